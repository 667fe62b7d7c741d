"""sparc_apply_H_noalloc: H X computed in the library's fixed scratch array.

Some callers cannot allocate device memory when they need H X: applications
whose device memory belongs to another allocator or to a fixed budget, and
latency-bound loops that may not block on cudaMalloc.  This checks, through the
C ABI, that the allocation-free entry point gives the same result as
sparc_apply_H on two calls in a row, that a call needing far more scratch than
the context has allocated leaves the device's free memory unchanged, and that a
problem larger than the fixed scratch is refused with a clear error.
"""
import numpy as np
import pytest

from paper_1603_04339_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1603_04339_gb300 import build, sparc
    build.build()
    c = sparc.Context(0)
    yield c
    c.close()


# FP32 and complex64: the allocating call takes the tiled kernels, the
# allocation-free one the generic pass, so they agree to FP32 rounding.
@pytest.mark.parametrize("dt,k,tol", [(torch.float64, (0.0, 0.0, 0.0), 1e-13),
                                      (torch.float32, (0.0, 0.0, 0.0), 1e-6),
                                      (torch.complex128, (0.15, 0.05, -0.2), 1e-13),
                                      (torch.complex64, (0.2, -0.1, 0.3), 1e-6)])
def test_noalloc_apply_matches_apply_on_two_calls(ctx, dt, k, tol):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(20, 18, 22), natom=3, k=k, seed=91)
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    cplx = dt.is_complex
    ns, ld = 45, wl.nd + 7
    outs = []
    for call in range(2):
        X = torch.zeros((ns, ld), dtype=dt, device="cuda")
        X[:, : wl.nd] = torch.from_numpy(synth.random_orbitals(wl.nd, ns, 100 + call, complex_=cplx)).to(dt).cuda()
        Yref = torch.zeros_like(X)
        sparc.sparc_apply_H(H, X, Yref, ns=ns, ld=ld)          # also uploads the projector values
        Y = torch.zeros_like(X)
        sparc.sparc_apply_H_noalloc(H, X, Y, ns=ns, ld=ld)
        torch.cuda.synchronize()
        a, b = Y[:, : wl.nd].cpu().numpy(), Yref[:, : wl.nd].cpu().numpy()
        err = np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1))
        assert err < tol, (call, err)
        outs.append(a)
    assert not np.allclose(outs[0], outs[1])                   # the second call saw new data


def test_noalloc_apply_rejects_problems_beyond_the_scratch(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(40, 40, 40), natom=1, seed=92)
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    X = torch.zeros((128, wl.nd), dtype=torch.float64, device="cuda")   # 2 x 65.5 MB of blocks
    Y = torch.zeros_like(X)
    sparc.sparc_apply_H(H, X[:1], Y[:1])
    with pytest.raises(sparc.SparcError) as e:
        sparc.sparc_apply_H_noalloc(H, X, Y)
    assert e.value.code == 1 and "scratch" in str(e.value)


def test_noalloc_apply_allocates_no_device_memory():
    """A context whose workspace only ever held a 1-orbital H-apply: a
    45-orbital call of the allocation-free entry point (about 2 x 2.5 MB of
    blocks, which sparc_apply_H would have to allocate) leaves the driver's
    free-memory count where it was.  The kernels and the scratch address are
    loaded first by a warm-up call on another context, so that lazy module
    loading does not count."""
    from paper_1603_04339_gb300 import build, sparc
    build.build()
    wl = synth.small_case(n=(20, 18, 22), natom=3, seed=93)
    ns = 45
    X = torch.from_numpy(synth.random_orbitals(wl.nd, ns, 8)).cuda()
    Y = torch.empty_like(X)
    Yref = torch.empty_like(X)
    x1 = X[:1].clone()
    y1 = torch.empty_like(x1)
    warm = sparc.Context(0)
    c = sparc.Context(0)
    try:
        Hw = sparc.Hamiltonian.from_workload(warm, wl)
        sparc.sparc_apply_H(Hw, x1, y1)
        sparc.sparc_apply_H_noalloc(Hw, X, Y, ns=ns)
        H = sparc.Hamiltonian.from_workload(c, wl)
        sparc.sparc_apply_H(H, x1, y1)                          # projector values; 1-orbital workspace
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        sparc.sparc_apply_H_noalloc(H, X, Y, ns=ns)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, (free0, free1)
        sparc.sparc_apply_H(H, X, Yref, ns=ns)                  # grows the workspace (allowed here)
        torch.cuda.synchronize()
        err = float(((Y - Yref).norm(dim=1) / Yref.norm(dim=1)).max())
        assert err < 1e-13, err
    finally:
        c.close()
        warm.close()
