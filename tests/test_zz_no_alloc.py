"""sparc_apply_H_noalloc: H X computed in the library's fixed scratch array.

Some callers cannot allocate device memory when they need H X (code under CUDA
graph capture, applications whose memory belongs to another pool, real-time
loops).  This checks, through the C ABI, that the allocation-free entry point
gives the same result as sparc_apply_H on two calls in a row, and that a
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


@pytest.mark.parametrize("dt,k,tol", [(torch.float64, (0.0, 0.0, 0.0), 1e-13),
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
