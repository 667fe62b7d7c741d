"""Failure detection through the C ABI, with every failure made on the host.

* a bounded device wait that runs out: the TMA-fed filter pass is told to stop
  filling its stages (sparc_debug_inject STALL, with a short wait limit), so its
  waits for that stage give up; the launch finishes, the status word carries the
  timeout and the next synchronising call returns SPARC_ERR_TIMEOUT; the context
  then runs the same filter correctly;
* an allocation that fails: the next workspace growth is refused, the call
  returns SPARC_ERR_OOM and the context stays usable;
* an SCF step whose Poisson solve cannot converge (its CG iteration cap is
  lowered): sparc_scf_step returns SPARC_ERR_NO_CONVERGENCE.
No kernel faults, traps or hangs: the injections change host-side decisions only.
"""
import numpy as np
import pytest

from oracle import sparc_oracle as O
from paper_1603_04339_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT, OOM, NO_CONVERGENCE = 6, 2, 5


@pytest.fixture(scope="module")
def ctx():
    from paper_1603_04339_gb300 import build, sparc
    build.build()
    c = sparc.Context(0)
    yield c
    c.close()


def _colerr(Y, Yref):
    return np.max(np.linalg.norm(Y - Yref, axis=1) / np.linalg.norm(Yref, axis=1))


def test_bounded_wait_runs_out_and_reports_timeout(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(32, 32, 30), natom=3, ns=16, m=3, seed=501)
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    X = torch.from_numpy(synth.random_orbitals(wl.nd, wl.ns, 502).astype(np.float32)).cuda()
    Y = torch.empty_like(X)
    a0, b = -3.0, 60.0
    a = a0 + 0.2 * (b - a0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, X, Y)      # warm-up on a healthy pipeline
    ctx.sync()
    ctx.inject("wait_limit", 1 << 20)                      # about half a millisecond
    ctx.inject("stall", 9)                                 # the next pass launch stalls at step 9
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, X, Y)      # returns: the launch is asynchronous
    with pytest.raises(sparc.SparcError) as e:
        ctx.sync()
    assert e.value.code == TIMEOUT, e.value
    ctx.inject("wait_limit", 0)
    ctx.sync()                                             # the status word was cleared
    Y.fill_(float("nan"))
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, X, Y)      # the context works as before
    ctx.sync()
    Yo = O.cheb_filter(O.OracleH(wl), X[:4].cpu().numpy().astype(np.float64), wl.m, a, b, a0)
    assert _colerr(Y[:4].cpu().numpy().astype(np.float64), Yo) < 1e-4
    H.close()


def test_injected_allocation_failure_returns_oom():
    from paper_1603_04339_gb300 import build, sparc
    build.build()
    c = sparc.Context(0)
    try:
        wl = synth.small_case(n=(20, 18, 22), natom=2, seed=503)
        H = sparc.Hamiltonian.from_workload(c, wl)
        X = torch.from_numpy(synth.random_orbitals(wl.nd, 24, 504)).cuda()
        Y = torch.empty_like(X)
        c.inject("alloc_fail", 1)
        with pytest.raises(sparc.SparcError) as e:
            sparc.sparc_apply_H(H, X, Y)                   # needs the first workspace
        assert e.value.code == OOM
        sparc.sparc_apply_H(H, X, Y)                       # the next growth succeeds
        c.sync()
        ref = O.OracleH(wl).apply(X[:3].cpu().numpy())
        assert _colerr(Y[:3].cpu().numpy(), ref) < 1e-12
        H.close()
    finally:
        c.close()


def test_injected_poisson_nonconvergence_fails_the_scf_step(ctx):
    from paper_1603_04339_gb300 import sparc
    sysd = synth.scf_small(n=(20, 20, 20), natom=4, ns=12, m=8, seed=505)
    H = sparc.Hamiltonian.from_workload(ctx, sysd.wl)
    S = sparc.Scf.from_system(H, sysd, kT=0.01, mix_beta=0.3, mix_history=7, poisson_tol=1e-13, first_passes=1)
    U = torch.from_numpy(sysd.U0.copy()).cuda()
    eig = torch.zeros(sysd.wl.ns, dtype=torch.float64, device="cuda")
    ctx.inject("cg_max_iters", 1)
    with pytest.raises(sparc.SparcError) as e:
        sparc.sparc_scf_step(S, U, eig, sysd.wl.m)
    assert e.value.code == NO_CONVERGENCE
    ctx.inject("cg_max_iters", 0)
    S.close()
    H.close()
