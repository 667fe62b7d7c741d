"""The k-point batched complex64 filter (sparc_cheb_filter_batch) and the filter
launch-shape autotuner, through the C ABI.

* bit-for-bit equality with one sparc_cheb_filter per k, for the cost model's
  grouping and for pinned groupings that split the blocks of a k over launches
  and put several k in one launch (small anisotropic cell, ragged ns);
* the oracle's filter per k on the small cell, element by element;
* the 40^3 Si-like cell with all 27 Monkhorst-Pack k-points in the launch shape
  the benchmark times: sampled (k, column) pairs against the oracle, whole blocks
  against the per-k filter;
* the autotuner: a tuned grouping leaves the result unchanged.
"""
import math

import numpy as np
import pytest

from oracle import sparc_oracle as O
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


def _colerr(Y, Yref):
    return np.max(np.linalg.norm(Y - Yref, axis=1) / np.linalg.norm(Yref, axis=1))


def _small_multi_k():
    base = synth.small_case(n=(16, 14, 15), h=(0.55, 0.6, 0.5), natom=3, ns=20, m=7, seed=31)
    L = np.array([base.n[s] * base.h[s] for s in range(3)])
    kap = np.array([[1 / 3, 0, 0], [0, -1 / 3, 1 / 3], [0.5, 0.5, 0.5], [-0.25, 0.1, 0.0],
                    [1 / 3, 1 / 3, -1 / 3]])
    kpts = 2 * math.pi * kap / L
    wl = synth.Workload("small_multi_k", base.n, base.h, 6, kpts, np.full(len(kpts), 1 / len(kpts)),
                        base.veff, base.atoms, base.proj, base.ns, base.m, base.seed)
    return wl


def _filter_each(sparc, Hs, m, a, b, a0, X):
    Y = torch.empty_like(X)
    for k, H in enumerate(Hs):
        sparc.sparc_cheb_filter(H, m, a[k], b[k], a0[k], X[k], Y[k])
    torch.cuda.synchronize()
    return Y


def _bounds(nk, nd, ns, a0=-3.0, b=60.0):
    a0s = [a0 - 0.1 * k for k in range(nk)]
    bs = [b + 0.5 * k for k in range(nk)]
    a = [a0s[k] + (bs[k] - a0s[k]) * (ns / nd) ** (2.0 / 3.0) for k in range(nk)]
    return a, bs, a0s


def test_batch_equals_per_k_filter_and_oracle_small(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = _small_multi_k()
    nk = len(wl.kpts)
    Hs = [sparc.Hamiltonian.from_workload(ctx, wl, k) for k in range(nk)]
    X = np.stack([synth.random_orbitals(wl.nd, wl.ns, 300 + k, complex_=True) for k in range(nk)])
    Xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    a, b, a0 = _bounds(nk, wl.nd, wl.ns)
    Yref = _filter_each(sparc, Hs, wl.m, a, b, a0, Xd)
    for units in (0, 1, 2, 4, 5, 100):   # 0: the cost model's grouping
        sparc.sparc_set_filter_units(ctx, sparc.C64, wl.nd, wl.ns, nk, units)
        Y = torch.full_like(Xd, float("nan"))
        sparc.sparc_cheb_filter_batch(Hs, wl.m, a, b, a0, Xd, Y)
        torch.cuda.synchronize()
        assert torch.equal(Y, Yref), units
    sparc.sparc_set_filter_units(ctx, sparc.C64, wl.nd, wl.ns, nk, 0)
    Yh = Yref.cpu().numpy().astype(np.complex128)
    for k in range(nk):
        Hor = O.OracleH(wl, k)
        Yo = O.cheb_filter(Hor, X[k].astype(np.complex64).astype(np.complex128), wl.m, a[k], b[k], a0[k])
        err = _colerr(Yh[k], Yo)
        assert err < 1e-4, (k, err)


def test_batch_runs_as_one_graph_launch_and_updates_bounds(ctx):
    """A complex64 batch call is one graph launch; a repeat with new bounds updates
    the captured graph in place and still equals the per-k filters bit for bit."""
    from paper_1603_04339_gb300 import sparc
    wl = _small_multi_k()
    nk = len(wl.kpts)
    Hs = [sparc.Hamiltonian.from_workload(ctx, wl, k) for k in range(nk)]
    X = np.stack([synth.random_orbitals(wl.nd, wl.ns, 310 + k, complex_=True) for k in range(nk)])
    Xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    Y = torch.empty_like(Xd)
    for shift in (0.0, 1.5, 0.0):
        a, b, a0 = _bounds(nk, wl.nd, wl.ns, a0=-3.0 - shift, b=60.0 + shift)
        g0 = ctx.graph_launches()
        for _ in range(2):
            sparc.sparc_cheb_filter_batch(Hs, wl.m, a, b, a0, Xd, Y)
        torch.cuda.synchronize()
        assert ctx.graph_launches() - g0 == 2
        assert torch.equal(Y, _filter_each(sparc, Hs, wl.m, a, b, a0, Xd)), shift
    for H in Hs:
        H.close()


def test_batch_rejects_mismatched_hamiltonians(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = _small_multi_k()
    H0 = sparc.Hamiltonian.from_workload(ctx, wl, 0)
    other = synth.small_case(n=(16, 14, 16), natom=3, ns=20, seed=31)
    H1 = sparc.Hamiltonian.from_workload(ctx, other, 0)
    X = torch.zeros((2, wl.ns, max(wl.nd, other.nd)), dtype=torch.complex64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(sparc.SparcError):
        sparc.sparc_cheb_filter_batch([H0, H1], 3, [0.0, 0.0], [1.0, 1.0], [-1.0, -1.0], X, Y)
    with pytest.raises(sparc.SparcError):   # a0 < a < b violated for the second k
        sparc.sparc_cheb_filter_batch([H0, H0], 3, [0.0, 2.0], [1.0, 1.0], [-1.0, -1.0], X, Y)


@pytest.fixture(scope="module")
def si27(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.config3()
    nk = len(wl.kpts)
    Hs = [sparc.Hamiltonian.from_workload(ctx, wl, k) for k in range(nk)]
    X = torch.empty((nk, wl.ns, wl.nd), dtype=torch.complex64, device="cuda")
    for k in range(nk):
        X[k] = torch.from_numpy(synth.random_orbitals(wl.nd, wl.ns, 4000 + k, complex_=True)
                                .astype(np.complex64))
    a, b, a0 = _bounds(nk, wl.nd, wl.ns, a0=-2.5, b=80.0)
    yield wl, Hs, X, (a, b, a0)
    for H in Hs:
        H.close()


def test_si_cell_27_kpoints_batched_against_oracle_and_per_k(ctx, si27):
    from paper_1603_04339_gb300 import sparc
    wl, Hs, X, (a, b, a0) = si27
    Y = torch.empty_like(X)
    sparc.sparc_cheb_filter_batch(Hs, wl.m, a, b, a0, X, Y)
    torch.cuda.synchronize()
    for k in (0, 13, 26):
        Yk = torch.empty_like(X[k])
        sparc.sparc_cheb_filter(Hs[k], wl.m, a[k], b[k], a0[k], X[k], Yk)
        torch.cuda.synchronize()
        assert torch.equal(Yk, Y[k]), k
    for k, col in ((1, 0), (8, 191), (20, 77), (26, 130)):
        Hor = O.OracleH(wl, k)
        x = X[k, col:col + 1].cpu().numpy().astype(np.complex128)
        yo = O.cheb_filter(Hor, x, wl.m, a[k], b[k], a0[k])
        err = _colerr(Y[k, col:col + 1].cpu().numpy().astype(np.complex128), yo)
        assert err < 2e-4, (k, col, err)


def test_autotuned_grouping_keeps_the_result(ctx, si27):
    from paper_1603_04339_gb300 import sparc
    wl, Hs, X, (a, b, a0) = si27
    Y0 = torch.empty_like(X)
    sparc.sparc_cheb_filter_batch(Hs, wl.m, a, b, a0, X, Y0)
    Yt = torch.empty_like(X)
    units, ms = sparc.sparc_autotune_filter(Hs, wl.m, a, b, a0, X, Yt)
    print(f"autotuned units per launch {units}, {ms:.2f} ms for degree 4")
    assert units > 0 and ms > 0
    Y1 = torch.empty_like(X)
    sparc.sparc_cheb_filter_batch(Hs, wl.m, a, b, a0, X, Y1)
    torch.cuda.synchronize()
    assert torch.equal(Y0, Y1)
    sparc.sparc_set_filter_units(ctx, sparc.C64, wl.nd, wl.ns, len(Hs), 0)


def test_batch_of_more_k_points_than_one_launch_holds(ctx):
    """35 k-points: launches hold at most 32 k slots, so the batch spans several
    launch groups; still bit-identical to the per-k filter."""
    from paper_1603_04339_gb300 import sparc
    base = synth.small_case(n=(16, 14, 15), h=(0.55, 0.6, 0.5), natom=2, ns=9, m=4, seed=5)
    L = np.array([base.n[s] * base.h[s] for s in range(3)])
    rng = np.random.default_rng(9)
    kpts = 2 * math.pi * rng.uniform(-0.5, 0.5, (35, 3)) / L
    wl = synth.Workload("small_35k", base.n, base.h, 6, kpts, np.full(35, 1 / 35), base.veff, base.atoms,
                        base.proj, base.ns, base.m, base.seed)
    Hs = [sparc.Hamiltonian.from_workload(ctx, wl, k) for k in range(35)]
    X = torch.from_numpy(np.stack([synth.random_orbitals(wl.nd, wl.ns, 50 + k, complex_=True)
                                   for k in range(35)]).astype(np.complex64)).cuda()
    a, b, a0 = _bounds(35, wl.nd, wl.ns)
    Yref = _filter_each(sparc, Hs, wl.m, a, b, a0, X)
    for units in (0, 3 * 2):
        sparc.sparc_set_filter_units(ctx, sparc.C64, wl.nd, wl.ns, 35, units)
        Y = torch.full_like(X, float("nan"))
        sparc.sparc_cheb_filter_batch(Hs, wl.m, a, b, a0, X, Y)
        torch.cuda.synchronize()
        assert torch.equal(Y, Yref), units
    sparc.sparc_set_filter_units(ctx, sparc.C64, wl.nd, wl.ns, 35, 0)
