"""The TMA-fed complex64 filter pass (k-point Hamiltonians) against the oracle, through
the C ABI.

The pass (hpass_tma.cu, k_pass_tma<true>) is the default complex64 filter pass where
n1 % 4 == 0 and every halo-frame row lies within one cell in y.  It runs the FP32
pass's frames and stencil on half-units of four complex orbitals; the Bloch factors of
Section 3.1 enter at the periodic faces (ghost nodes in x, wrapped frame rows in y,
wrapped halo planes in z) and in the projector slots, which are split by periodic image
so that each carries one factor exp(-i k.(t L)) (Eq. NonlocalPS:FD).  Its cases: one
tile with frames that cross both y faces and boxes that wrap on every axis; ragged x and
y tiles; several z-chunks; no projectors; k = 0 on complex data (a real Hamiltonian
takes the same pass); batches that mix the Gamma point with other k, and batches whose
projector values differ between k (run per k).
Tolerance: the FP32 filter's 1e-4 per column at m <= 9, 1e-5 for one degree.
"""
import dataclasses
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


def _with_k(wl, kap):
    """The workload at the k-point kap (in units of the reciprocal cell, 2 pi / L_s)."""
    L = np.array([wl.n[s] * wl.h[s] for s in range(3)])
    k = 2 * math.pi * np.asarray(kap, np.float64) / L
    return dataclasses.replace(wl, kpts=np.asarray([k]), kw=np.ones(1))


def _bounds(wl):
    a0, b = -3.0, 70.0
    return a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0), b, a0


CASES = [
    # n, natom, ns, m, k (reciprocal units)
    ((16, 14, 15), 6, 12, 6, (1 / 3, -0.25, 0.3)),   # one tile: frame rows cross both y faces; boxes wrap on x, y, z
    ((40, 24, 20), 5, 16, 7, (0.5, 0.5, -0.5)),      # ragged x tile (8 wide), tile rows 16 + 8; zone-boundary k
    ((20, 36, 70), 4, 8, 5, (-0.2, 0.15, 0.45)),     # ragged x (4) and y (4) tiles; four z-chunks (18, 18, 18, 16)
    ((24, 16, 16), 0, 9, 6, (0.1, 0.2, 0.3)),        # no projectors
    ((16, 20, 18), 3, 10, 6, (0.0, 0.0, 0.0)),       # k = 0 on complex data
]


@pytest.mark.parametrize("n,natom,ns,m,kap", CASES)
def test_tma_pass_c64_filter_matches_oracle(ctx, n, natom, ns, m, kap):
    from paper_1603_04339_gb300 import sparc
    base = synth.small_case(n=n, h=(0.5, 0.45, 0.55), natom=natom, ns=ns, m=m, seed=500 + n[0] + n[2])
    wl = _with_k(base, kap)
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    assert H.filter_kernel(sparc.C64) == sparc.KERNEL_TMA
    Hor = O.OracleH(wl)
    X = synth.random_orbitals(wl.nd, wl.ns, 501 + n[1], complex_=True)
    Xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    a, b, a0 = _bounds(wl)
    Y = torch.full_like(Xd, float("nan"))
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Y)
    torch.cuda.synchronize()
    ctx.sync()
    Yo = O.cheb_filter(Hor, X.astype(np.complex128), wl.m, a, b, a0)
    err = _colerr(Y.cpu().numpy().astype(np.complex128), Yo)
    Y1 = torch.full_like(Xd, float("nan"))
    sparc.sparc_cheb_filter(H, 1, a, b, a0, Xd, Y1)
    torch.cuda.synchronize()
    Y1o = O.cheb_filter(Hor, X.astype(np.complex128), 1, a, b, a0)
    err1 = _colerr(Y1.cpu().numpy().astype(np.complex128), Y1o)
    H.close()
    print(f"n={n} k={kap}: filter {err:.2e}, degree 1 {err1:.2e}")
    assert err < 1e-4, err
    assert err1 < 1e-5, err1


def test_tma_pass_c64_declines_frames_two_cells_away(ctx):
    """n2 = 18: a halo-frame row of the second tile row (y = 37) lies two cells away, which
    one Bloch factor per row cannot express, so the complex filter runs the tiled pass
    there (checked against the oracle)."""
    from paper_1603_04339_gb300 import sparc
    wl = _with_k(synth.small_case(n=(16, 18, 14), natom=2, ns=8, m=5, seed=41), (0.3, -0.2, 0.1))
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    assert H.filter_kernel(sparc.C64) == sparc.KERNEL_TILED
    Hor = O.OracleH(wl)
    X = synth.random_orbitals(wl.nd, wl.ns, 42, complex_=True)
    Xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    a, b, a0 = _bounds(wl)
    Y = torch.full_like(Xd, float("nan"))
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Y)
    torch.cuda.synchronize()
    Yo = O.cheb_filter(Hor, X.astype(np.complex128), wl.m, a, b, a0)
    H.close()
    assert _colerr(Y.cpu().numpy().astype(np.complex128), Yo) < 1e-4


def _batch(ctx, wl, kaps, proj_scale=None):
    from paper_1603_04339_gb300 import sparc
    Hs = []
    for i, kap in enumerate(kaps):
        w = _with_k(wl, kap)
        if proj_scale is not None and proj_scale[i] != 1.0:
            w = dataclasses.replace(w, proj=dataclasses.replace(w.proj, chi=w.proj.chi * proj_scale[i]))
        Hs.append(sparc.Hamiltonian.from_workload(ctx, w))
    return Hs


@pytest.mark.parametrize("proj_scale", [None, (1.0, 1.01, 1.0)])
def test_tma_batch_with_gamma_point_equals_per_k(ctx, proj_scale):
    """A batch holding k = 0 (a real Hamiltonian: its complex64 filter takes the split
    slots too) and two other k: bit for bit the per-k filters; with projector values that
    differ between k the batch runs per k, with the same result."""
    from paper_1603_04339_gb300 import sparc
    base = synth.small_case(n=(20, 24, 18), h=(0.5, 0.45, 0.55), natom=4, ns=19, m=5, seed=77)
    kaps = [(0.0, 0.0, 0.0), (1 / 3, 1 / 3, -1 / 3), (-0.5, 0.25, 0.5)]
    Hs = _batch(ctx, base, kaps, proj_scale)
    for H in Hs:
        assert H.filter_kernel(sparc.C64) == sparc.KERNEL_TMA
    nk = len(Hs)
    X = torch.from_numpy(np.stack([synth.random_orbitals(base.nd, base.ns, 90 + k, complex_=True)
                                   for k in range(nk)]).astype(np.complex64)).cuda()
    a, b, a0 = [], [], []
    for k in range(nk):
        ak, bk, a0k = _bounds(base)
        a.append(ak + 0.1 * k)
        b.append(bk)
        a0.append(a0k)
    Y = torch.full_like(X, float("nan"))
    g0 = ctx.graph_launches()
    sparc.sparc_cheb_filter_batch(Hs, base.m, a, b, a0, X, Y)
    torch.cuda.synchronize()
    batched = ctx.graph_launches() - g0 == 1
    assert batched == (proj_scale is None)
    for k in range(nk):
        Yk = torch.full_like(X[k], float("nan"))
        sparc.sparc_cheb_filter(Hs[k], base.m, a[k], b[k], a0[k], X[k], Yk)
        torch.cuda.synchronize()
        assert torch.equal(Yk, Y[k]), k
    w1 = _with_k(base, kaps[1])
    if proj_scale is not None:
        w1 = dataclasses.replace(w1, proj=dataclasses.replace(w1.proj, chi=w1.proj.chi * proj_scale[1]))
    x = X[1, :3].cpu().numpy().astype(np.complex128)
    yo = O.cheb_filter(O.OracleH(w1), x, base.m, a[1], b[1], a0[1])
    assert _colerr(Y[1, :3].cpu().numpy().astype(np.complex128), yo) < 1e-4
    for H in Hs:
        H.close()
