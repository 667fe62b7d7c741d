"""The TMA-fed FP32 filter pass against the oracle, through the C ABI.

The pass (hpass_tma.cu) is the default FP32 filter pass where n1 % 4 == 0.  Its
cases: halo frames that cross periodic faces (staged by per-row bulk copies, up
to three x segments per row when n1 < 28) and frames that do not (one tensor
box); ragged tiles in x and y; several z-chunks with a shorter last one; no
projectors at all; Yprev absent (degree 1) and aliasing Yout (degrees >= 2).
Tolerance: the FP32 filter's 1e-4 per column at m <= 9 (the 2e-4 of the full
filter is for m = 24).
"""
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


def _filter_vs_oracle(ctx, wl, seed, tol=1e-4):
    from paper_1603_04339_gb300 import sparc
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    Hor = O.OracleH(wl)
    X = synth.random_orbitals(wl.nd, wl.ns, seed).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.full_like(Xd, float("nan"))
    a0, b = -3.0, 70.0
    a = a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Yd)
    torch.cuda.synchronize()
    ctx.sync()
    Yo = O.cheb_filter(Hor, X.astype(np.float64), wl.m, a, b, a0)
    err = _colerr(Yd.cpu().numpy().astype(np.float64), Yo)
    # degree 1 (no Yprev) alone, element by element
    Y1 = torch.full_like(Xd, float("nan"))
    sparc.sparc_cheb_filter(H, 1, a, b, a0, Xd, Y1)
    torch.cuda.synchronize()
    Y1o = O.cheb_filter(Hor, X.astype(np.float64), 1, a, b, a0)
    err1 = _colerr(Y1.cpu().numpy().astype(np.float64), Y1o)
    H.close()
    return err, err1


@pytest.mark.parametrize("n,natom,ns,m", [
    ((40, 48, 45), 6, 20, 7),    # ragged x tile (8 wide), interior tiles, two z-chunks of 23 and 22
    ((20, 13, 14), 3, 11, 6),    # n1 < 28: up to three x segments per halo row; ragged y tile
    ((32, 32, 70), 4, 16, 5),    # three z-chunks (24, 24, 22)
    ((24, 20, 16), 0, 9, 6),     # no projectors
])
def test_tma_pass_filter_matches_oracle(ctx, n, natom, ns, m):
    wl = synth.small_case(n=n, h=(0.5, 0.45, 0.55), natom=natom, ns=ns, m=m, seed=300 + n[0] + n[2])
    err, err1 = _filter_vs_oracle(ctx, wl, seed=301 + n[1])
    print(f"n={n}: filter {err:.2e}, degree 1 {err1:.2e}")
    assert err < 1e-4, err
    assert err1 < 1e-5, err1


def test_tma_pass_differs_from_tiled_pass_only_by_rounding(ctx):
    """The TMA pass and the 16 x 16 tiled pass on the same filter: different kernels
    (their sums run in different orders, so the outputs are not equal bit for bit)
    that agree to FP32 rounding."""
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(36, 32, 30), natom=5, ns=24, m=8, seed=311)
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    X = torch.from_numpy(synth.random_orbitals(wl.nd, wl.ns, 312).astype(np.float32)).cuda()
    a0, b = -3.0, 70.0
    a = a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    outs = []
    for code in (0, 3):   # default (TMA) and the 16 x 16 tiled pass, 3 blocks per launch
        sparc.sparc_set_filter_units(ctx, sparc.F32, wl.nd, wl.ns, 1, code)
        Y = torch.full_like(X, float("nan"))
        sparc.sparc_cheb_filter(H, wl.m, a, b, a0, X, Y)
        torch.cuda.synchronize()
        outs.append(Y.cpu().numpy().astype(np.float64))
    sparc.sparc_set_filter_units(ctx, sparc.F32, wl.nd, wl.ns, 1, 0)
    d = _colerr(outs[0], outs[1])
    assert 0.0 < d < 2e-5, d
    H.close()
