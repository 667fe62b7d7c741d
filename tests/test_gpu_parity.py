"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  * FP64 / complex128 data: apply 1e-12 relative per column (same sums, another
    order); filter 1e-10 relative per column, eigenvalues 1e-10 * max|lambda|,
    spectral projectors 1e-9 (the FP64 targets of the method's specification);
  * FP32 / complex64 data: apply 1e-5 relative per column (about 40 * u_32 with
    the row sum of |FD coefficients| ~ 2 |H x| for random x), filter 2e-4 per
    column (m degrees, each adding that error, with the recurrence stable),
    mixed-mode eigenvalues 1e-6 Ha.
"""
import numpy as np
import pytest

from oracle import sparc_oracle as O
from paper_1603_04339_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32, "c128": torch.complex128, "c64": torch.complex64}
NPDT = {"f64": np.float64, "f32": np.float32, "c128": np.complex128, "c64": np.complex64}


@pytest.fixture(scope="module")
def ctx():
    from paper_1603_04339_gb300 import build, sparc
    build.build()
    c = sparc.Context(0)
    yield c
    c.close()


def _inputs(wl, ns, dt, seed, ld=None):
    """Seeded start block rounded to the test dtype; the oracle gets the same rounded values."""
    cplx = dt in ("c128", "c64")
    X = synth.random_orbitals(wl.nd, ns, seed, complex_=cplx).astype(NPDT[dt])
    ld = wl.nd if ld is None else ld
    Xd = torch.zeros((ns, ld), dtype=TDT[dt], device="cuda")
    Xd[:, : wl.nd] = torch.from_numpy(X).cuda()
    return X.astype(np.complex128 if cplx else np.float64), Xd


def _colerr(Y, Yref):
    return np.max(np.linalg.norm(Y - Yref, axis=1) / np.linalg.norm(Yref, axis=1))


def _ham(ctx, wl, kidx=0):
    from paper_1603_04339_gb300 import sparc
    return sparc.Hamiltonian.from_workload(ctx, wl, kidx)


CASES = [
    # (name, workload kwargs, dtype)
    ("gamma_f64", dict(n=(24, 20, 22), h=(0.5, 0.55, 0.45), natom=3, seed=31), "f64"),
    ("gamma_f32", dict(n=(24, 20, 22), h=(0.5, 0.55, 0.45), natom=3, seed=31), "f32"),
    ("bloch_c128", dict(n=(20, 22, 18), h=(0.5, 0.5, 0.6), natom=3, k=(0.21, -0.17, 0.09), seed=32), "c128"),
    ("bloch_c64", dict(n=(20, 22, 18), h=(0.5, 0.5, 0.6), natom=3, k=(0.21, -0.17, 0.09), seed=32), "c64"),
    ("gamma_c128", dict(n=(16, 16, 16), h=(0.5, 0.5, 0.5), natom=2, seed=33), "c128"),
    ("no_proj_f64", dict(n=(13, 14, 15), h=(0.5, 0.5, 0.5), natom=0, seed=34), "f64"),
    ("radius2_f64", dict(n=(9, 7, 8), h=(0.7, 0.6, 0.8), natom=1, fd_radius=2, rc=0.6, seed=35), "f64"),
]
APPLY_TOL = {"f64": 1e-12, "c128": 1e-12, "f32": 1e-5, "c64": 1e-5}
FILTER_TOL = {"f64": 1e-10, "c128": 1e-10, "f32": 2e-4, "c64": 2e-4}


@pytest.mark.parametrize("name,kw,dt", CASES, ids=[c[0] for c in CASES])
def test_apply_H_matches_oracle(ctx, name, kw, dt):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(**kw)
    H = _ham(ctx, wl)
    ns = 37                                    # two orbital blocks, the second ragged
    X, Xd = _inputs(wl, ns, dt, seed=5, ld=wl.nd + 3)
    Yd = torch.full_like(Xd, float("nan"))
    sparc.sparc_apply_H(H, Xd, Yd, ns=ns, ld=wl.nd + 3)
    torch.cuda.synchronize()
    Y = Yd[:, : wl.nd].cpu().numpy().astype(X.dtype)
    assert torch.isnan(Yd[:, wl.nd:]).all()    # padding rows untouched
    Yref = O.OracleH(wl).apply(X)
    assert _colerr(Y, Yref) < APPLY_TOL[dt]


def test_apply_H_single_column(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(15, 14, 13), natom=2, seed=41)
    H = _ham(ctx, wl)
    X, Xd = _inputs(wl, 1, "f64", seed=2)
    Yd = torch.empty_like(Xd)
    sparc.sparc_apply_H(H, Xd, Yd)
    torch.cuda.synchronize()
    assert _colerr(Yd.cpu().numpy(), O.OracleH(wl).apply(X)) < 1e-12


@pytest.mark.parametrize("name,kw,dt", CASES, ids=[c[0] for c in CASES])
def test_cheb_filter_matches_oracle(ctx, name, kw, dt):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(**kw)
    H = _ham(ctx, wl)
    Hor = O.OracleH(wl)
    ns, m = 33, 9
    X, Xd = _inputs(wl, ns, dt, seed=6)
    # bounds from the oracle's own Lanczos (an input here, not under test)
    a0, b, _ = O.lanczos_bounds(Hor, synth.lanczos_start(wl.nd, 1, complex_=Hor.is_complex), 10)
    a = a0 + 0.1 * (b - a0)
    Yd = torch.empty_like(Xd)
    sparc.sparc_cheb_filter(H, m, a, b, a0, Xd, Yd)
    torch.cuda.synchronize()
    Yref = O.cheb_filter(Hor, X, m, a, b, a0)
    assert _colerr(Yd.cpu().numpy().astype(X.dtype), Yref) < FILTER_TOL[dt]


def test_filter_degree_one_and_determinism(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(16, 15, 14), natom=2, seed=43)
    H = _ham(ctx, wl)
    X, Xd = _inputs(wl, 40, "f64", seed=9)
    Y1 = torch.empty_like(Xd)
    Y2 = torch.empty_like(Xd)
    sparc.sparc_cheb_filter(H, 1, 0.5, 40.0, -1.0, Xd, Y1)
    ref = O.cheb_filter(O.OracleH(wl), X, 1, 0.5, 40.0, -1.0)
    torch.cuda.synchronize()
    assert _colerr(Y1.cpu().numpy(), ref) < 1e-12
    sparc.sparc_cheb_filter(H, 7, 0.5, 40.0, -1.0, Xd, Y1)
    sparc.sparc_cheb_filter(H, 7, 0.5, 40.0, -1.0, Xd, Y2)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)                 # no atomics: bitwise reproducible


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.15)])
def test_lanczos_bounds_match_oracle(ctx, k):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(18, 17, 16), natom=3, k=k, seed=51)
    H = _ham(ctx, wl)
    Hor = O.OracleH(wl)
    v0 = synth.lanczos_start(wl.nd, 11, complex_=Hor.is_complex)
    v0d = torch.from_numpy(v0).cuda()
    a0, b = sparc.sparc_lanczos_bounds(H, 10, v0d)
    ra0, rb, _ = O.lanczos_bounds(Hor, v0, 10)
    scale = max(abs(ra0), abs(rb))
    assert abs(a0 - ra0) < 1e-10 * scale and abs(b - rb) < 1e-10 * scale


def _projector_err(U, Uref, lam, gap=1e-8):
    """Largest spectral-projector difference over clusters of (near-)degenerate Ritz values."""
    ns = len(lam)
    i, worst = 0, 0.0
    while i < ns:
        j = i + 1
        while j < ns and lam[j] - lam[j - 1] < gap * max(1.0, abs(lam[j])):
            j += 1
        P = U[i:j].T @ np.conj(U[i:j])
        Pr = Uref[i:j].T @ np.conj(Uref[i:j])
        worst = max(worst, np.linalg.norm(P - Pr))
        i = j
    return worst


@pytest.mark.parametrize("dt,k", [("f64", (0, 0, 0)), ("c128", (0.2, 0.1, -0.25))])
def test_rayleigh_ritz_fp64_matches_oracle(ctx, dt, k):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(16, 18, 17), natom=3, k=k, seed=61)
    H = _ham(ctx, wl)
    Hor = O.OracleH(wl)
    ns = 40
    X, Xd = _inputs(wl, ns, dt, seed=12)
    # filter first (oracle) so that the subspace is a realistic one
    a0, b, _ = O.lanczos_bounds(Hor, synth.lanczos_start(wl.nd, 2, complex_=Hor.is_complex), 10)
    Yf = O.cheb_filter(Hor, X, 8, a0 + 0.05 * (b - a0), b, a0)
    Ud = torch.from_numpy(Yf.astype(NPDT[dt])).cuda()
    eig = torch.zeros(ns, dtype=torch.float64, device="cuda")
    sparc.sparc_rayleigh_ritz(H, Ud, eig, sparc.RR_FP64)
    torch.cuda.synchronize()
    lam_ref, Uref, _, _ = O.rayleigh_ritz(Hor, Yf)
    lam = eig.cpu().numpy()
    assert np.max(np.abs(lam - lam_ref)) < 1e-10 * np.max(np.abs(lam_ref))
    U = Ud.cpu().numpy()
    assert np.allclose(U @ np.conj(U.T), np.eye(ns), atol=1e-10)
    assert _projector_err(U, Uref, lam_ref) < 1e-9


@pytest.mark.parametrize("dt,k,force", [("f32", (0, 0, 0), 0), ("f32", (0, 0, 0), 1), ("f32", (0, 0, 0), 2),
                                         ("c64", (0.2, 0.1, -0.25), 0)])
def test_rayleigh_ritz_mixed_matches_oracle(ctx, dt, k, force):
    """force: the FP32 path's FP64 fallbacks (1: second orthonormalisation, 2: both)."""
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(16, 18, 17), natom=3, k=k, seed=62)
    H = _ham(ctx, wl)
    Hor = O.OracleH(wl)
    ns = 40
    X, _ = _inputs(wl, ns, dt, seed=13)
    a0, b, _ = O.lanczos_bounds(Hor, synth.lanczos_start(wl.nd, 3, complex_=Hor.is_complex), 10)
    Yf = O.cheb_filter(Hor, X, 8, a0 + 0.05 * (b - a0), b, a0).astype(NPDT[dt])
    Ud = torch.from_numpy(Yf).cuda()
    eig = torch.zeros(ns, dtype=torch.float64, device="cuda")
    ctx.inject("fp64_ortho", force)
    try:
        sparc.sparc_rayleigh_ritz(H, Ud, eig, sparc.RR_MIXED)
        torch.cuda.synchronize()
    finally:
        ctx.inject("fp64_ortho", 0)
    lam_ref, _, _, _ = O.rayleigh_ritz(Hor, Yf.astype(np.complex128 if Hor.is_complex else np.float64))
    assert np.max(np.abs(eig.cpu().numpy() - lam_ref)) < 1e-6


@pytest.mark.parametrize("case", ["random_potential", "free_cubic_gamma", "free_axis_k"])
def test_complex64_mixed_rr_simple_and_degenerate_spectra(ctx, case):
    """The complex64 mixed Rayleigh-Ritz (tensor-core Grams and rotations on the real
    views, FP64 factorisations, complex Jacobi) on a simple spectrum (a random potential
    at a general k) and on degenerate ones: free electrons in a cube at k = 0 on complex
    data (clusters of 6, 12 and 24) and at k along an axis (clusters of up to 4).  Ritz
    values against the oracle to 1e-6 Ha or 1.5e-7 of the value, whichever is larger
    (the FP32 data's Grams carry about 1e-7 of relative bias, and these filtered blocks
    reach 7-16 Ha), orthonormal complex vectors."""
    from paper_1603_04339_gb300 import sparc
    if case == "random_potential":
        wl = synth.small_case(n=(16, 18, 17), natom=3, k=(0.2, 0.1, -0.25), seed=62)
    else:
        kap = (0.0, 0.0, 0.0) if case == "free_cubic_gamma" else (0.13, 0.0, 0.0)
        n, h = (14, 14, 14), (0.5, 0.5, 0.5)
        k = tuple(2 * np.pi * kap[i] / (n[i] * h[i]) for i in range(3))
        wl = synth.small_case(n=n, h=h, natom=0, k=k, seed=5, veff_scale=0.0)
    H = _ham(ctx, wl)
    Hor = O.OracleH(wl)
    ns = 48
    X = synth.random_orbitals(wl.nd, ns, 17, complex_=True)
    a0, b, _ = O.lanczos_bounds(Hor, synth.lanczos_start(wl.nd, 3, complex_=Hor.is_complex), 10)
    Yf = O.cheb_filter(Hor, X, 8, a0 + 0.05 * (b - a0), b, a0).astype(np.complex64)
    Ud = torch.from_numpy(Yf).cuda()
    eig = torch.zeros(ns, dtype=torch.float64, device="cuda")
    sparc.sparc_rayleigh_ritz(H, Ud, eig, sparc.RR_MIXED)
    torch.cuda.synchronize()
    lam_ref, _, _, _ = O.rayleigh_ritz(Hor, Yf.astype(np.complex128))
    dl = np.abs(eig.cpu().numpy() - lam_ref)
    U = Ud.cpu().numpy().astype(np.complex128)
    orth = np.max(np.abs(np.conj(U) @ U.T - np.eye(ns)))
    H.close()
    print(f"{case}: max |d lambda| {dl.max():.2e} Ha over [{lam_ref[0]:.3f}, {lam_ref[-1]:.3f}], "
          f"relative {np.max(dl / np.abs(lam_ref)):.2e}, orthonormality {orth:.1e}")
    assert np.all(dl <= np.maximum(1e-6, 1.5e-7 * np.abs(lam_ref))), dl.max()
    assert orth < 5e-5, orth


def test_mixed_not_positive_definite_is_reported(ctx):
    """A rank-deficient FP32 block: the FP32 Cholesky fails, its FP64 fallback fails
    too, and the call reports NOT_POSDEF with the status word cleared."""
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(14, 14, 14), natom=1, seed=73)
    H = _ham(ctx, wl)
    U = torch.randn((6, wl.nd), dtype=torch.float32, device="cuda")
    U[4] = U[2]
    eig = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(sparc.SparcError) as e:
        sparc.sparc_rayleigh_ritz(H, U, eig, sparc.RR_MIXED)
    assert e.value.code == 4
    ctx.sync()


def test_invalid_arguments_are_reported(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(14, 14, 14), natom=1, k=(0.1, 0, 0), seed=71)
    H = _ham(ctx, wl)
    X = torch.zeros((2, wl.nd), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(sparc.SparcError) as e:
        sparc.sparc_apply_H(H, X, Y)                  # real data at k != 0
    assert e.value.code == 1
    Xc = X.to(torch.complex128)
    Yc = torch.zeros_like(Xc)
    with pytest.raises(sparc.SparcError):
        sparc.sparc_cheb_filter(H, 5, 1.0, 2.0, 1.5, Xc, Yc)   # a0 >= a
    with pytest.raises(sparc.SparcError):
        sparc.sparc_apply_H(H, Xc, Xc)                # X and Y overlap
    with pytest.raises(sparc.SparcError):
        sparc.sparc_apply_H(H, Xc, Yc, ld=wl.nd - 1)  # ld < Nd
    with pytest.raises(sparc.SparcError):
        sparc.Hamiltonian(ctx, (12, 14, 14), (0.5,) * 3, 6, (0, 0, 0), np.zeros(12 * 14 * 14))  # n < 2 n_o + 1


def test_not_positive_definite_is_reported(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(14, 14, 14), natom=1, seed=72)
    H = _ham(ctx, wl)
    U = torch.randn((6, wl.nd), dtype=torch.float64, device="cuda")
    U[3] = U[1]                                        # rank deficient: M~ singular
    eig = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(sparc.SparcError) as e:
        sparc.sparc_rayleigh_ritz(H, U, eig, sparc.RR_FP64)
    assert e.value.code == 4
    ctx.sync()                                         # status word was cleared
