"""Parity at the sizes of the three synthetic workloads, through the C ABI.

* 24^3 cell, Ns=32, m=20, FP64: the whole CheFSI step (Lanczos bounds, filter,
  Rayleigh-Ritz) against the oracle, element by element.
* 64^3 benchmark cell, Ns=512, m=24: the FP32 filter in the launch the benchmark
  times, checked on sampled columns that the oracle filters one by one (columns
  are independent in the filter); FP64 Lanczos bounds against the oracle; the
  mixed Rayleigh-Ritz output against properties that hold at any size.
* 40^3 Si-like cell at one Monkhorst-Pack k-point, complex64 filter on sampled
  columns; the complex64 mixed Rayleigh-Ritz of the filtered Ns = 192 block against
  the oracle's.
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


def test_small_cell_full_chefsi_step_fp64(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.config1()
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    Hor = O.OracleH(wl)
    v0 = synth.lanczos_start(wl.nd, 2001)
    a0, b = sparc.sparc_lanczos_bounds(H, 10, torch.from_numpy(v0).cuda())
    ra0, rb, _ = O.lanczos_bounds(Hor, v0, 10)
    assert abs(a0 - ra0) < 1e-10 * abs(rb) and abs(b - rb) < 1e-10 * abs(rb)
    a = ra0 + (rb - ra0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    X = synth.random_orbitals(wl.nd, wl.ns, 2001)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    sparc.sparc_cheb_filter(H, wl.m, a, rb, ra0, Xd, Yd)
    Yf = O.cheb_filter(Hor, X, wl.m, a, rb, ra0)
    torch.cuda.synchronize()
    assert _colerr(Yd.cpu().numpy(), Yf) < 1e-10
    eig = torch.zeros(wl.ns, dtype=torch.float64, device="cuda")
    sparc.sparc_rayleigh_ritz(H, Yd, eig, sparc.RR_FP64)
    torch.cuda.synchronize()
    lam, U, _, _ = O.rayleigh_ritz(Hor, Yf)
    assert np.max(np.abs(eig.cpu().numpy() - lam)) < 1e-10 * np.max(np.abs(lam))
    Ug = Yd.cpu().numpy()
    assert np.allclose(Ug @ Ug.T, np.eye(wl.ns), atol=1e-10)
    # spectral projectors of clusters of (near-)degenerate Ritz values
    i = 0
    while i < wl.ns:
        j = i + 1
        while j < wl.ns and lam[j] - lam[j - 1] < 1e-8:
            j += 1
        P, Pr = Ug[i:j].T @ Ug[i:j], U[i:j].T @ U[i:j]
        assert np.linalg.norm(P - Pr) < 1e-9, (i, j)
        i = j


@pytest.fixture(scope="module")
def cell64():
    wl = synth.config2()
    return wl, O.OracleH(wl)


def test_benchmark_cell_lanczos_fp64(ctx, cell64):
    from paper_1603_04339_gb300 import sparc
    wl, Hor = cell64
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    v0 = synth.lanczos_start(wl.nd, 2003)
    a0, b = sparc.sparc_lanczos_bounds(H, 10, torch.from_numpy(v0).cuda())
    ra0, rb, _ = O.lanczos_bounds(Hor, v0, 10)
    assert abs(a0 - ra0) < 1e-10 * abs(rb) and abs(b - rb) < 1e-10 * abs(rb)


def test_benchmark_cell_fp32_filter_sampled_columns(ctx, cell64):
    """The benchmark's filter launch (all 512 columns, FP32); the oracle filters 3 of them."""
    from paper_1603_04339_gb300 import sparc
    wl, Hor = cell64
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    X32 = synth.random_orbitals(wl.nd, wl.ns, 2002).astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    Yd = torch.empty_like(Xd)
    a0, b = -2.5, 140.0
    a = a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Yd)
    torch.cuda.synchronize()
    cols = [0, 257, 511]
    Yref = O.cheb_filter(Hor, X32[cols].astype(np.float64), wl.m, a, b, a0)
    assert _colerr(Yd[cols].cpu().numpy().astype(np.float64), Yref) < 2e-4


def test_benchmark_cell_mixed_rayleigh_ritz_properties(ctx, cell64):
    """Orthonormal output, ascending Ritz values below the Lanczos upper bound, and
    lambda_i = u_i^T H u_i with H applied in FP64 (a property at any size)."""
    from paper_1603_04339_gb300 import sparc
    wl, _ = cell64
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    X32 = synth.random_orbitals(wl.nd, wl.ns, 2002).astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    Yd = torch.empty_like(Xd)
    a0, b = sparc.sparc_lanczos_bounds(H, 10, torch.from_numpy(synth.lanczos_start(wl.nd, 2003)).cuda())
    a = a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Yd)
    eig = torch.zeros(wl.ns, dtype=torch.float64, device="cuda")
    sparc.sparc_rayleigh_ritz(H, Yd, eig, sparc.RR_MIXED)
    torch.cuda.synchronize()
    lam = eig.cpu().numpy()
    # a0 (smallest Lanczos Ritz value) lies above lambda_min, so only b bounds the Ritz values
    assert np.all(np.diff(lam) >= 0), np.min(np.diff(lam))
    assert lam[-1] <= b, (lam[-1], b)
    U64 = Yd.to(torch.float64)
    G = (U64 @ U64.T).cpu().numpy()
    # Cholesky-QR pass, Rayleigh-Ritz in the orthonormal basis and an FP64 Newton-Schulz
    # step on the eigenvectors: |U^T U - I| is set by the FP32 rounding of U and the
    # 3xTF32 rotation (measured 6e-6 on this cell)
    print(f"mixed orthonormality {np.max(np.abs(G - np.eye(wl.ns))):.3e}")
    assert np.max(np.abs(G - np.eye(wl.ns))) < 5e-5, np.max(np.abs(G - np.eye(wl.ns)))
    HU = torch.empty_like(U64)
    sparc.sparc_apply_H(H, U64, HU)
    rq = (U64 * HU).sum(dim=1).cpu().numpy() / np.diag(G)
    print(f"mixed RQ consistency {np.max(np.abs(rq - lam)):.3e}")
    assert np.max(np.abs(rq - lam)) < 1e-5 * max(1.0, np.max(np.abs(lam))), np.max(np.abs(rq - lam))


def test_si_cell_one_kpoint_complex64_filter_sampled_columns(ctx):
    from paper_1603_04339_gb300 import sparc
    wl = synth.config3()
    kidx = 4
    H = sparc.Hamiltonian.from_workload(ctx, wl, kidx)
    Hor = O.OracleH(wl, kidx)
    X = synth.random_orbitals(wl.nd, wl.ns, 2013, complex_=True).astype(np.complex64)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    a0, b = -2.5, 80.0
    a = a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Yd)
    torch.cuda.synchronize()
    cols = [3, 191]
    Yref = O.cheb_filter(Hor, X[cols].astype(np.complex128), wl.m, a, b, a0)
    assert _colerr(Yd[cols].cpu().numpy().astype(np.complex128), Yref) < 2e-4


def test_benchmark_cell_mixed_vs_fp64_rayleigh_ritz(ctx, cell64):
    """The mixed Rayleigh-Ritz (FP32 data, tensor-core Grams and rotation, FP64
    Cholesky and eigensolve) against the FP64 Rayleigh-Ritz of the same filtered
    block (the FP32 values widened exactly): both compute the Ritz values of one
    subspace, so they differ only by the mixed path's own rounding."""
    from paper_1603_04339_gb300 import sparc
    wl, _ = cell64
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    X32 = synth.random_orbitals(wl.nd, wl.ns, 2004).astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    Yd = torch.empty_like(Xd)
    a0, b = sparc.sparc_lanczos_bounds(H, 10, torch.from_numpy(synth.lanczos_start(wl.nd, 2005)).cuda())
    a = a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Yd)
    Y64 = Yd.to(torch.float64)
    e32 = torch.zeros(wl.ns, dtype=torch.float64, device="cuda")
    e64 = torch.zeros_like(e32)
    sparc.sparc_rayleigh_ritz(H, Yd, e32, sparc.RR_MIXED)
    sparc.sparc_rayleigh_ritz(H, Y64, e64, sparc.RR_FP64)
    torch.cuda.synchronize()
    d = np.abs(e32.cpu().numpy() - e64.cpu().numpy())
    lam = e64.cpu().numpy()
    print(f"mixed vs FP64 Ritz values: max {d.max():.3e} Ha, lowest 256: {d[:256].max():.3e} Ha, "
          f"range [{lam[0]:.4f}, {lam[-1]:.4f}]")
    U64 = Yd.to(torch.float64)
    G = (U64 @ U64.T).cpu().numpy()
    print(f"mixed orthonormality: {np.max(np.abs(G - np.eye(wl.ns))):.3e}")
    # the mixed path's eigenvalue target is 1e-6 Ha (measured 7.6e-7 Ha on this cell);
    # 2e-6 leaves room for other seeds, and a single-TF32 product path misses it by 100x
    assert d.max() < 2e-6, d.max()
    assert np.max(np.abs(G - np.eye(wl.ns))) < 5e-5


def test_mixed_rayleigh_ritz_matches_oracle_at_ns256(ctx):
    """The mixed Rayleigh-Ritz at a production-like size (40^3 Si-like cell at
    Gamma, 64 s+p atoms, Ns = 256): tensor-core Grams accumulated over many
    chunks of the 64 000 grid rows, the Cholesky-QR pass and the Newton-Schulz
    step, against the oracle's FP64 Rayleigh-Ritz (Eq. SubspaceGeneralizedEigenproblem)
    of the same FP32 block.  Target: 1e-6 Ha on every Ritz value."""
    import dataclasses
    from paper_1603_04339_gb300 import sparc
    wl = dataclasses.replace(synth.config3(), kpts=np.zeros((1, 3)), kw=np.ones(1), ns=256)
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    Hor = O.OracleH(wl)
    ns = wl.ns
    Xd = torch.from_numpy(synth.random_orbitals(wl.nd, ns, 2011).astype(np.float32)).cuda()
    Yd = torch.empty_like(Xd)
    a0, b = sparc.sparc_lanczos_bounds(H, 10, torch.from_numpy(synth.lanczos_start(wl.nd, 2012)).cuda())
    a = a0 + (b - a0) * (ns / wl.nd) ** (2.0 / 3.0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Yd)
    Y = Yd.cpu().numpy().astype(np.float64)                 # the block both sides project
    lam_ref, _, _, _ = O.rayleigh_ritz(Hor, Y)
    # default: FP32 scaled Cholesky, then the series factorisation of I + E; then the
    # FP64 fallbacks of the second (1) and of both (2) orthonormalisations
    for force in (0, 1, 2):
        U32 = Yd.clone()
        eig = torch.zeros(ns, dtype=torch.float64, device="cuda")
        ctx.inject("fp64_ortho", force)
        try:
            sparc.sparc_rayleigh_ritz(H, U32, eig, sparc.RR_MIXED)
            torch.cuda.synchronize()
        finally:
            ctx.inject("fp64_ortho", 0)
        d = np.abs(eig.cpu().numpy() - lam_ref)
        err = ctx.last_ortho_err()
        print(f"mixed RR (fp64_ortho={force}) vs oracle at Ns=256: max {d.max():.3e} Ha over "
              f"[{lam_ref[0]:.4f}, {lam_ref[-1]:.4f}]; max |U1^T U1 - I| = {err:.2e}")
        assert d.max() < 1e-6, (force, d.max())
        if force == 0:
            assert 0.0 <= err <= 1e-3, err     # the series path ran
        U = U32.to(torch.float64)
        assert float((U @ U.T - torch.eye(ns, dtype=torch.float64, device="cuda")).abs().max()) < 5e-5


def test_si_cell_kpoint_mixed_rayleigh_ritz_complex64_matches_oracle(ctx):
    """The complex64 mixed Rayleigh-Ritz at the k-point workload's size (40^3 Si-like
    cell, one Monkhorst-Pack k-point, Ns = 192, m = 20; Section 3.3): tensor-core
    Grams and rotations on the real views of the Bloch orbitals, FP64 factorisations,
    against the oracle's FP64 Rayleigh-Ritz (Eq. SubspaceGeneralizedEigenproblem) of
    the same complex64 block.  Target: 1e-6 Ha on every Ritz value."""
    from paper_1603_04339_gb300 import sparc
    wl = synth.config3()
    kidx = 5
    H = sparc.Hamiltonian.from_workload(ctx, wl, kidx)
    Hor = O.OracleH(wl, kidx)
    ns = wl.ns
    X = synth.random_orbitals(wl.nd, ns, 2021, complex_=True).astype(np.complex64)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    v0 = synth.lanczos_start(wl.nd, 2022, complex_=True)
    a0, b = sparc.sparc_lanczos_bounds(H, 10, torch.from_numpy(v0).cuda())
    a = a0 + (b - a0) * (ns / wl.nd) ** (2.0 / 3.0)
    sparc.sparc_cheb_filter(H, wl.m, a, b, a0, Xd, Yd)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.complex128)       # the block both sides project
    lam_ref, _, _, _ = O.rayleigh_ritz(Hor, Y)
    U = Yd.clone()
    eig = torch.zeros(ns, dtype=torch.float64, device="cuda")
    sparc.sparc_rayleigh_ritz(H, U, eig, sparc.RR_MIXED)
    torch.cuda.synchronize()
    d = np.abs(eig.cpu().numpy() - lam_ref)
    Uc = U.to(torch.complex128)
    orth = float((Uc.conj() @ Uc.T - torch.eye(ns, dtype=torch.complex128, device="cuda")).abs().max())
    print(f"complex64 mixed RR vs oracle at 40^3, Ns={ns}: max {d.max():.3e} Ha over "
          f"[{lam_ref[0]:.4f}, {lam_ref[-1]:.4f}]; max |U^H U - I| = {orth:.2e}")
    H.close()
    assert d.max() < 1e-6, d.max()
    assert orth < 5e-5, orth
