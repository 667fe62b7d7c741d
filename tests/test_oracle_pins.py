"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: each checks a closed form, an
invariant, a special case that reduces to a textbook result, or brute force on
a tiny grid, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import sparc_oracle as O
from paper_1603_04339_gb300 import synth


# ---------------------------------------------------------------- FD weights (Eq. weightsLap)

@pytest.mark.parametrize("h", [1.0, 0.37])
def test_fd_second_order_is_three_point(h):
    w = O.fd_weights(1, h)
    # centre enters twice (p = 0 term of Eq. FD:Laplacian): [1, -2, 1] / h^2
    assert np.allclose([w[1], 2 * w[0], w[1]], np.array([1.0, -2.0, 1.0]) / h**2, rtol=1e-15)


@pytest.mark.parametrize("n_o", range(1, 9))
def test_fd_weights_annihilate_constants_and_differentiate_x2(n_o):
    h = 0.43
    w = O.fd_weights(n_o, h)
    assert abs(2 * w[0] + 2 * w[1:].sum()) * h * h < 1e-13
    # d2/dx2 x^2 = 2: sum_p w_p ((ph)^2 + (-ph)^2) = 2
    p = np.arange(1, n_o + 1)
    assert abs(np.sum(w[1:] * 2 * (p * h) ** 2) - 2.0) < 1e-12


@pytest.mark.parametrize("n_o", [1, 2, 3, 4, 6])
def test_fd_exact_on_polynomials(n_o):
    """A symmetric 2n_o+1 point second-derivative stencil is exact up to degree 2n_o+1."""
    h = 0.5
    x0 = 0.3
    w = O.fd_weights(n_o, h)
    for d in range(0, 2 * n_o + 2):
        f = lambda x: x ** d
        approx = 2 * w[0] * f(x0) + sum(w[p] * (f(x0 + p * h) + f(x0 - p * h)) for p in range(1, n_o + 1))
        exact = d * (d - 1) * x0 ** (d - 2) if d >= 2 else 0.0
        assert abs(approx - exact) < 1e-9 * max(1.0, abs(exact)) * 10 ** (d / 4), (d, approx, exact)


@pytest.mark.parametrize("n_o", [1, 2, 3])
def test_fd_convergence_order(n_o):
    """Symbol error on a fixed plane wave falls like h^(2 n_o)."""
    theta = 1.3
    errs = []
    for h in (0.2, 0.1):
        lam = O.fd_symbol(np.array([theta * h]), n_o, h)[0]
        errs.append(abs(lam - 0.5 * theta * theta))
    order = math.log(errs[0] / errs[1], 2)
    assert abs(order - 2 * n_o) < 0.15, order


# ---------------------------------------------------------------- H(k) local part

def _free(n, h, k, n_o=6):
    return O.OracleH(n=n, h=h, fd_radius=n_o, k=k, veff=np.zeros(n[0] * n[1] * n[2]),
                     proj=synth.Projectors.empty())


def _plane_wave(n, h, k, j):
    xs = synth.node_coords(n, h)
    L = [n[s] * h[s] for s in range(3)]
    th = [k[s] + 2 * math.pi * j[s] / L[s] for s in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return np.exp(1j * (th[0] * X + th[1] * Y + th[2] * Z)).reshape(-1), th


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.21, -0.13, 0.07)])
def test_plane_waves_are_eigenvectors_with_fd_symbol(k):
    """At V=0, exp(i(k+G).x) is Bloch with wavevector k and H acts as the FD symbol."""
    n, h = (14, 13, 15), (0.5, 0.6, 0.45)
    H = _free(n, h, k)
    for j in [(0, 0, 0), (1, -2, 3), (-7, 6, 7), (5, 0, -1)]:
        f, th = _plane_wave(n, h, k, j)
        lam = sum(O.fd_symbol(np.array([th[s] * h[s]]), 6, h[s])[0] for s in range(3))
        Hf = H.apply(f.astype(np.complex128))
        assert np.allclose(Hf, lam * f, atol=1e-10 * max(1.0, abs(lam)))


def test_full_free_spectrum_matches_symbol():
    n, h, k = (6, 7, 5), (0.7, 0.6, 0.8), (0.3, -0.2, 0.1)
    H = _free(n, h, k, n_o=2)
    ev = np.linalg.eigvalsh(H.dense())
    sym = []
    for a in range(n[0]):
        for b in range(n[1]):
            for c in range(n[2]):
                th = [k[0] + 2 * math.pi * a / (n[0] * h[0]), k[1] + 2 * math.pi * b / (n[1] * h[1]),
                      k[2] + 2 * math.pi * c / (n[2] * h[2])]
                sym.append(sum(O.fd_symbol(np.array([th[s] * h[s]]), 2, h[s])[0] for s in range(3)))
    assert np.allclose(ev, np.sort(sym), atol=1e-11)


def test_constant_potential_shifts_spectrum():
    n, h = (6, 6, 6), (0.6, 0.6, 0.6)
    H0 = _free(n, h, (0.1, 0.0, 0.0), n_o=2)
    H1 = O.OracleH(n=n, h=h, fd_radius=2, k=(0.1, 0.0, 0.0), veff=np.full(216, -0.731),
                   proj=synth.Projectors.empty())
    assert np.allclose(np.linalg.eigvalsh(H1.dense()), np.linalg.eigvalsh(H0.dense()) - 0.731, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_separable_potential_reduces_to_1d_problem(axis):
    """V depending on one coordinate only: spectrum = 1D (lap + V) spectrum + free symbol of the others."""
    n, h, n_o = (5, 6, 7), (0.7, 0.55, 0.6), 2
    rng = np.random.default_rng(3)
    v1 = rng.uniform(-1, 1, n[axis])
    idx = np.indices((n[2], n[1], n[0]))   # (z, y, x)
    coord = idx[2 - axis].reshape(-1)
    H = O.OracleH(n=n, h=h, fd_radius=n_o, k=(0, 0, 0), veff=v1[coord], proj=synth.Projectors.empty())
    ev = np.linalg.eigvalsh(H.dense())
    # 1D periodic matrix built directly from the weights of Eq. weightsLap
    w = O.fd_weights(n_o, h[axis])
    na = n[axis]
    A = np.zeros((na, na))
    for i in range(na):
        A[i, i] += 2 * w[0]
        for p in range(1, n_o + 1):
            A[i, (i + p) % na] += w[p]
            A[i, (i - p) % na] += w[p]
    e1 = np.linalg.eigvalsh(-0.5 * A + np.diag(v1))
    others = []
    for s in range(3):
        if s == axis:
            continue
        th = 2 * math.pi * np.arange(n[s]) / (n[s] * h[s])
        others.append(O.fd_symbol(th * h[s], n_o, h[s]))
    pred = (e1[:, None, None] + others[0][None, :, None] + others[1][None, None, :]).reshape(-1)
    assert np.allclose(ev, np.sort(pred), atol=1e-11)


# ---------------------------------------------------------------- nonlocal part

def test_projector_box_maps_to_analytic_function():
    """chi~ on the grid equals the analytic Gaussian of the nearest image (s projector, k=0)."""
    wl = synth.small_case(n=(14, 12, 13), natom=1, with_p=False, seed=11)
    H = O.OracleH(wl)
    gi, v = H.pidx[0], H.pval[0]
    xs = synth.node_coords(wl.n, wl.h)
    L = np.array(wl.L)
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)[gi]
    d = P - wl.atoms[0]
    d = d - L * np.round(d / L)         # nearest image
    g = np.exp(-np.sum(d * d, axis=1) / 0.9 ** 2)
    ratio = v / g
    assert np.allclose(ratio, ratio[0], rtol=1e-12)
    assert abs(wl.h[0] * wl.h[1] * wl.h[2] * np.sum(v * v) - 1.0) < 1e-12


def test_hermitian_with_projectors_at_k():
    wl = synth.small_case(k=(0.17, -0.29, 0.11), natom=2, seed=5)
    H = O.OracleH(wl)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(wl.nd) + 1j * rng.standard_normal(wl.nd)
    y = rng.standard_normal(wl.nd) + 1j * rng.standard_normal(wl.nd)
    lhs = np.vdot(x, H.apply(y))
    rhs = np.vdot(H.apply(x), y)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_gamma_point_operator_is_real_symmetric():
    wl = synth.small_case(n=(13, 13, 13), natom=2, seed=2)
    D = O.OracleH(wl).dense()
    assert D.dtype == np.float64
    assert np.allclose(D, D.T, atol=1e-12)


def test_rank_one_projector_secular_equation():
    """V=0 and one s projector: every new eigenvalue solves 1 = g h^3 sum |z_G|^2/(lam - eps_G)."""
    n, h, k = (13, 14, 13), (0.5, 0.5, 0.55), (0.11, 0.0, -0.2)
    wl = synth.small_case(n=n, h=h, natom=1, k=k, with_p=False, seed=21, veff_scale=0.0)
    H = O.OracleH(wl)
    gam = wl.proj.gamma[0]
    ev = np.linalg.eigvalsh(H.dense())
    # chi~ as a grid function, decomposed on Bloch plane waves by FFT
    chi = np.zeros(wl.nd, np.complex128)
    chi[H.pidx[0]] = H.pval[0]
    xs = synth.node_coords(n, h)
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    u = chi.reshape(n[2], n[1], n[0]) * np.exp(-1j * (k[0] * X + k[1] * Y + k[2] * Z))
    # z_G = <phi_G, chi~>, phi_G = exp(i(k+G).x)/sqrt(Nd); the FFT basis origin is node 0
    F = np.fft.fftn(u) / math.sqrt(wl.nd)
    eps = np.zeros_like(F, dtype=np.float64)
    for (c, b, a), _ in np.ndenumerate(F):
        th = [k[0] + 2 * math.pi * a / (n[0] * h[0]), k[1] + 2 * math.pi * b / (n[1] * h[1]),
              k[2] + 2 * math.pi * c / (n[2] * h[2])]
        eps[c, b, a] = sum(O.fd_symbol(np.array([th[s] * h[s]]), 6, h[s])[0] for s in range(3))
    z2, eps = (np.abs(F) ** 2).reshape(-1), eps.reshape(-1)
    dv = h[0] * h[1] * h[2]
    checked = 0
    for lam in ev:
        if np.min(np.abs(lam - eps)) < 1e-6:
            continue
        f = 1.0 - gam * dv * np.sum(z2 / (lam - eps))
        assert abs(f) < 1e-7, (lam, f)
        checked += 1
    assert checked >= 5


def test_lattice_translation_of_an_atom_leaves_H_unchanged():
    """chi~ of an atom and of its image one cell away differ by a phase only (Eq. NonlocalPS:FD)."""
    k = (0.23, -0.31, 0.17)
    wl = synth.small_case(n=(14, 13, 13), natom=1, k=k, seed=9)
    A = O.OracleH(wl).dense()
    p = wl.proj
    p2 = synth.Projectors(p.box_lo + np.array([wl.n[0], -wl.n[1], 0], np.int32), p.box_n, p.chi_off,
                          p.chi, p.gamma, p.atom, p.l)
    B = O.OracleH(wl, proj=p2).dense()
    assert np.allclose(A, B, atol=1e-12)


def test_grid_translation_across_boundary_preserves_spectrum():
    """Shifting V and the atom by whole nodes (box wrapping the face) keeps the spectrum at k != 0."""
    k = (0.41, 0.0, 0.0)
    n, h = (14, 13, 13), (0.5, 0.5, 0.5)
    base = synth.small_case(n=n, h=h, natom=1, k=k, seed=13)
    e_ref = None
    V = base.veff.reshape(n[2], n[1], n[0])
    for shift in (0, 3, 7, 11):
        L = np.array(base.L)
        atoms = base.atoms + np.array([shift * h[0], 0, 0])
        atoms = atoms - L * np.floor((atoms + L / 2) / L)
        proj = synth.make_projectors(n, h, atoms, 0.9, base.proj.gamma[:1], base.proj.gamma[1:2])
        H = O.OracleH(n=n, h=h, fd_radius=6, k=k, veff=np.roll(V, shift, axis=2).reshape(-1), proj=proj)
        e = np.linalg.eigvalsh(H.dense())
        if e_ref is None:
            e_ref = e
        else:
            assert np.allclose(e, e_ref, atol=1e-10), shift


def test_supercell_spectrum_folds_two_primitive_k_points():
    """Bloch's theorem (Section 2): the cell doubled along x, at wavevector K, has the
    spectrum of the primitive cell at K and at K + pi/L_x together.  V_eff and the atoms
    repeat with the primitive period, so this fixes the size and the sign convention of
    the Bloch phase on the stencil halo and on the projector images jointly (a phase of
    the wrong size, or one part taking exp(-ikL) where the other takes exp(+ikL), breaks
    the folding).  Radius-3 stencil to keep the dense supercell small."""
    n_o = 3
    n, h = (8, 7, 7), (0.55, 0.6, 0.6)
    L = np.array([n[s] * h[s] for s in range(3)])
    rng = np.random.default_rng(31)
    V = rng.uniform(-1.0, 0.5, (n[2], n[1], n[0]))
    R = np.array([-0.31, 0.17, -0.09]) * L            # R_x < 0, so R_x + L_x stays inside the doubled cell
    gs, gp = np.array([0.7]), np.array([-0.4])
    K = (0.21, -0.13, 0.37)
    spec = []
    for kx in (K[0], K[0] + math.pi / L[0]):
        proj = synth.make_projectors(n, h, R[None, :], 0.5, gs, gp)
        H = O.OracleH(n=n, h=h, fd_radius=n_o, k=(kx, K[1], K[2]), veff=V.reshape(-1), proj=proj)
        spec.append(np.linalg.eigvalsh(H.dense()))
    n2 = (2 * n[0], n[1], n[2])
    # node i' of the doubled cell (x = -L_x + i' h) is primitive node i' - n_x/2 (mod n_x)
    V2 = V[:, :, (np.arange(n2[0]) - n[0] // 2) % n[0]]
    atoms2 = np.stack([R, R + np.array([L[0], 0.0, 0.0])])
    proj2 = synth.make_projectors(n2, h, atoms2, 0.5, np.repeat(gs, 2), np.repeat(gp, 2))
    H2 = O.OracleH(n=n2, h=h, fd_radius=n_o, k=K, veff=V2.reshape(-1), proj=proj2)
    e2 = np.linalg.eigvalsh(H2.dense())
    e1 = np.sort(np.concatenate(spec))
    assert np.max(np.abs(e2 - e1)) < 1e-10 * np.max(np.abs(e1))
    # and the two primitive k-points do differ, so the check has teeth
    assert np.max(np.abs(spec[0] - spec[1])) > 1e-2


# ---------------------------------------------------------------- Chebyshev filter (Eq. ChebFilter)

def test_cheb_T_closed_form_matches_recurrence():
    x = np.linspace(-3, 3, 61)
    T0, T1 = np.ones_like(x), x.copy()
    for m in range(2, 12):
        T0, T1 = T1, 2 * x * T1 - T0
        assert np.allclose(O.cheb_T(m, x), T1, rtol=1e-11, atol=1e-11)


def _small_dense(k=(0.0, 0.0, 0.0), seed=4):
    wl = synth.small_case(n=(13, 13, 14), natom=2, k=k, seed=seed)
    H = O.OracleH(wl)
    ev, V = np.linalg.eigh(H.dense())
    return wl, H, ev, V


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.2, 0.1, -0.3)])
def test_filter_scales_eigenvectors_by_T_m(k):
    wl, H, ev, V = _small_dense(k)
    m, a0 = 9, ev[0] - 0.05
    a, b = ev[20], ev[-1] + 0.3
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    idx = [0, 3, 10, 30, 200, len(ev) - 1]
    X = V[:, idx].T
    Y = O.cheb_filter(H, X, m, a, b, a0)
    for r, i in enumerate(idx):
        f = O.cheb_T(m, np.array([(ev[i] - c) / e]))[0] / O.cheb_T(m, np.array([(a0 - c) / e]))[0]
        assert np.allclose(Y[r], f * X[r], atol=1e-9 * max(1.0, abs(f)))


def test_scaled_filter_equals_unscaled_over_T_m_tau0():
    wl, H, ev, V = _small_dense(seed=6)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, wl.nd))
    m, a, b, a0 = 11, ev[15], ev[-1] + 0.1, ev[0] - 0.2
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    Ys = O.cheb_filter(H, X, m, a, b, a0)
    Yu = O.cheb_filter_unscaled(H, X, m, a, b)
    t0 = O.cheb_T(m, np.array([(a0 - c) / e]))[0]
    assert np.allclose(Ys, Yu / t0, rtol=1e-12, atol=1e-12 * np.abs(Ys).max())


def test_degree_one_filter_is_shifted_matvec():
    wl, H, ev, V = _small_dense(seed=8)
    x = np.random.default_rng(2).standard_normal((2, wl.nd))
    a, b, a0 = 0.3, 50.0, -2.0
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    Y = O.cheb_filter(H, x, 1, a, b, a0)
    Yd = ((V * ((ev - c) / (a0 - c))) @ (np.conj(V.T) @ x.T)).T
    assert np.allclose(Y, Yd, atol=1e-11)


# ---------------------------------------------------------------- Lanczos bounds

@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.3, -0.1, 0.2)])
def test_lanczos_brackets_spectrum(k):
    wl, H, ev, V = _small_dense(k, seed=10)
    v0 = synth.lanczos_start(wl.nd, 3, complex_=any(k))
    a0, b, th = O.lanczos_bounds(H, v0, 10)
    assert ev[0] - 1e-10 <= a0
    assert th[-1] <= ev[-1] + 1e-10
    assert b >= ev[-1]


def test_lanczos_upper_bound_free_electron_closed_form():
    """V=0: lambda_max is the FD symbol at the grid's largest |theta h| on every axis."""
    n, h = (14, 14, 14), (0.5, 0.5, 0.5)
    H = _free(n, h, (0, 0, 0))
    lam_max = 3 * O.fd_symbol(np.array([math.pi]), 6, 0.5)[0]    # theta h = pi (n even)
    a0, b, th = O.lanczos_bounds(H, synth.lanczos_start(H.nd, 1), 12)
    assert b >= lam_max - 1e-9
    assert th[-1] <= lam_max + 1e-9


# ---------------------------------------------------------------- Rayleigh-Ritz (Eqs. 36-39)

def test_rayleigh_ritz_orthonormal_and_above_true_eigenvalues():
    wl, H, ev, V = _small_dense(seed=12)
    X = synth.random_orbitals(wl.nd, 10, 5)
    lam, U, Hs, Ms = O.rayleigh_ritz(H, X)
    assert np.allclose(U @ np.conj(U.T), np.eye(10), atol=1e-11)
    assert np.all(lam >= ev[:10] - 1e-10)              # Cauchy interlacing
    # Ritz pairs of a subspace that already is invariant are exact
    lam2, U2, _, _ = O.rayleigh_ritz(H, V[:, :6].T)
    assert np.allclose(lam2, ev[:6], atol=1e-10)


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, 0.0, -0.15)])
def test_repeated_chefsi_converges_to_lowest_eigenpairs(k):
    wl, H, ev, V = _small_dense(k, seed=14)
    ns = 12
    X = synth.random_orbitals(wl.nd, ns, 3, complex_=any(k))
    a0, b, _ = O.lanczos_bounds(H, synth.lanczos_start(wl.nd, 4, complex_=any(k)), 10)
    a = a0 + (b - a0) * 0.08
    for it in range(30):
        lam, X = O.chefsi_step(H, X, 12, a, b, a0)
        a = lam[-1]
        a0 = min(a0, lam[0])
    assert np.allclose(lam[:ns - 2], ev[:ns - 2], atol=1e-9)
    P = X[: ns - 2].T @ np.conj(X[: ns - 2])
    Pref = V[:, : ns - 2] @ np.conj(V[:, : ns - 2].T)
    # the subspace error is about the square root of the eigenvalue error
    if ev[ns - 2] - ev[ns - 3] > 1e-6:
        assert np.linalg.norm(P - Pref) < 1e-4


def test_free_electron_shell_closure():
    """V=0, no projectors, cubic cell, Ns=7 (shells 1+6): Ritz values = closed-form symbol values."""
    n, h = (14, 14, 14), (0.5, 0.5, 0.5)
    H = _free(n, h, (0, 0, 0))
    X = synth.random_orbitals(H.nd, 7, 8)
    a0, b, _ = O.lanczos_bounds(H, synth.lanczos_start(H.nd, 2), 10)
    t1 = O.fd_symbol(np.array([2 * math.pi / 7.0 * 0.5]), 6, 0.5)[0]
    a = 1.5 * t1
    for _ in range(25):
        lam, X = O.chefsi_step(H, X, 16, a, b, a0)
    assert abs(lam[0]) < 1e-9
    assert np.allclose(lam[1:], t1 + 2 * O.fd_symbol(np.array([0.0]), 6, 0.5)[0], atol=1e-9)


def test_fd_weights_match_textbook_table():
    """Eq. weightsLap with the centre counted twice reproduces the tabulated central
    second-derivative coefficients (tests/golden/fd_second_derivative_central.txt)."""
    from fractions import Fraction
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fd_second_derivative_central.txt")
    rows = 0
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        n_o = int(line[0])
        ref = [float(Fraction(t)) for t in line[1:]]
        assert len(ref) == n_o + 1
        w = O.fd_weights(n_o, 1.0)
        got = [2.0 * w[0]] + list(w[1:])
        assert np.allclose(got, ref, rtol=1e-14, atol=0), (n_o, got, ref)
        rows += 1
    assert rows == 4


def test_fd_weights_order12_solve_moment_equations_exactly():
    """n_o = 6 (the paper's twelfth order): the weights are the unique solution of the
    moment equations sum_p c_p (p^(2j) + (-p)^(2j)) = 2 [j == 1], j = 0..n_o (c_0 counted
    once at p = 0), solved here in exact rational arithmetic by Gaussian elimination."""
    from fractions import Fraction
    n_o = 6
    # unknowns c_0 .. c_6; equation j: c_0 [j == 0] + sum_p 2 p^(2j) c_p = 2 [j == 1]
    A = [[Fraction(1 if j == 0 else 0)] + [Fraction(2 * p ** (2 * j)) for p in range(1, n_o + 1)]
         for j in range(n_o + 1)]
    rhs = [Fraction(2 if j == 1 else 0) for j in range(n_o + 1)]
    n = n_o + 1
    for c in range(n):
        r = next(i for i in range(c, n) if A[i][c] != 0)
        A[c], A[r] = A[r], A[c]
        rhs[c], rhs[r] = rhs[r], rhs[c]
        for i in range(n):
            if i != c and A[i][c] != 0:
                f = A[i][c] / A[c][c]
                A[i] = [a - f * b for a, b in zip(A[i], A[c])]
                rhs[i] -= f * rhs[c]
    c = [float(rhs[i] / A[i][i]) for i in range(n)]
    w = O.fd_weights(n_o, 1.0)
    got = [2.0 * w[0]] + list(w[1:])
    assert np.allclose(got, c, rtol=1e-13, atol=0), (got, c)
