"""Pins of the SCF oracle (oracle/scf_oracle.py) to facts outside itself: closed forms,
limits, exact solutions of the discrete problems and a jellium fixed point."""
import math
import os

import numpy as np
import pytest

from oracle import scf_oracle as S
from oracle import sparc_oracle as O
from paper_1603_04339_gb300 import synth


def test_local_potential_limits():
    Z, rc = 3.0, 0.8
    assert abs(S.local_potential(np.array([0.0]), Z, rc)[0] - S.local_potential(np.array([1e-7]), Z, rc)[0]) < 1e-9
    r = np.array([12.0])
    assert abs(S.local_potential(r, Z, rc)[0] + Z / 12.0) < 1e-14   # erf(15) = 1


def test_pseudocharge_is_the_gaussian_of_charge_minus_z_and_its_self_energy():
    """-(1/4pi) lap V_I of V_I = -Z erf(r/rc)/r is -Z (pi^3/2 rc^3)^-1 exp(-r^2/rc^2) in the
    continuum; on a fine grid the discrete b_I matches it, integrates to -Z, and
    E_self = 1/2 int b V = Z^2 / (sqrt(2 pi) rc)."""
    n, h = (40, 40, 40), (0.2, 0.2, 0.2)
    Z, rc = 3.0, 0.8
    R = [[0.013, -0.021, 0.007]]
    b, e_self, q = S.pseudocharge(n, h, 6, R, [Z], [rc])
    assert abs(q[0] + Z) < 1e-8 * Z
    assert abs(b.sum() * 0.008 + Z) < 1e-8 * Z
    xs = [-0.5 * n[s] * h[s] + h[s] * np.arange(n[s]) - R[0][s] for s in range(3)]
    Zc, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    r2 = X * X + Y * Y + Zc * Zc
    ref = -Z / (math.pi ** 1.5 * rc ** 3) * np.exp(-r2 / rc ** 2)
    assert np.max(np.abs(b - ref.reshape(-1))) < 1e-5 * np.max(np.abs(ref))
    assert abs(e_self - Z * Z / (math.sqrt(2 * math.pi) * rc)) < 1e-6 * e_self


def test_pseudocharge_wraps_periodically():
    """An atom near a face: the same charge, b equal to that of the centred atom shifted."""
    n, h = (24, 24, 24), (0.5, 0.5, 0.5)
    b1, e1, _ = S.pseudocharge(n, h, 6, [[0.0, 0.0, 0.0]], [2.0], [0.7])
    b2, e2, _ = S.pseudocharge(n, h, 6, [[-6.0, 0.0, 0.0]], [2.0], [0.7])   # 12 nodes to the left
    assert abs(e1 - e2) < 1e-12 * e1
    assert np.allclose(np.roll(b1.reshape(24, 24, 24), -12, axis=2).reshape(-1), b2, atol=1e-14)


def test_poisson_plane_wave_closed_form():
    n, h, n_o = (12, 10, 8), (0.4, 0.5, 0.45), 6
    j = (2, 1, 3)
    xs = [h[s] * np.arange(n[s]) for s in range(3)]
    Zc, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    th = [2 * math.pi * j[s] / (n[s] * h[s]) for s in range(3)]
    f = np.cos(th[0] * X + th[1] * Y + th[2] * Zc).reshape(-1)
    lam = sum(2.0 * O.fd_symbol(np.array([th[s] * h[s]]), n_o, h[s])[0] for s in range(3))
    phi = S.poisson(f, n, h, n_o)
    assert np.allclose(phi, 4 * math.pi * f / lam, atol=1e-12 * np.max(np.abs(phi)))


def test_poisson_matches_dense_solve():
    n, h, n_o = (6, 5, 7), (0.5, 0.6, 0.4), 2
    nd = 210
    rng = np.random.default_rng(3)
    f = rng.standard_normal(nd)
    f -= f.mean()
    Lm = np.zeros((nd, nd))
    for c in range(nd):
        e = np.zeros(nd); e[c] = 1.0
        Lm[:, c] = O.laplacian(e.reshape(1, n[2], n[1], n[0]), n, h, n_o).reshape(-1).real
    phi_d = np.linalg.lstsq(-Lm / (4 * math.pi), f, rcond=None)[0]
    phi_d -= phi_d.mean()
    phi = S.poisson(f, n, h, n_o)
    assert np.allclose(phi, phi_d, atol=1e-10 * np.max(np.abs(phi_d)))


def test_lda_exchange_closed_form_and_potential_derivative():
    rs = np.array([0.5, 1.0, 2.0, 5.0])
    rho = 3.0 / (4.0 * math.pi * rs ** 3)
    eps, v = S.lda(rho)
    # exchange alone, the textbook form in rs: -(3/4pi)(9pi/4)^(1/3)/rs
    ex = -(3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
    A, a1, b1, b2, b3, b4 = S.PW92
    ec = eps - ex
    assert np.all(ec < 0) and np.all(np.diff(ec) > 0)      # negative, weaker at lower density
    # V_xc = d(rho eps_xc)/d rho, by central differences
    for r0 in rho:
        d = 1e-6 * r0
        e_p, _ = S.lda(np.array([r0 + d]))
        e_m, _ = S.lda(np.array([r0 - d]))
        num = ((r0 + d) * e_p[0] - (r0 - d) * e_m[0]) / (2 * d)
        _, v0 = S.lda(np.array([r0]))
        assert abs(num - v0[0]) < 1e-7 * abs(v0[0])


def test_pw92_high_density_limit_is_gell_mann_brueckner():
    """d eps_c / d ln rs -> (1 - ln 2)/pi^2 as rs -> 0 (exact high-density coefficient)."""
    A = (1.0 - math.log(2.0)) / math.pi ** 2
    assert abs(S.PW92[0] - A) < 2e-6
    rs1, rs2 = 1e-7, 2e-7
    rho = 3.0 / (4.0 * math.pi * np.array([rs1, rs2]) ** 3)
    eps, _ = S.lda(rho)
    ex = -(3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / np.array([rs1, rs2])
    ec = eps - ex
    slope = (ec[1] - ec[0]) / math.log(2.0)
    assert abs(slope - A) < 1e-3 * A


def test_fermi_level_symmetric_spectrum():
    lam = 0.1 * np.arange(20)
    mu = S.fermi_level(lam, 20.0, 0.01)        # 10 of 20 levels filled: midway by symmetry
    assert abs(mu - 0.95) < 1e-12
    g = S.occupations(lam, mu, 0.01)
    assert abs(2 * g.sum() - 20.0) < 1e-12
    assert abs(S.entropy_term(np.array([0.5]), 0.01) - 2 * 0.01 * math.log(0.5)) < 1e-15


def test_fermi_dirac_occupations_minimise_the_band_plus_entropy_functional():
    """Mermin's principle: at fixed electron count 2 sum g = N_e, the band energy plus the
    entropy term, 2 sum g lambda + 2 kT sum (g ln g + (1-g) ln(1-g)), is stationary at
    the Fermi-Dirac occupations with every partial derivative equal to 2 lambda_f, and
    any count-preserving change of the occupations raises it.  A wrong sign or factor
    of the entropy term, or of the occupation exponent, moves the minimum elsewhere."""
    rng = np.random.default_rng(12)
    lam = np.sort(rng.uniform(-0.4, 0.2, 24))
    kT, Ne = 0.02, 22.0
    mu = S.fermi_level(lam, Ne, kT)
    g = S.occupations(lam, mu, kT)
    F = lambda gg: 2.0 * float(np.sum(gg * lam)) + S.entropy_term(gg, kT)
    # F is a sum of one term per state: differentiate state n's term alone, with a step
    # inside (0, 1) that shrinks with g (1 - g) where ln g curves
    f_n = lambda n, x: 2.0 * x * lam[n] + S.entropy_term(np.array([x]), kT)
    checked = 0
    for n in range(len(lam)):
        eps = 1e-4 * min(g[n], 1.0 - g[n])
        if eps < 1e-14:
            continue
        dF = (f_n(n, g[n] + eps) - f_n(n, g[n] - eps)) / (2 * eps)
        assert abs(dF - 2.0 * mu) < 1e-6, (n, g[n], dF, 2 * mu)
        checked += 1
    assert checked >= 15
    F0 = F(g)
    for trial in range(20):
        d = rng.standard_normal(len(g))
        d -= d.mean()                             # keeps 2 sum g = N_e
        t = 0.5 * min(np.min(g / (np.abs(d) + 1e-300)), np.min((1 - g) / (np.abs(d) + 1e-300)))
        assert F(g + t * d) > F0


def test_anderson_solves_a_linear_fixed_point_exactly():
    rng = np.random.default_rng(5)
    dim = 5
    G = 0.5 * rng.standard_normal((dim, dim)) / math.sqrt(dim)
    c = rng.standard_normal(dim)
    x_star = np.linalg.solve(np.eye(dim) - G, c)
    xs, fs = [np.zeros(dim)], []
    for it in range(dim + 2):
        fs.append(G @ xs[-1] + c - xs[-1])
        xs.append(S.anderson(xs, fs, 0.3, 7))
    assert np.linalg.norm(xs[-1] - x_star) < 1e-10 * np.linalg.norm(x_star)


def test_jellium_is_a_fixed_point_with_closed_form_energy():
    """Uniform background b = -N_e/Omega, no projectors, 14 electrons in the 7 lowest
    plane waves (a closed shell at the Gamma point; 3 more orbitals from the next shell
    keep the filter cutoff above it and stay empty): the density is uniform, phi = 0,
    V_xc is constant, so V_in = V_xc(N_e/Omega) is self-consistent and the free
    energy is 2 sum g lambda + Omega (eps_xc - V_xc) rho + entropy, with lambda the FD
    free-electron values (Eq. FD:Laplacian symbol) shifted by V_xc."""
    n, h, n_o = (8, 8, 8), (0.5, 0.5, 0.5), 6
    nd = 512
    vol = nd * 0.125
    Ne, kT = 14.0, 1e-3
    rho0 = Ne / vol
    eps0, v0 = S.lda(np.array([rho0]))
    H = O.OracleH(n=n, h=h, fd_radius=n_o, k=(0, 0, 0), veff=np.full(nd, v0[0]),
                  proj=type("P", (), {"nproj": 0})())
    b = np.full(nd, -rho0)
    rng = np.random.default_rng(7)
    U = rng.standard_normal((10, nd))
    lam_prev = None
    for it in range(12):     # converge the subspace at fixed V_in
        out = S.scf_iteration(H, U, lam_prev, rng.standard_normal(nd), b, 0.0, Ne, kT, 12)
        U, lam_prev = out["U"], out["lam"]
    sym = lambda j: 2 * O.fd_symbol(np.array([2 * math.pi * j / 8]), n_o, 0.5)[0] / 2.0
    lam_ref = np.sort([v0[0]] + [v0[0] + sym(1)] * 6)
    assert np.allclose(out["lam"][:7], lam_ref, atol=1e-9)
    assert out["lam"][7] > lam_ref[-1] + 1.0
    assert np.allclose(out["rho"], rho0, atol=1e-9 * rho0)
    assert np.max(np.abs(out["phi"])) < 1e-9
    assert np.max(np.abs(out["v_out"] - v0[0])) < 1e-9
    g = out["g"]
    assert np.all(g[7:] < 1e-100)
    F_ref = 2 * np.sum(g[:7] * lam_ref) + vol * (eps0[0] - v0[0]) * rho0 + S.entropy_term(g, kT)
    assert abs(out["F"] - F_ref) < 1e-9 * abs(F_ref)


def test_gradient_weights_textbook():
    assert np.allclose(S.grad_weights(1, 1.0)[1:], [0.5])
    assert np.allclose(S.grad_weights(2, 1.0)[1:], [2.0 / 3.0, -1.0 / 12.0])
    x = np.linspace(0, 2 * math.pi, 24, endpoint=False)
    f = np.sin(3 * x)
    F = np.broadcast_to(f, (4, 5, 24)).copy()
    g = S.grad_h(F, (24, 5, 4), (2 * math.pi / 24, 1.0, 1.0), 6)
    assert np.allclose(g[0][0, 0], 3 * np.cos(3 * x), atol=2e-4)   # 12th-order error at 8 nodes/period
    assert np.max(np.abs(g[1])) < 1e-13 and np.max(np.abs(g[2])) < 1e-13


def test_forces_match_finite_differences_of_the_free_energy():
    """The analytic forces (local + nonlocal, Section 3.6) at the converged SCF state
    against -dF/dR by central differences of the converged free energy (the check the
    paper makes), for one atom of a two-atom cell, and Newton's third law."""
    from paper_1603_04339_gb300 import synth
    base = synth.scf_pair()
    n, h = base.wl.n, base.wl.h
    Z, rc = base.Z, base.rc
    R0 = base.wl.atoms
    U0, v0 = base.U0, base.v0

    def converged(R):
        proj = synth.scf_pair(R).wl.proj
        b, e_self, _ = S.pseudocharge(n, h, 6, R, Z, rc)
        v_in = S.lda(-b)[1]
        U, lam_prev, xh, fh = U0.copy(), None, [], []
        for it in range(80):
            H = O.OracleH(n=n, h=h, fd_radius=6, k=(0, 0, 0), veff=v_in, proj=proj)
            out = S.scf_iteration(H, U, lam_prev, v0, b, e_self, 2.0, 0.01, 12)
            if np.linalg.norm(out["v_out"] - v_in) < 1e-11 * np.linalg.norm(out["v_out"]):
                return out, proj
            xh.append(v_in)
            fh.append(out["v_out"] - v_in)
            v_in = S.anderson(xh, fh, 0.3, 7)
            U, lam_prev = out["U"], out["lam"]
        raise AssertionError("SCF did not converge")

    out, proj = converged(R0)
    f, _, _ = S.forces(n, h, 6, R0, Z, rc, out["phi"], proj, out["U"], out["g"])
    assert np.max(np.abs(f[0] + f[1])) < 1e-5            # no net force on an isolated pair
    d = 0.005
    for s in range(3):
        Rp, Rm = R0.copy(), R0.copy()
        Rp[0, s] += d
        Rm[0, s] -= d
        fd = -(converged(Rp)[0]["F"] - converged(Rm)[0]["F"]) / (2 * d)
        assert abs(fd - f[0, s]) < 5e-5, (s, fd, f[0, s])


def _smooth_bloch_orbitals(n, h, k, ns, rng):
    """ns orthonormal Bloch functions at k made of the 27 plane waves exp(i(k+G).x) with
    |G_s| <= 2 pi / L_s (smooth on the grid, so the discrete sums stand for integrals)."""
    import itertools
    L = np.array([n[s] * h[s] for s in range(3)])
    xs = synth.node_coords(n, h)
    Zg, Yg, Xg = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    P = np.stack([Xg.reshape(-1), Yg.reshape(-1), Zg.reshape(-1)], axis=1)
    U = np.zeros((ns, P.shape[0]), np.complex128)
    for t in itertools.product((-1, 0, 1), repeat=3):
        q = np.asarray(k) + np.array(t) * 2 * math.pi / L
        U += np.outer(rng.standard_normal(ns) + 1j * rng.standard_normal(ns), np.exp(1j * P @ q))
    return np.linalg.qr(U.T)[0].T


def test_bloch_nonlocal_force_is_minus_the_position_derivative_of_the_energy():
    """At k != 0, with the atom's projector box wrapping two faces: the Bloch nonlocal
    force (Section 3.6 with the phases of Eq. NonlocalPS:FD) equals minus the central
    difference, in the atom position, of the nonlocal energy 2 sum_n g_n sum_p gamma_p
    |Y_pn|^2 of fixed smooth orbitals (projectors rebuilt at each position).  The two
    agree to about 4e-5 relative (the box truncation at 3 rc and the per-box
    normalisation); a lost conjugate, a Bloch phase of the wrong sign in nabla_h or a
    wrong prefactor is an O(1) error."""
    n, h, n_o = (14, 13, 13), (0.5, 0.5, 0.5), 6
    L = np.array([n[s] * h[s] for s in range(3)])
    nd, dv = n[0] * n[1] * n[2], 0.125
    rng = np.random.default_rng(3)
    R = np.array([0.47, -0.41, 0.05]) * L
    gs, gp = np.array([0.8]), np.array([-0.6])
    k = (0.31, -0.17, 0.23)
    U = _smooth_bloch_orbitals(n, h, k, 6, rng)
    g = rng.uniform(0.2, 1.0, 6)

    def energy(Rx):
        proj = synth.make_projectors(n, h, Rx[None, :], 0.9, gs, gp)
        H = O.OracleH(n=n, h=h, fd_radius=n_o, k=k, veff=np.zeros(nd), proj=proj)
        c = H.nonlocal_coeffs(U / math.sqrt(dv))
        return 2.0 * sum(H.gamma[p] * float(np.sum(g * np.abs(c[p]) ** 2)) for p in range(len(H.gamma)))

    proj = synth.make_projectors(n, h, R[None, :], 0.9, gs, gp)
    f = S.nonlocal_forces_bloch(n, h, n_o, k, proj, U, g)
    d = 1e-3
    fd = np.array([-(energy(R + d * e) - energy(R - d * e)) / (2 * d) for e in np.eye(3)])
    assert np.max(np.abs(f[0] - fd)) < 3e-4 * np.max(np.abs(fd)), (f[0], fd)
    # the k-point weight scales the force
    assert np.allclose(S.nonlocal_forces_bloch(n, h, n_o, k, proj, U, g, w=0.25), 0.25 * f, rtol=1e-14, atol=0)


def test_bloch_nonlocal_force_at_gamma_is_the_real_orbital_formula():
    """At k = 0 with real orbitals the Bloch form reduces to the nonlocal part of the
    Gamma-point forces (same discrete sums, so to rounding)."""
    n, h, n_o = (14, 13, 13), (0.5, 0.5, 0.5), 6
    L = np.array([n[s] * h[s] for s in range(3)])
    nd = n[0] * n[1] * n[2]
    rng = np.random.default_rng(4)
    R = np.array([[0.45, -0.2, 0.1], [-0.3, 0.35, -0.44]]) * L
    proj = synth.make_projectors(n, h, R, 0.9, np.array([0.8, -0.5]), np.array([-0.6, 0.3]))
    U = np.linalg.qr(rng.standard_normal((nd, 5)))[0].T
    g = rng.uniform(0.2, 1.0, 5)
    _, _, f_nl = S.forces(n, h, n_o, R, np.array([1.0, 1.0]), np.array([0.7, 0.7]), np.zeros(nd), proj, U, g)
    f = S.nonlocal_forces_bloch(n, h, n_o, (0.0, 0.0, 0.0), proj, U, g)
    assert np.allclose(f, f_nl, rtol=0, atol=1e-12 * np.max(np.abs(f_nl)))


def test_starting_density_normalisation_and_atomic_special_case():
    """The learned starting density keeps N_e electrons for any correction, and with no
    correction reduces to the atomic superposition -b whose potential has phi = 0."""
    from paper_1603_04339_gb300 import synth
    sysd = synth.scf_small()
    wl = sysd.wl
    b, _, _ = S.pseudocharge(wl.n, wl.h, 6, wl.atoms, sysd.Z, sysd.rc)
    dv = wl.h[0] * wl.h[1] * wl.h[2]
    rng = np.random.default_rng(2)
    dy = rng.normal(0, 1, wl.nd)
    for scale in (0.0, 1e-3, 0.05):
        r = S.starting_density(b, dy, scale, sysd.nelec, wl.h)
        assert np.all(r >= 0.0)
        assert abs(dv * r.sum() - sysd.nelec) < 1e-12 * sysd.nelec
    r0 = S.starting_density(b, None, 0.0, sysd.nelec, wl.h)
    assert np.max(np.abs(r0 - np.maximum(-b, 0) * sysd.nelec / (dv * np.maximum(-b, 0).sum()))) < 1e-15
    assert abs(dv * (-b).sum() - sysd.nelec) < 1e-7          # int b = -N_e
    v = S.starting_potential(r0, b, wl.n, wl.h, 6)
    # rho0 + b vanishes up to the clipped truncation tail of b, so phi is small
    assert np.max(np.abs(v - S.lda(r0)[1])) < 1e-3 * np.max(np.abs(v))


def test_kpoint_iteration_reduces_to_gamma_for_repeated_kpoints():
    """The Brillouin-zone sum with the Gamma point twice at weights 1/2 is the Gamma-point
    iteration: the same Fermi level, density and free energy (a missing or doubled weight
    would change the electron count, the density or the band energy)."""
    from paper_1603_04339_gb300 import synth
    sysd = synth.scf_small()
    wl = sysd.wl
    b, e_self, _ = S.pseudocharge(wl.n, wl.h, 6, wl.atoms, sysd.Z, sysd.rc)
    H = O.OracleH(wl, veff=S.lda(-b)[1])
    one = S.scf_iteration(H, sysd.U0.copy(), None, sysd.v0, b, e_self, sysd.nelec, 0.01, wl.m)
    v0c = np.concatenate([sysd.v0, np.zeros(wl.nd)]).view(np.complex128)
    two = S.scf_iteration_k([H, H], [0.5, 0.5], [sysd.U0.copy(), sysd.U0.copy()], [None, None], v0c, b, e_self,
                            sysd.nelec, 0.01, wl.m)
    assert np.allclose(two["lam"], np.concatenate([one["lam"], one["lam"]]), rtol=0, atol=1e-12)
    assert abs(two["mu"] - one["mu"]) < 1e-12
    assert np.max(np.abs(two["rho"] - one["rho"])) < 1e-12 * np.max(one["rho"])
    assert abs(two["F"] - one["F"]) < 1e-11 * abs(one["F"])
    dv = wl.h[0] * wl.h[1] * wl.h[2]
    assert abs(dv * two["rho"].sum() - sysd.nelec) < 1e-9


def _golden_pw92():
    path = os.path.join(os.path.dirname(__file__), "golden", "pw92_correlation_expansions.txt")
    out = {}
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            out[line[0]] = (float(line[1]), float(line[2]))
    return out


def _pw92_expansion_from_parameters():
    """The high- and low-density coefficients implied by the oracle's six PW92
    parameters (series of G(rs) at rs -> 0 and rs -> infinity)."""
    A, a1, b1, b2, b3, b4 = S.PW92
    l = math.log(2.0 * A * b1)
    return {"c0": A, "c1": -2.0 * A * l, "c2": A * a1,
            "c3": -2.0 * A * a1 * l + 8.0 * A ** 3 * b1 ** 2 - 2.0 * A * b3 / b1,
            "d0": a1 / b4, "d1": a1 * b3 / b4 ** 2, "beta2": 2.0 * A * b1 ** 2}


def test_pw92_parameters_reproduce_the_published_expansion_coefficients():
    """Every one of A, alpha1, beta1..beta4 is tied to a coefficient of Perdew and
    Wang's Table I (tests/golden): a typo or a swap of any parameter moves at
    least one of c1 (beta1), beta2 = 2 A beta1^2, c2 (alpha1), c3 (beta3), d0 (beta4)
    or d1 far outside its tolerance."""
    gold = _golden_pw92()
    got = _pw92_expansion_from_parameters()
    for name, (val, tol) in gold.items():
        assert abs(got[name] - val) < tol, (name, got[name], val)
    assert abs(S.PW92[3] - got["beta2"]) < 1e-4
    # a planted swap or typo is caught: each single change breaks a coefficient
    base = list(S.PW92)
    for i in range(6):
        for bad in (base[i] * 1.01, base[(i + 1) % 6]):
            trial = base.copy()
            trial[i] = bad
            saved = S.PW92
            try:
                S.PW92 = tuple(trial)
                g2 = _pw92_expansion_from_parameters()
            finally:
                S.PW92 = saved
            off = [abs(g2[n] - v) > t for n, (v, t) in gold.items()]
            off.append(abs(trial[3] - g2["beta2"]) > 1e-4)
            assert any(off), (i, bad)


def test_pw92_correlation_has_the_published_asymptotic_series():
    """The oracle's eps_c (eps_xc minus Slater exchange) follows the high-density
    series c0 ln rs - c1 + c2 rs ln rs - c3 rs and the low-density series
    -d0/rs + d1/rs^1.5, with the coefficients implied by its parameters (which the
    previous test ties to Perdew and Wang's table): this pins the interpolation
    formula itself.  rs stays >= 1e-4 so that subtracting the exchange energy
    (which grows as 1/rs) keeps the rs terms above FP64 rounding."""
    c = _pw92_expansion_from_parameters()

    def ec(rs):
        rs = np.asarray(rs, dtype=np.float64)
        rho = 3.0 / (4.0 * math.pi * rs ** 3)
        eps, _ = S.lda(rho)
        ex = -(3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
        return eps - ex

    for rs in (1e-4, 3e-4):
        g = ec(rs) - (c["c0"] * math.log(rs) - c["c1"])            # the rs-order terms
        t = c["c2"] * rs * math.log(rs) - c["c3"] * rs
        assert abs(g - t) < 1e-3 * abs(t), (rs, g, t)
        # the c3 term alone is resolved (it is 1/7 of the rs-order terms here)
        assert abs((g - c["c2"] * rs * math.log(rs)) / (-c["c3"] * rs) - 1.0) < 1e-2
    for rs in (1e7, 1e8, 1e9):
        e = float(ec(rs))
        # remainder of the two-term series is O(1/rs^2) (coefficient about -3.7)
        assert abs(e * rs + c["d0"] - c["d1"] / math.sqrt(rs)) < 5.0 / rs, (rs, e)
        assert abs((e + c["d0"] / rs) * rs ** 1.5 - c["d1"]) < 5.0 / math.sqrt(rs), (rs, e)
