"""FP64 CPU oracle for one SCF iteration around the CheFSI step (SPARC, arXiv:1603.04339).

TEST INFRASTRUCTURE ONLY, like sparc_oracle.py: only the tests, the smoke check and
the benchmark's CPU baseline may import it, and it shares no code with the CUDA
library.  Each function restates one passage of the paper (cited in its docstring),
in the paper's order, with numpy (and scipy's Brent root finder as the library step
the paper names).

Readings where the paper is silent or leaves a choice (also in the design notes):
  * the local pseudopotential of atom I is V_I(r) = -Z_I erf(r/rc_I)/r (a stand-in
    for the Troullier-Martins tables); its discrete pseudocharge
    b_I = -(1/4pi) lap_h V_I (Eq. PseudochargeDiscrete) is kept on a cube of
    half-width ceil(6 rc_I / h) nodes around the atom's nearest node, which meets the
    paper's charge tolerance eps_b = 1e-8 (Eq. PseudochargeRadiusChoice), and it
    integrates to -Z_I (the sign that makes the cell neutral, int b = -N_e,
    Eq. IntegralPseudocharges);
  * E_c (overlapping pseudocharges) is zero: the Gaussian pseudocharges of the
    synthetic atoms do not overlap to 1e-12;
  * the Poisson problem -lap_h phi = 4 pi (rho + b) is periodic; phi has zero mean
    and the mean of the right-hand side (the truncation error of b) is removed;
  * LDA: Slater exchange and the Perdew-Wang 1992 parametrisation of the
    correlation energy of the unpolarised electron gas (Section 5);
  * Anderson extrapolation on V_eff with relaxation beta and history m (Section 5):
    with f = V_out - V_in, gamma solves the normal equations of min |f_k - dF gamma|
    over the last m differences (dF^T dF regularised by 1e-12 of its trace, so that a
    converged history stays solvable), V_next = (V_k - dX gamma) + beta (f_k - dF gamma);
  * the free energy (Eq. FreeEnergy:GroundState:DFT:discrete) is evaluated with the
    band energy of H[V_in] and the grid terms of the output density rho_out (its own
    phi and V_xc), which is the paper's expression at self-consistency;
  * the Fermi level is bracketed by [lambda_min - 1, lambda_max + 1] Ha and found to
    1e-12 Ha.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.optimize
from scipy.special import erf

from . import sparc_oracle as O

__all__ = ["local_potential", "pseudocharge", "occupations", "fermi_level", "density",
           "poisson", "lda", "anderson", "free_energy", "entropy_term", "PW92"]

# Perdew-Wang 1992 parameters of the correlation energy of the unpolarised gas
# (A, alpha1, beta1..beta4; p = 1).  A equals (1 - ln 2)/pi^2, the exact high-density
# coefficient of ln(rs), which the pins check.
PW92 = (0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294)


def _coords(n, h):
    """Node coordinates x_i = -L/2 + i h per axis (Section 3.1)."""
    return [(-0.5 * n[s] * h[s] + h[s] * np.arange(n[s])) for s in range(3)]


def local_potential(r: np.ndarray, Z: float, rc: float) -> np.ndarray:
    """V_I(r) = -Z erf(r/rc)/r, with its limit -2Z/(sqrt(pi) rc) at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = r < 1e-12
    out[~small] = -Z * erf(r[~small] / rc) / r[~small]
    out[small] = -2.0 * Z / (math.sqrt(math.pi) * rc)
    return out


def pseudocharge(n, h, n_o, R, Z, rc):
    """Discrete pseudocharge b and self energy E_self^h (Eqs. PseudochargeDiscrete and
    DiscreteEself; the loop over atoms of Algorithm "Pseudocharge density generation").

    For each atom: V_I on its cube plus an n_o halo (unwrapped node coordinates),
    b_I = -(1/4pi) lap_h V_I on the cube, added into b with periodic wrap, and
    E_self += 1/2 h1h2h3 sum_cube b_I V_I.  Returns (b[Nd], E_self, per-atom charges)."""
    n = tuple(int(v) for v in n)
    h = tuple(float(v) for v in h)
    L = [n[s] * h[s] for s in range(3)]
    w = [O.fd_weights(n_o, h[s]) for s in range(3)]
    dv = h[0] * h[1] * h[2]
    b = np.zeros(n[::-1], dtype=np.float64)          # [k][j][i]
    e_self = 0.0
    charges = []
    for I in range(len(Z)):
        nb = [int(math.ceil(6.0 * rc[I] / h[s])) for s in range(3)]
        c = [int(round((R[I][s] + 0.5 * L[s]) / h[s])) for s in range(3)]   # nearest node
        lo = [c[s] - nb[s] - n_o for s in range(3)]
        m = [2 * nb[s] + 1 + 2 * n_o for s in range(3)]
        xs = [(-0.5 * L[s] + h[s] * (lo[s] + np.arange(m[s]))) - R[I][s] for s in range(3)]
        X, Y, Zc = np.meshgrid(xs[0], xs[1], xs[2], indexing="ij")
        V = local_potential(np.sqrt(X * X + Y * Y + Zc * Zc), Z[I], rc[I])   # [i][j][k]
        inner = tuple(slice(n_o, n_o + 2 * nb[s] + 1) for s in range(3))
        lap = np.zeros([2 * nb[s] + 1 for s in range(3)])
        for s in range(3):
            acc = 2.0 * w[s][0] * V[inner]
            for p in range(1, n_o + 1):
                sl_p = list(inner)
                sl_m = list(inner)
                sl_p[s] = slice(n_o + p, n_o + p + 2 * nb[s] + 1)
                sl_m[s] = slice(n_o - p, n_o - p + 2 * nb[s] + 1)
                acc = acc + w[s][p] * (V[tuple(sl_p)] + V[tuple(sl_m)])
            lap = lap + acc
        bI = -lap / (4.0 * math.pi)
        e_self += 0.5 * dv * float(np.sum(bI * V[inner]))
        charges.append(dv * float(np.sum(bI)))
        ii = [np.mod(lo[s] + n_o + np.arange(2 * nb[s] + 1), n[s]) for s in range(3)]
        np.add.at(b, np.ix_(ii[2], ii[1], ii[0]), np.transpose(bI, (2, 1, 0)))
    return b.reshape(-1), e_self, np.array(charges)


def occupations(lam: np.ndarray, mu: float, kT: float) -> np.ndarray:
    """g_n = (1 + exp((lambda_n - lambda_f)/kT))^-1 (Eq. EL), written without overflow."""
    x = (np.asarray(lam, dtype=np.float64) - mu) / kT
    out = np.empty_like(x)
    pos = x > 0
    e = np.exp(-x[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def fermi_level(lam: np.ndarray, Ne: float, kT: float, wk=1.0) -> float:
    """lambda_f such that 2 sum_n w_n g_n = N_e, by Brent's method (Section 5); w: one
    weight, or the k-point weight of every value (the Brillouin-zone sum of Eq. EL)."""
    lam = np.asarray(lam, dtype=np.float64)
    f = lambda mu: 2.0 * float(np.sum(wk * occupations(lam, mu, kT))) - Ne
    return scipy.optimize.brentq(f, lam.min() - 1.0, lam.max() + 1.0, xtol=1e-14, maxiter=500)


def density(U: np.ndarray, g: np.ndarray, h, wk: float = 1.0) -> np.ndarray:
    """rho = 2 sum_n w g_n |u_n|^2 (Section 3.4, "Electron density calculation"), with the
    orbitals U (rows) orthonormal in the Euclidean sense, so u_n = U_n / sqrt(h1h2h3)."""
    dv = h[0] * h[1] * h[2]
    return 2.0 * wk * np.einsum("n,ng->g", np.asarray(g, dtype=np.float64), np.abs(U) ** 2) / dv


def poisson(rhs_density: np.ndarray, n, h, n_o: int) -> np.ndarray:
    """phi with -(1/4pi) lap_h phi = rhs_density (Eq. EL's Poisson equation, FD Laplacian
    of Eq. FD:Laplacian), periodic, zero mean.  The FD Laplacian is circulant on the
    periodic grid, so it is diagonal in the discrete Fourier basis with eigenvalues
    -2 fd_symbol (the oracle's own closed form), and the solve is exact up to rounding."""
    n = tuple(int(v) for v in n)
    f = np.asarray(rhs_density, dtype=np.float64).reshape(n[::-1])
    f = f - f.mean()
    F = np.fft.fftn(f)
    lam = np.zeros(n[::-1])
    for s, ax in ((0, 2), (1, 1), (2, 0)):
        theta_h = 2.0 * math.pi * np.fft.fftfreq(n[s])          # theta * h
        sym = 2.0 * O.fd_symbol(theta_h, n_o, h[s])              # -lap symbol along axis s
        shape = [1, 1, 1]
        shape[ax] = n[s]
        lam = lam + sym.reshape(shape)
    lam.flat[0] = 1.0
    P = 4.0 * math.pi * F / lam
    P.flat[0] = 0.0
    return np.real(np.fft.ifftn(P)).reshape(-1)


def lda(rho: np.ndarray):
    """(eps_xc, V_xc) of the LDA (Section 2, Exchange-correlation energy; Section 5: Slater
    exchange, Perdew-Wang 1992 correlation), for the unpolarised density rho."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    ok = rho > 1e-30
    r = rho[ok]
    ex = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * r ** (1.0 / 3.0)
    vx = (4.0 / 3.0) * ex
    A, a1, b1, b2, b3, b4 = PW92
    rs = (3.0 / (4.0 * math.pi * r)) ** (1.0 / 3.0)
    srs = np.sqrt(rs)
    Q0 = -2.0 * A * (1.0 + a1 * rs)
    Q1 = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    Q1p = A * (b1 / srs + 2.0 * b2 + 3.0 * b3 * srs + 4.0 * b4 * rs)
    L = np.log1p(1.0 / Q1)
    ec = Q0 * L
    dec = -2.0 * A * a1 * L - Q0 * Q1p / (Q1 * Q1 + Q1)
    vc = ec - rs / 3.0 * dec
    eps[ok] = ex + ec
    v[ok] = vx + vc
    return eps, v


def entropy_term(g: np.ndarray, kT: float, wk=1.0) -> float:
    """2 kT sum_n w_n (g ln g + (1-g) ln(1-g)), with 0 ln 0 = 0 (w as in fermi_level)."""
    g = np.asarray(g, dtype=np.float64)
    t = np.zeros_like(g)
    m = (g > 0) & (g < 1)
    t[m] = g[m] * np.log(g[m]) + (1.0 - g[m]) * np.log(1.0 - g[m])
    return 2.0 * kT * float(np.sum(wk * t))


def free_energy(lam, g, rho, b, phi, eps_xc, v_xc, h, e_self, kT, e_c=0.0, wk=1.0):
    """Eq. FreeEnergy:GroundState:DFT:discrete.  Returns (F, parts)."""
    dv = h[0] * h[1] * h[2]
    e_band = 2.0 * float(np.sum(wk * np.asarray(g) * np.asarray(lam)))
    e_xc = dv * float(np.sum(eps_xc * rho - v_xc * rho))
    e_el = dv * float(np.sum(0.5 * (b - rho) * phi))
    e_ent = entropy_term(g, kT, wk)
    F = e_band + e_xc + e_el - e_self + e_c + e_ent
    return F, {"band": e_band, "xc": e_xc, "el": e_el, "self": e_self, "entropy": e_ent}


def anderson(x_hist, f_hist, beta: float, m: int) -> np.ndarray:
    """Anderson extrapolation (Section 5): x_hist, f_hist are the lists of the inputs
    x_j = V_in and residuals f_j = V_out - V_in so far (last entry = current).  With
    dX, dF the differences of the last min(k, m) pairs, gamma minimises |f_k - dF gamma|
    (normal equations, regularised by 1e-12 of the trace of dF^T dF), and the next
    input is (x_k - dX gamma) + beta (f_k - dF gamma)."""
    xk, fk = x_hist[-1], f_hist[-1]
    k = len(x_hist) - 1
    mm = min(k, m)
    if mm == 0:
        return xk + beta * fk
    dX = np.stack([x_hist[-1 - j] - x_hist[-2 - j] for j in range(mm)], axis=1)
    dF = np.stack([f_hist[-1 - j] - f_hist[-2 - j] for j in range(mm)], axis=1)
    Gm = dF.T @ dF
    Gm = Gm + 1e-12 * np.trace(Gm) * np.eye(mm)   # keeps the normal equations solvable at convergence
    gamma = np.linalg.solve(Gm, dF.T @ fk)
    return (xk - dX @ gamma) + beta * (fk - dF @ gamma)


def scf_iteration(H: "O.OracleH", U, lam_prev, v0, b, e_self, Ne, kT, m, lanczos_k=10, passes=1):
    """One SCF iteration at fixed V_in = H.veff (Section 3.4 and Eq. EL), in the order
    the CUDA path takes it: filter bounds by Lanczos (Section 5; the cutoff is the
    largest previous Ritz value, or the Weyl estimate a0 + (b - a0)(Ns/Nd)^(2/3) at
    the first iteration, and a0 the smallest), scaled Chebyshev filter, Rayleigh-Ritz
    (`passes` times: Section 4 repeats CheFSI at the first iteration's fixed
    potential, each pass bounded by the previous pass's Ritz values), Fermi level,
    density, Poisson, LDA, V_out = phi + V_xc and the free energy.
    Returns a dict of every intermediate."""
    U = np.atleast_2d(U)
    ns = U.shape[0]
    a0l, bb, _ = O.lanczos_bounds(H, v0, lanczos_k)
    for _ in range(passes):
        if lam_prev is None:
            a0 = a0l
            a = a0 + (bb - a0) * (ns / H.nd) ** (2.0 / 3.0)
        else:
            a0 = float(lam_prev[0])
            a = float(lam_prev[-1])
        Yf = O.cheb_filter(H, U, m, a, bb, a0)
        lam, U, _, _ = O.rayleigh_ritz(H, Yf)
        lam_prev = lam
    Uo = U
    mu = fermi_level(lam, Ne, kT)
    g = occupations(lam, mu, kT)
    rho = density(Uo, g, H.h)
    phi = poisson(rho + b, H.n, H.h, H.n_o)
    eps, vxc = lda(rho)
    v_out = phi + vxc
    F, parts = free_energy(lam, g, rho, b, phi, eps, vxc, H.h, e_self, kT)
    return {"a0": a0, "a": a, "b": bb, "lam": lam, "U": Uo, "mu": mu, "g": g, "rho": rho,
            "phi": phi, "eps": eps, "vxc": vxc, "v_out": v_out, "F": F, "parts": parts}


def starting_density(b, dy, scale, Ne, h):
    """Starting density of the learned initial guess (project-added; the paper starts
    from the superposition of atomic densities, which is -b for the Gaussian atoms):
    rho0 = max(-b + scale dy, 0), scaled so that h1 h2 h3 sum rho0 = N_e."""
    r = -np.asarray(b, dtype=np.float64)
    if dy is not None:
        r = r + scale * np.asarray(dy, dtype=np.float64)
    r = np.maximum(r, 0.0)
    return r * (Ne / (h[0] * h[1] * h[2] * r.sum()))


def starting_potential(rho0, b, n, h, n_o):
    """V_in = phi[rho0 + b] + V_xc[rho0] (Poisson and LDA of this module)."""
    return poisson(rho0 + b, n, h, n_o) + lda(rho0)[1]


def scf_iteration_k(Hs, wk, Us, lam_prevs, v0, b, e_self, Ne, kT, m, lanczos_k=10, passes=1):
    """One SCF iteration with the Brillouin-zone sum over k-points (Section 2: the
    density and the electron count are k-point-weighted sums; Eq. EL): per k-point the
    CheFSI of scf_iteration (its Lanczos start vector v0 is complex; a k = 0
    Hamiltonian takes the first Nd doubles of its (re, im) storage, as the CUDA path
    does), then one Fermi level for all Ritz values with their k-point weights,
    rho = sum_k density(U_k, g_k, h, w_k), and the grid steps of scf_iteration."""
    nk = len(Hs)
    lams, Uo, bounds = [], [], []
    for k in range(nk):
        H = Hs[k]
        v = v0 if H.is_complex else np.ascontiguousarray(v0, dtype=np.complex128).view(np.float64)[: H.nd]
        a0l, bb, _ = O.lanczos_bounds(H, v, lanczos_k)
        U, lp = np.atleast_2d(Us[k]), lam_prevs[k]
        ns = U.shape[0]
        for _ in range(passes):
            if lp is None:
                a0 = a0l
                a = a0 + (bb - a0) * (ns / H.nd) ** (2.0 / 3.0)
            else:
                a0, a = float(lp[0]), float(lp[-1])
            Yf = O.cheb_filter(H, U, m, a, bb, a0)
            lp, U, _, _ = O.rayleigh_ritz(H, Yf)
        lams.append(lp)
        Uo.append(U)
        bounds.append((a0, a, bb))
    lam = np.concatenate(lams)
    w = np.concatenate([np.full(len(l), wk[k]) for k, l in enumerate(lams)])
    mu = fermi_level(lam, Ne, kT, w)
    g = occupations(lam, mu, kT)
    ns = len(lams[0])
    H0 = Hs[0]
    rho = sum(density(Uo[k], g[k * ns:(k + 1) * ns], H0.h, wk[k]) for k in range(nk))
    phi = poisson(rho + b, H0.n, H0.h, H0.n_o)
    eps, vxc = lda(rho)
    v_out = phi + vxc
    F, parts = free_energy(lam, g, rho, b, phi, eps, vxc, H0.h, e_self, kT, wk=w)
    return {"lam": lam, "U": Uo, "mu": mu, "g": g, "rho": rho, "phi": phi, "v_out": v_out, "F": F,
            "parts": parts, "bounds": bounds}


def grad_weights(n_o: int, h: float) -> np.ndarray:
    """Central first-derivative weights w~_p, p = 1..n_o (the gradient formula of
    Section 3.1): w~_p = (-1)^(p+1) (n_o!)^2 / (h p (n_o-p)! (n_o+p)!)."""
    fo = math.factorial(n_o)
    return np.array([0.0] + [(-1) ** (p + 1) * fo * fo / (h * p * math.factorial(n_o - p) * math.factorial(n_o + p))
                             for p in range(1, n_o + 1)])


def grad_h(F: np.ndarray, n, h, n_o: int) -> np.ndarray:
    """nabla_h F for F of shape (..., n3, n2, n1), periodic (Eq. gradient:approximate).
    Returns shape (3, ...)."""
    out = []
    for s in range(3):
        ax = F.ndim - 1 - s
        w = grad_weights(n_o, h[s])
        g = np.zeros_like(F)
        for p in range(1, n_o + 1):
            g = g + w[p] * (np.roll(F, -p, axis=ax) - np.roll(F, p, axis=ax))
        out.append(g)
    return np.stack(out)


def nonlocal_forces_bloch(n, h, n_o, k, proj, U, g, w=1.0, natom=None):
    """Nonlocal forces of the Bloch orbitals of one k-point (Section 3.6, Eq.
    NonlocForce:Discrete, with the image phases of Eq. NonlocalPS:FD):

      f_J = -4 w sum_n g_n sum_{p of atom J} gamma_p Re(conj(Y_pn) W_pn),
      Y_pn = h1h2h3 sum_g conj(chi~_p[g]) psi_n[g],
      W_pn = h1h2h3 sum_g conj(chi~_p[g]) (nabla_h psi_n)[g],

    psi = U / sqrt(h1h2h3) (rows of U), nabla_h the gradient of Eq.
    gradient:approximate with the Bloch wrap of Section 3.1 (a neighbour across a face
    carries exp(+-i k_s L_s)).  The derivative of chi~ with respect to the atom
    position is moved onto psi by summation by parts, exact for the antisymmetric
    nabla_h on two grid functions of the same k.  At k = 0 with real U this is the
    nonlocal part of forces(); over k-points the forces add with the weights w."""
    n = tuple(int(v) for v in n)
    h = tuple(float(v) for v in h)
    dv = h[0] * h[1] * h[2]
    nd = n[0] * n[1] * n[2]
    if natom is None:
        natom = int(np.max(proj.atom)) + 1 if proj.nproj else 0
    Hk = O.OracleH(n=n, h=h, fd_radius=n_o, k=k, veff=np.zeros(nd), proj=proj)
    U = np.atleast_2d(np.asarray(U)).astype(np.complex128)
    U3 = U.reshape((U.shape[0],) + n[::-1])
    grads = []
    for s in range(3):
        ax = U3.ndim - 1 - s
        kL = float(k[s]) * n[s] * h[s]
        wg = grad_weights(n_o, h[s])
        G = np.zeros_like(U3)
        for p in range(1, n_o + 1):
            G = G + wg[p] * (O._shift(U3, p, ax, n[s], kL) - O._shift(U3, -p, ax, n[s], kL))
        grads.append(G.reshape(U.shape[0], nd))
    gg = np.asarray(g, dtype=np.float64)
    f = np.zeros((natom, 3))
    for p, (gi, v) in enumerate(zip(Hk.pidx, Hk.pval)):
        J = int(proj.atom[p])
        Y = math.sqrt(dv) * (U[:, gi] @ np.conj(v))
        for s in range(3):
            W = math.sqrt(dv) * (grads[s][:, gi] @ np.conj(v))
            f[J, s] += -4.0 * w * Hk.gamma[p] * float(np.sum(gg * np.real(np.conj(Y) * W)))
    return f


def forces(n, h, n_o, R, Z, rc, phi, proj, U, g, gamma_atoms=None):
    """Atomic forces at the Gamma point (Section 3.6): f = f_loc + f_c + f_nloc, with
    f_c = 0 (no overlapping pseudocharges, see the readings).

    f_loc (Eq. LocalForce:Discrete): h1h2h3 sum over the atom's cube nodes of
      nabla_h b_J (phi - V_J), b_J = -(1/4pi) lap_h V_J evaluated at any node from the
      analytic V_J (the cube is the pseudocharge cube of the atom, images included).
    f_nloc (Eq. NonlocForce:Discrete): -4 sum_n g_n sum_lm gamma_Jl Y_Jnlm W_Jnlm with
      Y = h1h2h3 sum psi chi, W = h1h2h3 sum nabla_h psi chi over the projector box
      (psi = U / sqrt(h1h2h3), real at the Gamma point).
    Returns (f [natom, 3], f_loc, f_nloc)."""
    n = tuple(int(v) for v in n)
    h = tuple(float(v) for v in h)
    L = [n[s] * h[s] for s in range(3)]
    dv = h[0] * h[1] * h[2]
    wl = [O.fd_weights(n_o, h[s]) for s in range(3)]
    wg = [grad_weights(n_o, h[s]) for s in range(3)]
    phi3 = np.asarray(phi, dtype=np.float64).reshape(n[::-1])
    natom = len(Z)
    f_loc = np.zeros((natom, 3))
    for I in range(natom):
        nb = [int(math.ceil(6.0 * rc[I] / h[s])) for s in range(3)]
        c = [int(round((R[I][s] + 0.5 * L[s]) / h[s])) for s in range(3)]
        # V_I on the cube plus a 2 n_o halo; b_I on the cube plus an n_o halo
        H2 = 2 * n_o
        lo = [c[s] - nb[s] - H2 for s in range(3)]
        m = [2 * nb[s] + 1 + 2 * H2 for s in range(3)]
        xs = [(-0.5 * L[s] + h[s] * (lo[s] + np.arange(m[s]))) - R[I][s] for s in range(3)]
        X, Y, Zc = np.meshgrid(xs[0], xs[1], xs[2], indexing="ij")
        V = local_potential(np.sqrt(X * X + Y * Y + Zc * Zc), Z[I], rc[I])    # [i][j][k]
        mb = [2 * nb[s] + 1 + 2 * n_o for s in range(3)]
        inner_b = tuple(slice(n_o, n_o + mb[s]) for s in range(3))
        lap = np.zeros(mb)
        for s in range(3):
            acc = 2.0 * wl[s][0] * V[inner_b]
            for p in range(1, n_o + 1):
                sp, sm = list(inner_b), list(inner_b)
                sp[s] = slice(n_o + p, n_o + p + mb[s])
                sm[s] = slice(n_o - p, n_o - p + mb[s])
                acc = acc + wl[s][p] * (V[tuple(sp)] + V[tuple(sm)])
            lap = lap + acc
        bI = -lap / (4.0 * math.pi)                                             # cube + n_o halo
        cube = tuple(slice(n_o, n_o + 2 * nb[s] + 1) for s in range(3))
        ii = [np.mod(c[s] - nb[s] + np.arange(2 * nb[s] + 1), n[s]) for s in range(3)]
        phic = np.transpose(phi3[np.ix_(ii[2], ii[1], ii[0])], (2, 1, 0))      # [i][j][k]
        Vc = V[tuple(slice(H2, H2 + 2 * nb[s] + 1) for s in range(3))]
        for s in range(3):
            gb = np.zeros([2 * nb[t] + 1 for t in range(3)])
            for p in range(1, n_o + 1):
                sp, sm = list(cube), list(cube)
                sp[s] = slice(n_o + p, n_o + p + 2 * nb[s] + 1)
                sm[s] = slice(n_o - p, n_o - p + 2 * nb[s] + 1)
                gb = gb + wg[s][p] * (bI[tuple(sp)] - bI[tuple(sm)])
            f_loc[I, s] = dv * float(np.sum(gb * (phic - Vc)))
    # nonlocal
    f_nl = np.zeros((natom, 3))
    U3 = np.asarray(U, dtype=np.float64).reshape((-1,) + n[::-1])
    G = grad_h(U3, n, h, n_o)                                                  # (3, ns, n3, n2, n1)
    for p in range(proj.nproj):
        J = int(proj.atom[p])
        lo = proj.box_lo[p]
        bn = proj.box_n[p]
        chi = proj.chi[proj.chi_off[p]: proj.chi_off[p] + int(np.prod(bn))].reshape(bn[2], bn[1], bn[0])
        idx = [np.mod(lo[s] + np.arange(bn[s]), n[s]) for s in range(3)]
        Ub = U3[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]                       # (ns, bz, by, bx)
        Yp = math.sqrt(dv) * np.einsum("nzyx,zyx->n", Ub, chi)
        for s in range(3):
            Gb = G[s][:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
            Wp = math.sqrt(dv) * np.einsum("nzyx,zyx->n", Gb, chi)
            f_nl[J, s] += -4.0 * float(proj.gamma[p]) * float(np.sum(np.asarray(g) * Yp * Wp))
    return f_loc + f_nl, f_loc, f_nl
