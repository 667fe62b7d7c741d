"""FP64 CPU oracle for the CheFSI step of real-space Kohn-Sham DFT (SPARC, arXiv:1603.04339).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the tests, the smoke check and the timed
CPU baseline of the benchmark may import it; the product path never does.  It
shares no code with the CUDA library: it imports numpy (and, for one triangular
solve, scipy) and nothing else from this repository.

Every function follows one passage of the paper, cited in its docstring.  The
arithmetic is written in the paper's order and notation, vectorised with numpy
over the grid but with no blocking, fusion or reordering beyond that.

Data conventions:
  * grid index g = i + n1*(j + n2*k), node i on axis s at x_i = -L_s/2 + i*h_s
    (Section 3.1: cuboid cell with its origin at the centre, L_s = n_s*h_s);
  * a block of orbitals is an array of shape (Ns, Nd), i.e. the columns of the
    Nd x Ns matrix U(k) of Section 3.1 stored one after the other;
  * Bloch-periodic values: psi(x + L_s e_s) = exp(i k_s L_s) psi(x)
    (Bloch's theorem, Section 3, applied to psi = e^{ik.x} u).

Readings where the paper is silent (each is also listed in the design notes):
  * the Hamiltonian is discretised in psi-form: the finite-difference Laplacian
    acts on psi with Bloch-periodic wrap of indices, the nonlocal operator uses
    the image phases of Eq. NonlocalPS:FD, and H = -1/2 lap + V_eff + V_nl;
  * the FD sum of Eq. FD:Laplacian starts at p = 0, so the centre node enters
    with weight 2*w_0 per axis;
  * the filter is returned in the scaled form Y = C_m((H-c)/e) X / C_m((a0-c)/e),
    which spans the same subspace as Eq. ChebFilter;
  * the Lanczos bounds are a0 = min Ritz value and b = max Ritz value + |beta_k|;
  * the Rayleigh-Ritz step orthonormalises through a Cholesky factor of M~.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

__all__ = [
    "fd_weights", "laplacian", "OracleH", "cheb_filter", "cheb_filter_unscaled",
    "cheb_T", "lanczos_bounds", "rayleigh_ritz", "chefsi_step", "fd_symbol",
]


def fd_weights(n_o: int, h: float) -> np.ndarray:
    """Central FD weights w_{p,s}, p = 0..n_o, for the second derivative (Eq. weightsLap).

    w_0 = -(1/h^2) sum_{q=1}^{n_o} 1/q^2
    w_p = 2 (-1)^{p+1} (n_o!)^2 / (h^2 p^2 (n_o-p)! (n_o+p)!)
    """
    w = np.zeros(n_o + 1, dtype=np.float64)
    w[0] = -sum(1.0 / (q * q) for q in range(1, n_o + 1)) / (h * h)
    fo = math.factorial(n_o)
    for p in range(1, n_o + 1):
        w[p] = (2.0 * (-1) ** (p + 1) * fo * fo
                / (h * h * p * p * math.factorial(n_o - p) * math.factorial(n_o + p)))
    return w


def fd_symbol(theta_h: np.ndarray, n_o: int, h: float) -> np.ndarray:
    """-(1/2) times the FD Laplacian symbol on exp(i*theta*x) along one axis (Eq. FD:Laplacian)."""
    w = fd_weights(n_o, h)
    s = 2.0 * w[0] * np.ones_like(theta_h)
    for p in range(1, n_o + 1):
        s = s + 2.0 * w[p] * np.cos(p * theta_h)
    return -0.5 * s


def _shift(F: np.ndarray, p: int, axis: int, n: int, kL: float) -> np.ndarray:
    """Values F at node i+p along `axis`, indices mapped to their periodic image.

    Section 3.1: an index outside the grid is mapped to its periodic image; for
    a Bloch function the image carries the factor exp(i k_s L_s t) where t is
    the number of cells crossed, t = floor((i+p)/n).
    """
    out = np.roll(F, -p, axis=axis)
    if kL != 0.0:
        t = np.floor_divide(np.arange(n) + p, n)
        ph = np.exp(1j * kL * t)
        shape = [1] * F.ndim
        shape[axis] = n
        out = out * ph.reshape(shape)
    return out


def laplacian(F: np.ndarray, n, h, n_o: int, k=(0.0, 0.0, 0.0)) -> np.ndarray:
    """nabla_h^2 F on a block F of shape (Ns, n3, n2, n1) (Eq. FD:Laplacian).

    sum_s sum_{p=0}^{n_o} w_{p,s} (F(g + p e_s) + F(g - p e_s)), Bloch-periodic wrap.
    """
    out = np.zeros_like(F)
    for s in range(3):
        axis = F.ndim - 1 - s          # x is the last array axis
        w = fd_weights(n_o, h[s])
        kL = float(k[s]) * n[s] * h[s]
        out = out + w[0] * (F + F)
        for p in range(1, n_o + 1):
            out = out + w[p] * (_shift(F, p, axis, n[s], kL) + _shift(F, -p, axis, n[s], kL))
    return out


class OracleH:
    """Discrete Hamiltonian H(k) = -1/2 nabla_h^2 + V_eff + V_nl (Eqn. EL, Eq. NonlocalPS:FD).

    Built from plain arrays: n, h, fd_radius, k, veff and the projector boxes
    (box_lo, box_n, chi_off, chi, gamma).  `wl` may be any object with those
    attributes (kpts[kidx] gives k) or None if everything is passed explicitly.
    """

    def __init__(self, wl=None, kidx: int = 0, *, n=None, h=None, fd_radius=None, k=None,
                 veff=None, proj=None):
        self.n = tuple(int(v) for v in (n if n is not None else wl.n))
        self.h = tuple(float(v) for v in (h if h is not None else wl.h))
        self.n_o = int(fd_radius if fd_radius is not None else wl.fd_radius)
        kk = k if k is not None else wl.kpts[kidx]
        self.k = tuple(float(v) for v in kk)
        self.veff = np.asarray(veff if veff is not None else wl.veff, dtype=np.float64)
        self.proj = proj if proj is not None else wl.proj
        self.nd = self.n[0] * self.n[1] * self.n[2]
        self.dv = self.h[0] * self.h[1] * self.h[2]
        self.is_complex = any(v != 0.0 for v in self.k)
        self._build_projectors()

    def _build_projectors(self):
        """chi~_p[g] = sum_images exp(i k.T) chi_p(x_g - R - T), on the box nodes (Eq. NonlocalPS:FD).

        A box node q (unwrapped) lies in the image of the cell shifted by
        t = floor(q/n) cells; it is grid node q mod n.  Its contribution to
        chi~ at that node carries exp(-i k.(t L)) (the image of the atom seen
        from the home cell sits at R - t L).
        """
        P = self.proj
        self.pidx, self.pval, self.gamma = [], [], []
        for p in range(P.nproj):
            lo = [int(v) for v in P.box_lo[p]]
            nb = [int(v) for v in P.box_n[p]]
            size = nb[0] * nb[1] * nb[2]
            vals = np.asarray(P.chi[int(P.chi_off[p]): int(P.chi_off[p]) + size], np.float64)
            axes_g, axes_ph = [], []
            for s in range(3):
                q = lo[s] + np.arange(nb[s])
                g = np.mod(q, self.n[s])
                t = np.floor_divide(q, self.n[s])
                axes_g.append(g)
                axes_ph.append(np.exp(-1j * self.k[s] * self.n[s] * self.h[s] * t))
            gz, gy, gx = np.meshgrid(axes_g[2], axes_g[1], axes_g[0], indexing="ij")
            flat = (gx + self.n[0] * (gy + self.n[1] * gz)).reshape(-1)
            if self.is_complex:
                pz, py, px = np.meshgrid(axes_ph[2], axes_ph[1], axes_ph[0], indexing="ij")
                vals = vals * (px * py * pz).reshape(-1)
            self.pidx.append(flat)
            self.pval.append(vals)
            self.gamma.append(float(P.gamma[p]))

    def _dtype(self, X):
        return np.complex128 if (self.is_complex or np.iscomplexobj(X)) else np.float64

    def nonlocal_coeffs(self, X: np.ndarray) -> np.ndarray:
        """c_p[n] = h1 h2 h3 sum_g conj(chi~_p[g]) X[n, g] (trapezoidal rule, Eq. IntApprox)."""
        X = np.atleast_2d(X)
        c = np.zeros((len(self.pidx), X.shape[0]), dtype=self._dtype(X))
        for p, (gi, v) in enumerate(zip(self.pidx, self.pval)):
            c[p] = self.dv * (X[:, gi] @ np.conj(v))
        return c

    def apply_nonlocal(self, X: np.ndarray) -> np.ndarray:
        """V_nl X = sum_p gamma_p chi~_p c_p (Eq. NonlocalPS:FD)."""
        X = np.atleast_2d(X)
        out = np.zeros(X.shape, dtype=self._dtype(X))
        c = self.nonlocal_coeffs(X)
        for p, (gi, v) in enumerate(zip(self.pidx, self.pval)):
            np.add.at(out, (slice(None), gi), self.gamma[p] * np.outer(c[p], v))
        return out

    def apply_local(self, X: np.ndarray) -> np.ndarray:
        """(-1/2 nabla_h^2 + V_eff) X (Eqn. EL with Eq. FD:Laplacian)."""
        X = np.atleast_2d(X)
        if self.is_complex:
            X = X.astype(np.complex128)
        F = X.reshape(X.shape[0], self.n[2], self.n[1], self.n[0])
        lap = laplacian(F, self.n, self.h, self.n_o, self.k).reshape(X.shape)
        return -0.5 * lap + self.veff[None, :] * X

    def apply(self, X: np.ndarray) -> np.ndarray:
        """H X for a block X of shape (Ns, Nd) (or a single vector of shape (Nd,))."""
        single = (np.ndim(X) == 1)
        X2 = np.atleast_2d(X)
        Y = self.apply_local(X2)
        if self.pidx:
            Y = Y + self.apply_nonlocal(X2)
        return Y[0] if single else Y

    def dense(self) -> np.ndarray:
        """The Nd x Nd matrix H(k), column j = H e_j (brute force; tiny grids only)."""
        E = np.eye(self.nd, dtype=np.complex128 if self.is_complex else np.float64)
        return self.apply(E).T


def cheb_T(m: int, x: np.ndarray) -> np.ndarray:
    """Chebyshev polynomial T_m(x) from its closed form (cos/cosh of m times the angle)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    hi = x > 1.0
    out[hi] = np.cosh(m * np.arccosh(x[hi]))
    lo = x < -1.0
    out[lo] = (-1.0) ** m * np.cosh(m * np.arccosh(-x[lo]))
    return out


def cheb_filter_unscaled(H: OracleH, X: np.ndarray, m: int, a: float, b: float) -> np.ndarray:
    """U_f = C_m((H - c)/e) U with e = (b - a)/2, c = (b + a)/2 (Eq. ChebFilter).

    Three-term recurrence Y_0 = X, Y_1 = (H - c) X / e, Y_{j+1} = 2 (H - c) Y_j / e - Y_{j-1}.
    """
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    Y0 = np.atleast_2d(X).astype(np.result_type(X, np.float64))
    Y1 = (H.apply(Y0) - c * Y0) / e
    for _ in range(1, m):
        Y2 = 2.0 * (H.apply(Y1) - c * Y1) / e - Y0
        Y0, Y1 = Y1, Y2
    return Y1


def cheb_filter(H: OracleH, X: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """Scaled filter C_m((H-c)/e) X / C_m((a0-c)/e) (Eq. ChebFilter, normalised at a0).

    sigma_1 = e/(a0 - c), Y_1 = sigma_1 (H - c) X / e,
    sigma_{j+1} = 1/(2/sigma_1 - sigma_j),
    Y_{j+1} = 2 sigma_{j+1} (H - c) Y_j / e - sigma_j sigma_{j+1} Y_{j-1}.
    Follows from C_{j+1}(t) = 2 t C_j(t) - C_{j-1}(t) divided by C_{j+1}(tau0).
    """
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    sigma1 = e / (a0 - c)
    sigma = sigma1
    Y0 = np.atleast_2d(X).astype(np.result_type(X, np.float64))
    Y1 = (sigma1 / e) * (H.apply(Y0) - c * Y0)
    for _ in range(1, m):
        sigma_new = 1.0 / (2.0 / sigma1 - sigma)
        Y2 = (2.0 * sigma_new / e) * (H.apply(Y1) - c * Y1) - (sigma * sigma_new) * Y0
        Y0, Y1 = Y1, Y2
        sigma = sigma_new
    return Y1


def lanczos_bounds(H: OracleH, v0: np.ndarray, ksteps: int = 10):
    """Extremal-eigenvalue estimates of H by k steps of Lanczos (Section 4, 'Lanczos method').

    Full reorthogonalisation (one classical Gram-Schmidt pass).  Returns
    (a0, b) = (min Ritz value, max Ritz value + |beta_k|) and the Ritz values.
    """
    v = np.asarray(v0, dtype=np.complex128 if H.is_complex else np.float64)
    v = v / np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    for j in range(ksteps):
        w = H.apply(V[j])
        a_j = float(np.real(np.vdot(V[j], w)))
        w = w - a_j * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        Vm = np.array(V)
        w = w - Vm.T @ (np.conj(Vm) @ w)
        b_j = float(np.linalg.norm(w))
        alpha.append(a_j)
        beta.append(b_j)
        if j + 1 < ksteps:
            V.append(w / b_j)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    theta = np.linalg.eigvalsh(T)
    return float(theta[0]), float(theta[-1] + abs(beta[-1])), theta


def rayleigh_ritz(H: OracleH, Y: np.ndarray):
    """Projection, orthonormalisation, subspace eigenproblem and rotation (Eqs. 36-39).

    H~ = Y^H H Y, M~ = Y^H Y (Eq. SubspaceGeneralizedEigenproblem); both are
    symmetrised.  The generalised problem H~ y = lambda M~ y is solved through
    the Cholesky factor M~ = L L^H: C = L^{-1} H~ L^{-H}, C q = lambda q,
    y = L^{-H} q.  The rotation is U = Y [y_1 .. y_Ns] (Eq. OrbitalTransformation).
    Returns (lambda ascending, U with shape (Ns, Nd), Hs, Ms).
    """
    Y = np.atleast_2d(Y)
    HY = H.apply(Y)
    Yc = np.conj(Y)
    Hs = Yc @ HY.T          # Hs[i, j] = sum_g conj(Y[i, g]) (HY)[j, g]
    Ms = Yc @ Y.T
    Hs = 0.5 * (Hs + np.conj(Hs.T))
    Ms = 0.5 * (Ms + np.conj(Ms.T))
    L = np.linalg.cholesky(Ms)
    Linv_H = scipy.linalg.solve_triangular(L, Hs, lower=True)
    C = scipy.linalg.solve_triangular(L, np.conj(Linv_H.T), lower=True)
    C = 0.5 * (C + np.conj(C.T))
    lam, Q = np.linalg.eigh(C)
    Yrot = scipy.linalg.solve_triangular(np.conj(L.T), Q, lower=False)
    U = (Y.T @ Yrot).T
    return lam, U, Hs, Ms


def chefsi_step(H: OracleH, X: np.ndarray, m: int, a: float, b: float, a0: float):
    """One CheFSI pass: scaled filter, then Rayleigh-Ritz (Section 3.4)."""
    Yf = cheb_filter(H, X, m, a, b, a0)
    lam, U, _, _ = rayleigh_ritz(H, Yf)
    return lam, U
