"""Seeded synthetic inputs for the CheFSI hot path.

This module only draws inputs: the grid, the effective potential V_eff, atom
sites, Kleinman-Bylander projector boxes and start orbitals.  It holds none of
the arithmetic of the method (no stencil, no filter, no projection), so both the
CUDA path and the CPU oracle can consume what it produces without sharing any
of the computation.

Conventions (Section 3.1 of the paper, "Finite-difference discretization"):
  * the cell is a cuboid with its origin at the centre; node i (0-based) on axis
    s sits at x_i = -L_s/2 + i*h_s, L_s = n_s*h_s;
  * grid index g = i + n1*(j + n2*k) (x fastest);
  * orbitals are stored as arrays of shape (Ns, Nd), i.e. column-major
    Nd x Ns matrices with leading dimension Nd.

Projectors stand in for the Troullier-Martins tables the paper interpolates
(Eq. NonlocalPS:FD and Section 3.4): chi_lm(r) = N * r^l Y_lm(r) exp(-|r|^2/rc^2)
for l=0 (s) and l=1 (p_x, p_y, p_z), on a cube of (2*n_c+1)^3 nodes centred on
the node nearest to the atom, n_c = ceil(3*rc/h), normalised so that
h1*h2*h3 * sum_box chi^2 = 1 (then gamma is an energy in Ha).  Box corners are
given in unwrapped node coordinates and may lie outside [0, n); a node q of the
box maps to grid node q mod n of the periodic image shifted by floor(q/n)*L.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "Projectors", "make_projectors", "gaussian_veff", "fcc_sites",
    "diamond_sites", "monkhorst_pack", "config1", "config2", "config3",
    "small_case", "random_orbitals", "lanczos_start", "ScfSystem", "scf_small", "scf_fcc32", "scf_pair",
]


@dataclass
class Projectors:
    """Packed Kleinman-Bylander projector boxes (one entry per (atom, l, m))."""
    box_lo: np.ndarray      # (nproj, 3) int32, unwrapped first node per axis
    box_n: np.ndarray       # (nproj, 3) int32, nodes per axis
    chi_off: np.ndarray     # (nproj,) int64, offset of the box values in chi
    chi: np.ndarray         # packed real box values, x fastest inside a box
    gamma: np.ndarray       # (nproj,) float64, KB energies gamma_Jl (Ha)
    atom: np.ndarray        # (nproj,) int32, owning atom
    l: np.ndarray           # (nproj,) int32, angular momentum

    @property
    def nproj(self) -> int:
        return int(self.gamma.shape[0])

    @staticmethod
    def empty() -> "Projectors":
        return Projectors(np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32),
                          np.zeros(0, np.int64), np.zeros(0, np.float64),
                          np.zeros(0, np.float64), np.zeros(0, np.int32),
                          np.zeros(0, np.int32))


@dataclass
class Workload:
    name: str
    n: tuple            # (n1, n2, n3)
    h: tuple            # (h1, h2, h3) bohr
    fd_radius: int      # n_o
    kpts: np.ndarray    # (Nk, 3) Cartesian Bloch vectors, bohr^-1
    kw: np.ndarray      # (Nk,) Brillouin-zone weights
    veff: np.ndarray    # (Nd,) float64, Ha
    atoms: np.ndarray   # (natom, 3) bohr
    proj: Projectors
    ns: int
    m: int
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def nd(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def L(self) -> tuple:
        return tuple(self.n[s] * self.h[s] for s in range(3))

    @property
    def complex(self) -> bool:
        return bool(np.any(self.kpts != 0.0))


def node_coords(n, h):
    """Node coordinates per axis, origin at the cell centre."""
    return [(-0.5 * n[s] * h[s]) + h[s] * np.arange(n[s], dtype=np.float64) for s in range(3)]


def gaussian_veff(n, h, sites, depth, width, noise=0.0, rng=None):
    """V_eff(x) = sum_sites sum_{27 images} d * exp(-|x - R - T|^2 / w^2) (+ N(0, noise))."""
    xs = node_coords(n, h)
    L = np.array([n[s] * h[s] for s in range(3)])
    v = np.zeros((n[2], n[1], n[0]), dtype=np.float64)
    for R, d, w in zip(sites, depth, width):
        # the Gaussian and the 3x3x3 image set are both products over axes
        g = [sum(np.exp(-((xs[s] - R[s] - t * L[s]) ** 2) / (w * w)) for t in (-1, 0, 1)) for s in range(3)]
        v += d * (g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :])
    v = v.reshape(-1)
    if noise > 0.0:
        v = v + rng.normal(0.0, noise, size=v.shape)
    return v


def make_projectors(n, h, atoms, rc, gamma_s, gamma_p, with_p=True):
    """s (+p) Gaussian projectors on cubic boxes of half-width n_c = ceil(3 rc / h)."""
    L = [n[s] * h[s] for s in range(3)]
    box_lo, box_n, chi_off, chis, gam, atom, ll = [], [], [], [], [], [], []
    off = 0
    for J, R in enumerate(atoms):
        lo, nb, axes = [], [], []
        for s in range(3):
            nc = int(math.ceil(3.0 * rc / h[s]))
            qc = int(round((R[s] + 0.5 * L[s]) / h[s]))
            lo.append(qc - nc)
            nb.append(2 * nc + 1)
            if 2 * nc + 1 > n[s]:
                raise ValueError("projector box wider than the cell")
            q = np.arange(qc - nc, qc + nc + 1, dtype=np.float64)
            axes.append(-0.5 * L[s] + q * h[s] - R[s])
        rz, ry, rx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        g = np.exp(-(rx * rx + ry * ry + rz * rz) / (rc * rc))
        shapes = [(0, g)]
        if with_p:
            shapes += [(1, rx * g), (1, ry * g), (1, rz * g)]
        dv = h[0] * h[1] * h[2]
        for l, f in shapes:
            f = f / math.sqrt(dv * float(np.sum(f * f)))
            box_lo.append(lo)
            box_n.append(nb)
            chi_off.append(off)
            flat = f.reshape(-1)
            chis.append(flat)
            off += flat.size
            gam.append(gamma_s[J] if l == 0 else gamma_p[J])
            atom.append(J)
            ll.append(l)
    if not chis:
        return Projectors.empty()
    return Projectors(np.asarray(box_lo, np.int32), np.asarray(box_n, np.int32),
                      np.asarray(chi_off, np.int64), np.concatenate(chis),
                      np.asarray(gam, np.float64), np.asarray(atom, np.int32),
                      np.asarray(ll, np.int32))


def fcc_sites(cells, a, rng, sigma):
    """FCC conventional cells (4 sites each) tiling cells=(cx,cy,cz) with edges a=(ax,ay,az)."""
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = []
    for k in range(cells[2]):
        for j in range(cells[1]):
            for i in range(cells[0]):
                for b in basis:
                    pts.append((np.array([i, j, k]) + b) * np.asarray(a))
    pts = np.asarray(pts, dtype=np.float64)
    L = np.asarray(cells) * np.asarray(a)
    pts = pts - 0.5 * L + 0.25 * np.asarray(a) / 2.0
    if sigma > 0:
        pts = pts + rng.normal(0.0, sigma, size=pts.shape)
    return pts


def diamond_sites(cells, a):
    """Diamond lattice (8 sites per conventional cell), cell origin at the centre."""
    fcc = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    basis = np.concatenate([fcc, fcc + 0.25])
    pts = []
    for k in range(cells[2]):
        for j in range(cells[1]):
            for i in range(cells[0]):
                for b in basis:
                    pts.append((np.array([i, j, k]) + b) * a)
    pts = np.asarray(pts, dtype=np.float64)
    return pts - 0.5 * np.asarray(cells) * a + 0.01 * a


def monkhorst_pack(mesh, L):
    """Unshifted MP nodes kappa in (-1/2, 1/2], Cartesian k = 2*pi*kappa/L, equal weights."""
    ks = []
    for c in range(mesh[2]):
        for b in range(mesh[1]):
            for a_ in range(mesh[0]):
                kap = []
                for s, (idx, q) in enumerate(zip((a_, b, c), mesh)):
                    kap.append((2 * idx - q + 1) / (2.0 * q))
                ks.append([2.0 * math.pi * kap[s] / L[s] for s in range(3)])
    ks = np.asarray(ks, dtype=np.float64)
    return ks, np.full(len(ks), 1.0 / len(ks))


def random_orbitals(nd, ns, seed, complex_=False):
    """Seeded N(0,1) start block, shape (Ns, Nd)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((ns, nd))
    if complex_:
        x = x + 1j * rng.standard_normal((ns, nd))
    return x


def lanczos_start(nd, seed, complex_=False):
    """Seeded N(0,1) Lanczos start vector (not normalised: the method normalises it)."""
    return random_orbitals(nd, 1, seed + 7919, complex_)[0]


def _atoms_veff(n, h, atoms, rng, noise):
    d = rng.uniform(-2.0, 0.0, size=len(atoms))
    w = rng.uniform(0.8, 1.5, size=len(atoms))
    return gaussian_veff(n, h, atoms, d, w, noise=noise, rng=rng)


def config1(seed=1001) -> Workload:
    """24^3, h=0.5, 8 Gaussian wells on random sites, 8 s+p atoms, Ns=32, m=20, Gamma, FP64."""
    rng = np.random.default_rng(seed)
    n, h = (24, 24, 24), (0.5, 0.5, 0.5)
    L = np.array([12.0, 12.0, 12.0])
    sites = rng.uniform(-0.5, 0.5, size=(8, 3)) * L
    d = rng.uniform(-2.0, 0.0, size=8)
    w = rng.uniform(0.8, 1.5, size=8)
    veff = gaussian_veff(n, h, sites, d, w)
    atoms = rng.uniform(-0.5, 0.5, size=(8, 3)) * L
    proj = make_projectors(n, h, atoms, 1.2, rng.uniform(-1, 1, 8), rng.uniform(-1, 1, 8))
    return Workload("config1_24^3_ns32_m20_f64", n, h, 6, np.zeros((1, 3)), np.ones(1), veff,
                    atoms, proj, 32, 20, seed)


def config2(seed=1002) -> Workload:
    """64^3, h=0.4, 128 perturbed-FCC s+p atoms, V_eff atom Gaussians + N(0,0.01), Ns=512, m=24."""
    rng = np.random.default_rng(seed)
    n, h = (64, 64, 64), (0.4, 0.4, 0.4)
    atoms = fcc_sites((4, 4, 2), (6.4, 6.4, 12.8), rng, 0.05)
    veff = _atoms_veff(n, h, atoms, rng, 0.01)
    proj = make_projectors(n, h, atoms, 1.2, rng.uniform(-1, 1, len(atoms)),
                           rng.uniform(-1, 1, len(atoms)))
    return Workload("config2_64^3_128atoms_ns512_m24", n, h, 6, np.zeros((1, 3)), np.ones(1),
                    veff, atoms, proj, 512, 24, seed)


def config3(seed=1003) -> Workload:
    """40^3 Si-like 2x2x2 diamond cell (64 s+p atoms), 3x3x3 MP k-mesh, Ns=192, m=20, complex."""
    rng = np.random.default_rng(seed)
    n = (40, 40, 40)
    a = 10.68
    L = 2 * a
    h = (L / 40, L / 40, L / 40)
    atoms = diamond_sites((2, 2, 2), a)
    veff = _atoms_veff(n, h, atoms, rng, 0.01)
    proj = make_projectors(n, h, atoms, 1.2, rng.uniform(-1, 1, len(atoms)),
                           rng.uniform(-1, 1, len(atoms)))
    kpts, kw = monkhorst_pack((3, 3, 3), (L, L, L))
    return Workload("config3_40^3_64atoms_27k_ns192_m20", n, h, 6, kpts, kw, veff, atoms, proj,
                    192, 20, seed)


CELL_GRIDS = (("cube24", (24, 24, 24)), ("cube32", (32, 32, 32)), ("slab40x40x64", (40, 40, 64)),
              ("wire24x24x96", (24, 24, 96)), ("cube48", (48, 48, 48)))


def config4(seed=1004, ncell=16, h=0.45) -> list:
    """Uneven batch of independent Gamma-point cells for the filter graph.

    Per cell, drawn from the seed: the grid from {24^3, 32^3, 40x40x64 slab, 24x24x96
    wire, 48^3} at h = 0.45 bohr; 8..96 s+p atoms, at most one per 60 bohr^3 of the
    occupied region (slab: the middle half in z; wire: the middle half of each
    cross-section axis; cubes: everything), uniform there; V_eff = atom Gaussians
    (depth U[-2,0], width U[0.8,1.5]) + N(0, 0.01); projector width 1.0 bohr,
    energies U[-1,1]; Ns = 4 x atoms x U[0.8,1.2] clipped to [48, 384]; m from
    {16, 20, 24}."""
    rng = np.random.default_rng(seed)
    cells = []
    for c in range(ncell):
        kind, n = CELL_GRIDS[int(rng.integers(len(CELL_GRIDS)))]
        hh = (h, h, h)
        L = np.array([n[s] * h for s in range(3)])
        occ = np.ones(3)
        if kind.startswith("slab"):
            occ[2] = 0.5
        elif kind.startswith("wire"):
            occ[0] = occ[1] = 0.5
        vol = float(np.prod(L * occ))
        natom = int(rng.integers(8, max(9, min(96, int(vol / 60.0)) + 1)))
        atoms = (rng.uniform(-0.5, 0.5, size=(natom, 3)) * occ) * L
        veff = _atoms_veff(n, hh, atoms, rng, 0.01)
        proj = make_projectors(n, hh, atoms, 1.0, rng.uniform(-1, 1, natom), rng.uniform(-1, 1, natom))
        ns = int(np.clip(round(4 * natom * rng.uniform(0.8, 1.2)), 48, 384))
        m = int(rng.choice([16, 20, 24]))
        cells.append(Workload(f"cell{c:02d}_{kind}_{natom}atoms_ns{ns}_m{m}", tuple(n), hh, 6, np.zeros((1, 3)),
                              np.ones(1), veff, atoms, proj, ns, m, seed * 100 + c))
    return cells


def small_case(n=(14, 12, 13), h=(0.55, 0.6, 0.5), fd_radius=6, natom=2, k=(0.0, 0.0, 0.0),
               ns=8, m=6, seed=7, rc=0.9, veff_scale=1.0, with_p=True) -> Workload:
    """Tiny anisotropic cell for brute-force checks (dense H fits in memory)."""
    rng = np.random.default_rng(seed)
    L = np.array([n[s] * h[s] for s in range(3)])
    sites = rng.uniform(-0.5, 0.5, size=(3, 3)) * L
    veff = veff_scale * gaussian_veff(n, h, sites, rng.uniform(-2, 0, 3), rng.uniform(0.8, 1.5, 3))
    atoms = rng.uniform(-0.5, 0.5, size=(natom, 3)) * L
    proj = make_projectors(n, h, atoms, rc, rng.uniform(-1, 1, natom), rng.uniform(-1, 1, natom),
                           with_p=with_p) if natom else Projectors.empty()
    return Workload(f"small_{n[0]}x{n[1]}x{n[2]}", tuple(n), tuple(h), fd_radius,
                    np.asarray([k], np.float64), np.ones(1), veff, atoms, proj, ns, m, seed)


@dataclass
class ScfSystem:
    """Inputs of an SCF run: the workload (grid, projectors; its veff is unused, the SCF
    sets V_eff), valence charges Z and widths rc of the local pseudopotentials
    -Z erf(r/rc)/r, the Lanczos start vector and the start orbitals."""
    wl: Workload
    Z: np.ndarray
    rc: np.ndarray
    v0: np.ndarray
    U0: np.ndarray

    @property
    def nelec(self) -> float:
        return float(np.sum(self.Z))


def scf_small(n=(20, 20, 20), h=(0.5, 0.5, 0.5), natom=4, ns=12, m=12, seed=41, Z=1.0, rc_loc=0.7,
              rc_proj=0.9, gamma=0.3) -> ScfSystem:
    """A small cell for SCF parity against the oracle: atoms at random sites at least
    3.5 bohr apart (periodic images included), s+p projectors with energies U[-gamma, gamma]."""
    rng = np.random.default_rng(seed)
    L = np.array([n[s] * h[s] for s in range(3)])
    atoms = []
    while len(atoms) < natom:
        x = rng.uniform(-0.5, 0.5, 3) * L
        ok = True
        for y in atoms:
            d = x - y
            d -= L * np.round(d / L)
            ok = ok and float(np.linalg.norm(d)) > 3.5
        if ok:
            atoms.append(x)
    atoms = np.array(atoms)
    proj = make_projectors(n, h, atoms, rc_proj, rng.uniform(-gamma, gamma, natom),
                           rng.uniform(-gamma, gamma, natom))
    nd = n[0] * n[1] * n[2]
    wl = Workload(f"scf_{n[0]}x{n[1]}x{n[2]}", tuple(n), tuple(h), 6, np.zeros((1, 3)), np.ones(1),
                  np.zeros(nd), atoms, proj, ns, m, seed)
    return ScfSystem(wl, np.full(natom, float(Z)), np.full(natom, float(rc_loc)), lanczos_start(nd, seed + 1),
                     random_orbitals(nd, ns, seed + 2))


def scf_fcc32(seed=1005, a=8.1, h=0.45, sigma=0.05, Z=3.0, rc_loc=0.8, rc_proj=1.2, ns=72, m=20) -> ScfSystem:
    """32 atoms on 2x2x2 perturbed FCC cells (a = 8.1 bohr, 36^3 grid at h = 0.45),
    Z = 3 (N_e = 96), local pseudopotential width 0.8 bohr, s+p projectors with
    energies U[-0.5, 0.5] Ha, m = 20 (the SCF cell of the learned-density study).
    Ns = 72 = 1.5 N_e/2: with 1.2 N_e/2 = 58 states the highest one of this metallic
    cell lies 0.03 Ha above the Fermi level at k_B T = 0.01 Ha, keeps occupation 4e-2
    and, converging slowest in the filter, stalls the SCF near residual 1e-4."""
    rng = np.random.default_rng(seed)
    n = int(round(2 * a / h))
    sites = fcc_sites((2, 2, 2), a, rng, sigma)
    hh = (2 * a / n,) * 3
    proj = make_projectors((n, n, n), hh, sites, rc_proj, rng.uniform(-0.5, 0.5, len(sites)),
                           rng.uniform(-0.5, 0.5, len(sites)))
    nd = n ** 3
    wl = Workload("fcc32_scf", (n, n, n), hh, 6, np.zeros((1, 3)), np.ones(1), np.zeros(nd), sites, proj, ns, m,
                  seed)
    return ScfSystem(wl, np.full(len(sites), Z), np.full(len(sites), rc_loc), lanczos_start(nd, seed + 1),
                     random_orbitals(nd, ns, seed + 2))


def scf_pair(R=None, n=(18, 18, 18), h=(0.5, 0.5, 0.5)) -> ScfSystem:
    """Two atoms (Z = 1, local width 0.7 bohr, s+p projectors of width 0.9 bohr) in an
    18^3 cell, 8 orbitals, m = 12: the force checks."""
    if R is None:
        R = np.array([[-1.13, 0.37, 0.21], [1.41, -0.29, -0.52]])
    R = np.asarray(R, dtype=np.float64)
    proj = make_projectors(n, h, R, 0.9, np.array([0.25, -0.2]), np.array([0.15, 0.3]))
    nd = n[0] * n[1] * n[2]
    wl = Workload("pair_18", tuple(n), tuple(h), 6, np.zeros((1, 3)), np.ones(1), np.zeros(nd), R, proj, 8, 12, 5)
    return ScfSystem(wl, np.array([1.0, 1.0]), np.array([0.7, 0.7]), lanczos_start(nd, 6), random_orbitals(nd, 8, 5))
