"""Learned initial density (project-added; the paper starts each SCF from the
superposition of atomic densities): converged SCF densities of seeded cells become
(descriptor, density correction) pairs, the 16-128-128-1 network of the library is
trained on them with its own kernels, and its prediction seeds new SCF runs through
sparc_scf_set_density.

The network predicts t = (rho_converged - rho_atoms) / scale per grid node, where
rho_atoms = -b is the superposition of the Gaussian atoms' densities and `scale`
the standard deviation of that difference over the training set.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import sparc, synth

NFEAT = sparc.MLP_NFEAT


def widths():
    """Descriptor widths s_k = 0.4 * 10^(k/15) bohr, k = 0..15."""
    return 0.4 * 10.0 ** (np.arange(NFEAT) / (NFEAT - 1))


def init_params(seed):
    """Glorot-uniform weights and zero biases from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    nf, nh = NFEAT, sparc.MLP_NHID
    th = np.zeros(sparc.MLP_NPARAM)
    o = 0
    for shape, fan in (((nf, nh), nf + nh), ((nh,), 0), ((nh, nh), 2 * nh), ((nh,), 0), ((nh,), nh + 1), ((1,), 0)):
        sz = int(np.prod(shape))
        if fan:
            th[o:o + sz] = rng.uniform(-1, 1, sz) * np.sqrt(6.0 / fan)
        o += sz
    return th.astype(np.float32)


@dataclass
class ScfRun:
    iters: int
    seconds: float
    free_energy: float
    vresid: float
    rho: object          # CUDA float64 tensor, Nd
    b: object            # CUDA float64 tensor, Nd
    residuals: list      # V residual of every iteration

    def iterations_to(self, tol):
        """First iteration (1-based) whose V residual is below tol, or None."""
        for i, r in enumerate(self.residuals):
            if r < tol:
                return i + 1
        return None


def converge(ctx, sysd, dtype, tol=1e-6, max_iter=80, first_passes=4, dy=None, scale=0.0, kT=0.01):
    """Run sparc_scf_step until the V_eff residual is below tol (mixed path for FP32)."""
    import torch
    wl = sysd.wl
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    S = sparc.Scf.from_system(H, sysd, kT=kT, poisson_tol=1e-10, first_passes=first_passes)
    U = torch.from_numpy(sysd.U0.copy()).to(dtype).cuda()
    eig = torch.zeros(wl.ns, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if dy is not None:
        S.set_density(dy, scale)
    info = None
    it = 0
    res = []
    for it in range(1, max_iter + 1):
        info = sparc.sparc_scf_step(S, U, eig, wl.m)
        res.append(info["vresid"])
        if info["vresid"] < tol:
            break
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    rho = torch.empty(wl.nd, dtype=torch.float64, device="cuda")
    b = torch.empty_like(rho)
    S.read("rho", rho)
    S.read("b", b)
    torch.cuda.synchronize()
    S.close()
    H.close()
    return ScfRun(it, sec, info["free_energy"], info["vresid"], rho, b, res)


def descriptors(ctx, sysd):
    import torch
    wl = sysd.wl
    D = torch.empty((wl.nd, NFEAT), dtype=torch.float32, device="cuda")
    sparc.sparc_mlp_descriptors(ctx, wl.n, wl.h, wl.atoms, widths(), D)
    return D


def dataset(ctx, seeds, dtype, tol=1e-6):
    """Descriptors and density corrections rho - rho_atoms of the converged cells."""
    import torch
    Ds, Ts, runs = [], [], []
    for s in seeds:
        sysd = synth.scf_fcc32(seed=int(s))
        run = converge(ctx, sysd, dtype, tol=tol)
        Ds.append(descriptors(ctx, sysd))
        Ts.append((run.rho + run.b).to(torch.float32))   # rho - (-b)
        runs.append(run)
    return torch.cat(Ds), torch.cat(Ts), runs


def train(ctx, D, T, epochs=40, batch=8192, lr=1e-3, seed=0):
    """Adam on the standardised targets; returns (network, scale, loss before training
    and after each epoch)."""
    import torch
    scale = float(T.double().std().item())
    t = (T / scale).contiguous()
    net = sparc.Mlp(ctx, init_params(seed))
    rng = np.random.default_rng(seed + 1)
    n = D.shape[0]
    g = torch.empty(sparc.MLP_NPARAM, dtype=torch.float32, device="cuda")
    hist = [net.grad(D, t, g)]        # loss of the initial parameters, then after each epoch
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n).astype(np.int64)).cuda()
        for q in range(0, n, batch):
            net.train_step(D, t, lr, idx=perm[q:q + batch])
        hist.append(net.grad(D, t, g))
    return net, scale, hist


def predict(ctx, net, sysd):
    """Network output (the standardised correction) on the cell's grid."""
    import torch
    D = descriptors(ctx, sysd)
    y = torch.empty(D.shape[0], dtype=torch.float32, device="cuda")
    net.forward(D, y)
    return y
