"""Thin ctypes binding of libsparc.so (include/sparc.h).

Argument marshalling only: every step of the CheFSI path runs in the CUDA
library.  Device buffers are passed as torch tensors (or raw device pointers),
streams as torch.cuda.Stream (or raw handles).  Loading fails loudly when the
library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libsparc.so")

F64, F32, C128, C64 = 0, 1, 2, 3
TUNE_SHAPE = 1 << 20   # launch configuration code = blocks per launch + TUNE_SHAPE * tile shape
RR_FP64, RR_MIXED = 0, 1
STATUS = {0: "SPARC_OK", 1: "SPARC_ERR_INVALID_ARG", 2: "SPARC_ERR_OOM", 3: "SPARC_ERR_CUDA",
          4: "SPARC_ERR_NOT_POSDEF", 5: "SPARC_ERR_NO_CONVERGENCE", 6: "SPARC_ERR_TIMEOUT"}

EXPORTS = ["sparc_create", "sparc_destroy", "sparc_last_error", "sparc_sync", "sparc_ham_create",
           "sparc_ham_set_veff", "sparc_ham_destroy", "sparc_apply_H", "sparc_cheb_filter",
           "sparc_lanczos_bounds", "sparc_rayleigh_ritz", "sparc_timing_enable", "sparc_timing_read",
           "sparc_launch_count", "sparc_graph_launch_count", "sparc_apply_H_noalloc", "sparc_last_sweeps", "sparc_last_ortho_err", "sparc_gram_f32",
           "sparc_rotate_f32", "sparc_scf_create", "sparc_scf_step", "sparc_scf_read", "sparc_scf_destroy",
           "sparc_scf_forces", "sparc_cheb_filter_batch", "sparc_autotune_filter",
           "sparc_set_filter_units", "sparc_filter_graph_create", "sparc_filter_graph_set_bounds",
           "sparc_filter_graph_launch", "sparc_filter_graph_destroy", "sparc_scf_set_density",
           "sparc_mlp_create", "sparc_mlp_params", "sparc_mlp_descriptors", "sparc_mlp_forward", "sparc_mlp_grad",
           "sparc_mlp_train_step", "sparc_mlp_destroy", "sparc_scf_create_k", "sparc_debug_inject",
           "sparc_filter_kernel", "sparc_gram_c64", "sparc_rotate_c64"]
KERNEL_GENERIC, KERNEL_TILED, KERNEL_TMA = 0, 1, 2
TIMED = {"hpass": 0, "gather": 1, "gram": 2, "eig": 3, "rotation": 4, "jacobi": 5, "fpass": 6,
         "ortho": 7, "series": 8, "ritz": 9}


class SparcGrid(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("h", c_double * 3), ("fd_radius", c_int), ("k", c_double * 3)]


class SparcNonlocal(ctypes.Structure):
    _fields_ = [("nproj", c_int), ("box_lo", POINTER(c_int32)), ("box_n", POINTER(c_int32)),
                ("chi_off", POINTER(c_int64)), ("chi", POINTER(c_double)), ("chi_len", c_int64),
                ("gamma", POINTER(c_double))]


class SparcScfDesc(ctypes.Structure):
    _fields_ = [("natom", c_int), ("R", POINTER(c_double)), ("Z", POINTER(c_double)), ("rc", POINTER(c_double)),
                ("kT", c_double), ("mix_beta", c_double), ("mix_history", c_int), ("poisson_tol", c_double),
                ("v0", POINTER(c_double)), ("proj_atom", POINTER(c_int32)), ("first_passes", c_int)]


class SparcScfInfo(ctypes.Structure):
    _fields_ = [("free_energy", c_double), ("fermi", c_double), ("vresid", c_double), ("nelec", c_double),
                ("e_band", c_double), ("e_xc", c_double), ("e_el", c_double), ("e_self", c_double),
                ("e_entropy", c_double), ("poisson_iters", c_int), ("a0", c_double), ("a", c_double),
                ("b", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SparcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libsparc.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsparc.so not found at {path}; build it with "
                           "paper_1603_04339_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.sparc_create.argtypes = [POINTER(c_void_p), c_int]
    L.sparc_destroy.argtypes = [c_void_p]
    L.sparc_destroy.restype = None
    L.sparc_last_error.argtypes = [c_void_p]
    L.sparc_last_error.restype = ctypes.c_char_p
    L.sparc_sync.argtypes = [c_void_p, c_void_p]
    L.sparc_ham_create.argtypes = [c_void_p, POINTER(SparcGrid), POINTER(c_double),
                                   POINTER(SparcNonlocal), POINTER(c_void_p)]
    L.sparc_ham_set_veff.argtypes = [c_void_p, c_void_p, c_int, c_void_p]
    L.sparc_ham_destroy.argtypes = [c_void_p]
    L.sparc_ham_destroy.restype = None
    L.sparc_apply_H.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int64, c_void_p]
    L.sparc_cheb_filter.argtypes = [c_void_p, c_int, c_int, c_double, c_double, c_double, c_void_p,
                                    c_void_p, c_int, c_int64, c_void_p]
    L.sparc_lanczos_bounds.argtypes = [c_void_p, c_int, c_void_p, POINTER(c_double),
                                       POINTER(c_double), c_void_p]
    L.sparc_rayleigh_ritz.argtypes = [c_void_p, c_int, c_void_p, c_int, c_int64, c_void_p, c_int,
                                      c_void_p]
    L.sparc_timing_enable.argtypes = [c_void_p, c_int]
    L.sparc_launch_count.argtypes = [c_void_p, POINTER(c_int64)]
    L.sparc_last_sweeps.argtypes = [c_void_p, POINTER(c_int)]
    L.sparc_last_sweeps.restype = c_int
    L.sparc_last_ortho_err.argtypes = [c_void_p, POINTER(ctypes.c_double)]
    L.sparc_last_ortho_err.restype = c_int
    L.sparc_graph_launch_count.argtypes = [c_void_p, POINTER(c_int64)]
    L.sparc_graph_launch_count.restype = c_int
    L.sparc_debug_inject.argtypes = [c_void_p, c_int, c_int64]
    L.sparc_debug_inject.restype = c_int
    L.sparc_apply_H_noalloc.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int64, c_void_p]
    L.sparc_apply_H_noalloc.restype = c_int
    L.sparc_launch_count.restype = c_int
    L.sparc_timing_read.argtypes = [c_void_p, c_int, POINTER(c_double), POINTER(c_int64)]
    L.sparc_gram_f32.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int64, c_int, c_void_p,
                                 c_void_p]
    L.sparc_rotate_f32.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int, c_void_p, c_int64,
                                   c_void_p]
    L.sparc_gram_c64.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int64, c_int, c_void_p,
                                 c_void_p]
    L.sparc_rotate_c64.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int, c_void_p, c_int64,
                                   c_void_p]
    L.sparc_scf_create.argtypes = [c_void_p, POINTER(SparcScfDesc), POINTER(c_void_p)]
    L.sparc_scf_create_k.argtypes = [POINTER(c_void_p), c_int, POINTER(c_double), POINTER(SparcScfDesc),
                                     POINTER(c_void_p)]
    L.sparc_scf_step.argtypes = [c_void_p, c_int, c_int, c_void_p, c_int, c_int64, c_void_p,
                                 POINTER(SparcScfInfo), c_void_p]
    L.sparc_scf_read.argtypes = [c_void_p, c_int, c_void_p, c_void_p]
    L.sparc_scf_forces.argtypes = [c_void_p, c_int, c_void_p, c_int, c_int64, POINTER(c_double), c_void_p]
    L.sparc_filter_kernel.argtypes = [c_void_p, c_int, POINTER(c_int)]
    L.sparc_filter_kernel.restype = c_int
    L.sparc_cheb_filter_batch.argtypes = [POINTER(c_void_p), c_int, c_int, c_int, POINTER(c_double),
                                          POINTER(c_double), POINTER(c_double), c_void_p, c_void_p, c_int,
                                          c_int64, c_void_p]
    L.sparc_autotune_filter.argtypes = [POINTER(c_void_p), c_int, c_int, c_int, POINTER(c_double),
                                        POINTER(c_double), POINTER(c_double), c_void_p, c_void_p, c_int,
                                        c_int64, c_void_p, POINTER(c_int), POINTER(c_double)]
    L.sparc_set_filter_units.argtypes = [c_void_p, c_int, c_int64, c_int, c_int, c_int]
    L.sparc_filter_graph_create.argtypes = [POINTER(c_void_p), c_int, c_int, POINTER(c_int), POINTER(c_double),
                                            POINTER(c_double), POINTER(c_double), POINTER(c_void_p),
                                            POINTER(c_void_p), POINTER(c_int), POINTER(c_int64), c_int,
                                            POINTER(c_void_p)]
    L.sparc_filter_graph_set_bounds.argtypes = [c_void_p, POINTER(c_double), POINTER(c_double),
                                                POINTER(c_double)]
    L.sparc_filter_graph_launch.argtypes = [c_void_p, c_void_p]
    L.sparc_filter_graph_destroy.argtypes = [c_void_p]
    L.sparc_filter_graph_destroy.restype = None
    L.sparc_scf_set_density.argtypes = [c_void_p, c_void_p, c_double, c_void_p]
    L.sparc_mlp_create.argtypes = [c_void_p, c_void_p, POINTER(c_void_p)]
    L.sparc_mlp_params.argtypes = [c_void_p, c_void_p, c_int]
    L.sparc_mlp_descriptors.argtypes = [c_void_p, POINTER(c_int), POINTER(c_double), c_int, c_void_p, c_void_p,
                                        c_void_p, c_void_p]
    L.sparc_mlp_forward.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]
    L.sparc_mlp_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p,
                                 POINTER(c_double), c_void_p]
    L.sparc_mlp_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int64, ctypes.c_float,
                                       POINTER(c_double), c_void_p]
    L.sparc_mlp_destroy.argtypes = [c_void_p]
    L.sparc_mlp_destroy.restype = None
    L.sparc_scf_destroy.argtypes = [c_void_p]
    L.sparc_scf_destroy.restype = None
    for name in ("sparc_timing_enable", "sparc_timing_read", "sparc_create", "sparc_sync", "sparc_ham_create", "sparc_ham_set_veff",
                 "sparc_apply_H", "sparc_cheb_filter", "sparc_lanczos_bounds", "sparc_rayleigh_ritz",
                 "sparc_gram_f32", "sparc_rotate_f32", "sparc_gram_c64", "sparc_rotate_c64", "sparc_scf_create", "sparc_scf_step", "sparc_scf_read",
                 "sparc_scf_forces"):
        getattr(L, name).restype = c_int
    _lib = L
    return L


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def dtype_code(t) -> int:
    import torch
    return {torch.float64: F64, torch.float32: F32, torch.complex128: C128,
            torch.complex64: C64}[t.dtype]


class Context:
    """A libsparc context on one CUDA device (workspace + device status word)."""

    def __init__(self, device: int = 0):
        L = load()
        h = c_void_p()
        rc = L.sparc_create(ctypes.byref(h), int(device))
        if rc != 0:
            raise SparcError(rc, "sparc_create failed")
        self.handle = h
        self.device = device
        self._hams = weakref.WeakSet()   # Hamiltonians of this context, closed with it
        self._scfs = weakref.WeakSet()   # SCF states, closed before the Hamiltonians
        self._graphs = weakref.WeakSet()  # filter graphs, closed before the Hamiltonians

    def error(self) -> str:
        return load().sparc_last_error(self.handle).decode()

    def check(self, rc):
        if rc != 0:
            raise SparcError(rc, self.error())

    def sync(self, stream=None):
        self.check(load().sparc_sync(self.handle, _stream(stream)))

    def timing(self, on: bool):
        """Bracket the timed kernel classes with CUDA events (sparc_timing_enable)."""
        self.check(load().sparc_timing_enable(self.handle, 1 if on else 0))

    def timing_read(self, which: str):
        """(total ms, launches) of a timed kernel class since timing was enabled."""
        ms, n = c_double(), c_int64()
        self.check(load().sparc_timing_read(self.handle, TIMED[which], ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def last_sweeps(self) -> int:
        """Jacobi sweeps of the last Rayleigh-Ritz call (sparc_last_sweeps)."""
        n = c_int()
        self.check(load().sparc_last_sweeps(self.handle, ctypes.byref(n)))
        return n.value

    def graph_launches(self) -> int:
        """CUDA graph launches of this context (sparc_graph_launch_count)."""
        n = c_int64()
        self.check(load().sparc_graph_launch_count(self.handle, ctypes.byref(n)))
        return n.value

    def last_ortho_err(self) -> float:
        """max |U1^T U1 - I| of the last mixed FP32 Rayleigh-Ritz (sparc_last_ortho_err)."""
        e = ctypes.c_double(0.0)
        self.check(load().sparc_last_ortho_err(self.handle, ctypes.byref(e)))
        return e.value

    def inject(self, what: str, value: int):
        """Failure injection for tests of the error paths (sparc_debug_inject):
        what = 'alloc_fail' | 'wait_limit' | 'stall' | 'cg_max_iters' | 'fp64_ortho'."""
        code = {"alloc_fail": 1, "wait_limit": 2, "stall": 3, "cg_max_iters": 4, "fp64_ortho": 5}[what]
        self.check(load().sparc_debug_inject(self.handle, code, int(value)))

    def launches(self) -> int:
        """Kernels launched by this context so far (sparc_launch_count)."""
        n = c_int64()
        self.check(load().sparc_launch_count(self.handle, ctypes.byref(n)))
        return n.value

    def close(self):
        if self.handle:
            for Gr in list(self._graphs):
                Gr.close()
            for S in list(self._scfs):
                S.close()
            for H in list(self._hams):
                H.close()
            load().sparc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian:
    """H(k) on the device: grid, V_eff and projector boxes (sparc_ham_create)."""

    def __init__(self, ctx: Context, n, h, fd_radius, k, veff, proj=None):
        L = load()
        self.ctx = ctx
        g = SparcGrid()
        for s in range(3):
            g.n[s] = int(n[s])
            g.h[s] = float(h[s])
            g.k[s] = float(k[s])
        g.fd_radius = int(fd_radius)
        self.grid = g
        self.nd = int(n[0]) * int(n[1]) * int(n[2])
        self.cplx = any(float(v) != 0.0 for v in k)
        self._veff = np.ascontiguousarray(veff, dtype=np.float64)
        nl = SparcNonlocal()
        keep = []
        if proj is not None and proj.nproj > 0:
            arrs = [np.ascontiguousarray(proj.box_lo, np.int32).reshape(-1),
                    np.ascontiguousarray(proj.box_n, np.int32).reshape(-1),
                    np.ascontiguousarray(proj.chi_off, np.int64),
                    np.ascontiguousarray(proj.chi, np.float64),
                    np.ascontiguousarray(proj.gamma, np.float64)]
            keep = arrs
            nl.nproj = int(proj.nproj)
            nl.box_lo = arrs[0].ctypes.data_as(POINTER(c_int32))
            nl.box_n = arrs[1].ctypes.data_as(POINTER(c_int32))
            nl.chi_off = arrs[2].ctypes.data_as(POINTER(c_int64))
            nl.chi = arrs[3].ctypes.data_as(POINTER(c_double))
            nl.chi_len = int(arrs[3].size)
            nl.gamma = arrs[4].ctypes.data_as(POINTER(c_double))
        else:
            nl.nproj = 0
        self._keep = keep
        hh = c_void_p()
        rc = L.sparc_ham_create(ctx.handle, ctypes.byref(g),
                                self._veff.ctypes.data_as(POINTER(c_double)), ctypes.byref(nl),
                                ctypes.byref(hh))
        ctx.check(rc)
        self.handle = hh
        ctx._hams.add(self)

    @classmethod
    def from_workload(cls, ctx, wl, kidx=0):
        return cls(ctx, wl.n, wl.h, wl.fd_radius, wl.kpts[kidx], wl.veff, wl.proj)

    def filter_kernel(self, dtype) -> int:
        """The H-pass kernel sparc_cheb_filter runs for this H and dtype
        (sparc_filter_kernel: KERNEL_GENERIC, KERNEL_TILED or KERNEL_TMA)."""
        out = c_int(-1)
        self.ctx.check(load().sparc_filter_kernel(self.handle, int(dtype), ctypes.byref(out)))
        return out.value

    def close(self):
        if getattr(self, "handle", None):
            load().sparc_ham_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- the C entry points

def sparc_ham_set_veff(H: Hamiltonian, veff, stream=None):
    """Replace V_eff: a torch CUDA float64 tensor (async) or a numpy array (sync)."""
    if isinstance(veff, np.ndarray):
        a = np.ascontiguousarray(veff, np.float64)
        H.ctx.check(load().sparc_ham_set_veff(H.handle, a.ctypes.data, 0, None))
    else:
        H.ctx.check(load().sparc_ham_set_veff(H.handle, _ptr(veff), 1, _stream(stream)))


def sparc_apply_H(H: Hamiltonian, X, Y, ns=None, ld=None, stream=None, dtype=None):
    """Y = H X; X, Y are (ns, ld) CUDA tensors (column-major Nd x ns)."""
    ns = X.shape[0] if ns is None else ns
    ld = X.shape[-1] if ld is None else ld
    dt = dtype_code(X) if dtype is None else dtype
    H.ctx.check(load().sparc_apply_H(H.handle, dt, _ptr(X), _ptr(Y), int(ns), int(ld), _stream(stream)))


def sparc_apply_H_noalloc(H: Hamiltonian, X, Y, ns=None, ld=None, stream=None, dtype=None):
    """Y = H X in the library's fixed scratch array: the call allocates no device memory.

    For callers that cannot allocate when they need H X (device memory owned by
    another allocator or a fixed budget, loops that may not block on cudaMalloc).  Needs the projector values of H in this
    dtype on the device already (one sparc_apply_H call with the dtype uploads
    them); calls that overlap on the GPU share the scratch and race.
    """
    ns = X.shape[0] if ns is None else ns
    ld = X.shape[-1] if ld is None else ld
    dt = dtype_code(X) if dtype is None else dtype
    H.ctx.check(load().sparc_apply_H_noalloc(H.handle, dt, _ptr(X), _ptr(Y), int(ns), int(ld),
                                             _stream(stream)))


def sparc_cheb_filter(H: Hamiltonian, m, a, b, a0, X, Y, ns=None, ld=None, stream=None, dtype=None):
    """Y = C_m((H-c)/e) X / C_m((a0-c)/e), e=(b-a)/2, c=(b+a)/2."""
    ns = X.shape[0] if ns is None else ns
    ld = X.shape[-1] if ld is None else ld
    dt = dtype_code(X) if dtype is None else dtype
    H.ctx.check(load().sparc_cheb_filter(H.handle, dt, int(m), float(a), float(b), float(a0), _ptr(X),
                                         _ptr(Y), int(ns), int(ld), _stream(stream)))


def _batch_args(Hs, a, b, a0):
    nk = len(Hs)
    hs = (c_void_p * nk)(*[h.handle for h in Hs])
    arr = [(c_double * nk)(*[float(v) for v in x]) for x in (a, b, a0)]
    return nk, hs, arr


def sparc_cheb_filter_batch(Hs, m, a, b, a0, X, Y, stream=None, dtype=None):
    """The filter for Hamiltonians Hs[k] that differ only in k, in shared launches.

    X, Y: CUDA tensors of shape (nk, ns, ld) (block k = orbitals of k-point k);
    a, b, a0: sequences of nk bounds."""
    nk, hs, (aa, bb, cc) = _batch_args(Hs, a, b, a0)
    assert X.shape[0] == nk and Y.shape == X.shape
    dt = dtype_code(X) if dtype is None else dtype
    Hs[0].ctx.check(load().sparc_cheb_filter_batch(hs, nk, dt, int(m), aa, bb, cc, _ptr(X), _ptr(Y),
                                                   int(X.shape[1]), int(X.shape[2]), _stream(stream)))


def sparc_autotune_filter(Hs, m, a, b, a0, X, Y, stream=None, dtype=None):
    """Time the filter's launch shapes on (X, Y) and keep the fastest; returns (units, ms)."""
    nk, hs, (aa, bb, cc) = _batch_args(Hs, a, b, a0)
    if X.dim() == 2:
        X, Y = X.unsqueeze(0), Y.unsqueeze(0)
    dt = dtype_code(X) if dtype is None else dtype
    units, ms = c_int(), c_double()
    Hs[0].ctx.check(load().sparc_autotune_filter(hs, nk, dt, int(m), aa, bb, cc, _ptr(X), _ptr(Y),
                                                 int(X.shape[1]), int(X.shape[2]), _stream(stream),
                                                 ctypes.byref(units), ctypes.byref(ms)))
    return units.value, ms.value


def sparc_set_filter_units(ctx: Context, dtype, nd, ns, nk, units):
    """Pin (units > 0) or clear (0) the orbital blocks per filter launch for (dtype, Nd, ns, nk)."""
    ctx.check(load().sparc_set_filter_units(ctx.handle, int(dtype), int(nd), int(ns), int(nk), int(units)))


class FilterGraph:
    """The filters of independent cells captured into one CUDA graph (sparc_filter_graph_*).

    Hs, m, a, b, a0: per cell; X, Y: per-cell CUDA tensors of shape (ns, ld)."""

    def __init__(self, Hs, m, a, b, a0, X, Y, nbranch=8, dtype=None):
        n = len(Hs)
        self.ctx = Hs[0].ctx
        self._keep = (list(Hs), list(X), list(Y))
        dt = dtype_code(X[0]) if dtype is None else dtype
        hs = (c_void_p * n)(*[h.handle for h in Hs])
        xs = (c_void_p * n)(*[_ptr(x) for x in X])
        ys = (c_void_p * n)(*[_ptr(y) for y in Y])
        ms = (c_int * n)(*[int(v) for v in m])
        nss = (c_int * n)(*[int(x.shape[0]) for x in X])
        lds = (c_int64 * n)(*[int(x.shape[-1]) for x in X])
        dv = lambda v: (c_double * n)(*[float(t) for t in v])
        self.n = n
        h = c_void_p()
        self.ctx.check(load().sparc_filter_graph_create(hs, n, dt, ms, dv(a), dv(b), dv(a0), xs, ys, nss, lds,
                                                        int(nbranch), ctypes.byref(h)))
        self.handle = h
        self.ctx._graphs.add(self)

    def set_bounds(self, a, b, a0):
        dv = lambda v: (c_double * self.n)(*[float(t) for t in v])
        self.ctx.check(load().sparc_filter_graph_set_bounds(self.handle, dv(a), dv(b), dv(a0)))

    def launch(self, stream=None):
        self.ctx.check(load().sparc_filter_graph_launch(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().sparc_filter_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_NFEAT, MLP_NHID = 16, 128
MLP_NPARAM = MLP_NFEAT * MLP_NHID + MLP_NHID + MLP_NHID * MLP_NHID + MLP_NHID + MLP_NHID + 1


class Mlp:
    """The density network 16 -> 128 -> 128 -> 1 (sparc_mlp_*): parameters, Adam state."""

    def __init__(self, ctx: Context, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == MLP_NPARAM
        self.ctx = ctx
        h = c_void_p()
        ctx.check(load().sparc_mlp_create(ctx.handle, th.ctypes.data, ctypes.byref(h)))
        self.handle = h
        ctx._graphs.add(self)

    def params(self):
        out = np.zeros(MLP_NPARAM, np.float32)
        self.ctx.check(load().sparc_mlp_params(self.handle, out.ctypes.data, 0))
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        self.ctx.check(load().sparc_mlp_params(self.handle, th.ctypes.data, 1))

    def forward(self, D, y, stream=None):
        """y[p] = network(D[p]) for a float32 CUDA tensor D of shape (N, 16)."""
        self.ctx.check(load().sparc_mlp_forward(self.handle, _ptr(D), int(D.shape[0]), _ptr(y), _stream(stream)))

    def grad(self, D, t, grad, idx=None, stream=None):
        """Gradient of the mean squared error into the float32 CUDA tensor `grad`; returns the loss."""
        loss = c_double()
        n = int(idx.shape[0]) if idx is not None else int(D.shape[0])
        self.ctx.check(load().sparc_mlp_grad(self.handle, _ptr(D), _ptr(t), int(D.shape[0]), _ptr(idx), n,
                                             _ptr(grad), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def train_step(self, D, t, lr, idx=None, want_loss=False, stream=None):
        """One Adam step on the points idx (int64 CUDA tensor) or all rows of D."""
        loss = c_double()
        n = int(idx.shape[0]) if idx is not None else int(D.shape[0])
        self.ctx.check(load().sparc_mlp_train_step(self.handle, _ptr(D), _ptr(t), int(D.shape[0]), _ptr(idx), n,
                                                   float(lr), ctypes.byref(loss) if want_loss else None,
                                                   _stream(stream)))
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "handle", None):
            load().sparc_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sparc_mlp_descriptors(ctx: Context, n, h, atoms, widths, D, stream=None):
    """Descriptors D (float32 CUDA tensor (Nd, 16)) of the grid nodes for the atoms."""
    nn = (c_int * 3)(*[int(v) for v in n])
    hh = (c_double * 3)(*[float(v) for v in h])
    R = np.ascontiguousarray(atoms, dtype=np.float64).reshape(-1)
    w = np.ascontiguousarray(widths, dtype=np.float64)
    ctx.check(load().sparc_mlp_descriptors(ctx.handle, nn, hh, int(R.size // 3), R.ctypes.data, w.ctypes.data,
                                           _ptr(D), _stream(stream)))


def sparc_lanczos_bounds(H: Hamiltonian, ksteps, v0, stream=None):
    """(a0, b) from `ksteps` Lanczos steps started at the device vector v0."""
    a0 = c_double()
    b = c_double()
    H.ctx.check(load().sparc_lanczos_bounds(H.handle, int(ksteps), _ptr(v0), ctypes.byref(a0),
                                            ctypes.byref(b), _stream(stream)))
    return a0.value, b.value


def sparc_rayleigh_ritz(H: Hamiltonian, U, eig, mode, ns=None, ld=None, stream=None, dtype=None):
    """Rayleigh-Ritz in place on U (ns, ld); eig: CUDA float64 tensor of ns values."""
    ns = U.shape[0] if ns is None else ns
    ld = U.shape[-1] if ld is None else ld
    dt = dtype_code(U) if dtype is None else dtype
    H.ctx.check(load().sparc_rayleigh_ritz(H.handle, dt, _ptr(U), int(ns), int(ld), _ptr(eig), int(mode),
                                           _stream(stream)))


def sparc_gram_f32(ctx: Context, A, B, G, nd=None, stream=None):
    """G = A^T B (FP64, ns x ns) for FP32 CUDA tensors A, B of shape (ns, ld) (column-major nd x ns)."""
    ns = A.shape[0]
    nd = A.shape[-1] if nd is None else nd
    ctx.check(load().sparc_gram_f32(ctx.handle, _ptr(A), int(A.shape[-1]), _ptr(B), int(B.shape[-1]), int(nd),
                                    int(ns), _ptr(G), _stream(stream)))


def sparc_rotate_f32(ctx: Context, U, Yr, C, nd=None, stream=None):
    """C = U Yr for FP32 CUDA tensors U, C of shape (ns, ld) and an FP64 (ns, ns) tensor Yr
    holding the column-major ns x ns matrix (row n of the tensor is column n of Yr)."""
    ns = U.shape[0]
    nd = U.shape[-1] if nd is None else nd
    ctx.check(load().sparc_rotate_f32(ctx.handle, _ptr(U), int(U.shape[-1]), _ptr(Yr), int(nd), int(ns), _ptr(C),
                                      int(C.shape[-1]), _stream(stream)))


def sparc_gram_c64(ctx: Context, A, B, G, nd=None, stream=None):
    """G = A^H B (complex128, ns x ns) for complex64 CUDA tensors A, B of shape (ns, ld)
    (column-major nd x ns); row j of the tensor G is column j of the matrix."""
    ns = A.shape[0]
    nd = A.shape[-1] if nd is None else nd
    ctx.check(load().sparc_gram_c64(ctx.handle, _ptr(A), int(A.shape[-1]), _ptr(B), int(B.shape[-1]), int(nd),
                                    int(ns), _ptr(G), _stream(stream)))


def sparc_rotate_c64(ctx: Context, U, Yr, C, nd=None, stream=None):
    """C = U Yr for complex64 CUDA tensors U, C of shape (ns, ld) and a complex128 (ns, ns)
    tensor Yr holding the column-major ns x ns matrix (row n of the tensor is column n)."""
    ns = U.shape[0]
    nd = U.shape[-1] if nd is None else nd
    ctx.check(load().sparc_rotate_c64(ctx.handle, _ptr(U), int(U.shape[-1]), _ptr(Yr), int(nd), int(ns), _ptr(C),
                                      int(C.shape[-1]), _stream(stream)))


class Scf:
    """SCF state on a Hamiltonian (sparc_scf_create): pseudocharges, history, fields."""

    FIELDS = {"b": 0, "rho": 1, "phi": 2, "vxc": 3, "vout": 4, "veff": 5}

    def __init__(self, H, R, Z, rc, v0, kT=0.01, mix_beta=0.3, mix_history=7, poisson_tol=1e-10,
                 proj_atom=None, first_passes=1, wk=None):
        """H: a Hamiltonian, or a list of them (one per k-point, weights wk)."""
        Hs = list(H) if isinstance(H, (list, tuple)) else [H]
        H = Hs[0]
        self.H = H
        self.Hs = Hs
        self.nk = len(Hs)
        self._R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
        self._Z = np.ascontiguousarray(Z, dtype=np.float64)
        self._rc = np.ascontiguousarray(rc, dtype=np.float64)
        v = np.asarray(v0)
        if np.iscomplexobj(v):
            v = np.ascontiguousarray(v.astype(np.complex128)).view(np.float64)
        self._v0 = np.ascontiguousarray(v, dtype=np.float64)
        d = SparcScfDesc()
        d.natom = int(self._Z.size)
        d.R = self._R.ctypes.data_as(POINTER(c_double))
        d.Z = self._Z.ctypes.data_as(POINTER(c_double))
        d.rc = self._rc.ctypes.data_as(POINTER(c_double))
        d.kT = float(kT)
        d.mix_beta = float(mix_beta)
        d.mix_history = int(mix_history)
        d.poisson_tol = float(poisson_tol)
        d.v0 = self._v0.ctypes.data_as(POINTER(c_double))
        self._pa = None if proj_atom is None else np.ascontiguousarray(proj_atom, dtype=np.int32)
        d.proj_atom = None if self._pa is None else self._pa.ctypes.data_as(POINTER(c_int32))
        d.first_passes = int(first_passes)
        h = c_void_p()
        if self.nk == 1 and wk is None:
            H.ctx.check(load().sparc_scf_create(H.handle, ctypes.byref(d), ctypes.byref(h)))
        else:
            w = np.full(self.nk, 1.0 / self.nk) if wk is None else np.asarray(wk, dtype=np.float64)
            self._wk = np.ascontiguousarray(w, dtype=np.float64)
            hs = (c_void_p * self.nk)(*[x.handle for x in Hs])
            H.ctx.check(load().sparc_scf_create_k(hs, self.nk, self._wk.ctypes.data_as(POINTER(c_double)),
                                                  ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        H.ctx._scfs.add(self)

    @classmethod
    def from_system(cls, H: Hamiltonian, sysd, **kw):
        return cls(H, sysd.wl.atoms, sysd.Z, sysd.rc, sysd.v0, proj_atom=sysd.wl.proj.atom, **kw)

    def forces(self, U, ns=None, ld=None, stream=None, dtype=None):
        """(f, f_loc, f_nloc), each (natom, 3), at the state of the last step (sparc_scf_forces);
        U: (ns, ld) at Gamma, or (nk, ns, ld) Bloch orbitals of every k-point."""
        ns = U.shape[-2] if ns is None else ns
        ld = U.shape[-1] if ld is None else ld
        dt = dtype_code(U) if dtype is None else dtype
        na = int(self._Z.size)
        out = np.zeros(9 * na)
        self.H.ctx.check(load().sparc_scf_forces(self.handle, dt, _ptr(U), int(ns), int(ld),
                                                 out.ctypes.data_as(POINTER(c_double)), _stream(stream)))
        return out[:3 * na].reshape(na, 3), out[3 * na:6 * na].reshape(na, 3), out[6 * na:].reshape(na, 3)

    def set_density(self, dy=None, scale=0.0, stream=None):
        """Starting density max(-b + scale*dy, 0) normalised to N_e (sparc_scf_set_density);
        dy: float32 CUDA tensor of Nd values, or None for the atomic superposition."""
        self.H.ctx.check(load().sparc_scf_set_density(self.handle, _ptr(dy), float(scale), _stream(stream)))

    def read(self, name: str, out, stream=None):
        """Copy a grid field (b, rho, phi, vxc, vout, veff) into the float64 CUDA tensor `out`."""
        self.H.ctx.check(load().sparc_scf_read(self.handle, self.FIELDS[name], _ptr(out), _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().sparc_scf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sparc_scf_step(S: Scf, U, eig, m, ns=None, ld=None, stream=None, dtype=None) -> dict:
    """One SCF iteration on the orbitals U in place -- (ns, ld), or (nk, ns, ld) for a
    k-point SCF with eig of nk*ns values; returns the sparc_scf_info fields."""
    if ns is None:
        ns = U.shape[-2]
    ld = U.shape[-1] if ld is None else ld
    dt = dtype_code(U) if dtype is None else dtype
    info = SparcScfInfo()
    S.H.ctx.check(load().sparc_scf_step(S.handle, dt, int(m), _ptr(U), int(ns), int(ld), _ptr(eig),
                                        ctypes.byref(info), _stream(stream)))
    return info.as_dict()
