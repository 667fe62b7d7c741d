"""Tensor-core (tcgen05, 3xTF32) projections and rotation of Rayleigh-Ritz for FP32
data (Section 3.4, Eqs. SubspaceGeneralizedEigenproblem and OrbitalTransformation),
through the C ABI, against FP64 products of the same FP32 inputs.

Tolerances are relative to the Cauchy-Schwarz bound of each entry (|G_ij| <=
sqrt(G_ii G_jj); |C_ng| <= |Yr column n| |U row g|).  A 3xTF32 product keeps about
21 bits (the dropped a_lo b_lo term is 2^-22 relative) and the FP32 accumulation
runs over chunks of 1024 grid points before the FP64 sum, so 5e-6 holds with
margin; a single TF32 product (10 stored mantissa bits, truncated) misses it by
more than an order of magnitude.
"""
import numpy as np
import pytest

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


def _orbitals(nd, ns, ld, seed):
    X = np.zeros((ns, ld), dtype=np.float32)
    X[:, :nd] = synth.random_orbitals(nd, ns, seed).astype(np.float32)
    return X


@pytest.mark.parametrize("nd,ns,pad", [(4096, 128, 0), (3001, 130, 3), (8192, 300, 0), (777, 1, 1),
                                       (65536, 512, 0), (4100, 200, 4), (96, 40, 0)])
def test_gram_matches_fp64_product(ctx, nd, ns, pad):
    """Leading dimensions and nd that are multiples of 4 take the TMA-fed kernel
    (ragged last k-tile and columns past ns read as zero from the tensor map); the
    others the register-staged one."""
    from paper_1603_04339_gb300 import sparc
    # B = D A with a diagonal D on the grid, like H U: the exact G = A^T D A is symmetric,
    # which the library assumes (it computes the tiles on and above the diagonal)
    A = _orbitals(nd, ns, nd + pad, 11 + ns)
    d = np.random.default_rng(12 + ns).uniform(-2.0, 3.0, nd).astype(np.float32)
    B = np.zeros_like(A)
    B[:, :nd] = A[:, :nd] * d
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    G = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
    G2 = torch.zeros_like(G)
    sparc.sparc_gram_f32(ctx, Ad, Bd, G, nd=nd)
    sparc.sparc_gram_f32(ctx, Ad, Bd, G2, nd=nd)
    ctx.sync()
    g = G.cpu().numpy()
    assert torch.equal(G, G2), "not deterministic"
    assert np.array_equal(g, g.T), "not symmetric"
    A64, B64 = A[:, :nd].astype(np.float64), B[:, :nd].astype(np.float64)
    ref = A64 @ B64.T          # G[i, j] = a_i . b_j  (row i of the tensor is column i)
    ref = 0.5 * (ref + ref.T)  # symmetric up to the FP32 rounding of B
    scale = np.sqrt(np.outer(np.sum(A64 * A64, 1), np.sum(B64 * B64, 1)))
    err = np.max(np.abs(g - ref) / scale)
    assert err < 5e-6, err


def test_gram_of_equal_operands_is_positive_definite(ctx):
    from paper_1603_04339_gb300 import sparc
    nd, ns = 20000, 96
    A = _orbitals(nd, ns, nd, 5)
    Ad = torch.from_numpy(A).cuda()
    G = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
    sparc.sparc_gram_f32(ctx, Ad, Ad, G, nd=nd)
    ctx.sync()
    g = G.cpu().numpy()
    np.linalg.cholesky(g)
    A64 = A.astype(np.float64)
    assert np.max(np.abs(np.diag(g) - np.sum(A64 * A64, 1)) / np.diag(g)) < 3e-6


@pytest.mark.parametrize("nd,ns,pad", [(4096, 128, 0), (3001, 130, 3), (8192, 300, 1), (200, 1, 0),
                                       (262144, 512, 0)])
def test_rotation_matches_fp64_product(ctx, nd, ns, pad):
    from paper_1603_04339_gb300 import sparc
    U = _orbitals(nd, ns, nd + pad, 21 + ns)
    rng = np.random.default_rng(31 + ns)
    Yr = rng.standard_normal((ns, ns))      # tensor row n = column n of Yr
    Ud = torch.from_numpy(U).cuda()
    Yd = torch.from_numpy(Yr).cuda()
    C = torch.full((ns, nd + pad), 7.0, dtype=torch.float32, device="cuda")
    sparc.sparc_rotate_f32(ctx, Ud, Yd, C, nd=nd)
    ctx.sync()
    c = C.cpu().numpy()
    assert np.all(c[:, nd:] == 7.0), "wrote past nd"
    U64 = U[:, :nd].astype(np.float64)
    Y32 = Yr.astype(np.float32).astype(np.float64)   # Yr is rounded to FP32 on the way in
    ref = Y32 @ U64          # C column n = sum_k U column k * Yr[k, n]  (tensor: C[n] = sum_k Yr[n, k] U[k])
    # Cauchy-Schwarz scale |C[n, g]| <= |Yr column n| |U row g|, as for the Gram
    scale = np.outer(np.sqrt(np.sum(Y32 * Y32, 1)), np.sqrt(np.sum(U64 * U64, 0)))
    err = np.max(np.abs(c[:, :nd] - ref) / scale)
    assert err < 5e-6, err


def test_rotation_rejects_overlap(ctx):
    from paper_1603_04339_gb300 import sparc
    U = torch.zeros((4, 100), dtype=torch.float32, device="cuda")
    Yr = torch.eye(4, dtype=torch.float64, device="cuda")
    with pytest.raises(sparc.SparcError):
        sparc.sparc_rotate_f32(ctx, U, Yr, U)
