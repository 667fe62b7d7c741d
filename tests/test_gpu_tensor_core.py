"""Tensor-core (tcgen05, error-compensated TF32) projections and rotation of
Rayleigh-Ritz for FP32 and complex64 data (Section 3.4, Eqs.
SubspaceGeneralizedEigenproblem and OrbitalTransformation; complex64 for the Bloch
orbitals of Section 3.3), through the C ABI, against FP64 products of the same inputs.

Tolerances are relative to the Cauchy-Schwarz bound of each entry (|G_ij| <=
sqrt(G_ii G_jj); |C_ng| <= |Yr column n| |U row g|).  The rotation's 3xTF32 product
keeps about 22 bits (a_hi rounded to nearest, the dropped a_lo b_lo term 2^-22
relative; the Grams keep it), and the FP32 accumulation runs over chunks of 64 grid
points before the FP64 sum, so 5e-6 holds with margin; a single TF32 product (10
stored mantissa bits, truncated) misses it by more than an order of magnitude.  The
diagonal test pins the Grams' bias: the tensor core's FP32 accumulation rounds toward
zero, so every |u|^2 comes out low, by about 2.5e-7 of itself with chunks of 64
points (6e-7 with chunks of 256).
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
    rel = (np.diag(g) - np.sum(A64 * A64, 1)) / np.diag(g)
    assert np.max(np.abs(rel)) < 3e-6
    # the sums of squares' bias (the mean over the 96 columns; each column's own
    # scatter is far smaller): measured 2.5e-7 with 8 MMAs per FP32 chunk, 6e-7 with 32
    print(f"diagonal: mean {np.mean(rel):.2e}, max {np.max(np.abs(rel)):.2e}")
    assert abs(np.mean(rel)) < 3.5e-7, np.mean(rel)


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


def _corbitals(nd, ns, ld, seed):
    X = np.zeros((ns, ld), dtype=np.complex64)
    X[:, :nd] = synth.random_orbitals(nd, ns, seed, complex_=True).astype(np.complex64)
    return X


@pytest.mark.parametrize("nd,ns,pad", [(4096, 128, 0), (3001, 130, 3), (8192, 300, 0), (777, 1, 1),
                                       (64000, 192, 0), (96, 40, 2)])
def test_complex_gram_matches_fp64_product(ctx, nd, ns, pad):
    """G = A^H B for complex64 data (Section 3.3's Bloch orbitals) from two real Grams of
    the real views: the real part symmetric, the imaginary part antisymmetric (its
    tiles below the diagonal mirrored with a minus sign), so G is Hermitian exactly.
    Even leading dimensions and nd take the TMA-fed kernel, the others the
    register-staged one."""
    from paper_1603_04339_gb300 import sparc
    A = _corbitals(nd, ns, nd + pad, 41 + ns)
    d = np.random.default_rng(42 + ns).uniform(-2.0, 3.0, nd).astype(np.float32)
    B = np.zeros_like(A)
    B[:, :nd] = A[:, :nd] * d      # like H U: A^H D A is Hermitian
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    G = torch.zeros((ns, ns), dtype=torch.complex128, device="cuda")
    G2 = torch.zeros_like(G)
    sparc.sparc_gram_c64(ctx, Ad, Bd, G, nd=nd)
    sparc.sparc_gram_c64(ctx, Ad, Bd, G2, nd=nd)
    ctx.sync()
    assert torch.equal(G, G2), "not deterministic"
    g = G.cpu().numpy().T          # g[i, j] = a_i^H b_j
    assert np.array_equal(g, np.conj(g.T)), "not Hermitian"
    A64, B64 = A[:, :nd].astype(np.complex128), B[:, :nd].astype(np.complex128)
    ref = np.conj(A64) @ B64.T
    ref = 0.5 * (ref + np.conj(ref.T))
    scale = np.sqrt(np.outer(np.sum(np.abs(A64) ** 2, 1), np.sum(np.abs(B64) ** 2, 1)))
    err = np.max(np.abs(g - ref) / scale)
    assert err < 5e-6, err


def test_complex_gram_of_an_imaginary_hermitian_operator(ctx):
    """B = P A with P = i (S - S^T), S the cyclic shift of the grid index (a Hermitian
    operator with imaginary entries, like the momentum -i d/dx): A^H B is Hermitian and
    its imaginary parts are as large as its real parts, so a sign or conjugation slip in
    the antisymmetric half of the Gram fails."""
    from paper_1603_04339_gb300 import sparc
    nd, ns = 4096, 64
    A = _corbitals(nd, ns, nd, 7)
    B = (1j * (np.roll(A, -1, axis=1) - np.roll(A, 1, axis=1))).astype(np.complex64)
    G = torch.zeros((ns, ns), dtype=torch.complex128, device="cuda")
    sparc.sparc_gram_c64(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), G, nd=nd)
    ctx.sync()
    g = G.cpu().numpy().T
    A64, B64 = A.astype(np.complex128), B.astype(np.complex128)
    ref = np.conj(A64) @ B64.T
    # P is Hermitian (up to the complex64 rounding of B)
    assert np.max(np.abs(ref - np.conj(ref.T))) < 1e-6 * np.max(np.abs(ref))
    ref = 0.5 * (ref + np.conj(ref.T))
    assert np.max(np.abs(ref.imag)) > 0.3 * np.max(np.abs(ref))
    scale = np.sqrt(np.outer(np.sum(np.abs(A64) ** 2, 1), np.sum(np.abs(B64) ** 2, 1)))
    err = np.max(np.abs(g - ref) / scale)
    assert err < 5e-6, err


@pytest.mark.parametrize("nd,ns,pad", [(4096, 128, 0), (3001, 130, 3), (200, 1, 0), (64000, 192, 0),
                                       (8192, 300, 1)])
def test_complex_rotation_matches_fp64_product(ctx, nd, ns, pad):
    """C = U Yr for complex64 U: one real rotation over 2 ns values of k, the i U half
    formed from U as it is loaded."""
    from paper_1603_04339_gb300 import sparc
    U = _corbitals(nd, ns, nd + pad, 51 + ns)
    rng = np.random.default_rng(61 + ns)
    Yr = rng.standard_normal((ns, ns)) + 1j * rng.standard_normal((ns, ns))   # tensor row n = column n
    Ud = torch.from_numpy(U).cuda()
    Yd = torch.from_numpy(Yr).cuda()
    C = torch.full((ns, nd + pad), 7.0 + 3.0j, dtype=torch.complex64, device="cuda")
    sparc.sparc_rotate_c64(ctx, Ud, Yd, C, nd=nd)
    ctx.sync()
    c = C.cpu().numpy()
    assert np.all(c[:, nd:] == np.complex64(7.0 + 3.0j)), "wrote past nd"
    U64 = U[:, :nd].astype(np.complex128)
    Y32 = Yr.astype(np.complex64).astype(np.complex128)   # Yr is rounded to FP32 on the way in
    ref = Y32 @ U64
    scale = np.outer(np.sqrt(np.sum(np.abs(Y32) ** 2, 1)), np.sqrt(np.sum(np.abs(U64) ** 2, 0)))
    err = np.max(np.abs(c[:, :nd] - ref) / scale)
    assert err < 5e-6, err


def test_complex_rotation_rejects_overlap(ctx):
    from paper_1603_04339_gb300 import sparc
    U = torch.zeros((4, 100), dtype=torch.complex64, device="cuda")
    Yr = torch.eye(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(sparc.SparcError):
        sparc.sparc_rotate_c64(ctx, U, Yr, U)
