"""The uneven batch of 16 independent cells (grids 24^3 .. 48^3, slab and wire
shapes, 8..95 atoms, Ns 48..384, m 16..24) through the filter graph, FP32.

* every cell's output of one graph launch equals its own sparc_cheb_filter call
  bit for bit, with autotuned launch groupings in place and after new bounds;
* sampled columns of three cells against the oracle's filter.
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


def _bounds(cells, shift=0.0):
    a0 = [-2.5 - 0.05 * i + shift for i in range(len(cells))]
    b = [60.0 + i + shift for i in range(len(cells))]
    a = [a0[i] + (b[i] - a0[i]) * (c.ns / c.nd) ** (2.0 / 3.0) for i, c in enumerate(cells)]
    return a, b, a0


def test_cell_batch_graph_equals_per_cell_filters_and_oracle(ctx):
    from paper_1603_04339_gb300 import sparc
    cells = synth.config4()
    Hs = [sparc.Hamiltonian.from_workload(ctx, c) for c in cells]
    X = [torch.from_numpy(synth.random_orbitals(c.nd, c.ns, 5000 + i).astype(np.float32)).cuda()
         for i, c in enumerate(cells)]
    Y = [torch.full_like(x, float("nan")) for x in X]
    m = [c.m for c in cells]
    a, b, a0 = _bounds(cells)
    tuned = []
    for i, H in enumerate(Hs):
        u, ms = sparc.sparc_autotune_filter([H], m[i], [a[i]], [b[i]], [a0[i]], X[i], Y[i])
        tuned.append(u)
    print("tuned units per launch:", tuned)
    G = sparc.FilterGraph(Hs, m, a, b, a0, X, Y, nbranch=8)
    for shift in (0.0, -0.3):
        if shift:
            a, b, a0 = _bounds(cells, shift)
            G.set_bounds(a, b, a0)
        for y in Y:
            y.fill_(float("nan"))
        G.launch()
        torch.cuda.synchronize()
        for i, H in enumerate(Hs):
            ref = torch.empty_like(X[i])
            sparc.sparc_cheb_filter(H, m[i], a[i], b[i], a0[i], X[i], ref)
            torch.cuda.synchronize()
            assert torch.equal(ref, Y[i]), (shift, cells[i].name)
    small = sorted(range(len(cells)), key=lambda i: cells[i].nd * cells[i].m)[:3]
    for i in small:
        c = cells[i]
        Hor = O.OracleH(c)
        cols = [0, c.ns - 1]
        Yo = O.cheb_filter(Hor, X[i][cols].cpu().numpy().astype(np.float64), c.m, a[i], b[i], a0[i])
        err = _colerr(Y[i][cols].cpu().numpy().astype(np.float64), Yo)
        assert err < 1e-4, (c.name, err)
    G.close()


def test_filter_graph_rejects_bad_bounds(ctx):
    from paper_1603_04339_gb300 import sparc
    c = synth.small_case(n=(16, 14, 15), natom=2, ns=12, seed=3)
    H = sparc.Hamiltonian.from_workload(ctx, c)
    X = [torch.zeros((c.ns, c.nd), dtype=torch.float32, device="cuda")]
    Y = [torch.zeros_like(X[0])]
    with pytest.raises(sparc.SparcError):
        sparc.FilterGraph([H], [4], [1.0], [0.5], [-1.0], X, Y)
    G = sparc.FilterGraph([H], [4], [0.0], [1.0], [-1.0], X, Y)
    with pytest.raises(sparc.SparcError):
        G.set_bounds([0.0], [1.0], [0.5])
    G.launch()
    torch.cuda.synchronize()
    G.close()


def test_fp32_pass_shapes_match_each_other_and_oracle(ctx):
    """The FP32 pass with 16 x 8 tiles (256-thread CTAs, two per SM) takes every node
    and projector piece in the order of the 16 x 16 tile, so the filter is the same bit
    for bit; the TMA-fed pass (the default here) is the same bit for bit over any
    grouping of blocks per launch; all of them match the oracle."""
    from paper_1603_04339_gb300 import sparc
    wl = synth.small_case(n=(24, 22, 26), natom=4, ns=37, m=9, seed=77)
    H = sparc.Hamiltonian.from_workload(ctx, wl)
    X = torch.from_numpy(synth.random_orbitals(wl.nd, wl.ns, 808).astype(np.float32)).cuda()
    a0, b = -3.0, 60.0
    a = a0 + (b - a0) * (wl.ns / wl.nd) ** (2.0 / 3.0)
    TS = sparc.TUNE_SHAPE

    def run(codes):
        outs = []
        for code in codes:
            sparc.sparc_set_filter_units(ctx, sparc.F32, wl.nd, wl.ns, 1, code)
            Y = torch.full_like(X, float("nan"))
            sparc.sparc_cheb_filter(H, wl.m, a, b, a0, X, Y)
            torch.cuda.synchronize()
            outs.append(Y)
        sparc.sparc_set_filter_units(ctx, sparc.F32, wl.nd, wl.ns, 1, 0)
        return outs

    tiled = run((5, 2, 3 + TS, 1 + TS))             # 16 x 16 and 16 x 8 tiles, groups of 5, 2, 3, 1 blocks
    tma = run((0, 5 + 2 * TS, 2 + 2 * TS))          # default, and the TMA pass in groups of 5 and 2
    for Y in tiled[1:]:
        assert torch.equal(Y, tiled[0])
    for Y in tma[1:]:
        assert torch.equal(Y, tma[0])
    Hor = O.OracleH(wl)
    cols = [0, 17, 36]
    Yo = O.cheb_filter(Hor, X[cols].cpu().numpy().astype(np.float64), wl.m, a, b, a0)
    assert _colerr(tiled[2][cols].cpu().numpy().astype(np.float64), Yo) < 1e-4
    assert _colerr(tma[0][cols].cpu().numpy().astype(np.float64), Yo) < 1e-4


def test_filter_graph_of_complex_cells(ctx):
    """A graph of two complex64 cells at different k equals their own filter calls."""
    from paper_1603_04339_gb300 import sparc
    cells = [synth.small_case(n=(16, 14, 15), natom=2, ns=12, m=5, k=(0.2, -0.1, 0.3), seed=21),
             synth.small_case(n=(18, 16, 14), natom=3, ns=20, m=6, k=(-0.25, 0.0, 0.15), seed=22)]
    Hs = [sparc.Hamiltonian.from_workload(ctx, c) for c in cells]
    X = [torch.from_numpy(synth.random_orbitals(c.nd, c.ns, 70 + i, complex_=True).astype(np.complex64)).cuda()
         for i, c in enumerate(cells)]
    Y = [torch.full_like(x, float("nan")) for x in X]
    m = [c.m for c in cells]
    a, b, a0 = _bounds(cells)
    G = sparc.FilterGraph(Hs, m, a, b, a0, X, Y, nbranch=2)
    G.launch()
    torch.cuda.synchronize()
    for i, H in enumerate(Hs):
        ref = torch.empty_like(X[i])
        sparc.sparc_cheb_filter(H, m[i], a[i], b[i], a0[i], X[i], ref)
        torch.cuda.synchronize()
        assert torch.equal(ref, Y[i]), i
    G.close()
