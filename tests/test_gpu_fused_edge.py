"""GPU parity of the fused pass of undirected edge updates.

An undirected edge update {u, v} is, in G_D, two directed updates (u, v) and (v, u).
The fused pass takes both candidates of every row from the state before the update
(one rank-1 pass over two row lists, each with its own column vector) instead of two
sequential passes.  A shortest simple path uses the edge in at most one direction, so
both forms give the same d and sigma: checked here bit for bit against the two-pass
form (option fused_edges = 0) after every update, and against the oracle at the end;
dependencies and BC within |err| <= 1e-9 * max(1, |x|).
"""
import numpy as np
import pytest

from paper_1311_2147_gb300 import binding, synth
from tests.parity_util import close, compare_full

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


def _fused_vs_two_pass(g, ups, dist, label, pair_walk=None):
    a = binding.BCGraph(g, dist=dist)
    b = binding.BCGraph(g, dist=dist)
    b.bc_set_option("fused_edges", 0)
    if pair_walk is not None:
        for h in (a, b):
            h.bc_set_option("pair_walk", pair_walk)
    for i, up in enumerate(ups):
        for h in (a, b):
            rc, done = h.bc_apply_updates([up])
            assert rc == 0 and done == 1, (label, up, h.last_error())
        da, sa, la = a.bc_get_rows()
        db, sb, lb = b.bc_get_rows()
        assert np.array_equal(da, db), f"{label}: distances differ after {up}"
        assert np.array_equal(sa, sb), f"{label}: path counts differ after {up}"
        ok, worst = close(la, lb)
        assert ok, f"{label}: dependencies differ after update {i} ({worst:.3g} x tol)"
        ok, worst = close(a.bc_get_scores(), b.bc_get_scores())
        assert ok, f"{label}: BC differs after update {i} ({worst:.3g} x tol)"
    compare_full(a, synth.apply_updates(g, ups), label=label)
    return a.bc_get_info(), b.bc_get_info()


@pytest.mark.parametrize("dist", ["i32", "i64"])
@pytest.mark.parametrize("wmax", [1, 3, 1000])
def test_fused_matches_two_pass_er(dist, wmax):
    g = synth.erdos_renyi(96, 260, 1, wmax, 900 + wmax, directed=False)
    # unit weights admit new edges only (no weight can decrease)
    ups = synth.update_stream(g, 20, 0, 0, 901, 1, 1) if wmax == 1 else \
        synth.update_stream(g, 10, 10, 0, 901 + wmax, 1, wmax)
    ia, ib = _fused_vs_two_pass(g, ups, dist, f"ER w<={wmax} {dist}")
    # the fused form runs one rank-1 launch per edge update, the two-pass form two
    assert ia["kernel_launches"] < ib["kernel_launches"]


def test_fused_ties_cycles_and_components():
    # equal-length second routes (ties only), then an edge joining two components
    g = synth.cycle_graph(40, False, 1)
    _fused_vs_two_pass(g, [("edge", 0, 20, 20), ("edge", 10, 30, 20), ("edge", 5, 25, 3)], "i64", "cycle ties")
    a = synth.path_graph(12, False, 2)
    src = np.concatenate([a.src, a.src + 12]).astype(np.int32)
    dst = np.concatenate([a.dst, a.dst + 12]).astype(np.int32)
    w = np.concatenate([a.w, a.w]).astype(np.int64)
    g2 = synth.Graph(24, False, src, dst, w)
    _fused_vs_two_pass(g2, [("edge", 3, 15, 1), ("edge", 0, 23, 5), ("edge", 11, 12, 1)], "i32", "components")


def test_fused_decrease_on_shortest_paths_and_walks():
    g = synth.path_graph(64, False, 5)
    ups = [("edge", 10, 11, 2), ("edge", 20, 21, 1), ("edge", 0, 63, 3), ("edge", 30, 40, 7)]
    _fused_vs_two_pass(g, ups, "i32", "path decreases, column test", pair_walk=0)
    _fused_vs_two_pass(g, ups, "i32", "path decreases, DAG walks", pair_walk=1)


def test_fused_ba_stream_with_vertex_updates():
    # vertex updates keep the two-phase form; edge updates between them take the fused one
    g, ups = synth.workload_ba16384(n=512, n_updates=40)
    _fused_vs_two_pass(g, ups, "i32", "BA n=512 mixed")


def test_ragged_n_uses_the_two_pass_form():
    # n not a multiple of the vector width: the fused pass is not used, results unchanged
    g = synth.erdos_renyi(67, 200, 1, 9, 77, directed=False)
    ups = synth.update_stream(g, 6, 6, 0, 78, 1, 9)
    ia, ib = _fused_vs_two_pass(g, ups, "i32", "ragged n=67")
    assert ia["kernel_launches"] == ib["kernel_launches"]
