"""GPU parity of the DAG-walk form of the pair corrections (option "pair_walk") against
the column-test form and the oracle.

Both forms find the same columns (those on a shortest s-t path of each state) and add
the same terms; the walk form sums a row's terms as fixed-point integers (any order
gives the same sum), the column test in float-float in target order, so d and sigma
must be bit-identical between them and the dependency rows and BC equal within
|err| <= 1e-9 * max(1, |x|) after every update; at the end of each stream the walk form
is compared with the oracle.
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


def _walk_vs_test(g, ups, dist, label, every=1, cap=None):
    a = binding.BCGraph(g, dist=dist)
    a.bc_set_option("pair_walk", 1)
    if cap is not None:
        a.bc_set_option("walk_cap", cap)
    b = binding.BCGraph(g, dist=dist)
    b.bc_set_option("pair_walk", 0)
    for i, up in enumerate(ups):
        for h in (a, b):
            rc, done = h.bc_apply_updates([up])
            assert rc == 0 and done == 1, (label, up, h.last_error())
        if (i + 1) % every and i + 1 != len(ups):
            continue
        da, sa, la = a.bc_get_rows()
        db, sb, lb = b.bc_get_rows()
        assert np.array_equal(da, db), f"{label}: distances differ after {up}"
        assert np.array_equal(sa, sb), f"{label}: path counts differ after {up}"
        ok, worst = close(la, lb)
        assert ok, f"{label}: dependencies differ after update {i} {up} ({worst:.3g} x tol)"
        ok, worst = close(a.bc_get_scores(), b.bc_get_scores())
        assert ok, f"{label}: BC differs after update {i} ({worst:.3g} x tol)"
    compare_full(a, synth.apply_updates(g, ups), label=label)
    return a.bc_get_info()


@pytest.mark.parametrize("dist", ["i32", "i64"])
@pytest.mark.parametrize("wmax", [2, 9, 1000])
def test_walk_matches_column_test_er(dist, wmax):
    g = synth.erdos_renyi(80, 240, 1, wmax, 7000 + wmax, directed=False)
    ups = synth.update_stream(g, 8, 8, 6, 7100 + wmax, 1, wmax, kmin=1, kmax=6)
    info = _walk_vs_test(g, ups, dist, f"ER w<={wmax} {dist}")
    assert info["pair_rows"] > 0


def test_walk_matches_column_test_ba():
    g, ups = synth.workload_ba16384(n=700, n_updates=30)
    _walk_vs_test(g, ups, "i32", "BA n=700", every=5)


def test_walk_ties_and_cycles():
    # equal-length second routes: path counts grow, no distance drops
    g = synth.cycle_graph(40, False, 1)
    _walk_vs_test(g, [("edge", 0, 20, 20), ("edge", 10, 30, 20)], "i64", "cycle ties")


def test_walk_joining_components_and_new_edges():
    # new edges join components (their arcs did not exist in the old state)
    a = synth.path_graph(12, False, 2)
    k = 5
    src = np.concatenate([a.src + 12 * i for i in range(k)]).astype(np.int32)
    dst = np.concatenate([a.dst + 12 * i for i in range(k)]).astype(np.int32)
    w = np.concatenate([a.w] * k).astype(np.int64)
    g = synth.Graph(12 * k, False, src, dst, w)
    ups = [("edge", 3, 15, 1), ("edge", 30, 50, 4), ("vertex", 40, [(2, 1, 0), (27, 3, 0)])]
    _walk_vs_test(g, ups, "i32", "joining components")


def test_walk_decrease_on_a_shortest_path():
    # the lowered edge lay on old shortest paths: the old walks must use its old weight
    g = synth.path_graph(50, False, 5)
    ups = [("edge", 10, 11, 2), ("edge", 20, 21, 1), ("vertex", 30, [(29, 1, 0), (31, 2, 0), (5, 40, 0)])]
    _walk_vs_test(g, ups, "i32", "decreases on path edges")


def test_walk_long_paths_rows_for_whole_ctas():
    # closing a long unit path into a cycle: rows with up to the cap of changed targets,
    # each on a long path, so their walks find far more vertices than one warp takes
    g = synth.path_graph(300, False, 1)
    ups = [("edge", 0, 299, 1), ("edge", 100, 200, 3), ("edge", 50, 250, 1)]
    info = _walk_vs_test(g, ups, "i32", "path closed into a cycle")
    assert info["walk_pairs"] > 0 and info["walk_vertices"] > 0


def test_walk_mid_size_rows():
    # closing shorter unit paths into cycles: rows whose walks find between 129 and 512
    # vertices in all (the mid-size hash-table class) next to light and whole-CTA rows
    for n in (24, 40, 64):
        g = synth.path_graph(n, False, 1)
        info = _walk_vs_test(g, [("edge", 0, n - 1, 1), ("edge", 3, n - 4, 2)], "i32", f"path {n} closed")
        assert info["walk_vertices"] > 0


def test_walk_long_stream():
    g = synth.barabasi_albert(400, 3, 1, 30, 8181)
    ups = synth.update_stream(g, 40, 40, 20, 8282, 1, 30, kmin=1, kmax=5)
    _walk_vs_test(g, ups, "i32", "BA n=400, 100 updates", every=10)


def test_walk_buffer_overflow_falls_back_to_the_column_test():
    # a buffer too small for any walk: every update is done by the column test instead
    g = synth.erdos_renyi(64, 200, 1, 9, 4242, directed=False)
    ups = synth.update_stream(g, 6, 6, 4, 4343, 1, 9, kmin=1, kmax=5)
    _walk_vs_test(g, ups, "i32", "walk buffer of 1 entry", cap=1)


def test_row_lists_beyond_one_tile_of_flags():
    # n = 16400 > 1024 threads x 16 flags: the changed-row and full-row lists (one pass
    # over the flags, k_pair_lists) span two tiles.  Checked against a handle with the
    # pair corrections off (every changed row re-accumulated, lists from k_compact) on
    # BC and on rows of both tiles.
    n = 16400
    g = synth.erdos_renyi(n, 4 * n, 1, 50, 16400, directed=False)
    ups = synth.update_stream(g, 2, 2, 2, 16401, 1, 50, kmin=2, kmax=6)
    a = binding.BCGraph(g, dist="i32")
    a.bc_set_option("pair_walk", 1)
    b = binding.BCGraph(g, dist="i32")
    b.bc_set_option("pair_updates", 0)
    for h in (a, b):
        rc, done = h.bc_apply_updates(ups)
        assert rc == 0 and done == len(ups), h.last_error()
    assert a.bc_get_info()["pair_rows"] > 0
    for s0, cnt in ((0, 8), (16376, 24)):
        da, sa, la = a.bc_get_rows(s0, cnt)
        db, sb, lb = b.bc_get_rows(s0, cnt)
        assert np.array_equal(da, db) and np.array_equal(sa, sb), f"rows {s0}..{s0 + cnt}"
        ok, worst = close(la, lb)
        assert ok, f"dependencies of rows {s0}..{s0 + cnt} differ ({worst:.3g} x tol)"
    ok, worst = close(a.bc_get_scores(), b.bc_get_scores())
    assert ok, f"BC differs ({worst:.3g} x tol)"
    a.close()
    b.close()


def test_walk_option_rejected_on_directed_graphs():
    g = synth.erdos_renyi(20, 60, 1, 5, 3, directed=True)
    a = binding.BCGraph(g)
    with pytest.raises(binding.BCError) as e:
        a.bc_set_option("pair_walk", 1)
    assert e.value.code == binding.BC_ERR_ARG


def test_walk_through_hubs():
    # hubs with hundreds of E* arcs on the walks of many rows, and a vertex update of the
    # largest hub: results must equal the column test's bit for bit
    g = synth.barabasi_albert(3000, 4, 1, 3, 3003)
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n)
    assert deg.max() >= 64
    hub = int(np.argmax(deg))
    ups = synth.update_stream(g, 4, 4, 4, 3004, 1, 3, kmin=2, kmax=6)
    em = synth.EdgeMap.of(synth.apply_updates(g, ups))
    far = [x for x in range(g.n - 1, 0, -1) if x != hub and em.get(x, hub) is None][:6]
    ups.append(("vertex", hub, [(x, 1, 0) for x in far]))
    info = _walk_vs_test(g, ups, "i32", "BA n=3000 hubs", every=4)
    assert info["walk_pairs"] > 0
