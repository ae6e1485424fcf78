"""GPU parity of the pair-correction path ("pair_updates", on by default for undirected
graphs) against the full re-accumulation path and the oracle.

D and sigma must be bit-identical between the two paths (the option changes only how
dependency rows are updated); dependencies and BC agree within |err| <= 1e-9 * max(1, |x|)
with each other after every update and with the oracle at the end of each stream.
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


def _pair_vs_full(g, ups, dist, label, every=1):
    a = binding.BCGraph(g, dist=dist)
    b = binding.BCGraph(g, dist=dist)
    b.bc_set_option("pair_updates", 0)
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
    ia, ib = a.bc_get_info(), b.bc_get_info()
    assert ia["rows_reaccumulated"] == ib["rows_reaccumulated"]
    assert ib["rows_full"] == 0
    return ia


@pytest.mark.parametrize("dist", ["i32", "i64"])
@pytest.mark.parametrize("wmax", [2, 9, 1000])
def test_pair_matches_full_path_er(dist, wmax):
    g = synth.erdos_renyi(80, 240, 1, wmax, 7000 + wmax, directed=False)
    ups = synth.update_stream(g, 8, 8, 6, 7100 + wmax, 1, wmax, kmin=1, kmax=6)
    info = _pair_vs_full(g, ups, dist, f"ER w<={wmax} {dist}")
    assert info["rows_full"] < info["rows_reaccumulated"]


def test_pair_matches_full_path_ba():
    g, ups = synth.workload_ba16384(n=700, n_updates=30)
    info = _pair_vs_full(g, ups, "i32", "BA n=700", every=5)
    assert info["rows_full"] < info["rows_reaccumulated"]


def test_pair_rows_over_the_cap_take_the_full_path():
    # closing a long unit path into a cycle changes ~n/2 targets of the rows near its ends
    g = synth.path_graph(300, False, 1)
    ups = [("edge", 0, 299, 1), ("edge", 100, 200, 3), ("edge", 50, 250, 1)]
    info = _pair_vs_full(g, ups, "i32", "path closed into a cycle")
    assert info["rows_full"] > 0
    assert info["rows_full"] < info["rows_reaccumulated"]


def test_pair_tie_only_changes():
    # a second route of equal length: path counts grow, no distance drops
    g = synth.cycle_graph(40, False, 1)
    _pair_vs_full(g, [("edge", 0, 20, 20), ("edge", 10, 30, 20)], "i64", "cycle ties")


def test_pair_joining_components():
    a = synth.path_graph(12, False, 2)
    k = 5
    src = np.concatenate([a.src + 12 * i for i in range(k)]).astype(np.int32)
    dst = np.concatenate([a.dst + 12 * i for i in range(k)]).astype(np.int32)
    w = np.concatenate([a.w] * k).astype(np.int64)
    g = synth.Graph(12 * k, False, src, dst, w)
    ups = [("edge", 3, 15, 1), ("edge", 30, 50, 4), ("vertex", 40, [(2, 1, 0), (27, 3, 0)])]
    _pair_vs_full(g, ups, "i32", "joining components")


def test_pair_long_stream_no_drift():
    g = synth.barabasi_albert(400, 3, 1, 30, 8181)
    ups = synth.update_stream(g, 40, 40, 20, 8282, 1, 30, kmin=1, kmax=5)
    a = binding.BCGraph(g)
    rc, done = a.bc_apply_updates(ups)
    assert rc == 0 and done == len(ups), a.last_error()
    compare_full(a, synth.apply_updates(g, ups), label="BA n=400, 100 updates")


def test_pair_option_rejected_on_directed_graphs():
    g = synth.erdos_renyi(20, 60, 1, 5, 3, directed=True)
    a = binding.BCGraph(g)
    with pytest.raises(binding.BCError) as e:
        a.bc_set_option("pair_updates", 1)
    assert e.value.code == binding.BC_ERR_ARG
    a.bc_set_option("pair_updates", 0)


def _two_paths(n_each, w, w_join=None):
    a = synth.path_graph(n_each, False, w)
    src = np.concatenate([a.src, a.src + n_each]).astype(np.int32)
    dst = np.concatenate([a.dst, a.dst + n_each]).astype(np.int32)
    ww = np.concatenate([a.w, a.w]).astype(np.int64)
    return synth.Graph(2 * n_each, False, src, dst, ww)


def test_pair_joining_components_vector_columns():
    # n a multiple of the column vector: joining two components turns INF pairs finite
    g = _two_paths(32, 3)
    ups = [("edge", 5, 40, 2), ("edge", 20, 60, 1), ("vertex", 33, [(1, 2, 0), (31, 4, 0)])]
    _pair_vs_full(g, ups, "i32", "joining, n=64")


def test_pair_large_distances():
    # distances far above 16 bits, int64 state
    g = synth.path_graph(64, False, 30000)
    ups = [("edge", 0, 63, 5), ("edge", 10, 40, 7000)]
    _pair_vs_full(g, ups, "i64", "distances above 16 bits")


def test_pair_heavy_join():
    # small distances until a heavy edge joins the two halves
    g = _two_paths(32, 2)
    ups = [("edge", 3, 7, 1), ("edge", 10, 50, 60000), ("edge", 12, 45, 3), ("edge", 0, 31, 1)]
    _pair_vs_full(g, ups, "i32", "heavy join")
