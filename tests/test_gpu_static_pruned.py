"""GPU parity of the static computation with the all-pairs searches restricted to E*
(Algorithm 6 step 1: arcs found outside E* are left out of the later searches) against
the search over every arc and against the oracle: d and sigma bit for bit, delta and BC
within |err| <= 1e-9 * max(1, |x|)."""
import numpy as np
import pytest

from oracle import oracle
from paper_1311_2147_gb300 import binding, synth
from tests.parity_util import close, compare_full, compare_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


def _pruned_vs_all(g, dist):
    a = binding.BCGraph(g, dist=dist)
    b = binding.BCGraph(g, dist=dist, static_all_arcs=True)
    da, sa, la = a.bc_get_rows()
    db, sb, lb = b.bc_get_rows()
    assert np.array_equal(da, db) and np.array_equal(sa, sb)
    ok, worst = close(la, lb)
    assert ok, f"dependencies differ ({worst:.3g} x tol)"
    assert a.bc_get_info()["estar_arcs"] == b.bc_get_info()["estar_arcs"]
    return a


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("wmax", [1, 3, 1000])
def test_pruned_static_small(directed, wmax):
    g = synth.erdos_renyi(150, 700, 1, wmax, 4100 + wmax, directed=directed)
    a = _pruned_vs_all(g, "i32" if wmax < 1000 else "i64")
    compare_full(a, g, label=f"ER n=150 w<={wmax} directed={directed}")


def test_pruned_static_complete_graph():
    # E* is a small part of the arcs: most arcs are pruned early
    g = synth.complete_directed(300, 1, 300 * 300, 4242)
    a = _pruned_vs_all(g, "i64")
    assert a.bc_get_info()["estar_arcs"] < g.m // 4
    compare_full(a, g, label="complete n=300")


def test_pruned_static_components_and_sources():
    # two components and vertices without in- or out-arcs
    g = synth.Graph(9, True, np.array([0, 1, 2, 5, 6, 0], np.int32), np.array([1, 2, 3, 6, 7, 3], np.int32),
                    np.array([1, 1, 1, 2, 2, 3], np.int64))
    compare_full(_pruned_vs_all(g, "i32"), g, label="components")


def test_pruned_static_ba_4099():
    g = synth.barabasi_albert(4099, 8, 1, 100, 4099)
    a = _pruned_vs_all(g, "i32")
    rng = synth.Rng(4099)
    compare_rows(a, g, rng.below(g.n, 40).tolist() + [0, 1, 2, 4098], bc_too=True, label="BA n=4099")
