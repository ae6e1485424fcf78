"""Batches: many graphs updated in one CUDA graph launch per call.

Each graph's state after a batch must be bit-identical to the same updates applied to it
alone (same device functions, fixed summation orders), and must match the oracle.
"""
import numpy as np
import pytest

from paper_1311_2147_gb300 import binding, synth
from tests.parity_util import compare_full, compare_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


def _family(count, seed, nlo=40, nhi=400, vertex=True):
    rng = synth.Rng(seed)
    ns = synth.log_uniform_n(rng, nlo, nhi, count)
    out = []
    for i, n in enumerate(ns):
        if i % 2 == 0:
            g = synth.erdos_renyi_degree(n, 4, 1, 30, seed + i)
        else:
            g = synth.barabasi_albert(max(n, 9), 3, 1, 30, seed + i)
        nv = 2 if vertex else 0
        ups = synth.update_stream(g, 2, 2, nv, seed + 1000 + i, 1, 30, kmin=1, kmax=4)
        out.append((g, ups))
    return out


@pytest.mark.parametrize("pairs", [1, 0], ids=["pair-corrections", "full-reaccumulation"])
def test_batch_equals_alone_and_oracle(pairs):
    # undirected graphs: pair corrections (the default) or every changed row
    # re-accumulated, the same option on the handles alone and in the batch
    fam = _family(12, 77)
    alone = []
    for g, ups in fam:
        a = binding.BCGraph(g)
        if not g.directed:
            a.bc_set_option("pair_updates", pairs)
        rc, done = a.bc_apply_updates(ups)
        assert rc == 0 and done == len(ups)
        alone.append(a)
    mixed = [binding.BCGraph(g) for g, _ in fam]
    for m in mixed:
        if not m.directed:
            m.bc_set_option("pair_updates", pairs)
    batch = binding.BCBatch(mixed)
    rc, done = batch.bc_batch_apply([ups for _, ups in fam])
    assert rc == 0, batch.last_error()
    assert done.tolist() == [len(u) for _, u in fam]
    for (g, ups), a, m in zip(fam, alone, mixed):
        for x, y in zip(a.bc_get_rows(), m.bc_get_rows()):
            assert np.array_equal(x, y)
        assert np.array_equal(a.bc_get_scores(), m.bc_get_scores())
        compare_full(m, synth.apply_updates(g, ups), label=f"batch n={g.n}")
    if pairs:
        info = [m.bc_get_info() for (g, _), m in zip(fam, mixed) if not g.directed]
        assert sum(i["pair_rows"] for i in info) > 0


def test_batch_uneven_counts_and_repeat_calls():
    fam = _family(9, 5, nlo=64, nhi=300)
    graphs = [binding.BCGraph(g) for g, _ in fam]
    batch = binding.BCBatch(graphs)
    # first call: graph i gets i % 4 updates; second call: the rest
    first = [ups[: i % 4] for i, (_, ups) in enumerate(fam)]
    second = [ups[i % 4:] for i, (_, ups) in enumerate(fam)]
    for part in (first, second):
        rc, done = batch.bc_batch_apply(part)
        assert rc == 0, batch.last_error()
        assert done.tolist() == [len(p) for p in part]
    for (g, ups), m in zip(fam, graphs):
        compare_full(m, synth.apply_updates(g, ups), label=f"two calls n={g.n}")


def test_batch_stops_a_graph_at_its_invalid_update():
    fam = _family(4, 91, nlo=30, nhi=80, vertex=False)
    graphs = [binding.BCGraph(g) for g, _ in fam]
    batch = binding.BCBatch(graphs)
    lists = [list(ups) for _, ups in fam]
    bad = lists[1][1]
    lists[1][1] = ("edge", bad[1], bad[1], 1)       # self-loop: rejected
    rc, done = batch.bc_batch_apply(lists)
    assert rc == binding.BC_ERR_ARG
    assert done[1] == 1 and done[0] == len(lists[0])
    compare_full(graphs[1], synth.apply_updates(fam[1][0], lists[1][:1]))
    compare_full(graphs[0], synth.apply_updates(fam[0][0], lists[0]))


def test_batch_tiles_do_not_change_results():
    fam = _family(6, 33, nlo=50, nhi=200)
    outs = []
    for tiles in ([4, 8, 8, 0], [1, 2, 1, 1], [4, 8, 8, 0, 1, 0], [4, 8, 8, 0, 8, 1], [2, 4, 4, 1, 2, 1],
                  [4, 8, 8, 0, 4, 0, 256], [2, 8, 16, 1, 2, 1, 256], [4, 8, 8, 0, 4, 0, 128]):
        graphs = [binding.BCGraph(g) for g, _ in fam]
        batch = binding.BCBatch(graphs)
        batch.bc_batch_set_tiles(tiles)
        rc, _ = batch.bc_batch_apply([ups for _, ups in fam])
        assert rc == 0
        outs.append([m.bc_get_scores() for m in graphs])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)


def test_batch_config_shape_sample():
    # the 512-graph workload's distribution on a few graphs, 8 edge updates each
    fam = synth.workload_batch(count=16, nlo=64, nhi=700)
    graphs = [binding.BCGraph(g) for g, _ in fam]
    batch = binding.BCBatch(graphs)
    rc, done = batch.bc_batch_apply([ups for _, ups in fam])
    assert rc == 0 and all(d == 8 for d in done)
    for (g, ups), m in zip(fam, graphs):
        gg = synth.apply_updates(g, ups)
        compare_rows(m, gg, [0, g.n // 2, g.n - 1], label=f"batch workload n={g.n}")


def test_batch_pair_classes_int32():
    # int32 distances: the batched column test runs once per class of columns per
    # thread (8 where n is a multiple of 8, 4 where of 4, else 1); graphs of every class
    # in one batch, each bit for bit its result alone and matching the oracle
    ns = [64, 100, 101, 136, 77, 200]
    fam = []
    for i, n in enumerate(ns):
        g = synth.barabasi_albert(n, 3, 1, 30, 500 + i)
        ups = synth.update_stream(g, 3, 3, 2, 600 + i, 1, 30, kmin=1, kmax=4)
        fam.append((g, ups))
    alone = []
    for g, ups in fam:
        a = binding.BCGraph(g, dist="i32")
        rc, done = a.bc_apply_updates(ups)
        assert rc == 0 and done == len(ups)
        alone.append(a)
    mixed = [binding.BCGraph(g, dist="i32") for g, _ in fam]
    batch = binding.BCBatch(mixed)
    rc, done = batch.bc_batch_apply([ups for _, ups in fam])
    assert rc == 0, batch.last_error()
    for (g, ups), a, m in zip(fam, alone, mixed):
        for x, y in zip(a.bc_get_rows(), m.bc_get_rows()):
            assert np.array_equal(x, y), f"n={g.n}"
        assert np.array_equal(a.bc_get_scores(), m.bc_get_scores()), f"n={g.n}"
        compare_full(m, synth.apply_updates(g, ups), label=f"int32 batch n={g.n}")
    assert sum(m.bc_get_info()["pair_rows"] for m in mixed) > 0
