"""GPU parity: the CUDA path against the CPU oracle on the same seeded inputs.

d and sigma must match bit for bit; delta and BC within |err| <= 1e-9 * max(1, |x|)
(fp64 sums in a different order).  Every check calls the library through the C-ABI.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1311_2147_gb300 import binding, synth
from tests import golden_io
from tests.parity_util import close, compare_full, compare_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


# ------------------------------------------------------------------ static state

@pytest.mark.parametrize("dist", ["i32", "i64"])
@pytest.mark.parametrize("name", golden_io.all_fixtures())
def test_golden_fixtures_incremental(name, dist):
    fx = golden_io.load(name)
    g = golden_io.graph_of(fx)
    bg = binding.BCGraph(g, dist=dist)
    em = synth.EdgeMap.of(g)
    for blk in fx.blocks:
        if blk.update is not None:
            assert bg.bc_apply_edge_update(*blk.update[1:]) == binding.BC_OK, bg.last_error()
            synth.apply_update(em, blk.update)
        d, s, _ = bg.bc_get_rows()
        for a, b, dd, sig in blk.pairs:
            assert (d[a, b] == oracle.INF64) if dd is None else (d[a, b] == dd and s[a, b] == sig)
        bc = bg.bc_get_scores()
        for v, x in blk.bc.items():
            assert abs(bc[v] - float(x)) <= 1e-12, (name, blk.update, v, bc[v], x)
        compare_full(bg, em.to_graph(), label=f"{name} {blk.update}")


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("wmax", [1, 2, 1000])
def test_static_random(directed, wmax):
    for seed in range(6):
        n = [5, 17, 40, 64, 100, 129][seed]
        g = synth.erdos_renyi(n, min(3 * n, n * (n - 1) // 2), 1, wmax, 31 * seed + wmax, directed=directed)
        bg = binding.BCGraph(g, dist="i64" if seed % 2 else "i32")
        compare_full(bg, g, label=f"static n={n}")


def test_static_closed_forms():
    for g, exp in [(synth.star_graph(20), None), (synth.path_graph(33, False), None),
                   (synth.cycle_graph(16, False), None), (synth.complete_graph(12, True), None)]:
        bg = binding.BCGraph(g)
        compare_full(bg, g)
    bc = binding.BCGraph(synth.star_graph(20)).bc_get_scores()
    assert bc[0] == 19 * 18 / 2 and np.all(bc[1:] == 0)


def test_unreachable_and_isolated():
    g = synth.Graph(6, True, np.array([0, 1, 3], np.int32), np.array([1, 2, 4], np.int32),
                    np.array([2, 3, 1], np.int64))
    bg = binding.BCGraph(g)
    compare_full(bg, g)
    assert bg.bc_apply_edge_update(2, 3, 5) == 0
    compare_full(bg, synth.apply_updates(g, [("edge", 2, 3, 5)]))


# ------------------------------------------------------------- incremental

def _stream_check(g, ups, dist, every=1, full_scan=False, label=""):
    bg = binding.BCGraph(g, dist=dist)
    if full_scan:
        bg.bc_set_option("full_scan", 1)
    em = synth.EdgeMap.of(g)
    for i, up in enumerate(ups):
        rc, done = bg.bc_apply_updates([up])
        assert rc == binding.BC_OK and done == 1, (up, bg.last_error())
        synth.apply_update(em, up)
        if (i + 1) % every == 0 or i + 1 == len(ups):
            compare_full(bg, em.to_graph(), label=f"{label} after update {i}: {up}")
    return bg


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("wmax", [2, 5, 1000])
def test_edge_updates_random(directed, wmax):
    g = synth.erdos_renyi(48, 150, 1, wmax, 900 + wmax + directed, directed=directed)
    ups = synth.update_stream(g, 10, 10, 0, 77 + wmax, 1, wmax)
    _stream_check(g, ups, "i32", label=f"edge dir={directed} w<={wmax}")


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("wmax", [3, 100])
def test_vertex_updates_random(directed, wmax):
    g = synth.erdos_renyi(40, 140, 1, wmax, 400 + wmax + directed, directed=directed)
    ups = synth.update_stream(g, 4, 4, 12, 55 + wmax, 1, wmax, kmin=1, kmax=8)
    _stream_check(g, ups, "i64", label=f"vertex dir={directed} w<={wmax}")


@pytest.mark.parametrize("directed", [True, False])
def test_full_scan_option_same_result(directed):
    g = synth.erdos_renyi(36, 110, 1, 4, 123 + directed, directed=directed)
    ups = synth.update_stream(g, 5, 5, 6, 321, 1, 4, kmin=1, kmax=5)
    _stream_check(g, ups, "i32", full_scan=True, label="full scan")


def test_ragged_sizes_tiles():
    # n not a multiple of the vector width, and rows longer than one scan chunk
    for n, dist in [(2051, "i32"), (1029, "i64"), (4099, "i32")]:
        g = synth.erdos_renyi(n, 4 * n, 1, 50, n, directed=(n % 2 == 1))
        ups = synth.update_stream(g, 2, 2, 2, n + 1, 1, 50, kmin=1, kmax=4)
        bg = binding.BCGraph(g, dist=dist)
        rc, done = bg.bc_apply_updates(ups)
        assert rc == 0 and done == len(ups), bg.last_error()
        gg = synth.apply_updates(g, ups)
        rng = synth.Rng(n)
        compare_rows(bg, gg, rng.below(n, 12).tolist() + [0, n - 1], label=f"ragged n={n}")


def test_config_er256_every_update():
    g, ups = synth.workload_er256()
    _stream_check(g, ups, "i64", label="ER n=256")


def test_config_complete_small():
    g, ups = synth.workload_complete2048(n=192, n_updates=40)
    _stream_check(g, ups, "i64", every=5, label="complete n=192")
    st = oracle.brandes(g, want_rows=True, want_bc=False)
    dec = synth.effective_decreases(g, lambda a, b: st.D[a, b], 20, 9)
    _stream_check(g, dec, "i64", every=4, label="complete n=192 effective")


def test_config_ba_small_mixed():
    g, ups = synth.workload_ba16384(n=600, n_updates=40)
    _stream_check(g, ups, "i32", every=8, label="BA n=600")


def test_batch_of_updates_matches_one_by_one():
    g, ups = synth.workload_ba16384(n=300, n_updates=24)
    a = binding.BCGraph(g)
    rc, done = a.bc_apply_updates(ups)
    assert rc == 0 and done == len(ups)
    b = binding.BCGraph(g)
    for up in ups:
        assert b.bc_apply_updates([up])[0] == 0
    for x, y in zip(a.bc_get_rows(), b.bc_get_rows()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.bc_get_scores(), b.bc_get_scores())
    compare_full(a, synth.apply_updates(g, ups))


def test_estar_segment_moves_and_rebuilds():
    # vertex updates with many new edges at low-degree vertices overflow their E*
    # segments: the segments move to the free region, and once that is used up E* is
    # laid out again; results must not depend on either
    for directed in (False, True):
        g = synth.path_graph(160, directed, 3)
        em = synth.EdgeMap.of(g)
        rng = synth.Rng(44 + directed)
        ups = []
        for i in range(40):
            v = int(rng.below(g.n, 1)[0])
            nb = [int(x) for x in rng.below(g.n, 24) if int(x) != v]
            seen, edges = set(), []
            d = i % 2 if directed else 0
            for x in nb:
                exists = em.get(x, v) if d == 0 else em.get(v, x)
                if x in seen or exists is not None:
                    continue
                seen.add(x)
                edges.append((x, 1 + (x + v) % 5, d))
                if len(edges) == 16:
                    break
            up = ("vertex", v, edges)
            synth.apply_update(em, up)
            ups.append(up)
        bg = _stream_check(g, ups, "i32", every=3, label=f"E* moves directed={directed}")
        info = bg.bc_get_info()
        assert info["estar_moves"] > 0 and info["estar_rebuilds"] > 0, info


# ------------------------------------------------------------------ invariants

def test_lemma1_column_u_row_v_unchanged():
    g = synth.erdos_renyi(64, 256, 1, 20, 5, directed=True)
    bg = binding.BCGraph(g)
    d0, s0, _ = bg.bc_get_rows()
    ups = synth.update_stream(g, 6, 6, 0, 6, 1, 20)
    for up in ups:
        _, u, v, w = up
        d0, s0, _ = bg.bc_get_rows()
        assert bg.bc_apply_edge_update(u, v, w) == 0
        d1, s1, _ = bg.bc_get_rows()
        assert np.array_equal(d1[:, u], d0[:, u]) and np.array_equal(s1[:, u], s0[:, u])
        assert np.array_equal(d1[v], d0[v]) and np.array_equal(s1[v], s0[v])
        assert np.all(d1 <= d0)
        eq = d1 == d0
        assert np.all(s1[eq] >= s0[eq])


# ------------------------------------------------------------------ errors

def test_rejections_leave_state_untouched():
    g = synth.erdos_renyi(30, 90, 2, 9, 8, directed=True)
    bg = binding.BCGraph(g)
    before = bg.bc_get_rows(), bg.bc_get_scores()
    a, b, w = int(g.src[0]), int(g.dst[0]), int(g.w[0])
    assert bg.bc_apply_edge_update(a, b, w) == binding.BC_ERR_NOT_INCREMENTAL
    assert bg.bc_apply_edge_update(a, b, w + 5) == binding.BC_ERR_NOT_INCREMENTAL
    assert bg.bc_apply_edge_update(a, a, 1) == binding.BC_ERR_ARG
    assert bg.bc_apply_edge_update(-1, 2, 1) == binding.BC_ERR_ARG
    assert bg.bc_apply_edge_update(1, 2, 0) == binding.BC_ERR_ARG
    assert bg.bc_apply_vertex_update(3, [4, 4], [1, 1], [0, 0]) == binding.BC_ERR_ARG
    after = bg.bc_get_rows(), bg.bc_get_scores()
    for x, y in zip(before[0], after[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(before[1], after[1])


def test_sigma_overflow_detected_at_init():
    with pytest.raises(binding.BCError) as e:
        binding.BCGraph(synth.diamond_chain(64))
    assert e.value.code == binding.BC_ERR_OVERFLOW
    bg = binding.BCGraph(synth.diamond_chain(63))
    d, s, _ = bg.bc_get_rows(0, 1)
    assert int(s[0, 3 * 63]) == 2 ** 63


def test_sigma_overflow_detected_by_update_and_poisons():
    # 64 unit diamonds whose last diamond lacks one arc: sigma(0, 192) = 2^63 fits.
    # Adding the missing arc (191, 192) doubles it to 2^64, which must be reported.
    g = synth.diamond_chain(64)
    keep = ~((g.src == 191) & (g.dst == 192))
    g = synth.Graph(g.n, True, g.src[keep], g.dst[keep], g.w[keep])
    bg = binding.BCGraph(g)
    d, s, _ = bg.bc_get_rows(0, 1)
    assert int(s[0, 192]) == 2 ** 63
    assert bg.bc_apply_edge_update(191, 192, 1) == binding.BC_ERR_OVERFLOW
    assert bg.bc_apply_edge_update(0, 192, 1) == binding.BC_ERR_POISONED
    with pytest.raises(binding.BCError) as e:
        bg.bc_get_scores()
    assert e.value.code == binding.BC_ERR_POISONED


def test_distance_overflow_int32():
    g = synth.path_graph(4, True, w=(1 << 30))
    with pytest.raises(binding.BCError) as e:
        binding.BCGraph(g, dist="i32")
    assert e.value.code == binding.BC_ERR_DIST_OVERFLOW
    bg = binding.BCGraph(g, dist="i64")
    compare_full(bg, g)
