"""Pins for the CPU oracle (no GPU).

The oracle recomputes static Brandes on the current graph.  It is pinned here against
things other than itself:
* brute-force path enumeration with exact rationals on small graphs (Section 2
  definitions, Eq. 1-3), with tiny weight ranges so that ties and sigma > 1 are common;
* hand-derived fixtures under tests/golden/, including incremental steps;
* closed forms (star, path, cycles, complete graph, diamond chains);
* incremental closed forms (star plus a leaf-leaf edge, path closed into a cycle);
* invariants (Eq. 1 recurrence of sigma, triangle inequality, hop-count identity).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import brute, oracle
from paper_1311_2147_gb300 import synth
from tests import golden_io

INF = oracle.INF64


def _rel_close(a, b, tol=1e-12):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= tol * np.maximum(1.0, np.abs(b)))


def _check_against_brute(g):
    st = oracle.brandes(g, nthreads=2)
    d, sigma, delta, bc = brute.betweenness(g)
    n = g.n
    for s in range(n):
        for t in range(n):
            if d[s][t] is None:
                assert st.D[s, t] == INF and st.SIG[s, t] == 0, (s, t)
            else:
                assert st.D[s, t] == d[s][t], (s, t)
                assert int(st.SIG[s, t]) == sigma[s][t], (s, t)
        exp = [0.0 if v == s else float(delta[s][v]) for v in range(n)]
        assert _rel_close(st.DEL[s], exp), (s, st.DEL[s], exp)
    assert _rel_close(st.BC, [float(x) for x in bc]), (st.BC, bc)


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("wmax", [1, 2, 3, 10])
def test_brute_force_random(directed, wmax):
    count = 0
    for seed in range(40):
        n = 2 + seed % 6
        p = (0.3, 0.5, 0.8)[seed % 3]
        g = synth.random_small(n, p, 1, wmax, 1000 * wmax + seed + (7 if directed else 0), directed)
        _check_against_brute(g)
        count += 1
    assert count == 40


def test_brute_force_n8():
    for seed in range(4):
        g = synth.random_small(8, 0.45, 1, 2, 99 + seed, seed % 2 == 0)
        _check_against_brute(g)


@pytest.mark.parametrize("name", golden_io.all_fixtures())
def test_golden_fixture(name):
    fx = golden_io.load(name)
    g = golden_io.graph_of(fx)
    em = synth.EdgeMap.of(g)
    for blk in fx.blocks:
        if blk.update is not None:
            synth.apply_update(em, blk.update)
        st = oracle.brandes(em.to_graph(), nthreads=1)
        for s, t, d, sig in blk.pairs:
            if d is None:
                assert st.D[s, t] == INF and st.SIG[s, t] == 0
            else:
                assert st.D[s, t] == d and int(st.SIG[s, t]) == sig, (name, blk.update, s, t)
        for v, x in blk.bc.items():
            assert abs(st.BC[v] - float(x)) <= 1e-12, (name, blk.update, v, st.BC[v], x)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [3, 4, 7, 12, 33])
def test_star(n):
    st = oracle.brandes(synth.star_graph(n))
    assert st.BC[0] == (n - 1) * (n - 2) / 2
    assert np.all(st.BC[1:] == 0)


@pytest.mark.parametrize("n", [2, 5, 10, 31])
@pytest.mark.parametrize("directed", [True, False])
def test_path(n, directed):
    st = oracle.brandes(synth.path_graph(n, directed))
    assert np.array_equal(st.BC, np.array([i * (n - 1 - i) for i in range(n)], float))


@pytest.mark.parametrize("n", [3, 4, 5, 8, 9, 16, 17])
def test_undirected_cycle(n):
    st = oracle.brandes(synth.cycle_graph(n, False))
    exp = (n - 1) * (n - 3) / 8 if n % 2 else (n - 2) ** 2 / 8
    assert np.allclose(st.BC, exp, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [3, 6, 11])
def test_directed_cycle(n):
    st = oracle.brandes(synth.cycle_graph(n, True))
    assert np.all(st.BC == (n - 1) * (n - 2) / 2)


@pytest.mark.parametrize("directed", [True, False])
def test_complete_equal_weights(directed):
    st = oracle.brandes(synth.complete_graph(9, directed))
    assert np.all(st.BC == 0)
    off = ~np.eye(9, dtype=bool)
    assert np.all(st.SIG[off] == 1) and np.all(st.D[off] == 1)


@pytest.mark.parametrize("k", [1, 5, 20, 63])
def test_diamond_chain_sigma(k):
    g = synth.diamond_chain(k)
    st = oracle.brandes(g)
    assert int(st.SIG[0, 3 * k]) == 2 ** k
    assert st.D[0, 3 * k] == 2 * k


def test_diamond_chain_overflow():
    with pytest.raises(oracle.OracleError) as e:
        oracle.brandes(synth.diamond_chain(64))
    assert e.value.code == oracle.ERR_OVERFLOW


def test_distance_overflow():
    g = synth.path_graph(4, True, w=(1 << 62))
    with pytest.raises(oracle.OracleError) as e:
        oracle.brandes(g)
    assert e.value.code == oracle.ERR_DIST_OVERFLOW


def test_bad_graphs_rejected():
    for src, dst, w in [([0], [0], [1]), ([0], [5], [1]), ([0], [1], [0]), ([0, 0], [1, 1], [1, 2])]:
        g = synth.Graph(3, True, np.array(src, np.int32), np.array(dst, np.int32), np.array(w, np.int64))
        with pytest.raises(oracle.OracleError) as e:
            oracle.brandes(g)
        assert e.value.code == oracle.ERR_ARG
    g = synth.Graph(3, False, np.array([0, 1], np.int32), np.array([1, 0], np.int32), np.array([1, 1], np.int64))
    with pytest.raises(oracle.OracleError):
        oracle.brandes(g)


# ------------------------------------------------------ incremental closed forms

@pytest.mark.parametrize("wnew,drop", [(1, 1.0), (2, 0.5), (3, 0.0)])
def test_star_plus_leaf_edge(wnew, drop):
    n = 9
    g = synth.star_graph(n)
    before = oracle.brandes(g).BC
    after = oracle.brandes(synth.apply_updates(g, [("edge", 3, 6, wnew)])).BC
    assert before[0] - after[0] == drop
    assert np.all(after[1:] == 0)


@pytest.mark.parametrize("n", [6, 7])
def test_path_closed_into_cycle(n):
    g = synth.path_graph(n, False)
    st = oracle.brandes(synth.apply_updates(g, [("edge", 0, n - 1, 1)]))
    exp = (n - 1) * (n - 3) / 8 if n % 2 else (n - 2) ** 2 / 8
    assert np.allclose(st.BC, exp, atol=1e-12)


# ------------------------------------------------------------------ invariants

def _arcs(g):
    src, dst, w = g.src.astype(np.int64), g.dst.astype(np.int64), g.w
    if not g.directed:
        src, dst, w = np.concatenate([src, dst]), np.concatenate([dst, src]), np.concatenate([w, w])
    return src, dst, w


@pytest.mark.parametrize("directed", [True, False])
def test_invariants_random(directed):
    g = synth.erdos_renyi(120, 700, 1, 4, 4242 + directed, directed=directed)
    st = oracle.brandes(g)
    n = g.n
    a, b, w = _arcs(g)
    D, SIG, DEL = st.D, st.SIG, st.DEL
    assert np.all(np.diag(D) == 0) and np.all(np.diag(SIG) == 1)
    for s in range(0, n, 7):
        da, db = D[s, a], D[s, b]
        fin = da != INF
        # triangle inequality over E
        assert np.all(db[fin] <= da[fin] + w[fin])
        # Eq. 1 recurrence: sigma_st = sum over predecessors
        pred = fin & (da + np.where(fin, w, 0) == db)
        acc = np.zeros(n, dtype=object)
        for x, y in zip(a[pred].tolist(), b[pred].tolist()):
            acc[y] += int(SIG[s, x])
        for t in range(n):
            if t != s and D[s, t] != INF:
                assert acc[t] == int(SIG[s, t])
        # hop-count identity: sum_v delta_s.(v) = sum_t (H_st / sigma_st - 1),
        # H by the forward recurrence H_st = sum over preds (H_sa + sigma_sa)
        order = np.argsort(np.where(D[s] == INF, np.iinfo(np.int64).max, D[s]), kind="stable")
        H = [Fraction(0)] * n
        preds = [[] for _ in range(n)]
        for x, y in zip(a[pred].tolist(), b[pred].tolist()):
            preds[y].append(x)
        total = Fraction(0)
        for t in order.tolist():
            if D[s, t] == INF or t == s:
                continue
            H[t] = sum((H[x] + int(SIG[s, x]) for x in preds[t]), Fraction(0))
            total += H[t] / int(SIG[s, t]) - 1
        assert abs(DEL[s].sum() - float(total)) <= 1e-9 * max(1.0, float(total))
    assert np.all(st.BC >= 0)
    if directed:
        indeg = np.bincount(b, minlength=n)
        outdeg = np.bincount(a, minlength=n)
        assert np.all(st.BC[(indeg == 0) | (outdeg == 0)] == 0)


def test_sources_subset_matches_full():
    g = synth.erdos_renyi(80, 400, 1, 5, 77, directed=True)
    full = oracle.brandes(g, nthreads=3)
    srcs = np.array([5, 0, 79, 33], np.int32)
    part = oracle.brandes(g, sources=srcs, nthreads=2)
    assert np.array_equal(part.D, full.D[srcs])
    assert np.array_equal(part.SIG, full.SIG[srcs])
    assert np.array_equal(part.DEL, full.DEL[srcs])
    exp = full.DEL[srcs].sum(axis=0)
    assert np.allclose(part.BC, exp, rtol=1e-13, atol=1e-12)


def test_thread_count_does_not_change_rows():
    g = synth.barabasi_albert(200, 3, 1, 3, 5)
    a = oracle.brandes(g, nthreads=1)
    b = oracle.brandes(g, nthreads=5)
    assert np.array_equal(a.D, b.D) and np.array_equal(a.SIG, b.SIG) and np.array_equal(a.DEL, b.DEL)
    assert np.allclose(a.BC, b.BC, rtol=1e-13)
