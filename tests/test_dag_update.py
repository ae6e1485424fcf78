"""The paper's explicit DAG maintenance (oracle/dag_update.py: Algorithm 2 and
Algorithm 5 as written) against DAGs taken from the definition after the update, on
random directed graphs: Lemma 3 (Update-DAG gives DAG'(s)) for single-edge updates and
for updates of several in-edges of v, and Lemma 5 (Update-Reverse-DAG gives DAG'_R(s)).
Distances and path counts before and after come from the oracle."""
import numpy as np
import pytest

from oracle import dag_update as du
from oracle import oracle
from paper_1311_2147_gb300 import synth

INF = oracle.INF64


def _states(g, ups):
    g2 = synth.apply_updates(g, ups)
    a, b = oracle.brandes(g), oracle.brandes(g2)
    return g2, a.D.tolist(), a.SIG.tolist(), b.D.tolist(), b.SIG.tolist()


def _random_in_update(g, rng, kmax):
    """An update of 1..kmax arcs into one vertex v: decreases of existing arcs or new arcs."""
    em = synth.EdgeMap.of(g)
    n = g.n
    v = int(rng.integers(0, n))
    k = int(rng.integers(1, kmax + 1))
    cands = [x for x in range(n) if x != v]
    rng.shuffle(cands)
    out = []
    for x in cands[:k]:
        cur = em.get(x, v)
        if cur is None:
            out.append((x, v, int(rng.integers(1, 20))))
        elif cur > 1:
            out.append((x, v, int(rng.integers(1, cur))))
    return v, out


def _check(g, v, updated, tight_only=True):
    ups = [("vertex", v, [(x, w, 0) for x, _, w in updated])] if len(updated) > 1 else \
        [("edge", updated[0][0], v, updated[0][2])]
    g2, D, S, D2, S2 = _states(g, ups)
    arcs, arcs2 = du.arcs_of(g), du.arcs_of(g2)
    n = g.n
    dags = [du.dag(arcs, D, s, INF) for s in range(n)]
    dags2 = [du.dag(arcs2, D2, s, INF) for s in range(n)]
    ok3 = True
    for s in range(n):
        fl = [du.flag(D[s][t], S[s][t], D2[s][t], S2[s][t]) for t in range(n)]
        H = du.update_dag(s, v, dags[s], dags[v], fl, updated, D2, INF, tight_only=tight_only)
        ok3 &= H == dags2[s]
    R = du.reverse_sets(arcs2, D2, v, INF, dags2)
    ok5 = True
    for s in range(n):
        flr = [du.flag(D[b][s], S[b][s], D2[b][s], S2[b][s]) for b in range(n)]
        X = du.update_rdag(s, du.dag_rev(arcs, D, s, INF), flr, R)
        ok5 &= X == du.dag_rev(arcs2, D2, s, INF)
    return ok3, ok5


@pytest.mark.parametrize("wmax", [1, 3, 20])
def test_lemma3_and_lemma5_single_edge(wmax):
    rng = np.random.default_rng(100 + wmax)
    for trial in range(25):
        g = synth.erdos_renyi(12, 30, 1, wmax, 1000 * wmax + trial, directed=True)
        v, upd = _random_in_update(g, rng, 1)
        if not upd:
            continue
        ok3, ok5 = _check(g, v, upd, tight_only=False)   # one arc: the last step word for word
        assert ok3, (trial, v, upd)
        assert ok5, (trial, v, upd)


@pytest.mark.parametrize("wmax", [2, 9])
def test_lemma3_and_lemma5_several_in_edges(wmax):
    rng = np.random.default_rng(200 + wmax)
    for trial in range(25):
        g = synth.erdos_renyi(12, 30, 1, wmax, 2000 * wmax + trial, directed=True)
        v, upd = _random_in_update(g, rng, 4)
        if not upd:
            continue
        ok3, ok5 = _check(g, v, upd, tight_only=True)
        assert ok3, (trial, v, upd)
        assert ok5, (trial, v, upd)


def test_last_step_needs_tight_arcs_with_several_in_edges():
    # two new arcs into v = 2: (0,2) with weight 1 and (1,2) with weight 5, and 0 -> 1
    # with weight 1: from s = 0, only (0,2) is on a shortest path to 2, although
    # flag(0,2) is WT-changed; the last step word for word would add (1,2) as well
    g = synth.Graph(4, True, np.array([0, 2], np.int32), np.array([1, 3], np.int32), np.array([1, 1], np.int64))
    ok3, _ = _check(g, 2, [(0, 2, 1), (1, 2, 5)], tight_only=False)
    assert not ok3
    ok3, ok5 = _check(g, 2, [(0, 2, 1), (1, 2, 5)], tight_only=True)
    assert ok3 and ok5
