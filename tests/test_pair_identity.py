"""The pair-correction identity behind the "pair_updates" option, checked on the oracle
(no GPU).

The dependency of s on x is the sum over targets t of the pair dependencies
delta_st(x) = sigma_sx sigma_xt / sigma_st over x on shortest s-t paths (Section 2).
Under decreases, a pair whose distance and path count are both unchanged keeps its
shortest paths, so

    delta'_s(x) = delta_s(x) + sum over changed pairs (s,t) of [delta'_st(x) - delta_st(x)].

These tests evaluate both sides from oracle states before and after update streams on
undirected graphs (where column t equals row t), so a reading of the rule that drops
pairs with only new tied paths, or mixes old and new rows, fails here.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1311_2147_gb300 import synth

INF = oracle.INF64


def _pair_dep(D, SIG, s):
    """P[t, x] = delta_st(x) for row s, from the definition."""
    n = D.shape[0]
    P = np.zeros((n, n))
    ds = D[s]
    for t in range(n):
        if t == s or D[s, t] == INF or SIG[s, t] == 0:
            continue
        on = (ds != INF) & (D[:, t] != INF)
        on &= np.where(on, ds + np.where(on, D[:, t], 0), -1) == D[s, t]
        on[s] = on[t] = False
        P[t, on] = SIG[s, on].astype(np.float64) * SIG[on, t].astype(np.float64) / float(SIG[s, t])
    return P


def _check_stream(g, ups):
    before = oracle.brandes(g, nthreads=2)
    after_g = synth.apply_updates(g, ups)
    after = oracle.brandes(after_g, nthreads=2)
    n = g.n
    changed = (before.D != after.D) | (before.SIG != after.SIG)
    tie_only = (before.D == after.D) & (before.SIG != after.SIG)
    n_rows = 0
    for s in range(n):
        P0 = _pair_dep(before.D, before.SIG, s)
        P1 = _pair_dep(after.D, after.SIG, s)
        # the definition reproduces the oracle's dependencies
        assert np.allclose(P0.sum(axis=0), before.DEL[s], rtol=1e-12, atol=1e-12)
        assert np.allclose(P1.sum(axis=0), after.DEL[s], rtol=1e-12, atol=1e-12)
        # unchanged pairs keep every pair dependency
        keep = ~changed[s]
        assert np.allclose(P0[keep], P1[keep], rtol=0, atol=1e-12)
        corr = (P1[changed[s]] - P0[changed[s]]).sum(axis=0)
        assert np.allclose(before.DEL[s] + corr, after.DEL[s], rtol=1e-12, atol=1e-12)
        n_rows += int(changed[s].any())
    return n_rows, int(tie_only.sum())


@pytest.mark.parametrize("wmax", [2, 3, 50])
def test_identity_edge_and_vertex_updates(wmax):
    g = synth.erdos_renyi(36, 90, 1, wmax, 4100 + wmax, directed=False)
    ups = synth.update_stream(g, 3, 3, 2, 4200 + wmax, 1, wmax, kmin=1, kmax=4)
    rows, ties = _check_stream(g, ups)
    assert rows > 0


def test_identity_with_tie_only_changes():
    # unit weights: inserted edges mostly add tied paths without lowering distances
    g = synth.cycle_graph(12, False, 1)
    ups = [("edge", 0, 6, 6)]          # a second 6-hop route between 0 and 6
    rows, ties = _check_stream(g, ups)
    assert ties > 0 and rows > 0


def test_identity_joining_components():
    a = synth.path_graph(8, False, 2)
    # two disjoint paths 0..7 and 8..15, joined by one edge: pairs go from INF to finite
    src = np.concatenate([a.src, a.src + 8]).astype(np.int32)
    dst = np.concatenate([a.dst, a.dst + 8]).astype(np.int32)
    w = np.concatenate([a.w, a.w]).astype(np.int64)
    g = synth.Graph(16, False, src, dst, w)
    _check_stream(g, [("edge", 3, 12, 1)])


def test_dropping_tie_only_pairs_breaks_the_identity():
    """Planted mistake: correcting only the pairs whose distance dropped misses the
    pairs that gained tied paths."""
    g = synth.cycle_graph(12, False, 1)
    g2 = synth.apply_updates(g, [("edge", 0, 6, 6)])
    before, after = oracle.brandes(g, nthreads=1), oracle.brandes(g2, nthreads=1)
    lowered = before.D != after.D
    bad = 0
    for s in range(g.n):
        P0 = _pair_dep(before.D, before.SIG, s)
        P1 = _pair_dep(after.D, after.SIG, s)
        corr = (P1[lowered[s]] - P0[lowered[s]]).sum(axis=0)
        bad += int(not np.allclose(before.DEL[s] + corr, after.DEL[s], atol=1e-9))
    assert bad > 0
