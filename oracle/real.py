"""Static betweenness with real weights in exact rational arithmetic (test infrastructure).

Section 2 of the paper allows positive real edge weights.  Here a weight is the double
as given, taken as the exact rational it denotes (fractions.Fraction(w)), and every path
length is the exact sum of those rationals, so two paths tie exactly when their sums
are equal.  What is computed is the plain static definition, from scratch:

* d(s,t): Dijkstra from every source s over exact rationals (Section 2, Algorithm 7);
* sigma_ss = 1, sigma_st = sum of sigma_sa over the predecessors a of t on shortest
  paths, P_s(t) = { a : (a,t) in E, d(s,a) + w(a,t) = d(s,t) } (Eq. 1), taken over the
  vertices in order of distance;
* delta_s.(v) by Algorithm 1: vertices in non-increasing distance, each w pushing
  sigma_sv / sigma_sw * (1 + delta_s.(w)) to every v in P_s(w) (Eq. 4), in exact
  rationals; BC(v) = sum over s != v of delta_s.(v) (Eq. 3);
* undirected graphs run on G_D (Section 3) with BC halved (each unordered pair once).

Only the tests use this module; it is pure Python and meant for graphs of a few hundred
vertices.  It shares no code with the CUDA library or its binding.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass
from fractions import Fraction


@dataclass
class RealState:
    D: list      # D[s][t]: Fraction, or None when t is unreachable from s
    SIG: list    # SIG[s][t]: int
    DEL: list    # DEL[s][t]: Fraction (0 on the diagonal)
    BC: list     # BC[v]: Fraction


def _adjacency(n, directed, src, dst, w):
    adj = [[] for _ in range(n)]
    for a, b, x in zip(src, dst, w):
        q = Fraction(float(x))
        adj[int(a)].append((int(b), q))
        if not directed:
            adj[int(b)].append((int(a), q))
    return adj


def brandes_real(n, directed, src, dst, w) -> RealState:
    adj = _adjacency(n, directed, src, dst, w)
    D = [[None] * n for _ in range(n)]
    SIG = [[0] * n for _ in range(n)]
    DEL = [[Fraction(0)] * n for _ in range(n)]
    BC = [Fraction(0)] * n
    for s in range(n):
        dist = [None] * n
        sigma = [0] * n
        preds = [[] for _ in range(n)]
        order = []
        done = [False] * n
        dist[s] = Fraction(0)
        sigma[s] = 1
        heap = [(Fraction(0), s)]
        while heap:
            dx, x = heapq.heappop(heap)
            if done[x] or dx != dist[x]:
                continue
            done[x] = True
            order.append(x)
            for y, wt in adj[x]:
                nd = dx + wt
                if dist[y] is None or nd < dist[y]:
                    dist[y] = nd
                    sigma[y] = sigma[x]
                    preds[y] = [x]
                    heapq.heappush(heap, (nd, y))
                elif nd == dist[y] and not done[y]:
                    sigma[y] += sigma[x]
                    preds[y].append(x)
        delta = [Fraction(0)] * n
        for x in reversed(order):
            for a in preds[x]:
                delta[a] += Fraction(sigma[a], sigma[x]) * (1 + delta[x])
            if x != s:
                BC[x] += delta[x]
        D[s] = dist
        SIG[s] = sigma
        DEL[s] = [Fraction(0) if t == s else delta[t] for t in range(n)]
    if not directed:
        BC = [b / 2 for b in BC]
    return RealState(D, SIG, DEL, BC)
