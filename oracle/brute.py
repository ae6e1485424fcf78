"""Brute-force betweenness by path enumeration (test infrastructure, graphs with n <= 8).

Straight from the definitions of Section 2 of the paper:
* every simple s->t path is enumerated by depth-first search (with positive weights
  every shortest path is simple);
* d(s,t) is the least path weight, sigma_st the number of paths of that weight;
* sigma_st(v) counts the shortest s-t paths with v as an inner vertex (Eq. 2),
  delta_st(v) = sigma_st(v) / sigma_st;
* delta_s.(v) = sum over t not in {s, v} of delta_st(v); BC(v) is Eq. 3, the sum over
  s != v, t != v of delta_st(v), in exact rationals.
Undirected graphs count each unordered pair once (BC halved), as the oracle does.
"""
from __future__ import annotations

from fractions import Fraction


def _adjacency(g):
    adj = [[] for _ in range(g.n)]
    for a, b, w in zip(g.src.tolist(), g.dst.tolist(), g.w.tolist()):
        adj[a].append((b, w))
        if not g.directed:
            adj[b].append((a, w))
    return adj


def all_pairs(g):
    """Return (d, sigma, through) where d[s][t] is None if t is unreachable,
    sigma[s][t] is an int and through[s][t][v] = sigma_st(v)."""
    n = g.n
    adj = _adjacency(g)
    d = [[None] * n for _ in range(n)]
    sigma = [[0] * n for _ in range(n)]
    through = [[[0] * n for _ in range(n)] for _ in range(n)]
    for s in range(n):
        best: dict = {}
        paths: dict = {}

        def dfs(x, weight, visited, seq):
            t = x
            if t not in best or weight < best[t]:
                best[t] = weight
                paths[t] = [list(seq)]
            elif weight == best[t]:
                paths[t].append(list(seq))
            for y, w in adj[x]:
                if y not in visited:
                    visited.add(y)
                    seq.append(y)
                    dfs(y, weight + w, visited, seq)
                    seq.pop()
                    visited.remove(y)

        dfs(s, 0, {s}, [s])
        for t, wt in best.items():
            d[s][t] = wt
            sigma[s][t] = len(paths[t])
            for p in paths[t]:
                for v in p[1:-1]:
                    through[s][t][v] += 1
    return d, sigma, through


def betweenness(g):
    """Exact (d, sigma, delta, bc): delta[s][v] and bc[v] are Fractions."""
    n = g.n
    d, sigma, through = all_pairs(g)
    delta = [[Fraction(0)] * n for _ in range(n)]
    bc = [Fraction(0)] * n
    for s in range(n):
        for t in range(n):
            if t == s or d[s][t] is None:
                continue
            for v in range(n):
                if v in (s, t) or through[s][t][v] == 0:
                    continue
                dep = Fraction(through[s][t][v], sigma[s][t])
                delta[s][v] += dep
                bc[v] += dep
    if not g.directed:
        bc = [x / 2 for x in bc]
    return d, sigma, delta, bc
