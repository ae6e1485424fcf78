"""Seeded synthetic graphs and incremental-update streams.

This module only draws inputs: it holds none of the betweenness arithmetic, so both
the CPU oracle tests and the CUDA path can take their graphs and update streams from
it without sharing any part of the method.

Randomness comes from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based generator:
the i-th draw of a stream with seed ``s`` is ``mix(s + (i + 1) * GAMMA)``.  Every
draw is an exact 64-bit integer operation, so a seed gives the same graph on any
machine.

Graph conventions (the paper's Section 2 setting: positive integer weights):
* a graph is ``Graph(n, directed, src, dst, w)`` with int32 endpoints and int64
  weights; an undirected graph lists each edge {a, b} once;
* graphs are simple: no self-loops, no repeated (directed) pair / unordered pair.

Update conventions (the paper's Section 1 definition of an incremental update):
* ``("edge", u, v, w)``: add edge (u, v) with weight w, or lower its weight to w;
* ``("vertex", v, [(x, w, dir), ...])``: an incremental update of a subset of the
  edges incident to v; ``dir`` 0 is the edge (x, v), 1 is the edge (v, x); for an
  undirected graph ``dir`` is ignored and the edge is {v, x}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


class Rng:
    """Counter-based splitmix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed & M64
        self.ctr = 0

    def u64(self, k: int) -> np.ndarray:
        i = np.arange(self.ctr + 1, self.ctr + 1 + k, dtype=np.uint64)
        self.ctr += k
        with np.errstate(over="ignore"):
            x = np.uint64(self.seed) + i * np.uint64(GAMMA)
        return _mix(x)

    def below(self, bound: int, k: int) -> np.ndarray:
        """k integers uniform in [0, bound) by 32x32 multiply-shift (bound < 2**32)."""
        assert 0 < bound < (1 << 32)
        r = self.u64(k) >> np.uint64(32)
        with np.errstate(over="ignore"):
            return ((r * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)

    def uniform_int(self, lo: int, hi: int, k: int) -> np.ndarray:
        """k integers uniform in [lo, hi]."""
        return lo + self.below(hi - lo + 1, k)

    def unit(self, k: int) -> np.ndarray:
        """k doubles uniform in [0, 1) from the top 53 bits."""
        return (self.u64(k) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def one(self, bound: int) -> int:
        return int(self.below(bound, 1)[0])


def sub_seed(seed: int, index: int) -> int:
    """Derive the seed of item ``index`` of a family (graph number, config number)."""
    return int(_mix(np.array([(seed + (index + 1) * GAMMA) & M64], dtype=np.uint64))[0])


@dataclass
class Graph:
    n: int
    directed: bool
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def copy(self) -> "Graph":
        return Graph(self.n, self.directed, self.src.copy(), self.dst.copy(), self.w.copy())

    def arrays(self):
        return (np.ascontiguousarray(self.src, dtype=np.int32),
                np.ascontiguousarray(self.dst, dtype=np.int32),
                np.ascontiguousarray(self.w, dtype=np.int64))


def _graph(n, directed, pairs, weights) -> Graph:
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return Graph(n, directed, pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32),
                 np.asarray(weights, dtype=np.int64))


# ---------------------------------------------------------------------------
# graph families
# ---------------------------------------------------------------------------

def erdos_renyi(n: int, m: int, wlo: int, whi: int, seed: int, directed: bool = True) -> Graph:
    """G(n, m): m distinct pairs (ordered if directed), no self-loops, weights U[wlo, whi]."""
    rng = Rng(seed)
    cap = n * (n - 1) if directed else n * (n - 1) // 2
    assert m <= cap
    chosen: list[int] = []
    seen: set[int] = set()
    while len(chosen) < m:
        k = max(64, 2 * (m - len(chosen)))
        a = rng.below(n, k)
        b = rng.below(n, k)
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            if not directed and x > y:
                x, y = y, x
            key = x * n + y
            if key in seen:
                continue
            seen.add(key)
            chosen.append(key)
            if len(chosen) == m:
                break
    keys = np.array(chosen, dtype=np.int64)
    w = rng.uniform_int(wlo, whi, m)
    return Graph(n, directed, (keys // n).astype(np.int32), (keys % n).astype(np.int32), w)


def erdos_renyi_degree(n: int, avg_out_degree: int, wlo: int, whi: int, seed: int) -> Graph:
    """Directed ER with m = avg_out_degree * n (capped at the complete graph)."""
    m = min(avg_out_degree * n, n * (n - 1))
    return erdos_renyi(n, m, wlo, whi, seed, directed=True)


def barabasi_albert(n: int, k: int, wlo: int, whi: int, seed: int) -> Graph:
    """Undirected preferential attachment: a (k+1)-clique, then each new vertex joins
    k distinct earlier vertices drawn from the repeated-endpoint list."""
    rng = Rng(seed)
    n0 = k + 1
    assert n >= n0
    edges: list[tuple[int, int]] = [(a, b) for a in range(n0) for b in range(a + 1, n0)]
    ends: list[int] = [x for e in edges for x in e]
    block = rng.below(1 << 31, 4096).tolist()
    bi = 0
    for x in range(n0, n):
        targets: list[int] = []
        while len(targets) < k:
            if bi == len(block):
                block = rng.below(1 << 31, 4096).tolist()
                bi = 0
            r = block[bi]
            bi += 1
            t = ends[(r * len(ends)) >> 31]
            if t not in targets:
                targets.append(t)
        for t in targets:
            edges.append((t, x))
            ends.append(t)
            ends.append(x)
    w = rng.uniform_int(wlo, whi, len(edges))
    return _graph(n, False, edges, w)


def complete_directed(n: int, wlo: int, whi: int, seed: int) -> Graph:
    """Every ordered pair (a, b), a != b, with weight U[wlo, whi]."""
    rng = Rng(seed)
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mask = a != b
    src = a[mask].astype(np.int32)
    dst = b[mask].astype(np.int32)
    w = rng.uniform_int(wlo, whi, src.shape[0])
    return Graph(n, True, src, dst, w)


def random_small(n: int, p: float, wlo: int, whi: int, seed: int, directed: bool) -> Graph:
    """Each possible pair present with probability p (brute-force test graphs)."""
    rng = Rng(seed)
    pairs = [(a, b) for a in range(n) for b in range(n)
             if a != b and (directed or a < b)]
    keep = rng.unit(len(pairs)) < p
    chosen = [pq for pq, kp in zip(pairs, keep.tolist()) if kp]
    w = rng.uniform_int(wlo, whi, len(chosen))
    return _graph(n, directed, chosen if chosen else np.zeros((0, 2)), w)


def path_graph(n: int, directed: bool = False, w: int = 1) -> Graph:
    return _graph(n, directed, [(i, i + 1) for i in range(n - 1)], [w] * (n - 1))


def star_graph(n: int, w: int = 1) -> Graph:
    """Undirected star with centre 0 and leaves 1..n-1."""
    return _graph(n, False, [(0, i) for i in range(1, n)], [w] * (n - 1))


def cycle_graph(n: int, directed: bool = False, w: int = 1) -> Graph:
    return _graph(n, directed, [(i, (i + 1) % n) for i in range(n)], [w] * n)


def complete_graph(n: int, directed: bool = False, w: int = 1) -> Graph:
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b and (directed or a < b)]
    return _graph(n, directed, pairs, [w] * len(pairs))


def diamond_chain(k: int) -> Graph:
    """k unit diamonds in series: hubs h_0..h_k; diamond i joins h_i to h_{i+1} through
    two middle vertices.  Directed, so the hub-to-hub path count is exactly 2**k."""
    n = 3 * k + 1
    pairs = []
    for i in range(k):
        h, a, b, nxt = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        pairs += [(h, a), (h, b), (a, nxt), (b, nxt)]
    return _graph(n, True, pairs, [1] * len(pairs))


# ---------------------------------------------------------------------------
# update streams
# ---------------------------------------------------------------------------

@dataclass
class EdgeMap:
    """Host view of the current weights, used to draw valid incremental updates."""
    n: int
    directed: bool
    w: dict = field(default_factory=dict)
    adj: list = field(default_factory=list)
    keys: list = field(default_factory=list)   # keys in insertion order (for sampling)
    radj: list = field(default_factory=list)   # in-neighbours (directed graphs)

    @classmethod
    def of(cls, g: Graph) -> "EdgeMap":
        em = cls(g.n, g.directed, {}, [set() for _ in range(g.n)], [], [set() for _ in range(g.n)])
        for a, b, x in zip(g.src.tolist(), g.dst.tolist(), g.w.tolist()):
            em.set(a, b, x)
        return em

    def key(self, a, b):
        if not self.directed and a > b:
            a, b = b, a
        return (a, b)

    def get(self, a, b):
        return self.w.get(self.key(a, b))

    def set(self, a, b, x):
        k = self.key(a, b)
        if k not in self.w:
            self.adj[a].add(b)
            if not self.directed:
                self.adj[b].add(a)
            else:
                self.radj[b].add(a)
            self.keys.append(k)
        self.w[k] = x

    def to_graph(self) -> Graph:
        items = sorted(self.w.items())
        pairs = [k for k, _ in items]
        return _graph(self.n, self.directed, pairs if pairs else np.zeros((0, 2)),
                      [x for _, x in items])


def apply_update(em: EdgeMap, up) -> None:
    """Apply one update to the host weight map (graph edit only, no BC arithmetic)."""
    if up[0] == "edge":
        _, u, v, w = up
        em.set(u, v, w)
    else:
        _, v, edges = up
        for x, w, d in edges:
            if em.directed and d == 0:
                em.set(x, v, w)
            else:
                em.set(v, x, w)


def apply_updates(g: Graph, ups) -> Graph:
    em = EdgeMap.of(g)
    for up in ups:
        apply_update(em, up)
    return em.to_graph()


def _draw_edge_update(em: EdgeMap, rng: Rng, new_edge: bool, wlo: int, whi: int):
    n = em.n
    if new_edge:
        for _ in range(10000):
            u, v = rng.one(n), rng.one(n)
            if u != v and em.get(u, v) is None:
                return ("edge", u, v, int(rng.uniform_int(wlo, whi, 1)[0]))
        raise RuntimeError("no free pair for a new edge")
    # a uniformly drawn existing edge of weight >= 2 (rejection sampling)
    for _ in range(100000):
        a, b = em.keys[rng.one(len(em.keys))]
        if em.w[(a, b)] >= 2:
            break
    else:
        raise RuntimeError("no edge with weight >= 2 to decrease")
    if not em.directed and rng.one(2):
        a, b = b, a
    old = em.w[em.key(a, b)]
    return ("edge", a, b, int(rng.uniform_int(1, old - 1, 1)[0]))


def _draw_vertex_update(em: EdgeMap, rng: Rng, kmin: int, kmax: int, wlo: int, whi: int):
    n = em.n
    v = rng.one(n)
    k = int(rng.uniform_int(kmin, kmax, 1)[0])
    used: set = set()
    edges = []
    for _ in range(k):
        for _try in range(64):
            d = rng.one(2) if em.directed else 1
            decrease = rng.one(2) == 0
            if decrease:
                nbrs = sorted(x for x in (em.adj[v] if (d == 1 or not em.directed) else em.radj[v])
                              if (x, d) not in used)
                cand = [x for x in nbrs
                        if (em.get(v, x) if d == 1 else em.get(x, v)) is not None
                        and (em.get(v, x) if d == 1 else em.get(x, v)) >= 2]
                if not cand:
                    continue
                x = cand[rng.one(len(cand))]
                old = em.get(v, x) if d == 1 else em.get(x, v)
                edges.append((x, int(rng.uniform_int(1, old - 1, 1)[0]), d))
            else:
                x = rng.one(n)
                cur = em.get(v, x) if d == 1 else em.get(x, v)
                if x == v or cur is not None or (x, d) in used:
                    continue
                edges.append((x, int(rng.uniform_int(wlo, whi, 1)[0]), d))
            used.add((x, d))
            if not em.directed:
                used.add((x, 1 - d))
            break
    return ("vertex", v, edges)


def update_stream(g: Graph, n_edge_new: int, n_edge_dec: int, n_vertex: int, seed: int,
                  wlo: int, whi: int, kmin: int = 2, kmax: int = 16) -> list:
    """A shuffled stream of valid incremental updates, each drawn against the graph as
    left by the updates before it."""
    rng = Rng(seed)
    kinds = ["new"] * n_edge_new + ["dec"] * n_edge_dec + ["vtx"] * n_vertex
    order = np.argsort(rng.u64(len(kinds)), kind="stable")
    kinds = [kinds[i] for i in order.tolist()]
    em = EdgeMap.of(g)
    ups = []
    for kd in kinds:
        if kd == "vtx":
            up = _draw_vertex_update(em, rng, kmin, kmax, wlo, whi)
        else:
            up = _draw_edge_update(em, rng, kd == "new", wlo, whi)
        apply_update(em, up)
        ups.append(up)
    return ups


def effective_decreases(g: Graph, dist_uv, count: int, seed: int) -> list:
    """Weight decreases of random existing edges to U[1, d(u,v)] where ``dist_uv(u, v)``
    supplies the current distance (used for the 'effective decreases' variant of the
    complete-graph workload)."""
    rng = Rng(seed)
    em = EdgeMap.of(g)
    ups = []
    keys = sorted(em.w.keys())
    for _ in range(count):
        a, b = keys[rng.one(len(keys))]
        cap = min(em.w[(a, b)] - 1, int(dist_uv(a, b)))
        if cap < 1:
            continue
        up = ("edge", a, b, int(rng.uniform_int(1, cap, 1)[0]))
        apply_update(em, up)
        ups.append(up)
    return ups


# ---------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------

BASE_SEED = 0x13112147


def workload_er256(seed: int = BASE_SEED + 0):
    """Directed G(256, 2048), w ~ U[1,1000]; 16 updates: 8 new edges, 8 decreases."""
    g = erdos_renyi(256, 2048, 1, 1000, sub_seed(seed, 0), directed=True)
    ups = update_stream(g, 8, 8, 0, sub_seed(seed, 1), 1, 1000)
    return g, ups


def workload_complete2048(seed: int = BASE_SEED + 1, n: int = 2048, n_updates: int = 256):
    """Complete directed graph, w ~ U{1..n^2}; n_updates random weight decreases."""
    g = complete_directed(n, 1, n * n, sub_seed(seed, 0))
    ups = update_stream(g, 0, n_updates, 0, sub_seed(seed, 1), 1, n * n)
    return g, ups


def workload_ba16384(seed: int = BASE_SEED + 2, n: int = 16384, n_updates: int = 1024):
    """Undirected BA(n, 8), w ~ U[1,100]; half edge updates (half new, half decreases),
    half vertex updates on 2..16 incident edges."""
    g = barabasi_albert(n, 8, 1, 100, sub_seed(seed, 0))
    ne = n_updates // 2
    ups = update_stream(g, ne // 2, ne - ne // 2, n_updates - ne, sub_seed(seed, 1), 1, 100)
    return g, ups


def log_uniform_n(rng: Rng, lo: int, hi: int, k: int) -> list:
    u = rng.unit(k)
    return [int(math.floor(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo))))) for x in u]


def workload_batch(seed: int = BASE_SEED + 3, count: int = 512, nlo: int = 64, nhi: int = 2048,
                   n_updates: int = 8, rounds: int = 1):
    """count graphs, n log-uniform in [nlo, nhi]; even index directed ER (out-degree 8),
    odd index undirected BA(8); w ~ U[1,1000]; n_updates edge updates each."""
    rng = Rng(seed)
    ns = log_uniform_n(rng, nlo, nhi, count)
    out = []
    for i, n in enumerate(ns):
        gs = sub_seed(seed, 2 * i + 10)
        if i % 2 == 0:
            g = erdos_renyi_degree(n, 8, 1, 1000, gs)
        else:
            g = barabasi_albert(max(n, 9), 8, 1, 1000, gs)
        total = n_updates * rounds
        half = total // 2
        ups = update_stream(g, half, total - half, 0, sub_seed(seed, 2 * i + 11), 1, 1000)
        out.append((g, ups))
    return out
