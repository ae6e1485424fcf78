"""The paper's explicit DAG maintenance, as written (a CPU tool; test infrastructure).

The GPU path never stores DAG(s): it re-reads DAG'(s) off the E* superset with the
predicate d'(s,a) + w(a,b) = d'(s,b) (Eq. 1).  The paper instead maintains the DAGs as
edge sets, and this module implements that literally so that its lemmas can be checked
on random graphs against DAGs taken from the definition:

* flag(s,t) (Section 3): WT-changed if d'(s,t) < d(s,t); NUM-changed if d'(s,t) =
  d(s,t) and sigma'_st > sigma_st; UN-changed otherwise.
* Update-DAG (Algorithm 2) for an update of the in-edges E_in(v) of v (one edge (u,v)
  in Section 3; Section 4 step (C) runs it with every edge of E_in(v) in its last
  step): H = the arcs (a,b) of DAG(s) other than the updated ones with flag(s,b) UN- or
  NUM-changed, the arcs (a,b) of DAG(v) with flag(s,b) NUM- or WT-changed, and the
  updated arcs (u_j, v) when flag(s,v) is NUM- or WT-changed.  Lemma 3: H = DAG'(s).
  With several updated arcs, an updated arc that is not tight (d'(s,u_j) + w'_j >
  d'(s,v)) lies on no shortest path; `tight_only` keeps the last step to the tight
  ones (the reading the GPU path's predicate gives), `tight_only=False` is the last
  step word for word.
* Update-Reverse-DAG (Algorithm 5) for DAG_R(s), the shortest-path DAG of s in the
  reversed graph: X = the arcs (a,b) of DAG_R(s) with flag(b,s) UN- or NUM-changed,
  plus R_b for every b != s with flag(b,s) NUM- or WT-changed, where
  R_t = { (a,t) : (t,a) in DAG'(t) and w'(t,a) + d'(a,v) = d'(t,v) }.
  Lemma 5: X = DAG'_R(s).

Distances and path counts come from the oracle's states before and after the update.
"""
from __future__ import annotations

UN, NUM, WT = 0, 1, 2


def flag(d_old, s_old, d_new, s_new):
    if d_new < d_old:
        return WT
    if d_new == d_old and s_new > s_old:
        return NUM
    return UN


def arcs_of(g):
    """(a, b, w) for every arc of g (both arcs of an undirected edge)."""
    out = []
    for a, b, w in zip(g.src.tolist(), g.dst.tolist(), g.w.tolist()):
        out.append((a, b, w))
        if not g.directed:
            out.append((b, a, w))
    return out


def dag(arcs, D, s, inf):
    """DAG(s) from the definition: arcs (a,b) with d(s,a) finite and d(s,a) + w = d(s,b)."""
    return {(a, b) for a, b, w in arcs if D[s][a] != inf and D[s][a] + w == D[s][b]}


def dag_rev(arcs, D, s, inf):
    """DAG_R(s): arcs (a,b) of the reversed graph ((b,a) an arc of G) with d(a,s) finite
    and d(a,s) + w(b,a) = d(b,s)."""
    return {(a, b) for b, a, w in arcs if D[a][s] != inf and D[a][s] + w == D[b][s]}


def update_dag(s, v, dag_s, dag_v, flags_s, updated, d_new, inf, tight_only=True):
    """Algorithm 2 (Update-DAG) for source s after an update of the arcs `updated`
    ((u_j, v, w'_j), all into v).  flags_s[t] = flag(s,t)."""
    upd = {(u, vv) for u, vv, _ in updated}
    H = set()
    for a, b in dag_s:
        if (a, b) not in upd and flags_s[b] in (UN, NUM):
            H.add((a, b))
    for a, b in dag_v:
        if flags_s[b] in (NUM, WT):
            H.add((a, b))
    if flags_s[v] in (NUM, WT):
        for u, vv, w in updated:
            if not tight_only or (d_new[s][u] != inf and d_new[s][u] + w == d_new[s][v]):
                H.add((u, vv))
    return H


def reverse_sets(arcs_new, D_new, v, inf, dags_new):
    """R_t for every t: reversed out-arcs (t,a) of DAG'(t) on a shortest t -> v path."""
    n = len(D_new)
    R = [set() for _ in range(n)]
    for t in range(n):
        for a, b in dags_new[t]:
            if a != t:
                continue
            w = next(x for p, q, x in arcs_new if p == a and q == b)
            if D_new[b][v] != inf and D_new[t][v] != inf and w + D_new[b][v] == D_new[t][v]:
                R[t].add((b, t))
    return R


def update_rdag(s, rdag_s, flags_to_s, R):
    """Algorithm 5 (Update-Reverse-DAG) for source s.  flags_to_s[b] = flag(b,s)."""
    X = set()
    for a, b in rdag_s:
        if flags_to_s[b] in (UN, NUM):
            X.add((a, b))
    for b in range(len(R)):
        if b != s and flags_to_s[b] in (NUM, WT):
            X |= R[b]
    return X
