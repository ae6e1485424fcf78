"""GPU parity at the workloads' own sizes, against the oracle recomputed from scratch.

* BA n = 16384 (8 edges per new vertex, w ~ U[1,100]) with its whole 1024-update stream
  (edge updates and vertex updates on up to 16 edges), default options -- the DAG-walk
  pair corrections are on at this size.  At eight checkpoints the full BC vector is
  compared with static Brandes on the current graph, and at least 64 rows bit for bit
  (d, sigma) and within the tolerance (delta): the rows that the checkpoint's update
  changed most (counted on the device state just before and after it), rows at both
  ends of the vertex range, the highest-degree vertices and seeded random rows.  This
  checks the drift of the float-float dependency rows and the fixed-point BC words over
  the whole stream.
* Complete directed n = 2048 (w ~ U{1..n^2}) with its 256 weight decreases (nearly all
  no-ops), then the variant with effective decreases (w' <= d(u,v)): the full state
  at checkpoints and at the end.

d and sigma must match exactly; delta and BC within |err| <= 1e-9 * max(1, |x|).
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1311_2147_gb300 import binding, synth
from tests.parity_util import close, compare_full

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


def _rows(bg, rows, want=("d", "sigma")):
    d = np.empty((len(rows), bg.n), np.int64)
    s = np.empty((len(rows), bg.n), np.uint64)
    for i, r in enumerate(rows):
        dd, ss, _ = bg.bc_get_rows(int(r), 1, want=want)
        d[i], s[i] = dd[0], ss[0]
    return d, s


def _candidates(em, up, rng, n):
    """Rows likely to change most under ``up``: its endpoints and their neighbours, plus
    seeded random rows."""
    ends = [up[1], up[2]] if up[0] == "edge" else [up[1]] + [x for x, _, _ in up[2]]
    cand = set(int(x) for x in ends)
    for x in ends:
        nb = sorted(em.adj[x])
        cand.update(nb[:96])
    cand.update(int(x) for x in rng.below(n, 256).tolist())
    return sorted(cand)


def test_ba16384_whole_stream_against_oracle():
    g, ups = synth.workload_ba16384()
    n = g.n
    assert len(ups) == 1024
    bg = binding.BCGraph(g, dist="i32")
    em = synth.EdgeMap.of(g)
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=n)
    hubs = np.argsort(-deg, kind="stable")[:8].tolist()
    ends = [0, 1, 2, 3, n - 4, n - 3, n - 2, n - 1]
    checkpoints = set(range(128, 1025, 128))
    rng = synth.Rng(0xC3)
    checked = 0
    for i, up in enumerate(ups):
        last = (i + 1) in checkpoints
        if last:
            cand = _candidates(em, up, rng, n)
            d0, s0 = _rows(bg, cand)
        rc, done = bg.bc_apply_updates([up])
        assert rc == 0 and done == 1, (i, up, bg.last_error())
        synth.apply_update(em, up)
        if not last:
            continue
        d1, s1 = _rows(bg, cand)
        changed = ((d1 != d0) | (s1 != s0)).sum(axis=1)
        top = [cand[j] for j in np.argsort(-changed, kind="stable")[:32] if changed[j] > 0]
        rand = rng.below(n, 24).tolist()
        rows = sorted(set(top) | set(hubs) | set(ends) | set(int(x) for x in rand))
        assert len(rows) >= 64 or len(top) < 32
        gg = em.to_graph()
        st = oracle.brandes(gg, sources=np.asarray(rows, np.int32), want_bc=False)
        for k, r in enumerate(rows):
            d, s, dl = bg.bc_get_rows(r, 1)
            assert np.array_equal(d[0], st.D[k]), f"update {i + 1}: row {r} distances differ"
            assert np.array_equal(s[0], st.SIG[k]), f"update {i + 1}: row {r} path counts differ"
            ok, worst = close(dl[0], st.DEL[k])
            assert ok, f"update {i + 1}: row {r} dependencies differ ({worst:.3g} x tol)"
        full = oracle.brandes(gg, want_rows=False)
        ok, worst = close(bg.bc_get_scores(), full.BC)
        assert ok, f"update {i + 1}: BC differs ({worst:.3g} x tol)"
        checked += 1
    assert checked == 8
    info = bg.bc_get_info()
    assert info["walk_pairs"] > 0 and info["pair_rows"] > 0 and info["rows_full"] > 0
    bg.close()


def _complete_stream(g, ups, every, label):
    bg = binding.BCGraph(g, dist="i64")
    em = synth.EdgeMap.of(g)
    for i, up in enumerate(ups):
        rc, done = bg.bc_apply_updates([up])
        assert rc == 0 and done == 1, (label, i, up, bg.last_error())
        synth.apply_update(em, up)
        if (i + 1) % every == 0 or i + 1 == len(ups):
            compare_full(bg, em.to_graph(), label=f"{label}, after update {i + 1}")
    info = bg.bc_get_info()
    bg.close()
    return info


def test_complete2048_decreases_against_oracle():
    g, ups = synth.workload_complete2048()
    assert g.n == 2048 and g.m == 2048 * 2047 and len(ups) == 256
    info = _complete_stream(g, ups, 64, "complete n=2048")
    assert info["noop_updates"] >= len(ups) // 2


def test_complete2048_effective_decreases_against_oracle():
    g, _ = synth.workload_complete2048()
    st = oracle.brandes(g, want_rows=True, want_bc=False)
    dec = synth.effective_decreases(g, lambda a, b: st.D[a, b], 64, 0xEFFE)
    assert len(dec) >= 48
    info = _complete_stream(g, dec, 16, "complete n=2048, effective decreases")
    assert info["rows_reaccumulated"] > 0
