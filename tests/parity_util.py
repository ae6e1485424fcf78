"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on the same
seeded inputs and compare (d and sigma bit-exact, delta and BC within
|err| <= 1e-9 * max(1, |x|))."""
from __future__ import annotations

import numpy as np

from oracle import oracle
from paper_1311_2147_gb300 import synth

TOL = 1e-9


def close(got, exp, tol=TOL):
    got = np.asarray(got, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    err = np.abs(got - exp)
    lim = tol * np.maximum(1.0, np.abs(exp))
    return bool(np.all(err <= lim)), float(np.max(err / lim)) if err.size else 0.0


def compare_full(bg, g, label="", nthreads=None):
    """Compare every row and BC of the handle bg with a static oracle run on graph g."""
    st = oracle.brandes(g, nthreads=nthreads)
    d, s, dl = bg.bc_get_rows()
    assert np.array_equal(d, st.D), f"{label}: distances differ at {np.argwhere(d != st.D)[:5].tolist()}"
    assert np.array_equal(s, st.SIG), f"{label}: path counts differ at {np.argwhere(s != st.SIG)[:5].tolist()}"
    ok, worst = close(dl, st.DEL)
    assert ok, f"{label}: dependencies differ (worst {worst:.3g} x tol)"
    bc = bg.bc_get_scores()
    ok, worst = close(bc, st.BC)
    assert ok, f"{label}: BC differs (worst {worst:.3g} x tol)"
    return st


def compare_rows(bg, g, sources, bc_too=True, label="", nthreads=None):
    """Compare sampled rows (and BC when asked) with the oracle run from those sources."""
    srcs = np.asarray(sorted(set(int(x) for x in sources)), dtype=np.int32)
    st = oracle.brandes(g, sources=srcs, want_bc=False, nthreads=nthreads)
    for i, s in enumerate(srcs.tolist()):
        d, sg, dl = bg.bc_get_rows(s, 1)
        assert np.array_equal(d[0], st.D[i]), f"{label}: row {s} distances differ"
        assert np.array_equal(sg[0], st.SIG[i]), f"{label}: row {s} path counts differ"
        ok, worst = close(dl[0], st.DEL[i])
        assert ok, f"{label}: row {s} dependencies differ ({worst:.3g} x tol)"
    if bc_too:
        full = oracle.brandes(g, want_rows=False, nthreads=nthreads)
        ok, worst = close(bg.bc_get_scores(), full.BC)
        assert ok, f"{label}: BC differs ({worst:.3g} x tol)"


def dist_for(g) -> str:
    return "i64"
