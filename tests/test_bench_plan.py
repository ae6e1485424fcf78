"""bench.py's step plan: every valid --steps / --warmup fits the configured update stream
(fewer updates per step, or the stream continued), with the full-pass updates kept."""
import pytest

import bench


@pytest.mark.parametrize("W,K", [(3, 8), (5, 20), (3, 1), (10, 50), (3, 600), (5, 2000)])
@pytest.mark.parametrize("per_step", [1, 22, 32, 64])
def test_plan_fits_stream(W, K, per_step):
    U, extra = bench.plan_steps(1024, per_step, W, K)
    assert 1 <= U <= per_step
    assert (W + 2 * K) * U + bench.SCAN_UPDATES <= 1024 + extra
    if extra:
        assert U == 1          # the stream is continued only when one update per step does not fit
    else:
        # the largest U that fits (or the requested one)
        assert U == per_step or (W + 2 * K) * (U + 1) + bench.SCAN_UPDATES > 1024


def test_driver_command_uses_22_updates_per_step():
    assert bench.plan_steps(1024, 32, 5, 20) == (22, 0)


def test_default_command_keeps_32():
    assert bench.plan_steps(1024, 32, 3, 8) == (32, 0)


def test_stream_continuation_is_valid_and_seeded():
    from paper_1311_2147_gb300 import synth
    g = synth.barabasi_albert(200, 3, 1, 100, 5)
    ups = synth.update_stream(g, 4, 4, 4, 6, 1, 100)
    a = bench.extend_stream("ba16384", g, ups, 10, seed=77)
    b = bench.extend_stream("ba16384", g, ups, 10, seed=77)
    assert a == b and len(a) == 22 and a[:12] == ups
    em = synth.EdgeMap.of(g)
    for up in a:   # every update lowers a weight or adds an edge
        edges = [(up[1], up[2], up[3])] if up[0] == "edge" else [
            (up[1], x, w) if d else (x, up[1], w) for x, w, d in up[2]]
        for u, v, w in edges:
            cur = em.get(u, v)
            assert u != v and w >= 1 and (cur is None or w < cur)
        synth.apply_update(em, up)
