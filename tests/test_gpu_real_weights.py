"""GPU parity with real (fp64) weights (bc_init_static_f64 and the _f64 updates)
against the exact-rational oracle (oracle/real.py): distances equal exactly (the
device's integers times the handle's unit 2^E), path counts bit for bit, dependencies
and BC within |err| <= 1e-9 * max(1, |x|); and the rejections that keep sums exact."""
from fractions import Fraction

import numpy as np
import pytest

from oracle.real import brandes_real
from paper_1311_2147_gb300 import binding, synth
from tests.parity_util import TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()


def _check(h, n, directed, src, dst, w, label):
    st = brandes_real(n, directed, src, dst, w)
    e = h.bc_get_weight_unit()
    unit = Fraction(2) ** e
    d, s, dl = h.bc_get_rows()
    for a in range(n):
        for b in range(n):
            exp = st.D[a][b]
            if exp is None:
                assert s[a, b] == 0, (label, a, b)
            else:
                assert Fraction(int(d[a, b])) * unit == exp, (label, a, b, int(d[a, b]), exp)
                assert int(s[a, b]) == st.SIG[a][b], (label, a, b)
            x = float(st.DEL[a][b])
            assert abs(dl[a, b] - x) <= TOL * max(1.0, abs(x)), (label, a, b)
    bc = h.bc_get_scores()
    for v in range(n):
        x = float(st.BC[v])
        assert abs(bc[v] - x) <= TOL * max(1.0, abs(x)), (label, v, bc[v], x)


def _graph(n, m, directed, weights, seed):
    g = synth.erdos_renyi(n, m, 1, 1, seed, directed=directed)
    rng = np.random.default_rng(seed)
    return g.src.astype(np.int32), g.dst.astype(np.int32), rng.choice(weights, size=g.m)


@pytest.mark.parametrize("directed", [True, False])
@pytest.mark.parametrize("dist", ["i32", "i64"])
def test_dyadic_weights_static_and_updates(directed, dist):
    n = 90
    src, dst, w = _graph(n, 260, directed, np.arange(1, 33) / 8.0, 31 + directed)
    h = binding.BCGraphReal(n, directed, src, dst, w, dist=dist)
    assert h.bc_get_weight_unit() == -3
    _check(h, n, directed, src, dst, w, "static")
    em = {}
    for a, b, x in zip(src.tolist(), dst.tolist(), w.tolist()):
        em[(a, b) if directed or a < b else (b, a)] = x
    rng = np.random.default_rng(7)
    for step in range(10):
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        key = (a, b) if directed or a < b else (b, a)
        cur = em.get(key)
        new = 0.125 * int(rng.integers(1, 8)) if cur is None else max(0.125, cur - 0.125 * int(rng.integers(1, 4)))
        if cur is not None and new >= cur:
            continue
        assert h.bc_apply_edge_update_f64(a, b, new) == binding.BC_OK, h.last_error()
        em[key] = new
    # a vertex update on two edges of vertex 5
    dirs = [0, 1] if directed else None

    def key_of(x, dd):
        return ((x, 5) if dd == 0 else (5, x)) if directed else (min(x, 5), max(x, 5))
    nb = [x for x in range(n) if x != 5 and key_of(x, 0) not in em and key_of(x, 1) not in em][:2]
    ws = [0.125, 0.25]
    assert h.bc_apply_vertex_update_f64(5, nb, ws, dirs) == binding.BC_OK, h.last_error()
    for x, wv, dd in zip(nb, ws, dirs or [0, 0]):
        em[key_of(x, dd)] = wv
    keys = sorted(em)
    _check(h, n, directed, [k[0] for k in keys], [k[1] for k in keys], [em[k] for k in keys], "updated")


def test_arbitrary_doubles_ties_on_exact_sums():
    # weights 1.1, 2.2, 3.3 (as doubles 1.1 + 2.2 != 3.3) and 0.75 = 0.25 + 0.5 (exact)
    n = 6
    src = [0, 1, 0, 2, 3, 2, 4]
    dst = [1, 2, 2, 3, 5, 4, 5]
    w = [1.1, 2.2, 3.3, 0.25, 0.5, 0.5, 0.25]
    h = binding.BCGraphReal(n, True, src, dst, w)
    _check(h, n, True, src, dst, w, "exact sums")
    d, s, _ = h.bc_get_rows()
    assert int(s[0, 2]) == 1 and int(s[2, 5]) == 2


def test_random_doubles_in_one_octave_range():
    n = 100
    src, dst, _ = _graph(n, 300, False, [1.0], 99)
    w = 1.0 + 3.0 * np.random.default_rng(99).random(src.shape[0])   # full 53-bit mantissas in [1, 4)
    h = binding.BCGraphReal(n, False, src, dst, w)
    _check(h, n, False, src, dst, w, "random doubles")


def test_rejections_keep_the_state():
    src, dst, w = [0, 1, 2], [1, 2, 3], [0.25, 0.5, 0.75]
    h = binding.BCGraphReal(4, True, src, dst, w)
    before = h.bc_get_scores()
    assert h.bc_apply_edge_update_f64(0, 3, 0.125) == binding.BC_ERR_ARG    # finer than the unit 2^-2
    assert h.bc_apply_edge_update_f64(0, 3, float("nan")) == binding.BC_ERR_ARG
    assert h.bc_apply_edge_update_f64(0, 3, -1.0) == binding.BC_ERR_ARG
    assert h.bc_apply_edge_update_f64(1, 2, 0.75) == binding.BC_ERR_NOT_INCREMENTAL
    assert np.array_equal(h.bc_get_scores(), before)
    with pytest.raises(binding.BCError):   # 2^-60 next to 1.0 with int32 distances
        binding.BCGraphReal(4, True, src, dst, [1.0, 2.0 ** -60, 1.0], dist="i32")
    with pytest.raises(binding.BCError):
        binding.BCGraphReal(4, True, src, dst, [1.0, 0.0, 1.0])
    g = binding.BCGraph(synth.path_graph(4, True, 1))
    assert g.lib.bc_apply_edge_update_f64(g.h, 0, 2, 1.0) == binding.BC_ERR_ARG   # not a real-weight handle
