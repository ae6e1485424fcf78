"""Pins of the exact-rational oracle for real weights (oracle/real.py), no GPU.

* brute-force path enumeration (oracle/brute.py) on small graphs with rational weights,
  including exact ties between sums of dyadic weights;
* on integer weights it equals the C oracle (oracle/bc_oracle.c) exactly in d and
  sigma (an independent implementation of the same definition);
* scaling every weight by a power of two scales d and leaves sigma, delta and BC as
  they are;
* ties are decided on the exact sums of the doubles: 0.25 + 0.5 ties with 0.75, while
  0.1 + 0.2 does not tie with 0.3 (as doubles the sum is the larger);
* closed form: the star's centre scores (n-1)(n-2)/2 whatever the (equal) weight.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import brute, oracle
from oracle.real import brandes_real
from paper_1311_2147_gb300 import synth


class _G:
    def __init__(self, n, directed, src, dst, w):
        self.n, self.directed = n, directed
        self.src = np.asarray(src, dtype=np.int64)
        self.dst = np.asarray(dst, dtype=np.int64)
        self.w = np.asarray([Fraction(float(x)) for x in w], dtype=object)


@pytest.mark.parametrize("directed", [True, False])
def test_real_oracle_matches_brute_force(directed):
    rng = np.random.default_rng(11 if directed else 12)
    for trial in range(40):
        n = int(rng.integers(2, 7))
        pairs = [(a, b) for a in range(n) for b in range(n) if a != b and (directed or a < b)]
        k = int(rng.integers(1, len(pairs) + 1))
        sel = rng.choice(len(pairs), size=k, replace=False)
        src = [pairs[i][0] for i in sel]
        dst = [pairs[i][1] for i in sel]
        # dyadic weights from a small set: exact ties are frequent
        w = [float(x) for x in rng.choice([0.25, 0.5, 0.75, 1.0, 1.25], size=k)]
        st = brandes_real(n, directed, src, dst, w)
        d, sigma, delta, bc = brute.betweenness(_G(n, directed, src, dst, w))
        for s in range(n):
            for t in range(n):
                assert st.D[s][t] == d[s][t]
                assert st.SIG[s][t] == sigma[s][t]
                if s != t:
                    assert st.DEL[s][t] == delta[s][t]
        assert st.BC == bc


def test_real_oracle_equals_integer_oracle():
    for directed in (True, False):
        g = synth.erdos_renyi(40, 120, 1, 5, 77 + directed, directed=directed)
        st = brandes_real(g.n, g.directed, g.src, g.dst, g.w.astype(np.float64))
        ref = oracle.brandes(g)
        for s in range(g.n):
            for t in range(g.n):
                exp = None if ref.D[s, t] == oracle.INF64 else int(ref.D[s, t])
                assert st.D[s][t] == exp
                assert st.SIG[s][t] == int(ref.SIG[s, t])
        assert np.allclose([float(x) for x in st.BC], ref.BC, rtol=1e-12, atol=1e-12)


def test_power_of_two_scaling():
    g = synth.erdos_renyi(30, 90, 1, 9, 5, directed=False)
    a = brandes_real(g.n, False, g.src, g.dst, g.w.astype(np.float64))
    b = brandes_real(g.n, False, g.src, g.dst, g.w.astype(np.float64) * 2.0 ** -10)
    assert a.SIG == b.SIG and a.DEL == b.DEL and a.BC == b.BC
    assert all(b.D[s][t] == (None if a.D[s][t] is None else a.D[s][t] / 1024) for s in range(g.n) for t in range(g.n))


def test_ties_are_exact_sums_of_doubles():
    # 0 -> 1 -> 2 against 0 -> 2
    tie = brandes_real(3, True, [0, 1, 0], [1, 2, 2], [0.25, 0.5, 0.75])
    assert tie.SIG[0][2] == 2 and tie.BC[1] == Fraction(1, 2)
    no_tie = brandes_real(3, True, [0, 1, 0], [1, 2, 2], [0.1, 0.2, 0.3])
    assert Fraction(0.1) + Fraction(0.2) > Fraction(0.3)
    assert no_tie.SIG[0][2] == 1 and no_tie.BC[1] == 0 and no_tie.D[0][2] == Fraction(0.3)


def test_star_closed_form_with_real_weight():
    n = 9
    st = brandes_real(n, False, [0] * (n - 1), list(range(1, n)), [0.3] * (n - 1))
    assert st.BC[0] == Fraction((n - 1) * (n - 2), 2) and all(b == 0 for b in st.BC[1:])
