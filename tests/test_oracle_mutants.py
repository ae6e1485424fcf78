"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of bc_oracle.c (a dropped term, a swapped
ratio, a wrong index, a missing halving, an unweighted relaxation, a wrong sigma
seed), builds it with the host compiler into a temporary library, and checks that
the pins of test_oracle.py -- brute force, the hand-derived fixtures and the closed
forms -- reject it.  The mistakes are planted in the oracle only, on the CPU.
"""
import os
import subprocess

import numpy as np
import pytest

from oracle import brute, oracle
from paper_1311_2147_gb300 import synth
from tests import golden_io

MUTANTS = {
    "drop_one_plus": ("(1.0 + ws->delta[x])", "(ws->delta[x])"),
    "swap_sigma_ratio": ("(double)ws->sigma[v] / (double)ws->sigma[x]",
                         "(double)ws->sigma[x] / (double)ws->sigma[v]"),
    "no_undirected_halving": ("BC[v] *= 0.5;", "BC[v] *= 1.0;"),
    "bc_counts_source": ("if (x != s && bc) bc[x]", "if (bc) bc[x]"),
    "unweighted_relax": ("int64_t nd = ws->d[a] + wt;", "int64_t nd = ws->d[a] + 1;"),
    "sigma_seed_two": ("ws->sigma[s] = 1;", "ws->sigma[s] = 2;"),
    "delta_wrong_index": ("ws->delta[v] += ((double)", "ws->delta[x] += ((double)"),
    "pred_strict_less": ("ws->d[a] + g->in_w[e] == ws->d[t]", "ws->d[a] + g->in_w[e] >= ws->d[t]"),
}


def _pins_pass(so) -> bool:
    """Return True when every pin accepts the given oracle build."""
    try:
        # brute force on a few small graphs with ties, both kinds
        for seed in range(12):
            g = synth.random_small(4 + seed % 4, 0.5, 1, 3, 500 + seed, seed % 2 == 0)
            st = oracle.brandes(g, so=so, nthreads=1)
            d, sigma, delta, bc = brute.betweenness(g)
            for s in range(g.n):
                for t in range(g.n):
                    if d[s][t] is None:
                        if st.D[s, t] != oracle.INF64:
                            return False
                    elif st.D[s, t] != d[s][t] or int(st.SIG[s, t]) != sigma[s][t]:
                        return False
            if not np.allclose(st.BC, [float(x) for x in bc], rtol=1e-12, atol=1e-12):
                return False
        # hand-derived fixtures
        for name in golden_io.all_fixtures():
            fx = golden_io.load(name)
            em = synth.EdgeMap.of(golden_io.graph_of(fx))
            for blk in fx.blocks:
                if blk.update is not None:
                    synth.apply_update(em, blk.update)
                st = oracle.brandes(em.to_graph(), so=so, nthreads=1)
                for v, x in blk.bc.items():
                    if abs(st.BC[v] - float(x)) > 1e-12:
                        return False
        # closed forms
        n = 9
        if oracle.brandes(synth.star_graph(n), so=so).BC[0] != (n - 1) * (n - 2) / 2:
            return False
        if not np.all(oracle.brandes(synth.cycle_graph(7, True), so=so).BC == 15):
            return False
    except oracle.OracleError:
        return False
    return True


def _build_variant(tmp_path, name, old, new):
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(so), str(path)])
    return oracle.load_variant(str(so))


def test_unmutated_oracle_passes_pins():
    assert _pins_pass(oracle.lib())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    so = _build_variant(tmp_path, name, old, new)
    assert not _pins_pass(so), f"planted mistake {name} was not caught by the pins"
