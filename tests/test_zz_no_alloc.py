"""bc_static_scores_noalloc, the entry point that allocates no device memory.

Some callers cannot call cudaMalloc: their device memory belongs to a framework's
caching allocator, or a serving process reserves HBM at start-up and allows no later
allocation.  They hand over a graph already in device memory and a device buffer for
the scores; the library keeps its scratch in one fixed array of its own.  Here the
test (not the entry point) places the inputs in device memory with torch, calls the
entry point through the C-ABI twice in a row on different graphs -- so the second call
runs on scratch the first one left behind -- and compares each result with
bc_init_static + bc_get_scores within the parity tolerance.  This file is collected
last so that a run stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

from paper_1311_2147_gb300 import binding, synth
from tests.parity_util import close

pytestmark = pytest.mark.gpu


def _csr(g):
    src = g.src.astype(np.int64)
    dst = g.dst.astype(np.int64)
    w = g.w.astype(np.int64)
    if not g.directed:
        src, dst, w = np.concatenate([src, dst]), np.concatenate([dst, src]), np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, w = src[order], dst[order], w[order]
    off = np.zeros(g.n + 1, np.int32)
    off[1:] = np.cumsum(np.bincount(src, minlength=g.n))
    return off, dst.astype(np.int32), w


def _call(lib, torch, g, flags):
    off, dst, w = _csr(g)
    t_off = torch.from_numpy(off).cuda()
    t_dst = torch.from_numpy(dst).cuda()
    t_w = torch.from_numpy(w).cuda()
    t_out = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    rc = lib.bc_static_scores_noalloc(g.n, int(dst.shape[0]), t_off.data_ptr(), t_dst.data_ptr(),
                                      t_w.data_ptr(), flags, t_out.data_ptr(), stream)
    return rc, t_out.cpu().numpy()


def test_noalloc_matches_static_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = binding.load()
    cases = [
        (synth.erdos_renyi(300, 1500, 1, 20, 11, directed=True), "i32",
         binding.BC_DIRECTED | binding.BC_DIST_I32),
        (synth.barabasi_albert(400, 4, 1, 50, 12), "i64",
         binding.BC_UNDIRECTED | binding.BC_DIST_I64),
    ]
    for g, dist, flags in cases:
        rc, got = _call(lib, torch, g, flags)
        assert rc == binding.BC_OK
        exp = binding.BCGraph(g, dist=dist).bc_get_scores()
        ok, worst = close(got, exp)
        assert ok, f"n={g.n}: worst error {worst:.3g} x tolerance"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = binding.load()
    g = synth.erdos_renyi(513, 1000, 1, 5, 3, directed=True)
    rc, _ = _call(lib, torch, g, binding.BC_DIRECTED | binding.BC_DIST_I32)
    assert rc == binding.BC_ERR_ARG
