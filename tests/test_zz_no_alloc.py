"""bc_static_scores_noalloc, the entry point that allocates no device memory.

Some callers cannot call cudaMalloc: their device memory belongs to a framework's
caching allocator, or a serving process reserves HBM at start-up and allows no later
allocation.  They hand over a graph already in device memory and a device buffer for
the scores; the library keeps its scratch in one fixed array of its own.  Here the
test (not the entry point) places the inputs in device memory with torch, calls the
entry point through the C-ABI twice in a row on different graphs -- so the second call
runs on scratch the first one left behind -- and compares each result with
bc_init_static + bc_get_scores and with the oracle within the parity tolerance; a
repeated call must leave the device's free memory unchanged.  This file is collected
last so that a run stopping at the first failure has run every other test first.
"""
import gc

import numpy as np
import pytest

from oracle import oracle
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


def _device_inputs(torch, g):
    off, dst, w = _csr(g)
    t_off = torch.from_numpy(off).cuda()
    t_dst = torch.from_numpy(dst).cuda()
    t_w = torch.from_numpy(w).cuda()
    t_out = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    return t_off, t_dst, t_w, t_out


def _call(lib, torch, g, flags, inputs=None):
    t_off, t_dst, t_w, t_out = inputs or _device_inputs(torch, g)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.bc_static_scores_noalloc(g.n, int(t_dst.shape[0]), t_off.data_ptr(), t_dst.data_ptr(),
                                      t_w.data_ptr(), flags, t_out.data_ptr(), stream)
    return rc, t_out.cpu().numpy()


CASES = [
    (lambda: synth.erdos_renyi(300, 1500, 1, 20, 11, directed=True), "i32",
     binding.BC_DIRECTED | binding.BC_DIST_I32),
    (lambda: synth.barabasi_albert(400, 4, 1, 50, 12), "i64",
     binding.BC_UNDIRECTED | binding.BC_DIST_I64),
]


def test_noalloc_matches_static_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = binding.load()
    for make, dist, flags in CASES:
        g = make()
        rc, got = _call(lib, torch, g, flags)
        assert rc == binding.BC_OK
        exp = binding.BCGraph(g, dist=dist).bc_get_scores()
        ok, worst = close(got, exp)
        assert ok, f"n={g.n}: worst error {worst:.3g} x tolerance (against bc_init_static)"
        ok, worst = close(got, oracle.brandes(g, want_rows=False).BC)
        assert ok, f"n={g.n}: worst error {worst:.3g} x tolerance (against the oracle)"


def test_noalloc_second_call_allocates_nothing():
    # A repeated call (its kernels already loaded by the first) must leave the device's
    # free memory and torch's allocated bytes exactly as they were.
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = binding.load()
    for make, dist, flags in CASES:
        g = make()
        rc, first = _call(lib, torch, g, flags)
        assert rc == binding.BC_OK
        t_off, t_dst, t_w, t_out = _device_inputs(torch, g)
        stream = torch.cuda.current_stream().cuda_stream
        # handles of earlier tests freed by the garbage collector inside the window would
        # raise the free memory: collect them first and keep the collector off meanwhile
        gc.collect()
        torch.cuda.synchronize()
        gc.disable()
        try:
            free0, _ = torch.cuda.mem_get_info()
            alloc0 = torch.cuda.memory_allocated()
            rc = lib.bc_static_scores_noalloc(g.n, int(t_dst.shape[0]), t_off.data_ptr(), t_dst.data_ptr(),
                                              t_w.data_ptr(), flags, t_out.data_ptr(), stream)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            alloc1 = torch.cuda.memory_allocated()
        finally:
            gc.enable()
        assert rc == binding.BC_OK
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        assert alloc1 == alloc0
        ok, worst = close(t_out.cpu().numpy(), first)
        assert ok, f"n={g.n}: second call differs ({worst:.3g} x tolerance)"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = binding.load()
    g = synth.erdos_renyi(513, 1000, 1, 5, 3, directed=True)
    rc, _ = _call(lib, torch, g, binding.BC_DIRECTED | binding.BC_DIST_I32)
    assert rc == binding.BC_ERR_ARG


def test_noalloc_rejects_a_self_loop():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = binding.load()
    g = synth.path_graph(6, True, 2)
    g = synth.Graph(6, True, np.append(g.src, 3).astype(np.int32), np.append(g.dst, 3).astype(np.int32),
                    np.append(g.w, 1).astype(np.int64))
    rc, _ = _call(lib, torch, g, binding.BC_DIRECTED | binding.BC_DIST_I32)
    assert rc == binding.BC_ERR_ARG
