"""ctypes binding of libbcgpu.so (declared in include/bcgpu.h).

Argument marshalling only: every step of the computation runs in the CUDA library.
The module-level functions carry the C names; ``BCGraph`` wraps a handle.  Loading
fails loudly when the library has not been built (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

BC_OK = 0
BC_ERR_ARG = -1
BC_ERR_NOT_INCREMENTAL = -2
BC_ERR_OVERFLOW = -3
BC_ERR_DIST_OVERFLOW = -4
BC_ERR_OOM = -5
BC_ERR_CUDA = -6
BC_ERR_TIMEOUT = -7
BC_ERR_POISONED = -8

BC_DIRECTED = 1
BC_UNDIRECTED = 2
BC_DIST_I32 = 16
BC_DIST_I64 = 32
BC_STATIC_ALL_ARCS = 64
BC_UPD_EDGE = 0
BC_UPD_VERTEX = 1

UPDATE_DTYPE = np.dtype([("kind", "<i4"), ("u", "<i4"), ("v", "<i4"), ("k", "<i4"),
                         ("w", "<i8"), ("first", "<i8")], align=True)
VEDGE_DTYPE = np.dtype([("x", "<i4"), ("dir", "<i4"), ("w", "<i8")], align=True)
assert UPDATE_DTYPE.itemsize == 32 and VEDGE_DTYPE.itemsize == 16

INF64 = np.iinfo(np.int64).max

EXPORTS = ["bc_init_static", "bc_apply_edge_update", "bc_apply_vertex_update", "bc_apply_updates",
           "bc_stage_updates", "bc_run_staged", "bc_synchronize", "bc_query", "bc_get_scores",
           "bc_get_rows", "bc_get_info", "bc_get_profile", "bc_set_option", "bc_destroy", "bc_last_error",
           "bc_static_scores_noalloc", "bc_batch_create", "bc_batch_apply", "bc_batch_set_tiles",
           "bc_batch_last_ms", "bc_batch_last_error", "bc_batch_destroy", "bc_get_edges",
           "bc_server_create", "bc_server_add_graph", "bc_server_submit", "bc_server_poll",
           "bc_server_pending", "bc_server_graph", "bc_server_stats", "bc_server_destroy",
           "bc_init_static_f64", "bc_apply_edge_update_f64", "bc_apply_vertex_update_f64", "bc_get_weight_unit"]
PROFILE_CLASSES = ["scan", "accumulate", "bc_rows", "vertex_passes", "bookkeeping", "pair_corrections"]


class bc_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("directed", ctypes.c_int32), ("dist_bytes", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("m", ctypes.c_int64), ("estar_arcs", ctypes.c_int64),
                ("updates_applied", ctypes.c_int64), ("rows_reaccumulated", ctypes.c_int64),
                ("noop_updates", ctypes.c_int64), ("max_rows", ctypes.c_int64),
                ("rows_scanned", ctypes.c_int64), ("pairs_lowered", ctypes.c_int64),
                ("pairs_tied", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("state_bytes", ctypes.c_int64), ("last_init_ms", ctypes.c_double),
                ("rows_full", ctypes.c_int64), ("estar_rebuilds", ctypes.c_int64),
                ("estar_moves", ctypes.c_int64), ("pair_rows", ctypes.c_int64),
                ("pair_targets", ctypes.c_int64),
                ("walk_pairs", ctypes.c_int64),
                ("walk_vertices", ctypes.c_int64),
                ("walk_arcs", ctypes.c_int64)]


RESULT_DTYPE = np.dtype([("request_id", "<i8"), ("graph_id", "<i4"), ("status", "<i4"),
                         ("latency_ns", "<i8")], align=True)


class BCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bcgpu error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbcgpu.so (building it first when asked); raises when it cannot be had."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libbcgpu.so is not built ({path}); run paper_1311_2147_gb300.build")
    lib = ctypes.CDLL(path)
    p, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "bc_init_static": ([ctypes.POINTER(p), i32, i64, p, p, p, u32, p], ctypes.c_int),
        "bc_apply_edge_update": ([p, i32, i32, i64], ctypes.c_int),
        "bc_apply_vertex_update": ([p, i32, i32, p, p, p], ctypes.c_int),
        "bc_apply_updates": ([p, i32, p, p, i64, ctypes.POINTER(i32)], ctypes.c_int),
        "bc_stage_updates": ([p, i32, p, p, i64], ctypes.c_int),
        "bc_run_staged": ([p, ctypes.POINTER(i32)], ctypes.c_int),
        "bc_synchronize": ([p], ctypes.c_int),
        "bc_query": ([p, ctypes.POINTER(i32)], ctypes.c_int),
        "bc_get_scores": ([p, p], ctypes.c_int),
        "bc_get_rows": ([p, i32, i32, p, p, p], ctypes.c_int),
        "bc_get_info": ([p, ctypes.POINTER(bc_info)], ctypes.c_int),
        "bc_get_profile": ([p, p, p, i32], ctypes.c_int),
        "bc_set_option": ([p, ctypes.c_char_p, i64], ctypes.c_int),
        "bc_destroy": ([p], None),
        "bc_last_error": ([p], ctypes.c_char_p),
        "bc_static_scores_noalloc": ([i32, i64, p, p, p, u32, p, p], ctypes.c_int),
        "bc_batch_create": ([ctypes.POINTER(p), i32, p, p], ctypes.c_int),
        "bc_batch_apply": ([p, p, p, p, i64, p], ctypes.c_int),
        "bc_batch_set_tiles": ([p, p, i32], ctypes.c_int),
        "bc_batch_last_ms": ([p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "bc_batch_last_error": ([p], ctypes.c_char_p),
        "bc_batch_destroy": ([p], None),
        "bc_get_edges": ([p, ctypes.POINTER(i64), p, p, p], ctypes.c_int),
        "bc_server_create": ([ctypes.POINTER(p), i64, i32], ctypes.c_int),
        "bc_server_add_graph": ([p, i32, i64, p, p, p, u32, ctypes.POINTER(i32)], ctypes.c_int),
        "bc_server_submit": ([p, i32, p, p, ctypes.POINTER(i64)], ctypes.c_int),
        "bc_server_poll": ([p, i32, p, ctypes.POINTER(i32)], ctypes.c_int),
        "bc_server_pending": ([p, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "bc_server_graph": ([p, i32, ctypes.POINTER(p)], ctypes.c_int),
        "bc_server_stats": ([p, p], ctypes.c_int),
        "bc_server_destroy": ([p], None),
        "bc_init_static_f64": ([ctypes.POINTER(p), i32, i64, p, p, p, u32, p], ctypes.c_int),
        "bc_apply_edge_update_f64": ([p, i32, i32, ctypes.c_double], ctypes.c_int),
        "bc_apply_vertex_update_f64": ([p, i32, i32, p, p, p], ctypes.c_int),
        "bc_get_weight_unit": ([p, ctypes.POINTER(i32)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def encode_updates(ups):
    """Turn ("edge", u, v, w) / ("vertex", v, [(x, w, dir), ...]) tuples into the
    bc_update / bc_vedge arrays of the ABI."""
    rec = np.zeros(len(ups), dtype=UPDATE_DTYPE)
    edges = []
    for i, up in enumerate(ups):
        if up[0] == "edge":
            _, u, v, w = up
            rec[i] = (BC_UPD_EDGE, u, v, 0, w, 0)
        else:
            _, v, es = up
            rec[i] = (BC_UPD_VERTEX, -1, v, len(es), 0, len(edges))
            for x, w, d in es:
                edges.append((x, d, w))
    ed = np.array(edges, dtype=VEDGE_DTYPE) if edges else np.zeros(0, dtype=VEDGE_DTYPE)
    return rec, ed


class BCGraph:
    """One device-resident graph state."""

    def __init__(self, g, dist: str = "i32", stream=None, static_all_arcs: bool = False):
        lib = load()
        self.lib = lib
        self.n = int(g.n)
        self.directed = bool(g.directed)
        src = np.ascontiguousarray(g.src, dtype=np.int32)
        dst = np.ascontiguousarray(g.dst, dtype=np.int32)
        w = np.ascontiguousarray(g.w, dtype=np.int64)
        flags = (BC_DIRECTED if self.directed else BC_UNDIRECTED) | (BC_DIST_I32 if dist == "i32" else BC_DIST_I64)
        if static_all_arcs:
            flags |= BC_STATIC_ALL_ARCS
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        rc = lib.bc_init_static(ctypes.byref(h), self.n, int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(w),
                                flags, st)
        if rc != BC_OK:
            raise BCError(rc, lib.bc_last_error(None).decode())
        self.h = h

    # -- errors
    def _check(self, rc):
        if rc != BC_OK:
            raise BCError(rc, self.lib.bc_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.bc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- updates
    def bc_apply_edge_update(self, u, v, w):
        return self.lib.bc_apply_edge_update(self.h, int(u), int(v), int(w))

    def bc_apply_vertex_update(self, v, nbr, w, dirs=None):
        nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int64)
        d = None if dirs is None else np.ascontiguousarray(dirs, dtype=np.uint8)
        return self.lib.bc_apply_vertex_update(self.h, int(v), int(nbr.shape[0]), _ptr(nbr), _ptr(w), _ptr(d))

    def bc_apply_updates(self, ups):
        rec, ed = encode_updates(ups) if isinstance(ups, list) else ups
        done = ctypes.c_int32(0)
        rc = self.lib.bc_apply_updates(self.h, int(rec.shape[0]), _ptr(rec), _ptr(ed) if ed.size else None,
                                       int(ed.shape[0]), ctypes.byref(done))
        return rc, done.value

    def bc_stage_updates(self, ups):
        rec, ed = encode_updates(ups) if isinstance(ups, list) else ups
        self._staged = (rec, ed)
        return self.lib.bc_stage_updates(self.h, int(rec.shape[0]), _ptr(rec), _ptr(ed) if ed.size else None,
                                         int(ed.shape[0]))

    def bc_run_staged(self):
        done = ctypes.c_int32(0)
        rc = self.lib.bc_run_staged(self.h, ctypes.byref(done))
        return rc, done.value

    def bc_synchronize(self):
        return self.lib.bc_synchronize(self.h)

    def bc_query(self):
        done = ctypes.c_int32(0)
        rc = self.lib.bc_query(self.h, ctypes.byref(done))
        return rc, bool(done.value)

    def bc_set_option(self, name: str, value: int):
        return self._check(self.lib.bc_set_option(self.h, name.encode(), int(value)))

    # -- results
    def bc_get_scores(self):
        out = np.empty(self.n, dtype=np.float64)
        self._check(self.lib.bc_get_scores(self.h, _ptr(out)))
        return out

    def bc_get_rows(self, s0=0, count=None, want=("d", "sigma", "delta")):
        count = self.n - s0 if count is None else count
        d = np.empty((count, self.n), np.int64) if "d" in want else None
        s = np.empty((count, self.n), np.uint64) if "sigma" in want else None
        dl = np.empty((count, self.n), np.float64) if "delta" in want else None
        self._check(self.lib.bc_get_rows(self.h, int(s0), int(count), _ptr(d), _ptr(s), _ptr(dl)))
        return d, s, dl

    def bc_get_info(self):
        info = bc_info()
        self._check(self.lib.bc_get_info(self.h, ctypes.byref(info)))
        return {k: getattr(info, k) for k, _ in bc_info._fields_}

    def bc_get_profile(self, reset=True):
        ms = np.zeros(len(PROFILE_CLASSES), np.float64)
        nl = np.zeros(len(PROFILE_CLASSES), np.int64)
        self._check(self.lib.bc_get_profile(self.h, _ptr(ms), _ptr(nl), 1 if reset else 0))
        return {c: (float(ms[i]), int(nl[i])) for i, c in enumerate(PROFILE_CLASSES)}

    def last_error(self):
        return self.lib.bc_last_error(self.h).decode()


class BCGraphReal(BCGraph):
    """A device-resident graph state with real (fp64) weights: path lengths are the
    exact sums of the given doubles (bc_init_static_f64)."""

    def __init__(self, n, directed, src, dst, w, dist: str = "i64", stream=None):
        lib = load()
        self.lib = lib
        self.n = int(n)
        self.directed = bool(directed)
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float64)
        flags = (BC_DIRECTED if self.directed else BC_UNDIRECTED) | (BC_DIST_I32 if dist == "i32" else BC_DIST_I64)
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        rc = lib.bc_init_static_f64(ctypes.byref(h), self.n, int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(w),
                                    flags, st)
        if rc != BC_OK:
            raise BCError(rc, lib.bc_last_error(None).decode())
        self.h = h

    def bc_apply_edge_update_f64(self, u, v, w):
        return self.lib.bc_apply_edge_update_f64(self.h, int(u), int(v), float(w))

    def bc_apply_vertex_update_f64(self, v, nbr, w, dirs=None):
        nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float64)
        d = None if dirs is None else np.ascontiguousarray(dirs, dtype=np.uint8)
        return self.lib.bc_apply_vertex_update_f64(self.h, int(v), int(nbr.shape[0]), _ptr(nbr), _ptr(w), _ptr(d))

    def bc_get_weight_unit(self):
        e = ctypes.c_int32(0)
        self._check(self.lib.bc_get_weight_unit(self.h, ctypes.byref(e)))
        return e.value


class BCBatch:
    """A batch of device-resident graphs updated together (one CUDA graph launch per call)."""

    def __init__(self, graphs, stream=None):
        self.lib = load()
        self.graphs = list(graphs)
        hs = (ctypes.c_void_p * len(self.graphs))(*[g.h.value for g in self.graphs])
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        rc = self.lib.bc_batch_create(ctypes.byref(h), len(self.graphs), ctypes.cast(hs, ctypes.c_void_p), st)
        if rc != BC_OK:
            raise BCError(rc, "bc_batch_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.bc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bc_batch_apply(self, per_graph_updates):
        """per_graph_updates: one list of update tuples per graph.  Returns (rc, n_done)."""
        counts = np.array([len(u) for u in per_graph_updates], dtype=np.int32)
        flat = [u for us in per_graph_updates for u in us]
        rec, ed = encode_updates(flat)
        done = np.zeros(len(self.graphs), dtype=np.int32)
        rc = self.lib.bc_batch_apply(self.h, _ptr(counts), _ptr(rec) if rec.size else None,
                                     _ptr(ed) if ed.size else None, int(ed.shape[0]), _ptr(done))
        return rc, done

    def bc_batch_set_tiles(self, tiles):
        t = np.ascontiguousarray(tiles, dtype=np.int32)
        rc = self.lib.bc_batch_set_tiles(self.h, _ptr(t), int(t.shape[0]))
        if rc != BC_OK:
            raise BCError(rc, self.last_error())

    def bc_batch_last_ms(self):
        ms = ctypes.c_double(0.0)
        self.lib.bc_batch_last_ms(self.h, ctypes.byref(ms))
        return ms.value

    def last_error(self):
        return self.lib.bc_batch_last_error(self.h).decode()


class _Borrowed(BCGraph):
    """A handle owned by a server (not destroyed by Python)."""

    def __init__(self, lib, h, n, directed):
        self.lib, self.h, self.n, self.directed = lib, h, n, directed

    def close(self):
        self.h = None


class BCServer:
    """Continuous-batching server over many device-resident graphs."""

    def __init__(self, budget_bytes: int, max_batch: int = 64):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.bc_server_create(ctypes.byref(h), int(budget_bytes), int(max_batch))
        if rc != BC_OK:
            raise BCError(rc, "bc_server_create failed")
        self.h = h
        self.meta = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.bc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_graph(self, g, dist="i32") -> int:
        src, dst, w = g.arrays()
        flags = (BC_DIRECTED if g.directed else BC_UNDIRECTED) | (BC_DIST_I32 if dist == "i32" else BC_DIST_I64)
        gid = ctypes.c_int32(0)
        rc = self.lib.bc_server_add_graph(self.h, int(g.n), int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(w),
                                          flags, ctypes.byref(gid))
        if rc != BC_OK:
            raise BCError(rc, "bc_server_add_graph failed")
        self.meta.append((int(g.n), bool(g.directed)))
        return gid.value

    def submit(self, gid: int, up) -> int:
        rec, ed = encode_updates([up])
        rid = ctypes.c_int64(0)
        rc = self.lib.bc_server_submit(self.h, int(gid), _ptr(rec), _ptr(ed) if ed.size else None, ctypes.byref(rid))
        if rc != BC_OK:
            raise BCError(rc, "bc_server_submit failed")
        return rid.value

    def poll(self, max_results: int = 4096):
        out = np.zeros(max_results, dtype=RESULT_DTYPE)
        k = ctypes.c_int32(0)
        rc = self.lib.bc_server_poll(self.h, int(max_results), _ptr(out), ctypes.byref(k))
        if rc != BC_OK:
            raise BCError(rc, "bc_server_poll failed")
        return out[: k.value]

    def pending(self):
        q, f = ctypes.c_int64(0), ctypes.c_int64(0)
        self.lib.bc_server_pending(self.h, ctypes.byref(q), ctypes.byref(f))
        return q.value, f.value

    def drain(self):
        res = []
        while True:
            r = self.poll()
            if r.size:
                res.append(r)
            q, f = self.pending()
            if q == 0 and f == 0:
                break
        return np.concatenate(res) if res else np.zeros(0, dtype=RESULT_DTYPE)

    def graph(self, gid: int) -> BCGraph:
        h = ctypes.c_void_p()
        rc = self.lib.bc_server_graph(self.h, int(gid), ctypes.byref(h))
        if rc != BC_OK:
            raise BCError(rc, "bc_server_graph failed")
        n, directed = self.meta[gid]
        return _Borrowed(self.lib, h, n, directed)

    def stats(self):
        st = np.zeros(5, np.int64)
        self.lib.bc_server_stats(self.h, _ptr(st))
        return dict(zip(["resident", "bytes", "admissions", "evictions", "launches"], st.tolist()))
