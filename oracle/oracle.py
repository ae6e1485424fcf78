"""Python face of the CPU oracle (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this module.
It loads ``liboracle.so`` built from ``bc_oracle.c`` (plain static Brandes recomputed
on the current graph; see the header of that file for what each step follows in the
paper) and offers the graph-edit helpers the tests need.  It does not import, and is
not imported by, the CUDA library or its binding.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bc_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

OK = 0
ERR_ARG = -1
ERR_OVERFLOW = -3
ERR_DIST_OVERFLOW = -4
ERR_OOM = -5

INF64 = np.iinfo(np.int64).max


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (portable flags only)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        _lib.oracle_brandes_sources.argtypes = [i32, i32, i64, p, p, p, i32, p, p, p, p, p, i32]
        _lib.oracle_brandes_sources.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class State:
    """Static state of a graph: D (int64, INF64 = unreachable), SIG (uint64), DEL and BC."""
    D: np.ndarray | None
    SIG: np.ndarray | None
    DEL: np.ndarray | None
    BC: np.ndarray | None


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def load_variant(path: str):
    """Load another build of bc_oracle.c (the tests compile planted-mistake variants)."""
    so = ctypes.CDLL(path)
    p = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    so.oracle_brandes_sources.argtypes = [i32, i32, i64, p, p, p, i32, p, p, p, p, p, i32]
    so.oracle_brandes_sources.restype = ctypes.c_int
    return so


def brandes(g, sources=None, want_rows: bool = True, want_bc: bool = True,
            nthreads: int | None = None, so=None) -> State:
    """Static Brandes on ``g`` (a ``synth.Graph``-like object with n, directed, src, dst, w).

    ``sources`` None means every vertex; then BC is Eq. 3 over the whole graph.  With a
    list of sources, row i belongs to sources[i] and BC is the partial sum over them."""
    n = int(g.n)
    src = np.ascontiguousarray(g.src, dtype=np.int32)
    dst = np.ascontiguousarray(g.dst, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.int64)
    srcs = None if sources is None else np.ascontiguousarray(sources, dtype=np.int32)
    k = n if srcs is None else int(srcs.shape[0])
    D = np.empty((k, n), np.int64) if want_rows else None
    SIG = np.empty((k, n), np.uint64) if want_rows else None
    DEL = np.empty((k, n), np.float64) if want_rows else None
    BC = np.empty(n, np.float64) if want_bc else None
    rc = (so or lib()).oracle_brandes_sources(
        n, 1 if g.directed else 0, int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(w),
        k, _ptr(srcs), _ptr(D), _ptr(SIG), _ptr(DEL), _ptr(BC),
        int(nthreads or default_threads()))
    if rc != OK:
        raise OracleError(rc)
    return State(D, SIG, DEL, BC)
