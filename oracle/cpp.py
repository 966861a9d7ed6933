"""ctypes front of the plain C++17 oracle (pimi_ref.cpp) -- TEST INFRASTRUCTURE ONLY.

``build()`` compiles ``pimi_ref.cpp`` with the host C++ compiler (``-O2 -ffp-contract=off``,
threads for the replicas) into ``libpimi_oracle.so`` next to it; ``anneal`` takes the
arguments and returns the dict of ``oracle.pimi.anneal``.  Only the tests, the smoke check
and the benchmark's CPU-baseline legs use it; it shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pimi_ref.cpp")
LIB = os.path.join(HERE, "libpimi_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        raise RuntimeError("no host C++ compiler found to build the C++ oracle")
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", SRC,
           "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"building the C++ oracle failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.pimi_oracle_anneal.restype = C.c_int
        _lib.pimi_oracle_anneal.argtypes = (
            [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
             C.c_float, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
             C.c_uint64, C.c_uint32, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int]
            + [C.c_void_p] * 6)
        _lib.pimi_oracle_noise_levels.restype = None
        _lib.pimi_oracle_noise_levels.argtypes = [C.c_int, C.c_void_p]
        _lib.pimi_oracle_philox.restype = None
        _lib.pimi_oracle_philox.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def noise_levels(noise: str = "gauss") -> np.ndarray:
    out = np.empty(4096, np.float32)
    lib().pimi_oracle_noise_levels(0 if noise == "gauss" else 1, _p(out))
    return out


def philox4x32_10(ctr, k0: int, k1: int):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64) & 0xFFFFFFFF, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    lib().pimi_oracle_philox(_p(c), k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF, _p(out))
    return [int(x) for x in out]


def anneal(J, h, c: float, beta, eta, xi: float, *, replicas: int | None = None,
           sweeps: int | None = None, seed: int = 0, q: int = 0, t_begin: int = 0,
           init: np.ndarray | None = None, target: float | None = None, noise: str = "gauss",
           act: str = "tanh", lut_levels: int = 4, replica_ids=None, prev: dict | None = None,
           threads: int = 0) -> dict:
    """Same arguments and result keys as ``oracle.pimi.anneal`` (no recording)."""
    J = np.asarray(J)
    n = J.shape[0]
    real = not np.issubdtype(J.dtype, np.integer)
    if real:
        Jc = np.ascontiguousarray(J, dtype=np.float64)
        hc = None if h is None or not np.any(h) else np.ascontiguousarray(h, dtype=np.float64)
    else:
        Jc = np.ascontiguousarray(J, dtype=np.int8)
        hc = None if h is None or not np.any(h) else np.ascontiguousarray(h, dtype=np.int32)
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    eta = np.ascontiguousarray(eta, dtype=np.float32)
    if sweeps is None:
        sweeps = len(beta) - t_begin
    if t_begin + sweeps > len(beta):
        raise ValueError("t_begin + sweeps exceeds the schedule")
    if replica_ids is None:
        replica_ids = np.arange(replicas)
    rid = np.ascontiguousarray(replica_ids, dtype=np.int64)
    R = rid.size
    best_E = np.empty(R, np.float64)
    best_t = np.empty(R, np.int32)
    first_hit = np.empty(R, np.int32)
    final_E = np.empty(R, np.float64)
    best_state = np.empty((R, n), np.int8)
    final_state = np.empty((R, n), np.int8)
    cont = 0
    init_c = None
    if prev is not None:
        cont = 1
        best_E[:] = prev["best_E"]
        best_t[:] = prev["best_t"]
        first_hit[:] = prev["first_hit"]
        best_state[:] = prev["best_state"]
        final_state[:] = prev["final_state"]
    elif init is not None:
        init_c = np.ascontiguousarray(init, dtype=np.int8)
    rc = lib().pimi_oracle_anneal(
        n, 1 if real else 0, _p(Jc), None if hc is None else _p(hc), float(c), _p(beta), _p(eta),
        float(xi), 0 if noise == "gauss" else 1, 0 if act == "tanh" else 1, int(lut_levels), R,
        _p(rid), int(t_begin), int(sweeps), int(seed) & 0xFFFFFFFFFFFFFFFF, int(q) & 0xFFFFFFFF,
        None if init_c is None else _p(init_c), cont, 0 if target is None else 1,
        math.nan if target is None else float(target), int(threads), _p(best_E), _p(best_t),
        _p(first_hit), _p(final_E), _p(best_state), _p(final_state))
    if rc != 0:
        raise ValueError("pimi_oracle_anneal rejected its arguments")
    if not real:
        best_E = best_E.astype(np.int64)
        final_E = final_E.astype(np.int64)
    return dict(best_E=best_E, best_t=best_t.astype(np.int64),
                first_hit=first_hit.astype(np.int64), final_E=final_E, best_state=best_state,
                final_state=final_state)
