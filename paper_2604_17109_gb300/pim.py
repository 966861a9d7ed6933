"""Python binding of the C ABI in include/pim.h (argument marshalling only).

Each function has the name of the C entry point it calls and does nothing but convert
numpy arrays and Python values to the C arguments and raise ``PimError`` on a non-zero
status.  All computation happens in libpimi.so; importing this module without the built
library raises immediately -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpimi.so")

PIM_OK, PIM_PENDING = 0, 1
PIM_ERR_INVALID, PIM_ERR_NOMEM, PIM_ERR_CUDA = -1, -2, -3
PIM_ERR_STATE, PIM_ERR_TIMEOUT, PIM_ERR_UNSUPPORTED = -4, -5, -6
PIM_J_INT8, PIM_J_FP32, PIM_J_FP64 = 0, 1, 2
PIM_NOISE_GAUSS, PIM_NOISE_UNIFORM = 0, 1
PIM_ACT_TANH, PIM_ACT_LUT = 0, 1
PIM_CONTINUE, PIM_PATH_FP32REF, PIM_PATH_MID, PIM_PATH_BIG, PIM_RESULTS_TO_HOST = 1, 2, 4, 8, 16
PIM_PATH_FP8 = 32
PIM_NOALLOC_MAX_N, PIM_NOALLOC_MAX_STEPS, PIM_NOALLOC_MAX_REPLICAS = 256, 2048, 4096

# name -> (restype, argtypes); every symbol declared in include/pim.h
SIGNATURES = {
    "pim_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                             C.c_double]),
    "pim_set_schedule": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_float,
                                   C.c_int, C.c_int, C.c_int]),
    "pim_anneal": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                             C.c_void_p, C.c_double, C.c_int, C.c_void_p]),
    "pim_anneal_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                   C.c_uint64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "pim_sync": (C.c_int, [C.c_void_p]),
    "pim_energies": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pim_best_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pim_final_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pim_replicas": (C.c_int, [C.c_void_p]),
    "pim_kernel_ms": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "pim_set_fault_injection": (C.c_int, [C.c_int, C.c_uint64]),
    "pim_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_uint64)]),
    "pim_poll": (C.c_int, [C.c_uint64]),
    "pim_destroy": (None, [C.c_void_p]),
    "pim_last_error": (C.c_char_p, []),
    "pim_noise_levels": (C.c_int, [C.c_int, C.c_void_p]),
    "pim_activation_levels": (C.c_int, [C.c_float, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "pim_thresholds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pim_set_schedule_fixed": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_float,
                                         C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "pim_results_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "pim_state_words": (C.c_int, [C.c_void_p]),
    "pim_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "pim_autotune": (C.c_int, [C.c_int]),
    "pim_tune_report": (C.c_int, [C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "pim_anneal_sequential": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                        C.c_uint32, C.c_void_p, C.c_double, C.c_int, C.c_void_p]),
    "pim_mimo_formulate": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                     C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pim_mimo_reconstruct": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pim_mimo_formulate_depth": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                           C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                           C.c_void_p]),
    "pim_mimo_reconstruct_depth": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                             C.c_void_p]),
    "pim_mimo_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p]),
    "pim_mimo_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                         C.c_uint32, C.POINTER(C.c_uint64)]),
    "pim_mimo_server_poll": (C.c_int, [C.c_void_p, C.c_uint64]),
    "pim_mimo_server_result": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.c_void_p,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pim_mimo_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_size_t)]),
    "pim_mimo_server_replay": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pim_mimo_server_destroy": (None, [C.c_void_p]),
    "pim_mimo_server_idle_wait": (C.c_int, [C.c_void_p, C.c_double]),
    "pim_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p, C.c_int, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_int]),
    "pim_batch_run": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_void_p]),
    "pim_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pim_batch_route": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]),
    "pim_probe_tensor": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "pim_probe_ingest": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "pim_batch_destroy": (None, [C.c_void_p]),
    "pim_anneal_noalloc": (C.c_int, [C.c_int, C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                     C.c_void_p, C.c_float, C.c_int, C.c_uint64, C.c_uint32,
                                     C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}

_lib = None


def lib() -> C.CDLL:
    """Load libpimi.so (built by ``paper_2604_17109_gb300.build``); raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libpimi.so not built at {_LIB_PATH}; run the package build first")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PimError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise PimError(rc, where, lib().pim_last_error().decode())
    return rc


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


_NOISE = {"gauss": PIM_NOISE_GAUSS, "uniform": PIM_NOISE_UNIFORM}
_ACT = {"tanh": PIM_ACT_TANH, "lut": PIM_ACT_LUT}


def pim_last_error() -> str:
    return lib().pim_last_error().decode()


def pim_create(J: np.ndarray, h: np.ndarray | None = None, scale_c: float = 1.0) -> int:
    """Stage an instance; integer J -> PIM_J_INT8 (int32 h), float32 J -> PIM_J_FP32 (float32
    h), other float J -> PIM_J_FP64 (float64 h).  Returns the opaque handle (an int)."""
    J = np.asarray(J)
    n = J.shape[0]
    if J.shape != (n, n):
        raise ValueError("J must be square")
    if J.dtype == np.float32:
        jt, J = PIM_J_FP32, np.ascontiguousarray(J)
        hh = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
    elif np.issubdtype(J.dtype, np.floating):
        jt, J = PIM_J_FP64, np.ascontiguousarray(J, dtype=np.float64)
        hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    else:
        jt, J = PIM_J_INT8, np.ascontiguousarray(J, dtype=np.int8)
        hh = None if h is None else np.ascontiguousarray(h, dtype=np.int32)
    out = C.c_void_p()
    _check(lib().pim_create(C.byref(out), n, jt, _ptr(J), _ptr(hh), float(scale_c)), "pim_create")
    return out.value


def pim_set_schedule(inst: int, beta, eta, xi: float, noise="gauss", act="tanh",
                     lut_levels: int = 4) -> None:
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    eta = np.ascontiguousarray(eta, dtype=np.float32)
    if beta.shape != eta.shape:
        raise ValueError("beta and eta must have the same length")
    noise = _NOISE.get(noise, noise)
    act = _ACT.get(act, act)
    _check(lib().pim_set_schedule(inst, beta.size, _ptr(beta), _ptr(eta), float(xi), int(noise),
                                  int(act), int(lut_levels)), "pim_set_schedule")


def pim_set_schedule_fixed(inst: int, beta, eta, xi: float, total_bits: int, int_bits: int,
                           noise="gauss", act="tanh", lut_levels: int = 4) -> None:
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    eta = np.ascontiguousarray(eta, dtype=np.float32)
    if beta.shape != eta.shape:
        raise ValueError("beta and eta must have the same length")
    noise = _NOISE.get(noise, noise)
    act = _ACT.get(act, act)
    _check(lib().pim_set_schedule_fixed(inst, beta.size, _ptr(beta), _ptr(eta), float(xi),
                                        int(noise), int(act), int(lut_levels), int(total_bits),
                                        int(int_bits)), "pim_set_schedule_fixed")


def pim_anneal(inst: int, replicas: int, sweeps: int, seed: int, instance_id: int = 0,
               t_begin: int = 0, init_spins: np.ndarray | None = None, target=None,
               flags: int = 0, stream=None) -> None:
    init = None if init_spins is None else np.ascontiguousarray(init_spins, dtype=np.int8)
    tgt = math.nan if target is None else float(target)
    _check(lib().pim_anneal(inst, int(replicas), int(t_begin), int(sweeps), int(seed),
                            int(instance_id), _ptr(init), tgt, int(flags), _stream(stream)),
           "pim_anneal")


def pim_anneal_batch(insts, replicas, sweeps: int, seed: int, t_begin: int = 0,
                     instance_ids=None, targets=None, flags: int = 0, stream=None) -> None:
    count = len(insts)
    handles = (C.c_void_p * count)(*insts)
    reps = np.ascontiguousarray(np.broadcast_to(np.asarray(replicas, np.int32), (count,)))
    ids = None if instance_ids is None else np.ascontiguousarray(instance_ids, dtype=np.uint32)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.float64)
    _check(lib().pim_anneal_batch(C.cast(handles, C.c_void_p), count, _ptr(reps), int(t_begin),
                                  int(sweeps), int(seed), _ptr(ids), _ptr(tg), int(flags),
                                  _stream(stream)), "pim_anneal_batch")


def pim_anneal_sequential(inst: int, replicas: int, sweeps: int, seed: int,
                          instance_id: int = 0, t_begin: int = 0,
                          init_spins: np.ndarray | None = None, target=None, flags: int = 0,
                          stream=None) -> None:
    init = None if init_spins is None else np.ascontiguousarray(init_spins, dtype=np.int8)
    tgt = math.nan if target is None else float(target)
    _check(lib().pim_anneal_sequential(inst, int(replicas), int(t_begin), int(sweeps), int(seed),
                                       int(instance_id), _ptr(init), tgt, int(flags),
                                       _stream(stream)), "pim_anneal_sequential")


def _complex_ri(a) -> np.ndarray:
    """complex array -> contiguous interleaved (re, im) float64."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


def spins_per_component(qam: int) -> int:
    return {4: 2, 16: 2, 64: 3}[qam]


def pim_mimo_formulate(H, y, qam: int, mmse_reg: float, depth: int = 0):
    """(J n x n, h n, x_mmse nt complex) of the DI-MIMO instance of (H, y); depth 0 = the
    constellation's correction set, 2 = T = [I, I], 3 = T = [2I, I, I]."""
    H = np.asarray(H)
    nr, nt = H.shape
    n = (depth or spins_per_component(qam)) * 2 * nt
    J = np.empty((n, n), np.float64)
    h = np.empty(n, np.float64)
    xm = np.empty(2 * nt, np.float64)
    Hri, yri = _complex_ri(H), _complex_ri(y)
    if depth:
        _check(lib().pim_mimo_formulate_depth(nt, nr, int(qam), int(depth), _ptr(Hri), _ptr(yri),
                                              float(mmse_reg), _ptr(J), _ptr(h), _ptr(xm)),
               "pim_mimo_formulate_depth")
    else:
        _check(lib().pim_mimo_formulate(nt, nr, int(qam), _ptr(Hri), _ptr(yri), float(mmse_reg),
                                        _ptr(J), _ptr(h), _ptr(xm)), "pim_mimo_formulate")
    return J, h, xm.view(np.complex128)


def pim_mimo_reconstruct(x_mmse, spins, qam: int, depth: int = 0) -> np.ndarray:
    xm = _complex_ri(x_mmse)
    nt = xm.size // 2
    s = np.ascontiguousarray(spins, dtype=np.int8)
    out = np.empty(2 * nt, np.float64)
    if depth:
        _check(lib().pim_mimo_reconstruct_depth(nt, int(qam), int(depth), _ptr(xm), _ptr(s),
                                                _ptr(out)), "pim_mimo_reconstruct_depth")
    else:
        _check(lib().pim_mimo_reconstruct(nt, int(qam), _ptr(xm), _ptr(s), _ptr(out)),
               "pim_mimo_reconstruct")
    return out.view(np.complex128)


class MimoServerConfig(C.Structure):
    _fields_ = [("nt", C.c_int), ("nr", C.c_int), ("qam", C.c_int), ("replicas", C.c_int),
                ("sweeps", C.c_int), ("beta", C.c_void_p), ("eta", C.c_void_p), ("xi", C.c_float),
                ("scale_c", C.c_double), ("seed", C.c_uint64), ("max_batch", C.c_int),
                ("max_inflight", C.c_int), ("mem_budget", C.c_size_t),
                ("device_queue", C.c_int), ("idle_s", C.c_double)]


def pim_mimo_server_create(nt, nr, qam, replicas, beta, eta, xi, scale_c, seed=0, max_batch=64,
                           max_inflight=4, mem_budget=1 << 30, device_queue=False,
                           idle_s=0.05) -> int:
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    eta = np.ascontiguousarray(eta, dtype=np.float32)
    cfg = MimoServerConfig(int(nt), int(nr), int(qam), int(replicas), int(beta.size),
                           beta.ctypes.data, eta.ctypes.data, float(xi), float(scale_c), int(seed),
                           int(max_batch), int(max_inflight), int(mem_budget),
                           1 if device_queue else 0, float(idle_s))
    out = C.c_void_p()
    _check(lib().pim_mimo_server_create(C.byref(out), C.byref(cfg)), "pim_mimo_server_create")
    return out.value


def pim_mimo_server_submit(server: int, H, y, mmse_reg: float, request_id: int) -> int:
    Hri, yri = _complex_ri(H), _complex_ri(y)
    t = C.c_uint64()
    _check(lib().pim_mimo_server_submit(server, _ptr(Hri), _ptr(yri), float(mmse_reg),
                                        int(request_id), C.byref(t)), "pim_mimo_server_submit")
    return t.value


def pim_mimo_server_poll(server: int, ticket: int) -> int:
    return _check(lib().pim_mimo_server_poll(server, int(ticket)), "pim_mimo_server_poll")


def pim_mimo_server_result(server: int, ticket: int, nt: int, timeout_s: float = 60.0):
    """(x_hat nt complex, FP64 energy, latency us), or None on timeout."""
    x = np.empty(2 * nt, np.float64)
    e, lat = C.c_double(), C.c_double()
    rc = _check(lib().pim_mimo_server_result(server, int(ticket), float(timeout_s), _ptr(x),
                                             C.byref(e), C.byref(lat)), "pim_mimo_server_result")
    if rc == PIM_PENDING:
        return None
    return x.view(np.complex128), e.value, lat.value


def pim_mimo_server_stats(server: int) -> dict:
    c, p50, p99, mb, pk = C.c_uint64(), C.c_double(), C.c_double(), C.c_double(), C.c_size_t()
    rc = lib().pim_mimo_server_stats(server, C.byref(c), C.byref(p50), C.byref(p99), C.byref(mb),
                                     C.byref(pk))
    return {"completed": c.value, "p50_us": p50.value, "p99_us": p99.value,
            "mean_batch": mb.value, "peak_bytes": pk.value, "status": rc}


def pim_mimo_server_replay(server: int, H_all, y_all, reg_all, arrival_us, nt: int):
    """Native load driver; returns (x_hat (count, nt) complex, energies, latencies_us)."""
    Hri, yri = _complex_ri(H_all), _complex_ri(y_all)
    reg = np.ascontiguousarray(reg_all, dtype=np.float64)
    arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
    count = reg.size
    x = np.empty((count, 2 * nt), np.float64)
    e = np.empty(count, np.float64)
    lat = np.empty(count, np.float64)
    _check(lib().pim_mimo_server_replay(server, count, _ptr(Hri), _ptr(yri), _ptr(reg), _ptr(arr),
                                        _ptr(x), _ptr(e), _ptr(lat)), "pim_mimo_server_replay")
    return x.view(np.complex128), e, lat


def pim_mimo_server_destroy(server: int) -> None:
    lib().pim_mimo_server_destroy(server)


def pim_batch_create(insts, replicas, instance_ids=None, targets=None, flags: int = 0) -> int:
    count = len(insts)
    handles = (C.c_void_p * count)(*insts)
    reps = np.ascontiguousarray(np.broadcast_to(np.asarray(replicas, np.int32), (count,)))
    ids = None if instance_ids is None else np.ascontiguousarray(instance_ids, dtype=np.uint32)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.float64)
    out = C.c_void_p()
    _check(lib().pim_batch_create(C.byref(out), C.cast(handles, C.c_void_p), count, _ptr(reps),
                                  _ptr(ids), _ptr(tg), int(flags)), "pim_batch_create")
    return out.value


def pim_batch_run(batch: int, sweeps: int, seed: int, t_begin: int = 0, run_flags: int = 0,
                  stream=None) -> None:
    _check(lib().pim_batch_run(batch, int(t_begin), int(sweeps), int(seed), int(run_flags),
                               _stream(stream)), "pim_batch_run")


BIG_OPERANDS = {0: "fp8", 1: "bf16", 2: "e2m1_resident"}
KERNELS = {0: "fused", 1: "mid", 2: "large"}


def pim_batch_route(batch: int, index: int) -> dict:
    """Kernel of instance `index` of the batch; for the large-N kernel also its tile width
    and operand variant."""
    k, nt, op = C.c_int(), C.c_int(), C.c_int()
    _check(lib().pim_batch_route(batch, index, C.byref(k), C.byref(nt), C.byref(op)),
           "pim_batch_route")
    out = {"kernel": KERNELS[k.value]}
    if k.value == 2:
        out.update(tile_width=nt.value, operand=BIG_OPERANDS[op.value])
    return out


TENSOR_KINDS = {"fp8": 0, "bf16": 1, "e2m1": 2}


def pim_probe_tensor(kind: str, iters: int = 20000) -> float:
    """Measured dense tcgen05 rate (TFLOP/s, all SMs) of one operand kind."""
    out = C.c_double()
    if kind not in TENSOR_KINDS:
        raise PimError(PIM_ERR_INVALID, "pim_probe_tensor", f"unknown kind {kind!r}")
    _check(lib().pim_probe_tensor(TENSOR_KINDS[kind], int(iters), C.byref(out)), "pim_probe_tensor")
    return out.value


def pim_probe_ingest(nbytes: int = 32768, iters: int = 4000, shared: bool = False) -> float:
    """Measured cp.async.bulk ingest of one SM from L2 (GB/s) while every SM streams."""
    out = C.c_double()
    _check(lib().pim_probe_ingest(int(nbytes), int(iters), 1 if shared else 0, C.byref(out)),
           "pim_probe_ingest")
    return out.value


def pim_batch_info(batch: int) -> dict:
    k, g = C.c_int(), C.c_int()
    _check(lib().pim_batch_info(batch, C.byref(k), C.byref(g)), "pim_batch_info")
    return {"kernel_launches": k.value, "uses_graph": bool(g.value)}


def pim_batch_destroy(batch: int) -> None:
    lib().pim_batch_destroy(batch)


def pim_state_words(inst: int) -> int:
    return lib().pim_state_words(inst)


def pim_results_dev(inst: int, best_E=None, best_t=None, first_hit=None, final_E=None,
                    best_bits=None, final_bits=None, stream=None) -> None:
    """Device-to-device copies of the records into caller buffers given as device pointers
    (ints) or objects with a data_ptr() (e.g. torch tensors); None skips a record."""
    def dp(x):
        if x is None:
            return None
        return x if isinstance(x, int) else int(x.data_ptr())
    _check(lib().pim_results_dev(inst, dp(best_E), dp(best_t), dp(first_hit), dp(final_E),
                                 dp(best_bits), dp(final_bits), _stream(stream)), "pim_results_dev")


def pim_sync(inst: int) -> None:
    _check(lib().pim_sync(inst), "pim_sync")


def pim_replicas(inst: int) -> int:
    return lib().pim_replicas(inst)


def pim_set_fault_injection(mode: int, wait_limit_ns: int = 0) -> None:
    _check(lib().pim_set_fault_injection(int(mode), int(wait_limit_ns)), "pim_set_fault_injection")


def pim_kernel_ms(inst: int) -> float:
    ms = C.c_float()
    _check(lib().pim_kernel_ms(inst, C.byref(ms)), "pim_kernel_ms")
    return ms.value


def pim_energies(inst: int) -> dict:
    R = pim_replicas(inst)
    best_E = np.empty(R, np.float64)
    final_E = np.empty(R, np.float64)
    best_t = np.empty(R, np.int32)
    first = np.empty(R, np.int32)
    _check(lib().pim_energies(inst, _ptr(best_E), _ptr(best_t), _ptr(first), _ptr(final_E)),
           "pim_energies")
    return dict(best_E=best_E, best_t=best_t, first_hit=first, final_E=final_E)


def _state(fn, inst: int, n: int, where: str) -> np.ndarray:
    out = np.empty((pim_replicas(inst), n), np.int8)
    _check(fn(inst, _ptr(out)), where)
    return out


def pim_best_state(inst: int, n: int) -> np.ndarray:
    return _state(lib().pim_best_state, inst, n, "pim_best_state")


def pim_final_state(inst: int, n: int) -> np.ndarray:
    return _state(lib().pim_final_state, inst, n, "pim_final_state")


def pim_submit(inst: int, replicas: int, sweeps: int, seed: int) -> int:
    t = C.c_uint64()
    _check(lib().pim_submit(inst, int(replicas), int(sweeps), int(seed), C.byref(t)), "pim_submit")
    return t.value


def pim_poll(ticket: int) -> int:
    return _check(lib().pim_poll(int(ticket)), "pim_poll")


def pim_destroy(inst: int) -> None:
    lib().pim_destroy(inst)


def pim_noise_levels(noise="gauss") -> np.ndarray:
    out = np.empty(4096, np.float32)
    _check(lib().pim_noise_levels(int(_NOISE.get(noise, noise)), _ptr(out)), "pim_noise_levels")
    return out


def pim_activation_levels(b_t: float, imax: int, act="tanh", lut_levels: int = 4) -> np.ndarray:
    out = np.empty(max(0, 2 * imax + 1), np.float32)
    _check(lib().pim_activation_levels(float(b_t), int(imax), int(_ACT.get(act, act)),
                                       int(lut_levels), _ptr(out)), "pim_activation_levels")
    return out


def pim_thresholds(inst: int) -> tuple[np.ndarray, int]:
    """Device decision table as uint32 [steps, stride] and the field offset imax."""
    steps, imax, stride = C.c_int(), C.c_int(), C.c_int()
    _check(lib().pim_thresholds(inst, None, 0, C.byref(steps), C.byref(imax), C.byref(stride)),
           "pim_thresholds")
    out = np.empty((steps.value, stride.value), np.uint32)
    _check(lib().pim_thresholds(inst, _ptr(out), out.size, None, None, None), "pim_thresholds")
    return out, imax.value


def pim_anneal_noalloc(J: np.ndarray, scale_c: float, beta, eta, xi: float, replicas: int,
                       seed: int, instance_id: int, target, outputs: dict, stream=None) -> None:
    """Allocation-free anneal.  `outputs` maps best_E, best_t, first_hit, final_E, best_bits,
    final_bits to device pointers (ints) the caller owns."""
    J = np.ascontiguousarray(J, dtype=np.int8)
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    eta = np.ascontiguousarray(eta, dtype=np.float32)
    tgt = math.nan if target is None else float(target)
    o = outputs
    _check(lib().pim_anneal_noalloc(J.shape[0], _ptr(J), float(scale_c), beta.size, _ptr(beta),
                                    _ptr(eta), float(xi), int(replicas), int(seed),
                                    int(instance_id), tgt, o["best_E"], o["best_t"],
                                    o["first_hit"], o["final_E"], o["best_bits"],
                                    o["final_bits"], _stream(stream)), "pim_anneal_noalloc")


def pim_fields(inst, spins: np.ndarray, flags: int = 0, stream=None) -> np.ndarray:
    """FP32 fields I = J s + h of the states `spins` (R x n, +-1) as the sweep kernel forms
    them (real couplings); returns float32 R x n."""
    s = np.ascontiguousarray(spins, dtype=np.int8)
    out = np.empty(s.shape, np.float32)
    _check(lib().pim_fields(inst, s.shape[0], _ptr(s), _ptr(out), int(flags), _stream(stream)),
           "pim_fields")
    return out


def pim_autotune(mode: int) -> None:
    """0: analytic cost model only; 1: batch plans measure new shape classes first."""
    _check(lib().pim_autotune(int(mode)), "pim_autotune")


def pim_tune_report() -> str:
    """The measured kernel times, one line per shape class."""
    need = C.c_size_t()
    _check(lib().pim_tune_report(None, 0, C.byref(need)), "pim_tune_report")
    buf = C.create_string_buffer(need.value)
    _check(lib().pim_tune_report(buf, need.value, None), "pim_tune_report")
    return buf.value.decode()


def pim_mimo_server_idle_wait(server: int, timeout_s: float) -> int:
    """Device queue: PIM_ERR_TIMEOUT when the serving kernel ended on its idle limit, PIM_OK
    when it ended on a stop, PIM_PENDING while it runs (returned, not raised)."""
    rc = lib().pim_mimo_server_idle_wait(server, float(timeout_s))
    if rc in (PIM_OK, PIM_PENDING, PIM_ERR_TIMEOUT):
        return rc
    return _check(rc, "pim_mimo_server_idle_wait")
