"""Shared helpers of the GPU tests: run the library through its C ABI and compare with the
oracle element by element."""
import numpy as np

import oracle
from paper_2604_17109_gb300 import build as pkg_build

_built = False


def pim():
    global _built
    if not _built:
        pkg_build.build()
        _built = True
    from paper_2604_17109_gb300 import pim as mod
    return mod


def run_library(inst, beta, eta, xi, *, replicas, sweeps=None, seed=0, q=0, t_begin=0,
                init=None, target=None, noise="gauss", act="tanh", lut_levels=4, flags=0,
                handle=None, keep=False):
    """Stage `inst`, set the schedule, anneal once and return the oracle-format dict."""
    P = pim()
    h = None if not np.any(inst.h) else inst.h
    hd = handle if handle is not None else P.pim_create(inst.J, h, inst.c)
    try:
        if handle is None:
            P.pim_set_schedule(hd, beta, eta, xi, noise, act, lut_levels)
        if sweeps is None:
            sweeps = len(beta) - t_begin
        P.pim_anneal(hd, replicas, sweeps, seed, instance_id=q, t_begin=t_begin,
                     init_spins=init, target=target, flags=flags)
        out = collect(hd, inst.n)
    finally:
        if not keep and handle is None:
            P.pim_destroy(hd)
    if keep:
        out["handle"] = hd
    return out


def collect(hd, n):
    P = pim()
    e = P.pim_energies(hd)
    return dict(best_E=e["best_E"].astype(np.int64), best_t=e["best_t"].astype(np.int64),
                first_hit=e["first_hit"].astype(np.int64), final_E=e["final_E"].astype(np.int64),
                best_state=P.pim_best_state(hd, n), final_state=P.pim_final_state(hd, n))


KEYS = ("best_E", "best_t", "first_hit", "final_E", "best_state", "final_state")


def assert_same(got, want, rows=None, label=""):
    for k in KEYS:
        g = got[k] if rows is None else got[k][rows]
        w = want[k]
        if not np.array_equal(g, w):
            bad = np.argwhere(np.asarray(g) != np.asarray(w))
            raise AssertionError(f"{label} {k} differs at {bad[:5].tolist()} "
                                 f"(got {np.asarray(g).ravel()[:8]}, want {np.asarray(w).ravel()[:8]})")


def oracle_run(inst, beta, eta, xi, **kw):
    return oracle.anneal(inst.J, inst.h, inst.c, beta, eta, xi, **kw)
