"""Failure handling on the GPU without faulting it: a testing hook makes the sweep kernels
skip their first field computation, so their first bounded wait cannot complete.  The
kernel must give up after the (short) limit, report PIM_ERR_TIMEOUT through the host, and
leave the CUDA context usable: the next normal anneal matches the oracle."""
import numpy as np
import pytest

from oracle import pimi
from workloads import Instance, eta_power, linear_beta, maxcut_gauss, sk_pm1

from gpu_helpers import assert_same, collect, oracle_run, pim

pytestmark = pytest.mark.gpu


def _instance(kind):
    if kind == "fused":
        return sk_pm1(64, 0)
    if kind in ("large", "mid"):
        return sk_pm1(300, 1)
    base = maxcut_gauss(64, 2)
    return Instance("maxcut_gauss", 64, pimi.round_bf16(base.J), np.zeros(64), base.c, 2)


@pytest.mark.parametrize("kind", ["fused", "large", "mid", "real"])
def test_injected_wait_gives_up_and_context_survives(kind):
    P = pim()
    inst = _instance(kind)
    flags = {"large": P.PIM_PATH_BIG, "mid": P.PIM_PATH_MID}.get(kind, 0)
    T = 12
    beta = linear_beta(T)
    eta = eta_power(beta)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_set_fault_injection(1, 20_000_000)  # 20 ms wait limit
        try:
            P.pim_anneal(hd, 130, T, 3, flags=flags)
            with pytest.raises(P.PimError) as e:
                P.pim_sync(hd)
            assert e.value.code == P.PIM_ERR_TIMEOUT
        finally:
            P.pim_set_fault_injection(0, 0)
        P.pim_anneal(hd, 130, T, 3, flags=flags)
        P.pim_sync(hd)
        if kind != "real":
            want = oracle_run(inst, beta, eta, 0.5, replicas=130, seed=3)
            assert_same(collect(hd, inst.n), want, label=kind)
        else:
            e = P.pim_energies(hd)
            assert np.all(np.isfinite(e["final_E"]))
    finally:
        P.pim_destroy(hd)
