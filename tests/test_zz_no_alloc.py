"""The allocation-free entry point against the regular one.

pim_anneal_noalloc serves callers that may not allocate device memory while they run (a
real-time loop, a framework that owns all device memory through its own pool, a fixed
memory budget): they hand in their own output buffers and the library works inside one
fixed-size device array.  This test runs it twice in a row on different instances and
checks each result against pim_create / pim_set_schedule / pim_anneal on the same inputs,
bit for bit (the tolerance every integer-coupling test here uses).  It lives in its own
file so that a run which stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from workloads import eta_power, linear_beta, maxcut_er, sk_pm1

from gpu_helpers import pim, run_library

pytestmark = pytest.mark.gpu


def _unpack(bits: np.ndarray, n: int) -> np.ndarray:
    b = bits.astype(np.uint32)
    idx = np.arange(n)
    on = (b[:, idx >> 5] >> (idx & 31).astype(np.uint32)) & 1
    return np.where(on == 1, 1, -1).astype(np.int8)


def _noalloc(inst, beta, eta, xi, R, seed, q, target):
    torch = pytest.importorskip("torch")
    P = pim()
    words = ((inst.n + 63) // 64) * 2
    dev = torch.device("cuda", 0)
    out = {
        "best_E": torch.full((R,), np.nan, dtype=torch.float64, device=dev),
        "final_E": torch.full((R,), np.nan, dtype=torch.float64, device=dev),
        "best_t": torch.full((R,), -7, dtype=torch.int32, device=dev),
        "first_hit": torch.full((R,), -7, dtype=torch.int32, device=dev),
        "best_bits": torch.zeros((R, words), dtype=torch.int32, device=dev),
        "final_bits": torch.zeros((R, words), dtype=torch.int32, device=dev),
    }
    torch.cuda.synchronize()
    P.pim_anneal_noalloc(inst.J, inst.c, beta, eta, xi, R, seed, q, target,
                         {k: v.data_ptr() for k, v in out.items()})
    torch.cuda.synchronize()
    host = {k: v.cpu().numpy() for k, v in out.items()}
    return dict(best_E=host["best_E"].astype(np.int64), final_E=host["final_E"].astype(np.int64),
                best_t=host["best_t"].astype(np.int64),
                first_hit=host["first_hit"].astype(np.int64),
                best_state=_unpack(host["best_bits"].view(np.uint32), inst.n),
                final_state=_unpack(host["final_bits"].view(np.uint32), inst.n))


def test_noalloc_matches_regular_entry_point_twice():
    cases = [
        (sk_pm1(200, 3), 300, 400, 0.5, 11, 4, -1500.0),
        (maxcut_er(100, 5), 128, 250, 0.7, 12, 9, -1200.0),
    ]
    for inst, R, T, xi, seed, q, target in cases:
        beta = linear_beta(T)
        eta = eta_power(beta)
        got = _noalloc(inst, beta, eta, xi, R, seed, q, target)
        want = run_library(inst, beta, eta, xi, replicas=R, seed=seed, q=q, target=target)
        for key in ("best_E", "best_t", "first_hit", "final_E", "best_state", "final_state"):
            assert np.array_equal(got[key], want[key]), (inst.n, key)


def test_noalloc_at_the_maximum_sizes_allocates_nothing():
    """n = 256 (row sums 255, the table limit), the longest schedule and the most replicas
    the entry point takes: the tables, the diagonal region and the work list are used up
    to their last offsets.  After a warm-up call (the first call on a device may load the
    library's device code), a call leaves the device's free memory unchanged."""
    torch = pytest.importorskip("torch")
    inst = sk_pm1(256, 7)
    assert int(np.abs(inst.J.astype(np.int64)).sum(axis=1).max()) == 255
    P = pim()
    T, R, xi, seed, q, target = P.PIM_NOALLOC_MAX_STEPS, P.PIM_NOALLOC_MAX_REPLICAS, 0.5, 21, 2, -3000.0
    beta = linear_beta(T)
    eta = eta_power(beta)
    _noalloc(inst, linear_beta(8), eta_power(linear_beta(8)), xi, 4, 0, 0, None)  # warm-up
    words = ((inst.n + 63) // 64) * 2
    dev = torch.device("cuda", 0)
    out = {
        "best_E": torch.empty((R,), dtype=torch.float64, device=dev),
        "final_E": torch.empty((R,), dtype=torch.float64, device=dev),
        "best_t": torch.empty((R,), dtype=torch.int32, device=dev),
        "first_hit": torch.empty((R,), dtype=torch.int32, device=dev),
        "best_bits": torch.empty((R, words), dtype=torch.int32, device=dev),
        "final_bits": torch.empty((R, words), dtype=torch.int32, device=dev),
    }
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info(dev)[0]
    P.pim_anneal_noalloc(inst.J, inst.c, beta, eta, xi, R, seed, q, target,
                         {k: v.data_ptr() for k, v in out.items()})
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info(dev)[0]
    assert free_after == free_before, (free_before, free_after)
    host = {k: v.cpu().numpy() for k, v in out.items()}
    got = dict(best_E=host["best_E"].astype(np.int64), final_E=host["final_E"].astype(np.int64),
               best_t=host["best_t"].astype(np.int64), first_hit=host["first_hit"].astype(np.int64),
               best_state=_unpack(host["best_bits"].view(np.uint32), inst.n),
               final_state=_unpack(host["final_bits"].view(np.uint32), inst.n))
    want = run_library(inst, beta, eta, xi, replicas=R, seed=seed, q=q, target=target)
    for key in ("best_E", "best_t", "first_hit", "final_E", "best_state", "final_state"):
        assert np.array_equal(got[key], want[key]), key


def test_noalloc_rejects_sizes_beyond_the_maximum():
    P = pim()
    inst = sk_pm1(20, 0)
    beta = linear_beta(4)
    dummy = {k: 0 for k in ("best_E", "best_t", "first_hit", "final_E", "best_bits",
                            "final_bits")}
    with pytest.raises(P.PimError) as e:
        P.pim_anneal_noalloc(inst.J, inst.c, beta, eta_power(beta), 0.5, 5000, 0, 0, None, dummy)
    assert e.value.code == P.PIM_ERR_INVALID and "replicas" in str(e.value)
    big = sk_pm1(300, 0)
    with pytest.raises(P.PimError) as e:
        P.pim_anneal_noalloc(big.J, big.c, beta, eta_power(beta), 0.5, 4, 0, 0, None, dummy)
    assert e.value.code == P.PIM_ERR_INVALID
