"""GPU tests of MIMO detection serving: continuous batching with memory admission gives
every request the result it gets alone; the server's path equals the public API's; the
detector beats MMSE and approaches exhaustive ML (BER, synthetic Rayleigh channels)."""
import numpy as np
import pytest

import oracle
from oracle import mimo as om
from workloads import (MIMO_XI, bits_from_symbols, mimo_problem, mimo_scale, mimo_schedule)

from gpu_helpers import pim

pytestmark = pytest.mark.gpu

R = 32


def _server(P, nt, T, **kw):
    beta, eta = mimo_schedule(T)
    return P.pim_mimo_server_create(nt, nt, 16, R, beta, eta, MIMO_XI, mimo_scale(nt), seed=7, **kw)


def _problems(nt, count, snr=None, seed0=0):
    rng = np.random.default_rng(seed0)
    snrs = rng.uniform(10, 25, count) if snr is None else np.full(count, snr)
    return [mimo_problem(nt, nt, 16, float(s), seed0 + k) for k, s in enumerate(snrs)]


def _reg(p):
    return 1.0 / p.es_n0  # the paper's printed MMSE regulariser


def test_same_result_alone_and_in_the_mix():
    P = pim()
    nt, T = 16, 64
    probs = _problems(nt, 24)
    alone = []
    s1 = _server(P, nt, T, max_batch=1, max_inflight=1)
    try:
        for k, p in enumerate(probs):
            t = P.pim_mimo_server_submit(s1, p.H, p.y, _reg(p), k)
            alone.append(P.pim_mimo_server_result(s1, t, nt))
    finally:
        P.pim_mimo_server_destroy(s1)
    s2 = _server(P, nt, T, max_batch=8, max_inflight=3)
    try:
        H = np.stack([p.H for p in probs])
        y = np.stack([p.y for p in probs])
        x, e, lat = P.pim_mimo_server_replay(s2, H, y, [_reg(p) for p in probs],
                                             np.zeros(len(probs)), nt)
        st = P.pim_mimo_server_stats(s2)
    finally:
        P.pim_mimo_server_destroy(s2)
    assert st["mean_batch"] > 1.0 and st["completed"] == len(probs)
    for k in range(len(probs)):
        assert np.array_equal(alone[k][0], x[k]), k
        assert alone[k][1] == e[k], k
    assert np.all(lat > 0)


def test_server_equals_public_api_path():
    """The server's answer equals: formulate, stage, anneal with instance id = request id,
    take the replica of lowest reported energy, reconstruct; the reported energy is that
    state's FP64 energy."""
    P = pim()
    nt, T = 8, 32
    beta, eta = mimo_schedule(T)
    probs = _problems(nt, 6, seed0=50)
    s = P.pim_mimo_server_create(nt, nt, 16, R, beta, eta, MIMO_XI, mimo_scale(nt), seed=7)
    try:
        got = [P.pim_mimo_server_result(s, P.pim_mimo_server_submit(s, p.H, p.y, _reg(p), k), nt)
               for k, p in enumerate(probs)]
    finally:
        P.pim_mimo_server_destroy(s)
    for k, p in enumerate(probs):
        J, h, xm = P.pim_mimo_formulate(p.H, p.y, 16, _reg(p))
        hd = P.pim_create(J, h, mimo_scale(nt))
        try:
            P.pim_set_schedule(hd, beta, eta, MIMO_XI)
            P.pim_anneal(hd, R, T, 7, instance_id=k)
            S = P.pim_best_state(hd, J.shape[0])
            best = int(np.argmin(P.pim_energies(hd)["best_E"]))
        finally:
            P.pim_destroy(hd)
        xh = P.pim_mimo_reconstruct(xm, S[best], 16)
        E64 = oracle.energy(J, h, S[best:best + 1])[0]
        assert np.array_equal(xh, got[k][0]) and np.isclose(E64, got[k][1], rtol=1e-12)


def _ber_run(P, nt, T, probs):
    s = _server(P, nt, T, max_batch=32, max_inflight=4)
    try:
        H = np.stack([p.H for p in probs])
        y = np.stack([p.y for p in probs])
        x, _, _ = P.pim_mimo_server_replay(s, H, y, [_reg(p) for p in probs],
                                           np.zeros(len(probs)), nt)
    finally:
        P.pim_mimo_server_destroy(s)
    return x


def test_beats_mmse_16x16():
    P = pim()
    nt, T = 16, 64
    probs = _problems(nt, 64, snr=15.0, seed0=100)
    x = _ber_run(P, nt, T, probs)
    bits = np.stack([p.bits for p in probs])
    ber_pimi = om.ber(bits, bits_from_symbols(x, 16))
    ber_mmse = om.ber(bits, np.stack([bits_from_symbols(om.mmse(p.H, p.y, _reg(p), 4), 16)
                                      for p in probs]))
    assert ber_pimi < 0.6 * ber_mmse, (ber_pimi, ber_mmse)


def test_4x4_reaches_the_di_mimo_optimum():
    """4x4 16-QAM (16 spins): the server's answer has the exact ground-state energy of the
    DI-MIMO instance (enumerated) in at least 90 % of the problems, and the bit-error rates
    order as ML <= DI-MIMO optimum <= PIMI <= MMSE (the formulation, not the solver, limits
    the gap to ML: its corrections reach one constellation level)."""
    P = pim()
    nt, T = 4, 32
    probs = _problems(nt, 60, snr=10.0, seed0=200)
    s = _server(P, nt, T, max_batch=32, max_inflight=4)
    try:
        H = np.stack([p.H for p in probs])
        y = np.stack([p.y for p in probs])
        x, energy, _ = P.pim_mimo_server_replay(s, H, y, [_reg(p) for p in probs],
                                                np.zeros(len(probs)), nt)
    finally:
        P.pim_mimo_server_destroy(s)
    bits = np.stack([p.bits for p in probs])
    hits, x_opt = 0, []
    for k, p in enumerate(probs):
        xm = om.mmse(p.H, p.y, _reg(p), 4)
        J, h = om.di_mimo(p.H, p.y, xm, [1, 1])
        E_gs, s_gs = oracle.ground_state(J, h)
        hits += energy[k] <= E_gs + 1e-9 * abs(E_gs)
        x_opt.append(om.reconstruct(xm, s_gs, [1, 1], 4))
    ber = {
        "ml": om.ber(bits, np.stack([bits_from_symbols(om.ml_exhaustive(p.H, p.y, 4), 16) for p in probs])),
        "opt": om.ber(bits, bits_from_symbols(np.stack(x_opt), 16)),
        "pimi": om.ber(bits, bits_from_symbols(x, 16)),
        "mmse": om.ber(bits, np.stack([bits_from_symbols(om.mmse(p.H, p.y, _reg(p), 4), 16) for p in probs])),
    }
    assert hits >= 0.9 * len(probs), (hits, ber)
    assert ber["ml"] <= ber["opt"] + 1e-12 and ber["pimi"] <= ber["mmse"] + 1e-12, ber
    assert ber["pimi"] <= ber["opt"] + 0.01, ber


def test_memory_admission_bounds_admitted_bytes():
    P = pim()
    nt, T = 16, 64
    beta, eta = mimo_schedule(T)
    # a budget below one request is raised to exactly one: requests run one at a time
    s = P.pim_mimo_server_create(nt, nt, 16, R, beta, eta, MIMO_XI, mimo_scale(nt), seed=1,
                                 max_batch=16, max_inflight=4, mem_budget=1)
    try:
        one = P.pim_mimo_server_stats(s)  # budget raised to one request at creation
        probs = _problems(nt, 12, seed0=300)
        H = np.stack([p.H for p in probs])
        y = np.stack([p.y for p in probs])
        x, e, lat = P.pim_mimo_server_replay(s, H, y, [_reg(p) for p in probs],
                                             np.zeros(len(probs)), nt)
        st = P.pim_mimo_server_stats(s)
    finally:
        P.pim_mimo_server_destroy(s)
    assert one["completed"] == 0
    assert st["completed"] == 12 and st["mean_batch"] == 1.0
    assert st["p99_us"] >= st["p50_us"] > 0


# ------------------------------------------------ device-side request queue
def test_device_queue_equals_host_batching():
    """The persistent serving kernel fed from the device queue gives every request the same
    detected symbols and energy as host-side batched launches (same couplings, draws and
    decisions), for requests arriving all at once and one by one."""
    P = pim()
    nt, T = 16, 64
    probs = _problems(nt, 40, seed0=100)
    H = np.stack([p.H for p in probs])
    y = np.stack([p.y for p in probs])
    regs = [_reg(p) for p in probs]
    s1 = _server(P, nt, T, max_batch=8, max_inflight=3)
    try:
        x1, e1, _ = P.pim_mimo_server_replay(s1, H, y, regs, np.zeros(len(probs)), nt)
    finally:
        P.pim_mimo_server_destroy(s1)
    # 16 serving CTAs and 32 slots; then one CTA and two slots, so every request reuses a slot
    for batch, inflight in ((8, 2), (1, 1)):
        s2 = _server(P, nt, T, max_batch=batch, max_inflight=inflight, device_queue=True, idle_s=0.5)
        try:
            x2, e2, lat = P.pim_mimo_server_replay(s2, H, y, regs, np.zeros(len(probs)), nt)
            st = P.pim_mimo_server_stats(s2)
            single = []
            for k in (3, 17):
                t = P.pim_mimo_server_submit(s2, probs[k].H, probs[k].y, regs[k], k)
                single.append(P.pim_mimo_server_result(s2, t, nt))
        finally:
            P.pim_mimo_server_destroy(s2)
        assert st["completed"] == len(probs)
        bad = np.nonzero(np.any(x1 != x2, axis=1) | (e1 != e2))[0]
        assert bad.size == 0, (batch, inflight, bad)
        assert np.all(lat > 0)
        for (xs, es, _), k in zip(single, (3, 17)):
            assert np.array_equal(xs, x1[k]) and es == e1[k]


def test_device_queue_idle_wait_runs_out_and_the_kernel_comes_back():
    """With no request for idle_s the serving kernel's bounded wait runs out: it ends and the
    host sees PIM_ERR_TIMEOUT; the next requests launch it again and are served."""
    P = pim()
    nt, T = 16, 64
    probs = _problems(nt, 6, seed0=200)
    ref = []
    s1 = _server(P, nt, T, max_batch=4, max_inflight=1)
    try:
        for k, p in enumerate(probs):
            ref.append(P.pim_mimo_server_result(s1, P.pim_mimo_server_submit(s1, p.H, p.y, _reg(p), k), nt))
    finally:
        P.pim_mimo_server_destroy(s1)
    s2 = _server(P, nt, T, max_batch=4, max_inflight=1, device_queue=True, idle_s=0.05)
    try:
        got = []
        for k, p in enumerate(probs[:3]):
            got.append(P.pim_mimo_server_result(s2, P.pim_mimo_server_submit(s2, p.H, p.y, _reg(p), k), nt))
        assert P.pim_mimo_server_idle_wait(s2, 5.0) == P.PIM_ERR_TIMEOUT
        for k, p in enumerate(probs[3:], start=3):
            got.append(P.pim_mimo_server_result(s2, P.pim_mimo_server_submit(s2, p.H, p.y, _reg(p), k), nt))
        assert P.pim_mimo_server_idle_wait(s2, 5.0) == P.PIM_ERR_TIMEOUT
    finally:
        P.pim_mimo_server_destroy(s2)
    for (x, e, _), (xr, er, _) in zip(got, ref):
        assert np.array_equal(x, xr) and e == er


def test_device_queue_limits():
    P = pim()
    with pytest.raises(P.PimError) as e:
        _server(P, 65, 8, max_batch=1, max_inflight=1, device_queue=True)  # n = 260 spins
    assert e.value.code == P.PIM_ERR_UNSUPPORTED
    s = _server(P, 4, 8, max_batch=1, max_inflight=1)
    try:
        with pytest.raises(P.PimError) as e:
            P.pim_mimo_server_idle_wait(s, 0.01)
        assert e.value.code == P.PIM_ERR_UNSUPPORTED
    finally:
        P.pim_mimo_server_destroy(s)
