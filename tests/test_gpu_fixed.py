"""GPU tests of the fixed-point datapath mode (pim_set_schedule_fixed): bit-exact against
the oracle's ap_fixed<W, I> decision on every kernel, and the device tables equal the
oracle's quantized decision for every (step, field, spin, key)."""
import numpy as np
import pytest

import oracle
from oracle import pimi
from workloads import eta_power, linear_beta, maxcut_er, sk_pm1

from gpu_helpers import assert_same, collect, pim

pytestmark = pytest.mark.gpu

CASES = [
    # kind, n, R, sweeps, (W, I), act, flags
    ("maxcut", 100, 64, 60, (4, 2), "tanh", 0),
    ("sk", 200, 130, 30, (4, 2), "lut", 0),
    ("sk", 150, 40, 40, (6, 2), "tanh", 0),
    ("maxcut", 90, 50, 40, (16, 4), "tanh", 0),
    ("sk", 300, 70, 10, (4, 2), "tanh", 4),   # persistent mid-N kernel
    ("sk", 300, 70, 10, (5, 2), "lut", 8),    # large-N kernel
]


@pytest.mark.parametrize("kind,n,R,T,fmt,act,flags", CASES)
def test_fixed_point_matches_oracle(kind, n, R, T, fmt, act, flags):
    P = pim()
    inst = sk_pm1(n, 4) if kind == "sk" else maxcut_er(n, 4)
    beta = linear_beta(T)
    eta = eta_power(beta)
    xi = 0.5 if kind == "sk" else 0.7
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule_fixed(hd, beta, eta, xi, fmt[0], fmt[1], act=act, lut_levels=8)
        P.pim_anneal(hd, R, T, 6, instance_id=2, target=-0.5 * n, flags=flags)
        got = collect(hd, n)
    finally:
        P.pim_destroy(hd)
    want = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, xi, replicas=R, seed=6, q=2,
                         target=-0.5 * n, act=act, lut_levels=8, fixed=fmt)
    assert_same(got, want, label=f"{kind} n={n} fmt={fmt} {act}")


@pytest.mark.parametrize("fmt,act", [((4, 2), "tanh"), ((6, 3), "lut"), ((12, 4), "tanh")])
def test_fixed_point_tables_exhaustive(fmt, act):
    P = pim()
    inst = sk_pm1(40, 0)
    T = 6
    beta = linear_beta(T, 0.05, 4.0)
    eta = eta_power(beta)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule_fixed(hd, beta, eta, 0.5, fmt[0], fmt[1], act=act, lut_levels=4)
        tab, imax = P.pim_thresholds(hd)
    finally:
        P.pim_destroy(hd)
    Q = pimi.gaussian_quantiles()
    I = np.arange(-imax, imax + 1)
    m = np.arange(4096)
    for t in range(T):
        for s, shift in ((-1, 0), (1, 16)):
            M = (tab[t, : I.size] >> shift) & 0xFFFF
            dec = oracle.decide_fixed(np.repeat(I[:, None], 4096, 1), np.full((I.size, 4096), s),
                                      inst.c, beta[t], 0.5, eta[t], np.broadcast_to(Q, (I.size, 4096)),
                                      fmt[0], fmt[1], act, 4)
            assert np.array_equal(dec > 0, m[None, :] >= M[:, None]), (t, s)


# ------------------------------------------------ real couplings (the MIMO datapath)
def _mimo16(seed):
    from oracle import mimo as om
    from workloads import mimo_problem, mimo_scale
    mp = mimo_problem(16, 16, 16, 12.0, seed)
    xm = om.mmse(mp.H, mp.y, 1.0 / mp.es_n0, 4)
    J, h = om.di_mimo(mp.H, mp.y, xm, [1, 1])
    return J, h, mimo_scale(16)


REAL_CASES = [
    # name, (W, I), act, lut levels, R, sweeps
    ("mimo16x16", (16, 4), "tanh", 4, 64, 64),
    ("mimo16x16", (10, 4), "lut", 8, 40, 50),
    ("mimo16x16", (6, 3), "tanh", 4, 32, 40),
    ("gauss100_bias", (12, 4), "tanh", 4, 130, 30),
]


@pytest.mark.parametrize("name,fmt,act,L,R,T", REAL_CASES)
def test_fixed_point_real_couplings_match_oracle(name, fmt, act, L, R, T):
    """Real couplings in ap_fixed<W, I> (J_q = Q(c J), h_q = Q(c h), every datapath value
    quantized): the fields are exact, so states, steps and the (exact) energies of the
    quantized problem equal the oracle's run of the same datapath bit for bit."""
    from workloads import maxcut_gauss
    P = pim()
    if name.startswith("mimo"):
        J, h, c = _mimo16(5)
        xi = 1.0
    else:
        g = maxcut_gauss(100, 2)
        J, c = g.J, g.c
        h = 0.3 * np.random.default_rng(1).standard_normal(100)
        xi = 0.7
    beta = linear_beta(T)
    eta = eta_power(beta)
    Jq = pimi.quantize(c * J, *fmt)
    hq = pimi.quantize(c * h, *fmt)
    target = float(np.median(oracle.energy(Jq, hq, np.ones((1, J.shape[0]), np.int8))) - 1.0)
    hd = P.pim_create(J, h, c)
    try:
        P.pim_set_schedule_fixed(hd, beta, eta, xi, fmt[0], fmt[1], act=act, lut_levels=L)
        P.pim_anneal(hd, R, T, 9, instance_id=4, target=target)
        e = P.pim_energies(hd)
        got = dict(best_E=e["best_E"], best_t=e["best_t"].astype(np.int64),
                   first_hit=e["first_hit"].astype(np.int64), final_E=e["final_E"],
                   best_state=P.pim_best_state(hd, J.shape[0]),
                   final_state=P.pim_final_state(hd, J.shape[0]))
    finally:
        P.pim_destroy(hd)
    want = oracle.anneal(Jq, hq, 1.0, beta, eta, xi, replicas=R, seed=9, q=4, target=target,
                         act=act, lut_levels=L, fixed=fmt)
    assert_same(got, want, label=f"{name} fmt={fmt} {act}")


def test_fixed_point_real_rejects_large_n():
    from workloads import maxcut_gauss
    P = pim()
    g = maxcut_gauss(200, 0)
    hd = P.pim_create(g.J, None, g.c)
    try:
        beta = linear_beta(4)
        with pytest.raises(P.PimError) as e:
            P.pim_set_schedule_fixed(hd, beta, eta_power(beta), 0.7, 16, 4)
        assert e.value.code == P.PIM_ERR_UNSUPPORTED
    finally:
        P.pim_destroy(hd)
