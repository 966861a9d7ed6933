"""GPU tests of the sequential (conventional PIM) path and of the paper's comparison of
update schemes, through the C ABI:
  * sequential sweeps (Eq. 3, and Eq. 4 evaluated sequentially) are bit-exact against the
    oracle's sequential sweeps;
  * on the GPU, naive parallel updates (xi = 0) fail where sequential updates and parallel
    updates with inertia succeed (Fig. 1c, qualitatively);
  * the neighbour-triggered flip rate of GPU trajectories falls as xi grows (the
    supplementary section on coupled oscillations)."""
import numpy as np
import pytest

import oracle
from workloads import Instance, eta_power, linear_beta, maxcut_er, random_spins, sk_pm1

from gpu_helpers import assert_same, collect, pim

pytestmark = pytest.mark.gpu

CASES = [
    # kind, n, R, sweeps, xi, noise
    ("maxcut", 20, 37, 12, 0.0, "uniform"),
    ("sk", 100, 64, 8, 0.0, "uniform"),
    ("sk", 130, 33, 6, 0.5, "gauss"),
    ("maxcut", 300, 20, 4, 0.7, "gauss"),
    ("sk", 700, 9, 2, 0.0, "uniform"),
]


def _inst(kind, n, seed):
    return sk_pm1(n, seed) if kind == "sk" else maxcut_er(n, seed)


def _run_seq(inst, beta, eta, xi, noise, R, seed, q=0, init=None, target=None, h=None):
    P = pim()
    hd = P.pim_create(inst.J, h, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, xi, noise)
        P.pim_anneal_sequential(hd, R, len(beta), seed, instance_id=q, init_spins=init,
                                target=target)
        return collect(hd, inst.n)
    finally:
        P.pim_destroy(hd)


@pytest.mark.parametrize("kind,n,R,T,xi,noise", CASES)
def test_sequential_matches_oracle(kind, n, R, T, xi, noise):
    inst = _inst(kind, n, 3)
    beta = linear_beta(T)
    eta = eta_power(beta)
    got = _run_seq(inst, beta, eta, xi, noise, R, seed=5, q=4, target=-0.4 * n)
    want = oracle.anneal_sequential_sweeps(inst.J, inst.h, inst.c, beta, eta, xi, replicas=R,
                                           seed=5, q=4, target=-0.4 * n, noise=noise)
    assert_same(got, want, label=f"{kind} n={n}")


def test_sequential_bias_host_init_and_resume():
    """Non-zero h, host-given spins, and a run split in two with PIM_CONTINUE."""
    P = pim()
    base = sk_pm1(90, 2)
    h = np.random.default_rng(1).integers(-4, 5, 90).astype(np.int32)
    inst = Instance("sk", 90, base.J, h, base.c, 2)
    T = 10
    beta = linear_beta(T)
    eta = eta_power(beta)
    init = random_spins(90, 21, seed=8)
    want = oracle.anneal_sequential_sweeps(inst.J, inst.h, inst.c, beta, eta, 0.3, replicas=21,
                                           seed=6, init=init, noise="gauss")
    hd = P.pim_create(inst.J, inst.h, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.3, "gauss")
        P.pim_anneal_sequential(hd, 21, 4, 6, init_spins=init)
        P.pim_anneal_sequential(hd, 21, 6, 6, t_begin=4, flags=P.PIM_CONTINUE)
        assert_same(collect(hd, 90), want, label="sequential resume")
    finally:
        P.pim_destroy(hd)


def test_update_schemes_on_gpu():
    """Max-Cut N = 100, equal schedules and sweeps: naive parallel updates (xi = 0) reach
    far higher energies than sequential updates, while parallel updates with inertia
    (xi = 0.7) come close to the sequential result."""
    P = pim()
    n, R, T = 100, 256, 300
    beta = linear_beta(T)
    eta = eta_power(beta)
    means = {}
    for seed in range(3):
        inst = maxcut_er(n, seed)
        hd = P.pim_create(inst.J, None, inst.c)
        try:
            for name, xi, seq in (("naive", 0.0, False), ("pimi", 0.7, False), ("seq", 0.0, True)):
                P.pim_set_schedule(hd, beta, eta, xi, "uniform" if seq else "gauss")
                if seq:
                    P.pim_anneal_sequential(hd, R, T, seed)
                else:
                    P.pim_anneal(hd, R, T, seed)
                means.setdefault(name, []).append(P.pim_energies(hd)["best_E"].mean())
        finally:
            P.pim_destroy(hd)
    naive, pimi, seq = (np.mean(means[k]) for k in ("naive", "pimi", "seq"))
    assert naive > 0.5 * seq, (naive, pimi, seq)   # energies are negative: naive is far worse
    assert pimi < 0.9 * seq, (naive, pimi, seq)    # inertia brings parallel updates close


def test_flip_rate_of_gpu_trajectories_falls_with_inertia():
    """P_NT of trajectories produced on the GPU one sweep at a time (PIM_CONTINUE) falls
    as xi grows."""
    P = pim()
    n, R, T = 60, 64, 60
    inst = maxcut_er(n, 9)
    beta = linear_beta(T)
    eta = eta_power(beta)
    rates = []
    for xi in (0.0, 0.2, 0.5, 0.8):
        hd = P.pim_create(inst.J, None, inst.c)
        try:
            P.pim_set_schedule(hd, beta, eta, xi)
            P.pim_anneal(hd, R, 0, 1)
            states = [P.pim_final_state(hd, n)]
            for t in range(T):
                P.pim_anneal(hd, R, 1, 1, t_begin=t, flags=P.PIM_CONTINUE)
                states.append(P.pim_final_state(hd, n))
        finally:
            P.pim_destroy(hd)
        rates.append(oracle.neighbour_triggered_flip_rate(inst.J, np.stack(states)).mean())
    assert all(a > b for a, b in zip(rates, rates[1:])), rates
    assert rates[-1] < 0.3 * rates[0], rates
