"""Qualitative claims of the paper, checked on the oracle with synthetic instances (the
paper prints no per-instance values to compare with):
  * with fully parallel updates, the inertia term lets the machine reach low energies
    that the same schedule without inertia (naive parallel PIM) does not;
  * the neighbour-triggered flip rate P_NT falls as the inertia xi grows.
"""
import numpy as np

import oracle
from workloads import eta_power, linear_beta, maxcut_er


def test_inertia_beats_naive_parallel_updates():
    n, R, T = 40, 48, 400
    beta = linear_beta(T)
    eta = eta_power(beta)
    succ = {0.0: [], 0.7: []}
    for seed in range(4):
        inst = maxcut_er(n, seed)
        runs = {xi: oracle.anneal(inst.J, inst.h, inst.c, beta, eta, xi, replicas=R, seed=seed)
                for xi in succ}
        best = min(r["best_E"].min() for r in runs.values())
        for xi, r in runs.items():
            succ[xi].append(np.mean(r["best_E"] <= 0.999 * best))
    p0, p7 = np.mean(succ[0.0]), np.mean(succ[0.7])
    assert p7 > 0.3 and p7 > 3 * p0, (p0, p7)


def test_flip_rate_falls_with_inertia():
    n, R, T = 40, 32, 150
    inst = maxcut_er(n, 7)
    beta = linear_beta(T)
    eta = eta_power(beta)
    rates = []
    for xi in (0.0, 0.2, 0.5, 0.8):
        out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, xi, replicas=R, seed=1,
                            record_states=True)
        rates.append(oracle.neighbour_triggered_flip_rate(inst.J, out["states"]).mean())
    assert all(a > b for a, b in zip(rates, rates[1:])), rates
    assert rates[-1] < 0.25 * rates[0], rates


def test_flip_rate_definition_on_a_hand_case():
    """Path 0-1-2: step 1 flips spins 0 and 1 -> events: spin 1 (neighbour 0 flipped, 1
    flipped), spin 0 (neighbour 1 flipped, flipped), spin 2 (neighbour 1 flipped, not
    flipped) -> 2/3; step 2 flips nothing -> 0."""
    J = np.array([[0, -1, 0], [-1, 0, -1], [0, -1, 0]])
    states = np.array([[[1, 1, 1]], [[-1, -1, 1]], [[-1, -1, 1]]], dtype=np.int8)
    r = oracle.neighbour_triggered_flip_rate(J, states)
    assert np.allclose(r, [2 / 3, 0.0])
