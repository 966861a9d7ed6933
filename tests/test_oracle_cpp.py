"""The plain C++17 oracle (oracle/pimi_ref.cpp) against the pinned numpy oracle.

The C++ oracle is a second, independent statement of the update rule (it is what the
benchmark times as the CPU baseline).  Its Philox generator is pinned to the published
known-answer vectors, its noise levels to the numpy tables (scipy's ndtri), and whole
anneals to the numpy oracle bit for bit on integer couplings (Gaussian and uniform noise,
tanh and LUT activation, bias, given initial spins, targets, replica subsets, resume, any
thread count), and within float64 rounding on real couplings.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import cpp
from workloads import eta_power, linear_beta, maxcut_er, maxcut_gauss, random_spins, sk_pm1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KEYS = ("best_E", "best_t", "first_hit", "final_E", "best_state", "final_state")


def _same(a, b, label=""):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), f"{label}: {k}"


def test_cpp_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [[int(x, 16) for x in line.split()] for line in f
                if line.strip() and not line.startswith("#")]
    for row in rows:
        assert cpp.philox4x32_10(row[0:4], row[4], row[5]) == row[6:10]


def test_cpp_noise_levels_equal_the_numpy_tables():
    assert np.array_equal(cpp.noise_levels("gauss"), oracle.gaussian_quantiles())
    assert np.array_equal(cpp.noise_levels("uniform"), oracle.uniform_levels())


@pytest.mark.parametrize("case", ["sk_gauss_tanh", "maxcut_uniform_lut_bias", "init_target"])
def test_cpp_anneal_equals_numpy_oracle(case):
    if case == "sk_gauss_tanh":
        inst = sk_pm1(37, 4)
        beta = linear_beta(60)
        kw = dict(replicas=9, seed=0x1234_5678_9ABC, q=5, target=-120)
        args = (inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5)
    elif case == "maxcut_uniform_lut_bias":
        inst = maxcut_er(30, 2)
        h = (np.arange(30) % 5 - 2).astype(np.int32)
        beta = linear_beta(45)
        kw = dict(replicas=7, seed=3, q=1, noise="uniform", act="lut", lut_levels=8)
        args = (inst.J, h, inst.c, beta, eta_power(beta), 0.7)
    else:
        inst = sk_pm1(20, 9)
        beta = linear_beta(40)
        init = random_spins(20, 6, 3)
        kw = dict(replicas=6, seed=11, q=2, init=init, target=-30)
        args = (inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5)
    want = oracle.anneal(*args, **kw)
    for threads in (1, 4):
        got = cpp.anneal(*args, threads=threads, **kw)
        _same(got, want, f"{case}, {threads} threads")


def test_cpp_replica_subset_and_resume():
    inst = maxcut_er(24, 6)
    beta = linear_beta(50)
    eta = eta_power(beta)
    full = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, replicas=10, seed=2, q=3,
                         target=-40)
    sub = cpp.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, replica_ids=[1, 8, 9], seed=2, q=3,
                     target=-40)
    for k in KEYS:
        assert np.array_equal(np.asarray(full[k])[[1, 8, 9]], sub[k]), k
    part = cpp.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, replicas=10, seed=2, q=3,
                      target=-40, sweeps=17)
    rest = cpp.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, replicas=10, seed=2, q=3,
                      target=-40, t_begin=17, sweeps=33, prev=part)
    _same(rest, full, "resume")


def test_cpp_real_couplings_match_within_rounding():
    """Real couplings: both oracles form the fields in float64 in different summation orders,
    so energies agree to rounding; on a short run the decisions (float32, far from their
    thresholds in all but rare cases) and hence the states agree."""
    inst = maxcut_gauss(40, 1)
    beta = linear_beta(12)
    eta = eta_power(beta)
    J = oracle.round_bf16(inst.J)
    want = oracle.anneal(J, inst.h, inst.c, beta, eta, 0.7, replicas=8, seed=5)
    got = cpp.anneal(J, inst.h, inst.c, beta, eta, 0.7, replicas=8, seed=5)
    scale = np.abs(J).sum() / 2
    assert np.allclose(got["best_E"], want["best_E"], rtol=0, atol=1e-12 * scale)
    assert np.allclose(got["final_E"], want["final_E"], rtol=0, atol=1e-12 * scale)
    assert np.array_equal(got["final_state"], want["final_state"])
    assert np.array_equal(got["best_t"], want["best_t"])
