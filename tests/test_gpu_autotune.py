"""Autotuned batch plans: pim_batch_create measures each new shape class (fused and mid-N
units, large-N instance sweeps at both tile widths) and routes with the measured times.
Every candidate kernel is the same computation, so a tuned plan must give the results of
the cost-model plan and of the oracle bit for bit, whatever it chose."""
import numpy as np
import pytest

import oracle
from workloads import eta_power, linear_beta, maxcut_er, sk_pm1

from gpu_helpers import KEYS, collect, pim

pytestmark = pytest.mark.gpu


def _batch_results(P, insts, reps, T, mode):
    P.pim_autotune(mode)
    beta = linear_beta(T)
    eta = eta_power(beta)
    hds = [P.pim_create(i.J, None, i.c) for i in insts]
    try:
        for hd, i in zip(hds, insts):
            P.pim_set_schedule(hd, beta, eta, 0.5 if i.kind == "sk" else 0.7)
        b = P.pim_batch_create(hds, reps, instance_ids=list(range(10, 10 + len(insts))))
        try:
            P.pim_batch_run(b, T, seed=3)
            out = [collect(hd, i.n) for hd, i in zip(hds, insts)]
        finally:
            P.pim_batch_destroy(b)
    finally:
        for hd in hds:
            P.pim_destroy(hd)
        P.pim_autotune(1)
    return out


def test_autotuned_plan_equals_cost_model_plan_and_oracle():
    P = pim()
    insts = [sk_pm1(64, 1), maxcut_er(200, 2), sk_pm1(512, 3), maxcut_er(700, 4), sk_pm1(1100, 5)]
    reps = [200, 130, 256, 96, 128]
    T = 40
    tuned = _batch_results(P, insts, reps, T, 1)
    report = P.pim_tune_report()
    for kind in ("|fused|", "|mid|", "|big|"):
        assert kind in report, report
    model = _batch_results(P, insts, reps, T, 0)
    for k, (a, b) in enumerate(zip(tuned, model)):
        for key in KEYS:
            assert np.array_equal(a[key], b[key]), (k, key)
    beta = linear_beta(T)
    eta = eta_power(beta)
    for k in (0, 2, 4):  # oracle on a replica subset of some instances
        i = insts[k]
        rows = [0, reps[k] - 1]
        want = oracle.anneal(i.J, i.h, i.c, beta, eta, 0.5 if i.kind == "sk" else 0.7,
                             replica_ids=rows, seed=3, q=10 + k)
        for key in KEYS:
            assert np.array_equal(np.asarray(tuned[k][key])[rows], want[key]), (k, key)


def test_tune_report_lines_parse():
    P = pim()
    for line in P.pim_tune_report().strip().splitlines():
        key, us = line.rsplit(" ", 1)
        assert len(key.split("|")) == 6 and float(us) > 0.0
