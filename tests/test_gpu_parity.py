"""GPU parity: every sweep kernel (fused n <= 256, persistent mid-N, large-N cooperative)
and the plain FP32 path, called through the C ABI, against the CPU oracle -- bit-exact on
integer instances (spins, energies, steps)."""
import math

import numpy as np
import pytest

import oracle
from oracle import pimi
from workloads import (Instance, eta_power, linear_beta, maxcut_er, random_spins, sk_batch,
                       sk_pm1)

from gpu_helpers import assert_same, collect, oracle_run, pim, run_library

pytestmark = pytest.mark.gpu

# library's choice, plain FP32 path (PIM_PATH_FP32REF), persistent mid-N kernel for every
# integer n <= 1024 (PIM_PATH_MID), large-N kernel for every n > 256 (PIM_PATH_BIG: the
# coupling-resident E2M1 variant where the couplings allow it), large-N kernel with FP8
# couplings streamed every sweep (PIM_PATH_BIG | PIM_PATH_FP8)
PATHS = [0, 2, 4, 8, 8 | 32]

CASES = [
    # kind, n, replicas, sweeps, seed
    ("maxcut", 20, 32, 50, 1),
    ("sk", 1, 5, 7, 0),         # degenerate: no couplings, pure noise
    ("sk", 17, 40, 40, 2),      # ragged spins and replicas
    ("maxcut", 60, 70, 40, 9),  # last 16-spin chunk holds 12 spins
    ("sk", 100, 128, 80, 3),
    ("maxcut", 128, 96, 30, 4),  # exactly one K block
    ("sk", 129, 130, 25, 5),    # just past one K block and one replica tile
    ("sk", 200, 200, 60, 6),    # two K blocks, ragged replica tile
    ("maxcut", 256, 64, 20, 7),  # largest fused size
    ("sk2", 150, 140, 30, 8),   # couplings +-2: field range past 255, general-bias kernel
    ("sk", 300, 200, 25, 10),   # large-N kernel: 6 column blocks x 2 replica tiles
    ("maxcut", 520, 129, 15, 11),  # large-N kernel: ragged spins (last block) and replicas
    ("sk", 700, 257, 6, 14),    # three replica panels, ragged last chunk
    ("sk", 1000, 100, 8, 12),   # largest mid-N image (npad 1024), ragged
    ("maxcut", 1024, 130, 6, 13),  # exactly npad 1024
    ("sk", 1025, 64, 4, 15),    # past the mid-N limit: large-N kernel on every path
    # mid-N diagonal-encoded decisions from an E5M2 image with 2^k > field bound on the
    # diagonal: 256 (Max-Cut N = 300), 2048 (couplings +-2, N = 600); couplings with an odd
    # |J| > 8 have no E5M2 encoding and take the general table
    ("maxcut", 300, 64, 12, 18),
    ("sk2", 600, 130, 10, 16),
    ("sk9", 400, 96, 10, 17),
    # coupling-resident E2M1 variant: every E2M1 integer magnitude (1, 2, 3, 4, 6); 9
    # K-blocks of 256 spins (odd: the last ring stage holds one) with the threshold table in
    # shared memory; npad 3072 (12 K-blocks)
    ("sk12346", 700, 130, 8, 19),
    ("sk", 2100, 70, 4, 20),
    ("maxcut", 3000, 40, 3, 21),
]


def _inst(kind, n, seed):
    if kind == "sk2":
        base = sk_pm1(n, seed)
        return Instance("sk", n, (2 * base.J).astype(np.int8), base.h, base.c / 2, seed)
    if kind == "sk9":
        base = sk_pm1(n, seed)
        J = base.J.astype(np.int8).copy()
        i = np.arange(0, n - 1, 7)
        J[i, i + 1] = J[i + 1, i] = 9 * J[i, i + 1]
        return Instance("sk", n, J, base.h, base.c, seed)
    if kind == "sk12346":
        base = sk_pm1(n, seed)
        rng = np.random.default_rng(seed)
        mult = rng.choice(np.array([1, 2, 3, 4, 6], np.int8), size=(n, n))
        mult = np.triu(mult, 1)
        mult = mult + mult.T
        J = (base.J.astype(np.int16) * mult).astype(np.int8)
        return Instance("sk", n, J, base.h, base.c / 3, seed)
    return sk_pm1(n, seed) if kind == "sk" else maxcut_er(n, seed)


@pytest.mark.parametrize("flags", PATHS)
@pytest.mark.parametrize("kind,n,R,T,seed", CASES)
def test_matches_oracle(kind, n, R, T, seed, flags):
    inst = _inst(kind, n, seed)
    beta = linear_beta(T)
    eta = eta_power(beta)
    xi = 0.5 if kind == "sk" else 0.7
    target = -0.5 * n
    got = run_library(inst, beta, eta, xi, replicas=R, seed=seed * 7 + 1, q=3, target=target,
                      flags=flags)
    want = oracle_run(inst, beta, eta, xi, replicas=R, seed=seed * 7 + 1, q=3, target=target)
    assert_same(got, want, label=f"{kind} n={n} path={flags}")


@pytest.mark.parametrize("flags", [0, 2, 4])
def test_bias_uniform_noise_lut_and_host_init(flags):
    """Non-zero h, Eq. 3 uniform noise, the 4-level LUT activation and host-given spins."""
    inst = sk_pm1(70, 11)
    rng = np.random.default_rng(5)
    inst = Instance("sk", 70, inst.J, rng.integers(-4, 5, 70).astype(np.int32), inst.c, 11)
    T = 40
    beta = linear_beta(T, 0.2, 2.0)
    eta = np.full(T, 0.6, np.float32)
    init = random_spins(70, 33, seed=4)
    for noise, act in (("uniform", "tanh"), ("gauss", "lut")):
        got = run_library(inst, beta, eta, 0.3, replicas=33, seed=9, init=init, noise=noise,
                          act=act, lut_levels=4, flags=flags, target=-100)
        want = oracle_run(inst, beta, eta, 0.3, replicas=33, seed=9, init=init, noise=noise,
                          act=act, lut_levels=4, target=-100)
        assert_same(got, want, label=f"{noise}/{act} path={flags}")


@pytest.mark.parametrize("flags", [0, 2, 4])
def test_resume_matches_uninterrupted(flags):
    P = pim()
    inst = maxcut_er(60, 3)
    beta = linear_beta(90)
    eta = eta_power(beta)
    full = oracle_run(inst, beta, eta, 0.7, replicas=50, seed=2, target=-300)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.7)
        P.pim_anneal(hd, 50, 41, 2, target=-300, flags=flags)
        P.pim_anneal(hd, 50, 49, 2, t_begin=41, target=-300, flags=flags | P.PIM_CONTINUE)
        assert_same(collect(hd, 60), full, label="resume")
    finally:
        P.pim_destroy(hd)


def test_zero_sweeps_reports_initial_state():
    inst = sk_pm1(33, 1)
    beta = linear_beta(10)
    got = run_library(inst, beta, eta_power(beta), 0.5, replicas=10, sweeps=0, seed=4)
    want = oracle_run(inst, beta, eta_power(beta), 0.5, replicas=10, sweeps=0, seed=4)
    assert_same(got, want)
    assert np.all(got["best_t"] == 0)


def test_thresholds_equal_direct_evaluation_exhaustively():
    """Every entry of the device decision table equals the oracle's direct float32 decision
    for every key m in [0, 4096), both spins and every field of the table."""
    P = pim()
    inst = sk_pm1(40, 0)
    T = 12
    beta = linear_beta(T, 0.05, 4.0)
    eta = eta_power(beta)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.5)
        tab, imax = P.pim_thresholds(hd)
    finally:
        P.pim_destroy(hd)
    Q = pimi.gaussian_quantiles()
    I = np.arange(-imax, imax + 1)
    m = np.arange(4096)
    for t in range(T):
        b = np.float32(np.float64(beta[t]) * inst.c)
        tau = oracle.activation(b, I)
        for s, shift in ((-1, 0), (1, 16)):
            M = (tab[t, : I.size] >> shift) & 0xFFFF
            dec = pimi.decide(np.repeat(tau[:, None], 4096, 1), np.full((I.size, 4096), s), 0.5,
                              eta[t], np.broadcast_to(Q, (I.size, 4096)))
            assert np.array_equal(dec > 0, m[None, :] >= M[:, None]), (t, s)


def test_batch_equals_per_instance_oracle():
    """One launch over several instances (different n and R, both kernel sizes) gives each
    instance exactly its own oracle run with counter word q = its instance id."""
    P = pim()
    insts = [sk_pm1(200, 0), maxcut_er(100, 1), sk_pm1(150, 2), maxcut_er(37, 3)]
    reps = [300, 64, 129, 20]
    ids = [10, 11, 12, 13]
    T = 30
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.6)
        targets = [-1000.0, -150.0, -1000.0, -40.0]
        P.pim_anneal_batch(handles, reps, T, seed=77, instance_ids=ids, targets=targets)
        for hd, inst, R, q, tg in zip(handles, insts, reps, ids, targets):
            want = oracle_run(inst, beta, eta, 0.6, replicas=R, seed=77, q=q, target=tg)
            assert_same(collect(hd, inst.n), want, label=f"n={inst.n}")
    finally:
        for hd in handles:
            P.pim_destroy(hd)


@pytest.mark.parametrize("flags", [0, 4])
def test_uneven_batch_equals_per_instance_oracle(flags):
    """Instances of uneven size (n = 20 .. 1100) and replica count (32 .. 300), Max-Cut and
    SK mixed, in one call: the library's routing (fused / persistent / large-N) or every
    n <= 1024 on the persistent kernel; each instance is exactly its own oracle run."""
    P = pim()
    rng = np.random.default_rng(42)
    sizes = [20, 1100, 300, 96, 640, 257, 1000, 150, 513, 64]
    insts = [(sk_pm1 if k % 2 else maxcut_er)(n, 100 + k) for k, n in enumerate(sizes)]
    reps = [int(x) for x in rng.choice([32, 64, 96, 160, 224, 300], size=len(sizes))]
    ids = list(range(50, 50 + len(sizes)))
    T = 12
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.6)
        targets = [-0.4 * i.n for i in insts]
        P.pim_anneal_batch(handles, reps, T, seed=5, instance_ids=ids, targets=targets,
                           flags=flags)
        for hd, inst, R, q, tg in zip(handles, insts, reps, ids, targets):
            want = oracle_run(inst, beta, eta, 0.6, replicas=R, seed=5, q=q, target=tg)
            assert_same(collect(hd, inst.n), want, label=f"n={inst.n} R={R}")
    finally:
        for hd in handles:
            P.pim_destroy(hd)


def test_persistent_kernel_more_units_than_sms():
    """More (instance, panel) units than resident CTAs: every CTA of the persistent mid-N
    kernel takes several units in turn; sampled replicas of every instance are bit-exact."""
    P = pim()
    insts = [sk_pm1(300 + 7 * k, 200 + k) for k in range(40)]
    R, T = 512, 6
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal_batch(handles, R, T, seed=9, flags=P.PIM_PATH_MID)
        rows = [0, 200, 511]
        for q in range(0, 40, 3):
            got = collect(handles[q], insts[q].n)
            want = oracle_run(insts[q], beta, eta, 0.5, replica_ids=rows, seed=9, q=q)
            assert_same(got, want, rows=rows, label=f"q={q}")
            J, h = insts[q].J, insts[q].h
            assert np.array_equal(oracle.energy(J, h, got["final_state"]), got["final_E"])
    finally:
        for hd in handles:
            P.pim_destroy(hd)


def test_maxcut_n100_full_run_matches_oracle():
    """Max-Cut N = 100 (ER p = 0.5), 64 replicas x 1000 sweeps, linear beta 0.1 -> 3,
    seed 0: the whole run, every replica."""
    inst = maxcut_er(100, 0)
    T = 1000
    beta = linear_beta(T)
    eta = eta_power(beta)
    got = run_library(inst, beta, eta, 0.7, replicas=64, seed=0)
    want = oracle_run(inst, beta, eta, 0.7, replicas=64, seed=0)
    assert_same(got, want, label="maxcut-100")


def test_sk200_batch_full_size_sampled():
    """SK N = 200: 100 instances x 1024 replicas x 2000 sweeps in one launch (the
    configuration the bench times).  Sampled replicas are compared with the oracle bit for
    bit; every replica is checked for the energy identities."""
    P = pim()
    insts = sk_batch(200, 100)
    T, R = 2000, 1024
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal_batch(handles, R, T, seed=0)
        for q in (0, 57, 99):
            got = collect(handles[q], 200)
            rows = [0, 127, 128, 1023]
            want = oracle_run(insts[q], beta, eta, 0.5, replica_ids=rows, seed=0, q=q)
            assert_same(got, want, rows=rows, label=f"q={q}")
        for q in range(0, 100, 9):
            got = collect(handles[q], 200)
            J, h = insts[q].J, insts[q].h
            assert np.array_equal(oracle.energy(J, h, got["best_state"]), got["best_E"])
            assert np.array_equal(oracle.energy(J, h, got["final_state"]), got["final_E"])
            assert np.all(got["best_E"] <= got["final_E"])
            assert np.all((got["best_t"] >= 0) & (got["best_t"] <= T))
    finally:
        for hd in handles:
            P.pim_destroy(hd)


def test_errors_are_reported():
    P = pim()
    inst = sk_pm1(30, 0)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        with pytest.raises(P.PimError) as e:
            P.pim_anneal(hd, 4, 5, 0)
        assert e.value.code == P.PIM_ERR_STATE  # no schedule
        P.pim_set_schedule(hd, linear_beta(10), eta_power(linear_beta(10)), 0.5)
        with pytest.raises(P.PimError) as e:
            P.pim_anneal(hd, 4, 11, 0)
        assert e.value.code == P.PIM_ERR_INVALID  # more sweeps than schedule steps
        with pytest.raises(P.PimError) as e:
            P.pim_anneal(hd, 4, 3, 0, flags=P.PIM_CONTINUE)
        assert e.value.code == P.PIM_ERR_STATE  # nothing to continue from
        with pytest.raises(P.PimError) as e:
            P.pim_anneal(hd, 0, 3, 0)
        assert e.value.code == P.PIM_ERR_INVALID
        rng = np.random.default_rng(0)
        b40 = sk_pm1(40, 0)
        wide = Instance("sk", 40, (16 * b40.J).astype(np.int8),
                        rng.integers(-9, 9, 40).astype(np.int32), b40.c, 0)
        hb = P.pim_create(wide.J, wide.h, wide.c)
        try:
            P.pim_set_schedule(hb, linear_beta(4), eta_power(linear_beta(4)), 0.5)
            with pytest.raises(P.PimError) as e:
                P.pim_anneal(hb, 4, 2, 0)  # field range 16*39 > 511 for the fused kernel
            assert e.value.code == P.PIM_ERR_UNSUPPORTED
        finally:
            P.pim_destroy(hb)
    finally:
        P.pim_destroy(hd)


def test_submit_poll_completes():
    P = pim()
    inst = sk_pm1(64, 0)
    beta = linear_beta(100)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta_power(beta), 0.5)
        ticket = P.pim_submit(hd, 128, 100, 5)
        import time
        t0 = time.time()
        while P.pim_poll(ticket) == P.PIM_PENDING:
            assert time.time() - t0 < 30
            time.sleep(0.001)
        want = oracle_run(inst, beta, eta_power(beta), 0.5, replicas=128, seed=5)
        assert_same(collect(hd, 64), want)
    finally:
        P.pim_destroy(hd)


@pytest.mark.parametrize("flags", PATHS)
def test_large_n_bias_and_resume(flags):
    """Large-N kernel with a bias h and a resumed second segment."""
    P = pim()
    base = sk_pm1(400, 12)
    rng = np.random.default_rng(2)
    inst = Instance("sk", 400, base.J, rng.integers(-3, 4, 400).astype(np.int32), base.c, 12)
    T = 24
    beta = linear_beta(T)
    eta = eta_power(beta)
    full = oracle_run(inst, beta, eta, 0.5, replicas=70, seed=5, q=2, target=-2000)
    hd = P.pim_create(inst.J, inst.h, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal(hd, 70, 10, 5, instance_id=2, target=-2000, flags=flags)
        P.pim_anneal(hd, 70, 14, 5, instance_id=2, t_begin=10, target=-2000,
                     flags=flags | P.PIM_CONTINUE)
        assert_same(collect(hd, 400), full, label=f"large-N resume path={flags}")
    finally:
        P.pim_destroy(hd)


@pytest.mark.parametrize("flags", [0, 8 | 32])
def test_sk4096_sampled_replicas(flags):
    """SK N = 4096, 256 replicas (the library's choice: the coupling-resident E2M1 variant;
    and FP8 couplings streamed): sampled replicas bit for bit against the oracle, every
    replica's reported energies against its reported states."""
    P = pim()
    inst = sk_pm1(4096, 0)
    T = 40
    beta = linear_beta(T)
    eta = eta_power(beta)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal(hd, 256, T, 3, instance_id=1, flags=flags)
        got = collect(hd, 4096)
    finally:
        P.pim_destroy(hd)
    rows = [0, 77, 128, 255]
    want = oracle_run(inst, beta, eta, 0.5, replica_ids=rows, seed=3, q=1)
    assert_same(got, want, rows=rows, label=f"sk4096 path={flags}")
    assert np.array_equal(oracle.energy(inst.J, inst.h, got["final_state"]), got["final_E"])
    assert np.array_equal(oracle.energy(inst.J, inst.h, got["best_state"]), got["best_E"])


def test_results_dev_equal_host_getters():
    """pim_results_dev copies the records device to device, stream-ordered: they equal the
    host getters (energies, steps, and the bit words unpacked)."""
    import torch
    P = pim()
    inst = sk_pm1(70, 3)
    beta = linear_beta(20)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta_power(beta), 0.5)
        R = 150
        stream = torch.cuda.Stream()
        P.pim_anneal(hd, R, 20, 4, target=-40, stream=stream)
        words = P.pim_state_words(hd)
        dev = torch.device("cuda")
        bE, fE = torch.empty(R, dtype=torch.float64, device=dev), torch.empty(R, dtype=torch.float64, device=dev)
        bt, fh = torch.empty(R, dtype=torch.int32, device=dev), torch.empty(R, dtype=torch.int32, device=dev)
        bb, fb = (torch.empty(R * words, dtype=torch.int32, device=dev) for _ in range(2))
        P.pim_results_dev(hd, bE, bt, fh, fE, bb, fb, stream=stream)
        stream.synchronize()
        host = collect(hd, 70)
    finally:
        P.pim_destroy(hd)
    assert np.array_equal(bE.cpu().numpy(), host["best_E"]) and np.array_equal(fE.cpu().numpy(), host["final_E"])
    assert np.array_equal(bt.cpu().numpy(), host["best_t"]) and np.array_equal(fh.cpu().numpy(), host["first_hit"])
    for words_t, key in ((bb, "best_state"), (fb, "final_state")):
        w = words_t.cpu().numpy().view(np.uint32).reshape(R, words)
        bits = (w[:, np.arange(70) // 32] >> (np.arange(70) % 32)) & 1
        assert np.array_equal(np.where(bits > 0, 1, -1), host[key])


def test_sk4096_full_configuration_properties():
    """SK N = 4096, 256 replicas x 10 000 sweeps (the configuration the benchmark times):
    every replica's reported best / final energies are the exact energies of the reported
    states, best <= final, and the best step lies in range."""
    P = pim()
    inst = sk_pm1(4096, 0)
    T = 10000
    beta = linear_beta(T)
    eta = eta_power(beta)
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal(hd, 256, T, 0, instance_id=0)
        got = collect(hd, 4096)
    finally:
        P.pim_destroy(hd)
    assert np.array_equal(oracle.energy(inst.J, inst.h, got["final_state"]), got["final_E"])
    assert np.array_equal(oracle.energy(inst.J, inst.h, got["best_state"]), got["best_E"])
    assert np.all(got["best_E"] <= got["final_E"])
    assert np.all((got["best_t"] >= 0) & (got["best_t"] <= T))


def test_uneven4096_full_batch_plan():
    """The 4096-instance uneven batch (n ~ U[64, 1024], replicas ~ U{32..512}, 1000 sweeps)
    as one graph-replayed batch plan, the configuration the benchmark times: sampled
    instances bit-exact against the oracle on sampled replicas, energy identities for every
    replica of the sampled instances."""
    from workloads import uneven_batch
    P = pim()
    insts, reps = uneven_batch(4096, seed=0)
    T = 1000
    beta = linear_beta(T)
    eta = eta_power(beta)
    xis = [0.7 if k % 2 == 0 else 0.5 for k in range(len(insts))]
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    b = None
    try:
        for hd, xi in zip(handles, xis):
            P.pim_set_schedule(hd, beta, eta, xi)
        b = P.pim_batch_create(handles, reps, instance_ids=list(range(len(insts))))
        P.pim_batch_run(b, T, 0)
        P.pim_sync(handles[0])
        sizes = np.array([i.n for i in insts])
        small = [int(k) for k in np.flatnonzero(sizes <= 256)[:3]]
        mid = [int(k) for k in np.flatnonzero((sizes > 256) & (sizes <= 400))[:2]]
        for k in small + mid:
            got = collect(handles[k], insts[k].n)
            rows = [0, reps[k] - 1]
            want = oracle_run(insts[k], beta, eta, xis[k], replica_ids=rows, seed=0, q=k)
            assert_same(got, want, rows=rows, label=f"instance {k} n={insts[k].n}")
        for k in small + mid + [int(np.argmax(sizes))]:
            got = collect(handles[k], insts[k].n)
            J, h = insts[k].J, insts[k].h
            assert np.array_equal(oracle.energy(J, h, got["best_state"]), got["best_E"])
            assert np.array_equal(oracle.energy(J, h, got["final_state"]), got["final_E"])
    finally:
        if b is not None:
            P.pim_batch_destroy(b)
        for hd in handles:
            P.pim_destroy(hd)
