"""GPU tests of batch plans: an uneven batch routed once onto the fused, persistent mid-N
and large-N kernels, replayed as a CUDA graph; every run of every instance is bit-exact
against its own oracle run."""
import numpy as np
import pytest

from workloads import eta_power, linear_beta, maxcut_er, sk_pm1

from gpu_helpers import assert_same, collect, oracle_run, pim

pytestmark = pytest.mark.gpu


def _batch(sizes, reps, seed0=300):
    insts = [(sk_pm1 if k % 2 else maxcut_er)(n, seed0 + k) for k, n in enumerate(sizes)]
    return insts, list(reps)


def _check_all(P, handles, insts, reps, ids, beta, eta, xi, seed, sweeps=None, targets=None):
    for k, (hd, inst, R, q) in enumerate(zip(handles, insts, reps, ids)):
        tg = None if targets is None else targets[k]
        want = oracle_run(inst, beta, eta, xi, replicas=R, seed=seed, q=q, sweeps=sweeps, target=tg)
        assert_same(collect(hd, inst.n), want, label=f"n={inst.n} R={R} seed={seed}")


def test_batch_plan_graph_replays_match_oracle():
    """One plan over fused and mid-N instances: runs with two seeds replay a captured graph
    (updated in place for the new seed); a repeated seed reproduces its results."""
    P = pim()
    insts, reps = _batch([40, 300, 150, 700, 256, 1000, 64], [64, 130, 32, 100, 200, 64, 96])
    ids = list(range(20, 20 + len(insts)))
    targets = [-0.5 * i.n for i in insts]
    T = 10
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    b = None
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.6)
        b = P.pim_batch_create(handles, reps, instance_ids=ids, targets=targets)
        for seed in (3, 8, 3):
            P.pim_batch_run(b, T, seed)
            info = P.pim_batch_info(b)
            assert info["uses_graph"] and info["kernel_launches"] >= 3
            assert P.pim_kernel_ms(handles[0]) > 0.0  # timer events are graph nodes
            _check_all(P, handles, insts, reps, ids, beta, eta, 0.6, seed, targets=targets)
    finally:
        if b is not None:
            P.pim_batch_destroy(b)
        for hd in handles:
            P.pim_destroy(hd)


def test_batch_plan_resume_and_large_instance():
    """A plan that also holds a large-N instance (n = 1100): a run split in two with
    PIM_CONTINUE equals the uninterrupted oracle run."""
    P = pim()
    insts, reps = _batch([1100, 90, 520], [64, 40, 130], seed0=400)
    ids = [5, 6, 7]
    T = 12
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    b = None
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        b = P.pim_batch_create(handles, reps, instance_ids=ids)
        P.pim_batch_run(b, 5, 11)
        P.pim_batch_run(b, 7, 11, t_begin=5, run_flags=P.PIM_CONTINUE)
        assert P.pim_batch_info(b)["kernel_launches"] >= 2
        _check_all(P, handles, insts, reps, ids, beta, eta, 0.5, 11)
    finally:
        if b is not None:
            P.pim_batch_destroy(b)
        for hd in handles:
            P.pim_destroy(hd)


def test_batch_plan_rejects_changed_instance():
    P = pim()
    insts, reps = _batch([50, 60], [32, 32])
    beta = linear_beta(8)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    b = None
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        b = P.pim_batch_create(handles, reps)
        P.pim_batch_run(b, 8, 1)
        P.pim_sync(handles[0])
        P.pim_set_schedule(handles[1], linear_beta(9), eta_power(linear_beta(9)), 0.5)
        with pytest.raises(P.PimError) as e:
            P.pim_batch_run(b, 8, 1)
        assert e.value.code == P.PIM_ERR_STATE
        with pytest.raises(P.PimError) as e:
            P.pim_batch_run(b, 9, 1, t_begin=0, run_flags=4)
        assert e.value.code == P.PIM_ERR_INVALID
    finally:
        if b is not None:
            P.pim_batch_destroy(b)
        for hd in handles:
            P.pim_destroy(hd)


def test_results_to_host_matches_oracle_on_every_entry_point():
    """PIM_RESULTS_TO_HOST: the getters read the pinned copy taken at the end of the run.
    Results are bit-exact against the oracle after pim_anneal_batch, a graph-replayed batch
    plan (replays alternating with and without the flag, so a stale host copy would show)
    and a resumed run without the flag; the sequential loop reads the same way."""
    P = pim()
    F = P.PIM_RESULTS_TO_HOST
    insts, reps = _batch([120, 333, 64], [70, 96, 40], seed0=500)
    ids = [1, 2, 3]
    T = 12
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    b = None
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal_batch(handles, reps, T, 4, instance_ids=ids, flags=F)
        _check_all(P, handles, insts, reps, ids, beta, eta, 0.5, 4)
        b = P.pim_batch_create(handles, reps, instance_ids=ids)
        for seed, fl in ((5, F), (6, 0), (7, F), (7, 0)):
            P.pim_batch_run(b, T, seed, run_flags=fl)
            _check_all(P, handles, insts, reps, ids, beta, eta, 0.5, seed)
        P.pim_batch_destroy(b)
        b = None
        # first half with the host copy, second half resumed without it
        P.pim_anneal_batch(handles, reps, T // 2, 9, instance_ids=ids, flags=F)
        P.pim_anneal_batch(handles, reps, T - T // 2, 9, t_begin=T // 2, instance_ids=ids,
                           flags=P.PIM_CONTINUE)
        _check_all(P, handles, insts, reps, ids, beta, eta, 0.5, 9)
    finally:
        if b is not None:
            P.pim_batch_destroy(b)
        for hd in handles:
            P.pim_destroy(hd)
    inst = insts[0]
    hd = P.pim_create(inst.J, None, inst.c)
    try:
        P.pim_set_schedule(hd, beta, eta, 0.0)
        P.pim_anneal_sequential(hd, 33, T, 2, instance_id=4, flags=F)
        got = collect(hd, inst.n)
        P.pim_anneal_sequential(hd, 33, T, 2, instance_id=4)
        assert_same(got, collect(hd, inst.n), label="sequential host copy")
    finally:
        P.pim_destroy(hd)


def test_chunked_queue_matches_oracle():
    """More fused units than the two CTAs per SM that run at once: persistent CTAs take
    (chunk, unit) segments from a queue, each chunk after the first starting from the state
    its predecessor (run by another CTA) published.  Units of three sizes on one kernel
    variant; every unit equals the oracle after pim_anneal_batch (its results brought to the
    host by one gather launch), and sampled units after
    graph-replayed batch-plan runs of 1 and 2 sweeps (chunks down to one sweep) and a
    PIM_CONTINUE resumption to the full schedule."""
    import torch
    P = pim()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    K = int(2.5 * 2 * sms) + 3
    sizes = [64, 40, 100]
    insts = [(sk_pm1 if k % 2 else maxcut_er)(sizes[k % 3], 900 + k) for k in range(K)]
    reps = [128] * K
    ids = list(range(K))
    T = 12
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    b = None
    sample = list(range(0, K, 9)) + [K - 1]

    def pick(xs):
        return [xs[k] for k in sample]

    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        # results come back through one gather launch (many instances, PIM_RESULTS_TO_HOST)
        P.pim_anneal_batch(handles, reps, T, 21, instance_ids=ids, flags=P.PIM_RESULTS_TO_HOST)
        _check_all(P, handles, insts, reps, ids, beta, eta, 0.5, 21)
        b = P.pim_batch_create(handles, reps, instance_ids=ids)
        P.pim_batch_run(b, 1, 23)
        _check_all(P, pick(handles), pick(insts), pick(reps), pick(ids), beta, eta, 0.5, 23,
                   sweeps=1)
        P.pim_batch_run(b, 2, 22, run_flags=P.PIM_RESULTS_TO_HOST)  # gather after a replay
        _check_all(P, pick(handles), pick(insts), pick(reps), pick(ids), beta, eta, 0.5, 22,
                   sweeps=2)
        P.pim_batch_run(b, T - 2, 22, t_begin=2, run_flags=P.PIM_CONTINUE)
        _check_all(P, pick(handles), pick(insts), pick(reps), pick(ids), beta, eta, 0.5, 22)
        assert P.pim_batch_info(b)["uses_graph"]
    finally:
        if b is not None:
            P.pim_batch_destroy(b)
        for hd in handles:
            P.pim_destroy(hd)


def test_chunked_queue_general_bias_variants():
    """The chunked queue on the general-bias fused kernels (nonzero h): npad 128 (N = 100)
    and npad 256 (N = 200) groups, each with more units than two CTAs per SM, in one batch
    (one queue launch per group); sampled units equal the oracle."""
    import torch
    from workloads import Instance
    P = pim()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_group = int(2.2 * 2 * sms) + 5
    rng = np.random.default_rng(77)
    insts = []
    for k in range(2 * per_group):
        n = 100 if k % 2 else 200
        base = sk_pm1(n, 1200 + k)
        h = rng.integers(-3, 4, size=n).astype(np.int32)
        insts.append(Instance("sk", n, base.J, h, base.c, base.seed))
    K = len(insts)
    reps = [128] * K
    ids = list(range(K))
    T = 8
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(i.J, i.h, i.c) for i in insts]
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal_batch(handles, reps, T, 31, instance_ids=ids)
        sample = list(range(0, K, 5)) + [K - 2, K - 1]
        for k in sample:
            want = oracle_run(insts[k], beta, eta, 0.5, replicas=128, seed=31, q=ids[k])
            assert_same(collect(handles[k], insts[k].n), want, label=f"unit {k} n={insts[k].n}")
    finally:
        for hd in handles:
            P.pim_destroy(hd)


def test_mid_batch_mixes_diagonal_and_general_units():
    """One batch on the mid-N kernel with units of both kinds: SK N = 400 and Max-Cut N = 500
    (diagonal-encoded from E5M2 images), SK N = 400 with a bias h and SK N = 350 with some
    |J| = 9 (general table): the two kinds run as two persistent launches of one call and
    every instance equals the oracle."""
    from workloads import Instance
    P = pim()
    rng = np.random.default_rng(91)
    a = sk_pm1(400, 601)
    b = maxcut_er(500, 602)
    base = sk_pm1(400, 603)
    c = Instance("sk", 400, base.J, rng.integers(-2, 3, size=400).astype(np.int32), base.c, base.seed)
    base = sk_pm1(350, 604)
    J9 = base.J.astype(np.int8).copy()
    i = np.arange(0, 349, 5)
    J9[i, i + 1] = J9[i + 1, i] = 9 * J9[i, i + 1]
    d = Instance("sk", 350, J9, base.h, base.c, base.seed)
    insts = [a, b, c, d]
    reps = [130, 64, 96, 200]
    ids = [11, 12, 13, 14]
    T = 9
    beta = linear_beta(T)
    eta = eta_power(beta)
    handles = [P.pim_create(x.J, x.h if np.any(x.h) else None, x.c) for x in insts]
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta, 0.5)
        P.pim_anneal_batch(handles, reps, T, 41, instance_ids=ids, flags=P.PIM_PATH_MID)
        for hd, x, R, q in zip(handles, insts, reps, ids):
            want = oracle_run(x, beta, eta, 0.5, replicas=R, seed=41, q=q)
            assert_same(collect(hd, x.n), want, label=f"n={x.n} q={q}")
    finally:
        for hd in handles:
            P.pim_destroy(hd)


def test_batch_route_reports_kernel_and_large_n_variant():
    """pim_batch_route: fused for n <= 256; the E2M1 coupling-resident large-N variant for
    integer couplings in {0, +-1, +-2, +-3, +-4, +-6} (FP8 with PIM_PATH_FP8, and for a
    coupling magnitude E2M1 cannot hold); BF16 for real couplings."""
    from workloads import Instance, maxcut_gauss
    P = pim()
    sk = sk_pm1(1100, 5)
    J9 = sk.J.astype(np.int8).copy()
    J9[0, 1] = J9[1, 0] = 5
    insts = [sk_pm1(100, 4), sk, Instance("sk", 1100, J9, sk.h, sk.c, 5), maxcut_gauss(600, 6)]
    beta = linear_beta(4)
    handles = [P.pim_create(i.J, None, i.c) for i in insts]
    try:
        for hd in handles:
            P.pim_set_schedule(hd, beta, eta_power(beta), 0.5)
        for flags, want in ((P.PIM_PATH_BIG, ["fused", "e2m1_resident", "fp8", "bf16"]),
                            (P.PIM_PATH_BIG | P.PIM_PATH_FP8, ["fused", "fp8", "fp8", "bf16"])):
            b = P.pim_batch_create(handles, [128] * 4, flags=flags)
            try:
                got = [P.pim_batch_route(b, k) for k in range(4)]
            finally:
                P.pim_batch_destroy(b)
            assert got[0] == {"kernel": "fused"}
            assert [g.get("operand", "fused") for g in got] == want
            assert all(g["kernel"] == "large" and g["tile_width"] in (64, 128) for g in got[1:])
        with pytest.raises(P.PimError):
            b = P.pim_batch_create(handles, [128] * 4)
            try:
                P.pim_batch_route(b, 4)
            finally:
                P.pim_batch_destroy(b)
    finally:
        for hd in handles:
            P.pim_destroy(hd)
