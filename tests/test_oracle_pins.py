"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test names what it pins: published known answers (Philox), closed forms, exact
enumeration on tiny instances, textbook dynamics for special parameter values, and
invariants of the update rule (Eq. 4).
"""
import math
import os

import numpy as np
import pytest
from scipy.stats import chi2, norm

import oracle
from oracle import pimi
from workloads import maxcut_er, sk_pm1, linear_beta, eta_power, random_spins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- Philox
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    rows = _kat_rows()
    assert len(rows) == 3
    for row in rows:
        c, k, want = row[0:4], row[4:6], row[6:10]
        got = pimi.philox4x32_10(*[np.uint64(x) for x in c], k[0], k[1])
        assert [int(x) for x in got] == want


def test_draw_mapping_selects_words_and_halves():
    """d(i) takes word (i&7)>>1 of the block at counter (i>>3, r, t, q): low half for even
    i, high half for odd i; the key is (seed lo, seed hi)."""
    seed = 0x0123456789ABCDEF
    q, r, t = 7, 5, 11
    i = np.arange(16)
    d = pimi.noise_draw16(seed, q, r, t, i)
    for blk in range(2):
        w = pimi.philox4x32_10(np.uint64(blk), np.uint64(r), np.uint64(t), np.uint64(q),
                               seed & 0xFFFFFFFF, seed >> 32)
        w = [int(x) for x in w]
        for k in range(8):
            word = w[k >> 1]
            want = (word >> 16) if (k & 1) else (word & 0xFFFF)
            assert d[8 * blk + k] == want


def test_draws_are_uniform_16bit():
    d = pimi.noise_draw16(1, 0, np.arange(64)[:, None], 3, np.arange(1024)[None, :]).ravel()
    assert d.min() >= 0 and d.max() < 65536
    hist = np.bincount(d >> 12, minlength=16)
    stat = ((hist - d.size / 16) ** 2 / (d.size / 16)).sum()
    assert chi2.sf(stat, 15) > 1e-4


# ----------------------------------------------------------------------------- noise tables
def test_gaussian_quantiles_match_normal_cdf():
    """Phi(Q[m]) = (m+0.5)/4096 up to float32 rounding of Q; checked with the normal CDF
    (erfc based), a different routine from the inverse used to build the table."""
    Q = pimi.gaussian_quantiles()
    assert Q.dtype == np.float32 and Q.shape == (4096,)
    m = np.arange(4096)
    p = norm.cdf(Q.astype(np.float64))
    dens = norm.pdf(Q.astype(np.float64))
    tol = dens * np.abs(Q.astype(np.float64)) * 2.0 ** -23 + 1e-12
    assert np.all(np.abs(p - (m + 0.5) / 4096) <= tol)
    assert np.all(np.diff(Q) > 0)
    assert np.array_equal(Q[::-1], -Q)          # exact antisymmetry
    assert float(Q.astype(np.float64).sum()) == 0.0
    assert abs(float(Q[-1]) - 3.6683) < 1e-3    # largest |z|: Phi^-1(1 - 1/8192)


def test_uniform_levels_are_exact_grid():
    U = pimi.uniform_levels()
    assert U[0] == np.float32(-4095 / 4096) and U[-1] == np.float32(4095 / 4096)
    assert np.all(np.diff(U.astype(np.float64)) == 2 / 4096)


# ----------------------------------------------------------------------------- LUT tanh
@pytest.mark.parametrize("x,want", [
    (-3.0, -1.0), (-1.0, -1.0), (-0.7, -1.0), (-0.5, -1 / 3), (-0.2, -1 / 3),
    (0.0, 1 / 3), (0.2, 1 / 3), (0.5, 1.0), (0.99, 1.0), (1.0, 1.0), (7.0, 1.0),
])
def test_lut_tanh_four_levels(x, want):
    """Algorithm 'LUT-based tanh': L = 4 gives levels -1, -1/3, 1/3, 1 and breakpoints
    -1, -1/2, 0, 1/2, 1; outside [-1, 1] saturates."""
    assert math.isclose(pimi.lut_tanh(x, 4), want, abs_tol=1e-15)


# ----------------------------------------------------------------------------- energy
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_energy_quadratic_form_equals_pair_sum(seed):
    """-1/2 s^T J s - h^T s (used by the oracle) equals Eq. 1's explicit pair sum."""
    rng = np.random.default_rng(seed)
    n = 9
    up = rng.integers(-3, 4, (n, n))
    J = np.triu(up, 1)
    J = (J + J.T).astype(np.int8)
    h = rng.integers(-5, 6, n).astype(np.int32)
    S, E_pair = oracle.all_energies(J, h)
    assert np.array_equal(oracle.energy(J, h, S), E_pair.astype(np.int64))
    Jf = J.astype(np.float64) * 0.37
    hf = h.astype(np.float64) * -1.3
    S, E_pair = oracle.all_energies(Jf, hf)
    assert np.allclose(oracle.energy(Jf, hf, S), E_pair, rtol=0, atol=1e-12)


def test_maxcut_cut_identity():
    """With J = -A: H = |E| - 2 cut(s), i.e. cut = (|E| - H)/2, for cut counted edge by edge."""
    inst = maxcut_er(14, seed=3)
    A = -inst.J.astype(np.int64)
    n_edges = int(np.triu(A, 1).sum())
    S = random_spins(14, 50, seed=9)
    H = oracle.energy(inst.J, inst.h, S)
    for s, e in zip(S, H):
        cut = sum(1 for i in range(14) for j in range(i + 1, 14) if A[i, j] and s[i] != s[j])
        assert n_edges - 2 * cut == e


def test_instance_generators_shape():
    mc = maxcut_er(30, 0)
    assert np.array_equal(mc.J, mc.J.T) and np.all(np.diag(mc.J) == 0)
    assert set(np.unique(mc.J)) <= {0, -1}
    assert 0.35 < (-mc.J).sum() / (30 * 29) < 0.65
    sk = sk_pm1(30, 0)
    assert np.array_equal(sk.J, sk.J.T) and np.all(np.diag(sk.J) == 0)
    off = sk.J[~np.eye(30, dtype=bool)]
    assert set(np.unique(off)) == {-1, 1}
    assert math.isclose(sk.c, 1 / math.sqrt(30)) and math.isclose(mc.c, 2 / math.sqrt(30))


# ----------------------------------------------------------------------------- ground states
@pytest.mark.parametrize("kind,n,seed", [("sk", 14, 0), ("maxcut", 16, 1)])
def test_anneal_never_below_and_reaches_ground_state(kind, n, seed):
    """Brute-force ground state pins the tracked best energy: no replica reports a value
    below E_gs, every reported best equals the energy of its reported best state, and a
    modest run reaches E_gs."""
    inst = sk_pm1(n, seed) if kind == "sk" else maxcut_er(n, seed)
    e_gs, _ = oracle.ground_state(inst.J, inst.h)
    T = 300
    beta = linear_beta(T)
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta),
                        0.5 if kind == "sk" else 0.7, replicas=32, seed=seed)
    assert np.all(out["best_E"] >= e_gs)
    assert np.array_equal(oracle.energy(inst.J, inst.h, out["best_state"]), out["best_E"])
    assert np.array_equal(oracle.energy(inst.J, inst.h, out["final_state"]), out["final_E"])
    assert out["best_E"].min() == e_gs


# ----------------------------------------------------------------------------- special cases
def test_beta_zero_gives_fair_coins():
    """beta = 0, xi = 0: tau = 0 so s' = +1 iff z >= 0, i.e. exactly half of the keys."""
    inst = sk_pm1(64, 0)
    T = 40
    beta = np.zeros(T, np.float32)
    eta = np.ones(T, np.float32)
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.0, replicas=64, seed=5,
                        record=False)
    s = out["final_state"].ravel()
    k = int((s > 0).sum())
    nn = s.size
    assert abs(k - nn / 2) < 4 * math.sqrt(nn / 4)
    Q = pimi.gaussian_quantiles()
    assert int((Q >= 0).sum()) == 2048


def test_eta_zero_is_synchronous_threshold_dynamics():
    """eta = 0, xi = 0: Eq. 4 reduces to s' = sign(J s + h) with sign(0) = +1 (tanh keeps
    the sign for beta > 0).  Synchronous threshold networks with symmetric J end in a
    fixed point or a 2-cycle (Goles-Chacc et al. 1985), checked on the trajectory."""
    inst = sk_pm1(40, 2)
    h = np.random.default_rng(0).integers(-3, 4, 40).astype(np.int32)
    T = 60
    beta = np.full(T, 1.5, np.float32)
    eta = np.zeros(T, np.float32)
    init = random_spins(40, 8, seed=1)
    s = init.copy()
    traj = [s.copy()]
    for _ in range(T):
        I = s.astype(np.int64) @ inst.J.T.astype(np.int64) + h[None, :]
        s = np.where(I >= 0, 1, -1).astype(np.int8)
        traj.append(s)
    out = oracle.anneal(inst.J, h, inst.c, beta, eta, 0.0, replicas=8, init=init, seed=3)
    assert np.array_equal(out["final_state"], traj[-1])
    assert np.array_equal(traj[-1], traj[-3])


def test_large_inertia_freezes_spins():
    """xi > 1 + eta * max|z|: |tau + eta z| < xi, so sign(delta) = s(t) for every spin."""
    inst = maxcut_er(32, 4)
    T = 30
    beta = linear_beta(T)
    eta = np.full(T, 0.5, np.float32)
    xi = 1.0 + 0.5 * 3.7
    init = random_spins(32, 16, seed=2)
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, xi, replicas=16, init=init, seed=1)
    assert np.array_equal(out["final_state"], init)


def _sweep_transition_matrix(J, h, beta, eta):
    """16x16 transition matrix of one sequential sweep (spins 0..3 in order) computed by
    counting, for each state and spin, the keys m in [0, 4096) whose Eq. 3 decision is +1."""
    n = J.shape[0]
    U = pimi.uniform_levels()
    ns = 1 << n

    def single(i):
        P = np.zeros((ns, ns))
        for a in range(ns):
            s = np.array([1 if (a >> k) & 1 else -1 for k in range(n)], np.int8)
            I = int((J[i].astype(np.int64) * s).sum() + h[i])
            tau = pimi.activation(np.float32(beta), np.array([I]))[0]
            up = pimi.decide(np.full(4096, tau, np.float32), np.full(4096, s[i]), 0.0, eta, U)
            p_up = float((up > 0).mean())
            b_up, b_dn = a | (1 << i), a & ~(1 << i)
            P[a, b_up] += p_up
            P[a, b_dn] += 1.0 - p_up
        return P

    M = np.eye(ns)
    for i in range(n):
        M = M @ single(i)
    return M


def test_sequential_uniform_noise_is_heat_bath_exact():
    """Eq. 3 with eta = 1, uniform noise and constant beta: P(s_i=+1|rest) =
    (1 + tanh(beta I_i))/2, whose invariant law is exp(-beta H)/Z.  The stationary law
    of the exact 16-state sweep matrix built from the oracle's decisions matches the
    Boltzmann law up to the 12-bit key resolution (< 1e-3 total variation)."""
    J = np.array([[0, 1, -2, 1], [1, 0, 1, -1], [-2, 1, 0, 2], [1, -1, 2, 0]], np.int8)
    h = np.array([1, 0, -1, 0], np.int32)
    beta = 0.4
    M = _sweep_transition_matrix(J, h, beta, 1.0)
    w, v = np.linalg.eig(M.T)
    pi = np.real(v[:, np.argmin(np.abs(w - 1))])
    pi = pi / pi.sum()
    S, p = oracle.boltzmann(J, h, beta)
    # state index convention: bit k of the index -> spin k (+1 when set), same as brute
    assert 0.5 * np.abs(pi - p).sum() < 1e-3


def test_sequential_sampler_matches_boltzmann_chi2():
    """Empirical check of the full sequential loop (Philox draws, keys, tables): final
    states of 4000 independent chains after 40 sweeps follow exp(-beta H)/Z (chi^2)."""
    J = np.array([[0, 1, -2, 1], [1, 0, 1, -1], [-2, 1, 0, 2], [1, -1, 2, 0]], np.int8)
    h = np.array([1, 0, -1, 0], np.int32)
    beta = 0.4
    steps = 4 * 40
    s = oracle.anneal_sequential(J, h, 1.0, np.full(steps, beta, np.float32),
                                 np.ones(steps, np.float32), replicas=4000, steps=steps, seed=11)
    idx = ((s > 0).astype(np.int64) << np.arange(4)[None, :]).sum(axis=1)
    hist = np.bincount(idx, minlength=16)
    _, p = oracle.boltzmann(J, h, beta)
    expct = p * len(idx)
    stat = ((hist - expct) ** 2 / expct).sum()
    assert chi2.sf(stat, 15) > 1e-3


# ----------------------------------------------------------------------------- structure
def test_decision_monotone_in_key_and_field():
    """The decision is monotone in the noise key m and in the field I, which is what lets
    a threshold table M_t[s][I] = min{m : delta >= 0} represent it exactly."""
    Q = pimi.gaussian_quantiles()
    for b, xi, eta in [(0.07, 0.5, 0.3), (0.3, 0.7, 1.1), (0.01, 0.0, 0.05)]:
        I = np.arange(-60, 61)
        tau = pimi.activation(np.float32(b), I)
        assert np.all(np.diff(tau) >= 0)
        for s in (-1, 1):
            dec = pimi.decide(np.repeat(tau[:, None], 4096, 1), np.full((I.size, 4096), s),
                              xi, eta, np.broadcast_to(Q, (I.size, 4096)))
            assert np.all(np.diff(dec.astype(int), axis=1) >= 0)
            assert np.all(np.diff(dec.astype(int), axis=0) >= 0)


def test_replica_subset_reproduces_full_run():
    """Replicas only meet through the counter field r: any subset reproduces the full run."""
    inst = sk_pm1(24, 1)
    beta = linear_beta(50)
    eta = eta_power(beta)
    full = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.5, replicas=12, seed=4, q=3,
                         target=-40)
    sub = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.5, replica_ids=[3, 10], seed=4,
                        q=3, target=-40)
    for key in ("best_E", "best_t", "first_hit", "final_E", "best_state", "final_state"):
        assert np.array_equal(full[key][[3, 10]], sub[key])


def test_resume_is_bit_identical():
    """Running T sweeps equals running t0 sweeps and continuing from the saved state."""
    inst = maxcut_er(20, 2)
    beta = linear_beta(80)
    eta = eta_power(beta)
    kw = dict(replicas=6, seed=9, q=1, target=-45)
    full = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, sweeps=80, **kw)
    part = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, sweeps=33, **kw)
    rest = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, t_begin=33, sweeps=47,
                         prev=part, **kw)
    for key in ("best_E", "best_t", "first_hit", "final_E", "best_state", "final_state"):
        assert np.array_equal(full[key], rest[key]), key


def test_record_matches_per_state_energies():
    inst = sk_pm1(16, 5)
    beta = linear_beta(20)
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5, replicas=4,
                        seed=1, record=True)
    E = out["energies"]
    assert E.shape == (21, 4)
    assert np.array_equal(E.min(axis=0).astype(np.int64), out["best_E"])
    assert np.array_equal(E.argmin(axis=0), out["best_t"])


def _first_at_or_below(E, target, t_begin=0):
    """First step t_begin + k whose recorded energy E[k] is <= target, per replica, or -1."""
    hit = E <= target
    return np.where(hit.any(axis=0), hit.argmax(axis=0) + t_begin, -1)


def test_first_hit_is_the_first_recorded_energy_at_or_below_the_target():
    """first_hit = the first t in t_begin .. t_begin + sweeps (the final state s(T) included)
    whose energy is <= target, or -1: checked against the recorded trajectory for a target
    every replica meets at t = t_begin, a target that only the final state of some replica
    meets, a target between those, and one that nothing reaches."""
    inst = sk_pm1(16, 5)
    T = 20
    beta = linear_beta(T)
    kw = dict(replicas=64, seed=1)
    rec = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5, record=True, **kw)
    E = rec["energies"].astype(np.int64)                    # (T + 1, R): s(0) .. s(T)
    # a replica whose final energy is below every earlier one: its first hit at
    # target = E[T] is the final state s(T)
    final_only = np.nonzero(E[T] < E[:T].min(axis=0))[0]
    assert final_only.size > 0, "no replica improves on its last step; change the seed"
    targets = {"all at t = 0": int(E[0].max()),
               "final state only": int(E[T, final_only[0]]),
               "in between": int(np.median(E)),
               "never": int(E.min()) - 1}
    for label, target in targets.items():
        out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5, target=target, **kw)
        want = _first_at_or_below(E, target)
        assert np.array_equal(out["first_hit"], want), label
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5,
                        target=targets["all at t = 0"], **kw)
    assert np.all(out["first_hit"] == 0)
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5,
                        target=targets["final state only"], **kw)
    assert out["first_hit"][final_only[0]] == T
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5,
                        target=targets["never"], **kw)
    assert np.all(out["first_hit"] == -1)
    # a hit exactly at the target counts (<=, not <)
    r0 = 3
    out = oracle.anneal(inst.J, inst.h, inst.c, beta, eta_power(beta), 0.5, target=int(E[5, r0]),
                        **kw)
    assert out["first_hit"][r0] <= 5 and E[out["first_hit"][r0], r0] <= E[5, r0]


def test_first_hit_counts_absolute_steps_when_resuming():
    """A run that starts at t_begin reports first hits as schedule steps t_begin + k, and a
    resumed run keeps a hit found before the resume."""
    inst = maxcut_er(20, 2)
    beta = linear_beta(40)
    eta = eta_power(beta)
    kw = dict(replicas=32, seed=9, q=1)
    part = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, sweeps=15, record=True, **kw)
    rest = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, t_begin=15, sweeps=25, prev=part,
                         record=True, **kw)
    E_rest = rest["energies"].astype(np.int64)              # s(15) .. s(40)
    target = int(np.median(E_rest))
    part_t = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, sweeps=15, target=target, **kw)
    rest_t = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, t_begin=15, sweeps=25,
                           prev=part_t, target=target, **kw)
    E_all = np.concatenate([part["energies"][:15], E_rest]).astype(np.int64)  # s(0) .. s(40)
    assert np.array_equal(rest_t["first_hit"], _first_at_or_below(E_all, target))
    fresh = oracle.anneal(inst.J, inst.h, inst.c, beta, eta, 0.7, t_begin=15, sweeps=25,
                          init=part["final_state"], target=target, **kw)
    assert np.array_equal(fresh["first_hit"], _first_at_or_below(E_rest, target, t_begin=15))


def test_n_trials_closed_forms():
    """n = log(eps)/log(1-p): p = 1/2, eps = 1e-3 gives log2(1000); p = 1 needs one trial."""
    assert math.isclose(oracle.n_trials(0.5), math.log2(1000), rel_tol=1e-12)
    assert oracle.n_trials(1.0) == 1.0
    assert math.isclose(oracle.tts99(2.0, 0.9), 2.0 * 2.0, rel_tol=1e-12)


def test_round_bf16_examples():
    """bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie and rounds to even (1.0),
    1 + 3 * 2^-8 rounds up to 1 + 2^-6, and representable values are unchanged."""
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -3.140625, 0.0, 2.0 ** -130, 1.0 + 2 ** -7])
    want = np.array([1.0, 1.0 + 2.0 ** -6, -3.140625, 0.0, 2.0 ** -130, 1.0 + 2 ** -7])
    assert np.array_equal(pimi.round_bf16(x), want)
    r = pimi.round_bf16(np.random.default_rng(0).standard_normal(1000))
    assert np.array_equal(pimi.round_bf16(r), r)
    f32 = r.astype(np.float32).view(np.uint32)
    assert np.all(f32 & 0xFFFF == 0)


# ------------------------------------------------ sequential sweeps (conventional PIM, Eq. 3)
def test_sequential_sweeps_sample_boltzmann_chi2():
    """Sequential sweeps with xi = 0 and uniform noise are a heat-bath sampler: final
    states of 4000 chains after 40 sweeps follow exp(-beta H)/Z (chi^2)."""
    J = np.array([[0, 1, -2, 1], [1, 0, 1, -1], [-2, 1, 0, 2], [1, -1, 2, 0]], np.int8)
    h = np.array([1, 0, -1, 0], np.int32)
    beta = 0.4
    T = 40
    out = oracle.anneal_sequential_sweeps(J, h, 1.0, np.full(T, beta, np.float32),
                                          np.ones(T, np.float32), 0.0, replicas=4000, seed=5)
    s = out["final_state"]
    idx = ((s > 0).astype(np.int64) << np.arange(4)[None, :]).sum(axis=1)
    hist = np.bincount(idx, minlength=16)
    _, p = oracle.boltzmann(J, h, beta)
    expct = p * len(idx)
    stat = ((hist - expct) ** 2 / expct).sum()
    assert chi2.sf(stat, 15) > 1e-3


@pytest.mark.parametrize("n,zero_j", [(1, False), (10, True)])
def test_sequential_equals_parallel_without_interaction(n, zero_j):
    """With a single spin, or with J = 0, the order of the updates cannot matter: sequential
    sweeps equal the parallel loop record for record (same draws per sweep)."""
    rng = np.random.default_rng(n)
    J = np.zeros((n, n), np.int8)
    h = rng.integers(-3, 4, n).astype(np.int32)
    T = 30
    beta = linear_beta(T)
    eta = eta_power(beta)
    for xi in (0.0, 0.6):
        seq = oracle.anneal_sequential_sweeps(J, h, 0.5, beta, eta, xi, replicas=25, seed=7, q=2,
                                              target=-2.0, noise="gauss")
        par = oracle.anneal(J, h, 0.5, beta, eta, xi, replicas=25, seed=7, q=2, target=-2.0)
        for k in ("best_E", "best_t", "first_hit", "final_E", "best_state", "final_state"):
            assert np.array_equal(seq[k], par[k]), (k, xi)


def test_sequential_update_sees_the_new_spin():
    """Two ferromagnetically coupled spins starting anti-aligned, no noise: the parallel
    update swaps them (each follows the other's old value), the sequential update aligns
    them (spin 1 already sees the new spin 0)."""
    J = np.array([[0, 3], [3, 0]], np.int8)
    h = np.zeros(2, np.int32)
    beta = np.full(1, 2.0, np.float32)
    eta = np.zeros(1, np.float32)
    init = np.array([[1, -1]], np.int8)
    seq = oracle.anneal_sequential_sweeps(J, h, 1.0, beta, eta, 0.0, replicas=1, init=init)
    par = oracle.anneal(J, h, 1.0, beta, eta, 0.0, replicas=1, init=init)
    assert seq["final_state"].tolist() == [[-1, -1]]
    assert par["final_state"].tolist() == [[-1, 1]]


# ------------------------------------------------ fixed-point datapath (quantization section)
def test_quantize_truncates_toward_zero_and_saturates():
    q = oracle.quantize([0.3, -0.3, 1.9, -2.5, 1.75, 0.2499, -0.2499], 4, 2)
    assert q.tolist() == [0.25, -0.25, 1.75, -2.0, 1.75, 0.0, 0.0]
    step = 2.0 ** -12
    q = oracle.quantize([7.99999, -9.0, 3 * step + step / 2, -(3 * step + step / 2)], 16, 4)
    assert q.tolist() == [8 - step, -8.0, 3 * step, -3 * step]


def test_fixed_point_decision_hand_case():
    """ap_fixed<4,2> (step 1/4, range [-2, 1.75]), c = 1/2, I = 3, beta = 1: u = 1.5,
    x = 1.5, tanh(1.5) = 0.905 -> 0.75; s = -1, xi = 0.7 -> 0.5: a = 0.25; eta = 0.6 -> 0.5.
    z = -0.9 -> -0.75: n = Q(-0.375) = -0.25, delta = 0 -> +1.
    z = -1.3 -> -1.25: n = Q(-0.625) = -0.5, delta = -0.25 -> -1."""
    got = oracle.decide_fixed(np.array([3, 3]), np.array([-1, -1]), 0.5, 1.0, 0.7, 0.6,
                              np.array([-0.9, -1.3]), 4, 2)
    assert got.tolist() == [1, -1]


def test_fixed_point_decision_monotone_in_key():
    """The quantized decision never decreases with the noise key, so exact key thresholds
    represent it (the table form the kernels use)."""
    Q = pimi.gaussian_quantiles()
    I = np.arange(-40, 41)
    for W, Ib, act in ((4, 2, "tanh"), (6, 2, "lut"), (16, 4, "tanh")):
        for s in (-1, 1):
            dec = oracle.decide_fixed(np.repeat(I[:, None], 4096, 1), np.full((I.size, 4096), s),
                                      2 / np.sqrt(40), 1.3, 0.5, 0.8,
                                      np.broadcast_to(Q, (I.size, 4096)), W, Ib, act)
            assert np.all(np.diff(dec.astype(int), axis=1) >= 0), (W, Ib, act, s)


def test_fixed_point_at_high_precision_is_the_exact_rule():
    """With 32 fractional bits the datapath is Eq. 4 itself: decisions equal
    sign(tanh(beta c I) + xi s + eta z) evaluated in float64 wherever the margin exceeds
    1e-6 (a dropped or mis-signed term would fail this)."""
    rng = np.random.default_rng(3)
    I = rng.integers(-30, 31, 20000)
    s = np.where(rng.random(20000) < 0.5, -1, 1)
    z = rng.standard_normal(20000)
    c, beta, xi, eta = 2 / np.sqrt(50), 0.9, 0.7, 0.6
    beta32, xi32, eta32 = (float(np.float32(v)) for v in (beta, xi, eta))
    exact = np.tanh(beta32 * c * I) + xi32 * s + eta32 * z
    got = oracle.decide_fixed(I, s, c, beta, xi, eta, z, 40, 8)
    ok = np.abs(exact) > 1e-6
    assert np.array_equal(got[ok], np.where(exact[ok] >= 0, 1, -1))
