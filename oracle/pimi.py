"""Oracle of the PIMI update rule -- TEST INFRASTRUCTURE ONLY (see package docstring).

What it restates (paper section / equation):
  * Ising energy H(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i ............ Eq. 1
  * local field I_i(t) = sum_j J_ij s_j(t) + h_i ........................... Eq. 2
  * conventional (sequential) PIM update, one spin per step ............... Eq. 3, Box 1
  * PIMI update, all spins at once:
      s_i(t+1) = sign[ tanh(beta(t) I_i(t)) + xi s_i(t) + eta(t) N(0,1) ] . Eq. 4, Box 1
  * LUT tanh: L levels on [-1,1], saturating ............ Algorithm "LUT-based tanh"
  * success criterion min_{t<=T} H(t) <= target and the trial count
    n = log(eps)/log(1-p) .......................... supplementary CCTS section (Eqs. S)

Readings where the paper leaves a choice:
  * Coupling scale c (2/sqrt(N) Max-Cut, 1/sqrt(N) SK) is applied after the
    multiply-accumulate, as the fixed-point section describes: b_t = fl32(beta_t * c) and
    the activation argument is x = b_t * I computed in float64 (exact for integer I).
  * tanh is evaluated in float64 by the C library (math.tanh) and rounded to float32.
  * Noise N(0,1) is not pre-generated: a 16-bit draw d comes from Philox4x32-10
    (Salmon, Moraes, Dror, Shaw, SC'11) with key (seed_lo, seed_hi) and counter
    (i>>3, r, t, q); the 12-bit key m = d>>4 indexes a table of 4096 Gaussian
    quantiles Q[m] = fl32(Phi^-1((m+0.5)/4096)), made exactly antisymmetric.  The
    uniform noise of Eq. 3 uses the grid U[m] = (2m-4095)/4096.
  * The decision is taken in float32 (the kernel's precision), in this order:
      a = fl32(tau + (+xi if s>0 else -xi)),  n = fl32(fl32(eta_t) * z),
      delta = fl32(a + n),  s' = +1 if delta >= 0 else -1   (sign(0) = +1).
  * Initial spins, when not given, are bit 15 of the draw at step field 0xFFFFFFFF.
  * States s(t_begin) .. s(t_begin+sweeps) all count toward the best energy; the earliest
    minimum wins ties.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtri

# ---------------------------------------------------------------------------------------
# Philox4x32-10, written from its published definition (Salmon et al., SC'11, Sec. 4):
# each round multiplies counter words 0 and 2 by fixed 32-bit constants, splits the
# 64-bit products into hi/lo halves, and forms
#   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0));
# the key is bumped by the Weyl constants between rounds.
# ---------------------------------------------------------------------------------------
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_U32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x32-10.  Counter words are array-likes of 32-bit values
    (broadcast together); the key is two Python ints.  Returns four uint64 arrays that
    hold 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _U32 for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    m0 = np.uint64(_PHILOX_M0)
    m1 = np.uint64(_PHILOX_M1)
    k0 &= 0xFFFFFFFF
    k1 &= 0xFFFFFFFF
    for _ in range(10):
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _U32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _U32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def noise_draw16(seed: int, q: int, r, t: int, i) -> np.ndarray:
    """16-bit draw d for spin i, replica r, step t, instance q (arrays broadcast).

    Counter (i>>3, r, t, q), key (seed & 0xffffffff, seed >> 32); word (i&7)>>1 of the
    output, low half for even i and high half for odd i."""
    i = np.asarray(i, dtype=np.int64)
    r = np.asarray(r, dtype=np.int64)
    words = philox4x32_10(i >> 3, r, np.int64(t) & 0xFFFFFFFF, q, seed & 0xFFFFFFFF,
                          (seed >> 32) & 0xFFFFFFFF)
    sel = (i & 7) >> 1
    w = np.choose(np.broadcast_to(sel, words[0].shape), words)
    d = np.where(np.broadcast_to(i & 1, w.shape) == 1, w >> np.uint64(16), w & np.uint64(0xFFFF))
    return d.astype(np.int64)


def init_spin_draw(seed: int, q: int, replica_ids, n: int) -> np.ndarray:
    """Initial spins (replicas x n, int8): +1 where bit 15 of the draw at step field
    0xFFFFFFFF is set, else -1."""
    r = np.asarray(replica_ids, dtype=np.int64)[:, None]
    d = noise_draw16(seed, q, r, 0xFFFFFFFF, np.arange(n)[None, :])
    return np.where((d >> 15) & 1, 1, -1).astype(np.int8)


# ---------------------------------------------------------------------------------------
# Noise values z(m) for the 12-bit key m.
# ---------------------------------------------------------------------------------------
NOISE_LEVELS = 4096


def gaussian_quantiles() -> np.ndarray:
    """Q[m] = fl32(Phi^-1((m + 0.5)/4096)) for m < 2048 and Q[4095-m] = -Q[m]: the
    N(0,1) term of Eq. 4, sampled by inversion of a 12-bit uniform key."""
    m = np.arange(NOISE_LEVELS // 2, dtype=np.float64)
    lower = ndtri((m + 0.5) / NOISE_LEVELS).astype(np.float32)
    return np.concatenate([lower, -lower[::-1]]).astype(np.float32)


def uniform_levels() -> np.ndarray:
    """U[m] = (2m - 4095)/4096 (exact in float32): the U(-1,1) term of Eq. 3."""
    m = np.arange(NOISE_LEVELS, dtype=np.float64)
    return ((2.0 * m - (NOISE_LEVELS - 1)) / NOISE_LEVELS).astype(np.float32)


# ---------------------------------------------------------------------------------------
# Activation tau = tanh(beta_t I) (Eq. 4) or its L-level lookup table (Algorithm
# "LUT-based tanh approximation").
# ---------------------------------------------------------------------------------------
def lut_tanh(x: float, levels: int) -> float:
    """L output levels -1 + 2k/(L-1), k = 0..L-1; L+1 breakpoints -1 + 2k/L.  Inputs
    below -1 give -1 and above +1 give +1; otherwise the level of the interval
    [b_k, b_{k+1}) that holds x.  x = +1 exactly lies in no half-open interval and
    saturates to +1."""
    if x < -1.0:
        return -1.0
    if x > 1.0:
        return 1.0
    k = 0
    for kk in range(1, levels):
        if x >= -1.0 + 2.0 * kk / levels:
            k = kk
    return -1.0 + 2.0 * k / (levels - 1)


def activation(b_t: np.float32, I: np.ndarray, act: str = "tanh", lut_levels: int = 4) -> np.ndarray:
    """tau(I) in float32 for an integer-valued or real field array I.

    x = float64(b_t) * I; 'tanh' -> fl32(tanh(x)) using the C library tanh;
    'lut' -> the L-level staircase of x."""
    I = np.asarray(I, dtype=np.float64)
    flat = I.ravel()
    uniq, inv = np.unique(flat, return_inverse=True)
    b = float(np.float32(b_t))
    if act == "tanh":
        vals = np.array([math.tanh(b * v) for v in uniq], dtype=np.float64)
    elif act == "lut":
        vals = np.array([lut_tanh(b * v, lut_levels) for v in uniq], dtype=np.float64)
    else:
        raise ValueError(act)
    return vals.astype(np.float32)[inv].reshape(I.shape)


def delta(tau: np.ndarray, s: np.ndarray, xi: float, eta_t: float, z: np.ndarray) -> np.ndarray:
    """The argument of the sign in Eq. 4, in float32: (tau + xi*s) + eta*z."""
    tau = np.asarray(tau, dtype=np.float32)
    xi32 = np.float32(xi)
    a = tau + np.where(s > 0, xi32, -xi32).astype(np.float32)
    n = np.float32(eta_t) * np.asarray(z, dtype=np.float32)
    return (a + n).astype(np.float32)


def decide(tau: np.ndarray, s: np.ndarray, xi: float, eta_t: float, z: np.ndarray) -> np.ndarray:
    """Eq. 4 sign decision in float32: s' = +1 iff delta >= 0 (sign(0) = +1)."""
    return np.where(delta(tau, s, xi, eta_t, z) >= np.float32(0.0), 1, -1).astype(np.int8)


# ---------------------------------------------------------------------------------------
# Fixed-point emulation of the FPGA datapath (supplementary quantization section).
# ---------------------------------------------------------------------------------------
def quantize(v, total_bits: int, int_bits: int) -> np.ndarray:
    """ap_fixed<W, I, AP_TRN_ZERO, AP_SAT>: signed, I integer bits (sign included), W - I
    fractional bits; truncation toward zero, then saturation to [-2^(I-1), 2^(I-1) - 2^-F]."""
    F = total_bits - int_bits
    step = 2.0 ** -F
    q = np.trunc(np.asarray(v, dtype=np.float64) / step) * step
    return np.clip(q, -(2.0 ** (int_bits - 1)), 2.0 ** (int_bits - 1) - step)


def decide_fixed(I, s, c: float, beta_t, xi: float, eta_t, z, total_bits: int, int_bits: int,
                 act: str = "tanh", lut_levels: int = 4) -> np.ndarray:
    """Eq. 4 with every intermediate in ap_fixed<W, I> (the reading of the datapath order):
    u = Q(c I) (normalisation after the multiply-accumulate), x = Q(beta_t u),
    tau = Q(act(x)), a = Q(tau + s Q(xi)), n = Q(Q(eta_t) Q(z)), delta = Q(a + n),
    s' = +1 iff delta >= 0.  Products and sums of quantized values are formed exactly."""
    Q = lambda v: quantize(v, total_bits, int_bits)  # noqa: E731
    u = Q(float(c) * np.asarray(I, dtype=np.float64))
    x = Q(float(np.float32(beta_t)) * u)
    if act == "tanh":
        tau = Q(np.tanh(x))
    else:
        tau = Q(np.vectorize(lambda v: lut_tanh(float(v), lut_levels))(x))
    a = Q(tau + np.where(np.asarray(s) > 0, 1.0, -1.0) * Q(float(np.float32(xi))))
    n = Q(Q(float(np.float32(eta_t))) * Q(np.asarray(z, dtype=np.float64)))
    d = Q(a + n)
    return np.where(d >= 0.0, 1, -1).astype(np.int8)


def round_bf16(x) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 value (8 significant bits, ties to even),
    returned as float64: x = m 2^e with 1/2 <= |m| < 1, kept as rint(256 m) 2^(e-8)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0), e - 8)


# ---------------------------------------------------------------------------------------
# Field (Eq. 2) and energy (Eq. 1).
# ---------------------------------------------------------------------------------------
def _is_integer_valued(J) -> bool:
    return np.issubdtype(np.asarray(J).dtype, np.integer)


def field(J, h, S) -> np.ndarray:
    """I[r, i] = sum_j J_ij S[r, j] + h_i for a batch of spin rows S (R x n)."""
    Jf = np.asarray(J, dtype=np.float64)
    hf = np.asarray(h, dtype=np.float64)
    I = np.asarray(S, dtype=np.float64) @ Jf.T + hf[None, :]
    if _is_integer_valued(J) and _is_integer_valued(h):
        return np.rint(I).astype(np.int64)
    return I


def energy(J, h, S) -> np.ndarray:
    """H(s) = -1/2 s^T J s - h^T s for each row of S (J symmetric, zero diagonal), which
    is Eq. 1.  Integer J gives exact int64."""
    S = np.atleast_2d(S)
    I = field(J, h, S)
    hs = np.asarray(h, dtype=np.float64)[None, :]
    if _is_integer_valued(J) and _is_integer_valued(h):
        tot = (S.astype(np.int64) * (I + np.asarray(h, dtype=np.int64)[None, :])).sum(axis=1)
        return -(tot // 2)
    return -0.5 * (S.astype(np.float64) * (I + hs)).sum(axis=1)


def _imax(J, h) -> int:
    return int((np.abs(np.asarray(J, dtype=np.int64)).sum(axis=1) +
                np.abs(np.asarray(h, dtype=np.int64))).max())


# ---------------------------------------------------------------------------------------
# PIMI anneal (Eq. 4 / Box 1, blue) and conventional sequential PIM (Eq. 3 / Box 1, orange).
# ---------------------------------------------------------------------------------------
def anneal(J, h, c: float, beta, eta, xi: float, *, replicas: int | None = None,
           sweeps: int | None = None, seed: int = 0, q: int = 0, t_begin: int = 0,
           init: np.ndarray | None = None, target: float | None = None,
           noise: str = "gauss", act: str = "tanh", lut_levels: int = 4,
           replica_ids=None, record: bool = False, record_states: bool = False,
           prev: dict | None = None, fixed: tuple | None = None) -> dict:
    """Run fully parallel PIMI sweeps t = t_begin .. t_begin+sweeps-1.

    Each sweep: fields I(t) = J s(t) + h (Eq. 2); energy H(s(t)) (Eq. 1) with best and
    first-hit bookkeeping; then every spin decides s_i(t+1) from Eq. 4 with the draws
    described in the module docstring.  After the loop H(s(T)) is evaluated once more.
    Returns best_E, best_t, first_hit (-1 if never), final_E, best_state, final_state
    (and 'energies', shape (sweeps+1, R), when record=True).  fixed = (W, I) replaces the
    float32 decision by the ap_fixed<W, I> datapath of decide_fixed."""
    J = np.asarray(J)
    h = np.asarray(h)
    n = J.shape[0]
    beta = np.asarray(beta, dtype=np.float32)
    eta = np.asarray(eta, dtype=np.float32)
    if sweeps is None:
        sweeps = len(beta) - t_begin
    if replica_ids is None:
        replica_ids = np.arange(replicas)
    replica_ids = np.asarray(replica_ids, dtype=np.int64)
    R = len(replica_ids)
    integer = _is_integer_valued(J) and _is_integer_valued(h)
    z_table = gaussian_quantiles() if noise == "gauss" else uniform_levels()

    if prev is not None:
        s = prev["final_state"].copy()
        best_E = prev["best_E"].copy()
        best_t = prev["best_t"].copy()
        first_hit = prev["first_hit"].copy()
        best_state = prev["best_state"].copy()
    else:
        s = (np.asarray(init, dtype=np.int8).copy() if init is not None
             else init_spin_draw(seed, q, replica_ids, n))
        best_E = np.full(R, np.inf)
        best_t = np.full(R, -1, np.int64)
        first_hit = np.full(R, -1, np.int64)
        best_state = s.copy()

    traj = []
    states = [s.copy()] if record_states else None

    def bookkeep(E, t):
        nonlocal best_E
        better = E < best_E
        best_E = np.where(better, E, best_E)
        best_t[better] = t
        best_state[better] = s[better]
        if target is not None:
            hit = (E <= target) & (first_hit < 0)
            first_hit[hit] = t
        if record:
            traj.append(np.asarray(E, dtype=np.float64).copy())

    ivec = np.arange(n)
    for t in range(t_begin, t_begin + sweeps):
        I = field(J, h, s)                                  # Eq. 2, all i and r
        E = energy(J, h, s)                                 # Eq. 1 of s(t)
        bookkeep(E, t)
        d = noise_draw16(seed, q, replica_ids[:, None], t, ivec[None, :])
        z = z_table[d >> 4]
        if fixed is not None:                               # fixed-point datapath
            s = decide_fixed(I, s, c, beta[t], xi, eta[t], z, fixed[0], fixed[1], act,
                             lut_levels)
        else:
            b_t = np.float32(np.float64(beta[t]) * c)
            tau = activation(b_t, I, act, lut_levels)
            s = decide(tau, s, xi, eta[t], z)               # Eq. 4, synchronous
        if record_states:
            states.append(s.copy())
    E = energy(J, h, s)
    bookkeep(E, t_begin + sweeps)
    out = dict(best_E=best_E if not integer else best_E.astype(np.int64),
               best_t=best_t, first_hit=first_hit,
               final_E=E if not integer else E.astype(np.int64),
               best_state=best_state, final_state=s)
    if record:
        out["energies"] = np.stack(traj)
    if record_states:
        out["states"] = np.stack(states)
    return out


def neighbour_triggered_flip_rate(J, states) -> np.ndarray:
    """P_NT(t) of the supplementary section on coupled oscillations: over all spins i and
    replicas, the fraction of the events "some coupled neighbour j (J_ij != 0) flips at step
    t" in which spin i flips at the same step.  states: (T+1, R, n) -> P_NT: (T,)."""
    adj = (np.asarray(J) != 0).astype(np.int64)
    np.fill_diagonal(adj, 0)
    flips = (states[1:] != states[:-1]).astype(np.int64)          # (T, R, n)
    nb_flip = (flips @ adj.T) > 0                                  # neighbour flipped
    both = (flips > 0) & nb_flip
    den = nb_flip.sum(axis=(1, 2)).astype(np.float64)
    return np.where(den > 0, both.sum(axis=(1, 2)) / np.maximum(den, 1), 0.0)


def anneal_sequential(J, h, c: float, beta, eta, *, replicas: int, steps: int, seed: int = 0,
                      q: int = 0, init: np.ndarray | None = None, noise: str = "uniform",
                      xi: float = 0.0) -> np.ndarray:
    """Conventional PIM with sequential updates (Eq. 3, Box 1 orange): step t updates only
    spin i = t mod N, from the field of the current state, with draw counter
    (i>>3, r, t, q).  beta/eta are indexed by the step t.  Returns the final states.
    (xi is kept as a parameter so the same loop can show Eq. 4 sequentially; Eq. 3 is
    xi = 0.)"""
    J = np.asarray(J)
    h = np.asarray(h)
    n = J.shape[0]
    rids = np.arange(replicas)
    z_table = gaussian_quantiles() if noise == "gauss" else uniform_levels()
    s = (np.asarray(init, dtype=np.int8).copy() if init is not None
         else init_spin_draw(seed, q, rids, n))
    for t in range(steps):
        i = t % n
        Ii = (np.asarray(J[i], dtype=np.float64)[None, :] * s).sum(axis=1) + float(h[i])
        if _is_integer_valued(J):
            Ii = np.rint(Ii).astype(np.int64)
        b_t = np.float32(np.float64(beta[t]) * c)
        tau = activation(b_t, Ii, "tanh")
        d = noise_draw16(seed, q, rids, t, i)
        s[:, i] = decide(tau, s[:, i], xi, eta[t], z_table[d >> 4])
    return s


def anneal_sequential_sweeps(J, h, c: float, beta, eta, xi: float = 0.0, *, replicas: int,
                             sweeps: int | None = None, seed: int = 0, q: int = 0,
                             t_begin: int = 0, init: np.ndarray | None = None,
                             target: float | None = None, noise: str = "uniform",
                             act: str = "tanh", lut_levels: int = 4,
                             prev: dict | None = None) -> dict:
    """Conventional PIM with sequential updates (Eq. 3, Box 1 orange path), organised in
    sweeps like the parallel loop: sweep k (schedule entry k) updates spins i = 0 .. n-1 one
    after another, each from the field of the current state, with the draw of counter
    (i>>3, r, k, q), beta_k, eta_k and (for xi > 0) the inertia term of Eq. 4 -- the same
    numbers the parallel loop draws in sweep k.  Energies are evaluated on the state at the
    start of every sweep and on the final state, with the bookkeeping of `anneal`; the
    returned dict has the same keys."""
    J = np.asarray(J)
    h = np.asarray(h)
    n = J.shape[0]
    beta = np.asarray(beta, dtype=np.float32)
    eta = np.asarray(eta, dtype=np.float32)
    if sweeps is None:
        sweeps = len(beta) - t_begin
    rids = np.arange(replicas)
    integer = _is_integer_valued(J) and _is_integer_valued(h)
    z_table = gaussian_quantiles() if noise == "gauss" else uniform_levels()
    if prev is not None:
        s = prev["final_state"].copy()
        best_E = prev["best_E"].astype(np.float64)
        best_t = prev["best_t"].copy()
        first_hit = prev["first_hit"].copy()
        best_state = prev["best_state"].copy()
    else:
        s = (np.asarray(init, dtype=np.int8).copy() if init is not None
             else init_spin_draw(seed, q, rids, n))
        best_E = np.full(replicas, np.inf)
        best_t = np.full(replicas, -1, np.int64)
        first_hit = np.full(replicas, -1, np.int64)
        best_state = s.copy()

    def bookkeep(t):
        nonlocal best_E
        E = energy(J, h, s)
        better = E < best_E
        best_E = np.where(better, E, best_E)
        best_t[better] = t
        best_state[better] = s[better]
        if target is not None:
            hit = (E <= target) & (first_hit < 0)
            first_hit[hit] = t
        return E

    for k in range(t_begin, t_begin + sweeps):
        bookkeep(k)
        b_k = np.float32(np.float64(beta[k]) * c)
        for i in range(n):
            Ii = field(J[i:i + 1], h[i:i + 1], s)[:, 0]      # Eq. 2 for spin i, current state
            tau = activation(b_k, Ii, act, lut_levels)
            d = noise_draw16(seed, q, rids, k, i)
            s[:, i] = decide(tau, s[:, i], xi, eta[k], z_table[d >> 4])
    E = bookkeep(t_begin + sweeps)
    return dict(best_E=best_E.astype(np.int64) if integer else best_E, best_t=best_t,
                first_hit=first_hit, final_E=E.astype(np.int64) if integer else E,
                best_state=best_state, final_state=s)


# ---------------------------------------------------------------------------------------
# Trials to solution (supplementary CCTS section).
# ---------------------------------------------------------------------------------------
def n_trials(p_bar: float, eps: float = 1e-3) -> float:
    """n = log(eps) / log(1 - p_bar): independent trials needed for success with
    probability 1 - eps (no ceiling, as in the supplementary equation)."""
    if p_bar >= 1.0:
        return 1.0
    if p_bar <= 0.0:
        return math.inf
    return math.log(eps) / math.log(1.0 - p_bar)


def tts99(wall_seconds_per_trial: float, p_bar: float) -> float:
    """Time to solution at 99 % confidence: per-trial time x n_trials(p_bar, 0.01)."""
    return wall_seconds_per_trial * n_trials(p_bar, 0.01)
