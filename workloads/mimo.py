"""Seeded uplink MIMO detection problems (supplementary section on uplink MIMO instance
generation): i.i.d. Rayleigh channel, uniformly drawn Gray-coded QAM symbols, complex AWGN
whose variance is set from Eb/N0 and the empirical received power.

Only data is produced here (channels, symbols, their bits, received vectors); the
detection arithmetic (MMSE, the Ising formulation, reconstruction) lives elsewhere.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_DOMAIN_MIMO = 0x4D49  # "MI"


def pam_gray(m_levels: int):
    """Levels of one real dimension of square QAM (sqrt(M)-PAM: -L+1, -L+3, .., L-1) and the
    Gray code of each level (bits as an int, most significant first): adjacent levels differ
    in exactly one bit."""
    L = m_levels
    levels = np.arange(-L + 1, L, 2, dtype=np.float64)
    codes = np.array([k ^ (k >> 1) for k in range(L)], dtype=np.int64)
    return levels, codes


def qam_bits_per_symbol(qam: int) -> int:
    return int(round(np.log2(qam)))


def symbols_from_bits(bits: np.ndarray, qam: int) -> np.ndarray:
    """Gray-coded square QAM: the first half of a symbol's bits select the real level, the
    second half the imaginary level.  bits: (..., b) of 0/1 -> complex symbols (...)."""
    b = qam_bits_per_symbol(qam)
    half = b // 2
    L = int(round(np.sqrt(qam)))
    levels, codes = pam_gray(L)
    inv = np.empty(L, np.int64)
    inv[codes] = np.arange(L)
    w = 1 << np.arange(half - 1, -1, -1)
    re = (bits[..., :half] * w).sum(-1)
    im = (bits[..., half:] * w).sum(-1)
    return levels[inv[re]] + 1j * levels[inv[im]]


def bits_from_symbols(sym: np.ndarray, qam: int) -> np.ndarray:
    """Inverse of symbols_from_bits for constellation points."""
    b = qam_bits_per_symbol(qam)
    half = b // 2
    L = int(round(np.sqrt(qam)))
    levels, codes = pam_gray(L)
    def idx(v):
        return np.rint((np.asarray(v) + L - 1) / 2).astype(np.int64)
    cr = codes[idx(sym.real)]
    ci = codes[idx(sym.imag)]
    shifts = np.arange(half - 1, -1, -1)
    br = (cr[..., None] >> shifts) & 1
    bi = (ci[..., None] >> shifts) & 1
    return np.concatenate([br, bi], axis=-1)


@dataclasses.dataclass
class MimoProblem:
    nt: int
    nr: int
    qam: int
    ebn0_db: float
    H: np.ndarray      # complex (nr, nt), entries CN(0, 1)
    x: np.ndarray      # complex (nt,), transmitted symbols
    bits: np.ndarray   # (nt, log2 qam) of 0/1
    y: np.ndarray      # complex (nr,), received
    sigma2: float      # complex noise variance
    es_n0: float       # b * Eb/N0 (linear)
    seed: int


def mimo_problem(nt: int, nr: int, qam: int, ebn0_db: float, seed: int) -> MimoProblem:
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(
        [_DOMAIN_MIMO, nt, nr, qam, seed])))
    b = qam_bits_per_symbol(qam)
    H = (g.standard_normal((nr, nt)) + 1j * g.standard_normal((nr, nt))) / np.sqrt(2.0)
    bits = g.integers(0, 2, size=(nt, b))
    x = symbols_from_bits(bits, qam)
    y_rec = H @ x
    e_y = float(np.mean(np.abs(y_rec) ** 2))
    es_n0 = b * 10.0 ** (ebn0_db / 10.0)
    sigma2 = e_y / es_n0
    n = np.sqrt(sigma2 / 2.0) * (g.standard_normal(nr) + 1j * g.standard_normal(nr))
    return MimoProblem(nt, nr, qam, ebn0_db, H, x, bits, y_rec + n, sigma2, es_n0, seed)


def mimo_schedule(steps: int, gamma_init: float = 0.01, gamma_final: float = 1.0):
    """The MIMO schedule of the supplementary PIMI-for-MIMO section: beta(t) = 1 and
    eta(t) = sqrt(1 / (5 gamma(t))) with gamma linear from gamma_init to gamma_final (the
    paper does not print the two ends; these defaults are the values tuned here)."""
    t = np.arange(steps, dtype=np.float64)
    gamma = gamma_init + (gamma_final - gamma_init) * (t / max(steps - 1, 1))
    return np.ones(steps, np.float32), np.sqrt(1.0 / (5.0 * gamma)).astype(np.float32)


def mimo_scale(nr: int) -> float:
    """Coupling scale c = 2 / N_r applied to the accumulated field (tuned here; the paper's
    fixed-point MIMO pipeline does not print one)."""
    return 2.0 / nr


MIMO_XI = 1.0  # inertia used with the schedule above (tuned here; the paper uses 2 for its scaling)
