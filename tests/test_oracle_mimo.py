"""Pins of the MIMO-detection oracle (DI-MIMO formulation, MMSE, ML, reconstruction, BER)
against facts the mathematics fixes, and checks of the library's host-side formulation
(pim_mimo_formulate / pim_mimo_reconstruct: FP64 host code, no device work) against it."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import mimo as om
from workloads import bits_from_symbols, mimo_problem, pam_gray, symbols_from_bits

WEIGHTS = {4: [1, 1], 16: [1, 1], 64: [2, 1, 1]}
LEVELS = {4: 2, 16: 4, 64: 8}


def test_gray_code_neighbours_differ_in_one_bit_and_round_trip():
    for L in (2, 4, 8):
        _, codes = pam_gray(L)
        assert all(bin(a ^ b).count("1") == 1 for a, b in zip(codes, codes[1:]))
    for qam in (4, 16, 64):
        b = int(np.log2(qam))
        bits = np.array(list(itertools.product((0, 1), repeat=b)))
        sym = symbols_from_bits(bits, qam)
        assert len(set(sym.tolist())) == qam
        assert np.array_equal(bits_from_symbols(sym, qam), bits)


def test_slicer_picks_the_nearest_level():
    v = np.linspace(-6, 6, 1201)
    got = om.slice_pam(v, 4)
    levels = np.array([-3.0, -1.0, 1.0, 3.0])
    dist = np.abs(v[:, None] - levels[None, :])
    ok = np.isclose(np.abs(v - got), dist.min(axis=1))
    assert ok.all()


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_di_mimo_energy_is_the_residual_norm_up_to_a_constant(qam):
    """H(s) = -1/2 s^T J s - h^T s differs from ||y - H(x_m + T s)||^2 by one constant for
    every spin vector (the substitution of the DI-MIMO section)."""
    p = mimo_problem(4, 5, qam, 8.0, 3)
    L = LEVELS[qam]
    xm = om.mmse(p.H, p.y, 0.2, L)
    J, h = om.di_mimo(p.H, p.y, xm, WEIGHTS[qam])
    n = J.shape[0]
    rng = np.random.default_rng(0)
    S = np.where(rng.random((50, n)) < 0.5, -1, 1).astype(np.int8)
    E = oracle.energy(J, h, S)
    Hr, yr = om.real_equivalent(p.H, p.y)
    xr = np.concatenate([xm.real, xm.imag])
    T = om.transform(WEIGHTS[qam], 2 * p.nt)
    res = np.array([np.sum((yr - Hr @ (xr + T @ s)) ** 2) for s in S.astype(np.float64)])
    diff = res - E
    assert np.allclose(diff, diff[0], rtol=0, atol=1e-8 * np.abs(res).max())


def test_mmse_recovers_symbols_without_noise_and_ml_is_optimal():
    """Noise-free, a tiny regulariser (zero forcing) and exhaustive ML both return the
    transmitted vector; with noise ML's residual is never above MMSE's."""
    p = mimo_problem(4, 4, 16, 10.0, 5)
    y0 = p.H @ p.x
    assert np.array_equal(om.mmse(p.H, y0, 1e-9, 4), p.x)
    assert np.array_equal(om.ml_exhaustive(p.H, y0, 4), p.x)
    xml = om.ml_exhaustive(p.H, p.y, 4)
    assert om.residual(p.H, p.y, xml) <= om.residual(p.H, p.y, om.mmse(p.H, p.y, 0.1, 4)) + 1e-12
    assert om.residual(p.H, p.y, xml) <= om.residual(p.H, p.y, p.x) + 1e-12


def test_reconstruction_covers_one_step_corrections():
    """With T = [I, I] the pair (s1, s2) gives corrections s1 + s2 in {-2, 0, 2}: every
    constellation point one level away from the estimate is reached, and slicing keeps the
    result on the constellation."""
    xm = np.array([-3 + 1j, 1 - 1j])
    seen = set()
    for s in itertools.product((-1, 1), repeat=8):
        x = om.reconstruct(xm, np.array(s), [1, 1], 4)
        assert np.all(np.isin(x.real, [-3, -1, 1, 3])) and np.all(np.isin(x.imag, [-3, -1, 1, 3]))
        seen.add(tuple(x.round(6)))
    assert (-1 + 3j, 3 - 3j) in {(complex(a), complex(b)) for a, b in seen}


def test_ber_definition():
    p = mimo_problem(4, 4, 16, 10.0, 1)
    assert om.ber(p.bits, bits_from_symbols(p.x, 16)) == 0.0
    flipped = p.bits.copy()
    flipped[0, 0] ^= 1
    assert om.ber(p.bits, flipped) == 1.0 / p.bits.size


# ------------------------------------------- library host code (FP64, no device compute)
@pytest.mark.parametrize("nt,nr,qam", [(4, 4, 16), (16, 16, 16), (8, 10, 4), (4, 4, 64)])
def test_library_formulation_matches_oracle(nt, nr, qam):
    from paper_2604_17109_gb300 import build
    build.build()
    from paper_2604_17109_gb300 import pim as P
    p = mimo_problem(nt, nr, qam, 12.0, 2)
    J, h, xm = P.pim_mimo_formulate(p.H, p.y, qam, 0.1)
    xo = om.mmse(p.H, p.y, 0.1, LEVELS[qam])
    Jo, ho = om.di_mimo(p.H, p.y, xo, WEIGHTS[qam])
    assert np.array_equal(xm, xo)
    scale = np.abs(Jo).max()
    assert np.abs(J - Jo).max() <= 1e-12 * scale
    assert np.abs(h - ho).max() <= 1e-12 * max(1.0, np.abs(ho).max())
    rng = np.random.default_rng(1)
    for _ in range(5):
        s = np.where(rng.random(J.shape[0]) < 0.5, -1, 1).astype(np.int8)
        assert np.array_equal(P.pim_mimo_reconstruct(xm, s, qam),
                              om.reconstruct(xo, s, WEIGHTS[qam], LEVELS[qam]))


@pytest.mark.parametrize("nt,nr,qam,depth", [(4, 4, 16, 3), (8, 8, 4, 3), (4, 6, 64, 2), (16, 16, 16, 2)])
def test_library_formulation_with_explicit_depth_matches_oracle(nt, nr, qam, depth):
    """Either correction set on any constellation: T = [I, I] (depth 2) or [2I, I, I]
    (depth 3)."""
    from paper_2604_17109_gb300 import build
    build.build()
    from paper_2604_17109_gb300 import pim as P
    weights = (1.0, 1.0) if depth == 2 else (2.0, 1.0, 1.0)
    p = mimo_problem(nt, nr, qam, 12.0, 5)
    J, h, xm = P.pim_mimo_formulate(p.H, p.y, qam, 0.1, depth=depth)
    assert J.shape == (depth * 2 * nt, depth * 2 * nt)
    xo = om.mmse(p.H, p.y, 0.1, LEVELS[qam])
    Jo, ho = om.di_mimo(p.H, p.y, xo, weights)
    assert np.array_equal(xm, xo)
    assert np.abs(J - Jo).max() <= 1e-12 * np.abs(Jo).max()
    assert np.abs(h - ho).max() <= 1e-12 * max(1.0, np.abs(ho).max())
    rng = np.random.default_rng(3)
    for _ in range(5):
        s = np.where(rng.random(J.shape[0]) < 0.5, -1, 1).astype(np.int8)
        assert np.array_equal(P.pim_mimo_reconstruct(xm, s, qam, depth=depth),
                              om.reconstruct(xo, s, weights, LEVELS[qam]))
    with pytest.raises(P.PimError):
        P.pim_mimo_formulate(p.H, p.y, qam, 0.1, depth=4)
