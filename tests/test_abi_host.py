"""CPU-side checks of the C ABI library: it loads, exports every symbol include/pim.h
declares, its host-built constant tables equal the oracle's, and argument validation
rejects bad input before any device work.  No GPU is needed."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2604_17109_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pim():
    pkg_build.build()
    from paper_2604_17109_gb300 import pim as mod
    mod.lib()
    return mod


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "pim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(pim_[a-z_0-9]+)\s*\(", text))


def test_every_declared_symbol_is_exported(pim):
    declared = _declared_symbols()
    assert {"pim_create", "pim_set_schedule", "pim_anneal", "pim_anneal_batch", "pim_energies",
            "pim_best_state", "pim_submit", "pim_poll", "pim_destroy"} <= declared
    lib = pim.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(pim.SIGNATURES), "binding signatures out of step with the header"


def test_noise_levels_equal_oracle(pim):
    assert np.array_equal(pim.pim_noise_levels("gauss"), oracle.gaussian_quantiles())
    assert np.array_equal(pim.pim_noise_levels("uniform"), oracle.uniform_levels())


@pytest.mark.parametrize("b", [0.0, 0.0707107, 0.2121, 1.7, 12.5])
def test_activation_levels_equal_oracle(pim, b):
    imax = 300
    I = np.arange(-imax, imax + 1)
    assert np.array_equal(pim.pim_activation_levels(b, imax, "tanh"),
                          oracle.activation(np.float32(b), I, "tanh"))
    for L in (2, 3, 4, 16):
        assert np.array_equal(pim.pim_activation_levels(b, imax, "lut", L),
                              oracle.activation(np.float32(b), I, "lut", L))


def test_invalid_arguments_are_rejected_on_host(pim):
    J = np.zeros((4, 4), np.int8)
    J[0, 1] = 1  # asymmetric
    with pytest.raises(pim.PimError) as e:
        pim.pim_create(J)
    assert e.value.code == pim.PIM_ERR_INVALID
    J = np.eye(3, dtype=np.int8)  # non-zero diagonal
    with pytest.raises(pim.PimError) as e:
        pim.pim_create(J)
    assert e.value.code == pim.PIM_ERR_INVALID
    J = np.zeros((3, 3), np.int8)
    J[0, 1] = J[1, 0] = 17  # not exactly representable in the FP8 operand
    with pytest.raises(pim.PimError) as e:
        pim.pim_create(J)
    assert e.value.code == pim.PIM_ERR_INVALID
    with pytest.raises(pim.PimError) as e:
        pim.pim_create(np.zeros((3, 3), np.int8), scale_c=0.0)
    assert e.value.code == pim.PIM_ERR_INVALID
    with pytest.raises(pim.PimError) as e:
        pim.pim_activation_levels(1.0, -1)
    assert e.value.code == pim.PIM_ERR_INVALID
    with pytest.raises(pim.PimError) as e:
        pim.pim_poll(123456789)
    assert e.value.code == pim.PIM_ERR_INVALID


@pytest.mark.parametrize("n", [2, 7, 8, 9, 16, 23, 64, 200, 257])
def test_validation_finds_first_asymmetry_and_range_errors(pim, n):
    """The host checks of integer couplings (8 x 8 block transposes, byte row sums) report
    the first asymmetric pair in row-major order and the first out-of-range entry, at sizes
    with and without a ragged edge; a valid matrix passes them (it then fails only where no
    GPU is present, with a CUDA error)."""
    import re
    rng = np.random.default_rng(n)
    A = rng.integers(-16, 17, size=(n, n))
    J = np.triu(A, 1)
    J = (J + J.T).astype(np.int8)
    try:
        pim.pim_destroy(pim.pim_create(J))
    except pim.PimError as e:
        assert e.code != pim.PIM_ERR_INVALID, str(e)
    for _ in range(6):
        i, j = sorted(rng.choice(n, size=2, replace=False))
        K = J.copy()
        K[j, i] = np.int8(K[j, i] + (1 if K[j, i] < 16 else -1))  # lower triangle: first hit is (i, j)
        with pytest.raises(pim.PimError) as e:
            pim.pim_create(K)
        assert e.value.code == pim.PIM_ERR_INVALID
        assert re.search(rf"not symmetric at \({i}, {j}\)", str(e.value)), str(e.value)
        K = J.copy()
        K[i, j] = K[j, i] = -17 if _ % 2 else -128
        with pytest.raises(pim.PimError) as e:
            pim.pim_create(K)
        assert e.value.code == pim.PIM_ERR_INVALID
        assert re.search(rf"\|J\[{i}\]\[{j}\]\| = {17 if _ % 2 else 128} > 16", str(e.value)), str(e.value)


def test_autotune_mode_and_report_on_the_host(pim):
    """pim_autotune takes modes 0 and 1 only; the tuning report is text (empty when nothing
    was measured and no cache file is named)."""
    with pytest.raises(pim.PimError) as e:
        pim.pim_autotune(2)
    assert e.value.code == pim.PIM_ERR_INVALID
    pim.pim_autotune(0)
    pim.pim_autotune(1)
    assert isinstance(pim.pim_tune_report(), str)
