"""CPU oracle for the PIMI sweep path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy code that restates the paper's update rule step by
step (``pimi.py``), and a second plain statement of the anneal in C++17 (``pimi_ref.cpp``,
loaded through ``cpp.py``) that is pinned to it and timed as the CPU baseline.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never imports, links or calls anything
here, and nothing here imports the library.
"""
from .pimi import (  # noqa: F401
    philox4x32_10,
    noise_draw16,
    init_spin_draw,
    gaussian_quantiles,
    uniform_levels,
    lut_tanh,
    activation,
    decide,
    delta,
    round_bf16,
    quantize,
    decide_fixed,
    field,
    energy,
    anneal,
    anneal_sequential,
    anneal_sequential_sweeps,
    n_trials,
    tts99,
    neighbour_triggered_flip_rate,
)
from .brute import all_energies, ground_state, boltzmann  # noqa: F401
