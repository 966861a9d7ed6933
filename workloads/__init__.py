"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the bench.

This package draws problem instances, schedules and initial spins.  It holds none of
the annealing arithmetic (no fields, no noise stream, no decisions); both the oracle
and the CUDA library consume what it produces.
"""
from .generators import (  # noqa: F401
    maxcut_er,
    sk_pm1,
    maxcut_gauss,
    linear_beta,
    eta_power,
    coupling_scale,
    random_spins,
    Instance,
    sk_batch,
    uneven_batch,
    uneven_sizes,
    uneven_instance,
)
from .mimo import (  # noqa: F401
    MimoProblem,
    mimo_problem,
    pam_gray,
    qam_bits_per_symbol,
    symbols_from_bits,
    bits_from_symbols,
    mimo_schedule,
    mimo_scale,
    MIMO_XI,
)
