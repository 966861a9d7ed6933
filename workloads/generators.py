"""Instance, schedule and spin generators (seeded, platform independent).

Every generator takes an explicit integer seed and uses numpy's PCG64 through a
SeedSequence that also mixes in a per-generator domain tag and the size, so two
generators never share a stream.  Results are identical on x86-64 and aarch64.

Instance families follow the paper's benchmark section:
  * Max-Cut: Erdos-Renyi graph, edge probability 0.5, unit weights, J = -A, h = 0
    (supplementary "Max-Cut instance generation", graph construction and Ising mapping).
  * SK-1: symmetric J with i.i.d. +-1 off-diagonal entries, J_ii = 0, h = 0
    (supplementary "SK-1 instance generation").
  * Gaussian-weight Max-Cut (large dense variant): W_ij ~ N(0,1) on an ER(0.5) mask,
    J = -W.  This is a synthetic stand-in; the paper itself only uses unit weights.
Coupling normalisation (2/sqrt(N) for Max-Cut, 1/sqrt(N) for SK) is the scale c that
the library folds into beta; the stored J keeps its integer values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_DOMAIN_MAXCUT = 0x4D43  # "MC"
_DOMAIN_SK = 0x534B      # "SK"
_DOMAIN_GAUSS = 0x4747   # "GG"
_DOMAIN_SPINS = 0x5350   # "SP"
_DOMAIN_UNEVEN = 0x5542  # "UB"


def _rng(domain: int, n: int, seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([domain, n, seed])))


@dataclasses.dataclass
class Instance:
    """A coupling matrix J (row-major n x n), bias h and the coupling scale c."""
    kind: str
    n: int
    J: np.ndarray
    h: np.ndarray
    c: float
    seed: int


def coupling_scale(kind: str, n: int) -> float:
    """c = 2/sqrt(N) for Max-Cut and 1/sqrt(N) for SK-1 (preprocessing paragraphs of the
    two instance-generation sections)."""
    if kind in ("maxcut", "maxcut_gauss"):
        return 2.0 / math.sqrt(n)
    if kind == "sk":
        return 1.0 / math.sqrt(n)
    raise ValueError(kind)


def _upper_to_symmetric(upper: np.ndarray) -> np.ndarray:
    m = np.triu(upper, 1)
    return m + m.T


def maxcut_er(n: int, seed: int, p: float = 0.5) -> Instance:
    """Unweighted Erdos-Renyi Max-Cut: A_ij ~ Bernoulli(p) for i<j, J = -A, h = 0."""
    g = _rng(_DOMAIN_MAXCUT, n, seed)
    a = (g.random((n, n)) < p).astype(np.int8)
    J = (-_upper_to_symmetric(a)).astype(np.int8)
    return Instance("maxcut", n, J, np.zeros(n, np.int32), coupling_scale("maxcut", n), seed)


def sk_pm1(n: int, seed: int) -> Instance:
    """SK-1 spin glass: J_ij = J_ji uniform in {-1,+1} for i != j, J_ii = 0, h = 0."""
    g = _rng(_DOMAIN_SK, n, seed)
    u = np.where(g.random((n, n)) < 0.5, -1, 1).astype(np.int8)
    J = _upper_to_symmetric(u).astype(np.int8)
    return Instance("sk", n, J, np.zeros(n, np.int32), coupling_scale("sk", n), seed)


def sk_batch(n: int, count: int, first_seed: int = 0) -> list[Instance]:
    return [sk_pm1(n, first_seed + k) for k in range(count)]


def maxcut_gauss(n: int, seed: int, p: float = 0.5) -> Instance:
    """Gaussian-weight Max-Cut: W_ij ~ N(0,1) on an ER(p) mask, J = -W (float64)."""
    g = _rng(_DOMAIN_GAUSS, n, seed)
    w = g.standard_normal((n, n)) * (g.random((n, n)) < p)
    J = -_upper_to_symmetric(w)
    return Instance("maxcut_gauss", n, J, np.zeros(n, np.float64),
                    coupling_scale("maxcut_gauss", n), seed)


def linear_beta(steps: int, beta0: float = 0.1, beta1: float = 3.0) -> np.ndarray:
    """Linear inverse-temperature ramp beta_t = beta0 + (beta1-beta0) t/(T-1), float32."""
    if steps == 1:
        return np.array([beta0], np.float32)
    t = np.arange(steps, dtype=np.float64)
    return (beta0 + (beta1 - beta0) * t / (steps - 1)).astype(np.float32)


def eta_power(beta: np.ndarray, divisor: float = 5.0) -> np.ndarray:
    """Noise amplitude eta_t = sqrt(beta_t / 5), the Max-Cut/SK noise schedule as printed."""
    return np.sqrt(beta.astype(np.float64) / divisor).astype(np.float32)


def random_spins(n: int, replicas: int, seed: int) -> np.ndarray:
    """Initial spins in {-1,+1}, int8, shape (replicas, n)."""
    g = _rng(_DOMAIN_SPINS, n, seed)
    return np.where(g.random((replicas, n)) < 0.5, -1, 1).astype(np.int8)


def uneven_sizes(count: int, seed: int = 0, n_min: int = 64, n_max: int = 1024,
                 r_step: int = 32, r_max: int = 512):
    """Sizes and replica counts of uneven_batch: n ~ U{n_min .. n_max}, replicas
    ~ U{r_step, 2 r_step, .., r_max}."""
    g = _rng(_DOMAIN_UNEVEN, count, seed)
    sizes = g.integers(n_min, n_max + 1, size=count)
    reps = r_step * g.integers(1, r_max // r_step + 1, size=count)
    return [int(n) for n in sizes], [int(r) for r in reps]


def uneven_instance(k: int, n: int) -> Instance:
    """Instance k of an uneven batch: Max-Cut (ER 0.5) for even k, SK-1 for odd k, generator
    seed k of its family."""
    return (maxcut_er if k % 2 == 0 else sk_pm1)(n, k)


def uneven_batch(count: int, seed: int = 0, **kw):
    """A batch of `count` instances of uneven size for multi-instance scheduling (see
    uneven_sizes and uneven_instance).  Returns (instances, replicas)."""
    sizes, reps = uneven_sizes(count, seed, **kw)
    return [uneven_instance(k, n) for k, n in enumerate(sizes)], reps
