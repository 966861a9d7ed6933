"""CPU oracle of the MIMO-detection formulation -- TEST INFRASTRUCTURE ONLY.

Plain numpy in float64, written from the supplementary sections on MIMO detection:
  * real-valued equivalent of the complex model (section "Real-Valued equivalent");
  * linear MMSE filter with hard slicing (section "Baseline: linear MMSE detector", the
    printed filter (H^H H + I / (Es/N0))^-1 H^H);
  * Delta-Ising MIMO (DI-MIMO) formulation: correction d = u - x_m = T s, and the Ising
    parameters J = -zeroDiag(T^T H^T H T), h = 2 (y - H x_m)^T H T of the paper's Ising form
    -h^T s - s^T J s (section "Spin representation and Ising mapping"); the library's
    energy is Eq. 1, H(s) = -1/2 s^T J' s - h^T s, so J' = 2 J here;
  * reconstruction x_hat = slice(x_m + T s) (section "Reconstruction of the transmitted
    signal");
  * exhaustive maximum-likelihood detection (section "Maximum-Likelihood (ML) detection");
  * bit-error rate (section "Performance metric: bit-error rate").
Only the test-suite and the benchmark's verification may call it.
"""
from __future__ import annotations

import itertools

import numpy as np


def real_equivalent(H: np.ndarray, y: np.ndarray):
    """[[Re H, -Im H], [Im H, Re H]] and [Re y; Im y]."""
    Hr = np.block([[H.real, -H.imag], [H.imag, H.real]])
    return Hr, np.concatenate([y.real, y.imag])


def slice_pam(v: np.ndarray, levels: int) -> np.ndarray:
    """Nearest point of {-L+1, -L+3, .., L-1} (ties away from zero are impossible for the
    odd-integer grid except exactly at even integers; those go up)."""
    L = levels
    k = np.floor((np.asarray(v, dtype=np.float64) + L) / 2.0)
    k = np.clip(k, 0, L - 1)
    return 2.0 * k - L + 1


def mmse(H: np.ndarray, y: np.ndarray, reg: float, levels: int) -> np.ndarray:
    """Hard-sliced MMSE estimate: z = (H^H H + reg I)^-1 H^H y, each real / imaginary part
    sliced onto the PAM levels."""
    nt = H.shape[1]
    A = H.conj().T @ H + reg * np.eye(nt)
    z = np.linalg.solve(A, H.conj().T @ y)
    return slice_pam(z.real, levels) + 1j * slice_pam(z.imag, levels)


def transform(weights, two_nt: int) -> np.ndarray:
    """T = [w_1 I, w_2 I, ..] (2nt x len(weights) 2nt)."""
    return np.hstack([w * np.eye(two_nt) for w in weights])


def di_mimo(H: np.ndarray, y: np.ndarray, x_m: np.ndarray, weights):
    """Ising parameters of the residual problem around the estimate x_m (complex), in the
    library's convention H(s) = -1/2 s^T J s - h^T s:  J = -2 zeroDiag(T^T Hr^T Hr T),
    h = 2 T^T Hr^T (yr - Hr xr_m)."""
    Hr, yr = real_equivalent(H, y)
    xr = np.concatenate([x_m.real, x_m.imag])
    T = transform(weights, Hr.shape[1])
    G = T.T @ Hr.T @ Hr @ T
    J = -2.0 * (G - np.diag(np.diag(G)))
    h = 2.0 * T.T @ Hr.T @ (yr - Hr @ xr)
    return J, h


def reconstruct(x_m: np.ndarray, s: np.ndarray, weights, levels: int) -> np.ndarray:
    """slice(x_m + T s), back to complex."""
    nt = x_m.shape[0]
    xr = np.concatenate([x_m.real, x_m.imag])
    d = transform(weights, 2 * nt) @ np.asarray(s, dtype=np.float64)
    u = slice_pam(xr + d, levels)
    return u[:nt] + 1j * u[nt:]


def residual(H: np.ndarray, y: np.ndarray, x: np.ndarray) -> float:
    return float(np.sum(np.abs(y - H @ x) ** 2))


def ml_exhaustive(H: np.ndarray, y: np.ndarray, levels: int) -> np.ndarray:
    """argmin over all QAM vectors of ||y - H u||^2 (levels^(2 nt) candidates, all
    evaluated; the first minimum in enumeration order wins)."""
    nt = H.shape[1]
    pam = np.arange(-levels + 1, levels, 2, dtype=np.float64)
    pts = np.array([a + 1j * b for a in pam for b in pam])
    idx = np.array(list(itertools.product(range(len(pts)), repeat=nt)))
    U = pts[idx]                                    # (candidates, nt)
    res = np.sum(np.abs(y[None, :] - U @ H.T) ** 2, axis=1)
    return U[int(np.argmin(res))]


def ber(bits: np.ndarray, bits_hat: np.ndarray) -> float:
    return float(np.mean(np.asarray(bits) != np.asarray(bits_hat)))
