"""Per-step quantities of the block Davidson method (oracle; test infrastructure only).

App. A.2.1: start from orthonormal trial orbitals psi_i with eps_i = <psi_i|H|psi_i>; form the
residuals g_i = (H - eps_i S) psi_i and the corrections delta psi_i = D g_i, D a diagonal
approximation to (H - eps_i S)^{-1} in the PW basis, <k+G|D|k+G'> = delta_GG' / <k+G|H - eps S|k+G>;
solve the reduced problem sum_k (H_jk - eps S_jk) c_k = 0 in the span of {psi_i, delta psi_i}
with H_jk = <phi_j|H|phi_k>, S_jk = <phi_j|S|phi_k>; take psi_i <- sum_j c^(i)_j phi_j.

Readings (S = I for norm-conserving projectors):

* eps in the diagonal of D is taken per band, eps_i, and the denominator is kept away from
  zero: x -> x if |x| >= tau, else +tau for x >= 0 and -tau for x < 0 (tau = 0.1 Ha default);
* the diagonal <k+G|H|k+G> keeps the kinetic term, the mean of V and the nonlocal diagonal.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def residuals(hpsi: np.ndarray, psi: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """g_i = H psi_i - eps_i psi_i, [nb][npw]."""
    return hpsi - np.asarray(eps, dtype=np.float64)[:, None] * psi


def residual_norms(g: np.ndarray) -> np.ndarray:
    """||g_i||_2 per band."""
    return np.sqrt(np.sum(np.abs(g) ** 2, axis=1))


def clamp_denominator(x: np.ndarray, tau: float) -> np.ndarray:
    out = np.array(x, dtype=np.float64, copy=True)
    small = np.abs(out) < tau
    out[small] = np.where(out[small] >= 0.0, tau, -tau)
    return out


def precondition(g: np.ndarray, hdiag: np.ndarray, eps: np.ndarray, tau: float = 0.1) -> np.ndarray:
    """delta psi_i(G) = g_i(G) / (H_GG - eps_i), denominator clamped to |.| >= tau."""
    denom = clamp_denominator(np.asarray(hdiag)[None, :] - np.asarray(eps)[:, None], tau)
    return g / denom


def reduced_matrices(phi: np.ndarray, hphi: np.ndarray) -> tuple:
    """H_jk = <phi_j|H|phi_k>, S_jk = <phi_j|phi_k> for a basis phi [m][npw]."""
    h = np.conj(phi) @ hphi.T
    s = np.conj(phi) @ phi.T
    return h, s


def rayleigh_ritz(phi: np.ndarray, hphi: np.ndarray, nbnd: int) -> tuple:
    """Lowest nbnd solutions of (H_sub - eps S_sub) c = 0; returns (eps, psi, hpsi)."""
    h, s = reduced_matrices(phi, hphi)
    h = 0.5 * (h + h.conj().T)
    s = 0.5 * (s + s.conj().T)
    w, c = scipy.linalg.eigh(h, s)
    c = c[:, :nbnd]
    return w[:nbnd], c.T @ phi, c.T @ hphi
