"""Fock exchange at the Gamma point (oracle; test infrastructure only).

App. A.5: the exchange energy of an insulating, non-magnetic system sums, over pairs of occupied
bands, the Coulomb energy of their codensities psi_v'*(r) psi_v(r); the codensities are formed in
real space, transformed by FFT, and their electrostatic energies accumulated in reciprocal space.
Applying the Fock operator to a wavefunction takes further FFTs and real-space products.  The
integrable 1/q^2 divergence at q -> 0 is handled as Gygi and Baldereschi proposed: a function with
the same divergence is subtracted from the sum over the q grid and its analytic integral over the
Brillouin zone is added back.

Here k = q = 0 (the synthetic cells are Gamma-only).  With physical orbitals phi = psi / Omega^(1/2)
(psi(r) = sum_G psi(G) e^{iG.r}, sum |psi(G)|^2 = 1) and closed shells:
  (V_x phi)(r) = - sum_j phi_j(r) v_j(r),   v_j = Coulomb potential of n_j = phi_j* phi,
  v_j(G) = 4 pi n_j(G) / G^2 (G != 0),       v_j(0) = 4 pi n_j(0) x_div,
  E_x = sum_i <phi_i|V_x|phi_i> = - sum_ij (ij|ji),
with the Gygi-Baldereschi constant for the single q point, auxiliary function e^{-alpha G^2} / G^2:
  x_div = Omega / (2 pi)^3 * 2 pi^(3/2) / alpha^(1/2) - sum_{G != 0} e^{-alpha G^2} / G^2
(the Brillouin-zone integral of the auxiliary function minus its value on the q grid).

Readings:
* With one q point the paper's estimate of the 0/0 term at q = 0 from a twice coarser grid is
  not available; that term is left out (the paper notes the error it leaves falls as 1/Omega).
* alpha = 1 bohr^2 by default; the sum in x_div runs over the FFT box.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft

from . import hamiltonian, scf


def exx_div(lattice, fft, alpha: float = 1.0) -> float:
    omega = scf.cell_volume(lattice)
    g2 = scf.grid_g2(lattice, fft)
    nz = g2 > 1e-12
    return omega / (2.0 * math.pi) ** 3 * 2.0 * math.pi ** 1.5 / math.sqrt(alpha) - float(np.sum(np.exp(-alpha * g2[nz]) / g2[nz]))


def coulomb(n_r: np.ndarray, lattice, xdiv: float) -> np.ndarray:
    """Potential of a (complex) codensity on the grid: 4 pi n(G) / G^2, and 4 pi n(0) x_div at G = 0."""
    ng = scipy.fft.fftn(n_r) / n_r.size
    g2 = scf.grid_g2(lattice, n_r.shape)
    k = np.empty_like(g2)
    nz = g2 > 1e-12
    k[nz] = 4.0 * math.pi / g2[nz]
    k[~nz] = 4.0 * math.pi * xdiv
    return scipy.fft.ifftn(k * ng) * n_r.size


def apply_vx(psi: np.ndarray, occupied: np.ndarray, miller, fft, lattice, alpha: float = 1.0) -> np.ndarray:
    """V_x psi for the rows of psi [nb][npw], with the occupied orbitals [no][npw] (same convention)."""
    omega = scf.cell_volume(lattice)
    xdiv = exx_div(lattice, fft, alpha)
    pr = hamiltonian.to_real_space(np.asarray(psi, dtype=np.complex128), miller, fft)
    orr = hamiltonian.to_real_space(np.asarray(occupied, dtype=np.complex128), miller, fft)
    out = np.zeros_like(pr)
    for b in range(pr.shape[0]):
        for j in range(orr.shape[0]):
            v = coulomb(np.conj(orr[j]) * pr[b] / omega, lattice, xdiv)
            out[b] -= orr[j] * v
    return hamiltonian.to_reciprocal(out, miller, fft)


def exchange_energy(occupied: np.ndarray, miller, fft, lattice, alpha: float = 1.0) -> float:
    """E_x = sum_i <psi_i|V_x psi_i> over the occupied orbitals (closed shells)."""
    vx = apply_vx(occupied, occupied, miller, fft, lattice, alpha)
    return float(np.real(np.sum(np.conj(occupied) * vx)))
