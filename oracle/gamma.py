"""Gamma-point real-wavefunction form (oracle; test infrastructure only).

Sec. 4 (PWscf): when only k = 0 is used the Kohn-Sham orbitals can be taken real, so only half of
their Fourier components need to be stored.  A real function has psi(-G) = psi(G)*; with the half
sphere S+ = {0} and one G of every pair {G, -G}, psi is fixed by its components on S+ (psi(0) real).

This module gives
* the half sphere and the index of -G for every G of the full sphere;
* the maps between full and half storage, and the inner product in half storage,
  <a|b> = a(0)* b(0) + 2 Re sum_{G in S+, G != 0} a(G)* b(G);
* an orthonormal real basis of the real-in-r functions (cos and sin combinations of +-G), in which
  H at Gamma is a real symmetric matrix of the same order npw;
* the packing of two real orbitals into one complex FFT: phi = psi_a + i psi_b in real space; after
  the forward transform c(G) of (V phi), (V psi_a)(G) = (c(G) + c(-G)*) / 2 and
  (V psi_b)(G) = (c(G) - c(-G)*) / (2i), so one pair of FFTs serves two bands.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian


def partner_index(miller) -> np.ndarray:
    """idx[i] = the position of -G_i in the same Miller list (the sphere at k = 0 is symmetric)."""
    m = np.asarray(miller, dtype=np.int64)
    pos = {tuple(r): i for i, r in enumerate(m.tolist())}
    return np.array([pos[(-a, -b, -c)] for a, b, c in m.tolist()], dtype=np.int64)


def half_sphere(miller) -> np.ndarray:
    """Positions of S+: G = 0, and of every pair the member with the first nonzero Miller index > 0."""
    m = np.asarray(miller, dtype=np.int64)
    keep = []
    for i, (a, b, c) in enumerate(m.tolist()):
        first = a if a != 0 else (b if b != 0 else c)
        if first >= 0:
            keep.append(i)
    return np.array(keep, dtype=np.int64)


def to_half(psi: np.ndarray, miller) -> np.ndarray:
    return np.asarray(psi)[..., half_sphere(miller)]


def to_full(psi_half: np.ndarray, miller) -> np.ndarray:
    """Full coefficients of the real function whose half-sphere components are psi_half."""
    h = half_sphere(miller)
    par = partner_index(miller)
    ph = np.asarray(psi_half, dtype=np.complex128)
    out = np.zeros(ph.shape[:-1] + (len(par),), dtype=np.complex128)
    out[..., h] = ph
    out[..., par[h]] = np.conj(ph)
    return out


def half_dot(a_half: np.ndarray, b_half: np.ndarray, miller) -> float:
    """<a|b> of two real functions from their half-sphere components."""
    h = half_sphere(miller)
    zero = [j for j, i in enumerate(h) if not np.any(np.asarray(miller)[i])]
    w = np.full(len(h), 2.0)
    w[zero] = 1.0
    return float(np.real(np.sum(w * np.conj(a_half) * b_half)))


def real_basis(miller) -> np.ndarray:
    """U [npw][npw] complex: column j is a real-in-r function with unit norm; the columns are
    orthonormal.  G = 0 gives e_0; each pair (G, -G) gives (e_G + e_-G)/sqrt2 and
    (e_G - e_-G)/(i sqrt2)."""
    h = half_sphere(miller)
    par = partner_index(miller)
    n = len(par)
    u = np.zeros((n, n), dtype=np.complex128)
    col = 0
    for i in h:
        if par[i] == i:
            u[i, col] = 1.0
            col += 1
        else:
            u[i, col] = u[par[i], col] = 1.0 / np.sqrt(2.0)
            u[i, col + 1] = -1j / np.sqrt(2.0)
            u[par[i], col + 1] = 1j / np.sqrt(2.0)
            col += 2
    assert col == n
    return u


def real_h(h_full: np.ndarray, miller) -> np.ndarray:
    """U^H H U: H in the real basis (real symmetric at Gamma)."""
    u = real_basis(miller)
    return u.conj().T @ h_full @ u


def local_pair(vr: np.ndarray, miller, fft, psi_a: np.ndarray, psi_b: np.ndarray) -> tuple:
    """(V psi_a, V psi_b) for two real orbitals with one transform pair: psi_a + i psi_b to real
    space, times V, back to G, then the two results from c(G) and c(-G)*."""
    par = partner_index(miller)
    phi = hamiltonian.to_real_space(np.stack([psi_a + 1j * psi_b]), miller, fft)
    c = hamiltonian.to_reciprocal(phi * vr[None], miller, fft)[0]
    cm = np.conj(c[par])
    return 0.5 * (c + cm), (c - cm) / 2j
