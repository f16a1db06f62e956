"""Plane-wave basis at one k-point (oracle; test infrastructure only).

The wavefunctions are expanded in plane waves |k+G> with kinetic energy below the cutoff,
|k+G|^2/2 <= E_cut in Hartree units (paper Sec. 3: PW basis with periodic boundary
conditions; App. A.2.1 writes the PWs as |k+G>).  The paper leaves the boundary and the
order open; the readings taken here:

* the cutoff test is inclusive and uses |k+G|^2 computed in float64;
* G = m1 b1 + m2 b2 + m3 b3 with b = 2 pi (A^{-1})^T, A's rows being a1, a2, a3;
* the basis is ordered lexicographically by the signed Miller indices (m1, m2, m3).
"""
from __future__ import annotations

import math

import numpy as np


def reciprocal(lattice) -> np.ndarray:
    """Rows b_j with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * math.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def miller_bounds(lattice, ecut: float, k) -> list:
    """Per axis, the integer range that can hold |k+G| <= sqrt(2 E_cut).

    m_i = (k+G).a_i / (2 pi) - k.a_i / (2 pi), so |m_i + k.a_i/(2 pi)| <= sqrt(2 E_cut) |a_i| / (2 pi).
    """
    lat = np.asarray(lattice, dtype=np.float64)
    qmax = math.sqrt(2.0 * ecut)
    out = []
    for i in range(3):
        kf = float(np.dot(k, lat[i])) / (2.0 * math.pi)
        r = qmax * float(np.linalg.norm(lat[i])) / (2.0 * math.pi)
        out.append((int(math.floor(-kf - r)) - 1, int(math.ceil(-kf + r)) + 1))
    return out


def gsphere(lattice, ecut: float, k) -> np.ndarray:
    """Miller indices of {G : |k+G|^2 / 2 <= E_cut}, int32 [npw, 3], lexicographic (m1, m2, m3)."""
    k = np.asarray(k, dtype=np.float64)
    b = reciprocal(lattice)
    (l1, h1), (l2, h2), (l3, h3) = miller_bounds(lattice, ecut, k)
    m1, m2, m3 = np.meshgrid(np.arange(l1, h1 + 1), np.arange(l2, h2 + 1), np.arange(l3, h3 + 1), indexing="ij")
    m = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)      # already lexicographic
    q = k[None, :] + m[:, 0:1] * b[0][None, :] + m[:, 1:2] * b[1][None, :] + m[:, 2:3] * b[2][None, :]
    q2 = q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1] + q[:, 2] * q[:, 2]
    keep = 0.5 * q2 <= ecut
    return np.ascontiguousarray(m[keep].astype(np.int32))


def kplusg(lattice, k, miller) -> np.ndarray:
    """Cartesian k + G for each Miller triple, [npw, 3]."""
    b = reciprocal(lattice)
    m = np.asarray(miller, dtype=np.float64)
    return np.asarray(k, dtype=np.float64)[None, :] + m @ b


def kinetic(lattice, k, miller) -> np.ndarray:
    """T_G = |k+G|^2 / 2 (Ha), the diagonal kinetic term in the PW basis (App. A.2.1)."""
    q = kplusg(lattice, k, miller)
    return 0.5 * np.sum(q * q, axis=1)


def cutoff_margin(lattice, ecut: float, k, miller=None) -> float:
    """Smallest | |k+G|^2/2 - E_cut | over the bounding box (how far the nearest G is from a tie)."""
    k = np.asarray(k, dtype=np.float64)
    (l1, h1), (l2, h2), (l3, h3) = miller_bounds(lattice, ecut, k)
    m1, m2, m3 = np.meshgrid(np.arange(l1, h1 + 1), np.arange(l2, h2 + 1), np.arange(l3, h3 + 1), indexing="ij")
    m = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)
    q = kplusg(lattice, k, m)
    return float(np.min(np.abs(0.5 * np.sum(q * q, axis=1) - ecut)))


def min_box(miller) -> tuple:
    """Smallest FFT box into which the sphere maps one-to-one: n_i >= 2 max|m_i| + 1."""
    mm = np.max(np.abs(np.asarray(miller)), axis=0)
    return tuple(int(2 * x + 1) for x in mm)
