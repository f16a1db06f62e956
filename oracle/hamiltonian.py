"""H|psi> in the plane-wave basis (oracle; test infrastructure only).

The operator is the Kohn-Sham Hamiltonian at fixed potential of App. A.1 -- kinetic term
plus a local potential V(r) applied in real space -- plus the separable (Kleinman-Bylander)
norm-conserving nonlocal term of Sec. 3, sum_pq |beta_p> D_pq <beta_q|.  App. A.2 asks only
that H be available as an operator (H|psi> for any |psi>), with S = I for norm-conserving
projectors.

Readings of what the paper leaves open (Hartree units, bohr):

* r_j = sum_i (j_i / n_i) a_i on the n1 x n2 x n3 grid, V given as V[j1][j2][j3];
* psi(r_j) = sum_G psi(G) e^{+i G.r_j} (no normalisation), and
  (V psi)(G) = N_r^{-1} sum_j e^{-i G.r_j} V(r_j) psi(r_j), keeping G in the sphere only,
  so that <psi|psi> = sum_G |psi(G)|^2 (the 1/sqrt(Omega) of the plane waves is absorbed);
* the Bloch factor e^{ik.r} cancels between the two transforms: k enters only T and beta.

Equivalently, with V~(q) = N_r^{-1} sum_j V(r_j) e^{-i q.r_j},
    H_GG' = |k+G|^2/2 delta_GG' + V~(G - G') + sum_pq beta_p(G) D_pq conj(beta_q(G')).
``hpsi`` evaluates the first form with full-box FFTs; ``dense_h`` builds the second element
by element with a direct (non-FFT) DFT.  Both are exact for any box into which the sphere
maps one-to-one; they differ only in rounding order.
"""
from __future__ import annotations

import math
import os

import numpy as np
import scipy.fft

from .gsphere import kinetic, min_box


def _workers() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def check_box(miller, fft) -> None:
    need = min_box(miller)
    if any(int(n) < m for n, m in zip(fft, need)):
        raise ValueError(f"FFT box {tuple(fft)} too small for the sphere: need >= {need}")


def box_index(miller, fft) -> tuple:
    """Box position of each G: (m_i mod n_i)."""
    m = np.asarray(miller)
    return (np.mod(m[:, 0], fft[0]), np.mod(m[:, 1], fft[1]), np.mod(m[:, 2], fft[2]))


def to_real_space(psi_g: np.ndarray, miller, fft) -> np.ndarray:
    """psi(r_j) = sum_G psi(G) e^{+i G.r_j} for a block [nb][npw] -> [nb][n1][n2][n3]."""
    idx = box_index(miller, fft)
    nb = psi_g.shape[0]
    box = np.zeros((nb,) + tuple(fft), dtype=np.complex128)
    box[(slice(None),) + idx] = psi_g
    # scipy's inverse transform with norm="forward" is the unnormalised sum with e^{+i}
    return scipy.fft.ifftn(box, axes=(1, 2, 3), norm="forward", workers=_workers())


def to_reciprocal(phi_r: np.ndarray, miller, fft) -> np.ndarray:
    """(phi)(G) = N_r^{-1} sum_j e^{-i G.r_j} phi(r_j), for G in the sphere, [nb][npw]."""
    idx = box_index(miller, fft)
    # scipy's forward transform with norm="forward" carries the 1/N_r and e^{-i}
    full = scipy.fft.fftn(phi_r, axes=(1, 2, 3), norm="forward", workers=_workers())
    return full[(slice(None),) + idx]


def local_term(vr: np.ndarray, miller, fft, psi: np.ndarray) -> np.ndarray:
    """[V psi](G): to real space, multiply by V(r_j), back to the sphere."""
    check_box(miller, fft)
    return to_reciprocal(to_real_space(psi, miller, fft) * np.asarray(vr)[None], miller, fft)


def calbec(beta: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """<beta_p|psi_b> = sum_G conj(beta_p(G)) psi_b(G), [P][nb]."""
    return np.conj(beta) @ psi.T


def nonlocal_term(beta: np.ndarray, dmat: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """sum_pq beta_p(G) D_pq <beta_q|psi_b>, [nb][npw]."""
    if beta.shape[0] == 0:
        return np.zeros_like(psi)
    w = dmat @ calbec(beta, psi)          # [P][nb]
    return w.T @ beta


def hpsi(lattice, k, miller, fft, vr, beta, dmat, psi) -> np.ndarray:
    """H|psi> for a block of bands psi [nb][npw] (FFT form)."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    t = kinetic(lattice, k, miller)
    out = t[None, :] * psi
    out = out + local_term(vr, miller, fft, psi)
    out = out + nonlocal_term(np.asarray(beta, dtype=np.complex128), np.asarray(dmat, dtype=np.complex128), psi)
    return out


def vtilde_direct(vr: np.ndarray, q) -> np.ndarray:
    """V~(q) = N_r^{-1} sum_j V(r_j) e^{-2 pi i sum_i q_i j_i / n_i} by direct summation.

    ``q`` is an integer array [nq, 3].  The sum over j is carried out axis by axis with
    explicit DFT matrices E_i[q, j] = exp(-2 pi i q j / n_i) (no FFT), on the distinct
    components of q.
    """
    v = np.asarray(vr, dtype=np.float64)
    n1, n2, n3 = v.shape
    q = np.asarray(q, dtype=np.int64)
    u1, i1 = np.unique(q[:, 0], return_inverse=True)
    u2, i2 = np.unique(q[:, 1], return_inverse=True)
    u3, i3 = np.unique(q[:, 2], return_inverse=True)

    def dft_matrix(u, n):
        return np.exp(-2j * math.pi * np.outer(u, np.arange(n)) / n)

    e1, e2, e3 = dft_matrix(u1, n1), dft_matrix(u2, n2), dft_matrix(u3, n3)
    t = np.einsum("aj,jkl->akl", e1, v)
    t = np.einsum("bk,akl->abl", e2, t)
    t = np.einsum("cl,abl->abc", e3, t)
    return t[i1, i2, i3] / (n1 * n2 * n3)


def dense_local(vr: np.ndarray, miller) -> np.ndarray:
    """Matrix V~(G - G') over the sphere, [npw][npw]."""
    m = np.asarray(miller, dtype=np.int64)
    lo = m.min(axis=0) - m.max(axis=0)
    hi = m.max(axis=0) - m.min(axis=0)
    g1, g2, g3 = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                             np.arange(lo[2], hi[2] + 1), indexing="ij")
    qs = np.stack([g1.ravel(), g2.ravel(), g3.ravel()], axis=1)
    table = vtilde_direct(vr, qs).reshape(g1.shape)
    d = m[:, None, :] - m[None, :, :]
    return table[d[..., 0] - lo[0], d[..., 1] - lo[1], d[..., 2] - lo[2]]


def dense_h(lattice, k, miller, fft, vr, beta, dmat) -> np.ndarray:
    """H_GG' = T_G delta_GG' + V~(G - G') + sum_pq beta_p(G) D_pq conj(beta_q(G')), [npw][npw]."""
    check_box(miller, fft)
    h = dense_local(vr, miller).astype(np.complex128)
    h[np.diag_indices_from(h)] += kinetic(lattice, k, miller)
    beta = np.asarray(beta, dtype=np.complex128)
    if beta.shape[0]:
        h += beta.T @ np.asarray(dmat, dtype=np.complex128) @ np.conj(beta)
    return h


def h_diagonal(lattice, k, miller, vr, beta, dmat) -> np.ndarray:
    """<k+G|H|k+G> = T_G + V~(0) + sum_pq beta_p(G) D_pq conj(beta_q(G)) (real), [npw]."""
    t = kinetic(lattice, k, miller)
    vbar = float(np.mean(np.asarray(vr, dtype=np.float64)))
    beta = np.asarray(beta, dtype=np.complex128)
    nl = np.zeros_like(t)
    if beta.shape[0]:
        # sum_p beta_p(G) [D conj(beta)]_p(G)
        nl = np.real(np.sum(beta * (np.asarray(dmat, dtype=np.complex128) @ np.conj(beta)), axis=0))
    return t + vbar + nl
