"""Reference eigenvalues of H (oracle; test infrastructure only).

Eq. (diag) of App. A.2 with S = I: the lowest N eigenpairs of the Hermitian operator H.
Two independent routes:

* ``lowest_dense``: build H_GG' element by element (``hamiltonian.dense_h``) and call LAPACK
  (numpy.linalg.eigvalsh) -- the plain definition, for cells with a few thousand PWs;
* ``lowest_lobpcg``: scipy's LOBPCG on the FFT form of H|psi>, for cells whose dense matrix
  does not fit; a different algorithm from the block Davidson under test.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as sla

from . import hamiltonian


def lowest_dense(h: np.ndarray, nbnd: int) -> np.ndarray:
    """Lowest nbnd eigenvalues of a dense Hermitian matrix, ascending."""
    return np.linalg.eigvalsh(h)[:nbnd]


def lowest_lobpcg(lattice, k, miller, fft, vr, beta, dmat, nbnd: int, x0: np.ndarray,
                  tol: float = 1e-9, maxiter: int = 400, nguard: int = 8, verbose: bool = False,
                  chunk: int = 0):
    """Lowest nbnd eigenvalues by LOBPCG on the FFT H|psi>, with a guard block of extra vectors.

    ``chunk`` > 0 applies H to at most that many vectors at a time (the bands are independent, so
    this only bounds the memory of the full-box transforms).
    Returns (eigenvalues, residual norms of the returned vectors).
    """
    npw = len(miller)
    hdiag = hamiltonian.h_diagonal(lattice, k, miller, vr, beta, dmat)

    def matmat(x):
        x = np.asarray(x)
        step = chunk if chunk > 0 else max(1, x.shape[1])
        out = np.empty(x.shape, dtype=np.complex128)
        for j in range(0, x.shape[1], step):
            out[:, j:j + step] = hamiltonian.hpsi(lattice, k, miller, fft, vr, beta, dmat, x[:, j:j + step].T).T
        return out

    op = sla.LinearOperator((npw, npw), matmat=matmat, matvec=lambda v: matmat(v[:, None])[:, 0],
                            dtype=np.complex128)
    shift = float(np.min(hdiag)) - 1.0

    def prec(x):
        x = np.asarray(x)
        d = hdiag - shift
        return x / (d[:, None] if x.ndim == 2 else d)

    m = sla.LinearOperator((npw, npw), matmat=prec, matvec=prec, dtype=np.complex128)
    nb = nbnd + nguard
    x = np.asarray(x0[:nb], dtype=np.complex128).T
    w, v = sla.lobpcg(op, x, M=m, largest=False, tol=tol, maxiter=maxiter, verbosityLevel=1 if verbose else 0)
    order = np.argsort(w)
    w, v = w[order][:nbnd], v[:, order][:, :nbnd]
    hv = matmat(v)
    res = np.linalg.norm(hv - v * w[None, :], axis=0)
    return w, res
