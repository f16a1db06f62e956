"""Band-by-band preconditioned conjugate-gradient eigensolver (oracle; test infrastructure only).

App. A.2.2 recasts the eigenproblem as a sequence of constrained minimisations, one band at a time:
band i minimises <psi|H|psi> over unit vectors orthogonal to the bands j < i already found.  With a
diagonal preconditioner P and y = P^-1 psi the minimisation runs on H~ = P H P, S~ = P S P.  Each
step
  * takes the gradient g = (H~ - lambda S~) y with the multiplier lambda chosen so that g is
    S~-orthogonal to y: lambda = <y|S~ H~|y> / <y|S~^2|y>;
  * removes from P g its components along the lower bands (explicit Gram-Schmidt);
  * forms the conjugate direction h = g + gamma h_prev (Polak-Ribiere:
    gamma = <g - g_prev|S~|g> / <g_prev|S~|g_prev>), re-orthogonalises it to y, normalises it to
    n = h / <h|S~|h>^(1/2);
  * moves along y cos(theta) + n sin(theta), which keeps the norm, with the exact minimum of
    <y|H~|y> on that curve: theta = atan(a / (eps - b)) / 2, a = 2 Re<y|H~|n>, b = <n|H~|n>,
    eps = <y|H~|y>.
Only P g, P h and P^2 enter; P^2 is kinetic-only, <k+G|P^2|k+G> = 2m / (hbar^2 |k+G|^2).

Everything below works on psi = P y directly (S = I for norm-conserving projectors):
  H~ y = P H psi,  S~ y = P psi,  so  P g = P^2 (H psi - lambda psi),
  lambda = <psi|P^2 H|psi> / <psi|P^2|psi>,  <a|S~|b> = <P a|P b>,
  and the move is psi <- psi cos(theta) + (P n) sin(theta) with P n = P h / ||P h||.

Readings (where the paper is silent):
* P^2 = 1 / max(|k+G|^2 / 2, t_min) in Hartree units (2m / hbar^2 = 2): the kinetic form is
  undefined at k + G = 0, so the kinetic energy is floored at t_min (1 Ha by default).
* The gradients in the Polak-Ribiere ratio are the ones after the Gram-Schmidt step.
* Of the two stationary angles theta_0 and theta_0 + pi/2 the one with the lower energy is taken.
* A band stops when ||H psi - eps psi||_2 <= tol (eps = <psi|H|psi>), the test the Davidson solver
  uses, or after maxiter steps.
* The initial vector of band i is the given guess, orthogonalised to the finished bands j < i
  (two Gram-Schmidt passes) and normalised.  The bands are returned in the order found; no
  subspace rotation follows the sweep (the paper describes none).
"""
from __future__ import annotations

import numpy as np


def precond_p2(kinetic: np.ndarray, t_min: float = 1.0) -> np.ndarray:
    """Diagonal of P^2: 1 / max(|k+G|^2/2, t_min)."""
    return 1.0 / np.maximum(np.asarray(kinetic, dtype=np.float64), t_min)


def _orth(v: np.ndarray, lower: np.ndarray) -> np.ndarray:
    """v minus its components along the orthonormal rows of lower (two passes)."""
    if lower.shape[0] == 0:
        return v
    for _ in range(2):
        v = v - lower.T @ (np.conj(lower) @ v)
    return v


def gradient(psi: np.ndarray, hpsi: np.ndarray, p2: np.ndarray) -> tuple:
    """(lambda, P g) of the current vector: lambda = <psi|P^2 H|psi> / <psi|P^2|psi> and
    P g = P^2 (H psi - lambda psi), which that lambda makes orthogonal to psi."""
    lam = float(np.real(np.vdot(psi, p2 * hpsi)) / np.real(np.vdot(psi, p2 * psi)))
    return lam, p2 * (hpsi - lam * psi)


def line_angle(eps: float, a: float, b: float) -> float:
    """The angle of the minimum of E(t) = eps cos^2 t + b sin^2 t + a sin t cos t."""
    x = a / (eps - b) if eps != b else np.copysign(np.inf, a)
    t0 = 0.5 * np.arctan(x)
    e = lambda t: eps * np.cos(t) ** 2 + b * np.sin(t) ** 2 + a * np.sin(t) * np.cos(t)
    t1 = t0 + 0.5 * np.pi
    return t1 if e(t1) < e(t0) else t0


def cg_band(apply_h, psi0: np.ndarray, lower: np.ndarray, p2: np.ndarray, tol: float, maxiter: int) -> tuple:
    """One band: returns (psi, H psi, eps, residual norm, steps, eps after each step)."""
    psi = _orth(np.asarray(psi0, dtype=np.complex128), lower)
    psi = psi / np.linalg.norm(psi)
    hpsi = apply_h(psi)
    pg_prev = ph_prev = None
    gg_prev = 0.0
    history = []
    steps = 0
    while True:
        eps = float(np.real(np.vdot(psi, hpsi)))
        res = float(np.linalg.norm(hpsi - eps * psi))
        history.append(eps)
        if res <= tol or steps >= maxiter:
            return psi, hpsi, eps, res, steps, history
        _, pg = gradient(psi, hpsi, p2)
        pg = _orth(pg, lower)
        gg = float(np.real(np.vdot(pg, pg)))
        gamma = 0.0 if pg_prev is None else (gg - float(np.real(np.vdot(pg_prev, pg)))) / gg_prev
        ph = pg if ph_prev is None else pg + gamma * ph_prev
        ph = ph - psi * np.vdot(psi, ph)
        pn = ph / np.linalg.norm(ph)
        hpn = apply_h(pn)
        a = 2.0 * float(np.real(np.vdot(psi, hpn)))
        b = float(np.real(np.vdot(pn, hpn)))
        t = line_angle(eps, a, b)
        psi = np.cos(t) * psi + np.sin(t) * pn
        hpsi = np.cos(t) * hpsi + np.sin(t) * hpn
        pg_prev, gg_prev, ph_prev = pg, gg, ph
        steps += 1


def cg_solve(apply_h, x0: np.ndarray, kinetic: np.ndarray, tol: float, maxiter: int, t_min: float = 1.0) -> tuple:
    """All bands of x0 [nb][npw] in turn: returns (eigenvalues, psi [nb][npw], residual norms,
    steps per band)."""
    x0 = np.asarray(x0, dtype=np.complex128)
    nb, npw = x0.shape
    p2 = precond_p2(kinetic, t_min)
    psi = np.zeros((nb, npw), dtype=np.complex128)
    eig = np.zeros(nb)
    res = np.zeros(nb)
    steps = np.zeros(nb, dtype=np.int64)
    for i in range(nb):
        psi[i], _, eig[i], res[i], steps[i], _ = cg_band(apply_h, x0[i], psi[:i], p2, tol, maxiter)
    return eig, psi, res, steps
