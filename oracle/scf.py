"""Self-consistent field loop around H|psi> (oracle; test infrastructure only).

App. A.1 (self-consistency): the KS problem is a fixed point x = F[x] of the charge density; the
input density gives V_Hxc = V_H + V_xc, the lowest KS orbitals of H = T + V_ext + V_Hxc + V_NL give
the output density rho_out = sum_i f_i |psi_i|^2, and the input of the next iteration is chosen
from the previous few (x_in, x_out) pairs: the linear combination of past inputs that minimises the
scf norm of the residual x_out - x_in, plus a fraction of that optimal residual (simple mixing).
The scf norm is the Hartree energy of the density difference, computed in reciprocal space:
  ||d rho||^2 = (4 pi e^2 / Omega) sum_{G != 0} |d rho(G)|^2 / G^2.
The paper gives two variational energies that agree at self-consistency: the standard one on
rho_out and the Harris-Weinert-Foulkes one on rho_in (both below, without the ion-ion term).

Conventions (as in ``hamiltonian``): psi(r_j) = sum_G psi(G) e^{i(k+G).r_j} with sum_G |psi(G)|^2 = 1,
so the physical orbital is psi(r) / Omega^(1/2); densities are sampled on the FFT grid r_j, and a
density's Fourier components are rho(G) = (1/N_r) sum_j rho(r_j) e^{-iG.r_j}.

Readings (where the paper is silent or defers to its references):
* rho(G) in the scf norm is taken as Omega rho(G) of the convention above (the integral over the
  cell), so that ||d rho||^2 = 4 pi Omega sum_{G != 0} |d rho(G)|^2 / G^2 = 2 E_H[d rho]; the paper's
  first-order estimate E - E' ~ E_H[d rho] is then ||d rho||^2 / 2.
* The G = 0 component of the Hartree potential is zero (a uniform neutralising background), as
  it is for the local potential, which carries no G = 0 divergence here.
* LDA: Slater exchange and the Perdew-Zunger (1981) parametrisation of the Ceperley-Alder
  correlation energy of the unpolarised electron gas; V_xc = d(rho eps_xc)/d rho.
* Occupations: the lowest nocc bands, each holding two electrons (an insulator, as in the paper's
  energy estimate); the synthetic cells carry two electrons per atom.
* Mixing: the paper's description (the combination of the last nmix inputs that minimises the scf
  norm of the combined residual, then a step beta times the optimal residual), i.e. Anderson's form
  of the modified Broyden update; nmix = 8, beta = 0.5.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft

from . import gsphere, hamiltonian

# Perdew-Zunger (1981) fit to Ceperley-Alder, unpolarised gas, Hartree units
_PZ_GAMMA, _PZ_BETA1, _PZ_BETA2 = -0.1423, 1.0529, 0.3334
_PZ_A, _PZ_B, _PZ_C, _PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def cell_volume(lattice) -> float:
    return float(abs(np.linalg.det(np.asarray(lattice, dtype=np.float64))))


def grid_g2(lattice, fft) -> np.ndarray:
    """|G|^2 on the full FFT box, in numpy's FFT frequency order (signed Miller indices)."""
    b = gsphere.reciprocal(lattice)
    m = [np.fft.fftfreq(n, d=1.0 / n) for n in fft]
    m1, m2, m3 = np.meshgrid(*m, indexing="ij")
    g = m1[..., None] * b[0] + m2[..., None] * b[1] + m3[..., None] * b[2]
    return np.sum(g * g, axis=-1)


def density(psi: np.ndarray, occ: np.ndarray, miller, fft, lattice) -> np.ndarray:
    """rho(r_j) = sum_i f_i |psi_i(r_j)|^2 / Omega on the grid [n1][n2][n3] (real)."""
    phi = hamiltonian.to_real_space(np.asarray(psi, dtype=np.complex128), miller, fft)
    rho = np.tensordot(np.asarray(occ, dtype=np.float64), np.abs(phi) ** 2, axes=(0, 0))
    return rho / cell_volume(lattice)


def charge(rho: np.ndarray, lattice) -> float:
    """The integral of rho over the cell (Omega / N_r sum_j rho(r_j))."""
    return float(cell_volume(lattice) * np.mean(rho))


def hartree(rho: np.ndarray, lattice) -> tuple:
    """(V_H(r_j), E_H): V_H(G) = 4 pi rho(G) / G^2 for G != 0, 0 at G = 0; E_H = Omega / 2 sum
    4 pi |rho(G)|^2 / G^2."""
    fft = rho.shape
    rg = scipy.fft.fftn(rho) / rho.size
    g2 = grid_g2(lattice, fft)
    inv = np.zeros_like(g2)
    nz = g2 > 1e-12
    inv[nz] = 4.0 * math.pi / g2[nz]
    vh = np.real(scipy.fft.ifftn(inv * rg) * rho.size)
    eh = 0.5 * cell_volume(lattice) * float(np.sum(inv * np.abs(rg) ** 2))
    return vh, eh


def scf_norm2(drho: np.ndarray, lattice) -> float:
    """||d rho||^2 = 4 pi Omega sum_{G != 0} |d rho(G)|^2 / G^2 (= 2 E_H[d rho])."""
    return 2.0 * hartree(drho, lattice)[1]


def lda_xc(rho: np.ndarray) -> tuple:
    """(eps_xc, V_xc) per point: Slater exchange + Perdew-Zunger correlation; zero where rho <= 0."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    pos = rho > 1e-30
    r = rho[pos]
    rs = (3.0 / (4.0 * math.pi * r)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 * r / math.pi) ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    ec = np.empty_like(r)
    vc = np.empty_like(r)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + _PZ_BETA1 * s + _PZ_BETA2 * rs[hi]
    ec[hi] = _PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * _PZ_BETA1 * s + 4.0 / 3.0 * _PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    x = rs[lo]
    lx = np.log(x)
    ec[lo] = _PZ_A * lx + _PZ_B + _PZ_C * x * lx + _PZ_D * x
    vc[lo] = _PZ_A * lx + (_PZ_B - _PZ_A / 3.0) + 2.0 / 3.0 * _PZ_C * x * lx + (2.0 * _PZ_D - _PZ_C) / 3.0 * x
    eps[pos] = ex + ec
    v[pos] = vx + vc
    return eps, v


def hxc(rho: np.ndarray, lattice) -> tuple:
    """(V_Hxc(r_j), E_Hxc) of a density."""
    vh, eh = hartree(rho, lattice)
    exc, vxc = lda_xc(rho)
    e_xc = cell_volume(lattice) * float(np.mean(rho * exc))
    return vh + vxc, eh + e_xc


class AndersonMixer:
    """The paper's mixing: the combination of the last nmix inputs (coefficients summing to one)
    whose combined residual has the smallest scf norm, then a step beta along that residual.

    The constrained minimum is solved in the equivalent difference form, a least-squares problem on
    the residual differences r_{k+1} - r_k weighted by the scf-norm metric (no normal equations)."""

    def __init__(self, lattice, nmix: int = 8, beta: float = 0.5):
        self.lattice, self.nmix, self.beta = lattice, nmix, beta
        self.xin, self.res = [], []

    def _weighted(self, a: np.ndarray) -> np.ndarray:
        """Real vector whose dot products are the scf-norm inner products: (4 pi Omega)^(1/2) a(G)/|G|
        over G != 0, real and imaginary parts."""
        fa = scipy.fft.fftn(a) / a.size
        g2 = grid_g2(self.lattice, a.shape)
        nz = g2 > 1e-12
        w = fa[nz] * np.sqrt(4.0 * math.pi * cell_volume(self.lattice) / g2[nz])
        return np.concatenate([w.real, w.imag])

    def step(self, xin: np.ndarray, xout: np.ndarray) -> np.ndarray:
        self.xin.append(np.array(xin))
        self.res.append(np.array(xout) - np.array(xin))
        self.xin, self.res = self.xin[-self.nmix:], self.res[-self.nmix:]
        x, r = self.xin[-1], self.res[-1]
        if len(self.res) > 1:
            # sum_k c_k r_k with sum c_k = 1  <=>  r_n - sum_k g_k (r_{k+1} - r_k) over the history
            dr = np.stack([self._weighted(self.res[j + 1] - self.res[j]) for j in range(len(self.res) - 1)], axis=1)
            g = np.linalg.lstsq(dr, self._weighted(r), rcond=None)[0]
            for j, gj in enumerate(g):
                x = x - gj * (self.xin[j + 1] - self.xin[j])
                r = r - gj * (self.res[j + 1] - self.res[j])
        return x + self.beta * r


def energies(eig: np.ndarray, occ: np.ndarray, rho_in: np.ndarray, rho_out: np.ndarray, lattice) -> tuple:
    """(E, E'): the standard energy on rho_out and the Harris-Weinert-Foulkes one on rho_in, both
    from the band energies of H[rho_in] (no ion-ion term).  sum_i f_i <psi_i|T + V_ext + V_NL|psi_i>
    = sum_i f_i eps_i - int rho_out V_Hxc[rho_in]."""
    omega = cell_volume(lattice)
    v_in, ehxc_in = hxc(rho_in, lattice)
    band = float(np.dot(occ, eig))
    _, ehxc_out = hxc(rho_out, lattice)
    e_std = band - omega * float(np.mean(rho_out * v_in)) + ehxc_out
    e_hwf = band - omega * float(np.mean(rho_in * v_in)) + ehxc_in
    return e_std, e_hwf


def scf(lattice, k, miller, fft, vext: np.ndarray, beta, dmat, nocc: int, rho0: np.ndarray, tol: float = 1e-10,
        maxiter: int = 60, nmix: int = 8, mix_beta: float = 0.5) -> dict:
    """The SCF loop on a small cell with the dense H (exact eigenpairs at each step).  Returns the
    converged input density, eigenvalues, the two energies and the history of squared scf norms."""
    occ = np.full(nocc, 2.0)
    mixer = AndersonMixer(lattice, nmix, mix_beta)
    rho_in = np.array(rho0, dtype=np.float64)
    history = []
    for it in range(maxiter):
        v_hxc, _ = hxc(rho_in, lattice)
        h = hamiltonian.dense_h(lattice, k, miller, fft, vext + v_hxc, beta, dmat)
        w, v = np.linalg.eigh(h)
        psi = v[:, :nocc].T
        rho_out = density(psi, occ, miller, fft, lattice)
        n2 = scf_norm2(rho_out - rho_in, lattice)
        history.append(n2)
        if n2 < tol:
            e, e2 = energies(w[:nocc], occ, rho_in, rho_out, lattice)
            return {"rho": rho_in, "rho_out": rho_out, "eig": w[:nocc], "e": e, "e_hwf": e2, "norm2": history,
                    "iters": it + 1, "psi": psi}
        rho_in = mixer.step(rho_in, rho_out)
    raise RuntimeError(f"scf: no convergence in {maxiter} iterations (last ||d rho||^2 = {history[-1]:.3e})")
