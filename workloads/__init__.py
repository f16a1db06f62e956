"""Seeded synthetic inputs for the plane-wave H|psi> workloads.

This module draws and evaluates the *inputs* of the method and nothing else:
cells, atom positions, k-points, the synthetic local potential V(r) sampled on
the FFT grid, the synthetic separable projectors beta_p(k+G) evaluated at given
Miller indices, the projector matrix D and raw starting wavefunctions.  It holds
none of the method's arithmetic (no G-sphere selection, no FFT, no H|psi>, no
eigensolver): the Miller indices of the G-sphere are always passed in by the
caller, who takes them from the side under test.  Both the CPU oracle and the
CUDA path read their inputs from here, so they see the same arrays.

Physical setting (the paper's Sec. 3 and App. A.1-A.2): periodic cells, a plane-wave
basis |k+G> with |k+G|^2/2 <= E_cut (Hartree atomic units), a local potential
applied in real space and Kleinman-Bylander separable norm-conserving projectors.
The paper prints no workload of its own that fits this path, so these seeded cells
stand in for its systems; the recipe is:

* V(r) = sum_a sum_L -2 exp(-|r - R_a - L|^2 / 2)   (Gaussian wells, sigma = 1 bohr,
  periodic images L summed to convergence; terms beyond 12 bohr are < 6e-32).
* beta_{a,s}(q) = N exp(-0.32 q^2) e^{-i q.R_a},
  beta_{a,p_x}(q) = N q_x exp(-0.32 q^2) e^{-i q.R_a} (same for y, z), q = k + G,
  each normalised to unit 2-norm over the G-sphere of its k.
* D = diag(+1, -0.5, -0.5, -0.5) Ha per atom (block diagonal, Hermitian).
* psi0_b(G) = (x + i y)/sqrt(2) / (1 + |k+G|^2), x, y standard normal.

Seeds (numpy PCG64): atoms 1000 + config, psi0 2000 + config, k-points 3000,
multi-cell draw 4000.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi
V_DEPTH = -2.0          # Ha, depth of each Gaussian well
V_SIGMA2 = 1.0          # bohr^2, sigma^2 of each well
BETA_ALPHA = 0.32       # bohr^2, exp(-alpha q^2) radial factor (0.8^2 / 2)
D_DIAG = (1.0, -0.5, -0.5, -0.5)
IMAGE_CUTOFF = 12.0     # bohr


@dataclass
class Problem:
    """One independent H|psi> problem: a cell, its k-points and its inputs."""

    name: str
    lattice: np.ndarray            # [3,3] rows a1, a2, a3 (bohr)
    atoms: np.ndarray              # [nat,3] cartesian positions (bohr)
    ecut: float                    # Ha, |k+G|^2/2 <= ecut
    fft: tuple                     # (n1, n2, n3)
    kpts: np.ndarray               # [nk,3] cartesian (1/bohr)
    nbnd: int
    psi_seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nproj(self) -> int:
        return 4 * len(self.atoms)


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b1, b2, b3 with a_i . b_j = 2 pi delta_ij (used only to place inputs in q-space)."""
    return TWO_PI * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


# ---------------------------------------------------------------------------
# cells
# ---------------------------------------------------------------------------

def _cubic(a: float) -> np.ndarray:
    return np.diag([a, a, a]).astype(np.float64)


def _jittered_lattice(n: int, spacing: float, jitter: float, rng) -> np.ndarray:
    idx = np.array([(i, j, k) for i in range(n) for j in range(n) for k in range(n)], dtype=np.float64)
    return idx * spacing + rng.uniform(-jitter, jitter, size=idx.shape)


def smooth_235_at_least(n: int) -> int:
    """Smallest integer >= n whose only prime factors are 2, 3 and 5."""
    m = max(int(n), 1)
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def cubic_box(a: float, ecut: float) -> int:
    """FFT box edge for a cubic cell: smallest 2*3*5-smooth n >= 4 m_max + 1."""
    mmax = int(math.floor(math.sqrt(2.0 * ecut) * a / TWO_PI))
    return smooth_235_at_least(4 * mmax + 1)


def config1(nbnd: int = 16) -> Problem:
    """Simple cubic a = 10 bohr, 2 atoms at uniform fractional positions, Gamma, E_cut 10 Ha, box 32^3."""
    rng = np.random.default_rng(1001)
    lat = _cubic(10.0)
    atoms = rng.random((2, 3)) @ lat
    return Problem("sc10-2at", lat, atoms, 10.0, (32, 32, 32), np.zeros((1, 3)), nbnd, psi_seed=2001)


def config2(nbnd: int = 160) -> Problem:
    """Cubic a = 20.5 bohr, 64 atoms on a 4x4x4 lattice (spacing 5.125) +- 0.3 bohr jitter, E_cut 20 Ha, box 90^3."""
    rng = np.random.default_rng(1002)
    atoms = _jittered_lattice(4, 5.125, 0.3, rng)
    return Problem("sc20.5-64at", _cubic(20.5), atoms, 20.0, (90, 90, 90), np.zeros((1, 3)), nbnd, psi_seed=2002)


def config3(nbnd: int = 160) -> Problem:
    """The a = 10 bohr cell of config 1 with 160 (or 320) bands, for the mixed-precision form."""
    p = config1(nbnd)
    p.name = f"sc10-2at-{nbnd}b"
    p.psi_seed = 2003
    return p


def fold_to_bz(k: np.ndarray, recip: np.ndarray) -> np.ndarray:
    """Return k - G closest to the origin over the 5^3 nearest reciprocal-lattice vectors."""
    best = k.copy()
    rng = range(-2, 3)
    for i in rng:
        for j in rng:
            for l in rng:
                cand = k - (i * recip[0] + j * recip[1] + l * recip[2])
                if cand @ cand < best @ best - 1e-14:
                    best = cand
    return best


def config4a(nbnd: int = 24) -> Problem:
    """fcc a = 10.2 bohr, 2 atoms, E_cut 25 Ha, box 36^3, 16 seeded k-points folded into the first zone."""
    a = 10.2
    lat = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    rng = np.random.default_rng(1004)
    atoms = rng.random((2, 3)) @ lat
    recip = reciprocal(lat)
    krng = np.random.default_rng(3000)
    frac = krng.random((16, 3)) - 0.5
    kpts = np.array([fold_to_bz(f @ recip, recip) for f in frac])
    return Problem("fcc10.2-16k", lat, atoms, 25.0, (36, 36, 36), kpts, nbnd, psi_seed=2004)


def config4b() -> list:
    """32 independent cubic cells, a ~ U(8, 14) bohr, 1-4 atoms, 8-32 bands, E_cut 15 Ha, Gamma."""
    rng = np.random.default_rng(4000)
    cells = []
    for c in range(32):
        a = float(rng.uniform(8.0, 14.0))
        nat = int(rng.integers(1, 5))
        nb = int(rng.integers(8, 33))
        lat = _cubic(a)
        atoms = rng.random((nat, 3)) @ lat
        n = cubic_box(a, 15.0)
        cells.append(Problem(f"cell{c:02d}-a{a:.3f}", lat, atoms, 15.0, (n, n, n), np.zeros((1, 3)), nb,
                             psi_seed=20040 + c))
    return cells


def config5(nbnd: int = 512) -> Problem:
    """Cubic a = 30 bohr, 216 atoms on a 6x6x6 lattice (spacing 5) +- 0.3 bohr jitter, E_cut 25 Ha, box 144^3."""
    rng = np.random.default_rng(1005)
    atoms = _jittered_lattice(6, 5.0, 0.3, rng)
    return Problem("sc30-216at", _cubic(30.0), atoms, 25.0, (144, 144, 144), np.zeros((1, 3)), nbnd, psi_seed=2005)


def small_cell(ecut: float = 2.0, a: float = 10.0, nat: int = 2, fft=(16, 16, 16), nbnd: int = 8,
               seed: int = 7, k=(0.0, 0.0, 0.0), lattice=None) -> Problem:
    """A tiny cell for brute-force checks (dense matrices, direct DFTs)."""
    rng = np.random.default_rng(seed)
    lat = _cubic(a) if lattice is None else np.asarray(lattice, dtype=np.float64)
    atoms = rng.random((nat, 3)) @ lat
    return Problem(f"tiny-a{a}-e{ecut}", lat, atoms, ecut, tuple(fft), np.asarray([k], dtype=np.float64), nbnd,
                   psi_seed=seed + 100)


# ---------------------------------------------------------------------------
# inputs evaluated on the grid / at given Miller indices
# ---------------------------------------------------------------------------

def grid_points(lattice: np.ndarray, fft) -> np.ndarray:
    """Cartesian r_j = sum_i (j_i / n_i) a_i for the [n1][n2][n3] grid (C order), shape [N,3]."""
    n1, n2, n3 = fft
    f1 = np.arange(n1) / n1
    f2 = np.arange(n2) / n2
    f3 = np.arange(n3) / n3
    F = np.stack(np.meshgrid(f1, f2, f3, indexing="ij"), axis=-1).reshape(-1, 3)
    return F @ np.asarray(lattice, dtype=np.float64)


def _is_orthogonal_diag(lattice: np.ndarray) -> bool:
    lat = np.asarray(lattice)
    return bool(np.all(lat - np.diag(np.diag(lat)) == 0.0))


def vloc_r(lattice: np.ndarray, atoms: np.ndarray, fft, brute_force: bool = False) -> np.ndarray:
    """Synthetic local potential V(r_j) on the grid, float64 [n1][n2][n3] (C order), Ha.

    Periodic sum of -2 exp(-|r - R_a - L|^2/2) over atoms a and lattice vectors L, carried
    to convergence.  Orthorhombic cells use the exact factorisation of the Gaussian
    into per-axis image sums; other cells (and brute_force=True) sum images directly.
    """
    lat = np.asarray(lattice, dtype=np.float64)
    atoms = np.asarray(atoms, dtype=np.float64)
    n1, n2, n3 = fft
    if _is_orthogonal_diag(lat) and not brute_force:
        L = np.diag(lat)
        facs = []
        for ax, n in enumerate((n1, n2, n3)):
            x = np.arange(n) * (L[ax] / n)
            nimg = int(math.ceil(IMAGE_CUTOFF / L[ax])) + 2
            d = x[None, :, None] - atoms[:, ax][:, None, None] + L[ax] * np.arange(-nimg, nimg + 1)[None, None, :]
            facs.append(np.exp(-0.5 * d * d / V_SIGMA2).sum(axis=2))   # [nat, n]
        s12 = (facs[0][:, :, None] * facs[1][:, None, :]).reshape(len(atoms), n1 * n2)
        v = V_DEPTH * (s12.T @ facs[2])
        return np.ascontiguousarray(v.reshape(n1, n2, n3))
    r = grid_points(lat, fft)
    recip = reciprocal(lat)
    heights = TWO_PI / np.linalg.norm(recip, axis=1)      # spacing of lattice planes
    diam = np.linalg.norm(lat.sum(axis=0)) + np.linalg.norm(lat, axis=1).sum()
    nimg = [int(math.ceil((IMAGE_CUTOFF + diam) / h)) + 1 for h in heights]
    v = np.zeros(len(r))
    for Ra in atoms:
        for i in range(-nimg[0], nimg[0] + 1):
            for j in range(-nimg[1], nimg[1] + 1):
                for l in range(-nimg[2], nimg[2] + 1):
                    c = Ra + i * lat[0] + j * lat[1] + l * lat[2]
                    d = r - c
                    d2 = np.einsum("ij,ij->i", d, d)
                    m = d2 < (IMAGE_CUTOFF + 3.0) ** 2
                    if m.any():
                        v[m] += V_DEPTH * np.exp(-0.5 * d2[m] / V_SIGMA2)
    return v.reshape(n1, n2, n3)


def qvectors(lattice: np.ndarray, k: np.ndarray, miller: np.ndarray) -> np.ndarray:
    """Cartesian q = k + m1 b1 + m2 b2 + m3 b3 for the given Miller indices, [npw,3]."""
    return np.asarray(k, dtype=np.float64)[None, :] + np.asarray(miller, dtype=np.float64) @ reciprocal(lattice)


def beta(lattice: np.ndarray, atoms: np.ndarray, k: np.ndarray, miller: np.ndarray) -> np.ndarray:
    """Synthetic s + p projectors beta_p(k+G), complex128 [4 nat][npw], unit 2-norm per projector."""
    q = qvectors(lattice, k, miller)
    q2 = np.einsum("ij,ij->i", q, q)
    radial = np.exp(-BETA_ALPHA * q2)
    atoms = np.asarray(atoms, dtype=np.float64)
    out = np.empty((4 * len(atoms), len(q)), dtype=np.complex128)
    for a, Ra in enumerate(atoms):
        phase = np.exp(-1j * (q @ Ra))
        out[4 * a + 0] = radial * phase
        out[4 * a + 1] = q[:, 0] * radial * phase
        out[4 * a + 2] = q[:, 1] * radial * phase
        out[4 * a + 3] = q[:, 2] * radial * phase
    norms = np.sqrt(np.sum(np.abs(out) ** 2, axis=1))
    norms[norms == 0.0] = 1.0
    return out / norms[:, None]


def dmat(nat: int) -> np.ndarray:
    """D = diag(+1, -0.5, -0.5, -0.5) Ha per atom, complex128 [4 nat][4 nat]."""
    return np.diag(np.tile(np.asarray(D_DIAG, dtype=np.float64), nat)).astype(np.complex128)


def psi0(lattice: np.ndarray, k: np.ndarray, miller: np.ndarray, nbnd: int, seed: int) -> np.ndarray:
    """Raw starting wavefunctions, complex128 [nbnd][npw]: complex Gaussian damped by 1/(1+|k+G|^2)."""
    rng = np.random.default_rng(seed)
    q = qvectors(lattice, k, miller)
    damp = 1.0 / (1.0 + np.einsum("ij,ij->i", q, q))
    z = (rng.standard_normal((nbnd, len(q))) + 1j * rng.standard_normal((nbnd, len(q)))) / math.sqrt(2.0)
    return np.ascontiguousarray(z * damp[None, :])


def random_block(npw: int, nbnd: int, seed: int) -> np.ndarray:
    """Plain complex Gaussian block [nbnd][npw] (test vectors for H|psi> parity)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nbnd, npw)) + 1j * rng.standard_normal((nbnd, npw))) / math.sqrt(2.0)


def hermitian_matrix(n: int, seed: int, spectrum=None, scale: float = 1.0) -> np.ndarray:
    """Seeded dense Hermitian test matrix [n][n] (reduced-problem tests of the eigensolver).

    Without ``spectrum``: (B + B^H) / 2 for a complex Gaussian B, times ``scale``.  With it: U diag(spectrum) U^H
    for a Haar-like unitary U (QR of a complex Gaussian), so repeated values give exact degeneracies."""
    rng = np.random.default_rng(seed)
    b = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    if spectrum is None:
        return scale * (b + b.conj().T) / 2.0
    q, r = np.linalg.qr(b)
    q = q * (np.diag(r) / np.abs(np.diag(r)))[None, :]
    a = (q * np.asarray(spectrum, dtype=float)[None, :]) @ q.conj().T
    return (a + a.conj().T) / 2.0


CONFIGS = {
    "c1": config1,
    "c2": config2,
    "c3": config3,
    "c4a": config4a,
    "c5": config5,
}
