"""Pins of the CPU oracle to facts fixed outside it (closed forms, brute force, invariants)."""
import math

import numpy as np
import pytest

import oracle
import workloads
import _pins


# --- G-sphere ---------------------------------------------------------------------------

@pytest.mark.parametrize("lattice,k,ecut", [
    (np.diag([7.0, 8.0, 9.5]), (0.0, 0.0, 0.0), 3.0),
    (0.5 * 9.0 * np.array([[0.0, 1, 1], [1, 0, 1], [1, 1, 0]]), (0.13, -0.21, 0.07), 4.0),
    (np.array([[6.0, 0.5, 0.0], [0.3, 7.0, 0.2], [0.0, -0.4, 8.0]]), (0.05, 0.1, -0.2), 3.5),
])
def test_gsphere_bruteforce(lattice, k, ecut):
    """Pure-Python enumeration over a generous cube with G from a_i.G = 2 pi m_i."""
    got = oracle.gsphere.gsphere(lattice, ecut, k)
    ref = []
    R = 12
    for m1 in range(-R, R + 1):
        for m2 in range(-R, R + 1):
            for m3 in range(-R, R + 1):
                q = np.asarray(k) + _pins.g_cart(lattice, (m1, m2, m3))
                if 0.5 * float(q @ q) <= ecut:
                    ref.append((m1, m2, m3))
    assert max(abs(x) for m in ref for x in m) < R     # the cube was big enough
    assert [tuple(m) for m in got.tolist()] == sorted(ref)   # same set, lexicographic order


def test_gsphere_inversion_and_shift():
    lat = 0.5 * 10.2 * np.array([[0.0, 1, 1], [1, 0, 1], [1, 1, 0]])
    g0 = oracle.gsphere.gsphere(lat, 6.0, np.zeros(3))
    assert sorted(map(tuple, (-g0).tolist())) == sorted(map(tuple, g0.tolist()))
    b = oracle.gsphere.reciprocal(lat)
    k = np.array([0.11, 0.02, -0.05])
    gk = oracle.gsphere.gsphere(lat, 6.0, k)
    gkb = oracle.gsphere.gsphere(lat, 6.0, k + b[0])
    assert sorted(map(tuple, (gkb + np.array([1, 0, 0])).tolist())) == sorted(map(tuple, gk.tolist()))


@pytest.mark.parametrize("name,npw", [("c1", 1503), ("c2", 36785)])
def test_gsphere_counts_and_margins(name, npw):
    p = workloads.CONFIGS[name]()
    m = oracle.gsphere.gsphere(p.lattice, p.ecut, p.kpts[0])
    assert len(m) == npw
    # no G lies within 1e-8 Ha of the cutoff, so any rounding order gives the same set
    assert oracle.gsphere.cutoff_margin(p.lattice, p.ecut, p.kpts[0]) > 1e-8
    assert all(n >= b for n, b in zip(p.fft, oracle.gsphere.min_box(m)))


def test_gsphere_margins_fcc_kpoints():
    p = workloads.config4a()
    for k in p.kpts:
        assert oracle.gsphere.cutoff_margin(p.lattice, p.ecut, k) > 1e-8
        m = oracle.gsphere.gsphere(p.lattice, p.ecut, k)
        assert 1500 < len(m) < 1700


# --- H psi -------------------------------------------------------------------------------

def test_bruteforce_real_space():
    """FFT H psi equals explicit Cartesian sums on a tiny fcc cell, non-cubic box, k != 0, full D."""
    assert _pins.pin_bruteforce() < 1e-13


def test_dense_matches_fft():
    assert _pins.pin_dense_vs_fft() < 1e-13


def test_vtilde_closed_form():
    """Direct DFT of the sampled wells equals the analytic Gaussian transform with e^{-iG.R_a}."""
    assert _pins.pin_vtilde_analytic() < 1e-14


def test_plane_wave_column_orientation():
    assert _pins.pin_plane_wave_column() < 1e-14


def test_free_electron_exact():
    e_hpsi, e_eig = _pins.pin_free_electron()
    assert e_hpsi == 0.0 or e_hpsi < 1e-15
    assert e_eig < 1e-13


def test_constant_potential():
    assert _pins.pin_constant_potential() < 1e-14


def test_hermiticity():
    assert _pins.pin_hermiticity() < 1e-13


def test_secular_equation_rank_one():
    assert _pins.secular_residual() < 1e-9


def test_rigid_shift_invariance():
    """Eigenvalues do not change when every atom moves by the same off-grid vector."""
    lat = np.diag([10.0, 10.0, 10.0])
    rng = np.random.default_rng(21)
    atoms = rng.random((2, 3)) @ lat
    tau = np.array([1.234, -0.567, 2.345])
    e0 = _pins.eigs_dense_of(lat, atoms, 3.0, (32, 32, 32), (0, 0, 0), 12)
    e1 = _pins.eigs_dense_of(lat, atoms + tau, 3.0, (32, 32, 32), (0, 0, 0), 12)
    assert np.max(np.abs(e0 - e1)) < 1e-11
    # and the potential is not trivial: it moves the levels away from free electrons
    assert np.max(np.abs(e0 - _pins.eigs_dense_of(lat, atoms[:1], 3.0, (32, 32, 32), (0, 0, 0), 12))) > 1e-2


def test_k_periodicity_and_time_reversal():
    lat = 0.5 * 10.2 * np.array([[0.0, 1, 1], [1, 0, 1], [1, 1, 0]])
    rng = np.random.default_rng(22)
    atoms = rng.random((2, 3)) @ lat
    k = np.array([0.21, -0.13, 0.08])
    b = oracle.gsphere.reciprocal(lat)
    e_k = _pins.eigs_dense_of(lat, atoms, 4.0, (36, 36, 36), k, 10)
    e_kb = _pins.eigs_dense_of(lat, atoms, 4.0, (36, 36, 36), k + b[1], 10)
    e_mk = _pins.eigs_dense_of(lat, atoms, 4.0, (36, 36, 36), -k, 10)
    assert np.max(np.abs(e_k - e_kb)) < 1e-11
    assert np.max(np.abs(e_k - e_mk)) < 1e-11


def test_h_diagonal_two_routes():
    p, k, miller, vr, beta, d = _pins.tiny_problem(ecut=2.0, fft=(12, 13, 14), dense_d=True)
    h = oracle.hamiltonian.dense_h(p.lattice, k, miller, p.fft, vr, beta, d)
    hd = oracle.hamiltonian.h_diagonal(p.lattice, k, miller, vr, beta, d)
    assert np.max(np.abs(np.real(np.diag(h)) - hd)) < 1e-13
    assert np.max(np.abs(np.imag(np.diag(h)))) < 1e-14


# --- Davidson steps ----------------------------------------------------------------------

def test_preconditioner_exact_for_diagonal_h():
    """With H diagonal, D g_i = psi_i on every component whose denominator is not clamped."""
    rng = np.random.default_rng(2)
    hd = np.sort(rng.uniform(0.0, 5.0, 300))
    psi = workloads.random_block(300, 4, 1)
    eps = np.array([0.3, 1.1, 2.0, 3.3])
    g = oracle.davidson.residuals(hd[None, :] * psi, psi, eps)
    dpsi = oracle.davidson.precondition(g, hd, eps, tau=0.1)
    mask = np.abs(hd[None, :] - eps[:, None]) >= 0.1
    assert np.max(np.abs(dpsi[mask] - psi[mask])) < 1e-13
    # clamped components: g / (+-tau)
    x = hd[None, :] - eps[:, None]
    exp_small = g / np.where(x >= 0, 0.1, -0.1)
    assert np.max(np.abs(dpsi[~mask] - exp_small[~mask])) < 1e-15


def test_rayleigh_ritz_recovers_invariant_subspace():
    """A basis that contains the lowest eigenvectors (mixed and padded) returns the exact pairs."""
    p, k, miller, vr, beta, d = _pins.tiny_problem(ecut=2.0, fft=(12, 13, 14), dense_d=True)
    h = oracle.hamiltonian.dense_h(p.lattice, k, miller, p.fft, vr, beta, d)
    w, v = np.linalg.eigh(h)
    nb = 5
    rng = np.random.default_rng(4)
    u, _ = np.linalg.qr(rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb)))
    basis = np.concatenate([(v[:, :nb] @ u).T, workloads.random_block(len(miller), 4, 8)], axis=0)
    e, psi, hpsi = oracle.davidson.rayleigh_ritz(basis, (h @ basis.T).T, nb)
    assert np.max(np.abs(e - w[:nb])) < 1e-12
    assert np.max(np.abs(psi @ h.T - e[:, None] * psi)) < 1e-11
    assert np.max(np.abs(hpsi - psi @ h.T)) < 1e-11


# --- dense vs iterative routes -----------------------------------------------------------

@pytest.mark.slow
def test_lobpcg_matches_dense_c1():
    """The two oracle eigen-routes agree on the 1503-PW cell to 1e-10 Ha."""
    p = workloads.config1()
    k = np.zeros(3)
    miller = oracle.gsphere.gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, miller)
    d = workloads.dmat(len(p.atoms))
    h = oracle.hamiltonian.dense_h(p.lattice, k, miller, p.fft, vr, beta, d)
    e_dense = oracle.eigen.lowest_dense(h, p.nbnd)
    x0 = workloads.psi0(p.lattice, k, miller, p.nbnd + 8, p.psi_seed)
    e_lob, res = oracle.eigen.lowest_lobpcg(p.lattice, k, miller, p.fft, vr, beta, d, p.nbnd, x0, tol=1e-10)
    assert np.max(np.abs(e_lob - e_dense)) < 1e-10
