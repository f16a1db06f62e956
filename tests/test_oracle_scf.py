"""Pins of the oracle's self-consistency loop (App. A.1) to facts outside it: an Ewald closed form
for the Hartree energy, brute-force DFT sums, the LDA's derivative and limits, charge conservation,
a linear fixed point for the mixing, and the paper's statements about the two energy forms."""
import numpy as np

import oracle
import _pins


def test_hartree_gaussian_closed_form():
    assert _pins.pin_hartree_gaussian() < 1e-12


def test_hartree_bruteforce():
    assert _pins.pin_hartree_bruteforce() < 1e-12


def test_lda_potential_is_derivative():
    assert _pins.pin_lda_derivative() < 1e-6


def test_lda_limits():
    assert _pins.pin_lda_limits() <= 1.0


def test_density_charge():
    assert _pins.pin_density_charge() < 1e-12


def test_mixer_reaches_linear_fixed_point():
    assert _pins.pin_mixer_linear() < 1e-9


def test_scf_fixed_point_and_energy_forms():
    """At self-consistency rho_out(rho*) = rho*, and the standard and Harris-Weinert-Foulkes energies
    agree (both are variational and meet at the solution)."""
    lat, k, miller, fft, vr, beta, d = _pins.scf_small()
    rho0 = np.full(fft, 4.0 / oracle.scf.cell_volume(lat))
    out = oracle.scf.scf(lat, k, miller, fft, vr, beta, d, 2, rho0, tol=1e-20, maxiter=80)
    assert out["norm2"][-1] < 1e-20
    assert abs(oracle.scf.charge(out["rho"], lat) - 4.0) < 1e-9
    assert abs(out["e"] - out["e_hwf"]) < 1e-9
    # a different start reaches the same energy
    rho1 = oracle.scf.density(out["psi"][::-1], np.array([3.0, 1.0]), miller, fft, lat)
    out1 = oracle.scf.scf(lat, k, miller, fft, vr, beta, d, 2, rho1, tol=1e-20, maxiter=80)
    assert abs(out1["e"] - out["e"]) < 1e-9


def test_energy_forms_differ_to_second_order():
    """Both energy forms have no first-order term in the density error (the paper's variational
    statement), so E - E' shrinks four-fold when the input density's error is halved."""
    lat, k, miller, fft, vr, beta, d = _pins.scf_small()
    rho0 = np.full(fft, 4.0 / oracle.scf.cell_volume(lat))
    out = oracle.scf.scf(lat, k, miller, fft, vr, beta, d, 2, rho0, tol=1e-20, maxiter=80)
    rng = np.random.default_rng(3)
    pert = rng.standard_normal(fft)
    pert -= pert.mean()
    pert *= 1e-3 * np.max(out["rho"]) / np.max(np.abs(pert))
    diffs = []
    for s in (1.0, 0.5):
        rho_in = out["rho"] + s * pert
        v_hxc, _ = oracle.scf.hxc(rho_in, lat)
        h = oracle.hamiltonian.dense_h(lat, k, miller, fft, vr + v_hxc, beta, d)
        w, v = np.linalg.eigh(h)
        rho_out = oracle.scf.density(v[:, :2].T, np.array([2.0, 2.0]), miller, fft, lat)
        e, e2 = oracle.scf.energies(w[:2], np.array([2.0, 2.0]), rho_in, rho_out, lat)
        diffs.append(e - e2)
    assert 3.0 < diffs[0] / diffs[1] < 5.0
