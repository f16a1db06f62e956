"""Pins of the oracle's band-by-band conjugate-gradient eigensolver (App. A.2.2) to facts outside it."""
import numpy as np

import oracle
import _pins


def test_cg_matches_lapack_on_dense_h():
    """A small fcc cell at a general k: CG eigenvalues (in the order found) equal LAPACK's, the block
    is orthonormal and every residual is within tol."""
    assert _pins.pin_cg_dense() < 1e-9


def test_cg_free_electrons():
    """V = 0, no projectors: the sorted kinetic energies (closed form)."""
    assert _pins.pin_cg_free() < 1e-10


def test_cg_line_minimum_is_2x2_eigenvalue():
    assert _pins.pin_cg_angle() < 1e-12


def test_cg_gradient_orthogonal_to_psi():
    assert _pins.pin_cg_gradient() < 1e-12


def test_cg_kinetic_preconditioner_is_effective():
    assert _pins.pin_cg_precond_ratio() < 0.6


def test_cg_energy_decreases_monotonically():
    """Each step minimises <psi|H|psi> exactly on a curve through psi, so eps never rises."""
    h, kin, x0 = _pins.cg_problem()
    p2 = oracle.cg.precond_p2(kin)
    lower = np.zeros((0, h.shape[0]), dtype=np.complex128)
    for i in range(3):
        psi, hpsi, eps, res, steps, hist = oracle.cg.cg_band(lambda v: h @ v, x0[i], lower, p2, 1e-9, 500)
        assert np.all(np.diff(hist) <= 1e-12 * (1.0 + abs(eps)))
        lower = np.vstack([lower, psi[None, :]])
