"""Pins of the oracle's Gamma-point Fock exchange (App. A.5) to facts outside it: an Ewald closed
form for a Gaussian orbital's self-exchange with the Gygi-Baldereschi correction, Hermiticity, and
invariance under rotations of the occupied orbitals."""
import _pins


def test_fock_gaussian_closed_form():
    assert _pins.pin_fock_gaussian() < 1e-9


def test_fock_hermitian_and_subspace_invariant():
    assert _pins.pin_fock_hermitian_invariant() < 1e-12
