"""Pins of the oracle's Gamma-point real-wavefunction form (Sec. 4): storage of half the
components, the real basis in which H is real symmetric, and two bands per complex FFT."""
import _pins


def test_half_storage():
    assert _pins.pin_gamma_storage() < 1e-12


def test_real_symmetric_h_same_spectrum():
    assert _pins.pin_gamma_real_h() < 1e-11


def test_two_bands_per_fft():
    assert _pins.pin_gamma_pair_fft() < 1e-13
