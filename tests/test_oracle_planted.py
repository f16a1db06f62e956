"""Plant plausible mistakes in the oracle (on the CPU) and check that some pin catches each one."""
import numpy as np
import pytest
import scipy.fft

import oracle
import oracle.hamiltonian as H
import oracle.gsphere as GS
import oracle.davidson as DV
import _pins


def _fwd_wrong_sign(phi_r, miller, fft):
    idx = H.box_index(miller, fft)
    full = scipy.fft.ifftn(phi_r, axes=(1, 2, 3), norm="backward")     # e^{+i} with 1/N
    return full[(slice(None),) + idx]


def _fwd_no_norm(phi_r, miller, fft):
    idx = H.box_index(miller, fft)
    full = scipy.fft.fftn(phi_r, axes=(1, 2, 3), norm="backward")      # drops the 1/N_r
    return full[(slice(None),) + idx]


def _calbec_no_conj(beta, psi):
    return beta @ psi.T


def _nonlocal_dt(beta, dmat, psi):
    return ((dmat.T @ (np.conj(beta) @ psi.T)).T) @ beta


def _box_swapped(miller, fft):
    m = np.asarray(miller)
    return (np.mod(m[:, 0], fft[0]), np.mod(m[:, 2], fft[1]), np.mod(m[:, 1], fft[2]))


def _kinetic_no_half(lattice, k, miller):
    q = GS.kplusg(lattice, k, miller)
    return np.sum(q * q, axis=1)


def _vtilde_plus(vr, q):
    return np.conj(oracle.hamiltonian.__dict__["_orig_vtilde"](vr, q))


def _precondition_flipped(g, hdiag, eps, tau=0.1):
    return g / DV.clamp_denominator(np.asarray(eps)[:, None] - np.asarray(hdiag)[None, :], tau)


def _gsphere_gamma_only(lattice, ecut, k):
    return _orig_gsphere(lattice, ecut, np.zeros(3))


_orig_gsphere = GS.gsphere


@pytest.mark.parametrize("target,attr,bad,pin,thresh", [
    (H, "to_reciprocal", _fwd_wrong_sign, "bruteforce", 1e-3),
    (H, "to_reciprocal", _fwd_wrong_sign, "pwcol", 1e-3),
    (H, "to_reciprocal", _fwd_no_norm, "constV", 1e-3),
    (H, "calbec", _calbec_no_conj, "bruteforce", 1e-3),
    (H, "calbec", _calbec_no_conj, "herm", 1e-3),
    (H, "nonlocal_term", _nonlocal_dt, "bruteforce", 1e-3),
    (H, "box_index", _box_swapped, "bruteforce", 1e-3),
    (H, "kinetic", _kinetic_no_half, "free", 1e-3),
    (H, "vtilde_direct", _vtilde_plus, "vtilde", 1e-4),
    (DV, "precondition", _precondition_flipped, "precond", 1e-3),
])
def test_planted_mistake_is_caught(monkeypatch, target, attr, bad, pin, thresh):
    monkeypatch.setattr(H, "_orig_vtilde", H.vtilde_direct, raising=False)
    monkeypatch.setattr(target, attr, bad)
    if pin == "bruteforce":
        err = _pins.pin_bruteforce()
    elif pin == "pwcol":
        err = _pins.pin_plane_wave_column()
    elif pin == "constV":
        err = _pins.pin_constant_potential()
    elif pin == "herm":
        err = _pins.pin_hermiticity()
    elif pin == "free":
        err = max(_pins.pin_free_electron())
    elif pin == "vtilde":
        err = _pins.pin_vtilde_analytic()
    elif pin == "precond":
        hd = np.linspace(0.0, 5.0, 50)
        psi = np.ones((1, 50), dtype=np.complex128)
        eps = np.array([1.0])
        dpsi = DV.precondition(DV.residuals(hd[None, :] * psi, psi, eps), hd, eps)
        mask = np.abs(hd - 1.0) >= 0.1
        err = float(np.max(np.abs(dpsi[0, mask] - 1.0)))
    else:
        raise AssertionError(pin)
    assert err > thresh, f"pin {pin} missed a planted mistake in {attr}: err={err}"


def test_planted_gsphere_k_shift_is_caught(monkeypatch):
    monkeypatch.setattr(GS, "gsphere", _gsphere_gamma_only)
    lat = 0.5 * 9.0 * np.array([[0.0, 1, 1], [1, 0, 1], [1, 1, 0]])
    k = np.array([0.13, -0.21, 0.07])
    got = GS.gsphere(lat, 4.0, k)
    ok = all(0.5 * float(np.sum((k + _pins.g_cart(lat, m)) ** 2)) <= 4.0 for m in got)
    count = sum(1 for m1 in range(-8, 9) for m2 in range(-8, 9) for m3 in range(-8, 9)
                if 0.5 * float(np.sum((k + _pins.g_cart(lat, (m1, m2, m3))) ** 2)) <= 4.0)
    assert not (ok and count == len(got))


import oracle.cg as CG


def _orth_none(v, lower):
    return v


def _angle_maximum(eps, a, b):
    t = CG.__dict__["_orig_angle"](eps, a, b)
    return t + 0.5 * np.pi


def _gradient_rayleigh(psi, hpsi, p2):
    lam = float(np.real(np.vdot(psi, hpsi)))
    return lam, p2 * (hpsi - lam * psi)


def _p2_inverted(kinetic, t_min=1.0):
    return np.maximum(np.asarray(kinetic, dtype=np.float64), t_min)


@pytest.mark.parametrize("attr,bad,pin,bad_if", [
    ("_orth", _orth_none, "dense", lambda e: e > 1e-3),
    ("line_angle", _angle_maximum, "angle", lambda e: e > 1e-3),
    ("gradient", _gradient_rayleigh, "gradient", lambda e: e > 1e-6),
    ("precond_p2", _p2_inverted, "precond", lambda e: e > 0.6),
])
def test_planted_cg_mistake_is_caught(monkeypatch, attr, bad, pin, bad_if):
    monkeypatch.setattr(CG, "_orig_angle", CG.line_angle, raising=False)
    monkeypatch.setattr(CG, attr, bad)
    if pin == "dense":
        err = _pins.pin_cg_dense()
    elif pin == "angle":
        err = _pins.pin_cg_angle()
    elif pin == "gradient":
        err = _pins.pin_cg_gradient()
    else:
        err = _pins.pin_cg_precond_ratio()
    assert bad_if(err), f"pin {pin} missed a planted mistake in {attr}: err={err}"


import math

import oracle.scf as SCF

_hartree_ok = SCF.hartree
_lda_ok = SCF.lda_xc
_density_ok = SCF.density
_step_ok = SCF.AndersonMixer.step


def _hartree_no_4pi(rho, lattice):
    vh, eh = _hartree_ok(rho, lattice)
    return vh / (4 * math.pi), eh / (4 * math.pi)


def _hartree_over_g(rho, lattice):      # 1/|G| instead of 1/G^2
    import scipy.fft
    rg = scipy.fft.fftn(rho) / rho.size
    g2 = SCF.grid_g2(lattice, rho.shape)
    inv = np.zeros_like(g2)
    nz = g2 > 1e-12
    inv[nz] = 4 * math.pi / np.sqrt(g2[nz])
    return np.real(scipy.fft.ifftn(inv * rg) * rho.size), 0.5 * SCF.cell_volume(lattice) * float(np.sum(inv * np.abs(rg) ** 2))


def _lda_vx_equals_ex(rho):
    eps, v = _lda_ok(rho)
    r = np.asarray(rho, dtype=np.float64)
    ex = -0.75 * (3.0 * np.maximum(r, 0) / math.pi) ** (1.0 / 3.0)
    return eps, v - ex / 3.0          # V_x = eps_x instead of 4/3 eps_x


def _density_no_volume(psi, occ, miller, fft, lattice):
    return _density_ok(psi, occ, miller, fft, lattice) * SCF.cell_volume(lattice)


def _step_wrong_sign(self, xin, xout):
    x = _step_ok(self, xin, xout)
    return 2 * np.array(xin) - x + 0.0 * xout


@pytest.mark.parametrize("target,attr,bad,pin,bad_if", [
    (SCF, "hartree", _hartree_no_4pi, "gauss", lambda e: e > 1e-3),
    (SCF, "hartree", _hartree_over_g, "brute", lambda e: e > 1e-3),
    (SCF, "lda_xc", _lda_vx_equals_ex, "deriv", lambda e: e > 1e-3),
    (SCF, "density", _density_no_volume, "charge", lambda e: e > 1e-3),
    (SCF.AndersonMixer, "step", _step_wrong_sign, "mixer", lambda e: not (e < 1e-6)),
])
def test_planted_scf_mistake_is_caught(monkeypatch, target, attr, bad, pin, bad_if):
    monkeypatch.setattr(target, attr, bad)
    err = {"gauss": _pins.pin_hartree_gaussian, "brute": _pins.pin_hartree_bruteforce,
           "deriv": _pins.pin_lda_derivative, "charge": _pins.pin_density_charge,
           "mixer": _pins.pin_mixer_linear}[pin]()
    assert bad_if(err), f"pin {pin} missed a planted mistake in {attr}: err={err}"


import oracle.gamma as GM

_pair_ok = GM.local_pair
_basis_ok = GM.real_basis


def _partner_self(miller):
    return np.arange(len(miller))


def _pair_no_conj(vr, miller, fft, psi_a, psi_b):
    par = GM.partner_index(miller)
    phi = H.to_real_space(np.stack([psi_a + 1j * psi_b]), miller, fft)
    c = H.to_reciprocal(phi * vr[None], miller, fft)[0]
    return 0.5 * (c + c[par]), (c - c[par]) / 2j       # c(-G) without the conjugate


def _basis_no_i(miller):
    u = _basis_ok(miller)
    return np.where(np.abs(u.imag) > 0, np.abs(u.imag) * np.sign(u.imag), u.real).astype(np.complex128)


@pytest.mark.parametrize("attr,bad,pin", [
    ("partner_index", _partner_self, "storage"),
    ("local_pair", _pair_no_conj, "pair"),
    ("real_basis", _basis_no_i, "realh"),
])
def test_planted_gamma_mistake_is_caught(monkeypatch, attr, bad, pin):
    monkeypatch.setattr(GM, attr, bad)
    err = {"storage": _pins.pin_gamma_storage, "pair": _pins.pin_gamma_pair_fft,
           "realh": _pins.pin_gamma_real_h}[pin]()
    assert err > 1e-3, f"pin {pin} missed a planted mistake in {attr}: err={err}"


import oracle.fock as FK


def _xdiv_zero(lattice, fft, alpha=1.0):
    return 0.0


def _vx_codensity_swapped(psi, occupied, miller, fft, lattice, alpha=1.0):
    omega = SCF.cell_volume(lattice)
    xdiv = FK.exx_div(lattice, fft, alpha)
    pr = H.to_real_space(np.asarray(psi, dtype=np.complex128), miller, fft)
    orr = H.to_real_space(np.asarray(occupied, dtype=np.complex128), miller, fft)
    out = np.zeros_like(pr)
    for b in range(pr.shape[0]):
        for j in range(orr.shape[0]):
            out[b] -= orr[j] * FK.coulomb(orr[j] * np.conj(pr[b]) / omega, lattice, xdiv)
    return H.to_reciprocal(out, miller, fft)


@pytest.mark.parametrize("attr,bad,pin", [
    ("exx_div", _xdiv_zero, "gauss"),
    ("apply_vx", _vx_codensity_swapped, "herm"),
])
def test_planted_fock_mistake_is_caught(monkeypatch, attr, bad, pin):
    monkeypatch.setattr(FK, attr, bad)
    err = {"gauss": _pins.pin_fock_gaussian, "herm": _pins.pin_fock_hermitian_invariant}[pin]()
    assert err > 1e-3, f"pin {pin} missed a planted mistake in {attr}: err={err}"
