"""The seeded input generators: determinism, normalisation, two routes for V(r)."""
import numpy as np

import oracle
import workloads


def test_vloc_separable_matches_bruteforce():
    lat = np.diag([8.0, 9.0, 11.0])
    atoms = np.array([[0.5, 1.0, 10.5], [7.9, 4.0, 2.0], [3.0, 8.8, 0.1]])
    fft = (10, 12, 14)
    a = workloads.vloc_r(lat, atoms, fft)
    b = workloads.vloc_r(lat, atoms, fft, brute_force=True)
    assert np.max(np.abs(a - b)) < 1e-13
    assert a.max() < 0.0 and a.min() > -8.0


def test_beta_unit_norm_and_phase():
    p = workloads.config1()
    k = np.zeros(3)
    m = oracle.gsphere.gsphere(p.lattice, p.ecut, k)
    b = workloads.beta(p.lattice, p.atoms, k, m)
    assert b.shape == (8, len(m))
    assert np.allclose(np.sum(np.abs(b) ** 2, axis=1), 1.0, atol=1e-14)
    g0 = np.where((m == 0).all(axis=1))[0][0]
    assert np.all(b[1::4, g0] == 0.0)          # p projectors vanish at q = 0


def test_inputs_are_deterministic():
    a, b = workloads.config2(), workloads.config2()
    assert np.array_equal(a.atoms, b.atoms)
    c = workloads.config4b()
    assert len(c) == 32
    assert all(8.0 <= x.lattice[0, 0] <= 14.0 for x in c)
    assert all(1 <= len(x.atoms) <= 4 and 8 <= x.nbnd <= 32 for x in c)
    assert min(x.fft[0] for x in c) >= 25 and max(x.fft[0] for x in c) <= 50


def test_dmat_and_psi0():
    d = workloads.dmat(3)
    assert d.shape == (12, 12) and np.allclose(np.diag(d).real[:4], [1, -0.5, -0.5, -0.5])
    p = workloads.config1()
    m = oracle.gsphere.gsphere(p.lattice, p.ecut, np.zeros(3))
    x = workloads.psi0(p.lattice, np.zeros(3), m, 4, 1)
    y = workloads.psi0(p.lattice, np.zeros(3), m, 4, 1)
    assert np.array_equal(x, y) and x.shape == (4, len(m))
