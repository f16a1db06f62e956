"""GPU band-by-band conjugate-gradient eigensolver (App. A.2.2) through the C ABI, against the oracle.

Eigenvalues are compared with the oracle's dense LAPACK / LOBPCG values (tests/golden) and with the
oracle's own CG on the same start vectors; the returned block must be orthonormal, ordered and
within tol in every residual.  Step limits: the oracle's CG on the same problems needs at most
1933 steps for a band of c1 (16 bands; 4740 in all, the GPU took the same 4740), 61 for the
free-electron c1, 435 for c4a k-point 1 and 552 for the first four bands of c2; 3000 leaves room.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", "eigenvalues.json")
    return json.load(open(path))[name]["eigenvalues"]


def _setup(p, ik=0, precision=0, zero_potential=False):
    import torch
    from paper_0906_2569_gb300 import binding as B
    k = p.kpts[ik]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    if zero_potential:
        vr, beta, d = np.zeros(p.fft), None, None
    else:
        vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
        beta = workloads.beta(p.lattice, p.atoms, k, m)
        d = workloads.dmat(len(p.atoms))
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, None if beta is None else [beta], d, precision,
                       torch.cuda.current_stream().cuda_stream)
    return ctx, m, vr, beta, d


def _check_block(v, h_apply, eig, tol):
    nb = v.shape[0]
    assert np.max(np.abs(np.conj(v) @ v.T - np.eye(nb))) < 1e-12
    assert np.max(np.linalg.norm(h_apply(v) - eig[:, None] * v, axis=1)) <= 1.01 * tol


def test_cg_fp64_c1_against_dense_and_oracle_cg(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    x0 = workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)
    x = torch.from_numpy(x0.copy()).cuda()
    eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-8, 3000)
    ref = np.asarray(_golden("c1")[:p.nbnd])
    assert np.max(np.abs(eig - ref)) < 1e-10
    assert np.all(np.diff(eig) >= -1e-12)
    assert np.max(res) <= 1e-8
    h = oracle.hamiltonian.dense_h(p.lattice, p.kpts[0], m, p.fft, vr, beta, d)
    _check_block(x.cpu().numpy(), lambda v: v @ h.T, eig, 1e-8)
    kin = oracle.gsphere.kinetic(p.lattice, p.kpts[0], m)
    eo, _, _, so = oracle.cg.cg_solve(lambda v: h @ v, x0, kin, 1e-8, 3000)
    assert np.max(np.abs(eig - eo)) < 1e-10
    assert steps > 0


def test_cg_kpoint_complex_h_c4a(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config4a()
    ctx, m, vr, beta, d = _setup(p, ik=1)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[1], m, p.nbnd, p.psi_seed + 1)).cuda()
    eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-8, 3000)
    assert np.max(np.abs(eig - np.asarray(_golden("c4a")[1]))) < 1e-10
    h = oracle.hamiltonian.dense_h(p.lattice, p.kpts[1], m, p.fft, vr, beta, d)
    _check_block(x.cpu().numpy(), lambda v: v @ h.T, eig, 1e-8)


def test_cg_free_electron(lib):
    """V = 0, no projectors: the sorted kinetic energies (closed form)."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p, zero_potential=True)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-9, 400)
    t = np.sort(oracle.gsphere.kinetic(p.lattice, p.kpts[0], m))[:p.nbnd]
    assert np.max(np.abs(eig - t)) < 1e-12


def test_cg_c2_fp64_lowest_bands(lib):
    """The 36785-PW, 256-projector cell, the first four bands, against the oracle's LOBPCG values."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, m, vr, beta, d = _setup(p)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, 4, p.psi_seed)).cuda()
    eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-8, 3000)
    assert np.max(np.abs(eig - np.asarray(_golden("c2")[:4]))) < 1e-10
    v = x.cpu().numpy()
    assert np.max(np.abs(np.conj(v) @ v.T - np.eye(4))) < 1e-12
    assert np.max(res) <= 1e-8


def test_cg_host_buffer_and_errors(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    x = workloads.psi0(p.lattice, p.kpts[0], m, 4, p.psi_seed)
    eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-8, 400)
    assert np.max(np.abs(eig - np.asarray(_golden("c1")[:4]))) < 1e-10
    assert np.max(np.abs(np.conj(x) @ x.T - np.eye(4))) < 1e-12
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, 4, p.psi_seed)).cuda()
    eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-12, 2, raise_on_notconv=False)
    assert rc == B.HPSI_ENOTCONV
    zero_row = workloads.psi0(p.lattice, p.kpts[0], m, 2, p.psi_seed)
    zero_row[1] = 0.0
    with pytest.raises(B.HpsiError):
        B.cg_solve(ctx, 0, torch.from_numpy(zero_row).cuda(), 1e-8, 100)   # no start vector for band 1
    with pytest.raises(B.HpsiError):
        B.cg_solve(ctx, 0, x, 0.0, 10)
    with pytest.raises(B.HpsiError):
        B.hpsi_set_option(ctx, B.HPSI_OPT_CG_TMIN, 0.0)
