"""GPU Davidson (through the C ABI) against the oracle's eigenvalues.

Eigenvalues are unique, eigenvectors are not (degenerate shells): the test compares sorted
eigenvalues and checks that the returned vectors are orthonormal with small residuals.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _setup(p, precision=0, zero_potential=False):  # noqa: D103
    import torch
    from paper_0906_2569_gb300 import binding as B
    k = p.kpts[0]
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


def test_davidson_fp64_c1(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-8, 200)
    h = oracle.hamiltonian.dense_h(p.lattice, p.kpts[0], m, p.fft, vr, beta, d)
    e_ref = oracle.eigen.lowest_dense(h, p.nbnd)
    assert np.max(np.abs(eig - e_ref)) < 1e-10
    assert np.max(res) <= 1e-8
    v = x.cpu().numpy()
    assert np.max(np.abs(np.conj(v) @ v.T - np.eye(p.nbnd))) < 1e-12
    assert np.max(np.linalg.norm(v @ h.T - eig[:, None] * v, axis=1)) < 1e-7


def test_davidson_free_electron(lib):
    """V = 0, no projectors: eigenvalues are the sorted |k+G|^2/2.  The diagonal D is exact here, so
    each correction D g_i is parallel to psi_i; with one eps for all bands (the highest Ritz value)
    the corrections are not, and the lowest eigenpairs are found."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p, zero_potential=True)
    B.hpsi_set_option(ctx, B.HPSI_OPT_PRECOND_SHIFT, 1)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-8, 300)
    t = np.sort(oracle.gsphere.kinetic(p.lattice, p.kpts[0], m))[:p.nbnd]
    assert np.max(np.abs(eig - t)) < 1e-10


def test_davidson_notconv_and_errors(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-12, 2, raise_on_notconv=False)
    assert rc == B.HPSI_ENOTCONV and it == 2
    with pytest.raises(B.HpsiError):
        B.davidson_solve(ctx, 0, torch.zeros((p.nbnd, len(m)), dtype=torch.complex128, device="cuda"), 1e-8, 10)
    with pytest.raises(B.HpsiError):
        B.davidson_solve(ctx, 0, x, -1.0, 10)
    with pytest.raises(B.HpsiError):
        B.hpsi_set_option(ctx, 99, 1.0)
    with pytest.raises(B.HpsiError):
        B.hpsi_set_option(ctx, B.HPSI_OPT_PRECOND_TAU, 0.0)


def test_davidson_host_buffer(lib):
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    x = workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-8, 200)
    h = oracle.hamiltonian.dense_h(p.lattice, p.kpts[0], m, p.fft, vr, beta, d)
    assert np.max(np.abs(eig - oracle.eigen.lowest_dense(h, p.nbnd))) < 1e-10
    assert np.max(np.abs(np.conj(x) @ x.T - np.eye(p.nbnd))) < 1e-12


def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "eigenvalues.json")
    data = json.load(open(path))
    if name not in data:
        pytest.fail(f"golden eigenvalues for {name} missing: run tests/golden/make_golden.py {name}")
    return data[name]["eigenvalues"]


@pytest.mark.parametrize("nbnd", [16, 160])
def test_davidson_mixed_c1(lib, nbnd):
    """Mixed path: float32 subspace, float64 eigensolves / norms / final Rayleigh quotients: 1e-6 Ha."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config3(nbnd)
    ctx, m, vr, beta, d = _setup(p, precision=B.HPSI_MIXED)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-5, 400)
    ref = np.asarray(_golden("c3")[:nbnd])
    assert np.max(np.abs(eig - ref)) < 1e-6
    v = x.cpu().numpy()
    assert np.max(np.abs(np.conj(v) @ v.T - np.eye(nbnd))) < 1e-4


@pytest.mark.parametrize("precision,tol,etol", [(0, 1e-8, 1e-10), (1, 1e-5, 1e-6)])
def test_davidson_c2(lib, precision, tol, etol):
    """The 36785-PW, 256-projector cell, 160 bands, against the oracle's LOBPCG eigenvalues."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, m, vr, beta, d = _setup(p, precision=precision)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, tol, 300)
    ref = np.asarray(_golden("c2"))
    assert np.max(np.abs(eig - ref)) < etol


def test_davidson_kpoints_c4a(lib):
    """Two k-points of the fcc cell (k != 0, complex H), float64, against dense LAPACK."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config4a()
    ref = _golden("c4a")
    kp = p.kpts[:2]
    ms = [B.hpsi_gsphere(p.lattice, p.ecut, k) for k in kp]
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    betas = [workloads.beta(p.lattice, p.atoms, k, m) for k, m in zip(kp, ms)]
    ctx = B.hpsi_setup(p.lattice, p.ecut, kp, p.fft, vr, betas, workloads.dmat(len(p.atoms)), B.HPSI_FP64,
                       torch.cuda.current_stream().cuda_stream)
    for ik in range(2):
        x = torch.from_numpy(workloads.psi0(p.lattice, kp[ik], ms[ik], p.nbnd, p.psi_seed + ik)).cuda()
        eig, it, res, rc = B.davidson_solve(ctx, ik, x, 1e-8, 300)
        assert np.max(np.abs(eig - np.asarray(ref[ik]))) < 1e-10


@pytest.mark.parametrize("gemm", [3, 2])
def test_davidson_mixed_c2_subspace_gemm_options(lib, gemm):
    """The mixed solve with the split-bf16 cuBLAS subspace products (3) and with CGEMM3M (2) reaches
    the same eigenvalues, and its reduced problems all go through the library's eigensolver."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, m, vr, beta, d = _setup(p, precision=B.HPSI_MIXED)
    B.hpsi_set_option(ctx, B.HPSI_OPT_FP32_GEMM, gemm)
    B.hpsi_kernel_stats(ctx, -3, reset=True)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-5, 300)
    assert np.max(np.abs(eig - np.asarray(_golden("c2")))) < 1e-6
    calls, fallbacks = B.hpsi_kernel_stats(ctx, -3)
    assert calls >= it and fallbacks == 0


def test_davidson_cusolver_option_matches(lib):
    """HPSI_OPT_EIGENSOLVER = 0 (cuSOLVER zheevdx for the reduced problems) gives the same float64
    eigenvalues as the library's own eigensolver, and the library counters stay at zero."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    x0 = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    e1, _, _, _ = B.davidson_solve(ctx, 0, x0.clone(), 1e-8, 200)
    B.hpsi_set_option(ctx, B.HPSI_OPT_EIGENSOLVER, 0)
    B.hpsi_kernel_stats(ctx, -3, reset=True)
    e0, _, _, _ = B.davidson_solve(ctx, 0, x0.clone(), 1e-8, 200)
    assert B.hpsi_kernel_stats(ctx, -3)[0] == 0
    assert np.max(np.abs(e1 - e0)) < 1e-10


def test_davidson_mixed_c3_320_bands(lib):
    """The 320-band run of the mixed form on the 1500-PW cell: the reduced basis (up to 1280 vectors)
    nearly fills the plane-wave space and the float32 residuals sit near their rounding floor."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config3(320)
    ctx, m, vr, beta, d = _setup(p, precision=B.HPSI_MIXED)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-5, 400)
    assert np.max(np.abs(eig - np.asarray(_golden("c3")[:320]))) < 1e-6


@pytest.mark.parametrize("cfg,locking", [("c2", 1), ("c2", 2), ("c3", 2), ("c3_16", 2)])
def test_davidson_mixed_locking(lib, cfg, locking):
    """Hard locking (lowest converged run, or every converged band) reaches the same eigenvalues;
    the returned block is orthonormal to float32 accuracy and sorted."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2() if cfg == "c2" else workloads.config3(16 if cfg == "c3_16" else 160)
    ctx, m, vr, beta, d = _setup(p, precision=B.HPSI_MIXED)
    B.hpsi_set_option(ctx, B.HPSI_OPT_LOCKING, locking)
    B.hpsi_set_option(ctx, B.HPSI_OPT_LOCK_BATCH, 0.25)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-5, 300)
    ref = np.asarray(_golden("c2" if cfg == "c2" else "c3")[:p.nbnd])
    assert np.max(np.abs(eig - ref)) < 1e-6
    assert np.all(np.diff(eig) >= 0)
    v = x.cpu().numpy()
    assert np.max(np.abs(np.conj(v) @ v.T - np.eye(p.nbnd))) < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_davidson_plain_restart_option(lib, precision):
    """HPSI_OPT_THICK_RESTART = 0 (restart from the wanted Ritz vectors only) and the default thick
    restart reach the same eigenvalues; the Ritz-product chunking option changes nothing either."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1() if precision == 0 else workloads.config3(160)
    tol, etol = (1e-8, 1e-10) if precision == 0 else (1e-5, 1e-6)
    ctx, m, vr, beta, d = _setup(p, precision=precision)
    ref = np.asarray(_golden("c1" if precision == 0 else "c3")[:p.nbnd])
    x0 = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    its = {}
    for thick, split in ((1, 0), (0, 0), (1, 1)):
        B.hpsi_set_option(ctx, B.HPSI_OPT_THICK_RESTART, thick)
        B.hpsi_set_option(ctx, B.HPSI_OPT_RITZ_SPLIT, split)
        x = x0.clone()
        eig, it, res, rc = B.davidson_solve(ctx, 0, x, tol, 300)
        assert np.max(np.abs(eig - ref)) < etol
        its[(thick, split)] = it
    assert its[(1, 0)] <= its[(0, 0)]


def test_davidson_mixed_tc_inner_products(lib):
    """HPSI_OPT_FP32_GEMM = 4: the projections onto the basis, the H_sub columns and the overlaps run
    on the library's tcgen05 kernel (split bf16, float64 sums over K-splits).  Same eigenvalues on the
    160-band run of the small cell, orthonormal block, and the bf16 split kernels did run."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config3(160)
    ctx, m, vr, beta, d = _setup(p, precision=B.HPSI_MIXED)
    B.hpsi_set_option(ctx, B.HPSI_OPT_FP32_GEMM, 4)
    B.hpsi_kernel_stats(ctx, -1, reset=True)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-5, 300)
    assert np.max(np.abs(eig - np.asarray(_golden("c3")[:160]))) < 1e-6
    v = x.cpu().numpy()
    assert np.max(np.abs(np.conj(v) @ v.T - np.eye(160))) < 1e-4
    assert B.hpsi_kernel_stats(ctx, B.KERNELS.index("split"))[0] > 3 * it


@pytest.mark.parametrize("final", [0, 1, 2])
def test_davidson_mixed_c2_final_quotients(lib, final):
    """The final Rayleigh quotients of the mixed solve: 1 with the float64 H, 2 with float64
    projections <beta|psi> and D only (the rest at the working precision), 0 with the mixed H.
    Modes 1 and 2 stay within 1e-6 Ha of the oracle; every mode within 1e-5 Ha."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, m, vr, beta, d = _setup(p, precision=B.HPSI_MIXED)
    B.hpsi_set_option(ctx, B.HPSI_OPT_FINAL_FP64, final)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-5, 300)
    err = float(np.max(np.abs(eig - np.asarray(_golden("c2")))))
    print(f"c2 mixed, final quotients mode {final}: {it} iterations, max eigenvalue error {err:.2e} Ha")
    assert err < (1e-5 if final == 0 else 1e-6)
