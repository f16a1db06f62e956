"""The reduced Hermitian eigensolver (the Rayleigh-Ritz problem of App. A.2.1) through the C ABI,
against the oracle's LAPACK eigenvalues.

Eigenvalues are compared one by one; eigenvectors, unique only up to a phase (and a unitary
mixing inside a degenerate eigenvalue), are checked through their residuals and orthonormality.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    k = p.kpts[0]
    return B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, np.zeros(p.fft), None, None, B.HPSI_FP64,
                        torch.cuda.current_stream().cuda_stream)


def _solve(ctx, a, nwant, lda=None, lower_fill=None):
    import torch
    from paper_0906_2569_gb300 import binding as B
    n = a.shape[0]
    lda = n if lda is None else lda
    col = np.full((n, lda), np.nan + 1j * np.nan, dtype=np.complex128)   # row c of col = column c of a
    col[:, :n] = a.T
    if lower_fill is not None:
        for c in range(n):
            col[c, c + 1:n] = lower_fill                                      # strictly lower triangle
    at = torch.from_numpy(col).cuda()
    w = torch.empty(nwant, dtype=torch.float64, device="cuda")
    v = torch.empty((nwant, n), dtype=torch.complex128, device="cuda")
    B.hpsi_eigh_lowest(ctx, at, n, lda, nwant, w, v)
    torch.cuda.synchronize()
    return w.cpu().numpy(), v.cpu().numpy().T       # vectors as columns


def _check(a, w, x, tol_eig=1e-12, tol_res=1e-11):
    nwant = len(w)
    ref = oracle.eigen.lowest_dense(a, nwant)
    scale = max(1.0, float(np.max(np.abs(np.linalg.eigvalsh(a)))))
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(x))
    assert np.max(np.abs(w - ref)) <= tol_eig * scale, np.max(np.abs(w - ref))
    assert np.all(np.diff(w) >= -tol_eig * scale)
    res = np.linalg.norm(a @ x - x * w[None, :], axis=0)
    assert np.max(res) <= tol_res * scale, np.max(res)
    assert np.max(np.abs(x.conj().T @ x - np.eye(nwant))) <= 1e-12


@pytest.mark.parametrize("n,nwant", [(1, 1), (2, 1), (3, 3), (31, 8), (160, 40), (333, 160), (640, 160),
                                     (1024, 256)])
def test_random_hermitian(ctx, n, nwant):
    a = workloads.hermitian_matrix(n, 100 + n, scale=20.0)
    w, x = _solve(ctx, a, nwant)
    _check(a, w, x)


def test_degenerate_spectrum_cut_inside_a_multiplet(ctx):
    spec = np.repeat([-3.0, -1.0, 0.5, 2.0, 7.0], [6, 12, 24, 8, 150])
    a = workloads.hermitian_matrix(len(spec), 7, spectrum=spec)
    w, x = _solve(ctx, a, 30)          # the 24-fold value 0.5 is cut after 12 of its vectors
    _check(a, w, x)


def test_close_but_distinct_eigenvalues(ctx):
    spec = np.concatenate([1.0 + 1e-9 * np.arange(10), 1.0 + 1e-6 * np.arange(1, 11), np.linspace(2, 40, 180)])
    a = workloads.hermitian_matrix(len(spec), 8, spectrum=spec)
    w, x = _solve(ctx, a, 40)
    _check(a, w, x)


def test_diagonal_and_split_tridiagonal(ctx):
    d = np.array([5.0, -1.0, 3.0, 3.0, 0.0, -7.0, 2.5, 3.0] * 8)
    w, x = _solve(ctx, np.diag(d).astype(np.complex128), 20)
    _check(np.diag(d).astype(np.complex128), w, x)
    t = np.diag(np.arange(40, dtype=float)) + 0j
    for i in range(39):
        if i % 5 != 4:                 # zero couplings split the matrix into 5x5 blocks
            t[i, i + 1] = t[i + 1, i] = 0.7
    w, x = _solve(ctx, t, 25)
    _check(t, w, x)


def test_zero_matrix(ctx):
    a = np.zeros((17, 17), dtype=np.complex128)
    w, x = _solve(ctx, a, 5)
    assert np.max(np.abs(w)) <= 1e-12         # the bisection interval around 0 is ~1e-30 wide
    assert np.max(np.abs(x.conj().T @ x - np.eye(5))) <= 1e-12


def test_only_upper_triangle_read_and_lda(ctx):
    a = workloads.hermitian_matrix(200, 9, scale=5.0)
    w, x = _solve(ctx, a, 50, lda=213, lower_fill=np.nan)
    _check(a, w, x)


def test_reduced_problem_of_a_cell(ctx):
    """The dense H of the small synthetic cell (a Davidson-like spectrum with near-degenerate shells)."""
    p = workloads.small_cell()
    k = p.kpts[0]
    m = oracle.gsphere.gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    h = oracle.hamiltonian.dense_h(p.lattice, k, m, p.fft, vr, beta, workloads.dmat(len(p.atoms)))
    w, x = _solve(ctx, h, min(len(m), 60))
    _check(h, w, x)


def test_library_path_ran_and_matches_cusolver(ctx):
    from paper_0906_2569_gb300 import binding as B
    a = workloads.hermitian_matrix(400, 11, scale=30.0)
    keig = B.KERNELS.index("eigh")
    B.hpsi_kernel_stats(ctx, -1, reset=True)
    B.hpsi_kernel_stats(ctx, -4, reset=True)
    w1, x1 = _solve(ctx, a, 100)
    assert B.hpsi_kernel_stats(ctx, keig)[0] >= 3   # multisection, inverse iteration, back-transform helpers
    assert B.hpsi_kernel_stats(ctx, B.KERNELS.index("tridiag"))[0] == 1
    calls, flops = B.hpsi_kernel_stats(ctx, -4)
    assert calls == 1 and flops == pytest.approx(16.0 / 3.0 * 400 ** 3)
    B.hpsi_set_option(ctx, B.HPSI_OPT_EIGENSOLVER, 0)
    try:
        B.hpsi_kernel_stats(ctx, -1, reset=True)
        w0, x0 = _solve(ctx, a, 100)
        assert B.hpsi_kernel_stats(ctx, keig)[0] == 0
    finally:
        B.hpsi_set_option(ctx, B.HPSI_OPT_EIGENSOLVER, 1)
    scale = float(np.max(np.abs(np.linalg.eigvalsh(a))))
    assert np.max(np.abs(w1 - w0)) <= 1e-12 * scale
    # the same invariant subspace: projector difference
    assert np.linalg.norm(x1 @ x1.conj().T - x0 @ x0.conj().T, 2) < 1e-9


def test_above_the_kernel_limit_falls_back(ctx):
    a = workloads.hermitian_matrix(1100, 12, scale=10.0)
    w, x = _solve(ctx, a, 64)
    _check(a, w, x)


def test_errors(ctx):
    import torch
    from paper_0906_2569_gb300 import binding as B
    a = torch.zeros((8, 8), dtype=torch.complex128, device="cuda")
    w = torch.empty(8, dtype=torch.float64, device="cuda")
    v = torch.empty((8, 8), dtype=torch.complex128, device="cuda")
    for n, lda, nw in [(8, 8, 9), (0, 8, 1), (8, 7, 2), (8, 8, 0)]:
        with pytest.raises(B.HpsiError, match="HPSI_EINVAL"):
            B.hpsi_eigh_lowest(ctx, a, n, lda, nw, w, v)
