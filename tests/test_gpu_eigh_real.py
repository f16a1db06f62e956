"""The real symmetric reduced eigensolver (the Rayleigh-Ritz problem of the Gamma-point Davidson,
Sec. 4 with App. A.2.1) through the C ABI, against LAPACK (oracle.eigen.lowest_dense).

Eigenvalues are compared one by one; eigenvectors, unique only up to a sign (and a rotation inside a
degenerate eigenvalue), are checked through their residuals and orthonormality.
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
    return B.hpsi_setup(p.lattice, p.ecut, [p.kpts[0]], p.fft, np.zeros(p.fft), None, None, B.HPSI_FP64,
                        torch.cuda.current_stream().cuda_stream)


def _sym(n, seed, spectrum=None, scale=1.0):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(-scale, scale, n) if spectrum is None else np.asarray(spectrum, dtype=np.float64)
    return (q * lam[None, :]) @ q.T


def _solve(ctx, a, nwant, lda=None, lower_fill=None):
    import torch
    from paper_0906_2569_gb300 import binding as B
    n = a.shape[0]
    lda = n if lda is None else lda
    col = np.full((n, lda), np.nan)   # row c of col = column c of a
    col[:, :n] = a.T
    if lower_fill is not None:
        for c in range(n):
            col[c, c + 1:n] = lower_fill
    at = torch.from_numpy(col).cuda()
    w = torch.empty(nwant, dtype=torch.float64, device="cuda")
    v = torch.empty((nwant, n), dtype=torch.float64, device="cuda")
    B.hpsi_eigh_lowest_sym(ctx, at, n, lda, nwant, w, v)
    torch.cuda.synchronize()
    return w.cpu().numpy(), v.cpu().numpy().T


def _check(a, w, x, tol_eig=1e-12, tol_res=1e-11):
    nwant = len(w)
    ref = oracle.eigen.lowest_dense(a, nwant)
    scale = max(1.0, float(np.max(np.abs(np.linalg.eigvalsh(a)))))
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(x))
    assert np.max(np.abs(w - ref)) <= tol_eig * scale, np.max(np.abs(w - ref))
    assert np.all(np.diff(w) >= -tol_eig * scale)
    res = np.linalg.norm(a @ x - x * w[None, :], axis=0)
    assert np.max(res) <= tol_res * scale, np.max(res)
    assert np.max(np.abs(x.T @ x - np.eye(nwant))) <= 1e-12


@pytest.mark.parametrize("n,nwant", [(1, 1), (2, 1), (3, 3), (31, 8), (160, 40), (333, 160), (640, 160),
                                     (1024, 256), (1536, 512), (1824, 64)])
def test_random_symmetric(ctx, n, nwant):
    a = _sym(n, 100 + n, scale=20.0)
    w, x = _solve(ctx, a, nwant)
    _check(a, w, x)


def test_degenerate_spectrum_cut_inside_a_multiplet(ctx):
    spec = np.repeat([-3.0, -1.0, 0.5, 2.0, 7.0], [6, 12, 24, 8, 150])
    w, x = _solve(ctx, _sym(len(spec), 7, spectrum=spec), 30)
    _check(_sym(len(spec), 7, spectrum=spec), w, x)


def test_close_but_distinct_eigenvalues(ctx):
    spec = np.concatenate([1.0 + 1e-9 * np.arange(10), 1.0 + 1e-6 * np.arange(1, 11), np.linspace(2, 40, 180)])
    a = _sym(len(spec), 8, spectrum=spec)
    w, x = _solve(ctx, a, 40)
    _check(a, w, x)


def test_diagonal_split_and_zero(ctx):
    d = np.array([5.0, -1.0, 3.0, 3.0, 0.0, -7.0, 2.5, 3.0] * 8)
    w, x = _solve(ctx, np.diag(d), 20)
    _check(np.diag(d), w, x)
    w, x = _solve(ctx, np.zeros((50, 50)), 5)
    assert np.max(np.abs(w)) <= 1e-28 and np.max(np.abs(x.T @ x - np.eye(5))) <= 1e-12


def test_leading_dimension_and_unread_lower_triangle(ctx):
    a = _sym(200, 3, scale=5.0)
    w, x = _solve(ctx, a, 50, lda=217, lower_fill=np.nan)
    _check(a, w, x)


def test_real_form_of_a_cell(ctx):
    """H of the small fcc cell at Gamma in the real basis of Sec. 4 (oracle.gamma.real_h): real
    symmetric, the same spectrum as the complex Hermitian H."""
    import _pins
    lat, m, fft, vr, h = _pins.gamma_problem()
    hr = oracle.gamma.real_h(h, m)
    assert np.max(np.abs(hr.imag)) < 1e-12
    w, x = _solve(ctx, np.ascontiguousarray(hr.real), 12)
    _check(hr.real, w, x)
    assert np.max(np.abs(w - oracle.eigen.lowest_dense(h, 12))) < 1e-12


def test_too_large_is_refused(ctx):
    import torch
    from paper_0906_2569_gb300 import binding as B
    n = 2049
    a = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    w = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_eigh_lowest_sym(ctx, a, n, n, 1, w, w)
    assert e.value.status == B.HPSI_EINVAL


@pytest.fixture(scope="module")
def ctx_df(lib):
    """A context whose real reduction runs in double-float arithmetic (HPSI_OPT_EIGH_DF = 2)."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    c = B.hpsi_setup(p.lattice, p.ecut, [p.kpts[0]], p.fft, np.zeros(p.fft), None, None, B.HPSI_FP64,
                     torch.cuda.current_stream().cuda_stream)
    B.hpsi_set_option(c, B.HPSI_OPT_EIGH_DF, 2)
    return c


@pytest.mark.parametrize("n,nwant", [(1, 1), (2, 1), (3, 3), (31, 8), (333, 160), (1024, 256), (1536, 512),
                                     (1824, 64)])
def test_double_float_reduction(ctx_df, n, nwant):
    """The Householder reduction on pairs of float32 (~48-bit significands): eigenvalues and
    residuals within 5e-12 of the spectral radius, eigenvectors orthonormal to 1e-12."""
    a = _sym(n, 100 + n, scale=20.0)
    w, x = _solve(ctx_df, a, nwant)
    ref = oracle.eigen.lowest_dense(a, nwant)
    print(f"n {n}: double-float reduction, max eigenvalue error {np.max(np.abs(w - ref)) / 20.0:.2e} of the radius")
    _check(a, w, x, tol_eig=5e-12, tol_res=5e-11)


def test_double_float_reduction_clusters(ctx_df):
    spec = np.concatenate([np.repeat([-3.0, 0.5], [6, 24]), 1.0 + 1e-9 * np.arange(10),
                           1.0 + 1e-6 * np.arange(1, 11), np.linspace(2, 40, 150)])
    a = _sym(len(spec), 9, spectrum=spec)
    w, x = _solve(ctx_df, a, 60)
    _check(a, w, x, tol_eig=5e-12, tol_res=5e-11)
