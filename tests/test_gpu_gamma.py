"""GPU parity of the Gamma-point real form (Sec. 4): H on half-sphere storage with two real bands
per complex transform pair, and the block Davidson on real orbitals, through the C ABI.

Reference: the oracle's full-sphere H|psi> of the real function whose half-sphere coefficients are
given (oracle.gamma.to_full, then oracle.hamiltonian.hpsi, then oracle.gamma.to_half), and the
oracle's golden eigenvalues of the same cells (the real form has the same spectrum).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    return json.load(open(os.path.join(HERE, "golden", "eigenvalues.json")))[name]["eigenvalues"]


def _setup(p, precision=0):
    import torch
    from paper_0906_2569_gb300 import binding as B
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    d = workloads.dmat(len(p.atoms))
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], d, precision, torch.cuda.current_stream().cuda_stream)
    return ctx, m, vr, beta, d


def _half_block(m, nbnd, seed):
    """Half-sphere coefficients of nbnd random real orbitals (G = 0 component real)."""
    h = np.ascontiguousarray(oracle.gamma.to_half(workloads.random_block(len(m), nbnd, seed), m))
    h[:, 0] = h[:, 0].real
    return h


def _oracle_gamma(p, m, vr, beta, d, half):
    full = oracle.gamma.to_full(half, m)
    return oracle.gamma.to_half(oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, full), m)


def _apply(ctx, half):
    import torch
    from paper_0906_2569_gb300 import binding as B
    x = torch.from_numpy(half).cuda()
    y = torch.full_like(x, float("nan"))
    B.hpsi_apply_gamma(ctx, 0, x, y)
    B.hpsi_sync(ctx)
    return y.cpu().numpy()


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("nbnd", [1, 2, 7, 16])
def test_gamma_apply_fp64_c1(lib, nbnd):
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    half = _half_block(m, nbnd, 300 + nbnd)
    got = _apply(ctx, half)
    ref = _oracle_gamma(p, m, vr, beta, d, half)
    assert np.all(np.isfinite(got)) and _maxrel(got, ref) < 1e-12
    assert np.all(got[:, 0].imag == 0.0)
    ctx.close()


def test_gamma_apply_equals_complex_apply(lib):
    """hpsi_apply_gamma on half coefficients equals hpsi_apply on the full coefficients of the same
    real orbitals, restricted to the half sphere (float64, 1e-12)."""
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, m, vr, beta, d = _setup(p)
    half = _half_block(m, 9, 12)
    got = _apply(ctx, half)
    full = oracle.gamma.to_full(half, m)
    out = np.empty_like(full)
    B.hpsi_apply(ctx, 0, full, out)
    assert _maxrel(got, oracle.gamma.to_half(out, m)) < 1e-12
    sel = [0, 8]
    ref = _oracle_gamma(p, m, vr, beta, d, half[sel])
    assert _maxrel(got[sel], ref) < 1e-12
    ctx.close()


def test_gamma_apply_mixed_terms(lib):
    """Mixed precision: (H - T) psi on half storage matches the oracle's local + nonlocal terms
    element by element (the exact float64 kinetic term removed on both sides)."""
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, m, vr, beta, d = _setup(p, B.HPSI_MIXED)
    half = _half_block(m, 12, 4)
    got = _apply(ctx, half)
    sel = [0, 5, 11]
    ref = _oracle_gamma(p, m, vr, beta, d, half[sel])
    t = oracle.gamma.to_half(oracle.gsphere.kinetic(p.lattice, p.kpts[0], m)[None, :], m) * half[sel]
    err = _maxrel(got[sel] - t, ref - t)
    print(f"Gamma mixed (H - T) psi max-element error {err:.2e}")
    assert err < 1e-5
    ctx.close()


def _coupled_d(nat, seed, scale=0.3):
    """A dense Hermitian D that couples every projector pair and still allows the real form: real
    symmetric between projectors of the same parity under G -> -G (s with s, p with p), imaginary
    antisymmetric between s and p (whose beta(-G) = -conj(beta(G)))."""
    rng = np.random.default_rng(seed)
    P = 4 * nat
    odd = np.array([k % 4 != 0 for k in range(P)])
    a = rng.standard_normal((P, P))
    b = rng.standard_normal((P, P))
    cross = odd[:, None] != odd[None, :]
    return scale * np.where(cross, 1j * (b - b.T) / 2, (a + a.T) / 2 + 0j)


@pytest.mark.parametrize("precision", [0, 1])
def test_gamma_apply_coupled_d(lib, precision):
    """Projectors with beta(-G) = -conj(beta(G)) (p-type) coupled to s-type ones through a dense D:
    the real form rephases them, and D in the rephased basis has real off-diagonal entries.  H on
    half storage against the oracle (float64: 1e-12; mixed: (H - T) psi element by element, 1e-5)."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    d = _coupled_d(len(p.atoms), 5)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], d, precision, torch.cuda.current_stream().cuda_stream)
    half = _half_block(m, 7, 77)
    got = _apply(ctx, half)
    ref = _oracle_gamma(p, m, vr, beta, d, half)
    if precision == 0:
        err = _maxrel(got, ref)
        assert err < 1e-12
    else:
        t = oracle.gamma.to_half(oracle.gsphere.kinetic(p.lattice, k, m)[None, :], m) * half
        err = _maxrel(got - t, ref - t)
        assert err < 1e-5
    print(f"Gamma coupled D, precision {precision}: max-element error {err:.2e}")
    assert np.all(got[:, 0].imag == 0.0)
    ctx.close()


def test_gamma_davidson_coupled_d(lib):
    """Float64 Davidson on real orbitals with the coupled D reaches the eigenvalues of the complex
    form's Davidson on the same problem (1e-10 Ha)."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    d = _coupled_d(len(p.atoms), 9)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], d, B.HPSI_FP64,
                       torch.cuda.current_stream().cuda_stream)
    psi = workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed)
    xg = torch.from_numpy(np.ascontiguousarray(oracle.gamma.to_half(psi, m))).cuda()
    eg, _, _, _ = B.davidson_solve_gamma(ctx, 0, xg, 1e-9, 300)
    xc = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    ec, _, _, _ = B.davidson_solve(ctx, 0, xc, 1e-9, 300)
    assert np.max(np.abs(eg - ec)) < 1e-10
    ctx.close()


@pytest.mark.parametrize("cfg,precision,tol,bound", [("c1", 0, 1e-8, 1e-10), ("c2", 0, 1e-8, 1e-10),
                                                     ("c2", 1, 1e-5, 1e-6)])
def test_gamma_davidson(lib, cfg, precision, tol, bound):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.CONFIGS[cfg]()
    ctx, m, vr, beta, d = _setup(p, precision)
    x = torch.from_numpy(np.ascontiguousarray(
        oracle.gamma.to_half(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed), m))).cuda()
    eig, it, res, rc = B.davidson_solve_gamma(ctx, 0, x, tol, 300)
    gold = np.asarray(_golden(cfg)[:p.nbnd])
    err = float(np.max(np.abs(eig - gold)))
    print(f"{cfg} precision {precision}: {it} iterations, max eigenvalue error {err:.2e}, max residual {res.max():.2e}")
    assert err < bound and np.all(np.diff(eig) >= -1e-12)
    # the returned orbitals are orthonormal real functions: <a|b> = Re of the half-sphere form
    xh = x.cpu().numpy()
    assert np.all(xh[:, 0].imag == 0.0)
    w = np.full(xh.shape[1], 2.0)
    w[0] = 1.0
    s = np.real((xh.conj() * w[None, :]) @ xh.T)
    print(f"  orthonormality of the returned orbitals: {np.max(np.abs(s - np.eye(p.nbnd))):.2e}")
    assert np.max(np.abs(s - np.eye(p.nbnd))) < (1e-10 if precision == 0 else 1e-4)
    # and they are eigenvectors: residuals of the oracle's H on a few of them
    sel = [0, p.nbnd - 1]
    hx = _oracle_gamma(p, m, vr, beta, d, xh[sel])
    r = np.sqrt(np.real(((hx - eig[sel, None] * xh[sel]).conj() * w[None, :] * (hx - eig[sel, None] * xh[sel])).sum(1)))
    assert np.all(r < (10 * tol if precision == 0 else 1e-3))
    ctx.close()


def test_gamma_host_pointers(lib):
    """Host arrays work for both entry points (staged through the library's buffers)."""
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, m, vr, beta, d = _setup(p)
    half = _half_block(m, 5, 1)
    out = np.empty_like(half)
    B.hpsi_apply_gamma(ctx, 0, half, out)
    assert np.array_equal(out, _apply(ctx, half))
    x = np.ascontiguousarray(oracle.gamma.to_half(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed), m))
    eig, it, res, rc = B.davidson_solve_gamma(ctx, 0, x, 1e-8, 200)
    assert np.max(np.abs(eig - np.asarray(_golden("c1")[:p.nbnd]))) < 1e-10
    ctx.close()


def test_gamma_rejected_where_it_does_not_apply(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    s = torch.cuda.current_stream().cuda_stream
    p = workloads.config1()
    k = np.array([0.05, 0.0, 0.0])
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [workloads.beta(p.lattice, p.atoms, k, m)],
                       workloads.dmat(2), 0, s)
    x = np.zeros((2, (len(m) + 1) // 2), dtype=np.complex128)
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_apply_gamma(ctx, 0, x, np.zeros_like(x))
    assert e.value.status == B.HPSI_EINVAL and "k = 0" in str(e.value)
    ctx.close()
    # projectors without the beta(-G) = u conj(beta(G)) symmetry make the nonlocal term complex
    m = B.hpsi_gsphere(p.lattice, p.ecut, p.kpts[0])
    rng = np.random.default_rng(3)
    beta = rng.standard_normal((3, len(m))) + 1j * rng.standard_normal((3, len(m)))
    ctx = B.hpsi_setup(p.lattice, p.ecut, p.kpts, p.fft, vr, [beta], np.eye(3, dtype=np.complex128), 0, s)
    x = np.zeros((2, (len(m) + 1) // 2), dtype=np.complex128)
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_apply_gamma(ctx, 0, x, np.zeros_like(x))
    assert e.value.status == B.HPSI_EINVAL and "projector" in str(e.value)
    ctx.close()


def test_gamma_many_cells(lib):
    """The Gamma form on a context of independent cells (boxes 25^3..50^3): H on half storage for
    three cells against the oracle, and the Davidson eigenvalues of one cell against the golden
    dense-LAPACK values (float64)."""
    import json
    import torch
    from paper_0906_2569_gb300 import binding as B
    cells = workloads.config4b()
    ms = [B.hpsi_gsphere(c.lattice, c.ecut, c.kpts[0]) for c in cells]
    vrs = [workloads.vloc_r(c.lattice, c.atoms, c.fft) for c in cells]
    betas = [workloads.beta(c.lattice, c.atoms, c.kpts[0], m) for c, m in zip(cells, ms)]
    ds = [workloads.dmat(len(c.atoms)) for c in cells]
    ctx = B.hpsi_setup_cells([c.lattice for c in cells], [c.ecut for c in cells], [c.fft for c in cells], vrs,
                             betas, ds, B.HPSI_FP64, torch.cuda.current_stream().cuda_stream)
    for i in (0, 17, 31):
        c = cells[i]
        half = _half_block(ms[i], 5, 60 + i)
        x = torch.from_numpy(half).cuda()
        y = torch.full_like(x, float("nan"))
        B.hpsi_apply_gamma(ctx, i, x, y)
        B.hpsi_sync(ctx)
        full = oracle.gamma.to_full(half, ms[i])
        ref = oracle.gamma.to_half(oracle.hamiltonian.hpsi(c.lattice, c.kpts[0], ms[i], c.fft, vrs[i], betas[i], ds[i],
                                                           full), ms[i])
        assert _maxrel(y.cpu().numpy(), ref) < 1e-12
    i = 5
    c = cells[i]
    x = torch.from_numpy(np.ascontiguousarray(
        oracle.gamma.to_half(workloads.psi0(c.lattice, c.kpts[0], ms[i], c.nbnd, c.psi_seed), ms[i]))).cuda()
    eig, it, res, rc = B.davidson_solve_gamma(ctx, i, x, 1e-8, 300)
    gold = np.asarray(json.load(open(os.path.join(HERE, "golden", "eigenvalues.json")))["c4b"]["eigenvalues"][i])
    assert np.max(np.abs(eig - gold[:c.nbnd])) < 1e-10
    ctx.close()


@pytest.mark.parametrize("final", [1, 2])
def test_gamma_davidson_final_quotients(lib, final):
    """HPSI_OPT_FINAL_FP64 = 1 (float64 H) and 2 (float64 projections and D, the rest at the working
    precision; the default): eigenvalues of the mixed solve within 1e-6 Ha of the golden values."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, m, vr, beta, d = _setup(p, B.HPSI_MIXED)
    B.hpsi_set_option(ctx, B.HPSI_OPT_FINAL_FP64, final)
    x = torch.from_numpy(np.ascontiguousarray(
        oracle.gamma.to_half(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed), m))).cuda()
    eig, it, res, rc = B.davidson_solve_gamma(ctx, 0, x, 1e-5, 300)
    err = float(np.max(np.abs(eig - np.asarray(_golden("c2")[:p.nbnd]))))
    print(f"c2 Gamma mixed, final quotients mode {final}: {it} iterations, max eigenvalue error {err:.2e}")
    assert err < 1e-6
    ctx.close()
