"""GPU parity: libhpsi's H|psi> (through the C ABI) against the CPU oracle, element by element.

Tolerances: float64 path 1e-12 relative (Frobenius over the block) and 1e-12 max-element relative to
the block's largest entry; mixed path 1e-5 relative.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-5


def _torch():
    import torch
    return torch


def make_problem(p, ik=0, nbnd=None, seed=None, precision=0, lib=None, kpts=None):
    from paper_0906_2569_gb300 import binding as B
    torch = _torch()
    kpts = p.kpts if kpts is None else kpts
    millers = [B.hpsi_gsphere(p.lattice, p.ecut, k) for k in kpts]
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    betas = [workloads.beta(p.lattice, p.atoms, k, m) for k, m in zip(kpts, millers)]
    d = workloads.dmat(len(p.atoms))
    ctx = B.hpsi_setup(p.lattice, p.ecut, kpts, p.fft, vr, betas, d, precision,
                       torch.cuda.current_stream().cuda_stream)
    return ctx, millers, vr, betas, d


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def run_apply(ctx, ik, psi):
    from paper_0906_2569_gb300 import binding as B
    torch = _torch()
    x = torch.from_numpy(psi).cuda()
    y = torch.full_like(x, float("nan"))
    B.hpsi_apply(ctx, ik, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("nbnd", [1, 5, 16, 37])
def test_hpsi_fp64_c1(lib, nbnd):
    p = workloads.config1()
    ctx, (m,), vr, (beta,), d = make_problem(p)
    psi = workloads.random_block(len(m), nbnd, 100 + nbnd)
    got = run_apply(ctx, 0, psi)
    ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, psi)
    assert rel(got, ref) < TOL64 and maxrel(got, ref) < TOL64


def test_free_electron_is_kinetic(lib):
    """V = 0 and no projectors: H psi = |k+G|^2/2 psi (the transforms of zero are zero)."""
    from paper_0906_2569_gb300 import binding as B
    torch = _torch()
    p = workloads.config1()
    k = np.array([0.03, -0.02, 0.05])
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, np.zeros(p.fft), None, None, B.HPSI_FP64,
                       torch.cuda.current_stream().cuda_stream)
    psi = workloads.random_block(len(m), 7, 3)
    got = run_apply(ctx, 0, psi)
    t = oracle.gsphere.kinetic(p.lattice, k, m)
    assert maxrel(got, t[None, :] * psi) < 1e-15


def test_hpsi_fp64_oblique_cell_full_d(lib):
    """fcc cell, k != 0, non-cubic box (27 x 30 x 32), full Hermitian D, ragged band count."""
    from paper_0906_2569_gb300 import binding as B
    torch = _torch()
    lat = 0.5 * 9.0 * np.array([[0.0, 1, 1], [1, 0, 1], [1, 1, 0]])
    rng = np.random.default_rng(5)
    atoms = rng.random((3, 3)) @ lat
    k = np.array([0.13, -0.21, 0.07])
    fft = (27, 30, 32)
    m = B.hpsi_gsphere(lat, 6.0, k)
    vr = workloads.vloc_r(lat, atoms, fft)
    beta = workloads.beta(lat, atoms, k, m)
    a = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    d = 0.25 * (a + a.conj().T)
    ctx = B.hpsi_setup(lat, 6.0, [k], fft, vr, [beta], d, B.HPSI_FP64, torch.cuda.current_stream().cuda_stream)
    psi = workloads.random_block(len(m), 13, 8)
    got = run_apply(ctx, 0, psi)
    ref = oracle.hamiltonian.hpsi(lat, k, m, fft, vr, beta, d, psi)
    assert rel(got, ref) < TOL64 and maxrel(got, ref) < TOL64


def test_hpsi_fp64_kpoints(lib):
    p = workloads.config4a()
    kp = p.kpts[:3]
    ctx, ms, vr, betas, d = make_problem(p, kpts=kp)
    assert ctx.nprob() == 3
    for ik in range(3):
        psi = workloads.random_block(len(ms[ik]), 6, 40 + ik)
        got = run_apply(ctx, ik, psi)
        ref = oracle.hamiltonian.hpsi(p.lattice, kp[ik], ms[ik], p.fft, vr, betas[ik], d, psi)
        assert rel(got, ref) < TOL64


def test_hpsi_host_pointers_match_device(lib):
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, (m,), vr, (beta,), d = make_problem(p)
    psi = workloads.random_block(len(m), 9, 11)
    dev = run_apply(ctx, 0, psi)
    out = np.empty_like(psi)
    B.hpsi_apply(ctx, 0, psi, out)
    assert np.array_equal(out, dev)


def test_hpsi_errors(lib):
    from paper_0906_2569_gb300 import binding as B
    torch = _torch()
    p = workloads.config1()
    ctx, (m,), vr, (beta,), d = make_problem(p)
    x = torch.zeros((2, len(m)), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_apply(ctx, 1, x, torch.empty_like(x))
    assert e.value.status == B.HPSI_EINVAL
    with pytest.raises(B.HpsiError):
        B.hpsi_apply(ctx, 0, x, x)                  # aliasing
    with pytest.raises(B.HpsiError):
        B.hpsi_apply(ctx, 0, x, np.zeros((2, len(m)), dtype=np.complex128))   # host / device mix
    B.hpsi_apply(ctx, 0, x, torch.empty_like(x), 0)  # nbnd = 0 is a no-op
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_setup(p.lattice, p.ecut, p.kpts, (12, 12, 12), vr[:12, :12, :12], [beta], d)
    assert e.value.status == B.HPSI_EINVAL       # box too small for the sphere
    with pytest.raises(B.HpsiError):
        B.hpsi_setup(p.lattice, p.ecut, p.kpts, (33, 33, 33), np.zeros((33, 33, 33)), [beta], d)   # 33 = 3 * 11
    bad = d.copy()
    bad[0, 1] = 0.3j
    with pytest.raises(B.HpsiError):
        B.hpsi_setup(p.lattice, p.ecut, p.kpts, p.fft, vr, [beta], bad)      # D not Hermitian


def test_hpsi_fp64_c2_sampled(lib):
    """The 90^3 / 36785-PW / 256-projector cell, 160 bands in one call; 4 bands checked by the oracle."""
    p = workloads.config2()
    ctx, (m,), vr, (beta,), d = make_problem(p)
    psi = workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)
    got = run_apply(ctx, 0, psi)
    sel = [0, 57, 101, 159]
    ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, psi[sel])
    assert rel(got[sel], ref) < TOL64 and maxrel(got[sel], ref) < TOL64


def test_hpsi_mixed_c1(lib):
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config3(160)
    ctx, (m,), vr, (beta,), d = make_problem(p, precision=B.HPSI_MIXED)
    psi = workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)
    got = run_apply(ctx, 0, psi)
    ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, psi)
    assert rel(got, ref) < TOLMIX


def test_hpsi_mixed_c2_sampled(lib):
    """Mixed path on the 36785-PW / 256-projector cell: 160 bands, 4 checked by the oracle."""
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    ctx, (m,), vr, (beta,), d = make_problem(p, precision=B.HPSI_MIXED)
    psi = workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)
    got = run_apply(ctx, 0, psi)
    B.hpsi_sync(ctx)
    sel = [0, 63, 128, 159]
    ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, psi[sel])
    assert rel(got[sel], ref) < TOLMIX


@pytest.mark.parametrize("nbnd", [3, 130])
def test_hpsi_mixed_three_terms(lib, nbnd):
    """Six-product split (three bf16 terms per operand, the default) is at least as accurate as three."""
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, (m,), vr, (beta,), d = make_problem(p, precision=B.HPSI_MIXED)
    psi = workloads.random_block(len(m), nbnd, 7)
    ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, psi)
    e3 = rel(run_apply(ctx, 0, psi), ref)
    B.hpsi_set_option(ctx, B.HPSI_OPT_NL_TERMS, 2)
    e2 = rel(run_apply(ctx, 0, psi), ref)
    B.hpsi_sync(ctx)
    assert e2 < TOLMIX and e3 < TOLMIX and e3 <= e2 * 1.5


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOLMIX)])
def test_hpsi_c5_sampled(lib, precision, tol):
    """The large cell: 144^3 box, 161235 PWs, 864 projectors; 96 bands applied, 3 checked by the oracle."""
    p = workloads.config5()
    ctx, (m,), vr, (beta,), d = make_problem(p, precision=precision)
    assert len(m) == 161235
    psi = workloads.psi0(p.lattice, p.kpts[0], m, 96, p.psi_seed)
    got = run_apply(ctx, 0, psi)
    sel = [0, 47, 95]
    ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, psi[sel])
    assert rel(got[sel], ref) < tol
    ctx.close()


def test_bounded_wait_reports_timeout(lib):
    """A device wait that nothing satisfies expires, sets the error word, and the host sees
    HPSI_ETIMEOUT; the context keeps working afterwards (nothing faults or hangs)."""
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    ctx, (m,), vr, (beta,), d = make_problem(p, precision=B.HPSI_MIXED)
    B.hpsi_sync(ctx)
    B.hpsi_selftest_timeout(ctx)
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_sync(ctx)
    assert e.value.status == B.HPSI_ETIMEOUT
    B.hpsi_sync(ctx)                               # the word was cleared
    psi = workloads.random_block(len(m), 4, 1)
    ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, psi)
    assert rel(run_apply(ctx, 0, psi), ref) < TOLMIX
