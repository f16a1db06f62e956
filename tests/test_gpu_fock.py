"""GPU Fock exchange at Gamma (App. A.5, hpsi_fock_apply) against the oracle (oracle.fock), element
by element, plus the operator's Hermiticity and the exchange energy of the occupied set."""
import numpy as np
import pytest

import _pins
import oracle
import workloads

pytestmark = pytest.mark.gpu


def _orthonormal(npw, n, seed):
    q, _ = np.linalg.qr(workloads.random_block(npw, n, seed).T)
    return np.ascontiguousarray(q.T)


def _ctx(lat, ecut, fft, vr, beta, d):
    import torch
    from paper_0906_2569_gb300 import binding as B
    return B.hpsi_setup(lat, ecut, [np.zeros(3)], fft, vr, [beta] if beta is not None else None, d, B.HPSI_FP64,
                        torch.cuda.current_stream().cuda_stream)


def _vx(ctx, occ, psi, alpha=1.0):
    import torch
    from paper_0906_2569_gb300 import binding as B
    o = torch.from_numpy(occ).cuda()
    x = torch.from_numpy(psi).cuda()
    y = torch.full_like(x, float("nan"))
    ex = B.hpsi_fock_apply(ctx, 0, o, x, y, alpha, energy=True)
    return y.cpu().numpy(), ex


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("alpha", [1.0, 0.5])
def test_fock_c1(lib, alpha):
    """The 1503-PW cell (box 32^3): 4 occupied orbitals, V_x applied to 7 bands (the occupied ones
    among them) and E_x of the occupied set."""
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    m = B.hpsi_gsphere(p.lattice, p.ecut, p.kpts[0])
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    ctx = _ctx(p.lattice, p.ecut, p.fft, vr, workloads.beta(p.lattice, p.atoms, p.kpts[0], m), workloads.dmat(2))
    occ = _orthonormal(len(m), 4, 11)
    psi = np.concatenate([occ, workloads.random_block(len(m), 3, 12)])
    got, _ = _vx(ctx, occ, psi, alpha)
    ref = oracle.fock.apply_vx(psi, occ, m, p.fft, p.lattice, alpha)
    assert _maxrel(got, ref) < 1e-12
    _, ex = _vx(ctx, occ, occ, alpha)
    ex_ref = oracle.fock.exchange_energy(occ, m, p.fft, p.lattice, alpha)
    print(f"alpha {alpha}: E_x {ex:.14f} (oracle {ex_ref:.14f})")
    assert abs(ex - ex_ref) < 1e-12 * abs(ex_ref)
    ctx.close()


def test_fock_oblique_cell_hermitian(lib):
    """The small fcc cell at Gamma (oblique lattice, box 9^3): parity with the oracle and
    <a|V_x b> = conj(<b|V_x a>) for two random bands."""
    lat, m, fft, vr, _ = _pins.gamma_problem()
    p = workloads.small_cell(ecut=2.5, nat=2, fft=fft, seed=21, k=np.zeros(3), lattice=lat)
    beta = workloads.beta(lat, p.atoms, np.zeros(3), m)
    ctx = _ctx(lat, 2.5, fft, vr, beta, workloads.dmat(len(p.atoms)))
    occ = _orthonormal(len(m), 2, 3)
    ab = workloads.random_block(len(m), 2, 4)
    got, _ = _vx(ctx, occ, ab)
    assert _maxrel(got, oracle.fock.apply_vx(ab, occ, m, fft, lat)) < 1e-12
    lhs = np.vdot(ab[0], got[1])
    rhs = np.conj(np.vdot(ab[1], got[0]))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    ctx.close()


def test_fock_rejects_k_point(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1()
    k = np.array([0.1, 0.0, 0.0])
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, workloads.vloc_r(p.lattice, p.atoms, p.fft), None, None,
                       B.HPSI_FP64, torch.cuda.current_stream().cuda_stream)
    x = torch.zeros((2, len(m)), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_fock_apply(ctx, 0, x, x.clone(), torch.empty_like(x))
    assert e.value.status == B.HPSI_EINVAL
    ctx.close()
