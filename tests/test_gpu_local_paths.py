"""GPU parity of the two local-potential paths (register-codelet kernels for cubic boxes, generic
radix kernels otherwise) against the oracle, over the cubic box edges of the workloads."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _apply(ctx, psi, generic):
    import torch
    from paper_0906_2569_gb300 import binding as B
    B.hpsi_set_option(ctx, B.HPSI_OPT_LOCAL_PATH, 1 if generic else 0)
    x = torch.from_numpy(psi).cuda()
    y = torch.full_like(x, float("nan"))
    B.hpsi_apply(ctx, 0, x, y)
    B.hpsi_sync(ctx)
    return y.cpu().numpy()


@pytest.mark.parametrize("a,fft", [(8.0, 25), (9.0, 27), (9.3, 30), (10.0, 36), (11.0, 40), (12.5, 45), (13.0, 48),
                                   (14.0, 50)])
@pytest.mark.parametrize("precision", [0, 1])
def test_cubic_boxes_both_paths(lib, a, fft, precision):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.small_cell(ecut=15.0 if fft >= 30 else 12.0, a=a, nat=2, fft=(fft, fft, fft), seed=int(a * 10))
    k = np.array([0.02, -0.03, 0.01])
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    d = workloads.dmat(len(p.atoms))
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], d, precision,
                       torch.cuda.current_stream().cuda_stream)
    psi = workloads.random_block(len(m), 21, fft)
    ref = oracle.hamiltonian.hpsi(p.lattice, k, m, p.fft, vr, beta, d, psi)
    tol = 1e-12 if precision == 0 else 1e-5
    for generic in (False, True):
        got = _apply(ctx, psi, generic)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < tol, f"box {fft} precision {precision} generic={generic}: {err:.3e}"
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuner_does_not_change_results(lib, precision):
    """The plan the autotuner picks (staging, band block) leaves H|psi> bit-identical."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config2()
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    x = torch.from_numpy(workloads.psi0(p.lattice, k, m, 40, p.psi_seed)).cuda()
    outs = []
    for tune in (0, 1):
        ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], workloads.dmat(len(p.atoms)), precision,
                           torch.cuda.current_stream().cuda_stream)
        B.hpsi_set_option(ctx, B.HPSI_OPT_AUTOTUNE, tune)
        y = torch.empty_like(x)
        B.hpsi_apply(ctx, 0, x, y)
        B.hpsi_apply(ctx, 0, x, y)
        B.hpsi_sync(ctx)
        outs.append(y.cpu().numpy())
        ctx.close()
    assert np.array_equal(outs[0], outs[1])
