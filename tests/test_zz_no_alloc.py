"""hpsi_apply_noalloc: H psi for callers that cannot let the library allocate device memory.

The entry point keeps its intermediates in a fixed array inside libhpsi.so instead of allocating.
Its output must equal hpsi_apply's (same operator) within the tolerances the other parity tests
use, on two calls in a row (the second call sees the array the first one left behind), and the
oracle's.  One case has many projectors and a band count that leaves a short last chunk: the
nonlocal partial sums of that chunk are planned against the room the full chunk leaves, so they
stay inside the array.  This file is collected last so that a run stopping at the first failure
has run everything else.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _ctx(p, precision, beta=None, dmat=None):
    import torch
    from paper_0906_2569_gb300 import binding as B
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    if beta is None:
        beta = workloads.beta(p.lattice, p.atoms, k, m)
        dmat = workloads.dmat(len(p.atoms))
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], dmat, precision,
                       torch.cuda.current_stream().cuda_stream)
    return ctx, m, vr, beta, dmat


def _check_two_calls(ctx, x, ref, tol):
    import torch
    from paper_0906_2569_gb300 import binding as B
    for call in range(2):
        out = torch.full_like(x, float("nan"))
        B.hpsi_apply_noalloc(ctx, 0, x, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert np.all(np.isfinite(got)) and err < tol, f"call {call}: relative difference {err:.3e}"


@pytest.mark.parametrize("cfg,precision,tol", [("c1", 0, 1e-12), ("c1", 1, 1e-5), ("c2", 0, 1e-12)])
def test_noalloc_matches_hpsi_apply(lib, cfg, precision, tol):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.CONFIGS[cfg]()
    ctx, m, vr, beta, d = _ctx(p, precision)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    ref = torch.empty_like(x)
    B.hpsi_apply(ctx, 0, x, ref)
    torch.cuda.synchronize()
    _check_two_calls(ctx, x, ref.cpu().numpy(), tol)
    if cfg == "c1":
        want = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, d, x.cpu().numpy())
        _check_two_calls(ctx, x, want, tol)
    ctx.close()


def test_noalloc_short_last_chunk(lib):
    """512 random projectors on the 1503-PW cell, 308 bands in float64: the bands run as a chunk of
    180 and a last chunk of 128 whose calbec split, planned on its own, would need more room than
    the full chunk leaves.  The result must match hpsi_apply and the oracle."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1(308)
    m = oracle.gsphere.gsphere(p.lattice, p.ecut, p.kpts[0])
    rng = np.random.default_rng(77)
    nproj = 512
    beta = rng.standard_normal((nproj, len(m))) + 1j * rng.standard_normal((nproj, len(m)))
    beta /= np.linalg.norm(beta, axis=1, keepdims=True)
    dmat = np.diag(rng.uniform(-1.0, 1.0, nproj)).astype(np.complex128)
    ctx, m2, vr, beta, dmat = _ctx(p, 0, beta, dmat)
    assert np.array_equal(m, m2)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    ref = torch.empty_like(x)
    B.hpsi_apply(ctx, 0, x, ref)
    torch.cuda.synchronize()
    _check_two_calls(ctx, x, ref.cpu().numpy(), 1e-12)
    want = oracle.hamiltonian.hpsi(p.lattice, p.kpts[0], m, p.fft, vr, beta, dmat, x.cpu().numpy())
    _check_two_calls(ctx, x, want, 1e-12)
    ctx.close()


def test_noalloc_rejects_host_pointers(lib):
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1(4)
    ctx, m, _, _, _ = _ctx(p, 0)
    x = np.zeros((4, len(m)), dtype=np.complex128)
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_apply_noalloc(ctx, 0, x, np.zeros_like(x))
    assert e.value.status == B.HPSI_EINVAL
    ctx.close()
