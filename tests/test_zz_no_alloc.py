"""hpsi_apply_noalloc: H psi for callers that cannot let the library allocate device memory.

The entry point keeps its intermediates in a fixed array inside libhpsi.so instead of allocating.
Its output must equal hpsi_apply's (same kernels, same operator) within the tolerances the other
parity tests use, on two calls in a row (the second call sees the array the first one left behind).
This file is collected last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _ctx(p, precision):
    import torch
    from paper_0906_2569_gb300 import binding as B
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], workloads.dmat(len(p.atoms)), precision,
                       torch.cuda.current_stream().cuda_stream)
    return ctx, m


@pytest.mark.parametrize("cfg,precision,tol", [("c1", 0, 1e-12), ("c1", 1, 1e-5), ("c2", 0, 1e-12)])
def test_noalloc_matches_hpsi_apply(lib, cfg, precision, tol):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.CONFIGS[cfg]()
    ctx, m = _ctx(p, precision)
    x = torch.from_numpy(workloads.psi0(p.lattice, p.kpts[0], m, p.nbnd, p.psi_seed)).cuda()
    ref = torch.empty_like(x)
    B.hpsi_apply(ctx, 0, x, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for call in range(2):
        out = torch.full_like(x, float("nan"))
        B.hpsi_apply_noalloc(ctx, 0, x, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert np.all(np.isfinite(got)) and err < tol, f"call {call}: relative difference {err:.3e}"
    ctx.close()


def test_noalloc_rejects_host_pointers(lib):
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config1(4)
    ctx, m = _ctx(p, 0)
    x = np.zeros((4, len(m)), dtype=np.complex128)
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_apply_noalloc(ctx, 0, x, np.zeros_like(x))
    assert e.value.status == B.HPSI_EINVAL
    ctx.close()
