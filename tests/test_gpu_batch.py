"""Batched H|psi>: many k-points (one cell) and many independent cells in one launch sequence,
captured in a CUDA graph on the first call and replayed on identical calls."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _run_batch(ctx, xs):
    import torch
    from paper_0906_2569_gb300 import binding as B
    ys = [torch.full_like(x, float("nan")) for x in xs]
    B.hpsi_apply_batch(ctx, list(range(len(xs))), xs, ys)
    B.hpsi_sync(ctx)
    return [y.cpu().numpy() for y in ys]


def _run_each(ctx, xs):
    import torch
    from paper_0906_2569_gb300 import binding as B
    out = []
    for i, x in enumerate(xs):
        y = torch.full_like(x, float("nan"))
        B.hpsi_apply(ctx, i, x, y)
        out.append(y)
    B.hpsi_sync(ctx)
    return [y.cpu().numpy() for y in out]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_kpoints(lib, precision):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config4a()
    ms = [B.hpsi_gsphere(p.lattice, p.ecut, k) for k in p.kpts]
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    betas = [workloads.beta(p.lattice, p.atoms, k, m) for k, m in zip(p.kpts, ms)]
    d = workloads.dmat(len(p.atoms))
    ctx = B.hpsi_setup(p.lattice, p.ecut, p.kpts, p.fft, vr, betas, d, precision,
                       torch.cuda.current_stream().cuda_stream)
    xs = [torch.from_numpy(workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed + i)).cuda()
          for i, (k, m) in enumerate(zip(p.kpts, ms))]
    each = _run_each(ctx, xs)
    B.hpsi_set_option(ctx, B.HPSI_OPT_BATCH_NL, 1)   # mixed: the per-item tensor-core nonlocal form
    first = _run_batch(ctx, xs)      # eager + capture
    second = _run_batch(ctx, xs)     # graph replay
    for i in range(len(xs)):
        assert np.array_equal(first[i], each[i]) and np.array_equal(second[i], each[i])
    B.hpsi_set_option(ctx, B.HPSI_OPT_BATCH_NL, 0)
    B.hpsi_kernel_stats(ctx, -1, reset=True)
    third = _run_batch(ctx, xs)      # mixed: the float64 nonlocal term over the batch (8 projectors each)
    assert B.hpsi_kernel_stats(ctx, B.KERNELS.index("calbec") + B.HPSI_K_AT_FP64)[0] == 1
    tol = 1e-12 if precision == 0 else 1e-5
    for i in (0, 7, 15):
        ref = oracle.hamiltonian.hpsi(p.lattice, p.kpts[i], ms[i], p.fft, vr, betas[i], d, xs[i].cpu().numpy())
        for y in (first, third):
            assert np.linalg.norm(y[i] - ref) / np.linalg.norm(ref) < tol
    n, _ = B.hpsi_kernel_stats(ctx, -2)
    assert n == 4 * 16 * p.nbnd   # the per-item pass and three batches


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_cells(lib, precision):
    """32 cubic cells with 25^3 ... 50^3 boxes, 1-4 atoms, 8-32 bands, in float64 and mixed
    precision, against the oracle."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    cells = workloads.config4b()
    ms = [B.hpsi_gsphere(c.lattice, c.ecut, c.kpts[0]) for c in cells]
    vrs = [workloads.vloc_r(c.lattice, c.atoms, c.fft) for c in cells]
    betas = [workloads.beta(c.lattice, c.atoms, c.kpts[0], m) for c, m in zip(cells, ms)]
    ds = [workloads.dmat(len(c.atoms)) for c in cells]
    ctx = B.hpsi_setup_cells([c.lattice for c in cells], [c.ecut for c in cells], [c.fft for c in cells], vrs,
                             betas, ds, precision, torch.cuda.current_stream().cuda_stream)
    assert ctx.nprob() == 32
    xs = [torch.from_numpy(workloads.psi0(c.lattice, c.kpts[0], m, c.nbnd, c.psi_seed)).cuda()
          for c, m in zip(cells, ms)]
    each = _run_each(ctx, xs)
    B.hpsi_set_option(ctx, B.HPSI_OPT_BATCH_NL, 1)   # mixed: the per-item tensor-core nonlocal form
    first = _run_batch(ctx, xs)
    second = _run_batch(ctx, xs)
    for i in range(32):
        assert np.array_equal(first[i], each[i]) and np.array_equal(second[i], each[i])
    B.hpsi_set_option(ctx, B.HPSI_OPT_BATCH_NL, 0)
    third = _run_batch(ctx, xs)      # mixed: the float64 nonlocal term over the batch
    for i in (0, 5, 17, 31):
        c = cells[i]
        ref = oracle.hamiltonian.hpsi(c.lattice, c.kpts[0], ms[i], c.fft, vrs[i], betas[i], ds[i], xs[i].cpu().numpy())
        for y in (first, third):
            assert np.linalg.norm(y[i] - ref) / np.linalg.norm(ref) < (1e-12 if precision == 0 else 1e-5)


def test_batch_graph_invalidated_by_new_arguments(lib):
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config4a()
    kp = p.kpts[:3]
    ms = [B.hpsi_gsphere(p.lattice, p.ecut, k) for k in kp]
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    betas = [workloads.beta(p.lattice, p.atoms, k, m) for k, m in zip(kp, ms)]
    ctx = B.hpsi_setup(p.lattice, p.ecut, kp, p.fft, vr, betas, workloads.dmat(2), B.HPSI_FP64,
                       torch.cuda.current_stream().cuda_stream)
    xs = [torch.from_numpy(workloads.random_block(len(m), 5, i)).cuda() for i, m in enumerate(ms)]
    a = _run_batch(ctx, xs)
    xs2 = [x[:3].clone() for x in xs]          # new pointers and band counts
    b = _run_batch(ctx, xs2)
    c = _run_batch(ctx, xs)                    # back to the first list
    each = _run_each(ctx, xs)
    for i in range(3):
        assert np.array_equal(a[i], each[i]) and np.array_equal(c[i], each[i])
        assert np.array_equal(b[i], each[i][:3])


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_persistent_launch(lib, precision):
    """The 16 k-points of the fcc cell in one persistent launch (HPSI_OPT_PERSISTENT = 1): the same
    results, bit for bit, as one launch per kernel class, with a single launch of the batch class
    and none of the separate FFT kernels (float64: none of the nonlocal ones either)."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.config4a()
    ms = [B.hpsi_gsphere(p.lattice, p.ecut, k) for k in p.kpts]
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    betas = [workloads.beta(p.lattice, p.atoms, k, m) for k, m in zip(p.kpts, ms)]
    ctx = B.hpsi_setup(p.lattice, p.ecut, p.kpts, p.fft, vr, betas, workloads.dmat(len(p.atoms)), precision,
                       torch.cuda.current_stream().cuda_stream)
    xs = [torch.from_numpy(workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed + i)).cuda()
          for i, (k, m) in enumerate(zip(p.kpts, ms))]
    _run_each(ctx, xs)   # the autotuner settles the plans first
    B.hpsi_set_option(ctx, B.HPSI_OPT_PERSISTENT, 1)
    B.hpsi_kernel_stats(ctx, -1, reset=True)
    per = _run_batch(ctx, xs)
    k = {name: B.hpsi_kernel_stats(ctx, i)[0] for i, name in enumerate(B.KERNELS)}
    assert k["batch"] == 1 and k["inv_zy"] == 0 and k["xvx_y"] == 0 and k["fwd_z"] == 0
    assert k["calbec"] == 0 and k["addvus"] == 0   # mixed too: 8 projectors, the float64 batched form
    B.hpsi_set_option(ctx, B.HPSI_OPT_PERSISTENT, 0)
    B.hpsi_kernel_stats(ctx, -1, reset=True)
    sep = _run_batch(ctx, xs)
    assert B.hpsi_kernel_stats(ctx, B.KERNELS.index("batch"))[0] == 0
    for i in range(len(xs)):
        assert np.array_equal(per[i], sep[i])
    ctx.close()


def test_batch_persistent_per_box_edge(lib):
    """32 cells with nine box edges: one persistent launch per edge, the same results as one launch
    per kernel class (float64)."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    cells = workloads.config4b()
    ms = [B.hpsi_gsphere(c.lattice, c.ecut, c.kpts[0]) for c in cells]
    vrs = [workloads.vloc_r(c.lattice, c.atoms, c.fft) for c in cells]
    betas = [workloads.beta(c.lattice, c.atoms, c.kpts[0], m) for c, m in zip(cells, ms)]
    ds = [workloads.dmat(len(c.atoms)) for c in cells]
    ctx = B.hpsi_setup_cells([c.lattice for c in cells], [c.ecut for c in cells], [c.fft for c in cells], vrs,
                             betas, ds, B.HPSI_FP64, torch.cuda.current_stream().cuda_stream)
    xs = [torch.from_numpy(workloads.psi0(c.lattice, c.kpts[0], m, c.nbnd, c.psi_seed)).cuda()
          for c, m in zip(cells, ms)]
    _run_each(ctx, xs)
    B.hpsi_set_option(ctx, B.HPSI_OPT_PERSISTENT, 1)
    B.hpsi_kernel_stats(ctx, -1, reset=True)
    per = _run_batch(ctx, xs)
    edges = len({tuple(c.fft) for c in cells})
    assert B.hpsi_kernel_stats(ctx, B.KERNELS.index("batch"))[0] == edges
    B.hpsi_set_option(ctx, B.HPSI_OPT_PERSISTENT, 0)
    sep = _run_batch(ctx, xs)
    for i in range(len(xs)):
        assert np.array_equal(per[i], sep[i])
    ctx.close()
