"""Mixed-precision H|psi> term by term, element by element, against the oracle.

The kinetic term |k+G|^2/2 psi is added in float64 on the GPU, so a comparison of the whole H|psi>
dilutes the error of the float32 transforms and of the split-bf16 contractions by the size of
T psi.  Here each term is isolated and compared on its own:

* local term: a context without projectors returns T psi + V psi; T psi (float64, exact on both
  sides) is subtracted and the rest is compared with ``oracle.hamiltonian.local_term``;
* nonlocal term: a context with V = 0 returns T psi + sum beta D <beta|psi> (the transforms of zero
  are exactly zero); T psi is subtracted and the rest is compared with
  ``oracle.hamiltonian.nonlocal_term``.

Bound, per block: max over elements |got - ref| / max over elements |ref| < TOL_TERM.  With the
eigenvalue error bounded by ||H_mixed - H||_2 (Weyl), these per-term errors times the size of each
term bound the eigenvalue error of the mixed operator before the float64 Rayleigh quotients.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL_TERM = 1e-5


def _apply(ctx, psi):
    import torch
    from paper_0906_2569_gb300 import binding as B
    x = torch.from_numpy(psi).cuda()
    y = torch.full_like(x, float("nan"))
    B.hpsi_apply(ctx, 0, x, y)
    B.hpsi_sync(ctx)
    return y.cpu().numpy()


def _maxrel(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def _terms(cfg, nbnd, sel):
    """(local error, nonlocal error) of the mixed path on config cfg, nbnd bands applied, bands sel
    checked against the oracle."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    p = workloads.CONFIGS[cfg]()
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    d = workloads.dmat(len(p.atoms))
    psi = workloads.psi0(p.lattice, k, m, nbnd, p.psi_seed)
    t = oracle.gsphere.kinetic(p.lattice, k, m)[None, :] * psi[sel]
    s = torch.cuda.current_stream().cuda_stream
    loc = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, None, None, B.HPSI_MIXED, s)
    got_loc = _apply(loc, psi)[sel] - t
    loc.close()
    nl = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, np.zeros(p.fft), [beta], d, B.HPSI_MIXED, s)
    got_nl = _apply(nl, psi)[sel] - t
    nl.close()
    ref_loc = oracle.hamiltonian.local_term(vr, m, p.fft, psi[sel])
    ref_nl = oracle.hamiltonian.nonlocal_term(beta, d, psi[sel])
    return _maxrel(got_loc, ref_loc), _maxrel(got_nl, ref_nl)


@pytest.mark.parametrize("cfg,nbnd,sel", [("c1", 160, slice(None)), ("c2", 160, [0, 63, 128, 159]),
                                          ("c5", 96, [0, 95])])
def test_mixed_terms(lib, cfg, nbnd, sel):
    e_loc, e_nl = _terms(cfg, nbnd, sel)
    print(f"{cfg}: local term max-element error {e_loc:.2e}, nonlocal term {e_nl:.2e}")
    assert e_loc < TOL_TERM and e_nl < TOL_TERM


@pytest.mark.parametrize("batch_nl", [1, 0])
def test_mixed_batch_cells(lib, batch_nl):
    """The 32 independent cells at mixed precision through hpsi_apply_batch, with the per-item
    tensor-core nonlocal term (HPSI_OPT_BATCH_NL = 1: every item equals its own hpsi_apply) and with
    the default float64 nonlocal term over the batch (these cells have 4-16 projectors); on four
    cells (H - T) psi matches the oracle's local + nonlocal terms element by element."""
    import torch
    from paper_0906_2569_gb300 import binding as B
    cells = workloads.config4b()
    ms = [B.hpsi_gsphere(c.lattice, c.ecut, c.kpts[0]) for c in cells]
    vrs = [workloads.vloc_r(c.lattice, c.atoms, c.fft) for c in cells]
    betas = [workloads.beta(c.lattice, c.atoms, c.kpts[0], m) for c, m in zip(cells, ms)]
    ds = [workloads.dmat(len(c.atoms)) for c in cells]
    ctx = B.hpsi_setup_cells([c.lattice for c in cells], [c.ecut for c in cells], [c.fft for c in cells], vrs,
                             betas, ds, B.HPSI_MIXED, torch.cuda.current_stream().cuda_stream)
    xs = [torch.from_numpy(workloads.psi0(c.lattice, c.kpts[0], m, c.nbnd, c.psi_seed)).cuda()
          for c, m in zip(cells, ms)]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    B.hpsi_set_option(ctx, B.HPSI_OPT_BATCH_NL, batch_nl)
    B.hpsi_kernel_stats(ctx, -1, reset=True)
    B.hpsi_apply_batch(ctx, list(range(32)), xs, ys)
    B.hpsi_sync(ctx)
    nl64 = B.hpsi_kernel_stats(ctx, B.KERNELS.index("calbec") + B.HPSI_K_AT_FP64)[0]
    assert nl64 == (1 if batch_nl == 0 else 0)
    for i, x in enumerate(xs):
        y = torch.full_like(x, float("nan"))
        B.hpsi_apply(ctx, i, x, y)
        B.hpsi_sync(ctx)
        if batch_nl == 1:
            assert torch.equal(y, ys[i])
    for i in (0, 5, 17, 31):
        c = cells[i]
        psi = xs[i].cpu().numpy()
        t = oracle.gsphere.kinetic(c.lattice, c.kpts[0], ms[i])[None, :] * psi
        got = ys[i].cpu().numpy() - t
        ref = (oracle.hamiltonian.local_term(vrs[i], ms[i], c.fft, psi)
               + oracle.hamiltonian.nonlocal_term(betas[i], ds[i], psi))
        err = _maxrel(got, ref)
        print(f"cell {i}: (H - T) psi max-element error {err:.2e}")
        assert err < TOL_TERM
    ctx.close()
