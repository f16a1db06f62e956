"""A small, self-contained H|psi> case for profiler captures.

Runs ``--reps`` applications of H to the 160-band block of the 90^3 / 36785-PW / 256-projector
cell (or the cell named by ``--config``) at the chosen precision.  Two warm-up applications come
first (the first one runs the autotuner); the steady-state applications are bracketed by
cudaProfilerStart / cudaProfilerStop, so a profiler started with ``--profile-from-start off``
captures only them.

With ``--eigh N`` it instead solves the reduced Hermitian eigenproblem of order N (lowest
``--nwant`` pairs) on a seeded random matrix of the scale of a Davidson reduced H, the same way:
two warm-up solves, then ``--reps`` bracketed ones.

With ``--solve`` it runs the block-Davidson solve of the whole band block of the cell named by
``--config`` at the chosen precision (``--form gamma``: davidson_solve_gamma on the half-sphere
block, the default for a Gamma-only cell; ``--form complex``: davidson_solve), tolerance ``--tol``
(default 5e-5 mixed, 1e-8 float64): one warm-up solve, then one bracketed solve -- every launch of
a solve, the library's and cuBLAS's, falls inside the bracket.

With ``--eigh-real N`` the eigenproblem of order N is real symmetric (hpsi_eigh_lowest_sym);
``--df`` runs its reduction in double-float arithmetic (HPSI_OPT_EIGH_DF = 2).

With ``--batch c4a`` (the 16 k-points of the fcc cell) or ``--batch c4b`` (the 32 cells) it runs
hpsi_apply_batch on every item at the chosen precision: two warm-up batches (the first one eager,
then the captured graph), then ``--reps`` bracketed graph replays.  ``--batch-nl`` sets
HPSI_OPT_BATCH_NL and ``--persistent`` HPSI_OPT_PERSISTENT.

With ``--cg B`` it runs the band-by-band CG eigensolver on the first B bands of the cell named by
``--config`` in float64 (residual 1e-8, at most ``--cg-maxiter`` steps per band): one warm-up solve,
then one bracketed solve.  Every CG step's launches (three single-CTA kernels, the Gram-Schmidt
ZGEMVs and one single-band H|psi>) fall inside the bracket.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--nbnd", type=int, default=0)
    ap.add_argument("--eigh", type=int, default=0)
    ap.add_argument("--nwant", type=int, default=160)
    ap.add_argument("--cg", type=int, default=0)
    ap.add_argument("--cg-maxiter", type=int, default=3000)
    ap.add_argument("--solve", action="store_true")
    ap.add_argument("--form", default="auto", choices=["auto", "gamma", "complex"])
    ap.add_argument("--tol", type=float, default=0.0)
    ap.add_argument("--eigh-real", type=int, default=0)
    ap.add_argument("--df", action="store_true")
    ap.add_argument("--batch", default="", choices=["", "c4a", "c4b"])
    ap.add_argument("--batch-nl", type=int, default=0)
    ap.add_argument("--persistent", type=int, default=0)
    args = ap.parse_args()
    import torch
    import workloads
    from paper_0906_2569_gb300 import binding as B
    if args.eigh or args.eigh_real:
        eigh_case(args, torch, workloads, B)
        return
    if args.solve:
        solve_case(args, torch, workloads, B)
        return
    if args.cg:
        cg_case(args, torch, workloads, B)
        return
    if args.batch:
        batch_case(args, torch, workloads, B)
        return
    p = workloads.CONFIGS[args.config]()
    nb = args.nbnd or p.nbnd
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    prec = B.HPSI_MIXED if args.precision == "mixed" else B.HPSI_FP64
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], workloads.dmat(len(p.atoms)), prec,
                       torch.cuda.current_stream().cuda_stream)
    x = torch.from_numpy(workloads.psi0(p.lattice, k, m, nb, p.psi_seed)).cuda()
    y = torch.empty_like(x)
    for _ in range(2):
        B.hpsi_apply(ctx, 0, x, y)
    B.hpsi_sync(ctx)
    torch.cuda.profiler.start()
    for _ in range(args.reps):
        B.hpsi_apply(ctx, 0, x, y)
    B.hpsi_sync(ctx)
    torch.cuda.profiler.stop()
    print("ok", args.config, args.precision, nb, float(y.abs().sum()))


def eigh_case(args, torch, workloads, B):
    import numpy as np
    p = workloads.config1()
    ctx = B.hpsi_setup(p.lattice, p.ecut, [p.kpts[0]], p.fft, np.zeros(p.fft), None, None, B.HPSI_FP64,
                       torch.cuda.current_stream().cuda_stream)
    real = args.eigh_real > 0
    if args.df:
        B.hpsi_set_option(ctx, B.HPSI_OPT_EIGH_DF, 2)
    n = args.eigh_real if real else args.eigh
    nw = min(args.nwant, n)
    if real:
        rng = np.random.default_rng(n)
        q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        a = torch.from_numpy(np.ascontiguousarray(((q * rng.uniform(-20.0, 20.0, n)[None, :]) @ q.T).T)).cuda()
        v = torch.empty((nw, n), dtype=torch.float64, device="cuda")
        solve = B.hpsi_eigh_lowest_sym
    else:
        a = torch.from_numpy(np.ascontiguousarray(workloads.hermitian_matrix(n, n, scale=20.0).T)).cuda()
        v = torch.empty((nw, n), dtype=torch.complex128, device="cuda")
        solve = B.hpsi_eigh_lowest
    w = torch.empty(nw, dtype=torch.float64, device="cuda")
    for _ in range(2):
        solve(ctx, a, n, n, nw, w, v)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(args.reps):
        solve(ctx, a, n, n, nw, w, v)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("ok eigh", "real" if real else "complex", n, nw, float(w.sum()))


def solve_case(args, torch, workloads, B):
    import numpy as np
    import oracle
    p = workloads.CONFIGS[args.config]()
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    prec = B.HPSI_MIXED if args.precision == "mixed" else B.HPSI_FP64
    gamma = args.form == "gamma" or (args.form == "auto" and not np.any(k))
    tol = args.tol or (5e-5 if prec == B.HPSI_MIXED else 1e-8)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, workloads.vloc_r(p.lattice, p.atoms, p.fft),
                       [workloads.beta(p.lattice, p.atoms, k, m)], workloads.dmat(len(p.atoms)), prec,
                       torch.cuda.current_stream().cuda_stream)
    x0 = workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed)
    if gamma:
        x0 = np.ascontiguousarray(oracle.gamma.to_half(x0, m))
    x0 = torch.from_numpy(x0).cuda()
    solve = B.davidson_solve_gamma if gamma else B.davidson_solve
    solve(ctx, 0, x0.clone(), tol, 400, raise_on_notconv=False)
    torch.cuda.synchronize()
    x = x0.clone()
    torch.cuda.profiler.start()
    eig, it, res, rc = solve(ctx, 0, x, tol, 400, raise_on_notconv=False)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("ok solve", args.config, args.precision, "gamma" if gamma else "complex", it, rc, float(eig.sum()))


def cg_case(args, torch, workloads, B):
    p = workloads.CONFIGS[args.config]()
    k = p.kpts[0]
    m = B.hpsi_gsphere(p.lattice, p.ecut, k)
    ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, workloads.vloc_r(p.lattice, p.atoms, p.fft),
                       [workloads.beta(p.lattice, p.atoms, k, m)], workloads.dmat(len(p.atoms)), B.HPSI_FP64,
                       torch.cuda.current_stream().cuda_stream)
    x0 = torch.from_numpy(workloads.psi0(p.lattice, k, m, args.cg, p.psi_seed)).cuda()
    B.cg_solve(ctx, 0, x0.clone(), 1e-8, args.cg_maxiter)
    torch.cuda.synchronize()
    x = x0.clone()
    torch.cuda.profiler.start()
    eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-8, args.cg_maxiter)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("ok cg", args.config, args.cg, steps, float(eig.sum()))


def batch_case(args, torch, workloads, B):
    prec = B.HPSI_MIXED if args.precision == "mixed" else B.HPSI_FP64
    stream = torch.cuda.current_stream().cuda_stream
    if args.batch == "c4a":
        p = workloads.config4a()
        ms = [B.hpsi_gsphere(p.lattice, p.ecut, k) for k in p.kpts]
        betas = [workloads.beta(p.lattice, p.atoms, k, m) for k, m in zip(p.kpts, ms)]
        ctx = B.hpsi_setup(p.lattice, p.ecut, p.kpts, p.fft, workloads.vloc_r(p.lattice, p.atoms, p.fft), betas,
                           workloads.dmat(len(p.atoms)), prec, stream)
        xs = [torch.from_numpy(workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed + i)).cuda()
              for i, (k, m) in enumerate(zip(p.kpts, ms))]
    else:
        cells = workloads.config4b()
        ms = [B.hpsi_gsphere(c.lattice, c.ecut, c.kpts[0]) for c in cells]
        ctx = B.hpsi_setup_cells([c.lattice for c in cells], [c.ecut for c in cells], [c.fft for c in cells],
                                 [workloads.vloc_r(c.lattice, c.atoms, c.fft) for c in cells],
                                 [workloads.beta(c.lattice, c.atoms, c.kpts[0], m) for c, m in zip(cells, ms)],
                                 [workloads.dmat(len(c.atoms)) for c in cells], prec, stream)
        xs = [torch.from_numpy(workloads.psi0(c.lattice, c.kpts[0], m, c.nbnd, c.psi_seed)).cuda()
              for c, m in zip(cells, ms)]
    B.hpsi_set_option(ctx, B.HPSI_OPT_BATCH_NL, args.batch_nl)
    B.hpsi_set_option(ctx, B.HPSI_OPT_PERSISTENT, args.persistent)
    ys = [torch.empty_like(x) for x in xs]
    items = list(range(len(xs)))
    for _ in range(2):
        B.hpsi_apply_batch(ctx, items, xs, ys)
    B.hpsi_sync(ctx)
    torch.cuda.profiler.start()
    for _ in range(args.reps):
        B.hpsi_apply_batch(ctx, items, xs, ys)
    B.hpsi_sync(ctx)
    torch.cuda.profiler.stop()
    print("ok batch", args.batch, args.precision, len(xs), sum(int(x.shape[0]) for x in xs))


if __name__ == "__main__":
    main()
