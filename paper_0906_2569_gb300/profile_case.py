"""A small, self-contained H|psi> case for profiler captures.

Runs ``--reps`` applications of H to the 160-band block of the 90^3 / 36785-PW / 256-projector
cell (or the cell named by ``--config``) at the chosen precision.  Two warm-up applications come
first (the first one runs the autotuner); the steady-state applications are bracketed by
cudaProfilerStart / cudaProfilerStop, so a profiler started with ``--profile-from-start off``
captures only them.

With ``--eigh N`` it instead solves the reduced Hermitian eigenproblem of order N (lowest
``--nwant`` pairs) on a seeded random matrix of the scale of a Davidson reduced H, the same way:
two warm-up solves, then ``--reps`` bracketed ones.

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
    args = ap.parse_args()
    import torch
    import workloads
    from paper_0906_2569_gb300 import binding as B
    if args.eigh:
        eigh_case(args, torch, workloads, B)
        return
    if args.cg:
        cg_case(args, torch, workloads, B)
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
    n, nw = args.eigh, min(args.nwant, args.eigh)
    a = torch.from_numpy(np.ascontiguousarray(workloads.hermitian_matrix(n, n, scale=20.0).T)).cuda()
    w = torch.empty(nw, dtype=torch.float64, device="cuda")
    v = torch.empty((nw, n), dtype=torch.complex128, device="cuda")
    for _ in range(2):
        B.hpsi_eigh_lowest(ctx, a, n, n, nw, w, v)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(args.reps):
        B.hpsi_eigh_lowest(ctx, a, n, n, nw, w, v)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("ok eigh", n, nw, float(w.sum()))


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


if __name__ == "__main__":
    main()
