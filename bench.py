#!/usr/bin/env python
"""H|psi> band-applications/s on one GB300: mixed precision vs float64, plus the CPU oracle.

Workload (default, c5): the cubic a = 30 bohr cell with 216 atoms on a jittered 6x6x6 lattice,
E_cut 25 Ha, Gamma, FFT box 144^3, 161235 plane waves, 864 s+p projectors, 512 bands.

A step is one complete block-Davidson solve of the 512-band block through the C ABI, in the
Gamma-point real form of Sec. 4 (the cell is Gamma-only, so its orbitals are real: half the
coefficients, two bands per complex FFT, real subspace algebra): davidson_solve_gamma from the
seeded starting block to the residual tolerance.  It runs every step of the hot path (sphere
scatter, 3-D FFTs, x V(r), gather + kinetic, calbec, D, add_vuspsi, residuals, preconditioner,
Rayleigh-Ritz) as often as the solve needs them.  The metric counts the H|psi> band-applications
of the step (one real band through H) over the step's device time.  ``value`` is the mixed-precision
solve; ``config.fp64`` is the float64 solve of the same block; both report their largest eigenvalue
error against the oracle's reference eigenvalues (tests/golden/eigenvalues.json).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the library's
stream with the library's per-launch timing off; a 256 MB buffer is written between steps (outside
the events) so no step starts with the previous step's data in L2.  One more step with per-launch
timing on gives the per-kernel breakdown and the roofline of the dominant kernel.  Under torchrun
every rank runs its own replica of the block (the bands of different blocks are independent: no
collective on the data path) and rank 0 reports the whole-job rate with the max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H|psi> band-applications/s"
HBM_FALLBACK_GBS = 6800.0
FP64_ALU_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12    # 2 DFMA / clk / SM (measured), 2070 MHz max clock
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA x 2070 MHz

# DRAM bytes (read + write) per unit measured by ncu for a kernel class, keyed by (kernel, precision)
# with the hash of its source files at capture time; a mismatch reports null.  Units: a band of
# the kernel's launch for the H|psi> classes, a matrix element for the reduction.
#   xvx_y mixed: k_plane<float,9,10>, 48-band launch, 51.73 MB read + 4.81 MB write
#   calbec fp64: k_calbec64, 160-band launch, 270.83 MB read + 7.20 MB write
#   tridiag: k_eh_tridiag, one n = 640 launch, 3.372 MB read + 0.030 MB write
#   tridiag_real: k_eh_tridiag_r, one n = 1536 launch, 9.580 MB read + 2.8 KB write
NCU_TRAFFIC = {
    ("tridiag", -1): (("eigh_tridiag.cuh",), "7b3ca0b96a01", (3367936 + 31488) / 640 ** 2),
    ("tridiag_real", -1): (("eigh_tridiag_real.cuh",), "9dff8d240ee0", (9579520 + 2816) / 1536 ** 2),
    ("tridiag_df", -1): (("eigh_tridiag_df.cuh",), "d822de855785", (9583104 + 8704) / 1536 ** 2),
    ("xvx_y", 1): (("local_fast.cu", "fft_codelets.cuh"), "92564643ab55", (51.725568e6 + 4.813056e6) / 48),
    ("calbec", 0): (("nonlocal_fp64.cu",), "dc474a4712d7", (270.831104e6 + 7.199488e6) / 160),
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="c5")
    ap.add_argument("--form", default="auto", choices=["auto", "gamma", "complex"],
                    help="auto: the Gamma-point real form when the cell is Gamma-only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the side figures (c2 complex, batches, CG)")
    ap.add_argument("--tol-mixed", type=float, default=None)
    ap.add_argument("--tol-fp64", type=float, default=1e-8)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-warmup", type=int, default=0)
    ap.add_argument("--oracle-bands", type=int, default=4, help="bands per step of the oracle sample")
    return ap.parse_args(argv)


# Residual tolerance of the mixed solve: its float32 residuals stop at a floor set by the largest
# eigenvalue of H (the cutoff), so the larger cutoff of the 25-Ha cells takes a looser tolerance;
# the eigenvalues are float64 Rayleigh quotients either way and are judged against the oracle.
MIXED_TOL = {"c5": 5e-5}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def world_max(x, world, device):
    """Largest x over the ranks of the default process group (x itself when world == 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, max_ms, world):
    """Whole-job throughput of independent replicas: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def workload(cfg, form="complex"):
    import workloads
    p = workloads.CONFIGS[cfg]()
    cubic = np.all(p.lattice == np.diag(np.diag(p.lattice)))
    desc = (f"{cfg}: {p.name}, cell {np.diag(p.lattice).tolist() if cubic else 'oblique'} bohr, "
            f"{len(p.atoms)} atoms, E_cut {p.ecut} Ha, box {p.fft[0]}x{p.fft[1]}x{p.fft[2]}, {p.nproj} projectors, "
            f"{p.nbnd} bands, Gamma" + (", Gamma-point real form (Sec. 4)" if form == "gamma" else ""))
    return p, desc


def choose_form(p, form):
    if form != "auto":
        return form
    return "gamma" if len(p.kpts) == 1 and not np.any(p.kpts[0]) else "complex"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------------------------
# CPU oracle legs (the same sample for the reference arm and the GPU arm's cpu_baseline)
# ---------------------------------------------------------------------------------------------

def oracle_inputs(p, nb):
    import oracle
    import workloads
    k = p.kpts[0]
    m = oracle.gsphere.gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    d = workloads.dmat(len(p.atoms))
    psi = workloads.psi0(p.lattice, k, m, nb, p.psi_seed)
    return k, m, vr, beta, d, psi


def oracle_step(p, inputs, nb):
    """The oracle's H|psi> on nb bands (FFT form, scipy with all host cores) plus its Davidson
    residual, preconditioner and Rayleigh-Ritz on that sample; returns seconds."""
    import oracle
    k, m, vr, beta, d, psi = inputs
    t0 = time.perf_counter()
    x = psi[:nb]
    hx = oracle.hamiltonian.hpsi(p.lattice, k, m, p.fft, vr, beta, d, x)
    e, xr, hxr = oracle.davidson.rayleigh_ritz(x, hx, nb)
    g = oracle.davidson.residuals(hxr, xr, e)
    oracle.davidson.precondition(g, oracle.hamiltonian.h_diagonal(p.lattice, k, m, vr, beta, d), e)
    return time.perf_counter() - t0


def oracle_sample(p, nb, steps, warmup):
    """The oracle timed on `steps` samples of nb bands after `warmup` untimed ones: (value, seconds, text)."""
    inputs = oracle_inputs(p, nb)
    for _ in range(warmup):
        oracle_step(p, inputs, nb)
    ts = [oracle_step(p, inputs, nb) for _ in range(steps)]
    tot = sum(ts)
    return nb * len(ts) / tot, tot, (f"{nb} of the {p.nbnd} bands per step, {len(ts)} steps: oracle H|psi> (scipy.fft, "
                                     f"{host_cores()} workers) + residual, preconditioner and Rayleigh-Ritz on the "
                                     f"sample, {tot:.2f} s")


def cpu_baseline(p, nb):
    val, _, text = oracle_sample(p, nb, 3, 1)
    return {"value": val, "unit": "band-applications/s", "cores": host_cores(), "kind": "oracle", "sample": text}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    p, desc = workload(args.config)
    val, tot, text = oracle_sample(p, args.oracle_bands, args.steps, args.warmup)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "band-applications/s",
           "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": desc, "step": text},
           "cpu_baseline": {"value": val, "unit": "band-applications/s", "cores": host_cores(), "kind": "oracle",
                            "sample": text},
           "e2e": {"value": val, "unit": "band-applications/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

class Clocks:
    """nvidia-smi samples of SM clock, power and throttle reasons, every 200 ms while active."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.dir = tempfile.mkdtemp(prefix="hpsi_clocks_")
        self.path = os.path.join(self.dir, "clocks.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def source_hash(files):
    h = hashlib.sha256()
    for rel in files:
        with open(os.path.join(ROOT, "paper_0906_2569_gb300", "csrc", rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def kernel_breakdown(B, ctx):
    """Per-class launches and event time of the library's kernels, and the part of it made while H was
    applied in float64 (keys name@fp64)."""
    out = {}
    for kk, name in enumerate(B.KERNELS):
        n, t = B.hpsi_kernel_stats(ctx, kk)
        n64, t64 = B.hpsi_kernel_stats(ctx, kk + B.HPSI_K_AT_FP64)
        if n - n64:
            out[name] = {"launches": n - n64, "ms": t - t64}
        if n64:
            out[name + "@fp64"] = {"launches": n64, "ms": t64}
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import oracle
    import workloads
    from paper_0906_2569_gb300 import binding as B

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    p0, _ = workload(args.config)
    form = choose_form(p0, args.form)
    p, desc = workload(args.config, form)
    tol_mixed = args.tol_mixed if args.tol_mixed is not None else MIXED_TOL.get(args.config, 1e-5)
    k = p.kpts[0]
    miller = B.hpsi_gsphere(p.lattice, p.ecut, k)
    npw = len(miller)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, miller)
    d = workloads.dmat(len(p.atoms))
    full0 = workloads.psi0(p.lattice, k, miller, p.nbnd, p.psi_seed)
    gamma = form == "gamma"
    start = np.ascontiguousarray(oracle.gamma.to_half(full0, miller)) if gamma else full0
    psi0 = torch.from_numpy(start).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    nst, npl = stick_counts(miller, p.fft)
    solve = B.davidson_solve_gamma if gamma else B.davidson_solve

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    golden = None
    try:
        golden = json.load(open(os.path.join(ROOT, "tests", "golden", "eigenvalues.json"))).get(args.config)
    except (OSError, ValueError):
        golden = None

    def eig_error(eig):
        if golden is None:
            return None, 0
        g = np.asarray(golden["eigenvalues"])
        n = min(len(g), len(eig))
        return float(np.max(np.abs(eig[:n] - g[:n]))), n

    def measure(precision, tol, steps, warmup, e2e=False, breakdown=True):
        """Each step: one solve of the whole block to tol from the seeded start.  Warm-up: `warmup`
        solves, after one untimed H|psi> of the block (allocations and the autotuner)."""
        ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], d, precision, stream.cuda_stream)
        work = torch.empty_like(psi0)
        info = {}
        (B.hpsi_apply_gamma if gamma else B.hpsi_apply)(ctx, 0, psi0, work)

        def step():
            work.copy_(psi0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eig, it, res, rc = solve(ctx, 0, work, tol, 400, raise_on_notconv=False)
            e1.record(stream)
            info.update(eig=eig, iters=it, res=float(np.max(res)), rc=rc)
            return e0, e1

        for _ in range(warmup):
            step()
        barrier()
        B.hpsi_kernel_stats(ctx, -1, reset=True)
        B.hpsi_kernel_stats(ctx, -2, reset=True)
        evs = []
        with Clocks(local_rank) as clk:
            for _ in range(steps):
                evs.append(step())
            barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        launches, _ = B.hpsi_kernel_stats(ctx, -1)
        bapps, _ = B.hpsi_kernel_stats(ctx, -2)
        err, nerr = eig_error(info["eig"])
        res = {"total_ms": sum(ms), "ms": ms, "band_apps": bapps, "launches": launches, "clocks": clk.summary(),
               "iters": info["iters"], "max_residual": info["res"], "status": info["rc"], "max_eig_error_ha": err,
               "n_eig_checked": nerr}
        # one more solve with per-launch timing: the kernel breakdown and the roofline's durations
        res["kernels"] = {}
        if breakdown:
            for kk in range(len(B.KERNELS)):
                B.hpsi_kernel_stats(ctx, kk, reset=True)
            B.hpsi_kernel_stats(ctx, -2, reset=True)
            B.hpsi_kernel_stats(ctx, -4, reset=True)
            B.hpsi_set_option(ctx, B.HPSI_OPT_KERNEL_TIMING, 1)
            step()
            torch.cuda.synchronize()
            res["kernels"] = kernel_breakdown(B, ctx)
            res["timed_band_apps"] = B.hpsi_kernel_stats(ctx, -2)[0]
            res["tridiag_flops"] = B.hpsi_kernel_stats(ctx, -4)[1]
            B.hpsi_set_option(ctx, B.HPSI_OPT_KERNEL_TIMING, 0)
        # H|psi> alone on the block, for reference
        apply = B.hpsi_apply_gamma if gamma else B.hpsi_apply
        out = torch.empty_like(psi0)
        hms = []
        for _ in range(2):
            apply(ctx, 0, psi0, out)
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            apply(ctx, 0, psi0, out)
            e1.record(stream)
            torch.cuda.synchronize()
            hms.append(e0.elapsed_time(e1))
        res["hpsi_ms"] = statistics.median(hms)
        if e2e:
            host = torch.empty(psi0.shape, dtype=psi0.dtype, pin_memory=True)
            src = psi0.cpu()
            ts, b0 = [], None
            for i in range(1 + steps):
                host.copy_(src)
                flush.zero_()
                torch.cuda.synchronize()
                if i == 1:
                    b0, _ = B.hpsi_kernel_stats(ctx, -2)
                t0 = time.perf_counter()
                solve(ctx, 0, host, tol, 400, raise_on_notconv=False)
                t1 = time.perf_counter()
                if i >= 1:
                    ts.append(t1 - t0)
            b1, _ = B.hpsi_kernel_stats(ctx, -2)
            res["e2e_s"] = ts
            res["e2e_band_apps"] = b1 - b0
            res["e2e_bytes"] = int(psi0.numel() * 16)
        ctx.close()
        return res

    mixed = measure(B.HPSI_MIXED, tol_mixed, args.steps, args.warmup, e2e=not args.no_e2e)
    fp64 = measure(B.HPSI_FP64, args.tol_fp64, args.fp64_steps, args.fp64_warmup, breakdown=False)
    mix_ms = world_max(mixed["total_ms"], world, "cuda")
    f64_ms = world_max(fp64["total_ms"], world, "cuda")
    value = replica_value(mixed["band_apps"], mix_ms, world)
    v64 = replica_value(fp64["band_apps"], f64_ms, world)
    side = {}
    if not args.no_side:
        del psi0
        torch.cuda.empty_cache()
        side["c2_complex_solve"] = complex_solve(B, torch, flush)
        side["batched"] = batch_throughput(args, B, torch, flush)
        side["hpsi_apply_by_config"] = config_throughput(B, torch, flush)
        side["cg_solver"] = cg_throughput(B, torch)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    units = 2 if gamma else 1   # real bands per complex band through the H|psi> kernels
    roof = roofline(mixed, p, npw, nst, npl, B.HPSI_MIXED, units)
    out = {
        "metric": METRIC,
        "value": value, "unit": "band-applications/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mix_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("mixed: f32 FFT + xV, bf16 3-term split (6-product) tensor-core nonlocal with f32 accumulation, "
                  "f32 subspace GEMMs; f64-accurate residual norms, reduced eigenproblems (double-float Householder "
                  "reduction, f64 Sturm counts), Cholesky factors, and f64 projections <beta|psi>, D for the final "
                  "Rayleigh quotients"),
        "data": "synthetic",
        "config": {"workload": desc, "npw": npw, "form": form,
                   "fp64": {"value": v64, "ms_per_step": f64_ms / args.fp64_steps, "steps": args.fp64_steps,
                            "warmup": args.fp64_warmup, "tol": args.tol_fp64, "iterations": fp64["iters"],
                            "max_eig_error_ha_vs_oracle": fp64["max_eig_error_ha"],
                            "hpsi_apply_band_apps_per_s": p.nbnd / (fp64["hpsi_ms"] / 1e3)},
                   "mixed_over_fp64": value / v64,
                   "band_apps_per_step": mixed["band_apps"] // max(1, args.steps),
                   "step": (f"one {'davidson_solve_gamma' if gamma else 'davidson_solve'} of the {p.nbnd}-band block "
                            f"to max residual {tol_mixed:g} from the seeded start (every H|psi>, residual, "
                            "preconditioner and Rayleigh-Ritz of the solve; final Rayleigh quotients after one more "
                            "application of H with float64 projections and D)"),
                   "iterations": mixed["iters"], "max_residual": mixed["max_residual"],
                   "max_eig_error_ha_vs_oracle": mixed["max_eig_error_ha"],
                   "eigenvalues_checked": mixed["n_eig_checked"],
                   "hpsi_apply_band_apps_per_s": p.nbnd / (mixed["hpsi_ms"] / 1e3),
                   "l2": "256 MB buffer written between timed steps", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "clocks": mixed["clocks"],
        "gpu_launches": mixed["launches"],
    }
    if "e2e_s" in mixed:
        tot = sum(mixed["e2e_s"])
        out["e2e"] = {"value": mixed["e2e_band_apps"] / tot * world, "unit": "band-applications/s",
                      "h2d_bytes_per_step": mixed["e2e_bytes"], "d2h_bytes_per_step": mixed["e2e_bytes"] + 8 * p.nbnd}
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(p, args.oracle_bands)
    out["kernels"] = {k_: {"launches": v["launches"], "ms": round(v["ms"], 2)} for k_, v in
                      sorted(mixed["kernels"].items(), key=lambda kv: -kv[1]["ms"])}
    out.update(side)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def complex_solve(B, torch, flush, name="c2"):
    """The complex-form mixed Davidson solve of the 160-band block of the 36785-PW cell: the form a
    k-point calculation takes.  One untimed, two timed solves."""
    import workloads
    try:
        p = workloads.CONFIGS[name]()
        k = p.kpts[0]
        m = B.hpsi_gsphere(p.lattice, p.ecut, k)
        stream = torch.cuda.current_stream()
        ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, workloads.vloc_r(p.lattice, p.atoms, p.fft),
                           [workloads.beta(p.lattice, p.atoms, k, m)], workloads.dmat(len(p.atoms)), B.HPSI_MIXED,
                           stream.cuda_stream)
        x0 = torch.from_numpy(workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed)).cuda()
        gold = np.asarray(json.load(open(os.path.join(ROOT, "tests", "golden", "eigenvalues.json")))[name]["eigenvalues"])
        ms, bapps = [], 0
        for i in range(3):
            x = x0.clone()
            flush.zero_()
            B.hpsi_kernel_stats(ctx, -2, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eig, it, res, rc = B.davidson_solve(ctx, 0, x, 1e-5, 400, raise_on_notconv=False)
            e1.record(stream)
            torch.cuda.synchronize()
            if i:
                ms.append(e0.elapsed_time(e1))
                bapps += B.hpsi_kernel_stats(ctx, -2)[0]
        ctx.close()
        return {"workload": f"{name}: {p.nbnd} bands, {len(m)} PW, complex form, mixed, residual 1e-5",
                "band_apps_per_s": bapps / (sum(ms) / 1e3), "ms": sum(ms) / len(ms), "iterations": it,
                "max_eig_error_ha_vs_oracle": float(np.max(np.abs(eig - gold[:p.nbnd])))}
    except Exception as exc:   # noqa: BLE001 -- reported, the headline line still prints
        return {"error": str(exc)[:200]}


def batch_throughput(args, B, torch, flush):
    """hpsi_apply_batch (CUDA-graph replay) on the 16 k-points of the fcc cell and on the 32 cells:
    band-applications/s, float64 and mixed."""
    import workloads
    stream = torch.cuda.current_stream()
    out = {}
    p = workloads.config4a()
    ms = [B.hpsi_gsphere(p.lattice, p.ecut, k) for k in p.kpts]
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    betas = [workloads.beta(p.lattice, p.atoms, k, m) for k, m in zip(p.kpts, ms)]
    xs_k = [torch.from_numpy(workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed + i)).cuda()
            for i, (k, m) in enumerate(zip(p.kpts, ms))]
    cells = workloads.config4b()
    cm = [B.hpsi_gsphere(c.lattice, c.ecut, c.kpts[0]) for c in cells]
    cv = [workloads.vloc_r(c.lattice, c.atoms, c.fft) for c in cells]
    cb = [workloads.beta(c.lattice, c.atoms, c.kpts[0], m) for c, m in zip(cells, cm)]
    xs_c = [torch.from_numpy(workloads.psi0(c.lattice, c.kpts[0], m, c.nbnd, c.psi_seed)).cuda()
            for c, m in zip(cells, cm)]
    for prec, pname in ((B.HPSI_FP64, "fp64"), (B.HPSI_MIXED, "mixed")):
        for label, make, xs in (
                ("kpoints_fcc_16k_24b", lambda: B.hpsi_setup(p.lattice, p.ecut, p.kpts, p.fft, vr, betas,
                                                             workloads.dmat(len(p.atoms)), prec, stream.cuda_stream),
                 xs_k),
                ("cells_32", lambda: B.hpsi_setup_cells([c.lattice for c in cells], [c.ecut for c in cells],
                                                        [c.fft for c in cells], cv, cb,
                                                        [workloads.dmat(len(c.atoms)) for c in cells], prec,
                                                        stream.cuda_stream), xs_c)):
            ctx = make()
            ys = [torch.empty_like(x) for x in xs]
            probs = list(range(len(xs)))
            for _ in range(max(3, args.warmup)):
                B.hpsi_apply_batch(ctx, probs, xs, ys)
            torch.cuda.synchronize()
            ms_ = []
            for _ in range(5):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.hpsi_apply_batch(ctx, probs, xs, ys)
                e1.record(stream)
                torch.cuda.synchronize()
                ms_.append(e0.elapsed_time(e1))
            bands = sum(int(x.shape[0]) for x in xs)
            out.setdefault(label, {})[pname] = round(bands / (statistics.median(ms_) / 1e3), 1)
            ctx.close()
    return out


def config_throughput(B, torch, flush, names=("c1", "c2", "c5")):
    """Steady-state hpsi_apply (whole band block, CUDA events, L2 flushed) per configuration, complex
    form, band-applications/s."""
    import workloads
    stream = torch.cuda.current_stream()
    out = {}
    for name in names:
        p = workloads.CONFIGS[name]()
        k = p.kpts[0]
        m = B.hpsi_gsphere(p.lattice, p.ecut, k)
        vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
        beta = workloads.beta(p.lattice, p.atoms, k, m)
        x = torch.from_numpy(workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed)).cuda()
        y = torch.empty_like(x)
        res = {}
        for prec, pname in ((B.HPSI_FP64, "fp64"), (B.HPSI_MIXED, "mixed")):
            ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, vr, [beta], workloads.dmat(len(p.atoms)), prec,
                               stream.cuda_stream)
            for _ in range(2):
                B.hpsi_apply(ctx, 0, x, y)
            ms_ = []
            for _ in range(3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.hpsi_apply(ctx, 0, x, y)
                e1.record(stream)
                torch.cuda.synchronize()
                ms_.append(e0.elapsed_time(e1))
            res[pname] = round(p.nbnd / (statistics.median(ms_) / 1e3), 1)
            ctx.close()
        out[name] = res
        del x, y
        torch.cuda.empty_cache()
    return out


def cg_throughput(B, torch):
    """The band-by-band CG eigensolver (App. A.2.2) beside the Davidson headline: the 16 bands of the
    1503-PW cell (c1) in float64 to residual 1e-8, one untimed and one timed solve (CUDA events).
    Every step applies H to one band; the figure counts those band-applications over the solve.
    A failure here is reported in the JSON line instead of ending the run."""
    import workloads
    try:
        p = workloads.config1()
        k = p.kpts[0]
        m = B.hpsi_gsphere(p.lattice, p.ecut, k)
        stream = torch.cuda.current_stream()
        ctx = B.hpsi_setup(p.lattice, p.ecut, [k], p.fft, workloads.vloc_r(p.lattice, p.atoms, p.fft),
                           [workloads.beta(p.lattice, p.atoms, k, m)], workloads.dmat(len(p.atoms)), B.HPSI_FP64,
                           stream.cuda_stream)
        x0 = torch.from_numpy(workloads.psi0(p.lattice, k, m, p.nbnd, p.psi_seed)).cuda()
        golden = json.load(open(os.path.join(ROOT, "tests", "golden", "eigenvalues.json")))["c1"]["eigenvalues"]
        for timed in (False, True):
            x = x0.clone()
            B.hpsi_kernel_stats(ctx, -2, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eig, steps, res, rc = B.cg_solve(ctx, 0, x, 1e-8, 3000)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        bapps = B.hpsi_kernel_stats(ctx, -2)[0]
        ctx.close()
        return {"workload": "c1: 16 bands, 1503 PW, float64, residual 1e-8", "ms": ms, "steps": steps,
                "band_apps": bapps, "band_apps_per_s": bapps / (ms / 1e3),
                "max_eig_error_ha_vs_oracle": float(np.max(np.abs(eig - np.asarray(golden[:p.nbnd]))))}
    except Exception as exc:   # noqa: BLE001 -- reported, the headline line still prints
        return {"error": str(exc)[:200]}


def stick_counts(miller, fft):
    m = np.asarray(miller)
    sticks = {(a, b) for a, b in zip(m[:, 0].tolist(), m[:, 1].tolist())}
    planes = {a for a in m[:, 0].tolist()}
    return len(sticks), len(planes)


def kernel_work(name, p, npw, nst, npl, precision, nproj, real=False):
    """Algorithmic (bytes, flops) of one complex band through a kernel class of the fast path, or,
    with real (the Gamma form's nonlocal classes), of one real band in real-basis coordinates.

    Line FFTs count 5 n log2 n flops; bytes are the HBM data the method itself must move per band
    (psi in, H|psi> out, the stick rows between the z and the plane kernels).  The nonlocal GEMMs
    count 8 P npw flops per complex band, 2 P (npw + 1) per real band (x 6 bf16 products at mixed
    precision)."""
    n1, n2, n3 = p.fft
    cs = 16 if precision == 0 else 8
    fft = lambda n: 5.0 * n * math.log2(n)
    rows = n3 * nst * cs
    if name == "inv_zy":
        return 16 * npw + rows, nst * fft(n3)
    if name == "xvx_y":
        return 2 * rows, n3 * (2 * npl * fft(n2) + 2 * n2 * fft(n1) + 2 * n1 * n2)
    if name == "fwd_z":
        return rows + 2 * 16 * npw + 8 * npw, nst * fft(n3)
    if name in ("calbec", "addvus"):
        if real:
            return 8 * (npw + 1), 2.0 * nproj * (npw + 1) * (6 if precision == 1 else 1)
        return 16 * npw, 8.0 * nproj * npw * (6 if precision == 1 else 1)
    return None, None


def tridiag_roofline(res, kst, real=False, df=False):
    """Roofline of the Householder reduction of the reduced eigenproblems, against the float64 ALU
    roof (the precision it delivers; df: the double-float kernel of the mixed Gamma solve, which does
    that work on the float32 pipes).

    Algorithmic work per launch: 16 n^3 / 3 real flops for a complex Hermitian matrix, 4 n^3 / 3 for
    a real symmetric one (the Gamma-point form), summed by the library over the timed launches; the
    launches' n vary with the reduced basis."""
    secs = kst["ms"] / 1e3
    ach = res["tridiag_flops"] / secs / 1e12
    nlaunch = kst["launches"]
    n_eff = (res["tridiag_flops"] / nlaunch / ((4.0 if real else 16.0) / 3.0)) ** (1.0 / 3.0)
    traffic = None
    key = ("tridiag_df" if df else ("tridiag_real" if real else "tridiag"), -1)
    if key in NCU_TRAFFIC and NCU_TRAFFIC[key][1] == source_hash(NCU_TRAFFIC[key][0]):
        traffic = NCU_TRAFFIC[key][2] * n_eff ** 2      # bytes per matrix element, x n^2
    return {"kernel": "tridiag", "avg_launch_ms": kst["ms"] / nlaunch, "launches": nlaunch,
            "flops_per_launch": res["tridiag_flops"] / nlaunch, "n_cube_root_mean_cube": n_eff,
            "traffic": traffic, "bound": "alu", "achieved": ach, "peak": FP64_ALU_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_ALU_TFLOPS, "peak_source": "derived: 152 SMs x 2 DFMA/clk (measured) x 2 flop x 2070 MHz"}


HPSI_CLASSES = ("inv_zy", "xvx_y", "fwd_z", "calbec", "addvus")


def roofline(res, p, npw, nst, npl, precision, units_per_band=1):
    """Roofline of the library kernel class with the largest event time in the timed-breakdown solve.
    Launches made while H was applied in float64 inside a mixed solve form their own class
    (name@fp64), so each class has one precision."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    ks = res["kernels"]
    cand = {k: v for k, v in ks.items() if v["ms"] > 0 and (k.split("@")[0] in HPSI_CLASSES or k == "tridiag")}
    if not cand:
        return None
    name = max(cand, key=lambda k: cand[k]["ms"])
    if name == "tridiag" and res.get("tridiag_flops"):
        return tridiag_roofline(res, cand[name], real=units_per_band == 2, df=units_per_band == 2 and precision == 1)
    base = name.split("@")[0]
    prec = 0 if name.endswith("@fp64") else precision
    # bands through the class in that solve: the final float64 application of a mixed solve handles
    # the nbnd Ritz vectors, the rest of the band-applications ran at the working precision.  The
    # Gamma form (units_per_band 2) packs two real bands per complex band for the local classes and
    # runs the nonlocal classes on the real bands themselves.
    real_nl = units_per_band == 2 and base in ("calbec", "addvus")
    upb = 1 if real_nl else units_per_band
    total = res["timed_band_apps"] / upb
    final = p.nbnd / upb if precision == 1 else 0
    bands = final if name.endswith("@fp64") else total - final
    byt, flop = kernel_work(base, p, npw, nst, npl, prec, p.nproj, real=real_nl)
    secs = cand[name]["ms"] / 1e3
    avg_ms = cand[name]["ms"] / cand[name]["launches"]
    traffic = None
    key = (base, prec)
    per_launch = bands / cand[name]["launches"]
    if key in NCU_TRAFFIC and NCU_TRAFFIC[key][1] == source_hash(NCU_TRAFFIC[key][0]):
        traffic = NCU_TRAFFIC[key][2] * per_launch
    out = {"kernel": name, "avg_launch_ms": avg_ms, "launches": cand[name]["launches"], "traffic": traffic,
           "bytes_per_band": byt, "flops_per_band": flop, "bands_per_launch": per_launch}
    if base in ("calbec", "addvus") and prec == 1:
        peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
        ach = bands * flop / secs / 1e12
        out.update({"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "peak_source": "measured bf16 sustained"})
        return out
    alu = FP64_ALU_TFLOPS if prec == 0 else FP32_ALU_TFLOPS
    ridge = alu * 1e12 / (hbm * 1e9)
    if flop / byt > ridge:
        ach = bands * flop / secs / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": alu, "unit": "TFLOP/s", "frac": ach / alu,
                    "peak_source": ("derived: 152 SMs x 2 DFMA/clk (measured) x 2 flop x 2070 MHz" if prec == 0
                                    else "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz")})
    else:
        ach = bands * byt / secs / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"})
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
