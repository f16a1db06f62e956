"""Write reference eigenvalues of the synthetic cells, computed by the CPU oracle only.

The paper prints no eigenvalues for any system (it has no worked example), so every stored value
here is the oracle's: the lowest eigenvalues of H (App. A.2, Eq. (diag) with S = I) by dense
LAPACK (oracle.eigen.lowest_dense on the element-by-element H_GG') where the matrix fits, else by
LOBPCG on the FFT form of H|psi> (oracle.eigen.lowest_lobpcg).  Usage:

    python tests/golden/make_golden.py [c1 c3 c4a c2 c4b c5 scf_c1]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "eigenvalues.json")


def inputs(p, k):
    m = oracle.gsphere.gsphere(p.lattice, p.ecut, k)
    vr = workloads.vloc_r(p.lattice, p.atoms, p.fft)
    beta = workloads.beta(p.lattice, p.atoms, k, m)
    return m, vr, beta, workloads.dmat(len(p.atoms))


def dense(p, k, nbnd):
    m, vr, beta, d = inputs(p, k)
    h = oracle.hamiltonian.dense_h(p.lattice, k, m, p.fft, vr, beta, d)
    return oracle.eigen.lowest_dense(h, nbnd).tolist(), {"method": "dense LAPACK eigvalsh", "npw": len(m)}


def lobpcg(p, k, nbnd, tol=1e-9, chunk=0, verbose=False):
    m, vr, beta, d = inputs(p, k)
    x0 = workloads.psi0(p.lattice, k, m, nbnd + 16, p.psi_seed + 7)
    w, res = oracle.eigen.lowest_lobpcg(p.lattice, k, m, p.fft, vr, beta, d, nbnd, x0, tol=tol, maxiter=600,
                                        nguard=16, chunk=chunk, verbose=verbose)
    return w.tolist(), {"method": "LOBPCG on the FFT H|psi>", "npw": len(m), "max_residual": float(np.max(res))}


OUT_SCF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scf.json")


def main(names):
    for name in names:
        out = OUT_SCF if name.startswith("scf") else OUT
        data = json.load(open(out)) if os.path.exists(out) else {}
        if out == OUT:
            data["_about"] = ("Lowest eigenvalues (Ha) of the seeded synthetic cells of workloads/, from the CPU "
                              "oracle only (App. A.2 Eq. (diag), S = I); written by tests/golden/make_golden.py.")
        else:
            data["_about"] = ("Self-consistent solutions (App. A.1) of seeded synthetic cells of workloads/, from the "
                              "CPU oracle only (oracle.scf.scf); written by tests/golden/make_golden.py.")
        t0 = time.time()
        if name == "c1":
            p = workloads.config1()
            ev, info = dense(p, p.kpts[0], 64)
        elif name == "c3":
            p = workloads.config3(320)
            ev, info = dense(p, p.kpts[0], 320)
        elif name == "c4a":
            p = workloads.config4a()
            ev, info = [], {"method": "dense LAPACK eigvalsh per k-point", "npw": []}
            for k in p.kpts:
                e, i = dense(p, k, p.nbnd)
                ev.append(e)
                info["npw"].append(i["npw"])
        elif name == "c4b":
            ev, info = [], {"method": "dense LAPACK eigvalsh per cell", "npw": []}
            for cell in workloads.config4b():
                e, i = dense(cell, cell.kpts[0], cell.nbnd)
                ev.append(e)
                info["npw"].append(i["npw"])
        elif name == "c2":
            p = workloads.config2()
            ev, info = lobpcg(p, p.kpts[0], p.nbnd)
        elif name == "scf_c1":
            # the self-consistency loop of App. A.1 on the c1 cell: V_ext = the synthetic local
            # potential, two electrons per atom (nocc = 2), uniform starting density, dense H
            p = workloads.config1()
            k = p.kpts[0]
            m, vr, beta, d = inputs(p, k)
            omega = oracle.scf.cell_volume(p.lattice)
            rho0 = np.full(p.fft, 4.0 / omega)
            sol = oracle.scf.scf(p.lattice, k, m, p.fft, vr, beta, d, 2, rho0, tol=1e-16, maxiter=100)
            rng = np.random.default_rng(5000)
            idx = rng.choice(sol["rho"].size, 64, replace=False)
            ev = sol["eig"].tolist()
            info = {"method": "oracle.scf.scf, dense H, Anderson mixing (8, 0.5), tol 1e-16", "npw": len(m),
                    "nocc": 2, "e": sol["e"], "e_hwf": sol["e_hwf"], "iters": sol["iters"],
                    "charge": oracle.scf.charge(sol["rho"], p.lattice),
                    "rho_sample_index": idx.tolist(), "rho_sample": sol["rho"].reshape(-1)[idx].tolist(),
                    "rho_max": float(np.max(sol["rho"])), "rho_sum2": float(np.sum(sol["rho"] ** 2))}
        elif name.startswith("c5"):
            # the large cell: the lowest C5_NBND (default 64) of its 512 bands, H applied 16 bands
            # at a time to bound the memory of the 144^3 transforms
            nb = int(os.environ.get("C5_NBND", "64"))
            p = workloads.config5()
            ev, info = lobpcg(p, p.kpts[0], nb, chunk=16, verbose=True)
            name = "c5"
        else:
            raise SystemExit(f"unknown config {name}")
        info["seconds"] = round(time.time() - t0, 1)
        # re-read before writing: another run of this script may have added entries meanwhile
        data = json.load(open(out)) if os.path.exists(out) else data
        data[name] = {"eigenvalues": ev, **info}
        json.dump(data, open(out, "w"), indent=1)
        print(name, info, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1", "c3", "c4a"])
