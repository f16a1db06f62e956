"""Write reference eigenvalues of the synthetic cells, computed by the CPU oracle only.

The paper prints no eigenvalues for any system (it has no worked example), so every stored value
here is the oracle's: the lowest eigenvalues of H (App. A.2, Eq. (diag) with S = I) by dense
LAPACK (oracle.eigen.lowest_dense on the element-by-element H_GG') where the matrix fits, else by
LOBPCG on the FFT form of H|psi> (oracle.eigen.lowest_lobpcg).  Usage:

    python tests/golden/make_golden.py [c1 c3 c4a c2 c4b]
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


def lobpcg(p, k, nbnd, tol=1e-9):
    m, vr, beta, d = inputs(p, k)
    x0 = workloads.psi0(p.lattice, k, m, nbnd + 16, p.psi_seed + 7)
    w, res = oracle.eigen.lowest_lobpcg(p.lattice, k, m, p.fft, vr, beta, d, nbnd, x0, tol=tol, maxiter=600,
                                        nguard=16)
    return w.tolist(), {"method": "LOBPCG on the FFT H|psi>", "npw": len(m), "max_residual": float(np.max(res))}


def main(names):
    data = {}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    data["_about"] = ("Lowest eigenvalues (Ha) of the seeded synthetic cells of workloads/, from the CPU oracle "
                      "only (App. A.2 Eq. (diag), S = I); written by tests/golden/make_golden.py.")
    for name in names:
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
        else:
            raise SystemExit(f"unknown config {name}")
        info["seconds"] = round(time.time() - t0, 1)
        data[name] = {"eigenvalues": ev, **info}
        json.dump(data, open(OUT, "w"), indent=1)
        print(name, info, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1", "c3", "c4a"])
