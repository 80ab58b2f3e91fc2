"""Writes c2_cg_iterations.json: oracle CG iteration counts on the 2187^2 workload.

Workload: 2-D, N = 2187^2, seeded RSA polydisperse disks (radii uniform in
[8, 40] px) to digital volume fraction 0.4, matrix L = I, inclusions
L = rho I for rho in {1e1, 1e2, 1e3, 1e4}, L0 from Eq. (opt_ref), loads
E = (1, 0) and (0, 1), CG from e = E to relative residual 1e-6.
Calls only the oracle and the input generator; one process per solve.
Takes tens of minutes on one core per solve.
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

RHO = [1e1, 1e2, 1e3, 1e4]
TOL = 1e-6


def _solve(args):
    rho, b = args
    import numpy as np

    import oracle
    from paper_1004_1122_gb300 import microstructure as micro

    phase = micro.rsa_disks(2187, 0.4, 8, 40, seed=micro.config_seed(2))
    L = micro.isotropic_table([1.0, rho], 2)
    L0 = oracle.reference_medium(L)
    E = np.eye(2)[b]
    x, info = oracle.cg(phase, L, L0, E, tol=TOL, max_iter=5000)
    col = oracle.effective_tensor([x], phase, L)[:, 0]
    return {"rho": rho, "load": b, "iters": int(info["iters"]), "status": info["status"],
            "rel_res_true": float(info["rel_res_true"]), "L_eff_col": col.tolist()}


def main():
    jobs = [(r, b) for r in RHO for b in (0, 1)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(jobs)) as pool:
        rows = pool.map(_solve, jobs)
    out = {"source": "oracle.cg on the 2187^2 RSA-disk workload, tol 1e-6 (see module doc)",
           "tol": TOL, "solves": rows}
    with open(os.path.join(HERE, "c2_cg_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
