"""Writes full_size_parity.json: oracle effective-tensor columns of the grids on
which the library's compile-time-plan kernels run.

Cases (all inputs from paper_1004_1122_gb300.microstructure, seeds fixed here):

* c2_2187  -- 2-D N = 2187^2, the RSA polydisperse-disk workload (radii
  uniform in [8, 40] px, digital volume fraction 0.4, seed of config 2),
  matrix L = I, inclusions L = 10 I, L0 of Eq. (opt_ref), loads (1, 0) and
  (0, 1).  The 2187-point plan runs the float32 CG passes there.
* batch    -- eight 2-D cells of sizes 135, 243, 375 and 729 (two each):
  disks, ellipses and a laminate, contrasts 10..100, loads (1, 0) and (0, 1).
  The 729-point two-load plan runs the 729^2 group.
* c3_243   -- 3-D N = 243^3, Boolean overlapping spheres of radius 12 px to
  digital volume fraction 0.25 (seed of config 3), L = I / 10 I, the three
  unit loads.  The 243-point plan runs every 3-D pass.

Each (cell, load) is solved by oracle.cg from e = E to a relative residual of
1e-11 (ground truth for comparisons at 1e-7); the stored values are the
oracle's effective-tensor columns <L e> and its true relative residual.
Calls only the oracle and the input generator, one process per solve.
Takes about an hour of CPU time (the 243^3 solves dominate).
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

TOL = 1e-11

# (n, kind, contrast, seed item): kind 0 disks, 1 ellipses, 2 laminate along axis 0
BATCH_CELLS = [
    (135, 0, 10.0, 1), (135, 2, 100.0, 2), (243, 1, 30.0, 3), (243, 0, 100.0, 4),
    (375, 0, 10.0, 5), (375, 1, 50.0, 6), (729, 0, 20.0, 7), (729, 1, 10.0, 8),
]


def batch_phase(n, kind, item):
    from paper_1004_1122_gb300 import microstructure as micro

    seed = micro.config_seed(4, 900 + item)
    if kind == 0:
        return micro.rsa_disks(n, 0.3, n / 40.0, n / 15.0, seed=seed)
    if kind == 1:
        return micro.random_ellipses(n, 0.3, n / 30.0, n / 12.0, 3.0, seed=seed)
    return micro.laminate(n, [0.7, 0.3], axis=0, seed=seed)


def case_input(case, item):
    """(phase, L, loads) of one case; shared by the writer and the GPU test."""
    import numpy as np

    from paper_1004_1122_gb300 import microstructure as micro

    if case == "c2_2187":
        phase = micro.rsa_disks(2187, 0.4, 8, 40, seed=micro.config_seed(2))
        return phase, micro.isotropic_table([1.0, 10.0], 2), np.eye(2)
    if case == "c3_243":
        phase = micro.boolean_spheres(243, 12.0, 0.25, seed=micro.config_seed(3))
        return phase, micro.isotropic_table([1.0, 10.0], 3), np.eye(3)
    n, kind, rho, it = BATCH_CELLS[item]
    return batch_phase(n, kind, it), micro.isotropic_table([1.0, rho], 2), np.eye(2)


def _solve(job):
    case, item, b = job
    import oracle

    phase, L, loads = case_input(case, item)
    L0 = oracle.reference_medium(L)
    x, info = oracle.cg(phase, L, L0, loads[b], tol=TOL, max_iter=20000)
    col = oracle.effective_tensor([x], phase, L)[:, 0]
    return {"case": case, "item": item, "load": b, "iters": int(info["iters"]), "status": info["status"],
            "rel_res_true": float(info["rel_res_true"]), "L_eff_col": col.tolist()}


def main():
    jobs = [("c3_243", 0, b) for b in range(3)]
    jobs += [("c2_2187", 0, b) for b in range(2)]
    jobs += [("batch", k, b) for k in range(len(BATCH_CELLS)) for b in range(2)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 4)) as pool:
        rows = pool.map(_solve, jobs, chunksize=1)
    out = {"source": "oracle.cg to relative residual 1e-11 (see module doc)", "tol": TOL,
           "batch_cells": BATCH_CELLS, "solves": rows}
    with open(os.path.join(HERE, "full_size_parity.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
