"""Oracle parity at the sizes where the compile-time-plan kernels run.

The float32 CG passes switch to kernels with a compile-time FFT plan when the
grid matches one (2187^2 one load per launch, 729^2 two loads per launch,
243^3 one or three loads per launch); every other grid runs the run-time-plan
kernels.  These tests solve on exactly those grids, assert through
fh_info.ct_plans that the compile-time kernels ran, and compare with the
oracle's solutions stored in tests/golden/full_size_parity.json (written by
tests/golden/make_full_size_parity.py, which calls only the oracle):

* 2187^2 RSA disks (the benchmark microstructure) at contrast 10, both loads:
  effective-tensor columns, and the oracle's own true residual of the
  returned field;
* a batch with cells of 135, 243, 375 and 729 per axis, two loads each, with
  the default and with the autotuned launch shapes;
* 243^3 Boolean spheres at contrast 10: the full tensor (three loads per
  launch) and one single-load solve.

Bars: solves run to a float64 true relative residual of 1e-9 and the field
error is at most kappa times that residual (kappa <= contrast <= 100), so
effective-tensor columns must agree with the oracle's (solved to 1e-11) within
1e-7 relative; the oracle's residual of a returned field must meet the
requested 1e-9 up to the 1e-11 accuracy of the library's double-float
residual.
"""
import json
import os

import numpy as np
import pytest

import oracle
from golden.make_full_size_parity import BATCH_CELLS, case_input

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-9
LEFF_BAR = 1e-7


def _gold():
    with open(os.path.join(HERE, "golden", "full_size_parity.json")) as f:
        g = json.load(f)
    return {(r["case"], r["item"], r["load"]): r for r in g["solves"]}


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_2187_refined_cg_matches_oracle():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    gold = _gold()
    phase, L, loads = case_input("c2_2187", 0)
    L0 = oracle.reference_medium(L)
    with fh.Solver(phase, L, precision="fp32_refined") as s:
        for b in range(2):
            x, col, info = s.solve(loads[b], tol=TOL, method="cg", max_iter=20000)
            assert info["status"] == "FH_OK", info
            assert info["ct_plans"] == [2187], info
            ref = gold[("c2_2187", 0, b)]
            assert ref["status"] == "converged"
            assert _rel(col, ref["L_eff_col"]) <= LEFF_BAR, (b, col, ref["L_eff_col"])
            e0 = oracle.operator.macroscopic_field(loads[b], phase.shape)
            r = e0 - oracle.apply_A(x.cpu().numpy(), phase, L, L0)
            rel = float(np.linalg.norm(r) / np.linalg.norm(e0))
            assert rel <= TOL + 1e-11, (b, rel)
            assert abs(rel - info["rel_res_true"]) <= 1e-11, (rel, info["rel_res_true"])


def test_uneven_batch_with_729_cells_matches_oracle():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    gold = _gold()
    cells = [case_input("batch", k) for k in range(len(BATCH_CELLS))]
    with fh.Batch([c[0] for c in cells], [c[1] for c in cells], nloads=2, precision="fp32_refined") as bt:
        runs = [bt.solve(np.eye(2), tol=TOL, method="cg", max_iter=20000)]
        # the tuned launch shapes (for the 729^2 cells, tile widths with their
        # own compiled Green-pass instances) must give the oracle's solutions too
        bt.autotune()
        runs.append(bt.solve(np.eye(2), tol=TOL, method="cg", max_iter=20000))
    for Leff, st, it, info in runs:
        assert np.all(st == 0), st
        assert 729 in info["ct_plans"], info
        for k in range(len(BATCH_CELLS)):
            for b in range(2):
                ref = gold[("batch", k, b)]["L_eff_col"]
                assert _rel(Leff[k, :, b], ref) <= LEFF_BAR, (BATCH_CELLS[k], b, Leff[k, :, b], ref)


def test_243_cube_full_tensor_and_single_load_match_oracle():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    gold = _gold()
    phase, L, loads = case_input("c3_243", 0)
    ref = np.stack([gold[("c3_243", 0, b)]["L_eff_col"] for b in range(3)], axis=1)
    with fh.Solver(phase, L, precision="fp32_refined") as s:
        Le, infos = s.solve_all(tol=TOL, method="cg", max_iter=20000)
        assert all(i["status"] == "FH_OK" for i in infos), infos
        assert infos[0]["ct_plans"] == [243], infos[0]
        assert _rel(Le, ref) <= LEFF_BAR, (Le, ref)
        _, col, info = s.solve(loads[1], tol=TOL, method="cg", max_iter=20000, want_field=False)
        assert info["status"] == "FH_OK" and info["ct_plans"] == [243], info
        assert _rel(col, ref[:, 1]) <= LEFF_BAR, (col, ref[:, 1])
