"""Batches of independent 2-D cells of uneven sizes (fh_batch_*) against the oracle.

Every (cell, load) result must match the oracle's solution of that cell alone
(per-cell reference medium, Eq. opt_ref) at the same bars as single solves:
float64 <= 1e-10 relative on the effective-tensor column, float32 + float64
refinement <= 1e-6.
"""
import numpy as np
import pytest

import oracle
from paper_1004_1122_gb300 import microstructure as micro

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu


def _cells():
    cells = []
    rng = np.random.default_rng(77)
    specs = [(27, 27), (27, 27), (45, 45), (27, 27), (81, 45), (45, 45), (27, 27), (81, 45), (15, 21)]
    for k, N in enumerate(specs):
        kind = k % 3
        seed = micro.config_seed(4, k)
        if kind == 0:
            ph = micro.rsa_disks(N[0], 0.3, 2, 4, seed=seed) if N[0] == N[1] else \
                micro.laminate(N, [0.5, 0.5], axis=1, seed=seed)
        elif kind == 1:
            ph = micro.laminate(N, [0.4, 0.6], axis=k % 2, seed=seed)
        else:
            ph = micro.random_ellipses(N[0], 0.3, 2, 5, 2.0, seed=seed) if N[0] == N[1] else \
                micro.centred_disk(N, 0.3)
        rho = float(10 ** rng.uniform(1, 3))
        cells.append((ph, micro.isotropic_table([1.0, rho], 2)))
    return cells


def _oracle_cols(cells, tol):
    out = []
    for ph, L in cells:
        L0 = oracle.reference_medium(L)
        xs = [oracle.cg(ph, L, L0, np.eye(2)[b], tol=tol, max_iter=5000)[0] for b in range(2)]
        out.append(oracle.effective_tensor(xs, ph, L))
    return np.array(out)  # [cell, a, load]


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-12, 1e-10), ("fp32_refined", 1e-10, 1e-6)])
def test_batch_matches_oracle_per_cell(prec, tol, bar):
    cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    cells = _cells()
    ref = _oracle_cols(cells, 1e-13)
    with fh.Batch([c[0] for c in cells], [c[1] for c in cells], nloads=2, precision=prec) as b:
        Leff, st, it, info = b.solve(np.eye(2), tol=tol, method="cg", max_iter=20000)
    assert np.all(st == 0), st
    assert info["rel_res_true"] <= tol
    err = np.max(np.abs(Leff - ref), axis=(1, 2)) / np.max(np.abs(ref), axis=(1, 2))
    assert np.all(err < bar), err
    assert info["launches"] > 0


def test_batch_autotune_keeps_parity():
    """fh_batch_autotune re-plans every size group; the results stay those of the oracle."""
    cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    cells = _cells()
    ref = _oracle_cols(cells, 1e-13)
    with fh.Batch([c[0] for c in cells], [c[1] for c in cells], nloads=2, precision="fp32_refined") as b:
        before, after = b.autotune()
        assert 0.0 < after <= before * 1.05
        Leff, st, it, info = b.solve(np.eye(2), tol=1e-10, method="cg", max_iter=20000)
    assert np.all(st == 0), st
    err = np.max(np.abs(Leff - ref), axis=(1, 2)) / np.max(np.abs(ref), axis=(1, 2))
    assert np.all(err < 1e-6), err


@pytest.mark.parametrize("method", ["bicg", "fixed_point"])
def test_batch_other_methods_fp64(method):
    cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    cells = _cells()[:4]
    ref = _oracle_cols(cells, 1e-13)
    with fh.Batch([c[0] for c in cells], [c[1] for c in cells], nloads=2, precision="fp64") as b:
        Leff, st, it, info = b.solve(np.eye(2), tol=1e-11, method=method, max_iter=200000)
    assert np.all(st == 0), st
    err = np.max(np.abs(Leff - ref)) / np.max(np.abs(ref))
    assert err < 1e-9


def test_batch_single_load_and_iteration_cap():
    cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    cells = _cells()[:5]
    with fh.Batch([c[0] for c in cells], [c[1] for c in cells], nloads=1, precision="fp32_refined") as b:
        # a diagonal load is non-trivial for every cell (laminates included)
        E = np.array([0.6, 0.8])
        Leff, st, it, info = b.solve(E, tol=1e-12, max_iter=2)
        assert np.all(st == 6)  # FH_ERR_NOT_CONVERGED
        Leff, st, it, info = b.solve(E, tol=1e-8)
        assert np.all(st == 0)
    ref = _oracle_cols(cells, 1e-13) @ E
    assert np.max(np.abs(Leff[:, :, 0] - ref)) / np.max(np.abs(ref)) < 1e-5


def test_batch_rejects_bad_cells():
    cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    with pytest.raises(fh.FhError):
        fh.Batch([np.zeros((8, 9), np.uint8)], [micro.isotropic_table([1.0], 2)])
    with pytest.raises(fh.FhError):
        fh.Batch([np.full((9, 9), 2, np.uint8)], [micro.isotropic_table([1.0, 2.0], 2)])
