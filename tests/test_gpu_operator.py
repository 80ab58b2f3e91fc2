"""Parity of fh_apply (CUDA) with the oracle's collocation operator, element by element.

Tolerance (derived from the arithmetic): the product is e + F^-1 Gamma0 F (dL e);
each FFT stage adds O(u) relative error, with u = 2^-53 (float64) or 2^-24
(float32), and the FFT error is relative to the size of the polarisation
dL e, so the bound is  |err| <= c * u * log2|N| * (1 + max|dL|) * max|e|.
We use c * log2|N| <= 64, i.e. 64 u (1 + max|dL|) max|e|.
"""
import numpy as np
import pytest

import oracle
from paper_1004_1122_gb300 import microstructure as micro

from gpu_util import cuda_or_skip, spd

pytestmark = pytest.mark.gpu

U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}

CASES_2D = [
    ((81, 81), (1.0, 1.0)),        # 3^4, C1 grid
    ((27, 45), (1.0, 2.5)),        # non-square, 3^3 x 3^2 5, non-unit cell
    ((135, 21), (0.5, 1.0)),       # 3^3 5 x 3 7
    ((375, 9), (1.0, 1.0)),        # 3 5^3
    ((243, 729), (1.0, 1.0)),      # several tiles and a ragged tail
    ((7, 49), (1.0, 1.0)),         # 7^2
    ((15, 21), (1.0, 1.0)),        # single-stage radix-15 columns, one thread per FFT
    ((21, 15), (1.0, 1.0)),
    ((15, 15), (1.0, 1.0)),
    ((25, 9), (1.0, 1.0)),
    ((5, 7), (1.0, 1.0)),
    ((3, 3), (1.0, 1.0)),          # smallest odd grid: one radix-3 stage per axis
    ((3, 2187), (1.0, 1.0)),       # a single row of tiles along axis 0, long lines
    ((17, 17), (1.0, 1.0)),        # radix-17 stages (extended-radix plans)
    ((255, 255), (1.0, 1.0)),      # 3 * 5 * 17: the model-problem grid of Section 3
    ((51, 85), (1.0, 2.0)),        # 3 * 17 x 5 * 17, non-unit cell
    ((11, 13), (1.0, 1.0)),        # radix 11 and 13
    ((143, 9), (1.0, 1.0)),        # 11 * 13 along axis 0, a standard row axis
    ((8, 8), (1.0, 1.0)),          # even axes: radix 2/4/8, Nyquist frequencies
    ((6, 10), (1.0, 2.0)),
    ((16, 12), (1.0, 1.0)),
    ((256, 256), (1.0, 1.0)),      # 2^8: radix-16 stages
    ((3, 32), (1.0, 1.0)),         # even line, odd column
    ((30, 3), (1.0, 1.0)),         # even column, odd line
]
CASES_3D = [
    ((9, 15, 27), (1.0, 1.0, 1.0)),
    ((27, 27, 27), (1.0, 0.5, 2.0)),
    ((5, 21, 45), (1.0, 1.0, 1.0)),
    ((3, 5, 7), (1.0, 1.0, 1.0)),  # smallest mixed-radix 3-D grid
    ((243, 3, 9), (1.0, 1.0, 1.0)),
    ((17, 11, 13), (1.0, 1.0, 1.0)),  # every axis extended
    ((9, 17, 15), (1.0, 1.0, 1.0)),   # only the middle axis extended
    ((8, 6, 10), (1.0, 1.0, 1.0)),    # every axis even
    ((5, 4, 9), (1.0, 1.0, 1.0)),     # only the middle axis even
]


def _problem(N, seed, nphase=3, aniso=True):
    rng = np.random.default_rng(seed)
    d = len(N)
    phase = rng.integers(0, nphase, size=N).astype(np.uint8)
    if aniso:
        L = np.stack([spd(rng, d) for _ in range(nphase)])
        L0 = spd(rng, d, 1.0, 3.0)
    else:
        L = micro.isotropic_table(rng.uniform(1, 20, size=nphase), d)
        L0 = oracle.reference_medium(L)
    e = rng.normal(size=(d,) + tuple(N))
    return phase, L, L0, e


def _check(N, Y, prec, transpose, seed):
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase, L, L0, e = _problem(N, seed)
    ref = (oracle.apply_AT if transpose else oracle.apply_A)(e, phase, L, L0, Y)
    dt = torch.float64 if prec == "fp64" else torch.float32
    ctx_prec = "fp64" if prec == "fp64" else "fp32"
    with fh.Solver(phase, L, L0=L0, Y=Y, precision=ctx_prec) as s:
        et = torch.from_numpy(e).to(dt).cuda()
        got = s.apply(et, transpose=transpose).double().cpu().numpy()
    dl = np.max(np.abs(L - L0[None]))
    ein = e if prec == "fp64" else e.astype(np.float32).astype(np.float64)
    ref = (oracle.apply_AT if transpose else oracle.apply_A)(ein, phase, L, L0, Y)
    tol = 64 * U[prec] * (1.0 + dl) * np.max(np.abs(e)) * (4.0 if prec == "fp32" else 1.0)
    err = np.max(np.abs(got - ref))
    assert err <= tol, (N, prec, transpose, err, tol)


@pytest.mark.parametrize("N,Y", CASES_2D)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("transpose", [False, True])
def test_apply_2d(N, Y, prec, transpose):
    _check(N, Y, prec, transpose, seed=7 * N[0] + 13 * N[1] + 3 * (prec == "fp32") + int(transpose))


@pytest.mark.parametrize("N,Y", CASES_3D)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("transpose", [False, True])
def test_apply_3d(N, Y, prec, transpose):
    _check(N, Y, prec, transpose, seed=7 * N[0] + 13 * N[1] + 17 * N[2] + 3 * (prec == "fp32") + int(transpose))


def test_apply_in_place_and_homogeneous():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    N = (45, 63)
    phase = np.zeros(N, dtype=np.uint8)
    L = np.array([[[3.0, 0.5], [0.5, 2.0]]])
    with fh.Solver(phase, L, precision="fp64") as s:
        e = torch.zeros((2,) + N, dtype=torch.float64, device="cuda")
        e[0] = 0.7
        e[1] = -0.2
        keep = e.clone()
        s.apply(e, out=e)
        assert torch.max(torch.abs(e - keep)).item() < 1e-14


def test_apply_full_size_2187():
    """C2 grid 2187^2 at its own launch configuration, all outputs compared."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.rsa_disks(2187, 0.4, 8, 40, seed=micro.config_seed(2))
    L = micro.isotropic_table([1.0, 100.0], 2)
    L0 = oracle.reference_medium(L)
    rng = np.random.default_rng(5)
    e = rng.normal(size=(2, 2187, 2187))
    for prec in ("fp32", "fp64"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        with fh.Solver(phase, L, precision=prec) as s:
            got = s.apply(torch.from_numpy(e).to(dt).cuda()).double().cpu().numpy()
        ein = e if prec == "fp64" else e.astype(np.float32).astype(np.float64)
        ref = oracle.apply_A(ein, phase, L, L0)
        tol = 64 * U[prec] * (1.0 + np.max(np.abs(L - L0[None]))) * np.max(np.abs(e)) * (4.0 if prec == "fp32" else 1.0)
        assert np.max(np.abs(got - ref)) <= tol, (prec, np.max(np.abs(got - ref)), tol)


def test_autotune_keeps_parity():
    """fh_autotune rebuilds the pipeline with another launch shape; the product is unchanged."""
    torch = cuda_or_skip()
    import os
    import tempfile

    from paper_1004_1122_gb300 import fh

    phase, L, L0, e = _problem((243, 135), seed=21)
    old = os.environ.get("FH_TUNE_CACHE")
    with tempfile.TemporaryDirectory() as tmp:
        os.environ["FH_TUNE_CACHE"] = os.path.join(tmp, "tune.txt")
        try:
            with fh.Solver(phase, L, L0=L0, precision="fp32") as s:
                et = torch.from_numpy(e).float().cuda()
                before = s.apply(et).double().cpu().numpy()
                ms0, ms1 = s.autotune("fp32")
                after = s.apply(et).double().cpu().numpy()
            assert ms1 <= ms0 * 1.0001
            assert os.path.getsize(os.environ["FH_TUNE_CACHE"]) > 0
            with fh.Solver(phase, L, L0=L0, precision="fp32") as s2:  # starts from the cache
                again = s2.apply(et).double().cpu().numpy()
        finally:
            if old is None:
                del os.environ["FH_TUNE_CACHE"]
            else:
                os.environ["FH_TUNE_CACHE"] = old
    ein = e.astype(np.float32).astype(np.float64)
    ref = oracle.apply_A(ein, phase, L, L0)
    tol = 64 * U["fp32"] * 4 * (1.0 + np.max(np.abs(L - L0[None]))) * np.max(np.abs(e))
    for got in (before, after, again):
        assert np.max(np.abs(got - ref)) <= tol


def test_one_node_axis_is_refused():
    """An axis of one node (a 1-D problem embedded in 2-D) is outside the
    contract (every axis odd and >= 3): fh_create returns FH_ERR_ARG before any
    allocation or launch."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = np.zeros((1, 15), dtype=np.uint8)
    L = micro.isotropic_table([1.0], 2)
    with pytest.raises(fh.FhError) as ex:
        fh.Solver(phase, L, precision="fp64")
    assert ex.value.status == 1  # FH_ERR_ARG
