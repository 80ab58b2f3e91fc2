"""Parity of fh_solve (CUDA) with the oracle's solvers.

Bars (the accuracy targets of the method): float64 path <= 1e-10 relative error of the
field and of L_eff against the oracle's tight solution; float32 + float64
refinement <= 1e-6.  Comparisons are made at tolerances where the iteration
error is below those bars (the field error is at most kappa times the
relative residual, kappa <= contrast).
"""
import numpy as np
import pytest

import oracle
from paper_1004_1122_gb300 import microstructure as micro

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _c1():
    phase = micro.centred_disk(81, 0.3)
    L = micro.isotropic_table([1.0, 10.0], 2)
    return phase, L, oracle.reference_medium(L)


def test_c1_fp64_cg_matches_oracle_iterates():
    """C1: 81^2 centred disk, vf 0.3, L = 1 / 10, L0 = 5.5 I, E = (1, 0), FP64 CG to 1e-8.
    Same algorithm, same start: the iteration counts agree and the residual
    histories agree to round-off."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase, L, L0 = _c1()
    xo, io = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-8)
    with fh.Solver(phase, L, precision="fp64") as s:
        x, col, info = s.solve([1.0, 0.0], tol=1e-8, method="cg", history=512)
    assert info["status"] == "FH_OK"
    assert info["iters"] == io["iters"]
    h = info["history"]
    assert np.allclose(h, io["history"][: len(h)], rtol=1e-9, atol=1e-15)
    assert _rel_l2(x.cpu().numpy(), xo) < 1e-10
    assert info["rel_res_true"] <= 1e-8


@pytest.mark.parametrize("method", ["cg", "bicg", "fixed_point"])
def test_fp64_methods_reach_oracle_solution(method):
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.rsa_disks(135, 0.35, 6, 14, seed=micro.config_seed(2, 7))
    L = micro.isotropic_table([1.0, 20.0], 2)
    L0 = oracle.reference_medium(L)
    xo, io = oracle.cg(phase, L, L0, [0.0, 1.0], tol=1e-13)
    with fh.Solver(phase, L, precision="fp64") as s:
        x, col, info = s.solve([0.0, 1.0], tol=1e-12, method=method, max_iter=20000)
    assert info["status"] == "FH_OK", info
    assert _rel_l2(x.cpu().numpy(), xo) < 1e-10
    Lo = oracle.effective_tensor([xo], phase, L)[:, 0]
    assert np.max(np.abs(col - Lo)) / np.max(np.abs(Lo)) < 1e-10


@pytest.mark.parametrize("method", ["cg", "bicg", "fixed_point"])
def test_fp32_refined_meets_1e6(method):
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.rsa_disks(243, 0.4, 8, 20, seed=micro.config_seed(2, 3))
    rho = 100.0
    L = micro.isotropic_table([1.0, rho], 2)
    L0 = oracle.reference_medium(L)
    xo, _ = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-13)
    with fh.Solver(phase, L, precision="fp32_refined") as s:
        x, col, info = s.solve([1.0, 0.0], tol=1e-10, method=method, max_iter=50000)
    assert info["status"] == "FH_OK", info
    assert info["outer_iters"] >= 1
    assert _rel_l2(x.cpu().numpy(), xo) < 1e-6
    Lo = oracle.effective_tensor([xo], phase, L)[:, 0]
    assert np.max(np.abs(col - Lo)) / np.max(np.abs(Lo)) < 1e-6


@pytest.mark.parametrize("N,rho", [(81, 1e2), (243, 1e4), (135, 1e3)])
def test_refined_true_residual_is_float64_accurate(N, rho):
    """The outer residual of the refined solves (float64 fields, Green pass in
    double-float arithmetic) equals the oracle's float64 residual of the
    returned field to 1e-11 |e0|; a float32-accuracy Green pass would miss by
    ~1e-7.  (The two-load Green pass of fh_solve_all and of the batches is
    covered by their L_eff parity tests.)"""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.rsa_disks(N, 0.35, N / 40, N / 20, seed=micro.config_seed(5, N))
    L = micro.isotropic_table([1.0, rho], 2)
    L0 = oracle.reference_medium(L)
    E = [0.6, -0.8]
    with fh.Solver(phase, L, precision="fp32_refined") as s:
        x, _, info = s.solve(E, tol=1e-6, method="cg", max_iter=50000)
    assert info["status"] == "FH_OK", info
    assert info["outer_iters"] >= 1
    e0 = oracle.operator.macroscopic_field(E, (N, N))
    r = e0 - oracle.apply_A(x.cpu().numpy(), phase, L, L0)
    rel_o = float(np.linalg.norm(r) / np.linalg.norm(e0))
    assert 0.0 < rel_o <= 1e-6
    assert abs(info["rel_res_true"] - rel_o) <= 1e-11, (info["rel_res_true"], rel_o)


def test_fp32_plain_converges():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase, L, L0 = _c1()
    xo, _ = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-13)
    with fh.Solver(phase, L, precision="fp32") as s:
        x, col, info = s.solve([1.0, 0.0], tol=1e-5, method="cg")
    assert info["status"] == "FH_OK", info
    assert _rel_l2(x.cpu().numpy(), xo) < 1e-4


def test_3d_spheres_fp64_and_refined():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.boolean_spheres(27, 4.0, 0.25, seed=micro.config_seed(3, 1))
    L = micro.isotropic_table([1.0, 50.0], 3)
    L0 = oracle.reference_medium(L)
    xo, _ = oracle.cg(phase, L, L0, [0.0, 0.0, 1.0], tol=1e-13)
    for prec, tol, bar in (("fp64", 1e-12, 1e-10), ("fp32_refined", 1e-10, 1e-6)):
        with fh.Solver(phase, L, precision=prec) as s:
            x, col, info = s.solve([0.0, 0.0, 1.0], tol=tol, method="cg")
        assert info["status"] == "FH_OK", (prec, info)
        assert _rel_l2(x.cpu().numpy(), xo) < bar, prec


def test_effective_tensor_solve_all_symmetric_bounds():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.centred_disk(81, 0.45)
    f2 = micro.digital_fraction(phase)
    rho = 30.0
    L = micro.isotropic_table([1.0, rho], 2)
    L0 = oracle.reference_medium(L)
    with fh.Solver(phase, L, precision="fp64") as s:
        Le, infos = s.solve_all(tol=1e-12)
    xs = [oracle.cg(phase, L, L0, np.eye(2)[b], tol=1e-13)[0] for b in range(2)]
    Lo = oracle.effective_tensor(xs, phase, L)
    assert np.max(np.abs(Le - Lo)) / np.max(np.abs(Lo)) < 1e-10
    assert abs(Le[0, 1] - Le[1, 0]) < 1e-9 * Le[0, 0]
    voigt = (1 - f2) + f2 * rho
    reuss = 1.0 / ((1 - f2) + f2 / rho)
    assert reuss < Le[0, 0] < voigt


def test_homogeneous_zero_iterations_exact():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    N = (45, 45)
    phase = np.zeros(N, dtype=np.uint8)
    L = np.array([[[4.0, 1.0], [1.0, 3.0]]])
    with fh.Solver(phase, L, precision="fp64") as s:
        x, col, info = s.solve([0.3, -0.7], tol=1e-12)
    assert info["status"] == "FH_OK" and info["iters"] == 0
    xe = x.cpu().numpy()
    assert np.all(xe[0] == 0.3) and np.all(xe[1] == -0.7)
    assert np.allclose(col, L[0] @ np.array([0.3, -0.7]), rtol=1e-14)


def test_laminate_closed_form_gpu():
    """Layers normal to axis 0: harmonic mean across, arithmetic along (exact)."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    N = (81, 45)
    phase = micro.laminate(N, [1 / 3, 2 / 3], axis=0, seed=4)
    c = np.array([1.0, 10.0])
    L = micro.isotropic_table(c, 2)
    frac = np.bincount(phase[:, 0], minlength=2) / 81
    harm, arith = 1.0 / np.sum(frac / c), np.sum(frac * c)
    for prec in ("fp64", "fp32_refined"):
        with fh.Solver(phase, L, precision=prec) as s:
            Le, _ = s.solve_all(tol=1e-11)
        bar = 1e-10 if prec == "fp64" else 1e-6
        assert np.max(np.abs(Le - np.diag([harm, arith]))) / arith < bar, (prec, Le)


def test_reference_medium_independence_gpu():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.centred_disk(81, 0.4)
    rho = 50.0
    L = micro.isotropic_table([1.0, rho], 2)
    cols = []
    for omega in (0.25, 0.5, 0.75):
        L0 = (1 - omega + rho * omega) * np.eye(2)
        with fh.Solver(phase, L, L0=L0, precision="fp64") as s:
            _, col, info = s.solve([1.0, 0.0], tol=1e-12)
        assert info["status"] == "FH_OK"
        cols.append(col)
    assert np.max(np.abs(np.array(cols) - cols[1])) < 1e-10 * abs(cols[1][0])


def test_not_converged_and_infinite_contrast_status():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase, L, L0 = _c1()
    with fh.Solver(phase, L, precision="fp64") as s:
        _, _, info = s.solve([1.0, 0.0], tol=1e-12, max_iter=3)
    assert info["status"] == "FH_ERR_NOT_CONVERGED" and info["iters"] == 3
    Lr = micro.isotropic_table([1.0, 1e12], 2)
    with fh.Solver(phase, Lr, precision="fp64") as s:
        _, _, info = s.solve([1.0, 0.0], tol=1e-8, max_iter=200)
    assert info["status"] in ("FH_ERR_NOT_CONVERGED", "FH_ERR_BREAKDOWN")


def test_eta_e_matches_oracle():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.centred_disk(45, 0.3)
    L = micro.isotropic_table([1.0, 10.0], 2)
    L0 = oracle.reference_medium(L)
    rng = np.random.default_rng(3)
    e = rng.normal(size=(2, 45, 45))
    with fh.Solver(phase, L, precision="fp64") as s:
        got = s.eta_e(torch.from_numpy(e).cuda())
        x, _, info = s.solve([1.0, 0.0], tol=1e-12, eta_e=True)
        _, _, info_plain = s.solve([1.0, 0.0], tol=1e-12)
    assert abs(got - oracle.eta_e(e, phase, L)) < 1e-12 * oracle.eta_e(e, phase, L)
    assert info["eta_e"] < 1e-9
    assert np.isnan(info_plain["eta_e"])


def test_invalid_inputs_rejected():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    with pytest.raises(fh.FhError) as ex:  # 19 has no FFT plan (primes 2 .. 17 only)
        fh.Solver(np.zeros((19, 9), np.uint8), micro.isotropic_table([1.0], 2))
    assert ex.value.status == 9  # FH_ERR_UNSUPPORTED
    with pytest.raises(fh.FhError):
        fh.Solver(np.zeros((9, 9), np.uint8), np.array([[[1.0, 2.0], [2.0, 1.0]]]))
    with pytest.raises(fh.FhError):
        fh.Solver(np.full((9, 9), 3, np.uint8), micro.isotropic_table([1.0, 2.0], 2))


@pytest.mark.parametrize("N,axis", [((27, 27), 1), ((81, 45), 0), ((15, 21), None)])
def test_fp32_refined_reaches_tight_tolerance_on_noise_dominated_corrections(N, axis):
    """Once the float32 solution is accurate, the float64 residual is rounding
    noise with a large component outside the compatible fields, where I + B is
    not symmetric; the refinement starts each inner CG at the exact complement
    part (I - Q) r of the correction so that CG only sees compatible fields."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase = micro.laminate(N, [0.4, 0.6], axis=axis, seed=3) if axis is not None else micro.centred_disk(N, 0.3)
    L = micro.isotropic_table([1.0, 55.0], 2)
    L0 = oracle.reference_medium(L)
    E = np.array([0.6, 0.8])
    xo, _ = oracle.cg(phase, L, L0, E, tol=1e-13)
    for method in ("cg", "bicg"):
        with fh.Solver(phase, L, precision="fp32_refined") as s:
            x, col, info = s.solve(E, tol=1e-10, method=method, max_iter=5000)
        assert info["status"] == "FH_OK", (method, info)
        assert _rel_l2(x.cpu().numpy(), xo) < 1e-6


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-12, 1e-10), ("fp32_refined", 1e-10, 1e-6)])
def test_3d_full_tensor_loads_batched(prec, tol, bar, tmp_path, monkeypatch):
    """Config-3 path at a small size: all three unit loads in every launch
    (fh_solve_all), Boolean spheres, against three oracle solves; for float32
    + refinement also after tuning the all-loads pipeline (fh_autotune_loads)."""
    torch = cuda_or_skip()
    monkeypatch.setenv("FH_TUNE_CACHE", str(tmp_path / "tune.txt"))
    from paper_1004_1122_gb300 import fh

    phase = micro.boolean_spheres(27, 3.0, 0.25, seed=micro.config_seed(3, 2))
    L = micro.isotropic_table([1.0, 1e3], 3)
    L0 = oracle.reference_medium(L)
    xs = [oracle.cg(phase, L, L0, np.eye(3)[b], tol=1e-13, max_iter=3000)[0] for b in range(3)]
    Lo = oracle.effective_tensor(xs, phase, L)
    with fh.Solver(phase, L, precision=prec) as s:
        Le, infos = s.solve_all(tol=tol, max_iter=20000)
        tuned = None
        if prec == "fp32_refined":
            # tune the all-loads pipeline (tuning cache in a temporary file), solve again
            before, after = s.autotune(loads=True)
            assert after <= before * 1.05
            tuned, tinfos = s.solve_all(tol=tol, max_iter=20000)
            assert all(i["status"] == "FH_OK" for i in tinfos), tinfos
    assert all(i["status"] == "FH_OK" for i in infos), infos
    assert np.max(np.abs(Le - Lo)) / np.max(np.abs(Lo)) < bar
    assert np.max(np.abs(Le - Le.T)) < 10 * bar * np.max(np.abs(Lo))
    if tuned is not None:
        assert np.max(np.abs(tuned - Lo)) / np.max(np.abs(Lo)) < bar


def _x1(rho, omega):
    """Section 3's model problem: one centred disk at volume fraction 0.5 on
    255^2 nodes, matrix L = I, particle L = rho I, reference medium
    L0(omega) = (1 - omega + rho omega) I (Eq. ref_media_choice)."""
    phase = micro.centred_disk(255, 0.5)
    L = micro.isotropic_table([1.0, rho], 2)
    L0 = (1.0 - omega + rho * omega) * np.eye(2)
    return phase, L, L0


@pytest.mark.parametrize("method", ["cg", "bicg", "fixed_point"])
def test_model_problem_255_fp64_matches_oracle(method):
    """Radix-17 plans on the paper's own grid: float64 CG, BiCG and the
    fixed-point scheme reach the oracle's solution to 1e-10."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    # omega = 0.75: l0 = 7.75 > rho / 2, where the fixed-point series converges
    phase, L, L0 = _x1(10.0, 0.75)
    xo, io = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-13)
    with fh.Solver(phase, L, L0=L0, precision="fp64") as s:
        x, col, info = s.solve([1.0, 0.0], tol=1e-12, method=method, max_iter=20000)
    assert info["status"] == "FH_OK", info
    assert _rel_l2(x.cpu().numpy(), xo) < 1e-10
    if method == "cg":  # same algorithm, same start, same stopping tolerance
        _, i12 = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-12)
        assert abs(info["iters"] - i12["iters"]) <= 1, (info["iters"], i12["iters"])


def test_model_problem_255_refined_and_full_tensor():
    """Float32 iterations with float64 refinement on 255^2 (the float64
    residual runs float64 FFTs there), and fh_solve_all, which solves the loads
    of an extended-radix grid one by one."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase, L, L0 = _x1(100.0, 0.5)
    xo, _ = oracle.cg(phase, L, L0, [0.0, 1.0], tol=1e-13)
    with fh.Solver(phase, L, L0=L0, precision="fp32_refined") as s:
        x, col, info = s.solve([0.0, 1.0], tol=1e-10, method="cg", max_iter=20000)
        assert info["status"] == "FH_OK", info
        assert _rel_l2(x.cpu().numpy(), xo) < 1e-6
        Le, infos = s.solve_all(tol=1e-10, method="cg", max_iter=20000)
    assert all(i["status"] == "FH_OK" for i in infos)
    x0, _ = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-13)
    Lo = oracle.effective_tensor([x0, xo], phase, L)
    assert np.max(np.abs(Le - Lo)) / np.max(np.abs(Lo)) < 1e-6


@pytest.mark.parametrize("method", ["cg", "bicg", "fixed_point"])
def test_eta_histories_match_oracle(method):
    """Per-iteration norms of Section 3 on the C1 problem (float64): the
    eta_r history (Eq. errR_def, one entry per step) against the oracle's, and
    the eta_e history (Eq. errE_def of every iterate, one extra pass set per
    iteration) against oracle.eta_e of the oracle's iterates."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase, L, L0 = _c1()
    E = [1.0, 0.0]
    tol = 1e-6
    with fh.Solver(phase, L, precision="fp64") as s:
        _, _, info = s.solve(E, tol=tol, method=method, max_iter=5000, history=4096, norms=True)
    assert info["status"] == "FH_OK", info
    n = info["iters"]
    er, ee = info["eta_r_history"], info["eta_e_history"]
    assert len(er) == n and len(ee) == n + 1, (len(er), len(ee), n)
    solver = {"cg": oracle.cg, "bicg": oracle.bicg, "fixed_point": oracle.fixed_point}[method]
    _, io = solver(phase, L, L0, E, tol=1e-30, max_iter=n)
    k = min(n, 12)  # round-off grows along the iteration; the leading steps agree tightly
    assert np.allclose(er[:k], io["eta_r_history"][:k], rtol=1e-8, atol=0), (er[:k], io["eta_r_history"][:k])
    for m in sorted({0, 1, 2, min(5, n)}):
        xm, _ = solver(phase, L, L0, E, tol=1e-30, max_iter=m)
        # the fixed point's iterate after m steps is the oracle's with max_iter = m - 1
        if method == "fixed_point":
            xm = oracle.operator.macroscopic_field(E, phase.shape) if m == 0 else \
                solver(phase, L, L0, E, tol=1e-30, max_iter=m - 1)[0]
        ref = oracle.eta_e(xm, phase, L)
        assert abs(ee[m] - ref) <= 1e-9 * max(ref, 1e-300), (m, ee[m], ref)


@pytest.mark.parametrize("N", [(64, 48), (16, 12, 20)])
def test_even_grids_match_oracle(N):
    """Even axes (Green operator zero on the Nyquist frequencies, the reading
    the oracle's dense and equilibrium forms agree on): float64 CG and float32
    CG with float64 refinement reach the oracle's solution."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    rng = np.random.default_rng(sum(N))
    d = len(N)
    phase = (rng.random(N) < 0.35).astype(np.uint8)
    L = micro.isotropic_table([1.0, 30.0], d)
    L0 = oracle.reference_medium(L)
    E = np.eye(d)[0]
    xo, _ = oracle.cg(phase, L, L0, E, tol=1e-13)
    with fh.Solver(phase, L, precision="fp64") as s:
        x, col, info = s.solve(E, tol=1e-12, method="cg", max_iter=20000)
    assert info["status"] == "FH_OK", info
    assert _rel_l2(x.cpu().numpy(), xo) < 1e-10
    with fh.Solver(phase, L, precision="fp32_refined") as s:
        x, col, info = s.solve(E, tol=1e-10, method="cg", max_iter=20000)
    assert info["status"] == "FH_OK", info
    assert _rel_l2(x.cpu().numpy(), xo) < 1e-6
    eta = oracle.eta_e(xo, phase, L)
    assert eta < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cg_deferred_x_steps_are_exact(precision):
    """CG settles the x step of every second iteration together with the next
    one (x += alpha_k p_k, then += alpha_{k+1} p_{k+1}, in one pass) and owes
    the last step when it stops after an even iteration.  With the per-iteration
    norms requested x moves every iteration instead.  Both orders of work give
    the same float sums, so the fields and iteration counts must agree exactly,
    whichever parity the stopping iteration has."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    phase, L, _ = _c1()
    E = [1.0, 0.0]
    parities = set()
    with fh.Solver(phase, L, precision=precision) as s:
        for tol in (1e-3, 5e-4, 2e-4, 1e-4, 3e-5, 1e-5):
            x1, c1, i1 = s.solve(E, tol=tol, method="cg", max_iter=5000)
            x2, c2, i2 = s.solve(E, tol=tol, method="cg", max_iter=5000, history=4096, norms=True)
            assert i1["status"] == "FH_OK" and i2["status"] == "FH_OK", (i1, i2)
            assert i1["iters"] == i2["iters"], (tol, i1["iters"], i2["iters"])
            assert torch.equal(x1, x2), (tol, float((x1 - x2).abs().max()))
            assert np.array_equal(c1, c2), (tol, c1, c2)
            parities.add(i1["iters"] % 2)
    assert parities == {0, 1}, parities
