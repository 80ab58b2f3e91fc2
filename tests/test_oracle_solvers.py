"""Pins for the oracle's solvers and derived quantities (CPU only).

Closed forms (homogeneous, laminate), two independent dense formulations,
reference-medium independence, the bounds of Eq. (conv_rate), the CG == BiCG
observation of Section 3.1, Voigt/Reuss and Hashin-Shtrikman bounds on the
effective tensor, and the equilibrium norm of Eq. (errE_def).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1004_1122_gb300 import microstructure as micro

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spd(rng, d, lo=0.5, hi=5.0):
    q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    return q @ np.diag(rng.uniform(lo, hi, size=d)) @ q.T


@pytest.mark.parametrize("N,Y", [((15, 9), (1.0, 1.5)), ((5, 7, 5), (1.0, 1.0, 2.0)),
                                 ((8, 6), (1.0, 1.0)), ((6, 9), (1.5, 1.0)),   # even axes
                                 ((4, 6, 5), (1.0, 1.0, 1.0))])
def test_lu_equals_potential_formulation(N, Y):
    """Dense LU of Eq. (linear_system) == the L0-free equilibrium form (module doc of
    oracle.dense), anisotropic phases, both loads."""
    rng = np.random.default_rng(2)
    d = len(N)
    phase = rng.integers(0, 3, size=N).astype(np.uint8)
    L = np.stack([_spd(rng, d) for _ in range(3)])
    L0 = oracle.reference_medium(L)
    for b in range(d):
        E = np.eye(d)[b]
        x_lu = dense.solve_lu(phase, L, L0, E, Y)
        x_pot = dense.solve_potential(phase, L, E, Y)
        assert np.max(np.abs(x_lu - x_pot)) < 1e-11


@pytest.mark.parametrize("method", ["cg", "bicg", "fixed_point"])
def test_iterative_solvers_reach_dense_solution(method):
    phase = micro.rsa_disks(21, 0.35, 2, 4, seed=3)
    L = micro.isotropic_table([1.0, 8.0], 2)
    L0 = oracle.reference_medium(L)
    E = np.array([0.6, -0.8])
    x_lu = dense.solve_lu(phase, L, L0, E)
    x, info = oracle.solve(phase, L, L0, E, method=method, tol=1e-12, max_iter=5000)
    assert info["status"] == "converged"
    assert info["rel_res_true"] < 1e-11
    assert np.max(np.abs(x - x_lu)) < 1e-10


def test_reference_medium_independence():
    """Any SPD L0 gives the same discrete field (Section 3.1 'insensitive to the
    reference medium'; exact, since the solution is characterised without L0)."""
    rng = np.random.default_rng(4)
    phase = micro.centred_disk(15, 0.4)
    rho = 20.0
    L = micro.isotropic_table([1.0, rho], 2)
    E = np.array([1.0, 0.0])
    ref = dense.solve_lu(phase, L, oracle.reference_medium(L), E)
    for omega in (0.25, 0.5, 0.75):
        L0 = (1.0 - omega + rho * omega) * np.eye(2)  # Eq. (ref_media_choice)
        assert np.max(np.abs(dense.solve_lu(phase, L, L0, E) - ref)) < 1e-11
        x, info = oracle.cg(phase, L, L0, E, tol=1e-13)
        assert np.max(np.abs(x - ref)) < 1e-10
    L0 = _spd(rng, 2, 2.0, 15.0)
    assert np.max(np.abs(dense.solve_lu(phase, L, L0, E) - ref)) < 1e-11


def test_homogeneous_medium_zero_iterations():
    phase = np.zeros((27, 27), dtype=np.uint8)
    L = np.array([[[4.0, 1.0], [1.0, 3.0]]])
    L0 = oracle.reference_medium(L)
    for b in range(2):
        x, info = oracle.cg(phase, L, L0, np.eye(2)[b], tol=1e-12)
        assert info["iters"] == 0
        assert np.array_equal(x, oracle.operator.macroscopic_field(np.eye(2)[b], (27, 27)))
    xs = [oracle.cg(phase, L, L0, np.eye(2)[b])[0] for b in range(2)]
    assert np.allclose(oracle.effective_tensor(xs, phase, L), L[0], atol=1e-15)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_laminate_closed_form_golden():
    """Layers normal to axis 0: e_0 = E_0 <1/L>^-1 / L(x_0), e_1 = E_1 exactly,
    L_eff = diag(harmonic, arithmetic) over the digital layer fractions.
    The stored values are derived by hand (tests/golden/laminate_2d.json)."""
    g = _golden("laminate_2d.json")
    N = tuple(g["N"])
    phase = micro.laminate(N, g["fractions"], axis=g["axis"])
    L = micro.isotropic_table(g["conductivities"], 2)
    L0 = oracle.reference_medium(L)
    fields = []
    for b in range(2):
        E = np.eye(2)[b]
        x, info = oracle.cg(phase, L, L0, E, tol=1e-14, max_iter=200)
        assert info["rel_res_true"] < 1e-13
        fields.append(x)
    cond = np.asarray(g["conductivities"])[phase]
    harm = g["L_eff"][0][0]
    assert np.allclose(fields[0][0], harm / cond, atol=1e-12)
    assert np.allclose(fields[0][1], 0.0, atol=1e-12)
    assert np.allclose(fields[1][0], 0.0, atol=1e-12)
    assert np.allclose(fields[1][1], 1.0, atol=1e-12)
    assert np.allclose(oracle.effective_tensor(fields, phase, L), np.array(g["L_eff"]), atol=1e-12)


def test_laminate_3d_random_layers_dense():
    """Random layer order along axis 2 of a 3-D cell: harmonic along the layers'
    normal, arithmetic within, solved densely."""
    N = (5, 3, 9)
    phase = micro.laminate(N, [4 / 9, 3 / 9, 2 / 9], axis=2, d=3, seed=8)
    c = np.array([1.0, 6.0, 30.0])
    L = micro.isotropic_table(c, 3)
    L0 = oracle.reference_medium(L)
    frac = np.bincount(phase[0, 0, :], minlength=3) / 9.0
    harm = 1.0 / np.sum(frac / c)
    arith = np.sum(frac * c)
    xs = [dense.solve_lu(phase, L, L0, np.eye(3)[b]) for b in range(3)]
    assert np.allclose(oracle.effective_tensor(xs, phase, L), np.diag([arith, arith, harm]),
                       atol=1e-11)


def test_effective_tensor_bounds_and_symmetry():
    """L_eff symmetric; Reuss <= L_eff <= Voigt as quadratic forms (exact for the
    discrete minimum-energy problem); Hashin-Shtrikman for the square-symmetric
    single-disk cell (isotropic effective tensor)."""
    N = 45
    phase = micro.centred_disk(N, 0.45)
    f2 = micro.digital_fraction(phase)
    f1 = 1.0 - f2
    for rho in (10.0, 100.0):
        L = micro.isotropic_table([1.0, rho], 2)
        L0 = oracle.reference_medium(L)
        xs = [oracle.cg(phase, L, L0, np.eye(2)[b], tol=1e-12)[0] for b in range(2)]
        Le = oracle.effective_tensor(xs, phase, L)
        assert abs(Le[0, 1] - Le[1, 0]) < 1e-9 * Le[0, 0]
        assert abs(Le[0, 0] - Le[1, 1]) < 1e-9 * Le[0, 0]
        voigt = (f1 + f2 * rho) * np.eye(2)
        reuss = 1.0 / (f1 + f2 / rho) * np.eye(2)
        assert np.linalg.eigvalsh(voigt - 0.5 * (Le + Le.T)).min() > 0
        assert np.linalg.eigvalsh(0.5 * (Le + Le.T) - reuss).min() > 0
        hs_lo = 1.0 + f2 / (1.0 / (rho - 1.0) + f1 / 2.0)
        hs_hi = rho + f1 / (1.0 / (1.0 - rho) + f2 / (2.0 * rho))
        assert hs_lo <= Le[0, 0] <= hs_hi


def test_cg_and_bicg_iterates_coincide():
    """Section 3.1: CG and BiCG generate identical iterates (r0* = r0)."""
    phase = micro.rsa_disks(45, 0.4, 3, 7, seed=12)
    L = micro.isotropic_table([1.0, 100.0], 2)
    L0 = oracle.reference_medium(L)
    _, ic = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-8)
    _, ib = oracle.bicg(phase, L, L0, [1.0, 0.0], tol=1e-8)
    assert ic["iters"] == ib["iters"]
    hc, hb = ic["history"], ib["history"]
    assert np.allclose(hc[:20], hb[:20], rtol=1e-8)


def test_rate_bounds_eq_conv_rate():
    """Eq. (conv_rate): FFTH with omega = 0.5 contracts the residual at least by
    gamma_FFTH per step; CG's Euclidean residual obeys 2 sqrt(kappa) gamma_CG^m.
    Iteration counts are checked against the golden table derived from the
    same formulas (tests/golden/rate_bounds.json)."""
    g = _golden("rate_bounds.json")
    phase = micro.centred_disk(27, 0.5)
    for rho, row in zip(g["rho"], g["rows"]):
        if rho > 1e3:
            continue
        L = micro.isotropic_table([1.0, rho], 2)
        L0 = oracle.reference_medium(L)
        eps = 1e-4
        _, ffth = oracle.fixed_point(phase, L, L0, [1.0, 0.0], tol=eps, max_iter=20000)
        _, cgi = oracle.cg(phase, L, L0, [1.0, 0.0], tol=eps)
        gam_f = (rho - 1) / (rho + 1)
        gam_c = (math.sqrt(rho) - 1) / (math.sqrt(rho) + 1)
        assert math.ceil(math.log(eps) / math.log(gam_f)) == row["ffth"][0]
        assert math.ceil(math.log(eps) / math.log(gam_c)) == row["cg"][0]
        assert ffth["iters"] <= row["ffth"][0]
        cg_cap = math.ceil(math.log(eps / (2.0 * math.sqrt(rho))) / math.log(gam_c))
        assert cgi["iters"] <= cg_cap
        h = ffth["history"]
        ratios = h[1:] / h[:-1]
        assert np.all(ratios <= gam_f + 1e-9)


def test_cg_needs_fewer_iterations_sqrt_trend():
    """Section 3.2 / Fig. example2: CG iterations grow like sqrt(rho), FFTH like rho;
    CG needs a shrinking fraction of FFTH's iterations as the contrast grows
    (Section 3.1: 50 % at mild contrast down to a few percent)."""
    phase = micro.centred_disk(27, 0.5)
    it_cg, it_ff = {}, {}
    for rho in (10.0, 1000.0):
        L = micro.isotropic_table([1.0, rho], 2)
        L0 = oracle.reference_medium(L)
        it_cg[rho] = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-4)[1]["iters"]
        it_ff[rho] = oracle.fixed_point(phase, L, L0, [1.0, 0.0], tol=1e-4,
                                        max_iter=20000)[1]["iters"]
    assert it_cg[10.0] <= 0.6 * it_ff[10.0]
    assert it_cg[1000.0] <= 0.1 * it_ff[1000.0]
    grow_cg = it_cg[1000.0] / it_cg[10.0]
    grow_ff = it_ff[1000.0] / it_ff[10.0]
    assert 2.0 <= grow_cg <= 20.0
    assert grow_ff >= 30.0


def test_eta_e_vanishes_at_solution():
    """Eq. (errE_def): the converged field is in equilibrium, the cold start is not."""
    phase = micro.centred_disk(27, 0.3)
    L = micro.isotropic_table([1.0, 10.0], 2)
    L0 = oracle.reference_medium(L)
    x, _ = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-13)
    assert oracle.eta_e(x, phase, L) < 1e-10
    cold = oracle.operator.macroscopic_field([1.0, 0.0], (27, 27))
    assert oracle.eta_e(cold, phase, L) > 1e-2


def test_infinite_contrast_does_not_converge():
    """Section 3.2 / conjecture iii: as rho -> infinity CG stalls; a near-rigid
    inclusion within a small iteration budget must end 'not_converged', never hang."""
    phase = micro.centred_disk(27, 0.5)
    L = micro.isotropic_table([1.0, 1e12], 2)
    L0 = oracle.reference_medium(L)
    _, info = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-8, max_iter=200)
    assert info["status"] in ("not_converged", "breakdown")


def test_fixed_point_eta_r_is_l0_times_residual():
    """Eq. (errR_def) for FFTH: ||L0 (e^(m+1) - e^(m))|| / ||e^0|| = l0 * relative residual."""
    phase = micro.centred_disk(15, 0.3)
    L = micro.isotropic_table([1.0, 4.0], 2)
    L0 = oracle.reference_medium(L)
    _, info = oracle.fixed_point(phase, L, L0, [1.0, 0.0], tol=1e-6)
    assert np.isclose(info["eta_r"], L0[0, 0] * info["history"][-1], rtol=1e-12)


def test_bicg_biorthogonality_nonsymmetric():
    """Saad Alg. 7.3 invariant: (r_i, r*_j) = 0 for i != j.  An anisotropic L0
    makes A non-symmetric, so this holds only if the shadow sequence really uses
    A^T (a CG-like shadow r* = r loses it)."""
    rng = np.random.default_rng(21)
    phase = micro.rsa_disks(21, 0.35, 2, 4, seed=6)
    L = np.stack([_spd(rng, 2, 1.0, 2.0), _spd(rng, 2, 5.0, 9.0)])
    L0 = np.array([[6.0, 2.5], [2.5, 3.0]])
    A = np.eye(882) + dense.assemble_B(phase, L, L0)
    assert np.max(np.abs(A - A.T)) > 1e-3
    rec = []
    oracle.bicg(phase, L, L0, [1.0, 0.3], tol=1e-10, max_iter=8, record=rec)
    R = np.stack([r.ravel() / np.linalg.norm(r) for r, _ in rec])
    S = np.stack([s.ravel() / np.linalg.norm(s) for _, s in rec])
    M = R @ S.T
    off = M - np.diag(np.diag(M))
    assert np.max(np.abs(off)) < 1e-8
    assert np.min(np.abs(np.diag(M))) > 1e-6


def test_eta_r_history_is_the_printed_norm_of_every_step():
    """Eq. (errR_def) per step, checked against brute force: the CG iterate
    after m steps is the oracle's result with max_iter = m, so
    ||L0 (e_{m+1} - e_m)|| / ||e0|| comes from two separate solves; for the
    fixed-point scheme the step is the residual, so eta_r = l0 * rel.res."""
    rng = np.random.default_rng(41)
    N = (15, 21)
    phase = rng.integers(0, 2, size=N).astype(np.uint8)
    L = micro.isotropic_table([1.0, 7.0], 2)
    L0 = oracle.reference_medium(L)
    E = [0.3, 1.0]
    nb = np.linalg.norm(oracle.operator.macroscopic_field(E, N))
    xs = [oracle.cg(phase, L, L0, E, tol=1e-30, max_iter=m)[0] for m in range(6)]
    _, info = oracle.cg(phase, L, L0, E, tol=1e-30, max_iter=5)
    assert len(info["eta_r_history"]) == 5
    for m in range(5):
        ref = np.linalg.norm(np.einsum("ab,b...->a...", L0, xs[m + 1] - xs[m])) / nb
        assert abs(info["eta_r_history"][m] - ref) <= 1e-12 * ref, (m, info["eta_r_history"][m], ref)
    _, fi = oracle.fixed_point(phase, L, L0, E, tol=1e-30, max_iter=6)
    assert np.allclose(fi["eta_r_history"], L0[0, 0] * fi["history"], rtol=1e-13, atol=0)


def test_even_grid_solvers_reach_the_dense_solution_and_equilibrium():
    """Even axes (zero Green operator on the Nyquist frequencies): CG and the
    fixed point reach the dense LU solution, eta_e (without the Nyquist
    frequencies) vanishes there, and the solution has no Nyquist mode."""
    rng = np.random.default_rng(43)
    N = (8, 10)
    phase = rng.integers(0, 2, size=N).astype(np.uint8)
    L = micro.isotropic_table([1.0, 6.0], 2)
    L0 = oracle.reference_medium(L)
    E = [1.0, -0.5]
    xd = dense.solve_lu(phase, L, L0, E)
    for solver in (oracle.cg, oracle.fixed_point):
        x, info = solver(phase, L, L0, E, tol=1e-13, max_iter=20000)
        assert info["status"] == "converged"
        assert np.max(np.abs(x - xd)) < 1e-10
    assert oracle.eta_e(xd, phase, L) < 1e-12
    xh = np.fft.fft2(xd - np.asarray(E)[:, None, None])
    nyq = oracle.operator.nyquist_mask(N)
    assert np.max(np.abs(xh[:, nyq])) < 1e-10 * np.max(np.abs(xh))
