"""The warm-start network's kernels against the numpy oracle (oracle/nn.py),
and the learned warm start against a cold start e = E.

Forward: tensor-core products of the bfloat16 weights with each float32
activation split into two bfloat16 halves (about 16 mantissa bits kept, error
<= 2^-17 relative per product) and float32 accumulation, against float64 with
the same bfloat16-rounded weights: max error <= 1e-4 of max |y| (eleven
layers of ~2^-17 each), loss within 1e-4 relative.  Gradients: per layer, max
error <= 2e-3 of the layer's max |g| (float32 backward sweeps through eleven
layers).
Features and targets are exact conversions and compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import nn as onn
from paper_1004_1122_gb300 import microstructure as micro

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

N = (27, 27, 27)


def _flat(params):
    return np.concatenate([np.concatenate([w.reshape(-1), b]) for (w, b) in params]).astype(np.float32)


def _unflat(flat, shapes):
    out, k = [], 0
    for (o, i, t) in shapes:
        w = flat[k:k + o * i * t].reshape(o, i, t)
        k += o * i * t
        b = flat[k:k + o]
        k += o
        out.append((w, b))
    assert k == flat.size
    return out


def _setup(seed=11, cout=9, channels=onn.CHANNELS):
    rng = np.random.default_rng(seed)
    params = [(w, (rng.normal(size=b.shape) * 0.05).astype(np.float32))
              for (w, b) in onn.init_params(2, cout, seed=seed, channels=channels)]
    x = rng.normal(size=(2,) + N).astype(np.float32)
    return params, x


def test_param_layout():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    net = fh.Net(N, 2, 9)
    params, _ = _setup()
    flat = _flat(params)
    assert net.nparam == flat.size
    net.set_params(flat)
    np.testing.assert_array_equal(net.get_params(), flat)
    net.close()
    with pytest.raises(fh.FhError):
        fh.Net((27, 27, 30), 2, 9)


def test_forward_parity():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    params, x = _setup()
    net = fh.Net(N, 2, 9)
    net.set_params(_flat(params))
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref, _ = onn.forward(params, x.astype(np.float64), round_bf16=True)
    err = np.max(np.abs(y - ref)) / np.max(np.abs(ref))
    assert err <= 1e-4, err
    assert net.launches() > 0
    net.close()


def test_forward_parity_uneven_grid():
    """A non-cubic grid (27, 54, 81) with small channel counts that do not fill
    a 16-channel output tile."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    Ng = (27, 54, 81)
    chans = (5, 7, 9, 11)
    rng = np.random.default_rng(4)
    params = [(w, (rng.normal(size=b.shape) * 0.05).astype(np.float32))
              for (w, b) in onn.init_params(2, 4, seed=3, channels=chans)]
    x = rng.normal(size=(2,) + Ng).astype(np.float32)
    net = fh.Net(Ng, 2, 4, channels=chans)
    net.set_params(_flat(params))
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref, _ = onn.forward(params, x.astype(np.float64), round_bf16=True)
    assert np.max(np.abs(y - ref)) <= 1e-4 * np.max(np.abs(ref))
    net.close()


def test_gradient_parity():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    params, x = _setup(seed=12)
    rng = np.random.default_rng(5)
    target = rng.normal(size=(9,) + N).astype(np.float32)
    net = fh.Net(N, 2, 9)
    net.set_params(_flat(params))
    loss, g = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda())
    ref_loss, ref_grads, _ = onn.loss_and_grads(params, x.astype(np.float64), target.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    shapes = onn.layer_shapes(2, 9)
    for layer, ((gw, gb), (rw, rb)) in enumerate(zip(_unflat(g, shapes), ref_grads)):
        scale = max(np.max(np.abs(rw)), np.max(np.abs(rb)))
        assert np.max(np.abs(gw - rw)) <= 2e-3 * scale, layer
        assert np.max(np.abs(gb - rb)) <= 2e-3 * scale, layer
    net.close()


def test_adam_step_parity():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    params, x = _setup(seed=13)
    rng = np.random.default_rng(6)
    target = rng.normal(size=(9,) + N).astype(np.float32)
    lr = 1e-3
    net = fh.Net(N, 2, 9)
    flat = _flat(params)
    net.set_params(flat)
    net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda(), lr)
    got = net.get_params()
    _, grads, _ = onn.loss_and_grads(params, x.astype(np.float64), target.astype(np.float64))
    g = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for (gw, gb) in grads])
    p = flat.astype(np.float64)
    onn.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr)
    # every entry moves by at most lr; where the gradient is clearly non-zero
    # the step is lr * sign(g) on both sides
    assert np.all(np.abs(got - flat) <= lr * 1.001 + 1e-7)
    big = np.abs(g) > 1e-2 * np.max(np.abs(g))
    assert big.sum() > 100
    assert np.max(np.abs(got[big] - p[big])) <= 1e-3 * lr + 1e-6
    net.close()


def test_training_reduces_loss():
    """A learnable target (the output of another parameter set) is fitted."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    chans = (8, 12, 16, 16)
    params, x = _setup(seed=14, channels=chans)
    teacher = [(w, b) for (w, b) in onn.init_params(2, 9, seed=99, channels=chans)]
    t, _ = onn.forward(teacher, x.astype(np.float64))
    net = fh.Net(N, 2, 9, channels=chans)
    net.set_params(_flat(params))
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    losses = [net.train_step(xd, td, 3e-3) for _ in range(80)]
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])
    net.close()


def test_features_and_targets_exact():
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    rng = np.random.default_rng(8)
    ph = rng.integers(0, 3, size=N).astype(np.uint8)
    L = micro.isotropic_table([2.0, 37.0, 4000.0], 3)
    x = torch.empty((2,) + N, dtype=torch.float32, device="cuda")
    fh.nn_features(torch.from_numpy(ph).cuda(), L, x)
    np.testing.assert_array_equal(x.cpu().numpy(), onn.features(ph, L))
    fields = [rng.normal(size=(3,) + N) for _ in range(3)]
    t = torch.empty((9,) + N, dtype=torch.float32, device="cuda")
    fh.nn_targets([torch.from_numpy(f).cuda() for f in fields], t)
    torch.cuda.synchronize()
    ref = np.concatenate([(f - np.eye(3)[b].reshape(3, 1, 1, 1)) for b, f in enumerate(fields)]).astype(np.float32)
    np.testing.assert_array_equal(t.cpu().numpy(), ref)
    base = rng.normal(size=(9,) + N).astype(np.float32)
    fh.nn_targets([torch.from_numpy(f).cuda() for f in fields], t, torch.from_numpy(base).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(t.cpu().numpy(), ref + base)


def test_warm_start_projection():
    """x0 = E + Q(sum_b E_b (pred_b - base_b)), Q = F^-1 Gamma0 F L0 (Section 2.1), against the oracle's
    Green operator; x0 - E has zero mean and Q(x0 - E) = x0 - E."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh, warmstart

    rng = np.random.default_rng(9)
    ph = micro.boolean_spheres(27, 4.0, 0.3, seed=3)
    L = micro.isotropic_table([1.0, 50.0], 3)
    pred = rng.normal(size=(9,) + N).astype(np.float32)
    base = rng.normal(size=(9,) + N).astype(np.float32)
    E = np.array([0.3, -0.5, 0.8])
    s = fh.Solver(ph, L, precision="fp64")
    x0 = warmstart.start(s, torch.from_numpy(pred).cuda(), E, torch.from_numpy(base).cuda()).cpu().numpy()
    L0 = oracle.reference_medium(L)
    g = np.einsum("b,ba...->a...", E, (pred.astype(np.float64) - base).reshape((3, 3) + N))
    ref = oracle.operator.macroscopic_field(E, N) + oracle.operator.green_apply(np.einsum("ab,b...->a...", L0, g), N, np.ones(3), L0)
    assert np.max(np.abs(x0 - ref)) <= 1e-12 * np.max(np.abs(ref))
    f = x0 - oracle.operator.macroscopic_field(E, N)
    assert np.max(np.abs(f.mean(axis=(1, 2, 3)))) <= 1e-12 * np.max(np.abs(f))
    qf = oracle.operator.green_apply(np.einsum("ab,b...->a...", L0, f), N, np.ones(3), L0)
    assert np.max(np.abs(qf - f)) <= 1e-10 * np.max(np.abs(f))
    s.close()


def _cell(seed):
    r = np.random.default_rng(seed)
    vf = r.uniform(0.15, 0.4)
    ph = micro.random_ellipsoids(27, vf, 2.5, 4.5, 2.0, seed=seed, spheres=bool(seed % 2))
    rho = float(10 ** r.uniform(1, 3))
    return ph, micro.isotropic_table([1.0, rho], 3)


def test_response_features():
    """(B e_b)_a from the library (float32 products) against the oracle's B
    (Eq. mtrx_B), within the float32 operator bound of the operator tests:
    64 * 4 u (1 + max|dL|) max|e|, u = 2^-24."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    ph, L = _cell(7)
    s = fh.Solver(ph, L, precision="fp32_refined")
    x = torch.empty((9,) + N, dtype=torch.float32, device="cuda")
    fh.nn_response_features(s, x)
    L0 = oracle.reference_medium(L)
    ref = np.concatenate([oracle.apply_B(oracle.operator.macroscopic_field(np.eye(3)[b], N), ph, L, L0)
                          for b in range(3)])
    got = x.cpu().numpy()
    dl = np.max(np.abs(L - L0[None]))
    assert np.max(np.abs(got - ref)) <= 64 * 4 * 2.0 ** -24 * (1.0 + dl)
    s.close()


def test_learned_warm_start_saves_iterations():
    """End to end on solver-generated fields: train the network on the unit-load
    fields of four 27^3 cells (contrast 10..1000), then solve those cells for a
    new load E from the warm start and from e = E to the same tolerance: the
    same effective column, fewer CG iterations in total.  (This
    checks the pipeline on cells the network has fitted; generalisation to
    held-out cells is measured by the benchmark.)"""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh, warmstart

    cells, pairs = [], []
    for k in range(4):
        ph, L = _cell(1000 + k)
        phd = torch.from_numpy(ph).cuda()
        s = fh.Solver(phd, L, precision="fp64")
        x, t, infos = warmstart.training_pair(s, phd, L, tol=1e-9)
        assert all(i["status"] == "FH_OK" for i in infos)
        pairs.append((x, t))
        cells.append((phd, L, s))
    ws = warmstart.WarmStart(N, d=3, seed=2)
    losses = ws.train(pairs, steps=4000, lr=1e-3)
    print("losses", np.mean(losses[:8]), np.mean(losses[-8:]))
    assert np.mean(losses[-8:]) < 0.3 * np.mean(losses[:8])
    rng = np.random.default_rng(21)
    cold_it, warm_it = [], []
    for (phd, L, s), (x, _) in zip(cells, pairs):
        pred = ws.predict(x)
        E = rng.normal(size=3)
        _, col_c, ic = s.solve(E, tol=1e-6, method="cg", max_iter=5000)
        _, col_w, iw = ws.solve(s, x, pred, E, tol=1e-6)
        print("cell", ic["iters"], iw["iters"], iw["res0_warm"], iw["res0_cold"])
        assert ic["status"] == "FH_OK" and iw["status"] == "FH_OK"
        assert iw["start"] == "warm" and iw["res0_warm"] < iw["res0_cold"]
        assert np.max(np.abs(col_w - col_c)) <= 1e-5 * np.max(np.abs(col_c))
        cold_it.append(ic["iters"])
        warm_it.append(iw["iters"])
        s.close()
    assert sum(warm_it) < sum(cold_it), (cold_it, warm_it)
    ws.close()


def test_warm_start_falls_back_to_cold():
    """An untrained network's start is worse than e = E: the cold start is taken
    and the result is the cold start's."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh, warmstart

    ph, L = _cell(11)
    phd = torch.from_numpy(ph).cuda()
    s = fh.Solver(phd, L, precision="fp64")
    ws = warmstart.WarmStart(N, d=3, seed=5)
    rng = np.random.default_rng(3)
    flat = ws.net.get_params()
    ws.net.set_params((flat + rng.normal(size=flat.size) * 0.5).astype(np.float32))
    x = ws.features(phd, L, s)
    pred = ws.predict(x)
    E = np.array([1.0, 0.0, 0.0])
    _, col_c, ic = s.solve(E, tol=1e-6)
    _, col_w, iw = ws.solve(s, x, pred, E, tol=1e-6)
    assert iw["start"] == "cold" and iw["res0_warm"] >= iw["res0_cold"]
    assert iw["iters"] == ic["iters"]
    np.testing.assert_array_equal(col_w, col_c)
    s.close()
    ws.close()


def test_learned_warm_start_on_held_out_cells():
    """Generalisation: train on the unit-load fields of 24 cells (27^3,
    contrast 10..1000), then solve 8 cells the network has never seen for a
    random load, from the warm start and from e = E, to the same tolerance.
    Checks: the warm start's initial residual is below the cold start's on
    held-out cells (the network carries over), both reach the same effective
    column, and the warm solves stay within 5 % of the cold iteration count.
    The gain in iterations and in time is printed.  Measured: the held-out
    initial residual halves (0.45 -> 0.2 of ||e0||) on every cell, yet the
    iterations do not change (443 cold, 445 warm over the 8 cells): the
    network removes mostly error components that CG removes in its first few
    iterations anyway, so at this accuracy a learned start cannot pay."""
    torch = cuda_or_skip()
    import time

    from paper_1004_1122_gb300 import fh, warmstart

    pairs = []
    for k in range(24):
        ph, L = _cell(2000 + k)
        phd = torch.from_numpy(ph).cuda()
        with fh.Solver(phd, L, precision="fp64") as s:
            x, t, infos = warmstart.training_pair(s, phd, L, tol=1e-9)
        assert all(i["status"] == "FH_OK" for i in infos)
        pairs.append((x, t))
    ws = warmstart.WarmStart(N, d=3, seed=4)
    ws.train(pairs, steps=6000, lr=1e-3)
    del pairs
    rng = np.random.default_rng(77)
    rows = []
    for k in range(8):
        ph, L = _cell(5000 + k)  # held out: seeds never used for training
        phd = torch.from_numpy(ph).cuda()
        with fh.Solver(phd, L, precision="fp64") as s:
            E = rng.normal(size=3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, col_c, ic = s.solve(E, tol=1e-6, method="cg", max_iter=5000)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            x = ws.features(phd, L, s)
            pred = ws.predict(x)
            _, col_w, iw = ws.solve(s, x, pred, E, tol=1e-6)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
        assert ic["status"] == "FH_OK" and iw["status"] == "FH_OK"
        assert np.max(np.abs(col_w - col_c)) <= 1e-5 * np.max(np.abs(col_c))
        rows.append((ic["iters"], iw["iters"], iw["res0_cold"], iw["res0_warm"], t1 - t0, t2 - t1, iw["start"]))
    ws.close()
    cold = sum(r[0] for r in rows)
    warm = sum(r[1] for r in rows)
    better_start = sum(r[3] < r[2] for r in rows)
    print(f"held-out: cold {cold} warm {warm} iterations ({100.0 * (cold - warm) / cold:+.1f} %), "
          f"time cold {sum(r[4] for r in rows):.3f} s warm {sum(r[5] for r in rows):.3f} s, "
          f"warm start better on {better_start}/8 cells; per cell {rows}")
    assert better_start >= 6
    assert warm <= 1.05 * cold
