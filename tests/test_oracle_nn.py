"""Pins for the warm-start network oracle (CPU only): the convolution against
its index-loop definition, every backward formula against central finite
differences, the pool / upsample adjoint identity, bfloat16 rounding and Adam."""
import numpy as np
import pytest

from oracle import nn


def test_conv3_matches_index_loops():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 5))
    w = rng.normal(size=(3, 2, 27))
    b = rng.normal(size=3)
    y = nn.conv3(x, w, b)
    C, n0, n1, n2 = x.shape
    ref = np.zeros((3, n0, n1, n2))
    for o in range(3):
        for z in range(n0):
            for yy in range(n1):
                for xx in range(n2):
                    s = b[o]
                    t = 0
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                for c in range(C):
                                    s += w[o, c, t] * x[c, (z + dz) % n0, (yy + dy) % n1, (xx + dx) % n2]
                                t += 1
                    ref[o, z, yy, xx] = s
    assert np.allclose(y, ref, atol=1e-12)


def test_pool_upsample_adjoint():
    """<pool3(a), b> = <a, up3(b)> / 27 and pool3(up3(b)) = b."""
    rng = np.random.default_rng(1)
    a = rng.normal(size=(2, 9, 6, 3))
    b = rng.normal(size=(2, 3, 2, 1))
    assert np.isclose(np.vdot(nn.pool3(a), b), np.vdot(a, nn.up3(b)) / 27.0)
    assert np.allclose(nn.pool3(nn.up3(b)), b)
    assert np.allclose(nn.up3_backward(nn.up3(b)), 27 * b)


def _fd(f, p, eps=1e-6, idx=None):
    flat = p.reshape(-1)
    out = []
    for i in idx:
        old = flat[i]
        flat[i] = old + eps
        fp = f()
        flat[i] = old - eps
        fm = f()
        flat[i] = old
        out.append((fp - fm) / (2 * eps))
    return np.array(out)


def test_conv3_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 4, 3, 5))
    w = rng.normal(size=(2, 3, 27))
    b = rng.normal(size=2)
    gy = rng.normal(size=(2, 4, 3, 5))
    gx, gw, gb = nn.conv3_backward(x, w, gy)
    f = lambda: float(np.sum(gy * nn.conv3(x, w, b)))
    idx = rng.choice(x.size, 12, replace=False)
    assert np.allclose(_fd(f, x, idx=idx), gx.reshape(-1)[idx], rtol=1e-6, atol=1e-8)
    idx = rng.choice(w.size, 12, replace=False)
    assert np.allclose(_fd(f, w, idx=idx), gw.reshape(-1)[idx], rtol=1e-6, atol=1e-8)
    assert np.allclose(_fd(f, b, idx=[0, 1]), gb, rtol=1e-6)


def test_network_backward_finite_differences():
    """The whole network in float64 (no bfloat16 rounding), N = 27 so that the
    coarsest level is a single voxel."""
    rng = np.random.default_rng(3)
    chans = (4, 5, 6, 7)
    params = [(w.astype(np.float64), b.astype(np.float64) + rng.normal(size=b.shape) * 0.1)
              for (w, b) in nn.init_params(2, 3, seed=5, channels=chans)]
    x = rng.normal(size=(2, 27, 27, 27))
    target = rng.normal(size=(3, 27, 27, 27))
    loss, grads, _ = nn.loss_and_grads(params, x, target, round_bf16=False)
    for layer in (0, 2, 3, 4, 5, 8, 9, 10):
        w, b = params[layer]
        f = lambda: nn.loss_and_grads(params, x, target, round_bf16=False)[0]
        idx = rng.choice(w.size, 4, replace=False)
        fd = _fd(f, w, eps=1e-5, idx=idx)
        assert np.allclose(fd, grads[layer][0].reshape(-1)[idx], rtol=1e-4, atol=1e-9), layer
        fdb = _fd(f, b, eps=1e-5, idx=[0])
        assert np.allclose(fdb, grads[layer][1][:1], rtol=1e-4, atol=1e-9), layer


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.14159265, 65504.0, 1e-20], dtype=np.float32)
    r = nn.bf16(v)
    # exactly representable values are kept; others go to the nearest bf16 (8 mantissa bits)
    assert r[0] == 1.0
    for a, q in zip(v, r):
        assert abs(q - a) <= abs(a) * 2 ** -8
        bits = np.array([q], dtype=np.float32).view(np.uint32)[0]
        assert bits & 0xFFFF == 0
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert nn.bf16(np.array([1.0 + 2 ** -8], dtype=np.float32))[0] == 1.0


def test_adam_scalar_recurrence():
    p = np.array([1.0])
    m = np.zeros(1)
    v = np.zeros(1)
    gs = [0.5, -0.2, 0.3]
    mm = vv = 0.0
    q = 1.0
    for t, g in enumerate(gs, start=1):
        nn.adam(p, np.array([g]), m, v, t, lr=0.01)
        mm = 0.9 * mm + 0.1 * g
        vv = 0.999 * vv + 0.001 * g * g
        q -= 0.01 * (mm / (1 - 0.9 ** t)) / (np.sqrt(vv / (1 - 0.999 ** t)) + 1e-8)
    assert np.isclose(p[0], q)


def test_adam_matches_kingma_ba_by_hand():
    """Adam (Kingma & Ba, Algorithm 1) with lr 0.01, beta1 0.9, beta2 0.999,
    eps 1e-8, from m = v = 0, values written out by hand.

    Step 1 (g = 0.5): m = 0.05, v = 2.5e-4, m_hat = g, v_hat = g^2, so the
    update is lr g / (|g| + eps) = 0.01 * 0.5 / 0.50000001 and
    p = 1 - 0.0099999998 = 0.9900000002.
    Step 2 (g = -0.2): m = 0.9 * 0.05 - 0.02 = 0.025,
    v = 0.999 * 2.5e-4 + 0.001 * 0.04 = 2.8975e-4, m_hat = 0.025 / 0.19,
    v_hat = 2.8975e-4 / 0.001999, p = 0.9900000002 - 0.01 m_hat / (sqrt(v_hat) + eps)
    = 0.98654394181165106 (evaluated to 30 digits).
    A wrong bias correction (none, or beta^(t-1)) or a swapped beta moves
    either step by far more than the tolerance."""
    p = np.array([1.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    nn.adam(p, np.array([0.5, -3.0]), m, v, 1, lr=0.01)
    assert abs(p[0] - 0.9900000002) < 1e-15
    # the first step is lr * sign(g) up to eps whatever |g|: -2 + 0.01 * 3 / (3 + 1e-8)
    assert abs(p[1] - (-2.0 + 0.03 / 3.00000001)) < 1e-15
    assert np.allclose(m, [0.05, -0.3], rtol=0, atol=1e-16)
    assert np.allclose(v, [2.5e-4, 9e-3], rtol=1e-15, atol=0)
    nn.adam(p, np.array([-0.2, 0.0]), m, v, 2, lr=0.01)
    assert abs(m[0] - 0.025) < 1e-16 and abs(v[0] - 2.8975e-4) < 1e-18
    assert abs(p[0] - 0.98654394181165106) < 1e-14


def test_leaky_and_mse_literal_values():
    """Leaky ReLU with slope 0.1 on the negative side, and the mean squared
    error over every entry with gradient 2 (y - t) / count, on literal values."""
    x = np.array([-2.0, -0.5, 0.0, 0.3, 4.0])
    assert np.array_equal(nn.leaky(x), np.array([-0.2, -0.05, 0.0, 0.3, 4.0]))
    g = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    assert np.allclose(nn.leaky_backward(x, g), [0.1, 0.2, 0.3, 4.0, 5.0], rtol=0, atol=1e-15)
    y = np.array([[1.0, 2.0], [3.0, 4.0]])
    t = np.array([[0.0, 0.0], [1.0, 6.0]])
    loss, gy = nn.mse(y, t)
    # diff = [[1, 2], [2, -2]]: squares 1 + 4 + 4 + 4 = 13 over 4 entries
    assert loss == 13.0 / 4.0
    assert np.array_equal(gy, np.array([[0.5, 1.0], [1.0, -1.0]]))
