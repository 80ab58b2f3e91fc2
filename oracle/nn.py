"""Oracle of the learned warm-start network (test infrastructure only).

Plain numpy, float64 unless a float32 / bfloat16 step is stated.  The
network maps a 3-D phase description to the fluctuation fields of the d unit
loads, e^(b) - e_b, from which a warm start for CG is formed.  The paper has
no network; this is the warm-start pattern the build adds on top of the
method, and its arithmetic is written out here so that the CUDA kernels can be
checked element by element:

* conv3 : 3 x 3 x 3 convolution with periodic (circular) padding,
          y[o, z] = b[o] + sum_c sum_t w[o, c, t] x[c, z + t],  t in {-1,0,1}^3
* pool3 : mean over disjoint 3 x 3 x 3 blocks (stride 3)
* up3   : nearest-neighbour upsampling by 3 (each coarse voxel copied 27 times)
* leaky : max(x, 0) + 0.1 min(x, 0)
* loss  : mean squared error over channels and voxels
* adam  : Kingma & Ba's Adam with bias correction
* bf16  : round-to-nearest-even float32 -> bfloat16 (weights in the forward)

Architecture (channels c = (16, 32, 48, 64), levels N, N/3, N/9, N/27;
layers numbered 0..10 in parameter order):
  a0 = leaky(conv3(x; W0))                     c0 at N
  a1 = leaky(conv3(pool3(a0); W1))             c1 at N/3
  a2 = leaky(conv3(pool3(a1); W2))             c2 at N/9
  a3 = leaky(conv3(pool3(a2); W3))             c3 at N/27
  v2 = up3(leaky(conv3(a3; W4))) + a2 ; u2 = leaky(conv3(v2; W5))    c2 at N/9
  v1 = up3(leaky(conv3(u2; W6))) + a1 ; u1 = leaky(conv3(v1; W7))    c1 at N/3
  v0 = up3(leaky(conv3(u1; W8))) + a0 ; u0 = leaky(conv3(v0; W9))    c0 at N
  y  = conv3(u0; W10)                                                cout at N

Pinned by ``tests/test_oracle_nn.py``: the convolution against explicit index
loops, every backward formula against central finite differences, the
pool / upsample adjoint identity, and Adam against its scalar recurrence.
"""
from __future__ import annotations

import numpy as np

SLOPE = 0.1
CHANNELS = (16, 32, 48, 64)


# ---------------------------------------------------------------------------
# elementary layers
# ---------------------------------------------------------------------------
def _taps():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3(x, w, b):
    """y[o] = b[o] + sum_c sum_t w[o, c, t] x[c](. + t), periodic; w: (O, C, 27)."""
    O = w.shape[0]
    y = np.zeros((O,) + x.shape[1:], dtype=np.result_type(x, w))
    for t, (dz, dy, dx) in enumerate(_taps()):
        xs = np.roll(x, shift=(-dz, -dy, -dx), axis=(1, 2, 3))  # xs[c, z] = x[c, z + t]
        y += np.einsum("oc,c...->o...", w[:, :, t], xs)
    return y + b.reshape((O, 1, 1, 1))


def conv3_backward(x, w, gy):
    """Gradients of sum(gy * conv3(x, w, b)) with respect to x, w and b."""
    gx = np.zeros_like(x, dtype=np.result_type(x, w, gy))
    gw = np.zeros(w.shape, dtype=np.result_type(x, gy))
    for t, (dz, dy, dx) in enumerate(_taps()):
        xs = np.roll(x, shift=(-dz, -dy, -dx), axis=(1, 2, 3))
        gw[:, :, t] = gy.reshape(gy.shape[0], -1) @ xs.reshape(xs.shape[0], -1).T
        # d/dx[c, z'] of sum_o gy[o, z] w[o, c, t] x[c, z + t] with z' = z + t
        gx += np.roll(np.einsum("oc,o...->c...", w[:, :, t], gy), shift=(dz, dy, dx), axis=(1, 2, 3))
    gb = gy.sum(axis=(1, 2, 3))
    return gx, gw, gb


def pool3(x):
    C, n0, n1, n2 = x.shape
    return x.reshape(C, n0 // 3, 3, n1 // 3, 3, n2 // 3, 3).mean(axis=(2, 4, 6))


def pool3_backward(gy):
    return up3(gy) / 27.0


def up3(x):
    return x.repeat(3, axis=1).repeat(3, axis=2).repeat(3, axis=3)


def up3_backward(gy):
    C, n0, n1, n2 = gy.shape
    return gy.reshape(C, n0 // 3, 3, n1 // 3, 3, n2 // 3, 3).sum(axis=(2, 4, 6))


def leaky(x):
    return np.where(x > 0, x, SLOPE * x)


def leaky_backward(x, gy):
    return np.where(x > 0, gy, SLOPE * gy)


def mse(y, target):
    """Mean squared error and its gradient with respect to y."""
    diff = y - target
    return float(np.mean(diff * diff)), 2.0 * diff / diff.size


def bf16(w):
    """Round float32 values to bfloat16 (round to nearest, ties to even), as float32."""
    u = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def adam(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place; t is the 1-based step count."""
    m *= beta1
    m += (1.0 - beta1) * grad
    v *= beta2
    v += (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    param -= lr * mh / (np.sqrt(vh) + eps)


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def layer_shapes(cin, cout, channels=CHANNELS):
    c0, c1, c2, c3 = channels
    io = [(cin, c0), (c0, c1), (c1, c2), (c2, c3),
          (c3, c2), (c2, c2), (c2, c1), (c1, c1), (c1, c0), (c0, c0),
          (c0, cout)]
    return [(o, i, 27) for (i, o) in io]


def init_params(cin, cout, seed, channels=CHANNELS):
    """He-normal weights, zero biases, float32 (seeded input, shared by both sides)."""
    rng = np.random.default_rng(seed)
    params = []
    for (o, i, t) in layer_shapes(cin, cout, channels):
        w = rng.normal(0.0, np.sqrt(2.0 / (27.0 * i)), size=(o, i, t)).astype(np.float32)
        params.append((w, np.zeros(o, dtype=np.float32)))
    return params


def forward(params, x, round_bf16=True):
    """Returns (y, cache).  Weights are rounded to bfloat16 when round_bf16."""
    W = [(bf16(w) if round_bf16 else w, b) for (w, b) in params]
    c = {"x": x, "W": W}
    c["z0"] = conv3(x, *W[0]); c["a0"] = leaky(c["z0"])
    for l in (1, 2, 3):
        c[f"p{l - 1}"] = pool3(c[f"a{l - 1}"])
        c[f"z{l}"] = conv3(c[f"p{l - 1}"], *W[l])
        c[f"a{l}"] = leaky(c[f"z{l}"])
    u = c["a3"]
    for l, (ku, kp) in zip((2, 1, 0), ((4, 5), (6, 7), (8, 9))):
        c[f"u{l + 1}_in"] = u                      # input of the up convolution
        c[f"z{ku}"] = conv3(u, *W[ku])
        c[f"v{l}"] = up3(leaky(c[f"z{ku}"])) + c[f"a{l}"]
        c[f"z{kp}"] = conv3(c[f"v{l}"], *W[kp])
        u = leaky(c[f"z{kp}"])
        c[f"u{l}"] = u
    y = conv3(u, *W[10])
    return y, c


def backward(cache, gy):
    """Gradients of sum(gy * y) with respect to every (w, b), in layer order."""
    c, W = cache, cache["W"]
    grads = [None] * 11
    g_u, grads[10] = _conv_grads(c["u0"], W[10], gy)
    g_skip = {}
    for l, (ku, kp) in zip((0, 1, 2), ((8, 9), (6, 7), (4, 5))):
        g_zp = leaky_backward(c[f"z{kp}"], g_u)
        g_v, grads[kp] = _conv_grads(c[f"v{l}"], W[kp], g_zp)
        g_skip[l] = g_v                            # v_l = up(...) + a_l
        g_zu = leaky_backward(c[f"z{ku}"], up3_backward(g_v))
        g_u, grads[ku] = _conv_grads(c[f"u{l + 1}_in"], W[ku], g_zu)
    g_a = g_u                                      # gradient at a3
    for l in (3, 2, 1):
        g_z = leaky_backward(c[f"z{l}"], g_a)
        g_p, grads[l] = _conv_grads(c[f"p{l - 1}"], W[l], g_z)
        g_a = g_skip[l - 1] + pool3_backward(g_p)
    g_z0 = leaky_backward(c["z0"], g_a)
    _, grads[0] = _conv_grads(c["x"], W[0], g_z0)
    return grads


def _conv_grads(x, wb, gy):
    gx, gw, gb = conv3_backward(x, wb[0], gy)
    return gx, (gw, gb)


def loss_and_grads(params, x, target, round_bf16=True):
    y, cache = forward(params, x, round_bf16)
    loss, gy = mse(y, target)
    return loss, backward(cache, gy), y


def features(phase, L):
    """Network input: channel 0 = log10(L(x) / L_matrix) / 4, channel 1 = inclusion indicator.
    Isotropic phases; L_matrix is phase 0."""
    cond = np.asarray([Lp[0, 0] for Lp in np.asarray(L)])
    lc = np.log10(cond / cond[0]) / 4.0
    ph = np.asarray(phase)
    return np.stack([lc[ph], (ph > 0).astype(np.float64)]).astype(np.float32)
