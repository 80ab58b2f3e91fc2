"""Host-side logic of the learned warm start (CPU only): the parameter layout
the driver initialises matches the network's definition layer by layer, and
the learning-rate schedule is the stated warm-up + cosine decay."""
import math

import numpy as np

from oracle import nn as onn
from paper_1004_1122_gb300 import warmstart


def test_init_params_layout_matches_network():
    for cin, d, ch in ((2, 3, None), (11, 3, (8, 16, 24, 32)), (6, 2, (5, 7, 9, 11))):
        flat = warmstart.init_params(cin, d, seed=4, channels=ch)
        shapes = onn.layer_shapes(cin, d * d, ch if ch else onn.CHANNELS)
        assert flat.dtype == np.float32
        assert flat.size == sum(o * i * t + o for (o, i, t) in shapes)
        k = 0
        for (o, i, t) in shapes:
            w = flat[k:k + o * i * t]
            k += o * i * t
            b = flat[k:k + o]
            k += o
            assert np.all(b == 0.0)
            # He-normal scale sqrt(2 / (27 fan_in)) within sampling error
            if w.size >= 400:
                assert abs(np.std(w) / math.sqrt(2.0 / (27.0 * i)) - 1.0) < 0.15


def test_learning_rate_schedule():
    """Linear warm-up to lr over `warmup` steps, then cosine decay to lr_final."""

    class Net:
        def __init__(self):
            self.lrs = []

        def train_step(self, x, t, lr):
            self.lrs.append(lr)
            return 0.0

    ws = warmstart.WarmStart.__new__(warmstart.WarmStart)
    ws.net = Net()
    steps, lr, lr_final, warmup = 1000, 1e-3, 2e-5, 100
    ws.train([(None, None)] * 3, steps=steps, lr=lr, lr_final=lr_final, warmup=warmup)
    lrs = np.array(ws.net.lrs)
    assert lrs.size == steps
    assert np.isclose(lrs[0], lr / warmup) and np.isclose(lrs[warmup - 1], lr)
    assert np.all(np.diff(lrs[:warmup]) > 0)
    assert np.isclose(lrs[warmup], lr) and np.isclose(lrs[-1], lr_final)
    assert np.all(np.diff(lrs[warmup:]) <= 1e-15)
    mid = warmup + (steps - warmup - 1) // 2
    assert abs(lrs[mid] - 0.5 * (lr + lr_final)) < 0.01 * lr
