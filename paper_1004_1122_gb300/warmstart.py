"""Learned warm start for the CG solve of Eq. (linear_system).

The solution of (I + B) e = E is linear in the macroscopic field E, so one
network prediction per microstructure serves every load: the network
(``fh_nn_*``, hand-written kernels) maps the phase image to the fluctuation
fields e^(b) - e_b of the d unit loads, and the warm start for a load E is

    x0 = E + Q ( sum_b E_b (e^(b) - e_b) ),

with Q the compatible projection of Section 2.1 (``fh_nn_warm_start``), so
that x0 - E is a zero-mean compatible field, the subspace on which the
Krylov iterates of Section 3 live.  Plain CG from e = E stays the fallback
and the yardstick: the warm start is used only when its true residual is
below the cold start's, and both run to the same tolerance on the same
operator.

This module sequences the library calls (features, targets, training steps,
prediction, solves); every arithmetic step runs in the library's kernels.
"""
from __future__ import annotations

import math
import time
from typing import Sequence

import numpy as np

from . import fh


def init_params(cin: int, d: int, seed: int, channels=None) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (27 * fan_in))) and zero biases, flat float32,
    in the library's parameter order (per layer: weights [out][in][27], biases)."""
    c0, c1, c2, c3 = channels if channels is not None else (16, 32, 48, 64)
    io = [(cin, c0), (c0, c1), (c1, c2), (c2, c3),
          (c3, c2), (c2, c2), (c2, c1), (c1, c1), (c1, c0), (c0, c0),
          (c0, d * d)]
    rng = np.random.default_rng(seed)
    parts = []
    for (ci, co) in io:
        parts.append(rng.normal(0.0, math.sqrt(2.0 / (27.0 * ci)), size=co * ci * 27))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def features(phase_dev, L, solver: fh.Solver | None = None):
    """Network input, float32 on the device: channel 0 = log10(L_p / L_0) / 4,
    channel 1 = inclusion indicator, and, when a solver of the same cell is
    given, d*d more channels (B e_b)_a: the first-order response of the cell
    to each unit load (d operator products)."""
    import torch

    V = int(np.prod(phase_dev.shape))
    d = phase_dev.dim()
    c = 2 + (d * d if solver is not None else 0)
    x = torch.empty((c,) + tuple(phase_dev.shape), dtype=torch.float32, device=phase_dev.device)
    fh.nn_features(phase_dev, L, x)
    if solver is not None:
        fh.nn_response_features(solver, x.view(c, V)[2:])
    return x


def training_pair(solver: fh.Solver, phase_dev, L, tol: float = 1e-6, max_iter: int = 20000,
                  response: bool = True):
    """(input, target) for one microstructure: the d unit loads solved to tol.

    Returns (x, target, infos); target[b * d + a] = e^(b)_a - delta_ab."""
    import torch

    d = solver.d
    fields = []
    infos = []
    for b in range(d):
        E = np.zeros(d)
        E[b] = 1.0
        e, _, info = solver.solve(E, tol=tol, method="cg", max_iter=max_iter)
        fields.append(e)
        infos.append(info)
    t = torch.empty((d * d,) + solver.N, dtype=torch.float32, device=solver.dev)
    x = features(phase_dev, L, solver if response else None)
    fh.nn_targets(fields, t, base(x, d))
    return x, t, infos


def base(x, d: int):
    """The part of the input the network's output is measured from: the
    first-order response channels (B e_b)_a when present, else None.  The
    network then learns the correction e^(b) - e_b + B e_b to the
    fluctuation of the first fixed-point iterate of Eq. (orig_fft)."""
    return x[2:] if x.shape[0] == 2 + d * d else None


def start(solver: fh.Solver, pred, E, base_=None):
    """x0 = E + Q(sum_b E_b (pred_b - base_b)), device float64 [d][N...]."""
    import torch

    x0 = torch.empty((solver.d,) + solver.N, dtype=torch.float64, device=solver.dev)
    return fh.nn_warm_start(solver, pred, E, x0, base_)


class WarmStart:
    """A network for grids N (each a multiple of 27) predicting d unit-load fluctuations."""

    def __init__(self, N: Sequence[int], d: int = 3, channels=None, seed: int = 0, response: bool = True):
        self.N = tuple(int(n) for n in N)
        self.d = d
        self.response = response
        self.cin = 2 + (d * d if response else 0)
        self.net = fh.Net(self.N, self.cin, d * d, channels)
        self.net.set_params(init_params(self.cin, d, seed, channels))

    def close(self):
        self.net.close()

    def features(self, phase_dev, L, solver: fh.Solver):
        return features(phase_dev, L, solver if self.response else None)

    def train(self, pairs, steps: int, lr: float = 1e-3, lr_final: float = 2e-5, warmup: int = 200,
              seed: int = 0):
        """Adam on the mean squared error, one pair per step (order shuffled per
        epoch); linear warm-up over `warmup` steps, then cosine decay from lr to
        lr_final.  Returns the losses."""
        rng = np.random.default_rng(seed)
        losses = []
        order = []
        warmup = min(warmup, max(steps // 4, 1))
        for s in range(steps):
            if not order:
                order = list(rng.permutation(len(pairs)))
            x, t = pairs[order.pop()]
            if s < warmup:
                cur = lr * (s + 1) / warmup
            else:
                q = (s - warmup) / max(steps - warmup - 1, 1)
                cur = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * q))
            losses.append(self.net.train_step(x, t, cur))
        return losses

    def loss(self, x, t) -> float:
        return self.net.gradients(x, t)[0]

    def predict(self, x):
        return self.net.forward(x)

    def start(self, solver: fh.Solver, x, pred, E):
        return start(solver, pred, E, base(x, self.d))

    def solve(self, solver: fh.Solver, x, pred, E, tol: float = 1e-6, method: str = "cg",
              max_iter: int = 20000, x0=None):
        """Solve for load E from the warm start built from input x and prediction
        pred, falling back to e = E when the warm start's true residual is not
        smaller.  Returns (field, column, info) with info["start"] in
        {"warm", "cold"} and the two initial residuals."""
        if x0 is None:
            x0 = self.start(solver, x, pred, E)
        _, _, probe_w = solver.solve(E, tol=tol, method=method, max_iter=0, e_init=x0, want_field=False)
        _, _, probe_c = solver.solve(E, tol=tol, method=method, max_iter=0, want_field=False)
        warm = probe_w["rel_res_true"] < probe_c["rel_res_true"]
        e, col, info = solver.solve(E, tol=tol, method=method, max_iter=max_iter,
                                    e_init=x0 if warm else None)
        info["start"] = "warm" if warm else "cold"
        info["res0_warm"] = probe_w["rel_res_true"]
        info["res0_cold"] = probe_c["rel_res_true"]
        return e, col, info


def timed(fn, *args, **kw):
    """(result, wall seconds) with a device synchronisation on both sides."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn(*args, **kw)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0
