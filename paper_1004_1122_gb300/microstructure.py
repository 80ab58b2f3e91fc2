"""Seeded synthetic microstructures (phase images) and phase-tensor tables.

This module produces the *inputs* of the homogenization problem of Section 2.1
(the periodic conductivity field L(x), given as a phase image plus a per-phase
tensor table) and nothing else: it holds none of the solver's arithmetic.
Both the CPU oracle tests and the CUDA path consume what it returns.

Conventions shared by every generator:

* A grid ``N = (N_0, ..., N_{d-1})`` is stored C-order, last axis contiguous.
  Node ``i`` sits at pixel coordinate ``i`` (pixel-centred nodes, Section 2.2);
  the paper's centred indices ``k in Z^N`` differ by a constant integer shift,
  which commutes with the periodic operator.
* A node belongs to an inclusion iff its periodic minimum-image distance to the
  inclusion centre satisfies ``|x - c|^2 <= r^2`` (ellipses/ellipsoids: the
  quadratic form ``<= 1``).
* Phase 0 is the matrix; phase ``p >= 1`` are inclusions.  ``phase`` is
  ``uint8``.
* Volume fractions quoted by the generators are *digital*: count / |N|.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

__all__ = [
    "centred_disk",
    "rsa_disks",
    "random_ellipses",
    "laminate",
    "boolean_spheres",
    "random_ellipsoids",
    "isotropic_table",
    "digital_fraction",
    "config_seed",
]


def config_seed(config: int, item: int = 0) -> int:
    """Seed rule used for every synthetic workload: 1000 + 100*config + item."""
    return 1000 + 100 * int(config) + int(item)


def _periodic_delta(coord: np.ndarray, centre: float, n: int) -> np.ndarray:
    """Minimum-image signed distance along one periodic axis of length n."""
    dlt = coord - centre
    return dlt - n * np.round(dlt / n)


def digital_fraction(phase: np.ndarray) -> float:
    """Fraction of nodes whose phase is non-zero."""
    return float(np.count_nonzero(phase)) / phase.size


def _stamp_ball(img: np.ndarray, centre: Sequence[float], radius: float, value: int,
                semi_axes: Sequence[float] | None = None,
                rotation: np.ndarray | None = None) -> None:
    """Set ``img`` to ``value`` inside a periodic ball / ellipsoid.

    Works on a bounding box around the centre with periodic wrap, so the cost
    is proportional to the inclusion volume, not to the grid.
    """
    d = img.ndim
    shape = img.shape
    reach = radius if semi_axes is None else max(semi_axes)
    idx = []
    for a in range(d):
        lo = int(math.floor(centre[a] - reach)) - 1
        hi = int(math.ceil(centre[a] + reach)) + 1
        span = np.arange(lo, hi + 1)
        if span.size > shape[a]:
            span = np.arange(shape[a])
        idx.append(span)
    grids = np.meshgrid(*idx, indexing="ij")
    deltas = [_periodic_delta(grids[a].astype(np.float64), centre[a], shape[a]) for a in range(d)]
    if semi_axes is None:
        inside = sum(dl * dl for dl in deltas) <= radius * radius
    else:
        vec = np.stack(deltas, axis=-1)
        if rotation is not None:
            vec = vec @ rotation  # coordinates in the body frame
        q = sum((vec[..., a] / semi_axes[a]) ** 2 for a in range(d))
        inside = q <= 1.0
    wrapped = tuple(np.mod(g[inside], shape[a]) for a, g in enumerate(grids))
    img[wrapped] = value


def centred_disk(n: int | Sequence[int], vf: float, d: int = 2) -> np.ndarray:
    """One centred circular (spherical) inclusion at volume fraction ``vf``.

    The radius is chosen so the *continuous* disk/ball has area fraction vf:
    2-D ``r = sqrt(vf |N| / pi)``; 3-D ``r = (3 vf |N| / (4 pi))^(1/3)``.
    The centre is the middle node ``(N-1)/2`` of each axis.  This is the
    single-particle unit cell of the paper's square-array model problem
    (Section 3).
    """
    shape = (n,) * d if isinstance(n, int) else tuple(n)
    size = float(np.prod(shape))
    if len(shape) == 2:
        r = math.sqrt(vf * size / math.pi)
    else:
        r = (3.0 * vf * size / (4.0 * math.pi)) ** (1.0 / 3.0)
    img = np.zeros(shape, dtype=np.uint8)
    _stamp_ball(img, [(s - 1) / 2.0 for s in shape], r, 1)
    return img


def rsa_disks(n: int, vf: float, rmin: float, rmax: float, seed: int,
              max_attempts: int = 2_000_000) -> np.ndarray:
    """Random sequential addition of non-overlapping periodic disks.

    Radii are uniform in [rmin, rmax]; centres uniform on the torus.  A new
    disk is accepted iff its periodic centre distance to every accepted disk is
    at least the sum of the radii.  Disks are added until the digital volume
    fraction reaches ``vf``.
    """
    rng = np.random.default_rng(seed)
    img = np.zeros((n, n), dtype=np.uint8)
    centres = np.zeros((0, 2))
    radii = np.zeros((0,))
    attempts = 0
    filled = 0
    target = vf * n * n
    while filled < target:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError("rsa_disks: jammed before reaching the volume fraction")
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(0.0, n, size=2)
        if radii.size:
            dl = c[None, :] - centres
            dl -= n * np.round(dl / n)
            if np.any(np.einsum("ij,ij->i", dl, dl) < (radii + r) ** 2):
                continue
        centres = np.vstack([centres, c])
        radii = np.append(radii, r)
        _stamp_ball(img, c, r, 1)
        filled = int(np.count_nonzero(img))
    return img


def random_ellipses(n: int, vf: float, amin: float, amax: float, aspect: float,
                    seed: int) -> np.ndarray:
    """Overlapping randomly oriented periodic ellipses until digital vf."""
    rng = np.random.default_rng(seed)
    img = np.zeros((n, n), dtype=np.uint8)
    while digital_fraction(img) < vf:
        a = rng.uniform(amin, amax)
        th = rng.uniform(0.0, math.pi)
        rot = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        _stamp_ball(img, rng.uniform(0.0, n, size=2), a, 1, semi_axes=(a, a / aspect),
                    rotation=rot)
    return img


def laminate(n: int | Sequence[int], fractions: Sequence[float], axis: int = 0,
             d: int = 2, seed: int | None = None) -> np.ndarray:
    """Layered medium: the phase depends on the coordinate along ``axis`` only.

    ``fractions[p]`` is the share of node layers (rounded to whole layers)
    carrying phase ``p``.  Without a seed the phases are stacked in order; with
    a seed the sequence of node layers is a random permutation of that stack.
    """
    shape = (n,) * d if isinstance(n, int) else tuple(n)
    m = shape[axis]
    counts = [int(round(f * m)) for f in fractions]
    counts[0] += m - sum(counts)
    profile = np.concatenate([np.full(c, p, dtype=np.uint8) for p, c in enumerate(counts)])
    if seed is not None:
        profile = np.random.default_rng(seed).permutation(profile)
    view = [1] * len(shape)
    view[axis] = m
    return np.broadcast_to(profile.reshape(view), shape).copy()


def boolean_spheres(n: int, radius: float, vf: float, seed: int) -> np.ndarray:
    """Boolean model: overlapping periodic balls of fixed radius until digital vf."""
    rng = np.random.default_rng(seed)
    img = np.zeros((n, n, n), dtype=np.uint8)
    filled = 0
    target = vf * n ** 3
    while filled < target:
        _stamp_ball(img, rng.uniform(0.0, n, size=3), radius, 1)
        filled = int(np.count_nonzero(img))
    return img


def random_ellipsoids(n: int, vf: float, amin: float, amax: float, aspect_max: float,
                      seed: int, spheres: bool = False) -> np.ndarray:
    """Overlapping randomly oriented periodic ellipsoids (or balls) until digital vf."""
    rng = np.random.default_rng(seed)
    img = np.zeros((n, n, n), dtype=np.uint8)
    while digital_fraction(img) < vf:
        a = rng.uniform(amin, amax)
        c = rng.uniform(0.0, n, size=3)
        if spheres:
            _stamp_ball(img, c, a, 1)
            continue
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        asp = rng.uniform(1.0, aspect_max, size=2)
        _stamp_ball(img, c, a, 1, semi_axes=(a, a / asp[0], a / asp[1]), rotation=q)
    return img


def isotropic_table(conductivities: Sequence[float], d: int) -> np.ndarray:
    """Per-phase tensor table ``L[p] = c_p * I`` of shape (nphase, d, d), float64."""
    c = np.asarray(conductivities, dtype=np.float64)
    return c[:, None, None] * np.eye(d)[None, :, :]
