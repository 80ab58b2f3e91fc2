"""Seeded input generators (phase images and tables): each checked against its
definition by brute force over the whole grid, plus the recipe properties the
workloads rely on (digital volume fractions, determinism per seed).  CPU only."""
import math

import numpy as np
import pytest

from paper_1004_1122_gb300 import microstructure as micro


def _brute_inside(shape, centre, radius=None, semi_axes=None, rotation=None):
    """Every node against the inclusion definition: periodic minimum-image
    offset, then |x - c|^2 <= r^2 or the body-frame quadratic form <= 1."""
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    deltas = []
    for a, s in enumerate(shape):
        dl = grids[a] - centre[a]
        deltas.append(dl - s * np.round(dl / s))
    if semi_axes is None:
        return sum(dl * dl for dl in deltas) <= radius * radius
    vec = np.stack(deltas, axis=-1)
    if rotation is not None:
        vec = vec @ rotation
    return sum((vec[..., a] / semi_axes[a]) ** 2 for a in range(len(shape))) <= 1.0


@pytest.mark.parametrize("shape,centre,radius", [
    ((31, 31), (0.2, 30.7), 6.3),          # wraps across both axes
    ((27, 45), (13.0, 22.0), 10.0),        # non-square grid, integer centre
    ((15, 15, 15), (14.5, 0.0, 7.2), 4.1),  # 3-D, wraps
    ((9, 9), (4.0, 4.0), 20.0),            # larger than the grid: everything
])
def test_stamp_ball_matches_definition(shape, centre, radius):
    img = np.zeros(shape, dtype=np.uint8)
    micro._stamp_ball(img, centre, radius, 1)
    assert np.array_equal(img.astype(bool), _brute_inside(shape, centre, radius))


def test_stamp_rotated_ellipse_and_ellipsoid_match_definition():
    th = 0.7
    rot2 = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    img = np.zeros((41, 41), dtype=np.uint8)
    micro._stamp_ball(img, (39.3, 2.1), 9.0, 1, semi_axes=(9.0, 3.0), rotation=rot2)
    assert np.array_equal(img.astype(bool), _brute_inside((41, 41), (39.3, 2.1), semi_axes=(9.0, 3.0),
                                                          rotation=rot2))
    q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    img = np.zeros((21, 21, 21), dtype=np.uint8)
    micro._stamp_ball(img, (1.0, 19.5, 10.2), 7.0, 1, semi_axes=(7.0, 3.5, 2.5), rotation=q)
    assert np.array_equal(img.astype(bool), _brute_inside((21, 21, 21), (1.0, 19.5, 10.2),
                                                          semi_axes=(7.0, 3.5, 2.5), rotation=q))


def test_centred_disk_radius_and_symmetry():
    img = micro.centred_disk(81, 0.3)
    r = math.sqrt(0.3 * 81 * 81 / math.pi)
    assert r == pytest.approx(25.03, abs=5e-3)
    assert np.array_equal(img.astype(bool), _brute_inside((81, 81), (40.0, 40.0), r))
    # centred on the middle node: symmetric under both reflections and the transpose
    assert np.array_equal(img, img[::-1, :]) and np.array_equal(img, img[:, ::-1])
    assert np.array_equal(img, img.T)
    assert abs(micro.digital_fraction(img) - 0.3) < 0.01
    ball = micro.centred_disk(27, 0.2, d=3)
    r3 = (3 * 0.2 * 27 ** 3 / (4 * math.pi)) ** (1 / 3)
    assert np.array_equal(ball.astype(bool), _brute_inside((27, 27, 27), (13.0, 13.0, 13.0), r3))


def test_rsa_disks_recipe():
    a = micro.rsa_disks(243, 0.4, 8, 20, seed=micro.config_seed(2, 1))
    b = micro.rsa_disks(243, 0.4, 8, 20, seed=micro.config_seed(2, 1))
    c = micro.rsa_disks(243, 0.4, 8, 20, seed=micro.config_seed(2, 2))
    assert a.dtype == np.uint8 and set(np.unique(a)) == {0, 1}
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    vf = micro.digital_fraction(a)
    # filled until the target is reached; the last disk adds at most pi rmax^2 nodes
    assert 0.4 <= vf <= 0.4 + math.pi * 21 ** 2 / 243 ** 2


def test_rsa_disks_do_not_overlap():
    # a single seed's disks, re-stamped one by one with distinct labels: with no
    # overlap every node is claimed at most once
    rng_seed = micro.config_seed(2, 7)
    n, vf, rmin, rmax = 101, 0.35, 5, 9
    img = micro.rsa_disks(n, vf, rmin, rmax, seed=rng_seed)
    rng = np.random.default_rng(rng_seed)
    claims = np.zeros((n, n), dtype=np.int32)
    centres, radii, filled = np.zeros((0, 2)), np.zeros((0,)), 0
    while filled < vf * n * n:
        r = rng.uniform(rmin, rmax)
        cc = rng.uniform(0.0, n, size=2)
        if radii.size:
            dl = cc[None, :] - centres
            dl -= n * np.round(dl / n)
            if np.any(np.einsum("ij,ij->i", dl, dl) < (radii + r) ** 2):
                continue
        centres = np.vstack([centres, cc])
        radii = np.append(radii, r)
        claims += _brute_inside((n, n), cc, r)
        filled = int(np.count_nonzero(claims))
    assert claims.max() == 1
    assert np.array_equal(claims.astype(bool), img.astype(bool))


def test_laminate_layers():
    lam = micro.laminate(27, [1 / 3, 2 / 3], axis=0)
    assert np.array_equal(lam[:, 0], np.r_[np.zeros(9), np.ones(18)].astype(np.uint8))
    assert (lam == lam[:, :1]).all()  # depends on the axis-0 coordinate only
    p = micro.laminate((15, 21), [0.4, 0.6], axis=1, seed=4)
    assert (p == p[:1, :]).all()
    assert np.count_nonzero(p[0]) == round(0.6 * 21)
    assert np.array_equal(p, micro.laminate((15, 21), [0.4, 0.6], axis=1, seed=4))
    t = micro.laminate(9, [0.5, 0.25, 0.25], axis=2, d=3)
    assert t.shape == (9, 9, 9) and (t == t[:1, :1, :]).all()
    assert [int(np.count_nonzero(t[0, 0] == k)) for k in range(3)] == [5, 2, 2]


def test_overlapping_models_reach_their_fraction():
    sph = micro.boolean_spheres(45, 4.0, 0.25, seed=micro.config_seed(3))
    assert 0.25 <= micro.digital_fraction(sph) <= 0.25 + 4 / 3 * math.pi * 5 ** 3 / 45 ** 3
    assert np.array_equal(sph, micro.boolean_spheres(45, 4.0, 0.25, seed=micro.config_seed(3)))
    ell = micro.random_ellipses(81, 0.3, 4, 8, 3.0, seed=micro.config_seed(4, 1))
    assert 0.3 <= micro.digital_fraction(ell) <= 0.3 + math.pi * 9 * 3 / 81 ** 2
    e3 = micro.random_ellipsoids(27, 0.2, 2, 4, 3.0, seed=micro.config_seed(5, 2))
    b3 = micro.random_ellipsoids(27, 0.2, 2, 4, 3.0, seed=micro.config_seed(5, 3), spheres=True)
    for v in (e3, b3):
        assert 0.2 <= micro.digital_fraction(v) <= 0.2 + 4 / 3 * math.pi * 5 ** 3 / 27 ** 3


def test_tables_and_seed_rule():
    L = micro.isotropic_table([1.0, 10.0, 100.0], 3)
    assert L.shape == (3, 3, 3) and L.dtype == np.float64
    assert np.array_equal(L[2], 100.0 * np.eye(3))
    assert micro.config_seed(2) == 1200 and micro.config_seed(4, 17) == 1417
    assert micro.digital_fraction(np.array([[0, 2], [1, 0]], dtype=np.uint8)) == 0.5
