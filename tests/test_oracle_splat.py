"""Pins of the splat oracle (the interactive view of Sec. 2, Fig. 1, restated
headless): the Boyer-Lindquist -> Cartesian map against an independent inverse
and against straight photon paths in flat space, the camera against closed
forms, and the sprite deposit against brute force."""
import math

import numpy as np
import pytest

import oracle
from oracle import splat as S

import theory as T


def _cam(**kw):
    c = dict(eye=(50.0, 0.0, 0.0), look=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), fov=math.radians(40.0),
             half_height=10.0, width=64, height=48, sprite=0.0)
    c.update(kw)
    return c


def test_transform_inverts_with_the_oblate_inverse():
    rng = np.random.default_rng(3)
    for a in (0.0, 0.5, 0.999):
        r = rng.uniform(1.0, 40.0, 200)
        th = rng.uniform(0.01, math.pi - 0.01, 200)
        ph = rng.uniform(-math.pi, math.pi, 200)
        X, Y, Z = S.bl_to_cartesian(a, r, th, ph)
        for k in range(200):
            r2, th2, ph2 = T.cart_to_oblate(a, (X[k], Y[k], Z[k]))
            assert r2 == pytest.approx(r[k], rel=1e-12)
            assert th2 == pytest.approx(th[k], abs=1e-10)
            assert T.angle_diff(ph2, ph[k]) == pytest.approx(0.0, abs=1e-12)
        if a == 0.0:
            assert np.allclose(np.sqrt(X * X + Y * Y + Z * Z), r, rtol=1e-14)


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_flat_space_photons_move_on_straight_lines(a):
    """M = 0: the oracle's traced positions, mapped to Cartesian space, lie on
    the straight line of the initial point and direction (a wrong map, e.g.
    r in place of sqrt(r^2 + a^2), bends it)."""
    y0 = oracle.initial(0.0, a, 60.0, math.radians(50.0), 3.0, -2.5)
    P0 = np.array(S.bl_to_cartesian(a, y0[1], y0[2], y0[3]))
    pts = []
    for k in (50, 150, 400):
        rec = oracle.trace(a, 60.0, y0, oracle.Options(M=0.0, max_steps=k))
        y = rec[8:16]
        pts.append(np.array(S.bl_to_cartesian(a, y[1], y[2], y[3])))
    d = pts[-1] - P0
    d /= np.linalg.norm(d)
    for P in pts:
        off = (P - P0) - np.dot(P - P0, d) * d
        # RK4 truncation of the curvilinear straight line is ~1e-7 relative
        assert np.linalg.norm(off) < 1e-6 * max(1.0, np.linalg.norm(P - P0))


def test_camera_closed_forms():
    cam = _cam()
    k = 0.5 * 48 / math.tan(math.radians(20.0))
    px, py, z, vis = S.project(cam, np.array([0.0, 0.0, 0.0, 0.0, 60.0]), np.array([0.0, 2.0, 0.0, 0.0, 0.0]),
                               np.array([0.0, 0.0, 3.0, 0.0, 0.0]))
    assert px[0] == 32.0 and py[0] == 24.0 and z[0] == pytest.approx(50.0)
    assert px[1] == pytest.approx(32.0 + k * 2.0 / 50.0, abs=1e-12) and py[1] == pytest.approx(24.0)
    assert py[2] == pytest.approx(24.0 - k * 3.0 / 50.0, abs=1e-12) and px[2] == pytest.approx(32.0)
    assert vis[:4].all() and not vis[4]  # the last point is behind the eye
    ortho = _cam(fov=0.0, half_height=8.0)
    px, py, _, _ = S.project(ortho, np.array([-30.0]), np.array([2.0]), np.array([-1.0]))
    assert px[0] == pytest.approx(32.0 + 3.0 * 2.0) and py[0] == pytest.approx(24.0 + 3.0 * 1.0)


def _brute(cam, px, py, z, vis):
    W, H, rad = cam["width"], cam["height"], cam["sprite"]
    count = np.zeros((H, W), np.uint32)
    zmin = np.full((H, W), np.inf, np.float32)
    for j in range(H):
        for i in range(W):
            for x, y, d, ok in zip(px, py, z, vis):
                if not ok:
                    continue
                hit = (i <= x < i + 1 and j <= y < j + 1) if rad <= 0 else \
                    (i + 0.5 - x) ** 2 + (j + 0.5 - y) ** 2 <= rad * rad
                if hit:
                    count[j, i] += 1
                    zmin[j, i] = min(zmin[j, i], np.float32(d))
    return count, zmin


@pytest.mark.parametrize("rad", [0.0, 0.7, 2.5])
def test_sprites_match_brute_force(rad):
    rng = np.random.default_rng(11)
    cam = _cam(width=17, height=13, sprite=rad)
    n = 40
    px, py = rng.uniform(-3, 20, n), rng.uniform(-3, 16, n)
    z, vis = rng.uniform(1, 9, n), rng.uniform(0, 1, n) < 0.9
    c1, z1 = S.splat(cam, px, py, z, vis)
    c2, z2 = _brute(cam, px, py, z, vis)
    assert np.array_equal(c1, c2) and np.array_equal(z1, z2)


def test_sprite_area_and_point_count():
    cam = _cam(width=200, height=200, sprite=30.0)
    c, _ = S.splat(cam, np.array([100.3]), np.array([99.8]), np.array([1.0]), np.array([True]))
    assert abs(int(c.sum()) - math.pi * 900.0) < 4 * 2 * math.pi * 30.0 ** 0.7  # Gauss circle bound
    cam0 = _cam(width=10, height=10, sprite=0.0)
    rng = np.random.default_rng(2)
    px, py = rng.uniform(0, 10, 500), rng.uniform(0, 10, 500)
    c0, _ = S.splat(cam0, px, py, np.ones(500), np.ones(500, bool))
    assert int(c0.sum()) == 500
