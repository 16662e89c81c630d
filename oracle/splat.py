"""Headless restatement of GRay's interactive view (Sec. 2, Fig. 1): photon
positions in Boyer-Lindquist coordinates -> Cartesian space -> a camera ->
point sprites deposited into an image.  Plain numpy.

Test infrastructure only: the parity reference for the CUDA splat.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
use it.  Nothing here imports the CUDA library.

The paper draws the live photons of the device buffer with a shader that
performs "coordinate transformation and sprite drawing" and prints neither.
Readings used here:
* transform: the Cartesian coordinates for which Boyer-Lindquist (r, theta,
  phi) are oblate spheroidal, x = sqrt(r^2 + a^2) sin(theta) cos(phi),
  y = sqrt(r^2 + a^2) sin(theta) sin(phi), z = r cos(theta) (flat-space
  Cartesian coordinates when M = 0; a sphere of radius r when a = 0);
* camera: eye point, look-at point and up vector give the orthonormal basis
  forward f = (look - eye)/|look - eye|, right s = f x up / |f x up|,
  true up u = s x f.  A point P at d = P - eye has camera coordinates
  (d.s, d.u, d.f) and is drawn only in front of the eye (d.f > 0).
  Perspective (vertical field of view fov): scale k = (H/2) / tan(fov/2),
  image position (W/2 + k x/z, H/2 - k y/z) in pixels, row 0 at the top;
  orthographic (fov = 0): k = (H/2) / half_height, (W/2 + k x, H/2 - k y);
* sprite: every pixel whose centre lies within `sprite` pixels of the image
  position gets one count; sprite = 0 draws the single pixel containing the
  position.  Counts are integers (additive blending), the depth image keeps
  the smallest d.f per pixel, both independent of drawing order.
"""
import math

import numpy as np


def bl_to_cartesian(a, r, th, ph):
    """Oblate-spheroidal map of Boyer-Lindquist (r, theta, phi)."""
    rho = np.sqrt(np.asarray(r, dtype=np.float64) ** 2 + a * a)
    st = np.sin(th)
    return rho * st * np.cos(ph), rho * st * np.sin(ph), np.asarray(r) * np.cos(th)


def camera_basis(eye, look, up):
    """(right, true up, forward) unit vectors of the camera."""
    eye, look, up = (np.asarray(v, dtype=np.float64) for v in (eye, look, up))
    f = look - eye
    f = f / np.sqrt(np.dot(f, f))
    s = np.cross(f, up)
    s = s / np.sqrt(np.dot(s, s))
    u = np.cross(s, f)
    return s, u, f


def project(cam, X, Y, Z):
    """Image position (px, py) in pixels and depth d.f of Cartesian points;
    visible = in front of the eye."""
    s, u, f = camera_basis(cam["eye"], cam["look"], cam["up"])
    e = np.asarray(cam["eye"], dtype=np.float64)
    dx, dy, dz = np.asarray(X) - e[0], np.asarray(Y) - e[1], np.asarray(Z) - e[2]
    x = dx * s[0] + dy * s[1] + dz * s[2]
    y = dx * u[0] + dy * u[1] + dz * u[2]
    z = dx * f[0] + dy * f[1] + dz * f[2]
    W, H = cam["width"], cam["height"]
    visible = z > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        if cam["fov"] > 0:
            k = 0.5 * H / math.tan(0.5 * cam["fov"])
            px = 0.5 * W + k * x / z
            py = 0.5 * H - k * y / z
        else:
            k = 0.5 * H / cam["half_height"]
            px = 0.5 * W + k * x
            py = 0.5 * H - k * y
    visible &= np.isfinite(px) & np.isfinite(py)
    return px, py, z, visible


def splat(cam, px, py, depth, visible):
    """Count and depth images (H, W) of sprites at (px, py)."""
    W, H, rad = cam["width"], cam["height"], float(cam["sprite"])
    count = np.zeros((H, W), dtype=np.uint32)
    zmin = np.full((H, W), np.inf, dtype=np.float32)
    for x, y, z, ok in zip(px, py, depth, visible):
        if not ok:
            continue
        if rad <= 0:
            i, j = math.floor(x), math.floor(y)
            cells = [(i, j)] if (0 <= i < W and 0 <= j < H) else []
        else:
            i0, i1 = math.ceil(x - rad - 0.5), math.floor(x + rad - 0.5)
            j0, j1 = math.ceil(y - rad - 0.5), math.floor(y + rad - 0.5)
            cells = [(i, j) for j in range(max(j0, 0), min(j1, H - 1) + 1)
                     for i in range(max(i0, 0), min(i1, W - 1) + 1)
                     if (i + 0.5 - x) ** 2 + (j + 0.5 - y) ** 2 <= rad * rad]
        for i, j in cells:
            count[j, i] += 1
            zmin[j, i] = min(zmin[j, i], np.float32(z))
    return count, zmin


def splat_states(cam, a, r, th, ph):
    """Transform, project and splat photon positions (Boyer-Lindquist)."""
    X, Y, Z = bl_to_cartesian(a, r, th, ph)
    px, py, z, vis = project(cam, X, Y, Z)
    return splat(cam, px, py, z, vis)


__all__ = ["bl_to_cartesian", "camera_basis", "project", "splat", "splat_states"]
