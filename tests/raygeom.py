"""Independent numpy geometry for pinning the oracle: camera directions from the pinhole
definition, ray-box clipping by the slab method, and brute-force line integrals by dense
sampling. Nothing here walks voxels the way the oracle or the CUDA path does."""
import math

import numpy as np


def halton(base: int, i: int) -> float:
    f, r = 1.0, 0.0
    while i > 0:
        f /= base
        r += f * (i % base)
        i //= base
    return r


def pixel_dir(scene, c, px, py):
    tx = math.tan(0.5 * scene.cam_fov[c])
    ty = tx * scene.cam_h[c] / scene.cam_w[c]
    x = (2.0 * px / scene.cam_w[c] - 1.0) * tx
    y = (2.0 * py / scene.cam_h[c] - 1.0) * ty
    R = scene.cam_rot[c]
    d = R[6:9] + x * R[0:3] + y * R[3:6]
    return d / np.linalg.norm(d)


def subpixel_dirs(scene, c, i, j):
    return [pixel_dir(scene, c, i + halton(2, r), j + halton(3, r)) for r in range(1, scene.n_rays + 1)]


def box(scene):
    lo = np.array(scene.origin, dtype=np.float64)
    return lo, lo + np.array(scene.shape) * np.array(scene.h)


def ray_box(o, d, lo, hi):
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        if d[a] == 0.0:
            if o[a] < lo[a] or o[a] > hi[a]:
                return None
            continue
        ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    if t0 >= t1:
        return None
    return t0, t1


def chord(o, d, lo, hi):
    r = ray_box(o, d, lo, hi)
    if r is None:
        return 0.0
    return max(0.0, r[1] - max(r[0], 0.0))


def voxel_of(scene, pts):
    lo, _ = box(scene)
    idx = np.floor((pts - lo) / np.array(scene.h)).astype(np.int64)
    nx, ny, nz = scene.shape
    inside = np.all((idx >= 0) & (idx < np.array(scene.shape)), axis=1)
    lin = idx[:, 0] + nx * (idx[:, 1] + ny * idx[:, 2])
    return np.where(inside, lin, -1)


def line_integral(scene, field, o, d, t0, t1, n=200_000):
    """Midpoint rule of field(voxel) along o + t d for t in [t0, t1]."""
    if t1 <= t0:
        return 0.0
    t = t0 + (np.arange(n) + 0.5) * (t1 - t0) / n
    k = voxel_of(scene, o[None, :] + t[:, None] * d[None, :])
    vals = np.where(k >= 0, field[np.maximum(k, 0)], 0.0)
    return float(vals.sum() * (t1 - t0) / n)
