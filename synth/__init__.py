"""Seeded synthetic scenes shaped like the paper's workloads.

This module only builds inputs: extinction fields, camera rigs and parameter
sets. It holds none of the rendering or gradient arithmetic, so both the CUDA
path and the CPU oracle can take their inputs from here without sharing any of
the method's code.

Units are SI throughout: lengths in metres, extinction in 1/m. The paper's
scenes (Sec. 4: 80x80x120 voxels, 36 ground cameras, haze blobs of aides2013)
are not available, so these generators stand in for them: Gaussian haze blobs,
lognormal-modulated blobs and a Kolmogorov-spectrum cumulus field.

Grid convention: voxel (ix, iy, iz) has linear index ix + nx*(iy + ny*iz)
(x fastest). Arrays are returned flattened in that order. Voxel (ix,iy,iz)
covers [origin + i*h, origin + (i+1)*h) on each axis; z is up, the top face
z = origin_z + nz*dz is the top of the atmosphere.

Camera convention: rot = (right, up, forward) as three consecutive 3-vectors
(world-from-camera columns). Pixel (i, j) is column i of W, row j of H; row j
grows along `up`, column i along `right`.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

KM = 1e-3  # 1/km -> 1/m


@dataclasses.dataclass
class Scene:
    shape: tuple            # (nx, ny, nz)
    h: tuple                # (dx, dy, dz) metres
    origin: tuple           # (ox, oy, oz) metres
    beta: np.ndarray        # [nvox] float64, x fastest, 1/m
    cam_pos: np.ndarray     # [C, 3] float64
    cam_rot: np.ndarray     # [C, 9] float64: right, up, forward
    cam_w: np.ndarray       # [C] int32
    cam_h: np.ndarray       # [C] int32
    cam_fov: np.ndarray     # [C] float64, horizontal field of view, radians
    n_rays: int = 10        # sub-pixel rays per pixel (N_rays, Sec. 3.1)
    reg_wz: Optional[np.ndarray] = None  # [nz] altitude weights of the regulariser, None: all 1
    beta_air: Optional[np.ndarray] = None  # [nvox] air (Rayleigh) extinction, None: one species

    @property
    def nvox(self) -> int:
        return int(self.shape[0] * self.shape[1] * self.shape[2])

    @property
    def n_cams(self) -> int:
        return int(self.cam_pos.shape[0])

    @property
    def n_pix(self) -> int:
        return int(np.sum(self.cam_w.astype(np.int64) * self.cam_h))

    def extent(self) -> np.ndarray:
        return np.array(self.shape, dtype=np.float64) * np.array(self.h)

    def with_beta(self, beta: np.ndarray) -> "Scene":
        return dataclasses.replace(self, beta=np.ascontiguousarray(beta, dtype=np.float64).ravel())


@dataclasses.dataclass
class Params:
    albedo: float = 0.99
    g: float = 0.85
    sun_zenith: float = math.radians(30.0)
    sun_azimuth: float = 0.0
    sun_irradiance: float = 1.0
    n_photons: int = 100_000
    photon_offset: int = 0
    n_photons_total: int = 0       # 0: same as n_photons
    seed: int = 3
    max_order: int = 0             # 0: unlimited
    max_events: int = 100_000
    rr_threshold: float = 0.01     # Russian roulette below this fraction of I0
    rr_survival: float = 0.1       # survival probability in roulette
    albedo_air: float = 1.0        # single-scattering albedo of air (two species)

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------------------------
# cameras


def look_up_rot() -> np.ndarray:
    """Camera looking along +z: right = +x, up = +y, forward = +z."""
    return np.array([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=np.float64)


def look_at_rot(forward: Sequence[float], up_hint=(0.0, 0.0, 1.0)) -> np.ndarray:
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    uh = np.asarray(up_hint, dtype=np.float64)
    if abs(np.dot(uh, f)) > 0.999:
        uh = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, uh)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return np.concatenate([r, u, f])


def make_cameras(positions, w: int, h: int, fov_deg: float, rots=None):
    positions = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    c = positions.shape[0]
    if rots is None:
        rots = np.tile(look_up_rot(), (c, 1))
    return dict(cam_pos=positions.copy(), cam_rot=np.asarray(rots, dtype=np.float64).reshape(c, 9),
                cam_w=np.full(c, w, np.int32), cam_h=np.full(c, h, np.int32),
                cam_fov=np.full(c, math.radians(fov_deg), np.float64))


def lattice_xy(extent_x: float, extent_y: float, dx: float, dy: float, n: int = 3) -> np.ndarray:
    """n x n lattice at ((i+0.5)/n)*L, shifted a quarter voxel so no camera sits on a voxel face."""
    pts = []
    for j in range(n):
        for i in range(n):
            pts.append(((i + 0.5) / n * extent_x + 0.25 * dx, (j + 0.5) / n * extent_y + 0.25 * dy))
    return np.array(pts)


def cloud_base_heights(beta: np.ndarray, shape, h, xy: np.ndarray, thresh: float) -> np.ndarray:
    """Lowest voxel layer above (x, y) whose extinction exceeds `thresh` (nz if none)."""
    nx, ny, nz = shape
    b = beta.reshape(nz, ny, nx)
    out = []
    for x, y in xy:
        ix = min(max(int(x // h[0]), 0), nx - 1)
        iy = min(max(int(y // h[1]), 0), ny - 1)
        col = np.nonzero(b[:, iy, ix] > thresh)[0]
        out.append(int(col[0]) if col.size else nz)
    return np.array(out)


def insitu_lattice_cameras(beta, shape, h, w: int, fov_deg: float, n_raised: int = 2,
                           floor_z: float = 1.0, thresh: float = 0.1 * KM):
    """3x3 ground lattice; the n_raised points with the lowest cloud base are lifted to
    the centre height of their cloud-base voxel (in-situ, inside the cloud base)."""
    ext = np.array(shape, dtype=np.float64) * np.array(h)
    xy = lattice_xy(ext[0], ext[1], h[0], h[1], 3)
    base = cloud_base_heights(beta, shape, h, xy, thresh)
    z = np.full(len(xy), floor_z)
    order = np.argsort(base, kind="stable")
    for idx in order[:n_raised]:
        if base[idx] < shape[2]:
            z[idx] = (base[idx] + 0.5) * h[2]
    pos = np.column_stack([xy, z])
    return make_cameras(pos, w, w, fov_deg)


# --------------------------------------------------------------------------------------------
# extinction fields


def _centres(shape, h):
    nx, ny, nz = shape
    x = (np.arange(nx) + 0.5) * h[0]
    y = (np.arange(ny) + 0.5) * h[1]
    z = (np.arange(nz) + 0.5) * h[2]
    return np.meshgrid(x, y, z, indexing="ij")  # each [nx, ny, nz]


def _flat(f_xyz: np.ndarray) -> np.ndarray:
    """[nx, ny, nz] -> flat x-fastest."""
    return np.ascontiguousarray(np.transpose(f_xyz, (2, 1, 0))).ravel()


def blob_field(shape, h, n_blobs: int, sigma_range, max_ext: float, background: float,
               seed: int, inner: float = 0.6) -> np.ndarray:
    """Sum of isotropic Gaussian blobs, centres uniform over the inner fraction of the box,
    scaled so the maximum is max_ext, on top of a uniform background. Returns 1/m, flat."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _centres(shape, h)
    ext = np.array(shape, dtype=np.float64) * np.array(h)
    f = np.zeros(X.shape)
    for _ in range(n_blobs):
        c = ext * (0.5 - inner / 2 + inner * rng.random(3))
        s = rng.uniform(*sigma_range)
        f += np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))
    f = f / f.max() * (max_ext - background) + background
    return _flat(f)


def _smooth_noise(shape, sigma_vox: float, rng) -> np.ndarray:
    g = rng.standard_normal(shape)
    k = [np.fft.fftfreq(n) for n in shape]
    KX, KY, KZ = np.meshgrid(*k, indexing="ij")
    filt = np.exp(-2 * (math.pi ** 2) * (sigma_vox ** 2) * (KX ** 2 + KY ** 2 + KZ ** 2))
    out = np.real(np.fft.ifftn(np.fft.fftn(g) * filt))
    return out / out.std()


def lognormal_blob_field(shape, h, seed: int, n_blobs: int = 6, mean_ext: float = 5 * KM,
                         max_ext: float = 40 * KM, thresh: float = 0.1 * KM) -> np.ndarray:
    """Gaussian blobs modulated by exp(0.5 G), G unit Gaussian noise smoothed over 2 voxels;
    rescaled to the given mean over voxels above `thresh`, clipped at max_ext."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _centres(shape, h)
    ext = np.array(shape, dtype=np.float64) * np.array(h)
    f = np.zeros(X.shape)
    for _ in range(n_blobs):
        c = ext * (0.2 + 0.6 * rng.random(3))
        s = rng.uniform(0.08, 0.18) * ext.min()
        f += np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))
    f = f * np.exp(0.5 * _smooth_noise(shape, 2.0, rng))
    f = f / f.max()
    cloud = f > 0.05
    f = np.where(cloud, f, 0.0)
    f = f * (mean_ext / f[cloud].mean())
    f = np.minimum(f, max_ext)
    f = np.where(f > thresh, f, 0.0) + 0.001 * KM   # thin background
    return _flat(f)


def fractal_field(shape, h, seed: int, cloud_fraction: float = 0.3, max_ext: float = 80 * KM,
                  background: float = 0.0) -> np.ndarray:
    """Gaussian random field with amplitude filter |k|^(-11/6) (1-D spectrum k^(-5/3)),
    thresholded at the (1 - cloud_fraction) quantile; extinction rises linearly from the
    threshold to max_ext at the field maximum."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape)
    k = [np.fft.fftfreq(n) for n in shape]
    KX, KY, KZ = np.meshgrid(*k, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kk[0, 0, 0] = 1.0
    amp = kk ** (-11.0 / 6.0)
    amp[0, 0, 0] = 0.0
    f = np.real(np.fft.ifftn(np.fft.fftn(g) * amp))
    thr = np.quantile(f, 1.0 - cloud_fraction)
    beta = np.where(f > thr, max_ext * (f - thr) / (f.max() - thr), 0.0) + background
    return _flat(beta)


def homogeneous(shape, value: float) -> np.ndarray:
    return np.full(int(np.prod(shape)), float(value))


def air_profile(shape, h, beta0: float, scale_height: float = 8000.0, origin_z: float = 0.0) -> np.ndarray:
    """Air (Rayleigh) extinction beta0 exp(-z / scale_height) at each voxel centre's altitude z,
    flattened x fastest. The molecular scattering coefficient of sea-level air is about 0.0116
    1/km at 550 nm and scales as wavelength^-4; the test scenes raise it so that events on
    air and on aerosol are both frequent."""
    nx, ny, nz = (int(s) for s in shape)
    z = origin_z + (np.arange(nz) + 0.5) * float(h[2])
    col = beta0 * np.exp(-z / scale_height)
    return np.ascontiguousarray(np.broadcast_to(col[:, None, None], (nz, ny, nx)).ravel(), dtype=np.float64)


# --------------------------------------------------------------------------------------------
# named workloads


def make_scene(shape, h, beta, cams: dict, n_rays: int = 10, origin=(0.0, 0.0, 0.0)) -> Scene:
    return Scene(shape=tuple(int(s) for s in shape), h=tuple(float(v) for v in h),
                 origin=tuple(float(v) for v in origin),
                 beta=np.ascontiguousarray(beta, dtype=np.float64).ravel(), n_rays=n_rays, **cams)


def cfg_blobs16(n_photons: int = 100_000):
    """16^3 grid of 50 m voxels, 3 Gaussian blobs (sigma 100-200 m) to 20 1/km over
    0.01 1/km; albedo 0.99, g 0.85, sun zenith 30 deg; 5 floor cameras 32x32, 60 deg."""
    shape, h = (16, 16, 16), (50.0, 50.0, 50.0)
    beta = blob_field(shape, h, 3, (100.0, 200.0), 20 * KM, 0.01 * KM, seed=1)
    L = 16 * 50.0
    cx, cy = L / 2 + 12.5, L / 2 + 12.5
    pos = [(cx, cy, 1.0)] + [(cx + sx * L / 4, cy + sy * L / 4, 1.0) for sx in (-1, 1) for sy in (-1, 1)]
    scene = make_scene(shape, h, beta, make_cameras(pos, 32, 32, 60.0))
    params = Params(albedo=0.99, g=0.85, sun_zenith=math.radians(30.0), n_photons=n_photons, seed=3)
    return scene, params


def cfg_lognormal32(n_photons: int = 10_000_000):
    """32^3 grid of 40 m voxels, lognormal-modulated blobs (mean 5, max 40 1/km), albedo
    0.999, g 0.85, sun zenith 45 deg; 9 cameras 64x64 on a 3x3 lattice, 2 in the cloud base."""
    shape, h = (32, 32, 32), (40.0, 40.0, 40.0)
    beta = lognormal_blob_field(shape, h, seed=1)
    cams = insitu_lattice_cameras(beta, shape, h, 64, 60.0)
    scene = make_scene(shape, h, beta, cams)
    params = Params(albedo=0.999, g=0.85, sun_zenith=math.radians(45.0), n_photons=n_photons, seed=3)
    return scene, params


def cfg_cumulus64(n_photons: int = 100_000_000):
    """64^3 grid of 20 m voxels, k^-5/3 cumulus field at cloud fraction 0.3 up to 80 1/km,
    albedo 0.999, g 0.85, sun zenith 45 deg; 9 in-situ cameras 128x128, 60 deg."""
    shape, h = (64, 64, 64), (20.0, 20.0, 20.0)
    beta = fractal_field(shape, h, seed=1)
    cams = insitu_lattice_cameras(beta, shape, h, 128, 60.0)
    scene = make_scene(shape, h, beta, cams)
    params = Params(albedo=0.999, g=0.85, sun_zenith=math.radians(45.0), n_photons=n_photons, seed=3)
    return scene, params


def haze_field(coarse_shape, coarse_h, seed: int, n_blobs: int = 4, max_ext: float = 0.2 * KM,
               background: float = 0.005 * KM, sigma_xy=(4000.0, 9000.0), sigma_z=(500.0, 1200.0),
               top: float = 3000.0, inner: float = 0.6) -> np.ndarray:
    """Aerosol haze blobs of the kind the paper reconstructs (Sec. 7): Gaussian blobs wide
    across and shallow in altitude (horizontal sigma in sigma_xy, vertical in sigma_z),
    centres uniform over the inner fraction of the box across and below `top` in altitude,
    scaled so the maximum is max_ext over a uniform background. Evaluated at the centres of
    the coarse cells; returns 1/m, flat, x fastest, on the coarse grid."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _centres(coarse_shape, coarse_h)
    ext = np.array(coarse_shape, dtype=np.float64) * np.array(coarse_h)
    f = np.zeros(X.shape)
    for _ in range(n_blobs):
        cx, cy = ext[:2] * (0.5 - inner / 2 + inner * rng.random(2))
        cz = top * rng.random()
        sx, sy = rng.uniform(*sigma_xy, size=2)
        sz = rng.uniform(*sigma_z)
        f += np.exp(-0.5 * (((X - cx) / sx) ** 2 + ((Y - cy) / sy) ** 2 + ((Z - cz) / sz) ** 2))
    f = f / f.max() * (max_ext - background) + background
    return _flat(f)


def refine(coarse: np.ndarray, coarse_shape, factor) -> np.ndarray:
    """A coarse field (flat, x fastest) held constant over blocks of factor = (fx, fy, fz)
    fine voxels: the fine field, flat, x fastest."""
    cx, cy, cz = (int(v) for v in coarse_shape)
    f3 = np.asarray(coarse, dtype=np.float64).reshape(cz, cy, cx)
    f3 = np.repeat(np.repeat(np.repeat(f3, factor[2], 0), factor[1], 1), factor[0], 2)
    return np.ascontiguousarray(f3).ravel()


def cfg_haze80(n_photons: int = 100_000_000, seed: int = 1, fov_deg: float = 150.0):
    """The paper's rendering and reconstruction setting (Secs. 4 and 7), synthetic: a 50 x 50 x
    10 km atmosphere on 80 x 80 x 120 voxels (625 x 625 x 83.3 m); aerosol haze blobs defined on
    the coarse 20 x 20 x 40 grid (blocks of 4 x 4 x 3 voxels) over air at 550 nm (0.0116 1/km at
    the ground, 8 km scale height); sun at 45 deg zenith; 36 ground cameras 7 km apart on a 6 x 6 lattice,
    looking up, 64 x 64 pixels. The paper's cameras are hemispherical; these are pinholes of
    fov_deg horizontal field of view (150 deg: the image corners see 79 deg from the zenith).
    Aerosol albedo 0.9 and g 0.7 (the paper leaves both to its haze model). Returns (scene with
    beta = aerosol and beta_air = air, params, coarse shape, block)."""
    coarse, block = (20, 20, 40), (4, 4, 3)
    shape = tuple(c * b for c, b in zip(coarse, block))
    h = (625.0, 625.0, 10000.0 / 120)
    ch = tuple(v * b for v, b in zip(h, block))
    aer = refine(haze_field(coarse, ch, seed), coarse, block)
    air = air_profile(shape, h, 0.0116 * KM)
    xs = 25000.0 + 7000.0 * (np.arange(6) - 2.5) + 100.0  # off the voxel faces
    pos = [(x, y, 1.0) for y in xs for x in xs]
    scene = make_scene(shape, h, aer, make_cameras(pos, 64, 64, fov_deg))
    scene = dataclasses.replace(scene, beta_air=air)
    params = Params(albedo=0.9, g=0.7, sun_zenith=math.radians(45.0), n_photons=n_photons, seed=3,
                    albedo_air=1.0)
    return scene, params, coarse, block


def smoothed(beta: np.ndarray, shape, frac: float = 0.3) -> np.ndarray:
    """A nearby but different field: (1-frac)*beta + frac*mean(beta)."""
    return (1.0 - frac) * beta + frac * float(beta.mean())


def batch_scenes(n: int = 16, seed: int = 11, max_photons: float = 1e8, min_photons: float = 1e7):
    """Uneven scenes: grids n^3 for n in {24..96}, 20 m voxels, blob or fractal fields,
    albedo U[0.99,0.999], g U[0.75,0.9], sun zenith U[0,60] deg, 3-12 cameras of 64 or 128 px,
    photons log-uniform in [min_photons, max_photons]."""
    rng = np.random.default_rng(seed)
    sizes = [24, 32, 48, 64, 80, 96]
    out = []
    for s in range(n):
        m = int(sizes[s % len(sizes)])
        shape, h = (m, m, m), (20.0, 20.0, 20.0)
        if s % 2 == 0:
            beta = blob_field(shape, h, 4, (3 * 20.0, 8 * 20.0), 40 * KM, 0.01 * KM, seed=100 + s)
        else:
            beta = fractal_field(shape, h, seed=100 + s)
        ncam = int(rng.integers(3, 13))
        px = int(rng.choice([64, 128]))
        ext = m * 20.0
        xy = ext * (0.15 + 0.7 * rng.random((ncam, 2))) + 5.0
        pos = np.column_stack([xy, np.ones(ncam)])
        scene = make_scene(shape, h, beta, make_cameras(pos, px, px, 60.0))
        params = Params(albedo=float(rng.uniform(0.99, 0.999)), g=float(rng.uniform(0.75, 0.9)),
                        sun_zenith=math.radians(float(rng.uniform(0.0, 60.0))),
                        n_photons=int(10 ** rng.uniform(math.log10(min_photons), math.log10(max_photons))),
                        seed=3 + s)
        out.append((scene, params))
    return out
