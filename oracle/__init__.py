"""ctypes wrapper of the FP64 CPU oracle (oracle/mst_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
bench.py use it to check the CUDA path. The product package never imports it,
and it imports nothing from the product package.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mst_oracle.c")
_LIB = os.path.join(_HERE, "libmst_oracle.so")

ST_NAMES = ["esc_xm", "esc_xp", "esc_ym", "esc_yp", "esc_zm", "esc_zp", "absorbed", "rr_killed",
            "rr_gained", "forced", "events", "segments", "capped", "escaped_n", "launched", "traced"]
COND = {"none": 0, "inv_count": 1, "count": 2}


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("n_cams", ctypes.c_int),
                ("n_rays", ctypes.c_int), ("pad_", ctypes.c_int),
                ("h", ctypes.c_double * 3), ("o", ctypes.c_double * 3),
                ("beta", ctypes.c_void_p), ("cam_pos", ctypes.c_void_p), ("cam_rot", ctypes.c_void_p),
                ("cam_w", ctypes.c_void_p), ("cam_h", ctypes.c_void_p), ("cam_fov", ctypes.c_void_p),
                ("reg_wz", ctypes.c_void_p), ("beta_air", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("albedo", ctypes.c_double), ("g", ctypes.c_double), ("sun_zenith", ctypes.c_double),
                ("sun_azimuth", ctypes.c_double), ("sun_irradiance", ctypes.c_double),
                ("rr_threshold", ctypes.c_double), ("rr_survival", ctypes.c_double),
                ("n_photons", ctypes.c_uint64), ("photon_offset", ctypes.c_uint64),
                ("n_photons_total", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("max_order", ctypes.c_int), ("max_events", ctypes.c_int), ("albedo_air", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_u01.argtypes = [ctypes.c_uint32]
        L.or_u01.restype = ctypes.c_double
        L.or_hg_phase.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_hg_phase.restype = ctypes.c_double
        L.or_hg_sample.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_hg_sample.restype = ctypes.c_double
        L.or_rayleigh_phase.argtypes = [ctypes.c_double]
        L.or_rayleigh_phase.restype = ctypes.c_double
        L.or_rayleigh_sample.argtypes = [ctypes.c_double]
        L.or_rayleigh_sample.restype = ctypes.c_double
        L.or_rotate.argtypes = [P, ctypes.c_double, ctypes.c_double, P]
        L.or_radical_inverse.argtypes = [ctypes.c_int, ctypes.c_int]
        L.or_radical_inverse.restype = ctypes.c_double
        L.or_render.argtypes = [P, P, P, P, P, P, P, ctypes.c_int, P]
        L.or_transmittance.argtypes = [P, P, P]
        L.or_los_adjoint.argtypes = [P, P, P]
        L.or_images.argtypes = [P, P, P, P]
        L.or_backproject.argtypes = [P, P, P]
        L.or_ray_counts.argtypes = [P, P]
        L.or_laplacian.argtypes = [P, P, P, P]
        L.or_surrogate_grad.argtypes = [P, P, P, P, P, ctypes.c_int, ctypes.c_double, P, P, P]
        L.or_full_grad.argtypes = [P, P, P, P, ctypes.c_double, ctypes.c_int, P, P, P, P, P, P]
        L.or_full_grad_classic.argtypes = [P, P, P, P, ctypes.c_double, ctypes.c_int, P, P, P, P, P]
        L.or_bmc_pixel.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, P, P]
        L.or_sun_mask.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P]
        L.or_particle_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        L.or_particle_uniform.restype = ctypes.c_double
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _Bound:
    """Keeps the numpy arrays behind a scene struct alive for the call."""

    def __init__(self, scene, beta=None):
        self.beta = np.ascontiguousarray(scene.beta if beta is None else beta, dtype=np.float64)
        self.pos = np.ascontiguousarray(scene.cam_pos, dtype=np.float64)
        self.rot = np.ascontiguousarray(scene.cam_rot, dtype=np.float64)
        self.w = np.ascontiguousarray(scene.cam_w, dtype=np.int32)
        self.h = np.ascontiguousarray(scene.cam_h, dtype=np.int32)
        self.fov = np.ascontiguousarray(scene.cam_fov, dtype=np.float64)
        s = _Scene()
        s.nx, s.ny, s.nz = scene.shape
        s.n_cams = scene.n_cams
        s.n_rays = scene.n_rays
        s.h = (ctypes.c_double * 3)(*scene.h)
        s.o = (ctypes.c_double * 3)(*scene.origin)
        s.beta, s.cam_pos, s.cam_rot = _ptr(self.beta), _ptr(self.pos), _ptr(self.rot)
        s.cam_w, s.cam_h, s.cam_fov = _ptr(self.w), _ptr(self.h), _ptr(self.fov)
        air = getattr(scene, "beta_air", None)
        if air is not None:  # two species: the oracle's beta is the total extinction
            self.air = np.ascontiguousarray(air, dtype=np.float64)
            self.beta = np.ascontiguousarray(self.beta + self.air)
            s.beta = _ptr(self.beta)
            s.beta_air = _ptr(self.air)
        wz = getattr(scene, "reg_wz", None)
        self.wz = None if wz is None else np.ascontiguousarray(wz, dtype=np.float64)
        s.reg_wz = None if self.wz is None else _ptr(self.wz)
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _params(p) -> _Params:
    q = _Params()
    q.albedo, q.g = p.albedo, p.g
    q.sun_zenith, q.sun_azimuth, q.sun_irradiance = p.sun_zenith, p.sun_azimuth, p.sun_irradiance
    q.rr_threshold, q.rr_survival = p.rr_threshold, p.rr_survival
    q.n_photons, q.photon_offset, q.n_photons_total, q.seed = p.n_photons, p.photon_offset, p.n_photons_total, p.seed
    q.max_order, q.max_events = p.max_order, p.max_events
    q.albedo_air = getattr(p, "albedo_air", 1.0)
    return q


# ------------------------------------------------------------------------------------------
# primitives


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(x: int) -> float:
    return lib().or_u01(int(x))


def hg_phase(g: float, mu: float) -> float:
    return lib().or_hg_phase(g, mu)


def hg_sample(g: float, u: float) -> float:
    return lib().or_hg_sample(g, u)


def particle_uniform(seed: int, photon: int, event: int) -> float:
    return lib().or_particle_uniform(int(seed), int(photon), int(event))


def rayleigh_phase(mu: float) -> float:
    return lib().or_rayleigh_phase(mu)


def rayleigh_sample(u: float) -> float:
    return lib().or_rayleigh_sample(u)


def rotate(d, ct: float, phi: float):
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(3)
    lib().or_rotate(_ptr(dd), ct, phi, _ptr(out))
    return out


def radical_inverse(base: int, i: int) -> float:
    return lib().or_radical_inverse(base, i)


# ------------------------------------------------------------------------------------------
# the method


def render(scene, params, want_L=True, classic=False, hashes=False, skip=None, nthreads=0, points=False):
    """Forward MC. Returns dict(L [C,nvox] or None, classic [npix] or None, stats, hash, point):
    point [n, 3] (points=True) is each photon's last event point in grid coordinates (metres
    from the grid origin; the launch point for a photon without events)."""
    b = _Bound(scene)
    q = _params(params)
    L = np.zeros((scene.n_cams, scene.nvox)) if want_L else None
    ci = np.zeros(scene.n_pix) if classic else None
    st = np.zeros(16)
    h = np.zeros(params.n_photons, np.uint32) if hashes else None
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.uint8)
    pt = np.zeros((params.n_photons, 3)) if points else None
    lib().or_render(b.ref, ctypes.byref(q), _ptr(L), _ptr(ci), _ptr(st), _ptr(h), _ptr(sk), int(nthreads), _ptr(pt))
    return dict(L=L, classic=ci, stats=dict(zip(ST_NAMES, st.tolist())), hash=h, point=pt)


def transmittance(scene, beta=None):
    b = _Bound(scene, beta)
    tau = np.zeros((scene.n_cams, scene.nvox))
    T = np.zeros((scene.n_cams, scene.nvox))
    lib().or_transmittance(b.ref, _ptr(tau), _ptr(T))
    return tau, T


def los_adjoint(scene, sv):
    b = _Bound(scene)
    s = np.ascontiguousarray(sv, dtype=np.float64).reshape(scene.n_cams, scene.nvox)
    out = np.zeros((scene.n_cams, scene.nvox))
    lib().or_los_adjoint(b.ref, _ptr(s), _ptr(out))
    return out


def images(scene, L, T):
    b = _Bound(scene)
    Lc = np.ascontiguousarray(L, dtype=np.float64).reshape(scene.n_cams, scene.nvox)
    Tc = np.ascontiguousarray(T, dtype=np.float64).reshape(scene.n_cams, scene.nvox)
    img = np.zeros(scene.n_pix)
    lib().or_images(b.ref, _ptr(Lc), _ptr(Tc), _ptr(img))
    return img


def backproject(scene, rr):
    b = _Bound(scene)
    r = np.ascontiguousarray(rr, dtype=np.float64).ravel()
    out = np.zeros((scene.n_cams, scene.nvox))
    lib().or_backproject(b.ref, _ptr(r), _ptr(out))
    return out


def ray_counts(scene):
    b = _Bound(scene)
    out = np.zeros((scene.n_cams, scene.nvox))
    lib().or_ray_counts(b.ref, _ptr(out))
    return out


def laplacian(scene, beta=None):
    b = _Bound(scene, beta)
    psi = ctypes.c_double()
    g = np.zeros(scene.nvox)
    lib().or_laplacian(b.ref, _ptr(b.beta), ctypes.byref(psi), _ptr(g))
    return psi.value, g


def surrogate_grad(scene, L_ref, beta_ref, meas, mask=None, conditioning="none", eta=0.0):
    b = _Bound(scene)
    Lr = np.ascontiguousarray(L_ref, dtype=np.float64).reshape(scene.n_cams, scene.nvox)
    br = np.ascontiguousarray(beta_ref, dtype=np.float64)
    m = np.ascontiguousarray(meas, dtype=np.float64).ravel()
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).ravel()
    img = np.zeros(scene.n_pix)
    g = np.zeros(scene.nvox)
    loss = ctypes.c_double()
    lib().or_surrogate_grad(b.ref, _ptr(Lr), _ptr(br), _ptr(m), _ptr(mk), COND[conditioning], float(eta),
                            _ptr(img), _ptr(g), ctypes.byref(loss))
    return dict(images=img, grad=g, loss=loss.value)


def full_grad(scene, params, meas, mask=None, eta=0.0, nthreads=0, skip=None, classic=False):
    """Loss and full gradient (score replay) of the voxel estimator, or of the classic local
    estimator with classic=True (images by Eq. fle; no L)."""
    b = _Bound(scene)
    q = _params(params)
    m = np.ascontiguousarray(meas, dtype=np.float64).ravel()
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).ravel()
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.uint8)
    img = np.zeros(scene.n_pix)
    g = np.zeros(scene.nvox)
    L = np.zeros((scene.n_cams, scene.nvox))
    st = np.zeros(16)
    loss = ctypes.c_double()
    if classic:
        lib().or_full_grad_classic(b.ref, ctypes.byref(q), _ptr(m), _ptr(mk), float(eta), int(nthreads), _ptr(img),
                                   _ptr(g), ctypes.byref(loss), _ptr(st), _ptr(sk))
        L = None
    else:
        lib().or_full_grad(b.ref, ctypes.byref(q), _ptr(m), _ptr(mk), float(eta), int(nthreads), _ptr(img),
                           _ptr(g), ctypes.byref(loss), _ptr(L), _ptr(st), _ptr(sk))
    return dict(images=img, grad=g, loss=loss.value, L=L, stats=dict(zip(ST_NAMES, st.tolist())))


def channels_grad(scene, beta_ref, channels, mask=None, eta=0.0, skip=None, nthreads=0, classic=False,
                  surrogate=False, conditioning="none"):
    """Multi-channel loss and gradient w.r.t. the reference aerosol field (Eq. channelBeta,
    Eq. Cost, Eq. divCost1). Channel mu renders the two-species medium with aerosol
    sigma_mu * beta_ref and its own air field: beta_mu = beta_air_mu + sigma_mu beta_ref. The loss
    is the sum of the channels' masked L2 losses plus eta Psi(beta_ref), once; the gradient is
    sum_mu sigma_mu dE_mu/dbeta_aerosol_mu + eta dPsi/dbeta_ref (chain rule through
    Eq. channelBeta). channels: dicts with params (albedo_air inside), sigma, meas and beta_air
    (None: no air in that channel). surrogate=True: each channel's dE_mu/dbeta_mu is the
    surrogate with j = L_mu / beta_mu fixed (Eq. divCost1 with Q_c), L_mu rendered here at the
    channel's total field."""
    import dataclasses
    beta_ref = np.asarray(beta_ref, dtype=np.float64)
    loss, grad, imgs = 0.0, np.zeros(scene.nvox), []
    for ch in channels:
        sc = dataclasses.replace(scene, beta=ch["sigma"] * beta_ref, beta_air=ch.get("beta_air"))
        if surrogate:
            L = render(sc, ch["params"], skip=skip, nthreads=nthreads)["L"]
            tot = sc.beta + (0.0 if sc.beta_air is None else np.asarray(sc.beta_air, dtype=np.float64))
            r = surrogate_grad(sc, L, tot, ch["meas"], mask, conditioning, eta=0.0)
        else:
            r = full_grad(sc, ch["params"], ch["meas"], mask, eta=0.0, nthreads=nthreads, skip=skip,
                          classic=classic)
        loss += r["loss"]
        grad += ch["sigma"] * r["grad"]
        imgs.append(r["images"])
    if eta != 0.0:
        psi, dpsi = laplacian(dataclasses.replace(scene, beta_air=None), beta_ref)
        loss += eta * psi
        grad += eta * dpsi
    return dict(loss=loss, grad=grad, images=imgs)


def sun_mask(scene, zenith, azimuth, radius):
    """M_c of Eq. Cost: uint8 [n_pix], 0 where the pixel's centre ray is within radius of the
    direction to the sun."""
    b = _Bound(scene)
    m = np.zeros(scene.n_pix, np.uint8)
    lib().or_sun_mask(b.ref, float(zenith), float(azimuth), float(radius), _ptr(m))
    return m


def bmc_pixel(scene, params, cam: int, i: int, j: int, n: int):
    b = _Bound(scene)
    q = _params(params)
    mean, var = ctypes.c_double(), ctypes.c_double()
    lib().or_bmc_pixel(b.ref, ctypes.byref(q), cam, i, j, int(n), ctypes.byref(mean), ctypes.byref(var))
    return mean.value, math.sqrt(max(var.value, 0.0))


def forward_images(scene, params, nthreads=0, skip=None):
    """The voxelised method end to end: L by MC, T by LOS, images by Eq. Icpixel."""
    r = render(scene, params, skip=skip, nthreads=nthreads)
    _, T = transmittance(scene)
    return images(scene, r["L"], T), r
