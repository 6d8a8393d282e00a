"""Python binding of libmst (include/mst.h): GB300-native in-situ multi-scattering tomography.

Argument marshalling only. Every step of the render and gradient runs in the CUDA library;
torch provides device memory and the current stream. If libmst.so has not been built this
module raises at import time: there is no CPU fallback.

Units: metres, 1/m, radians. Layouts follow include/mst.h: voxel k = ix + nx*(iy + ny*iz);
per-camera fields [C, nvox]; images flat [sum_c W_c*H_c], camera blocks in order, pixel
(i, j) of a block at j*W + i.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmst.so")

MST_OK = 0
ERRORS = {-1: "invalid argument", -2: "CUDA error", -3: "out of device memory", -4: "no CUDA device",
          -5: "unsupported", -6: "grid too large for the no-allocation scratch"}
EST = {"voxel": 0, "classic": 1}
GRID_DTYPE = {"f32": 0, "f16": 1, "bf16": 2}
GRAD = {"surrogate": 0, "full": 1}
COND = {"none": 0, "inv_count": 1, "count": 2}
NSTATS = 32
STAT_NAMES = ["esc_xm", "esc_xp", "esc_ym", "esc_yp", "esc_zm", "esc_zp", "absorbed", "rr_killed", "rr_gained",
              "forced", "events", "segments", "capped", "escaped_n", "launched", "traced", "replay_segments",
              "replay_events", "los_segments", "pixel_segments", "backproj_segments", "losadj_segments",
              "replay_scatters", "lost", "events_stored", "bmc_paths", "bmc_events", "bmc_segments",
              "air_events", "shadow_rays", "shadow_segments"]
EXPORTS = ["mst_version", "mst_default_params", "mst_create_grid", "mst_destroy", "mst_render", "mst_render_grad",
           "mst_transmittance", "mst_form_images", "mst_surrogate_grad", "mst_ray_counts", "mst_regularizer",
           "mst_set_debug", "mst_set_debug_points", "mst_get_stats", "mst_sync", "mst_last_error", "mst_set_profiling",
           "mst_get_phase_times", "mst_transmittance_noalloc", "mst_batch_create", "mst_batch_render_grad",
           "mst_batch_last_error", "mst_batch_destroy", "mst_set_replay_memory", "mst_render_bmc",
           "mst_set_reg_weights", "mst_set_air", "mst_render_grad_channels", "mst_sun_mask",
           "mst_set_wavefront", "mst_autotune", "mst_batch_set_form", "mst_batch_get_form", "mst_batch_set_wavefront",
           "mst_batch_autotune"]
PHASES = ["stage", "transport", "fold", "los", "images", "backproject", "los_adjoint", "replay", "combine", "replay2",
          "replay_list", "event_adjoint", "bmc"]


class MSTError(RuntimeError):
    pass


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("dz", ctypes.c_double), ("origin", ctypes.c_double * 3)]


class Camera(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("rot", ctypes.c_double * 9), ("width", ctypes.c_int),
                ("height", ctypes.c_int), ("fov_x_rad", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("albedo", ctypes.c_double), ("g", ctypes.c_double), ("sun_zenith_rad", ctypes.c_double),
                ("sun_azimuth_rad", ctypes.c_double), ("sun_irradiance", ctypes.c_double),
                ("rr_threshold", ctypes.c_double), ("rr_survival", ctypes.c_double),
                ("n_photons", ctypes.c_uint64), ("photon_offset", ctypes.c_uint64),
                ("n_photons_total", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("max_order", ctypes.c_int), ("max_events", ctypes.c_int), ("estimator", ctypes.c_int),
                ("grid_dtype", ctypes.c_int), ("grad_mode", ctypes.c_int), ("conditioning", ctypes.c_int),
                ("reg_eta", ctypes.c_double)]


class Channel(ctypes.Structure):  # mst_channel
    _fields_ = [("params", Params), ("beta_air", ctypes.c_void_p), ("albedo_air", ctypes.c_double),
                ("sigma_ratio", ctypes.c_double), ("images_meas", ctypes.c_void_p), ("images", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    L.mst_version.restype = I
    L.mst_default_params.argtypes = [P]
    L.mst_create_grid.argtypes = [P, I, P, I, ctypes.POINTER(P)]
    L.mst_create_grid.restype = I
    L.mst_destroy.argtypes = [P]
    L.mst_render.argtypes = [P, P, P, P, P, P]
    L.mst_render_grad.argtypes = [P, P, P, P, P, P, P, P, P]
    L.mst_transmittance.argtypes = [P, P, I, P, P]
    L.mst_form_images.argtypes = [P, P, I, P, P, P]
    L.mst_surrogate_grad.argtypes = [P, P, P, P, P, P, P, P, P, P, P]
    L.mst_ray_counts.argtypes = [P, P, P]
    L.mst_regularizer.argtypes = [P, P, D, P, P, P]
    L.mst_set_debug.argtypes = [P, P, P]
    L.mst_set_debug_points.argtypes = [P, P]
    L.mst_set_replay_memory.argtypes = [P, ctypes.c_uint64]
    L.mst_set_reg_weights.argtypes = [P, P]
    L.mst_set_air.argtypes = [P, P, ctypes.c_double]
    L.mst_sun_mask.argtypes = [P, D, D, D, P, P]
    L.mst_set_wavefront.argtypes = [P, I, I, I, I]
    L.mst_autotune.argtypes = [P, P, P, ctypes.c_uint64, P, P]
    L.mst_render_grad_channels.argtypes = [P, P, I, P, P, D, P, P, P]
    L.mst_render_bmc.argtypes = [P, P, P, ctypes.c_uint32, P, P, P]
    L.mst_get_stats.argtypes = [P, P]
    L.mst_set_profiling.argtypes = [P, I]
    L.mst_get_phase_times.argtypes = [P, P, P]
    L.mst_transmittance_noalloc.argtypes = [P, I, P, P, P, P]
    L.mst_batch_create.argtypes = [I, P, ctypes.POINTER(P)]
    L.mst_batch_render_grad.argtypes = [P, P, P, P, P, P, P, P, P]
    L.mst_batch_last_error.argtypes = [P]
    L.mst_batch_last_error.restype = ctypes.c_char_p
    L.mst_batch_destroy.argtypes = [P]
    L.mst_batch_set_form.argtypes = [P, I]
    L.mst_batch_get_form.argtypes = [P]
    L.mst_batch_set_wavefront.argtypes = [P, I, I, I, I]
    L.mst_batch_autotune.argtypes = [P, P, P, P, I, P, P]
    L.mst_sync.argtypes = [P]
    L.mst_last_error.argtypes = [P]
    L.mst_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("mst_last_error", "mst_default_params", "mst_destroy", "mst_version", "mst_batch_last_error",
                        "mst_batch_destroy"):
            getattr(L, name).restype = I
    L.mst_destroy.restype = None
    L.mst_batch_destroy.restype = None
    L.mst_default_params.restype = None
    return L


lib = _load()


def default_params() -> Params:
    p = Params()
    lib.mst_default_params(ctypes.byref(p))
    return p


def make_params(src=None, **kw) -> Params:
    """mst_params from any object with the fields of synth.Params (albedo, g, sun_zenith, ...)
    plus keyword overrides (estimator, grid_dtype, grad_mode, conditioning, reg_eta, ...)."""
    p = default_params()
    alias = {"sun_zenith": "sun_zenith_rad", "sun_azimuth": "sun_azimuth_rad"}
    fields = {f for f, _ in Params._fields_}
    items = {}
    if src is not None:
        d = dataclasses.asdict(src) if dataclasses.is_dataclass(src) else dict(vars(src))
        items.update(d)
    items.update(kw)
    for k, v in items.items():
        k = alias.get(k, k)
        if k == "estimator" and isinstance(v, str):
            v = EST[v]
        elif k == "grid_dtype" and isinstance(v, str):
            v = GRID_DTYPE[v]
        elif k == "grad_mode" and isinstance(v, str):
            v = GRAD[v]
        elif k == "conditioning" and isinstance(v, str):
            v = COND[v]
        if k in fields:
            setattr(p, k, v)
    return p


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Grid:
    """A handle (mst_grid) with its cameras: geometry pre-calculation of Sec. 3."""

    def __init__(self, shape, h, origin, cam_pos, cam_rot, cam_w, cam_h, cam_fov, n_rays: int = 10):
        self.shape = tuple(int(s) for s in shape)
        self.nvox = int(np.prod(self.shape))
        cam_pos = np.asarray(cam_pos, dtype=np.float64).reshape(-1, 3)
        self.n_cams = cam_pos.shape[0]
        cam_rot = np.asarray(cam_rot, dtype=np.float64).reshape(self.n_cams, 9)
        cam_w = np.asarray(cam_w).reshape(-1)
        cam_h = np.asarray(cam_h).reshape(-1)
        cam_fov = np.asarray(cam_fov, dtype=np.float64).reshape(-1)
        self.cam_w, self.cam_h = cam_w.astype(np.int64), cam_h.astype(np.int64)
        self.n_pix = int(np.sum(self.cam_w * self.cam_h))
        self.pix_off = np.concatenate([[0], np.cumsum(self.cam_w * self.cam_h)]).astype(np.int64)
        desc = GridDesc(self.shape[0], self.shape[1], self.shape[2], float(h[0]), float(h[1]), float(h[2]),
                        (ctypes.c_double * 3)(*[float(o) for o in origin]))
        cams = (Camera * self.n_cams)()
        for c in range(self.n_cams):
            cams[c].pos = (ctypes.c_double * 3)(*cam_pos[c])
            cams[c].rot = (ctypes.c_double * 9)(*cam_rot[c])
            cams[c].width, cams[c].height = int(cam_w[c]), int(cam_h[c])
            cams[c].fov_x_rad = float(cam_fov[c])
        handle = ctypes.c_void_p()
        rc = lib.mst_create_grid(ctypes.byref(desc), self.n_cams, cams, int(n_rays), ctypes.byref(handle))
        if rc != MST_OK:
            raise MSTError(f"mst_create_grid: {ERRORS.get(rc, rc)}")
        self._h = handle
        self.device = torch.device("cuda", torch.cuda.current_device())

    @classmethod
    def from_scene(cls, scene) -> "Grid":
        return cls(scene.shape, scene.h, scene.origin, scene.cam_pos, scene.cam_rot, scene.cam_w, scene.cam_h,
                   scene.cam_fov, scene.n_rays)

    # -- helpers ------------------------------------------------------------------------------
    def _check(self, rc, what):
        if rc != MST_OK:
            msg = lib.mst_last_error(self._h)
            raise MSTError(f"{what}: {ERRORS.get(rc, rc)}: {msg.decode() if msg else ''}")

    def _t(self, t, n, dtype, name):
        if t is None:
            return None
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor of {n} elements, got "
                             f"{t.device} {t.dtype} {tuple(t.shape)}")
        return t

    def _new(self, n, dtype=torch.float64):
        return torch.empty(n, dtype=dtype, device=self.device)

    # -- calls --------------------------------------------------------------------------------
    def render(self, beta, params: Params, images=True, L=False, stream=None):
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        img = self._new(self.n_pix) if images else None
        Lt = self._new(self.n_cams * self.nvox) if L else None
        self._check(lib.mst_render(self._h, _ptr(beta), ctypes.byref(params), _ptr(img), _ptr(Lt), _stream(stream)),
                    "mst_render")
        return dict(images=img, L=None if Lt is None else Lt.view(self.n_cams, self.nvox))

    def render_grad(self, beta, params: Params, meas, mask=None, images=True, stream=None):
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        meas = self._t(meas, self.n_pix, torch.float64, "images_meas")
        mask = self._t(mask, self.n_pix, torch.uint8, "mask")
        img = self._new(self.n_pix) if images else None
        grad = self._new(self.nvox)
        loss = self._new(1)
        self._check(lib.mst_render_grad(self._h, _ptr(beta), ctypes.byref(params), _ptr(meas), _ptr(mask), _ptr(img),
                                        _ptr(grad), _ptr(loss), _stream(stream)), "mst_render_grad")
        return dict(loss=loss, grad=grad, images=img)

    def transmittance(self, beta, grid_dtype: int = 0, stream=None):
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        T = self._new(self.n_cams * self.nvox, torch.float32)
        self._check(lib.mst_transmittance(self._h, _ptr(beta), int(grid_dtype), _ptr(T), _stream(stream)),
                    "mst_transmittance")
        return T.view(self.n_cams, self.nvox)

    def form_images(self, beta, L, grid_dtype: int = 0, stream=None):
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        L = self._t(L.reshape(-1), self.n_cams * self.nvox, torch.float64, "L")
        img = self._new(self.n_pix)
        self._check(lib.mst_form_images(self._h, _ptr(beta), int(grid_dtype), _ptr(L), _ptr(img), _stream(stream)),
                    "mst_form_images")
        return img

    def surrogate_grad(self, beta, L_ref, beta_ref, params: Params, meas, mask=None, stream=None):
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        L_ref = self._t(L_ref.reshape(-1), self.n_cams * self.nvox, torch.float64, "L_ref")
        beta_ref = self._t(beta_ref, self.nvox, torch.float32, "beta_ref")
        meas = self._t(meas, self.n_pix, torch.float64, "images_meas")
        mask = self._t(mask, self.n_pix, torch.uint8, "mask")
        img, grad, loss = self._new(self.n_pix), self._new(self.nvox), self._new(1)
        self._check(lib.mst_surrogate_grad(self._h, _ptr(beta), _ptr(L_ref), _ptr(beta_ref), ctypes.byref(params),
                                           _ptr(meas), _ptr(mask), _ptr(img), _ptr(grad), _ptr(loss),
                                           _stream(stream)), "mst_surrogate_grad")
        return dict(loss=loss, grad=grad, images=img)

    def sun_mask(self, sun_zenith: float, sun_azimuth: float, radius: float, stream=None):
        """M_c of Eq. Cost: uint8 [n_pix], 0 where the pixel's centre ray is within radius of
        the direction to the sun."""
        m = self._new(self.n_pix, torch.uint8)
        self._check(lib.mst_sun_mask(self._h, float(sun_zenith), float(sun_azimuth), float(radius), _ptr(m),
                                     _stream(stream)), "mst_sun_mask")
        return m

    def ray_counts(self, stream=None):
        Q = self._new(self.n_cams * self.nvox, torch.float32)
        self._check(lib.mst_ray_counts(self._h, _ptr(Q), _stream(stream)), "mst_ray_counts")
        return Q.view(self.n_cams, self.nvox)

    def regularizer(self, beta, eta: float = 1.0, grad=None, stream=None):
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        grad = self._t(grad, self.nvox, torch.float64, "grad")
        psi = self._new(1)
        self._check(lib.mst_regularizer(self._h, _ptr(beta), float(eta), _ptr(psi), _ptr(grad), _stream(stream)),
                    "mst_regularizer")
        return psi

    def set_debug(self, photon_hash=None, photon_skip=None):
        self._check(lib.mst_set_debug(self._h, _ptr(photon_hash), _ptr(photon_skip)), "mst_set_debug")
        self._dbg = (photon_hash, photon_skip)  # keep alive while attached

    def set_debug_points(self, points=None):
        """points: float32 CUDA tensor [n_photons, 4] receiving each photon's last event point
        (offset inside the voxel, then the packed voxel as uint32 bits), or None."""
        self._check(lib.mst_set_debug_points(self._h, _ptr(points)), "mst_set_debug_points")
        self._dbg_points = points  # keep alive while attached

    def stats(self) -> dict:
        out = np.zeros(NSTATS)
        self._check(lib.mst_get_stats(self._h, out.ctypes.data_as(ctypes.c_void_p)), "mst_get_stats")
        return dict(zip(STAT_NAMES, out.tolist()))

    def render_bmc(self, beta, params: Params, n_per_pixel: int, var=True, stream=None):
        """Backward MC images (Eq. ble): dict(images=[total pix] means, var=variance of each mean)."""
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        img = self._new(self.n_pix)
        v = self._new(self.n_pix) if var else None
        self._check(lib.mst_render_bmc(self._h, _ptr(beta), ctypes.byref(params), int(n_per_pixel), _ptr(img), _ptr(v),
                                       _stream(stream)), "mst_render_bmc")
        return dict(images=img, var=v)

    def set_reg_weights(self, wz=None):
        """Altitude weights W of the regulariser, one per layer ([nz]); None restores W = I."""
        if wz is None:
            self._check(lib.mst_set_reg_weights(self._h, None), "mst_set_reg_weights")
            return
        w = np.ascontiguousarray(wz, dtype=np.float64)
        if w.shape != (self.shape[2],):
            raise ValueError(f"need {self.shape[2]} weights, one per layer")
        self._check(lib.mst_set_reg_weights(self._h, w.ctypes.data_as(ctypes.c_void_p)), "mst_set_reg_weights")

    def set_air(self, beta_air=None, albedo_air: float = 1.0):
        """Two-species medium: air extinction [nvox] (float32 on the device) beside the aerosol
        beta of later calls, Rayleigh phase and albedo albedo_air; None restores one species.
        The tensor is kept referenced here while attached (the library borrows it)."""
        beta_air = self._t(beta_air, self.nvox, torch.float32, "beta_air")
        self._check(lib.mst_set_air(self._h, _ptr(beta_air), float(albedo_air)), "mst_set_air")
        self._air = beta_air

    def render_grad_channels(self, beta, channels, mask=None, eta: float = 0.0, images=True, stream=None):
        """Multi-channel loss and gradient w.r.t. the reference aerosol field beta (Eq. channelBeta,
        Eq. Cost, Eq. divCost1). channels: list of dicts with keys params (Params, grad_mode full),
        meas ([n_pix] float64 CUDA tensor), sigma (sigma~_mu), and optionally beta_air ([nvox]
        float32 CUDA tensor) and albedo_air (default 1). Returns dict(loss, grad, images=[per
        channel] or None)."""
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        mask = self._t(mask, self.n_pix, torch.uint8, "mask")
        n = len(channels)
        arr = (Channel * max(n, 1))()
        keep, imgs = [], []
        for i, c in enumerate(channels):
            meas = self._t(c["meas"], self.n_pix, torch.float64, f"channel {i} meas")
            air = self._t(c.get("beta_air"), self.nvox, torch.float32, f"channel {i} beta_air")
            img = self._new(self.n_pix) if images else None
            arr[i].params = c["params"]
            arr[i].beta_air = _ptr(air)
            arr[i].albedo_air = float(c.get("albedo_air", 1.0))
            arr[i].sigma_ratio = float(c["sigma"])
            arr[i].images_meas = _ptr(meas)
            arr[i].images = _ptr(img)
            keep += [meas, air]
            imgs.append(img)
        grad, loss = self._new(self.nvox), self._new(1)
        self._check(lib.mst_render_grad_channels(self._h, _ptr(beta), n, arr, _ptr(mask), float(eta), _ptr(grad),
                                                 _ptr(loss), _stream(stream)), "mst_render_grad_channels")
        return dict(loss=loss, grad=grad, images=imgs if images else None)

    def set_wavefront(self, forward_trip=0, forward_blocks=0, replay_trip=0, replay_blocks=0):
        """Voxels per loop trip and blocks per SM of the forward and pass-2 kernels (0: default)."""
        self._check(lib.mst_set_wavefront(self._h, int(forward_trip), int(forward_blocks), int(replay_trip),
                                          int(replay_blocks)), "mst_set_wavefront")

    def autotune(self, beta, params: Params, n_sample: int = 1 << 24, stream=None) -> dict:
        """Times candidate wavefront shapes on this scene and keeps the fastest (mst_autotune)."""
        beta = self._t(beta, self.nvox, torch.float32, "beta")
        c = (ctypes.c_int * 4)()
        self._check(lib.mst_autotune(self._h, _ptr(beta), ctypes.byref(params), int(n_sample), c, _stream(stream)),
                    "mst_autotune")
        return dict(forward_trip=c[0], forward_blocks_per_sm=c[1], replay_trip=c[2], replay_blocks_per_sm=c[3])

    def set_replay_memory(self, nbytes: int):
        """Budget for the events a full-gradient forward render stores (0: W by replay)."""
        self._check(lib.mst_set_replay_memory(self._h, int(nbytes)), "mst_set_replay_memory")

    def set_profiling(self, enable: bool = True):
        self._check(lib.mst_set_profiling(self._h, int(bool(enable))), "mst_set_profiling")

    def phase_times(self) -> dict:
        """{phase: (ms, launches)} of the last call; needs set_profiling(True) before it."""
        ms = np.zeros(len(PHASES))
        n = np.zeros(len(PHASES), dtype=np.int32)
        self._check(lib.mst_get_phase_times(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                            n.ctypes.data_as(ctypes.c_void_p)), "mst_get_phase_times")
        return {k: (float(a), int(b)) for k, a, b in zip(PHASES, ms, n)}

    def sync(self):
        self._check(lib.mst_sync(self._h), "mst_sync")

    def close(self):
        if getattr(self, "_h", None):
            lib.mst_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """mst_batch: forward + gradient of several scenes (one Grid each) in one CUDA graph."""

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g._h.value for g in self.grids])
        h = ctypes.c_void_p()
        rc = lib.mst_batch_create(len(self.grids), arr, ctypes.byref(h))
        if rc != MST_OK:
            raise MSTError(f"mst_batch_create: {ERRORS.get(rc, rc)}")
        self._h = h
        self._keep = None

    def render_grad(self, betas, params, meas, masks=None, images=False, stream=None):
        """Lists (one entry per scene) of CUDA tensors as in Grid.render_grad; returns
        dict(loss=[n] tensor, grad=[...], images=[...] or None)."""
        n = len(self.grids)
        P = ctypes.c_void_p
        for g, b, m in zip(self.grids, betas, meas):
            g._t(b, g.nvox, torch.float32, "beta")
            g._t(m, g.n_pix, torch.float64, "images_meas")
        grads = [g._new(g.nvox) for g in self.grids]
        imgs = [g._new(g.n_pix) for g in self.grids] if images else None
        losses = torch.empty(n, dtype=torch.float64, device=self.grids[0].device)
        pa = (Params * n)(*params)
        arr = lambda ts: (P * n)(*[None if t is None else t.data_ptr() for t in ts])
        self._keep = (betas, meas, masks, grads, imgs, losses)
        rc = lib.mst_batch_render_grad(self._h, arr(betas), pa, arr(meas), None if masks is None else arr(masks),
                                       None if imgs is None else arr(imgs), arr(grads), _ptr(losses),
                                       _stream(stream))
        if rc != MST_OK:
            msg = lib.mst_batch_last_error(self._h)
            raise MSTError(f"mst_batch_render_grad: {ERRORS.get(rc, rc)}: {msg.decode() if msg else ''}")
        return dict(loss=losses, grad=grads, images=imgs)

    def _check(self, rc, what):
        if rc != MST_OK:
            msg = lib.mst_batch_last_error(self._h)
            raise MSTError(f"{what}: {ERRORS.get(rc, rc)}: {msg.decode() if msg else ''}")

    def set_form(self, form: str):
        """"persistent" (default): the transport of all scenes in single persistent launches;
        "branches": one graph branch per scene (mst_batch_set_form)."""
        self._check(lib.mst_batch_set_form(self._h, {"branches": 0, "persistent": 1}[form]), "mst_batch_set_form")

    def form(self) -> str:
        """Form of the last captured graph."""
        return {0: "branches", 1: "persistent"}.get(lib.mst_batch_get_form(self._h), "none")

    def set_wavefront(self, forward_trip=0, forward_blocks=0, replay_trip=0, replay_blocks=0):
        self._check(lib.mst_batch_set_wavefront(self._h, int(forward_trip), int(forward_blocks), int(replay_trip),
                                                int(replay_blocks)), "mst_batch_set_wavefront")

    def autotune(self, betas, params, meas, sample_div: int = 8, stream=None) -> dict:
        """Times the persistent form's wavefront candidates on a sample of this call (mst_batch_autotune)."""
        n = len(self.grids)
        P = ctypes.c_void_p
        arr = lambda ts: (P * n)(*[t.data_ptr() for t in ts])
        pa = (Params * n)(*params)
        c = (ctypes.c_int * 4)()
        self._check(lib.mst_batch_autotune(self._h, arr(betas), pa, arr(meas), int(sample_div), c, _stream(stream)),
                    "mst_batch_autotune")
        return dict(forward_trip=c[0], forward_blocks_per_sm=c[1], replay_trip=c[2], replay_blocks_per_sm=c[3])

    def close(self):
        if getattr(self, "_h", None):
            lib.mst_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def transmittance_noalloc(shape, h, origin, cam_pos, cam_rot, cam_w, cam_h, cam_fov, beta, T=None, stream=None):
    """mst_transmittance_noalloc: T_c(k) without a handle; the library allocates nothing (its
    scratch is a fixed device array). beta: CUDA float32 [nvox]; T: CUDA float32 [C, nvox]
    (created here if not given). Raises MSTError with MST_ERR_TOO_LARGE for grids past the
    array's size."""
    nvox = int(np.prod(shape))
    cam_pos = np.asarray(cam_pos, dtype=np.float64).reshape(-1, 3)
    nc = cam_pos.shape[0]
    desc = GridDesc(int(shape[0]), int(shape[1]), int(shape[2]), float(h[0]), float(h[1]), float(h[2]),
                    (ctypes.c_double * 3)(*[float(o) for o in origin]))
    cams = (Camera * nc)()
    rot = np.asarray(cam_rot, dtype=np.float64).reshape(nc, 9)
    for c in range(nc):
        cams[c].pos = (ctypes.c_double * 3)(*cam_pos[c])
        cams[c].rot = (ctypes.c_double * 9)(*rot[c])
        cams[c].width, cams[c].height = int(np.ravel(cam_w)[c]), int(np.ravel(cam_h)[c])
        cams[c].fov_x_rad = float(np.ravel(cam_fov)[c])
    if not (beta.is_cuda and beta.dtype == torch.float32 and beta.is_contiguous() and beta.numel() == nvox):
        raise ValueError("beta: need a contiguous CUDA float32 tensor of nvox elements")
    if T is None:
        T = torch.empty(nc, nvox, dtype=torch.float32, device=beta.device)
    rc = lib.mst_transmittance_noalloc(ctypes.byref(desc), nc, cams, _ptr(beta), _ptr(T), _stream(stream))
    if rc != MST_OK:
        raise MSTError(f"mst_transmittance_noalloc: {ERRORS.get(rc, rc)}")
    return T


from .autograd import Blocks, RenderLoss, Scaled, reconstruct  # noqa: E402  (needs `lib` above)
