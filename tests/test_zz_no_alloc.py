"""mst_transmittance_noalloc, the entry point for callers that cannot allocate device memory
(hosts with their own memory arena, plugins that may not allocate after start-up). It must give the same
transmittance as the handle-based mst_transmittance, call after call, using only its fixed
device scratch array. Collected last on purpose: a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_util import dev, f32_scene, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return need_gpu()


def _noalloc(m, sc, beta):
    return m.transmittance_noalloc(sc.shape, sc.h, sc.origin, sc.cam_pos, sc.cam_rot, sc.cam_w, sc.cam_h,
                                   sc.cam_fov, beta)


def test_noalloc_matches_handle_twice(m):
    import torch
    sc = f32_scene(synth.cfg_lognormal32()[0])
    grid = m.Grid.from_scene(sc)
    for scale in (1.0, 0.37):   # two calls in a row: the shared scratch must not leak the first grid
        beta = dev(sc.beta * scale, np.float32)
        ref = grid.transmittance(beta)
        got = _noalloc(m, sc, beta)
        torch.cuda.synchronize()
        err = float(((got - ref).abs() / ref.clamp_min(1e-30)).max())
        assert err <= 1e-6, (scale, err)   # same kernels; the tolerance of the LOS tests is 2e-6 + 2e-5 tau


def test_noalloc_rejects_grids_past_its_scratch(m):
    import torch
    lib = m.lib
    cam = (m.Camera * 1)()
    cam[0].pos = (ctypes.c_double * 3)(10.0, 10.0, 1.0)
    cam[0].rot = (ctypes.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    cam[0].width = cam[0].height = 4
    cam[0].fov_x_rad = 1.0
    beta = torch.zeros(8, dtype=torch.float32, device="cuda")
    T = torch.zeros(8, dtype=torch.float32, device="cuda")
    big = m.GridDesc(136, 128, 128, 1.0, 1.0, 1.0, (ctypes.c_double * 3)(0, 0, 0))
    rc = lib.mst_transmittance_noalloc(ctypes.byref(big), 1, cam, ctypes.c_void_p(beta.data_ptr()),
                                       ctypes.c_void_p(T.data_ptr()), None)
    assert rc == -6
    ok = m.GridDesc(2, 2, 2, 1.0, 1.0, 1.0, (ctypes.c_double * 3)(0, 0, 0))
    T8 = torch.zeros(8, dtype=torch.float32, device="cuda")
    rc = lib.mst_transmittance_noalloc(ctypes.byref(ok), 1, cam, ctypes.c_void_p(beta.data_ptr()),
                                       ctypes.c_void_p(T8.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == 0 and float(T8.min()) == 1.0
