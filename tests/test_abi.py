"""The C-ABI library (CPU checks): it builds, loads, exports every symbol include/mst.h declares,
its struct layout matches the ctypes mirror, and argument validation needs no GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mst.h")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_02110_gb300 as m
    return m


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mst_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(pkg):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mst_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(pkg.lib, n)
    assert set(pkg.EXPORTS) == set(names)


def test_struct_layout_matches_header(pkg):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "mst.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(mst_grid_desc), sizeof(mst_camera), sizeof(mst_params));
  printf("%zu %zu %zu %zu\n", offsetof(mst_params, n_photons), offsetof(mst_params, seed),
         offsetof(mst_params, max_order), offsetof(mst_params, reg_eta));
  printf("%zu %zu\n", offsetof(mst_camera, width), offsetof(mst_camera, fov_x_rad));
  printf("%zu %zu %zu %zu %zu\n", sizeof(mst_channel), offsetof(mst_channel, beta_air_dev),
         offsetof(mst_channel, sigma_ratio), offsetof(mst_channel, images_meas_dev), offsetof(mst_channel, images_dev));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        lines = subprocess.run([exe], capture_output=True, text=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    coffs = [int(x) for x in lines[2].split()]
    assert sizes == [ctypes.sizeof(pkg.GridDesc), ctypes.sizeof(pkg.Camera), ctypes.sizeof(pkg.Params)]
    P = pkg.Params
    assert offs == [P.n_photons.offset, P.seed.offset, P.max_order.offset, P.reg_eta.offset]
    assert coffs == [pkg.Camera.width.offset, pkg.Camera.fov_x_rad.offset]
    ch = [int(x) for x in lines[3].split()]
    C = pkg.Channel
    assert ch == [ctypes.sizeof(C), C.beta_air.offset, C.sigma_ratio.offset, C.images_meas.offset, C.images.offset]


def test_defaults_and_version(pkg):
    p = pkg.default_params()
    assert pkg.lib.mst_version() >= 1
    assert (p.albedo, p.g, p.rr_threshold, p.rr_survival, p.seed) == (0.99, 0.85, 0.01, 0.1, 3)
    assert p.estimator == 0 and p.grid_dtype == 0 and p.grad_mode == 0 and p.conditioning == 0


def test_create_grid_validates_before_touching_a_device(pkg):
    L = pkg.lib
    cam = (pkg.Camera * 1)()
    cam[0].pos = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    cam[0].rot = (ctypes.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    cam[0].width = cam[0].height = 4
    cam[0].fov_x_rad = 1.0
    h = ctypes.c_void_p()
    good = pkg.GridDesc(4, 4, 4, 10.0, 10.0, 10.0, (ctypes.c_double * 3)(0, 0, 0))
    bad_cases = [
        (pkg.GridDesc(0, 4, 4, 10.0, 10.0, 10.0, (ctypes.c_double * 3)(0, 0, 0)), 1, 10),
        (pkg.GridDesc(4, 4, 4, -1.0, 10.0, 10.0, (ctypes.c_double * 3)(0, 0, 0)), 1, 10),
        (good, 0, 10),
        (good, 65, 10),
        (good, 1, 0),
        (good, 1, 65),
        # past the packed voxel index (11 + 11 + 10 bits) or 2^30 voxels
        (pkg.GridDesc(2049, 4, 4, 10.0, 10.0, 10.0, (ctypes.c_double * 3)(0, 0, 0)), 1, 10),
        (pkg.GridDesc(4, 2049, 4, 10.0, 10.0, 10.0, (ctypes.c_double * 3)(0, 0, 0)), 1, 10),
        (pkg.GridDesc(4, 4, 1025, 10.0, 10.0, 10.0, (ctypes.c_double * 3)(0, 0, 0)), 1, 10),
        (pkg.GridDesc(2048, 2048, 257, 10.0, 10.0, 10.0, (ctypes.c_double * 3)(0, 0, 0)), 1, 10),
    ]
    for desc, nc, nr in bad_cases:
        assert L.mst_create_grid(ctypes.byref(desc), nc, cam, nr, ctypes.byref(h)) == -1
        assert not h.value
    assert L.mst_create_grid(None, 1, cam, 10, ctypes.byref(h)) == -1
    cam[0].fov_x_rad = 3.5
    assert L.mst_create_grid(ctypes.byref(good), 1, cam, 10, ctypes.byref(h)) == -1
    L.mst_destroy(None)  # NULL-safe
    assert L.mst_render(None, None, None, None, None, None) == -1
    assert L.mst_sync(None) == -1
    assert L.mst_set_air(None, None, 1.0) == -1
    assert L.mst_sun_mask(None, 0.0, 0.0, 0.1, None, None) == -1
    assert L.mst_render_grad_channels(None, None, 1, None, None, 0.0, None, None, None) == -1
    assert L.mst_set_wavefront(None, 8, 3, 5, 3) == -1
    assert L.mst_autotune(None, None, None, 1 << 20, None, None) == -1


def test_package_refuses_without_library(tmp_path):
    """Importing the binding with the library absent fails loudly (no CPU fallback)."""
    code = ("import sys, os; sys.path.insert(0, %r); import paper_1512_02110_gb300 as m; "
            "m.LIB_PATH='/nonexistent/libmst.so'; m._load()") % ROOT
    r = subprocess.run(["python", "-c", code], capture_output=True, text=True)
    assert r.returncode != 0 and "missing" in r.stderr
