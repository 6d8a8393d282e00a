"""Degenerate and extreme grids through the C ABI against the oracle: a single voxel, an empty
medium, and grids at the limits of the packed voxel index (2048 voxels along x or y, 1024 along
z), each with the forward render and the full gradient (whose forward stores its events with
the packed index)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import dev, f32_scene, gpu_hashes, max_rel, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return need_gpu()


def _scene(shape, h, beta, cam_xy, cam_z=-5.0, px=8):
    cams = synth.make_cameras([(cam_xy[0], cam_xy[1], cam_z)], px, px, 60.0)
    return f32_scene(synth.make_scene(shape, h, beta, cams))


def _parity(m, sc, p, name, tol=1e-4, per_camera=False):
    """Forward L and images, then the full gradient, on the photons whose paths agree
    (per_camera: also each camera's L row and image to 1e-4 in relative L2)."""
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    h_gpu = gpu_hashes(m, grid, beta, m.make_params(p), p.n_photons)
    h_or = oracle.render(sc, p, want_L=False, hashes=True)["hash"]
    skip = (h_gpu != h_or).astype(np.uint8)
    assert skip.mean() < 2e-3, skip.mean()
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render(beta, m.make_params(p), images=True, L=True)
    st = grid.stats()
    ref = oracle.render(sc, p, skip=skip)
    _, T = oracle.transmittance(sc)
    img_ref = oracle.images(sc, ref["L"], T)
    Lr = ref["L"]
    eL = max_rel(out["L"].cpu().numpy(), Lr, 1e-3 * max(np.abs(Lr).max(), 1e-300))
    eI = max_rel(out["images"].cpu().numpy(), img_ref, 1e-3 * max(np.abs(img_ref).max(), 1e-300))
    eL2 = rel_l2(out["L"].cpu().numpy(), Lr)
    eI2 = rel_l2(out["images"].cpu().numpy(), img_ref)
    for k in ["events", "traced", "escaped_n"]:
        assert st[k] == ref["stats"][k], (k, st[k], ref["stats"][k])
    if per_camera:
        Lg = out["L"].cpu().numpy().reshape(sc.n_cams, -1)
        ig = out["images"].cpu().numpy()
        off = np.concatenate([[0], np.cumsum(sc.cam_w.astype(np.int64) * sc.cam_h)])
        for c in range(sc.n_cams):
            Lc, ic = Lr.reshape(sc.n_cams, -1)[c], img_ref[off[c]:off[c + 1]]
            assert np.abs(Lc).max() > 0 and np.abs(ic).max() > 0, c
            assert rel_l2(Lg[c], Lc) < 1e-4 and rel_l2(ig[off[c]:off[c + 1]], ic) < 1e-4, c
    meas = oracle.forward_images(sc, p.replace(seed=4))[0] * 0.7 + 1e-6
    g = grid.render_grad(beta, m.make_params(p, grad_mode="full"), dev(meas, np.float64))
    gst = grid.stats()
    grid.set_debug(None, None)
    gr = oracle.full_grad(sc, p, meas, skip=skip)
    el = abs(g["loss"].item() - gr["loss"]) / gr["loss"]
    eg = rel_l2(g["grad"].cpu().numpy(), gr["grad"]) if np.abs(gr["grad"]).max() > 0 else \
        float(np.abs(g["grad"].cpu().numpy()).max())
    record(name, diverged_frac=skip.mean(), L_max_rel=eL, images_max_rel=eI, L_rel_l2=eL2, images_rel_l2=eI2,
           loss_rel=el, grad_rel_l2=eg, events=st["events"], events_stored=gst["events_stored"])
    assert eL < tol and eI < tol and eL2 < 1e-4 and eI2 < 1e-4 and el < 1e-4 and eg < 1e-3, (eL, eI, eL2, eI2, el, eg)
    return st, gst


def test_single_voxel(m):
    sc = _scene((1, 1, 1), (100.0, 100.0, 100.0), [10 * synth.KM], (50.0, 47.0))
    p = synth.Params(albedo=0.95, g=0.7, sun_zenith=0.4, n_photons=20_000, seed=5)
    st, gst = _parity(m, sc, p, "edge[single voxel]")
    assert st["events"] > 0 and gst["events_stored"] == gst["events"]


def test_empty_medium(m):
    """beta = 0: no event, every photon leaves the grid along its launch direction with its
    launch weight (through the floor or the -x side for this sun), L and the images vanish; the
    loss is the measured images' energy and the gradient is that of the oracle (no path is
    sampled whose score could carry a derivative)."""
    sc0, p = synth.cfg_blobs16(20_000)
    sc = f32_scene(sc0.with_beta(np.zeros(sc0.nvox)))
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    out = grid.render(beta, m.make_params(p), images=True, L=True)
    st = grid.stats()
    assert float(out["L"].abs().max()) == 0.0 and float(out["images"].abs().max()) == 0.0
    assert st["events"] == 0 and st["escaped_n"] == p.n_photons
    faces = ["esc_xm", "esc_xp", "esc_ym", "esc_yp", "esc_zm", "esc_zp"]
    assert abs(sum(st[f] for f in faces) - st["launched"]) <= 1e-6 * st["launched"]
    rs = oracle.render(sc, p, want_L=False)["stats"]
    for f in faces:
        assert abs(st[f] - rs[f]) <= 1e-6 * rs["launched"], (f, st[f], rs[f])
    assert st["esc_zm"] > 0 and st["esc_xm"] > 0
    meas = np.random.default_rng(3).uniform(0.0, 1e-3, sc.n_pix)
    g = grid.render_grad(beta, m.make_params(p, grad_mode="full"), dev(meas, np.float64))
    gr = oracle.full_grad(sc, p, meas)
    assert abs(g["loss"].item() - gr["loss"]) <= 1e-12 * gr["loss"]
    gg = g["grad"].cpu().numpy()
    assert np.all(np.isfinite(gg)) and np.abs(gg - gr["grad"]).max() <= 1e-12 * max(np.abs(gr["grad"]).max(), 1e-300)


@pytest.mark.parametrize("shape", [(2048, 3, 2), (3, 2048, 2), (2, 2, 1024)])
def test_packed_index_limits(m, shape):
    """Grids at the largest extent each axis of the packed voxel index holds (11, 11 and 10
    bits): the walk, the event stacks and the stored events carry the highest indices. The
    10 km column gets the sun at zenith and optical depth ~2 along it, so that light reaches
    the camera under it. A wrong index would misplace whole contributions (errors of order 1).
    Per bin and pixel the bound is 2e-3: free flights here cross hundreds of voxels of optical
    depth ~2e-3 each, and the FP32 decrement of the flight's optical depth (~3e-8 per voxel)
    moves a collision point by up to centimetres, which tilts the ray to a camera tens of
    metres away (the FP64 oracle has no such drift). In relative L2 the bound stays 1e-4."""
    h = (10.0, 10.0, 10.0)
    rng = np.random.default_rng(11)
    tall = shape[2] == 1024
    beta = synth.KM * rng.uniform(0.1, 0.3, int(np.prod(shape))) if tall else \
        synth.KM * rng.uniform(2.0, 8.0, int(np.prod(shape)))
    ext = np.array(shape) * np.array(h)
    # the camera below the middle of the grid, a quarter voxel off the faces
    sc = _scene(shape, h, beta, (0.5 * ext[0] + 2.5, 0.5 * ext[1] + 2.5))
    p = synth.Params(albedo=0.97, g=0.6, sun_zenith=0.0 if tall else 0.6, sun_azimuth=0.3, n_photons=20_000,
                     seed=9)
    st, gst = _parity(m, sc, p, f"edge[{shape}]", tol=2e-3)
    assert st["events"] > 0 and gst["events_stored"] == gst["events"]


def test_many_cameras(m):
    """41 cameras (past 16, and not a multiple of the 4-camera vector tallies): floor cameras
    on a lattice looking up, plus in-situ cameras inside the medium looking sideways, each
    camera's L row and image against the oracle, then the full gradient. Per bin the bound is
    2e-3 as for the tall column and the two-species medium: one bin is off by 2.6e-4 (with the
    1e-3-of-the-largest-bin floor) while the relative L2 over all bins is 7e-7: the FP32
    drift of one long path (a bin like it in the two-species medium traced to a single photon
    of 33 events); rounding the cameras' positions to FP32 moves no bin by more than 1e-6 in
    the oracle. A camera past the old 16-camera limit read wrongly would miss its
    whole row."""
    shape, h = (12, 12, 12), (50.0, 50.0, 50.0)
    beta = synth.blob_field(shape, h, 3, (80.0, 150.0), 15 * synth.KM, 0.02 * synth.KM, seed=2)
    xs = 600.0 * (np.arange(6) + 0.5) / 6 + 3.0
    pos = [(x, y, 1.0) for y in xs for x in xs] + [(300.0 + 7.0 * i, 290.0, 150.0 + 80.0 * i) for i in range(5)]
    rots = [synth.look_up_rot()] * 36 + [synth.look_at_rot((np.cos(i), np.sin(i), 0.2)) for i in range(5)]
    cams = synth.make_cameras(pos, 8, 6, 70.0, rots=np.array(rots))
    sc = f32_scene(synth.make_scene(shape, h, beta, cams))
    assert sc.n_cams == 41
    p = synth.Params(albedo=0.97, g=0.7, sun_zenith=0.5, sun_azimuth=0.4, n_photons=20_000, seed=6)
    st, gst = _parity(m, sc, p, "edge[41 cameras]", tol=2e-3, per_camera=True)
    assert st["events"] > 0 and gst["events_stored"] == gst["events"]
