"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (derived from the arithmetic: FP32 walks and weights, FP64 final sums):
  deterministic ray kernels (T, images from a given L, surrogate gradient): 1e-4 relative
    per element where the value is not negligible, FP32 walk lengths carry ~1e-6 relative.
  MC forward on photons whose path checksum agrees on both sides: 1e-4 relative per L bin
    and per pixel (spec tolerance); photons whose FP32/FP64 face or roulette
    decisions differ are excluded from both sides through the skip mask.
  gradients: 1e-3 relative L2.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import dev, f32_scene, gpu_hashes, max_rel, need_gpu, quantised, record, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return need_gpu()


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _small_scene():
    shape, h = (12, 10, 9), (40.0, 45.0, 50.0)
    beta = synth.blob_field(shape, h, 3, (60.0, 150.0), 15 * synth.KM, 0.02 * synth.KM, seed=5)
    pos = [(250.0, 230.0, 1.0), (120.0, 300.0, 230.0), (-60.0, 200.0, 210.0)]
    rots = [synth.look_up_rot(), synth.look_at_rot([0.3, -0.2, 1.0]), synth.look_at_rot([1.0, 0.1, 0.2])]
    cams = synth.make_cameras(pos, 24, 20, 60.0, rots=rots)
    return synth.make_scene(shape, h, beta, cams)


SCENES = {"blobs16": lambda: synth.cfg_blobs16()[0], "small": _small_scene,
          "lognormal32": lambda: synth.cfg_lognormal32()[0]}


# ------------------------------------------------------------------------------------------
# deterministic kernels fed identical inputs


@pytest.mark.parametrize("name", ["blobs16", "small", "lognormal32"])
def test_transmittance(m, name):
    sc = f32_scene(SCENES[name]())
    grid = m.Grid.from_scene(sc)
    T = grid.transmittance(dev(sc.beta, np.float32)).cpu().numpy()
    tau, T_or = oracle.transmittance(sc)
    err = np.abs(T - T_or) / np.maximum(T_or, 1e-30)
    tol = 2e-5 * np.maximum(tau, 1.0) + 2e-6
    worst = np.unravel_index(np.argmax(err / tol), err.shape)
    record(f"transmittance[{name}]", max_rel_T=err.max(), worst_over_tol=(err / tol).max(), tau_at_worst=tau[worst])
    assert np.all(err <= tol), (float(np.max(err / tol)), name, worst, tau[worst], T[worst], T_or[worst])


@pytest.mark.parametrize("name", ["blobs16", "small"])
def test_images_from_given_L(m, name):
    sc = f32_scene(SCENES[name]())
    p = synth.Params(n_photons=20_000, seed=11)
    L = oracle.render(sc, p)["L"]
    _, T = oracle.transmittance(sc)
    ref = oracle.images(sc, L, T)
    grid = m.Grid.from_scene(sc)
    img = grid.form_images(dev(sc.beta, np.float32), dev(L, np.float64)).cpu().numpy()
    e = max_rel(img, ref, 1e-3 * np.abs(ref).max())
    record(f"images_from_L[{name}]", max_rel=e)
    assert e < 1e-4


def test_ray_counts(m):
    sc = f32_scene(_small_scene())
    Q = m.Grid.from_scene(sc).ray_counts().cpu().numpy()
    ref = oracle.ray_counts(sc)
    diff = np.abs(Q - ref)
    record("ray_counts", frac_equal=np.mean(diff == 0), max_diff=diff.max())
    # a count differs only where a chord lies within FP32 rounding of the 1e-4 h threshold
    assert diff.max() <= 1
    assert np.mean(diff == 0) > 0.9995


@pytest.mark.parametrize("zen_deg,az,rho_deg", [(0.0, 0.0, 12.0), (20.0, 0.7, 8.0), (30.0, 0.0, 35.0)])
def test_sun_mask(m, zen_deg, az, rho_deg):
    """M_c of Eq. Cost: bit-exact with the oracle except for pixels whose centre ray lies within
    1e-5 rad of the mask edge (the camera axes are FP32 on the device)."""
    from tests import raygeom as rg
    sc = f32_scene(synth.cfg_blobs16()[0])
    zen, rho = math.radians(zen_deg), math.radians(rho_deg)
    mk = m.Grid.from_scene(sc).sun_mask(zen, az, rho).cpu().numpy()
    ref = oracle.sun_mask(sc, zen, az, rho)
    s = np.array([math.sin(zen) * math.cos(az), math.sin(zen) * math.sin(az), math.cos(zen)])
    ang = np.concatenate([[math.acos(min(1.0, float(np.dot(rg.pixel_dir(sc, c, i + 0.5, j + 0.5), s))))
                           for j in range(int(sc.cam_h[c])) for i in range(int(sc.cam_w[c]))]
                          for c in range(sc.n_cams)])
    far = np.abs(ang - rho) > 1e-5
    record(f"sun_mask[{zen_deg},{rho_deg}]", masked=int((ref == 0).sum()), near_edge=int((~far).sum()),
           mismatched_far=int((mk[far] != ref[far]).sum()))
    assert 0 < (ref == 0).sum() < ref.size
    assert np.array_equal(mk[far], ref[far])


@pytest.mark.parametrize("weighted", [False, True])
def test_regularizer(m, torch, weighted):
    import dataclasses
    sc = f32_scene(_small_scene())
    if weighted:  # altitude weights W of Sec. 6, one per layer
        sc = dataclasses.replace(sc, reg_wz=np.linspace(2.0, 0.25, sc.shape[2]))
    grid = m.Grid.from_scene(sc)
    grid.set_reg_weights(sc.reg_wz)
    g = torch.zeros(sc.nvox, dtype=torch.float64, device="cuda")
    psi = grid.regularizer(dev(sc.beta, np.float32), 0.7, g)
    psi_or, g_or = oracle.laplacian(sc)
    assert abs(psi.item() - psi_or) <= 1e-12 * psi_or
    assert rel_l2(g.cpu().numpy(), 0.7 * g_or) < 1e-12
    grid.set_reg_weights(None)
    psi_u = grid.regularizer(dev(sc.beta, np.float32), 0.7, None)
    assert weighted or abs(psi_u.item() - psi_or) <= 1e-12 * psi_or


@pytest.mark.parametrize("cond", ["none", "inv_count"])
def test_surrogate_gradient(m, cond):
    sc0 = f32_scene(synth.cfg_blobs16()[0])
    p = synth.Params(n_photons=30_000, seed=3)
    L_ref = oracle.render(sc0, p)["L"]
    beta_ref = sc0.beta.copy()
    meas = oracle.forward_images(sc0, p.replace(seed=4))[0]
    beta = synth.smoothed(beta_ref, sc0.shape, 0.3).astype(np.float32).astype(np.float64)
    sc = sc0.with_beta(beta)
    mask = (np.arange(sc.n_pix) % 5 != 0).astype(np.uint8)
    ref = oracle.surrogate_grad(sc, L_ref, beta_ref, meas, mask, cond, eta=0.3)
    grid = m.Grid.from_scene(sc)
    out = grid.surrogate_grad(dev(beta, np.float32), dev(L_ref, np.float64), dev(beta_ref, np.float32),
                              m.make_params(conditioning=cond, reg_eta=0.3), dev(meas, np.float64),
                              dev(mask, np.uint8))
    ei = max_rel(out["images"].cpu().numpy(), ref["images"], 1e-3 * np.abs(ref["images"]).max())
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    record(f"surrogate_gradient[{cond}]", images_max_rel=ei, grad_rel_l2=eg, loss_rel=el)
    assert ei < 1e-4 and el < 1e-4 and eg < 1e-3


# ------------------------------------------------------------------------------------------
# Monte-Carlo forward: same Philox streams, per-photon checksums


def _diverged(m, grid, sc, params, beta_dev):
    h_gpu = gpu_hashes(m, grid, beta_dev, m.make_params(params), params.n_photons)
    h_or = oracle.render(sc, params, want_L=False, hashes=True)["hash"]
    return (h_gpu != h_or).astype(np.uint8), h_gpu, h_or


def _forward_parity(m, torch, sc, params, kind="f32", tol=1e-4, name="forward"):
    sc = sc.with_beta(quantised(sc.beta, kind))
    grid = m.Grid.from_scene(sc)
    beta_dev = dev(sc.beta, np.float32)
    mp = m.make_params(params, grid_dtype=kind)
    skip, h_gpu, h_or = _diverged(m, grid, sc, params, beta_dev)
    frac = skip.mean()
    assert frac < 2e-3, frac
    skip_dev = dev(skip, np.uint8)
    grid.set_debug(None, skip_dev)
    out = grid.render(beta_dev, mp, images=True, L=True)
    st = grid.stats()
    grid.set_debug(None, None)
    ref = oracle.render(sc, params, skip=skip)
    _, T = oracle.transmittance(sc)
    img_ref = oracle.images(sc, ref["L"], T)
    L = out["L"].cpu().numpy()
    Lr = ref["L"]
    eL = max_rel(L, Lr, 1e-3 * np.abs(Lr).max())
    eI = max_rel(out["images"].cpu().numpy(), img_ref, 1e-3 * np.abs(img_ref).max())
    record(name, diverged_frac=frac, L_max_rel=eL, images_max_rel=eI,
           segments_rel=abs(st["segments"] - ref["stats"]["segments"]) / ref["stats"]["segments"])
    assert eL < tol and eI < tol, (eL, eI)
    rs = ref["stats"]
    for k in ["events", "traced", "escaped_n", "capped"]:
        assert st[k] == rs[k], (k, st[k], rs[k])
    # zero-length visits at exact voxel-edge crossings may be counted on one side only
    assert abs(st["segments"] - rs["segments"]) <= 1e-5 * rs["segments"], (st["segments"], rs["segments"])
    for k in ["esc_xm", "esc_xp", "esc_ym", "esc_yp", "esc_zm", "esc_zp", "absorbed", "launched"]:
        assert abs(st[k] - rs[k]) <= 1e-5 * rs["launched"], (k, st[k], rs[k])
    return grid, skip, out


def test_forward_blobs16(m, torch):
    sc, p = synth.cfg_blobs16(100_000)
    _forward_parity(m, torch, f32_scene(sc), p, name="forward[blobs16]")


def test_forward_small_scene_roulette_and_order(m, torch):
    """Roulette below 0.6 of the launch weight (reached at the 5th event at albedo 0.9) and the
    order cap at 6 events both end photons."""
    sc = _small_scene()
    p = synth.Params(albedo=0.9, g=0.6, sun_zenith=math.radians(50), sun_azimuth=1.1, n_photons=60_001, seed=77,
                     rr_threshold=0.6, rr_survival=0.3, max_order=6)
    grid, _, _ = _forward_parity(m, torch, f32_scene(sc), p, name="forward[small,roulette,order6]")
    st = grid.stats()
    assert st["rr_killed"] > 0 and st["forced"] > 0, (st["rr_killed"], st["forced"])


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_forward_half_precision_grid(m, torch, kind):
    sc, p = synth.cfg_blobs16(50_000)
    _forward_parity(m, torch, sc, p, kind=kind, name=f"forward[blobs16,{kind}]")


def test_forward_isotropic_vertical_sun(m, torch):
    sc = _small_scene()
    p = synth.Params(albedo=0.95, g=0.0, sun_zenith=0.0, n_photons=30_000, seed=5)
    _forward_parity(m, torch, f32_scene(sc), p, name="forward[small,isotropic,zenith]")


def test_zero_albedo_and_single_photon(m, torch):
    sc = f32_scene(_small_scene())
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    out = grid.render(beta, m.make_params(synth.Params(albedo=0.0, n_photons=5000)), images=True, L=True)
    assert float(out["L"].abs().max()) == 0.0 and float(out["images"].abs().max()) == 0.0
    p1 = synth.Params(n_photons=1, photon_offset=123456, n_photons_total=1000, seed=9)
    h = gpu_hashes(m, grid, beta, m.make_params(p1), 1)
    assert h[0] == oracle.render(sc, p1, want_L=False, hashes=True)["hash"][0]


def _tiny_scene():
    shape, h = (4, 4, 4), (60.0, 60.0, 60.0)
    beta = synth.blob_field(shape, h, 1, (60.0, 90.0), 8 * synth.KM, 0.1 * synth.KM, seed=2)
    return f32_scene(synth.make_scene(shape, h, beta, synth.make_cameras([(121.0, 117.0, 1.0)], 8, 8, 70.0)))


def test_chunk_boundary_and_ragged_count(m, torch):
    """4M photons with a ragged count into a 256-bin tile: the rolling fold sweeps the tile
    (2 slices of 128 bins) every 128 photons while the transport keeps adding to it."""
    p = synth.Params(albedo=0.99, g=0.85, sun_zenith=0.5, n_photons=(1 << 22) + 1003, seed=17)
    _forward_parity(m, torch, _tiny_scene(), p, name="forward[4^3,chunk+ragged]")


@pytest.mark.slow
def test_full_gradient_across_replay_chunks(m, torch):
    """More photons than one replay chunk (2^24), W by replay: two pass-1 / list / pass-2
    rounds, the second ragged, against the oracle's full gradient."""
    sc = _tiny_scene()
    p = synth.Params(albedo=0.99, g=0.85, sun_zenith=0.5, n_photons=(1 << 24) + 1003, seed=23)
    rng = np.random.default_rng(4)
    meas = rng.uniform(0.0, 2e-3, sc.n_pix)
    mask = np.ones(sc.n_pix, np.uint8)
    grid = m.Grid.from_scene(sc)
    grid.set_replay_memory(0)  # W by replay pass 1, chunk by chunk
    beta = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta)
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render_grad(beta, m.make_params(p, grad_mode="full"), dev(meas, np.float64), dev(mask, np.uint8))
    st = grid.stats()
    assert st["events_stored"] == 0
    grid.set_debug(None, None)
    ref = oracle.full_grad(sc, p, meas, mask, skip=skip)
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    record("full_gradient_replay_chunks", diverged_frac=skip.mean(), loss_rel=el, grad_rel_l2=eg)
    assert st["traced"] == p.n_photons - int(skip.sum())
    assert el < 1e-4 and eg < 1e-3, (el, eg)


def test_photon_offset_split(m, torch):
    sc, p = synth.cfg_blobs16(40_000)
    sc = f32_scene(sc)
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    full = grid.render(beta, m.make_params(p), images=False, L=True)["L"].cpu().numpy()
    a = grid.render(beta, m.make_params(p, n_photons=15_000, n_photons_total=40_000), images=False,
                    L=True)["L"].cpu().numpy()
    b = grid.render(beta, m.make_params(p, n_photons=25_000, photon_offset=15_000, n_photons_total=40_000),
                    images=False, L=True)["L"].cpu().numpy()
    e = max_rel(a + b, full, 1e-3 * np.abs(full).max())
    record("photon_offset_split", max_rel=e)
    assert e < 1e-5


def test_classic_estimator(m, torch):
    shape, h = (10, 10, 8), (50.0, 50.0, 50.0)
    beta = synth.blob_field(shape, h, 2, (80.0, 150.0), 6 * synth.KM, 0.2 * synth.KM, seed=8)
    cams = synth.make_cameras([(262.0, 238.0, -40.0), (130.0, 140.0, -25.0)], 12, 12, 60.0)
    sc = f32_scene(synth.make_scene(shape, h, beta, cams))
    p = synth.Params(albedo=0.99, g=0.7, sun_zenith=0.4, n_photons=50_000, seed=19)
    grid = m.Grid.from_scene(sc)
    beta_dev = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta_dev)
    grid.set_debug(None, dev(skip, np.uint8))
    img = grid.render(beta_dev, m.make_params(p, estimator="classic"), images=True)["images"].cpu().numpy()
    grid.set_debug(None, None)
    ref = oracle.render(sc, p, want_L=False, classic=True, skip=skip)["classic"]
    e = max_rel(img, ref, 1e-3 * np.abs(ref).max())
    record("classic_estimator", diverged_frac=skip.mean(), images_max_rel=e)
    assert e < 2e-4


# ------------------------------------------------------------------------------------------
# gradients through mst_render_grad


def _grad_case():
    sc, p = synth.cfg_blobs16(30_000)
    sc = f32_scene(sc)
    meas = oracle.forward_images(sc, p.replace(seed=4))[0]
    beta = synth.smoothed(sc.beta, sc.shape, 0.3).astype(np.float32).astype(np.float64)
    mask = (np.arange(sc.n_pix) % 7 != 3).astype(np.uint8)
    return sc.with_beta(beta), p, meas, mask


def test_full_gradient(m, torch):
    sc, p, meas, mask = _grad_case()
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta)
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render_grad(beta, m.make_params(p, grad_mode="full", reg_eta=0.05), dev(meas, np.float64),
                           dev(mask, np.uint8))
    grid.set_debug(None, None)
    ref = oracle.full_grad(sc, p, meas, mask, eta=0.05, skip=skip)
    ei = max_rel(out["images"].cpu().numpy(), ref["images"], 1e-3 * np.abs(ref["images"]).max())
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    record("full_gradient", diverged_frac=skip.mean(), images_max_rel=ei, loss_rel=el, grad_rel_l2=eg)
    assert ei < 1e-4 and el < 1e-4 and eg < 1e-3


@pytest.mark.parametrize("order", [1, 3])
def test_full_gradient_max_order(m, torch, order):
    """The model truncated at `order` scatterings (order 1: the single-scattering model the
    reconstruction study fits as the paper's baseline): paths end at that event in the forward,
    the stored-event adjoint and replay pass 2 alike."""
    sc, p, meas, mask = _grad_case()
    p = p.replace(max_order=order)
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta)
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render_grad(beta, m.make_params(p, grad_mode="full", reg_eta=0.05), dev(meas, np.float64),
                           dev(mask, np.uint8))
    st = grid.stats()
    grid.set_debug(None, None)
    ref = oracle.full_grad(sc, p, meas, mask, eta=0.05, skip=skip)
    ei = max_rel(out["images"].cpu().numpy(), ref["images"], 1e-3 * np.abs(ref["images"]).max())
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    record(f"full_gradient[max_order={order}]", diverged_frac=skip.mean(), images_max_rel=ei, loss_rel=el,
           grad_rel_l2=eg, events_per_photon=st["events"] / p.n_photons)
    assert st["events_stored"] == st["events"] <= order * p.n_photons
    assert ei < 1e-4 and el < 1e-4 and eg < 1e-3, (ei, el, eg)


def test_full_gradient_classic_estimator(m, torch):
    """Full gradient of the classic local estimate (path score plus shadow-ray terms) against
    the oracle's, photons that FP32 and FP64 send apart excluded from both."""
    sc, p, meas, mask = _grad_case()
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta)
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render_grad(beta, m.make_params(p, grad_mode="full", estimator="classic", reg_eta=0.05),
                           dev(meas, np.float64), dev(mask, np.uint8))
    st = grid.stats()
    grid.set_debug(None, None)
    ref = oracle.full_grad(sc, p, meas, mask, eta=0.05, skip=skip, classic=True)
    ei = max_rel(out["images"].cpu().numpy(), ref["images"], 1e-3 * np.abs(ref["images"]).max())
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    record("full_gradient_classic", diverged_frac=skip.mean(), images_max_rel=ei, loss_rel=el, grad_rel_l2=eg)
    assert st["events_stored"] == 0 and st["replay_segments"] > 0
    assert ei < 2e-4 and el < 1e-4 and eg < 1e-3, (ei, el, eg)


@pytest.mark.parametrize("budget", ["replay", "overflow"])
def test_full_gradient_stored_events_match_replay(m, torch, budget):
    """W from the forward's stored events (the default) against W from replay pass 1: same
    loss and gradient up to the order of floating-point additions. "overflow": a budget of
    2048 events (60 B each with its step), far fewer than the call makes, so the device falls
    back to pass 1."""
    sc, p, meas, mask = _grad_case()
    beta = dev(sc.beta, np.float32)
    args = (beta, m.make_params(p, grad_mode="full", reg_eta=0.05), dev(meas, np.float64), dev(mask, np.uint8))
    g_st = m.Grid.from_scene(sc)
    a = g_st.render_grad(*args)
    st_a = g_st.stats()
    g_rp = m.Grid.from_scene(sc)
    g_rp.set_replay_memory(0 if budget == "replay" else 2048 * 60)
    b = g_rp.render_grad(*args)
    st_b = g_rp.stats()
    assert st_a["events_stored"] == st_a["events"] > 2048
    assert st_b["events_stored"] == 0
    el = abs(a["loss"].item() - b["loss"].item()) / abs(b["loss"].item())
    eg = rel_l2(a["grad"].cpu().numpy(), b["grad"].cpu().numpy())
    record(f"stored_events_vs_{budget}", loss_rel=el, grad_rel_l2=eg, replay_segments_stored=st_a["replay_segments"],
           replay_segments_replay=st_b["replay_segments"])
    assert el < 1e-6 and eg < 1e-5, (el, eg)  # the forward L sums in FP32 atomics in any order
    # pass 2 walks the same photons either way; the replay also walks every path in pass 1
    assert st_b["replay_segments"] > st_a["replay_segments"]


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_full_gradient_half_precision_grid(m, torch, kind):
    """Full gradient with the extinction staged in FP16 / BF16 (FP32 arithmetic): the kernels of
    that grid type (forward storing its events, the stored-event adjoint, replay pass 2 on the
    stored steps, the LOS and image walks) against the oracle on the rounded beta."""
    sc, p, meas, mask = _grad_case()
    sc = sc.with_beta(quantised(sc.beta, kind))
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta)
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render_grad(beta, m.make_params(p, grad_mode="full", grid_dtype=kind, reg_eta=0.05),
                           dev(meas, np.float64), dev(mask, np.uint8))
    st = grid.stats()
    grid.set_debug(None, None)
    ref = oracle.full_grad(sc, p, meas, mask, eta=0.05, skip=skip)
    ei = max_rel(out["images"].cpu().numpy(), ref["images"], 1e-3 * np.abs(ref["images"]).max())
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    record(f"full_gradient[{kind}]", diverged_frac=skip.mean(), images_max_rel=ei, loss_rel=el, grad_rel_l2=eg)
    assert st["events_stored"] == st["events"] > 0 and st["lost"] == 0
    assert ei < 1e-4 and el < 1e-4 and eg < 1e-3, (ei, el, eg)


def test_full_gradient_roulette_on_stored_events(m, torch):
    """Full gradient on the stored events where Russian roulette ends and reweights photons (small
    scene, three cameras in and around the grid, one of them inside the medium; roulette below
    half the launch weight, reached after ~7 events at albedo 0.9): pass 2 must stop where the
    forward stopped and carry the reweighted I, against the oracle."""
    sc = f32_scene(_small_scene())
    p = synth.Params(albedo=0.9, g=0.6, sun_zenith=math.radians(50), sun_azimuth=1.1, n_photons=60_001, seed=77,
                     rr_threshold=0.5, rr_survival=0.3)
    meas = oracle.forward_images(sc, p.replace(seed=4))[0]
    sc = sc.with_beta(synth.smoothed(sc.beta, sc.shape, 0.3).astype(np.float32).astype(np.float64))
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta)
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render_grad(beta, m.make_params(p, grad_mode="full"), dev(meas, np.float64))
    st = grid.stats()
    grid.set_debug(None, None)
    ref = oracle.full_grad(sc, p, meas, skip=skip)
    ei = max_rel(out["images"].cpu().numpy(), ref["images"], 1e-3 * np.abs(ref["images"]).max())
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    record("full_gradient[roulette]", diverged_frac=skip.mean(), images_max_rel=ei, loss_rel=el,
           grad_rel_l2=eg, rr_killed=st["rr_killed"])
    assert st["events_stored"] == st["events"] > 0 and st["lost"] == 0 and st["rr_killed"] > 0
    assert ei < 1e-4 and el < 1e-4 and eg < 1e-3, (ei, el, eg)


def test_record_buffer_follows_the_first_count(m, torch):
    """An optically thick, nearly conservative cube (beta 40 1/km over 0.8 km, albedo 0.999) makes
    tens of events per photon, more than the first call's buffer holds (sized for 4 per photon
    and one chunk per resident warp): that call computes W by replay pass 1 on the device. The
    handle waits for that call's count at its next call, and stores every event from then on,
    with the same loss and gradient."""
    shape, h = (16, 16, 16), (50.0, 50.0, 50.0)
    beta = np.full(int(np.prod(shape)), 40.0 * synth.KM)
    cams = synth.make_cameras([(400.0, 400.0, -30.0), (100.0, 700.0, -30.0)], 16, 16, 60.0)
    sc = f32_scene(synth.make_scene(shape, h, beta, cams))
    p = synth.Params(albedo=0.999, g=0.85, sun_zenith=0.3, n_photons=200_000, seed=5)
    grid = m.Grid.from_scene(sc)
    args = (dev(sc.beta, np.float32), m.make_params(p, grad_mode="full"), dev(np.zeros(sc.n_pix), np.float64))
    a = grid.render_grad(*args)
    s1 = grid.stats()
    b = grid.render_grad(*args)
    s2 = grid.stats()
    el = abs(a["loss"].item() - b["loss"].item()) / abs(b["loss"].item())
    eg = rel_l2(a["grad"].cpu().numpy(), b["grad"].cpu().numpy())
    record("record_buffer_first_count", events_per_photon=s1["events"] / p.n_photons, loss_rel=el, grad_rel_l2=eg)
    assert s1["events"] > 15 * p.n_photons, s1["events"]  # ~27 per photon (oracle)
    assert s1["events_stored"] == 0 and s2["events_stored"] == s2["events"] == s1["events"], (s1, s2)
    assert el < 1e-6 and eg < 1e-5, (el, eg)


def test_surrogate_mode_of_render_grad(m, torch):
    sc, p, meas, mask = _grad_case()
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    skip, _, _ = _diverged(m, grid, sc, p, beta)
    grid.set_debug(None, dev(skip, np.uint8))
    out = grid.render_grad(beta, m.make_params(p, grad_mode="surrogate", conditioning="inv_count"),
                           dev(meas, np.float64), dev(mask, np.uint8))
    grid.set_debug(None, None)
    L = oracle.render(sc, p, skip=skip)["L"]
    ref = oracle.surrogate_grad(sc, L, sc.beta, meas, mask, "inv_count")
    el = abs(out["loss"].item() - ref["loss"]) / ref["loss"]
    eg = rel_l2(out["grad"].cpu().numpy(), ref["grad"])
    record("render_grad_surrogate", loss_rel=el, grad_rel_l2=eg)
    assert el < 1e-4 and eg < 1e-3


def test_invalid_arguments_raise(m, torch):
    sc = f32_scene(_small_scene())
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    with pytest.raises(m.MSTError, match="invalid"):
        grid.render(beta, m.make_params(g=1.0))
    with pytest.raises(m.MSTError, match="invalid"):
        grid.render(beta, m.make_params(estimator="classic"), L=True)
    with pytest.raises(m.MSTError, match="unsupported"):
        grid.render_grad(beta, m.make_params(estimator="classic"), dev(np.zeros(sc.n_pix), np.float64))
    with pytest.raises(ValueError):
        grid.render(dev(sc.beta, np.float64), m.make_params())
    grid.sync()
