"""Parity at the full benchmark size (64^3 cumulus field, 9 in-situ 128x128 cameras, 1e8
photons, forward + full gradient in the benchmark's launch configuration), on outputs the
oracle can compute one by one (sampled photon paths, LOS transmittance, image formation from
an oracle L) and on invariants that hold at any size (energy balance)."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import dev, f32_scene, max_rel, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return need_gpu()


@pytest.fixture(scope="module")
def case(m):
    import torch
    sc, p = synth.cfg_cumulus64()
    sc = f32_scene(sc)
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    hashes = torch.zeros(p.n_photons, dtype=torch.int32, device="cuda")
    grid.set_debug(hashes, None)
    meas = dev(np.zeros(sc.n_pix), np.float64)
    out = grid.render_grad(beta, m.make_params(p, grad_mode="full"), meas)
    st = grid.stats()
    grid.set_debug(None, None)
    return dict(sc=sc, p=p, grid=grid, beta=beta, out=out, stats=st, hashes=hashes.cpu().numpy().view(np.uint32))


def test_sampled_photon_paths(case):
    sc, p, h = case["sc"], case["p"], case["hashes"]
    rng = np.random.default_rng(0)
    starts = rng.integers(0, p.n_photons - 200, 16)
    agree = total = 0
    for s in starts:
        q = p.replace(n_photons=200, photon_offset=int(s), n_photons_total=p.n_photons)
        ho = oracle.render(sc, q, want_L=False, hashes=True)["hash"]
        agree += int(np.sum(ho == h[s:s + 200]))
        total += 200
    record("fullsize_photon_paths", agree_frac=agree / total)
    assert agree / total > 0.99, agree / total


def test_energy_balance_full_size(case):
    st, sc, p = case["stats"], case["sc"], case["p"]
    esc = sum(st[k] for k in ["esc_xm", "esc_xp", "esc_ym", "esc_yp", "esc_zm", "esc_zp"])
    out = esc + st["absorbed"] + st["rr_killed"] + st["forced"] - st["rr_gained"]
    incident = math.cos(p.sun_zenith) * sc.extent()[0] * sc.extent()[1]
    assert st["traced"] == p.n_photons
    assert abs(st["launched"] - incident) < 1e-5 * incident
    record("fullsize_energy", launched_rel=abs(st["launched"] - incident) / incident,
           balance_rel=abs(out - incident) / incident)
    assert abs(out - incident) < 1e-4 * incident
    # the forward stored every event (17 GB within the default budget), so W came from them and
    # the replay is pass 2 alone: it walks the scoring photons up to their last event
    assert st["events_stored"] == st["events"]
    assert 0 < st["replay_segments"] < st["segments"]
    g = case["out"]["grad"].cpu().numpy()
    assert np.all(np.isfinite(g)) and np.abs(g).max() > 0


def test_transmittance_full_size(m, case):
    sc, grid = case["sc"], case["grid"]
    T = grid.transmittance(case["beta"]).cpu().numpy()
    tau, T_or = oracle.transmittance(sc)
    err = np.abs(T - T_or) / np.maximum(T_or, 1e-30)
    tol = 2e-5 * np.maximum(tau, 1.0) + 2e-6
    worst = np.unravel_index(np.argmax(err / tol), err.shape)
    record("fullsize_transmittance", max_rel_T=err.max(), worst_over_tol=(err / tol).max())
    assert np.all(err <= tol), ((err / tol).max(), worst, tau[worst], T[worst], T_or[worst])


def test_images_full_size_from_oracle_L(m, case):
    sc, grid = case["sc"], case["grid"]
    L = oracle.render(sc, case["p"].replace(n_photons=100_000, n_photons_total=100_000))["L"]
    _, T = oracle.transmittance(sc)
    ref = oracle.images(sc, L, T)
    img = grid.form_images(case["beta"], dev(L, np.float64)).cpu().numpy()
    e = max_rel(img, ref, 1e-3 * np.abs(ref).max())
    record("fullsize_images_from_L", max_rel=e)
    assert e < 1e-4
