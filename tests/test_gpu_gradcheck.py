"""The GPU gradients against central finite differences of the GPU's own loss: the full gradient
with common random numbers (the same Philox streams at beta +- h; a t-test over seeds, since a
perturbation moves some collisions across voxel faces), and the surrogate gradient, whose loss
(j held fixed) is deterministic."""
import math

import numpy as np
import pytest

import synth
from tests.gpu_util import dev, f32_scene, need_gpu, record

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return need_gpu()


def _case():
    sc, p = synth.cfg_blobs16(4_000_000)
    sc = f32_scene(sc)
    beta = synth.smoothed(sc.beta, sc.shape, 0.4).astype(np.float32).astype(np.float64)
    return sc, p.replace(rr_threshold=0.0), beta


def test_full_gradient_matches_fd_crn(m):
    sc, p, beta = _case()
    grid = m.Grid.from_scene(sc)
    meas = grid.render(dev(sc.beta, np.float32), m.make_params(p, seed=4))["images"]
    voxels = np.argsort(-beta)[[0, 5, 20, 60, 150]]
    nseed = 8
    diffs = np.zeros((nseed, len(voxels)))
    gs = np.zeros((nseed, len(voxels)))
    for s in range(nseed):
        prm = m.make_params(p, seed=100 + s, grad_mode="full")
        g = grid.render_grad(dev(beta, np.float32), prm, meas, images=False)["grad"].cpu().numpy()
        for i, k in enumerate(voxels):
            hstep = 0.02 * beta[k]
            bp, bm = beta.copy(), beta.copy()
            bp[k] += hstep
            bm[k] -= hstep
            # the FP32 grid holds beta +- h exactly enough: the difference is taken on the values staged
            hp = float(np.float32(bp[k])) - float(np.float32(beta[k]))
            hm = float(np.float32(beta[k])) - float(np.float32(bm[k]))
            Ep = grid.render_grad(dev(bp, np.float32), prm, meas, images=False)["loss"].item()
            Em = grid.render_grad(dev(bm, np.float32), prm, meas, images=False)["loss"].item()
            diffs[s, i] = g[k] - (Ep - Em) / (hp + hm)
            gs[s, i] = g[k]
    t = diffs.mean(0) / (diffs.std(0, ddof=1) / math.sqrt(nseed))
    tg = gs.mean(0) / (gs.std(0, ddof=1) / math.sqrt(nseed))
    record("gpu_full_gradient_fd_crn", max_abs_t=float(np.abs(t).max()), median_abs_t_grad=float(np.median(np.abs(tg))))
    assert np.all(np.abs(t) < 5.0), t
    assert np.median(np.abs(tg)) > 5.0, tg  # the gradient is resolved, many standard errors from zero


def test_surrogate_gradient_matches_central_differences(m):
    """Without conditioning (Q_c reweights the gradient away from the loss's derivative)."""
    sc, p, beta = _case()
    grid = m.Grid.from_scene(sc)
    ref = grid.render(dev(sc.beta, np.float32), m.make_params(p.replace(n_photons=200_000)), L=True)
    L_ref, meas = ref["L"], ref["images"] * 0.8
    beta_ref = dev(beta, np.float32)
    prm = m.make_params(p, conditioning="none")

    def surrogate(b):
        return grid.surrogate_grad(dev(b, np.float32), L_ref, beta_ref, prm, meas)

    g = surrogate(beta)["grad"].cpu().numpy()
    worst = 0.0
    for k in np.argsort(-beta)[[0, 7, 30, 90]]:
        hstep = 0.01 * beta[k]
        bp, bm = beta.copy(), beta.copy()
        bp[k] += hstep
        bm[k] -= hstep
        hp = float(np.float32(bp[k])) - float(np.float32(beta[k]))
        hm = float(np.float32(beta[k])) - float(np.float32(bm[k]))
        fd = (surrogate(bp)["loss"].item() - surrogate(bm)["loss"].item()) / (hp + hm)
        worst = max(worst, abs(g[k] - fd) / abs(fd))
    record("gpu_surrogate_fd", max_rel=worst)
    assert worst < 2e-3, worst
    assert np.all(np.isfinite(g)) and np.abs(g).max() > 0
