"""Autograd wrapper and reconstruction drivers on the GPU (the host-side optimizers call only
the C ABI). Measured images come from the oracle; beta starts at a uniform 1 1/km."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import dev, f32_scene, need_gpu, record

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return need_gpu()


@pytest.fixture(scope="module")
def case():
    sc, p = synth.cfg_blobs16(200_000)
    sc = f32_scene(sc)
    meas = oracle.forward_images(sc, p.replace(seed=4))[0]
    return sc, p, meas


def test_autograd_matches_render_grad(m, case):
    import torch
    sc, p, meas = case
    grid = m.Grid.from_scene(sc)
    beta = dev(synth.smoothed(sc.beta, sc.shape, 0.4), np.float32).requires_grad_(True)
    params = m.make_params(p, grad_mode="full", reg_eta=0.01)
    meas_d = dev(meas, np.float64)
    loss = m.RenderLoss.apply(beta, grid, params, meas_d)
    loss.backward()
    ref = grid.render_grad(beta.detach(), params, meas_d)
    assert beta.grad.dtype == torch.float32
    g, gr = beta.grad.double(), ref["grad"]
    err = float((g - gr).norm() / gr.norm())
    assert err < 1e-5, err
    assert abs(loss.item() - ref["loss"].item()) <= 1e-6 * ref["loss"].item()  # FP32 atomic order differs per call


def test_projected_lbfgs_reduces_loss_and_error(m, case):
    sc, p, meas = case
    grid = m.Grid.from_scene(sc)
    params = m.make_params(p, grad_mode="full")
    beta0 = np.full(sc.nvox, 1e-3)
    st = m.reconstruct(grid, dev(meas, np.float64), beta0, params, iters=8, method="lbfgs")
    truth = sc.beta
    eps0 = np.abs(beta0 - truth).sum() / truth.sum()
    eps = np.abs(st.beta - truth).sum() / truth.sum()
    record("lbfgs", loss0=st.losses[0], loss=st.losses[-1], eps0=eps0, eps=eps, renders=st.n_renders)
    assert st.it == 8 and np.all(np.diff(st.losses) <= 0)
    assert st.losses[-1] < 0.3 * st.losses[0]
    assert eps < eps0 and np.all(st.beta >= 0)


def test_paper_surrogate_gd_loop(m, case):
    import torch
    sc, p, meas = case
    grid = m.Grid.from_scene(sc)
    params = m.make_params(p, grad_mode="surrogate", conditioning="inv_count")
    meas_d = dev(meas, np.float64)
    beta0 = np.full(sc.nvox, 1e-3)
    g0 = grid.render_grad(dev(beta0, np.float32), params, meas_d)["grad"].abs().max().item()
    step = 0.05 * 1e-3 / g0
    st = m.reconstruct(grid, meas_d, beta0, params, iters=4, method="gd", step=step, n_gd=5)
    record("gd_ngd5", loss0=st.losses[0], loss=st.losses[-1], renders=st.n_renders)
    assert len(st.losses) == 20 and st.n_renders == 4
    assert st.losses[-1] < st.losses[0]
    torch.cuda.synchronize()
