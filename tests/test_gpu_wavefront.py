"""Wavefront shape of the persistent transport kernels (voxels per loop trip, blocks per SM) and
its autotuner: the shape moves work between lanes but not a photon's path (fixed by its Philox
key), so the images, loss and gradient only change by the order of FP32 additions, and the
event and segment counts not at all."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, f32_scene, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return need_gpu()


def _case(m):
    sc, p = synth.cfg_blobs16(200_000)
    sc = f32_scene(sc)
    grid = m.Grid.from_scene(sc)
    beta = dev(sc.beta, np.float32)
    meas = grid.render(beta, m.make_params(p, seed=p.seed + 1))["images"]
    return sc, p, grid, beta, meas


@pytest.mark.parametrize("shape", [(8, 2, 4, 2), (16, 1, 10, 3), (10, 3, 8, 1)])
def test_wavefront_shape_changes_no_result(m, shape):
    sc, p, grid, beta, meas = _case(m)
    prm = m.make_params(p, grad_mode="full")
    a = grid.render_grad(beta, prm, meas)
    sa = grid.stats()
    grid.set_wavefront(*shape)
    b = grid.render_grad(beta, prm, meas)
    sb = grid.stats()
    for k in ["events", "segments", "replay_segments", "events_stored"]:
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    ei = rel_l2(b["images"].cpu().numpy(), a["images"].cpu().numpy())
    eg = rel_l2(b["grad"].cpu().numpy(), a["grad"].cpu().numpy())
    el = abs(b["loss"].item() - a["loss"].item()) / a["loss"].item()
    record(f"wavefront{shape}", images_rel_l2=ei, grad_rel_l2=eg, loss_rel=el)
    assert ei < 1e-6 and el < 1e-6 and eg < 1e-5, (ei, el, eg)
    for bad in [(7, 0, 0, 0), (0, 0, 3, 0), (0, 9, 0, 0)]:  # trips outside the instantiated sets
        with pytest.raises(m.MSTError):
            grid.set_wavefront(*bad)


def test_autotune_picks_a_candidate_and_keeps_results(m):
    sc, p, grid, beta, meas = _case(m)
    prm = m.make_params(p, grad_mode="full")
    a = grid.render_grad(beta, prm, meas)
    c = grid.autotune(beta, prm, n_sample=1 << 18)
    assert c["forward_trip"] in (8, 10, 12, 16) and c["replay_trip"] in (4, 6, 8, 10)
    assert 1 <= c["forward_blocks_per_sm"] <= 8 and 1 <= c["replay_blocks_per_sm"] <= 8
    b = grid.render_grad(beta, prm, meas)
    eg = rel_l2(b["grad"].cpu().numpy(), a["grad"].cpu().numpy())
    record("autotune", grad_rel_l2=eg, **{k: float(v) for k, v in c.items()})
    assert eg < 1e-5, eg
