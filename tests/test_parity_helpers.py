"""CPU checks of the parity tests' own helpers (no GPU): the pixel-edge move signature used by
the classic-estimator image checks (Eq. fle's pixel of an event on a pixel edge is not unique
between FP32 and FP64)."""
import types

import numpy as np

from tests.gpu_util import pixel_edge_moves


def _scene(ws, hs):
    return types.SimpleNamespace(cam_w=np.array(ws, np.int32), cam_h=np.array(hs, np.int32))


def test_a_move_between_neighbours_is_explained():
    sc = _scene([4, 3], [3, 2])
    ref = np.ones(18)
    gpu = ref.copy()
    gpu[5] += 0.5     # camera 0, pixel (1, 1)
    gpu[6] -= 0.48    # camera 0, pixel (2, 1): the same contribution, 4 % apart (solid angles)
    bad, unexplained = pixel_edge_moves(gpu, ref, sc, 2e-4, 1e-2)
    assert list(bad) == [5, 6] and unexplained == []


def test_a_lone_error_is_not_explained():
    sc = _scene([4, 3], [3, 2])
    ref = np.ones(18)
    gpu = ref.copy()
    gpu[13] += 0.3    # camera 1, nothing to cancel it
    gpu[5] += 0.5
    gpu[6] -= 0.3     # a neighbour that cancels only 60 %
    bad, unexplained = pixel_edge_moves(gpu, ref, sc, 2e-4, 1e-2)
    assert sorted(unexplained) == [5, 6, 13]


def test_no_move_across_a_row_end_or_between_cameras():
    sc = _scene([4, 3], [3, 2])
    ref = np.ones(18)
    gpu = ref.copy()
    gpu[3] += 0.5     # camera 0, pixel (3, 0)
    gpu[4] -= 0.5     # camera 0, pixel (0, 1): adjacent in memory, not in the image
    gpu[11] += 0.5    # camera 0, last pixel
    gpu[12] -= 0.5    # camera 1, first pixel
    _, unexplained = pixel_edge_moves(gpu, ref, sc, 2e-4, 1e-2)
    assert sorted(unexplained) == [3, 4, 11, 12]


def test_faint_pixels_below_the_floor_are_held_to_the_floor():
    sc = _scene([4], [1])
    ref = np.array([1.0, 1e-6, 1.0, 1.0])
    gpu = ref.copy()
    gpu[1] += 1e-7    # 10 % of a faint pixel, 1e-5 of the floor (1e-2 of the brightest)
    bad, _ = pixel_edge_moves(gpu, ref, sc, 2e-4, 1e-2)
    assert list(bad) == []
