"""Shared helpers of the GPU parity tests: device marshalling and oracle-side twins of a scene."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_02110_gb300 as m
    return m


def dev(x, dtype):
    import torch
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return torch.from_numpy(a).to("cuda").contiguous()


def f32_scene(scene):
    """The scene with beta rounded to float32: the GPU reads float32, so the oracle does too."""
    return scene.with_beta(scene.beta.astype(np.float32).astype(np.float64))


def quantised(beta, kind):
    if kind == "f16":
        return beta.astype(np.float32).astype(np.float16).astype(np.float64)
    if kind == "bf16":
        b = beta.astype(np.float32).view(np.uint32).astype(np.uint64)
        r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16   # round to nearest even
        return (r.astype(np.uint32)).view(np.float32).astype(np.float64)
    return beta.astype(np.float32).astype(np.float64)


def record(name, **vals):
    """Appends measured parity errors to the JSON-lines file named by MST_PARITY_REPORT."""
    import json
    import os
    path = os.environ.get("MST_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, **{k: float(v) for k, v in vals.items()}}) + "\n")


def rel_l2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b, floor):
    """max |a - b| / max(|b|, floor)"""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def gpu_hashes(m, grid, beta_dev, params, n):
    import torch
    h = torch.zeros(n, dtype=torch.int32, device="cuda")
    grid.set_debug(h, None)
    grid.render(beta_dev, params, images=False)
    grid.set_debug(None, None)
    return h.cpu().numpy().view(np.uint32)


def last_point_drift(m, grid, sc, p, beta_dev, params=None):
    """Per photon: whether its GPU voxel sequence (path checksum) differs from the oracle's, and the
    distance (m) between the two sides' last event points. FP32 and FP64 carry a photon along
    paths that drift apart (a collision point l = tau / beta amplifies the rounding of the free
    path where beta is small, and later flights carry the offset on), so the parity tests compare
    the photons whose checksum agrees and whose last event point stays close to the oracle's."""
    import torch
    import oracle
    n = p.n_photons
    h = torch.zeros(n, dtype=torch.int32, device="cuda")
    pts = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    grid.set_debug(h, None)
    grid.set_debug_points(pts)
    grid.render(beta_dev, params if params is not None else m.make_params(p), images=True)
    grid.set_debug(None, None)
    grid.set_debug_points(None)
    pg = pts.cpu().numpy()
    vox = pg[:, 3].copy().view(np.uint32).astype(np.int64)
    ijk = np.stack([vox & 2047, (vox >> 11) & 2047, vox >> 22], axis=1)
    xg = ijk * np.array(sc.h) + pg[:, :3].astype(np.float64)
    ro = oracle.render(sc, p, want_L=False, hashes=True, points=True)
    return h.cpu().numpy().view(np.uint32) != ro["hash"], np.linalg.norm(xg - ro["point"], axis=1)


def pixel_edge_moves(gpu, ref, sc, tol, floor_frac):
    """Classic local estimate (Eq. fle): an event within FP32 rounding of a pixel edge lands in one
    pixel on the GPU and in its neighbour in the FP64 oracle, and carries its whole contribution
    with it (scaled by the two pixels' solid angles, which differ by a few per cent). Returns the
    pixels whose error exceeds tol relative to max(|ref|, floor_frac * max |ref|), and those of them
    that no such move explains: a move shows as a neighbouring pixel of the same camera whose error
    cancels at least 90 % of the pixel's own."""
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    err = gpu - ref
    rel = np.abs(err) / np.maximum(np.abs(ref), floor_frac * np.abs(ref).max())
    bad = np.nonzero(rel > tol)[0]
    offs = np.concatenate([[0], np.cumsum(sc.cam_w.astype(np.int64) * sc.cam_h)])
    unexplained = []
    for q in bad:
        c = int(np.searchsorted(offs, q, side="right") - 1)
        w, hgt = int(sc.cam_w[c]), int(sc.cam_h[c])
        x, y = (q - offs[c]) % w, (q - offs[c]) // w
        best = np.inf
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx or dy) and 0 <= x + dx < w and 0 <= y + dy < hgt:
                    best = min(best, abs(err[q] + err[offs[c] + (y + dy) * w + x + dx]))
        if not best <= 0.1 * abs(err[q]):
            unexplained.append(int(q))
    return bad, unexplained
