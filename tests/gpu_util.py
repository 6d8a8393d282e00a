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
