"""Autograd wrapper and reconstruction drivers (Sec. 5: Eq. minobjective, Eq. GD).

`RenderLoss` exposes mst_render_grad as a torch.autograd.Function of beta. `reconstruct`
runs either projected L-BFGS on beta >= 0 (FP64 two-loop recursion and Armijo line search on
the host), or the paper's surrogate loop: N_GD gradient-descent steps with j held fixed
(mst_surrogate_grad), then a new forward render refreshes j (Eq. GD). All renders and
gradients run in the CUDA library; the host only holds the optimizer's vectors.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np
import torch


class RenderLoss(torch.autograd.Function):
    """E(beta) = sum M (i(beta) - i_meas)^2 + eta Psi(beta) with dE/dbeta from the library."""

    @staticmethod
    def forward(ctx, beta, grid, params, meas, mask=None):
        out = grid.render_grad(beta.detach().contiguous(), params, meas, mask, images=False)
        ctx.save_for_backward(out["grad"])
        ctx.beta_dtype = beta.dtype
        return out["loss"][0]

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return (gout * grad).to(ctx.beta_dtype), None, None, None, None


@dataclasses.dataclass
class ReconState:
    beta: np.ndarray
    it: int = 0
    s_hist: List[np.ndarray] = dataclasses.field(default_factory=list)
    y_hist: List[np.ndarray] = dataclasses.field(default_factory=list)
    losses: List[float] = dataclasses.field(default_factory=list)
    n_renders: int = 0
    x: Optional[np.ndarray] = None  # block values when the field is block-parametrised

    def save(self, path: str):
        n = self.beta.size if self.x is None else self.x.size
        np.savez(path, beta=self.beta, it=self.it, losses=np.array(self.losses), n_renders=self.n_renders,
                 s=np.array(self.s_hist) if self.s_hist else np.zeros((0, n)),
                 y=np.array(self.y_hist) if self.y_hist else np.zeros((0, n)),
                 x=self.x if self.x is not None else np.zeros(0))

    @classmethod
    def load(cls, path: str) -> "ReconState":
        z = np.load(path)
        x = z["x"] if "x" in z.files and z["x"].size else None
        return cls(beta=z["beta"], it=int(z["it"]), s_hist=list(z["s"]), y_hist=list(z["y"]),
                   losses=z["losses"].tolist(), n_renders=int(z["n_renders"]), x=x)


class Blocks:
    """beta = B theta: beta piecewise constant over 3-D blocks of bx x by x bz voxels (Sec. 5,
    the paper's dimensionality reduction; blocks at the far faces may be smaller). expand
    gives beta from the block values, reduce applies B^T (sums a voxel field over each
    block: the gradient with respect to theta), restrict gives the block means."""

    def __init__(self, shape, block):
        nx, ny, nz = (int(v) for v in shape)
        bx, by, bz = (int(v) for v in block)
        if min(bx, by, bz) < 1:
            raise ValueError("block sizes must be >= 1")
        nbx, nby, nbz = -(-nx // bx), -(-ny // by), -(-nz // bz)
        ix = np.arange(nx) // bx
        iy = np.arange(ny) // by
        iz = np.arange(nz) // bz
        self.bid = (ix[None, None, :] + nbx * (iy[None, :, None] + nby * iz[:, None, None])).ravel()
        self.n = nbx * nby * nbz
        self.count = np.bincount(self.bid, minlength=self.n).astype(np.float64)

    def expand(self, theta):
        return np.asarray(theta, dtype=np.float64)[self.bid]

    def reduce(self, g):
        return np.bincount(self.bid, weights=np.asarray(g, dtype=np.float64), minlength=self.n)

    def restrict(self, beta):
        return self.reduce(beta) / self.count


class Scaled:
    """beta = w x with fixed positive weights w (a diagonal preconditioner): the optimizer works
    on x, its gradient is w * dE/dbeta. With w the start field, every voxel moves in proportion to
    its own extinction and voxels outside the start's support stay at 0."""

    def __init__(self, w):
        self.w = np.asarray(w, dtype=np.float64)
        if not np.all(self.w > 0):
            raise ValueError("scaling weights must be > 0")
        self.n = self.w.size

    def expand(self, x):
        return self.w * np.asarray(x, dtype=np.float64)

    def reduce(self, g):
        return self.w * np.asarray(g, dtype=np.float64)

    def restrict(self, beta):
        return np.asarray(beta, dtype=np.float64) / self.w


def _eval(grid, params, meas, mask, x, P=None):
    """Loss and gradient at parameter vector x (beta itself, or block values under P)."""
    beta_np = x if P is None else P.expand(x)
    beta = torch.from_numpy(beta_np.astype(np.float32)).to(grid.device)
    out = grid.render_grad(beta, params, meas, mask, images=False)
    g = out["grad"].cpu().numpy()
    return float(out["loss"].item()), (g if P is None else P.reduce(g))


def reconstruct(grid, meas, beta0, params, iters: int = 50, method: str = "lbfgs", mask=None, history: int = 10,
                step: float = 1e-3, n_gd: int = 5, state: Optional[ReconState] = None,
                callback: Optional[Callable[[ReconState], None]] = None, block=None) -> ReconState:
    """Recovers beta >= 0 from measured images.

    method="lbfgs": projected L-BFGS. The photon seed is held fixed across iterations (common
    random numbers), so the objective is one deterministic function of beta.
    method="gd": the paper's loop (Eq. GD): a forward render gives L and j = L/beta; then n_gd
    projected steps beta <- max(0, beta - step * dE/dbeta) with j fixed; repeat.
    block=(bx, by, bz): optimise one value per block of voxels (Blocks); the state's x holds the
    block values and its beta the expanded field. block may also be a parametrisation object
    with expand / reduce / restrict (Blocks, Scaled).
    """
    if block is None or hasattr(block, "expand"):
        P = block
    else:
        P = Blocks(grid.shape, block)
    b0 = np.maximum(np.asarray(beta0, dtype=np.float64), 0.0)
    if state is None:
        x0 = b0 if P is None else P.restrict(b0)
        st = ReconState(beta=x0 if P is None else P.expand(x0), x=None if P is None else x0)
    else:
        st = state
    if method == "gd":
        return _run_gd(grid, meas, params, mask, iters, step, n_gd, st, callback, P)
    cur = lambda: st.beta if P is None else st.x  # noqa: E731
    f, g = _eval(grid, params, meas, mask, cur(), P)
    st.n_renders += 1
    if not st.losses:
        st.losses.append(f)
    while st.it < iters:
        x = cur()
        free = (x > 0) | (g < 0)
        gf = np.where(free, g, 0.0)
        d = -_two_loop(gf, st.s_hist, st.y_hist)
        d = np.where(free, d, 0.0)
        if not np.dot(d, gf) < 0:
            d = -gf
            st.s_hist.clear()
            st.y_hist.clear()
        if len(st.s_hist) == 0:
            d *= min(1.0, 0.1 * max(np.abs(x).max(), 1e-12) / max(np.abs(d).max(), 1e-300))
        alpha, ok = 1.0, False
        for _ in range(20):
            xn = np.maximum(x + alpha * d, 0.0)
            fn, gn = _eval(grid, params, meas, mask, xn, P)
            st.n_renders += 1
            if fn <= f + 1e-4 * np.dot(gf, xn - x):
                ok = True
                break
            alpha *= 0.5
        if not ok:
            if not st.s_hist:
                break  # no descent along the projected gradient either
            st.s_hist.clear()  # stale curvature pairs: retry from the projected gradient
            st.y_hist.clear()
            continue
        s, y = xn - x, gn - g
        if np.dot(s, y) > 1e-12 * np.dot(y, y):
            st.s_hist.append(s)
            st.y_hist.append(y)
            if len(st.s_hist) > history:
                st.s_hist.pop(0)
                st.y_hist.pop(0)
        if P is None:
            st.beta = xn
        else:
            st.x, st.beta = xn, P.expand(xn)
        f, g = fn, gn
        st.it += 1
        st.losses.append(f)
        if callback:
            callback(st)
    return st


def _two_loop(g, S, Y):
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / np.dot(y, s)
        a = rho * np.dot(s, q)
        alphas.append((a, rho))
        q -= a * y
    if S:
        q *= np.dot(S[-1], Y[-1]) / np.dot(Y[-1], Y[-1])
    for (s, y), (a, rho) in zip(zip(S, Y), reversed(alphas)):
        b = rho * np.dot(y, q)
        q += (a - b) * s
    return q


def _run_gd(grid, meas, params, mask, iters, step, n_gd, st, callback, P=None):
    while st.it < iters:
        beta_ref = torch.from_numpy(st.beta.astype(np.float32)).to(grid.device)
        L_ref = grid.render(beta_ref, params, images=False, L=True)["L"]
        st.n_renders += 1
        for _ in range(n_gd):
            beta = torch.from_numpy(st.beta.astype(np.float32)).to(grid.device)
            out = grid.surrogate_grad(beta, L_ref, beta_ref, params, meas, mask)
            st.losses.append(float(out["loss"].item()))
            g = out["grad"].cpu().numpy()
            if P is None:
                st.beta = np.maximum(st.beta - step * g, 0.0)
            else:
                st.x = np.maximum(st.x - step * P.reduce(g), 0.0)
                st.beta = P.expand(st.x)
        st.it += 1
        if callback:
            callback(st)
    return st
