"""Host logic of the reconstruction drivers: checkpoint / resume of their state, and the projected
L-BFGS and surrogate GD loops on a CPU stand-in for the grid (a quadratic loss)."""
import numpy as np


def test_recon_state_roundtrip(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_02110_gb300.autograd import ReconState, _two_loop
    rng = np.random.default_rng(0)
    st = ReconState(beta=rng.random(50), it=7, s_hist=[rng.random(50) for _ in range(3)],
                    y_hist=[rng.random(50) for _ in range(3)], losses=[3.0, 2.0, 1.5], n_renders=11)
    path = str(tmp_path / "state.npz")
    st.save(path)
    r = ReconState.load(path)
    assert r.it == 7 and r.n_renders == 11 and r.losses == [3.0, 2.0, 1.5]
    assert np.array_equal(r.beta, st.beta)
    assert all(np.array_equal(a, b) for a, b in zip(r.s_hist, st.s_hist))
    # the two-loop recursion reproduces the inverse of a quadratic's Hessian on its secant pairs
    A = np.diag(np.linspace(1.0, 5.0, 6))
    S = [np.eye(6)[i] for i in range(6)]
    Y = [A @ s for s in S]
    g = rng.random(6)
    assert np.allclose(_two_loop(g, S, Y), np.linalg.solve(A, g), rtol=1e-10)


class _QuadGrid:
    """Stand-in for a Grid on the CPU: E(beta) = |A beta - y|^2, the shape of the paper's loss
    with a linear image model, so the drivers' host logic runs without a GPU."""

    device = "cpu"

    def __init__(self, A, y):
        import torch
        self.A, self.y, self.torch = torch.from_numpy(A), torch.from_numpy(y), torch

    def _f(self, beta):
        r = self.A @ beta.double() - self.y
        return (r @ r).reshape(1), 2.0 * (self.A.T @ r)

    def render_grad(self, beta, params, meas, mask=None, images=False):
        loss, grad = self._f(beta)
        return {"loss": loss, "grad": grad}

    def render(self, beta, params, images=False, L=False):
        return {"L": beta.double().clone()}

    def surrogate_grad(self, beta, L_ref, beta_ref, params, meas, mask=None):
        loss, grad = self._f(beta)
        return {"loss": loss, "grad": grad}


def _nnls_case(seed=3, m=40, n=25):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, n))
    x_true = np.maximum(rng.normal(size=n), 0.0)
    y = A @ x_true + 0.3 * rng.normal(size=m)  # noisy: some bounds are active at the optimum
    return A, y


def test_projected_lbfgs_reaches_the_nonnegative_least_squares_optimum():
    scipy_opt = __import__("pytest").importorskip("scipy.optimize")
    from paper_1512_02110_gb300.autograd import reconstruct
    A, y = _nnls_case()
    x_ref, _ = scipy_opt.nnls(A, y)
    st = reconstruct(_QuadGrid(A, y), None, np.full(A.shape[1], 0.5), None, iters=300, method="lbfgs")
    f_ref = float(np.sum((A @ x_ref - y) ** 2))
    assert st.losses[-1] <= f_ref * (1 + 1e-6)
    assert np.all(st.beta >= 0.0)
    assert np.allclose(st.beta, x_ref, atol=1e-4)


def test_surrogate_gd_loop_descends_with_a_safe_step():
    from paper_1512_02110_gb300.autograd import reconstruct
    A, y = _nnls_case(seed=5)
    step = 0.5 / np.linalg.norm(A, 2) ** 2  # below 1 / Lipschitz constant of the gradient
    st = reconstruct(_QuadGrid(A, y), None, np.full(A.shape[1], 0.5), None, iters=20, method="gd", step=step, n_gd=5)
    assert st.it == 20 and st.n_renders == 20 and len(st.losses) == 100
    assert all(b <= a + 1e-12 for a, b in zip(st.losses, st.losses[1:]))
    assert np.all(st.beta >= 0.0)


def test_blocks_parametrisation():
    """beta = B theta over ragged 3-D blocks: B^T is the adjoint of B, block means invert the
    expansion, and every voxel lands in the block its coordinates give."""
    from paper_1512_02110_gb300.autograd import Blocks
    shape, block = (5, 4, 3), (2, 3, 2)
    P = Blocks(shape, block)
    assert P.n == 3 * 2 * 2 and P.count.sum() == 60
    for k in range(60):
        ix, iy, iz = k % 5, (k // 5) % 4, k // 20
        assert P.bid[k] == ix // 2 + 3 * (iy // 3 + 2 * (iz // 2))
    rng = np.random.default_rng(2)
    th, g = rng.random(P.n), rng.random(60)
    assert abs(np.dot(P.expand(th), g) - np.dot(th, P.reduce(g))) < 1e-12
    assert np.allclose(P.restrict(P.expand(th)), th)


def test_block_reconstruction_reaches_the_block_optimum(tmp_path):
    scipy_opt = __import__("pytest").importorskip("scipy.optimize")
    from paper_1512_02110_gb300.autograd import Blocks, ReconState, reconstruct
    A, y = _nnls_case(m=40, n=24)
    grid = _QuadGrid(A, y)
    grid.shape = (4, 3, 2)
    P = Blocks(grid.shape, (2, 2, 1))
    B = np.stack([P.expand(np.eye(P.n)[b]) for b in range(P.n)], axis=1)  # [nvox, nblocks]
    th_ref, _ = scipy_opt.nnls(A @ B, y)
    st = reconstruct(grid, None, np.full(24, 0.5), None, iters=200, method="lbfgs", block=(2, 2, 1))
    assert np.allclose(st.x, th_ref, atol=1e-4) and np.allclose(st.beta, B @ st.x)
    path = str(tmp_path / "s.npz")
    st.save(path)
    r = ReconState.load(path)
    assert np.array_equal(r.x, st.x) and np.array_equal(r.beta, st.beta)
    g = reconstruct(grid, None, np.full(24, 0.5), None, iters=10, method="gd", step=0.5 / np.linalg.norm(A @ B, 2) ** 2,
                    n_gd=5, block=(2, 2, 1))
    assert all(b2 <= b1 + 1e-12 for b1, b2 in zip(g.losses, g.losses[1:])) and np.allclose(g.beta, B @ g.x)


def test_haze_scene_is_the_coarse_field_on_blocks():
    """The paper-shaped haze scene: its aerosol field is the coarse 20 x 20 x 40 field held
    constant over 4 x 4 x 3 voxel blocks (synth.refine agrees with Blocks.expand), the 36
    cameras sit inside the domain and within the library's camera limit, and the optical depths
    are those of haze (aerosol column 0.05-0.5, air 0.07)."""
    import re

    import synth
    from paper_1512_02110_gb300.autograd import Blocks
    sc, p, coarse, block = synth.cfg_haze80(1000)
    P = Blocks(sc.shape, block)
    assert P.n == int(np.prod(coarse))
    assert np.allclose(P.expand(P.restrict(sc.beta)), sc.beta, rtol=1e-14, atol=0)
    th = np.random.default_rng(1).random(P.n)
    assert np.array_equal(synth.refine(th, coarse, block), P.expand(th))
    hdr = open(__import__("os").path.join(__import__("os").path.dirname(__file__), "..", "include", "mst.h")).read()
    assert sc.n_cams == 36 <= int(re.search(r"#define MST_MAX_CAMERAS (\d+)", hdr).group(1))
    ext = sc.extent()
    assert np.all(sc.cam_pos > 0) and np.all(sc.cam_pos < ext)
    dz = sc.h[2]
    col = sc.beta.reshape(sc.shape[::-1]).sum(0) * dz
    assert 0.04 < col.min() and col.max() < 0.5
    assert abs(sc.beta_air.reshape(sc.shape[::-1]).sum(0).mean() * dz - 0.066) < 0.002
