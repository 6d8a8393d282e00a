"""Checkpoint / resume of the reconstruction driver state (host only)."""
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
