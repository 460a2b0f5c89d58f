"""Host-side pins of the Newton-Krylov building block (no GPU): restarted
GMRES against a dense solve, on CPU tensors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2105_08632_gb300 import implicit  # noqa: E402


@pytest.mark.parametrize("n,restart", [(40, 50), (60, 12)])
def test_gmres_matches_a_dense_solve(n, restart):
    rng = np.random.default_rng(8)
    A = np.eye(n) * 4 + rng.normal(0, 0.3, (n, n))            # non-symmetric, well conditioned
    b = rng.normal(0, 1, n)
    At = torch.from_numpy(A)
    x, it, rel = implicit.gmres(lambda v: At @ v, torch.from_numpy(b), tol=1e-12, restart=restart, maxiter=500)
    want = np.linalg.solve(A, b)
    assert rel <= 1e-12 and it <= 500
    assert np.abs(x.numpy() - want).max() < 1e-10 * np.abs(want).max()


def test_gmres_of_the_backward_euler_operator():
    """(I - dt J) x = b with J the upwind difference operator of a periodic
    grid (the linear system of one backward-Euler step)."""
    n, dt = 64, 0.5
    J = -np.eye(n) + np.roll(np.eye(n), -1, axis=1)           # (J u)_i = u_{i-1} - u_i
    M = torch.from_numpy(np.eye(n) - dt * J)
    b = torch.from_numpy(np.sin(2 * np.pi * np.arange(n) / n))
    x, it, rel = implicit.gmres(lambda v: M @ v, b, tol=1e-13, restart=30)
    assert rel <= 1e-13
    assert torch.allclose(M @ x, b, atol=1e-12)


def test_gmres_zero_right_hand_side():
    x, it, rel = implicit.gmres(lambda v: 2 * v, torch.zeros(5, dtype=torch.float64))
    assert it == 0 and rel == 0.0 and float(x.abs().max()) == 0.0
