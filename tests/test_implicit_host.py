"""Host logic of the Newton-Krylov step: restarted GMRES (device-resident
Arnoldi basis, one transfer per iteration) against a dense solve, on CPU
tensors; restarts and early exits on an exactly reached Krylov space."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_08632_gb300.implicit import gmres  # noqa: E402


@pytest.mark.parametrize("n,restart", [(120, 40), (200, 15)])
def test_gmres_matches_dense_solve(n, restart):
    rng = np.random.default_rng(n)
    A = np.eye(n) * 4 + rng.normal(size=(n, n)) * 0.08
    b = rng.normal(size=n)
    At = torch.from_numpy(A)
    x, it, rel = gmres(lambda v: At @ v, torch.from_numpy(b), tol=1e-12, restart=restart, maxiter=400)
    want = np.linalg.solve(A, b)
    assert rel <= 1e-12
    assert np.abs(x.numpy() - want).max() <= 1e-9 * np.abs(want).max()
    assert np.linalg.norm(A @ x.numpy() - b) <= 1.1e-12 * np.linalg.norm(b)


def test_gmres_small_krylov_space_and_zero_rhs():
    # diagonal with 3 distinct eigenvalues: the Krylov space closes after 3 steps
    d = np.repeat([1.0, 2.0, 5.0], 10)
    b = np.random.default_rng(1).normal(size=30)
    x, it, rel = gmres(lambda v: torch.from_numpy(d) * v, torch.from_numpy(b), tol=1e-14)
    assert it <= 4 and np.allclose(x.numpy(), b / d, rtol=1e-12, atol=1e-12)
    x, it, rel = gmres(lambda v: v, torch.zeros(5, dtype=torch.float64))
    assert it == 0 and rel == 0.0 and not x.any()
