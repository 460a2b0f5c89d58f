"""Implicit backward-Euler step by Newton-Krylov (GMRES on the library's JVP)
on the GPU.

- Linear advection: the step equals the oracle's dense solve
  (I - dt J) X = U with J the oracle-assembled RHS Jacobian.
- Euler (nonlinear): the converged X satisfies the implicit equation
  X - U - dt R(X) = 0 with R evaluated by the oracle, to the solver
  tolerance; Newton converges quadratically (the residual history falls
  super-linearly)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import residual as ores  # noqa: E402
from tests import gpu_util as gu  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    c = sdrt.Context(0)
    yield c
    c.close()


def test_backward_euler_linear_advection_matches_dense_solve(ctx):
    from paper_2105_08632_gb300 import implicit
    M, geom, oph, _ = gu.build_pair(ctx, "tri", (4, 4), 2, "advection", "upwind", "fp64", a=(1.0, 0.5))
    rng = np.random.default_rng(61)
    U = [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    dt = 0.05
    Ud = torch.from_numpy(M.pack(U)).cuda()
    X, info = implicit.backward_euler_step(M, Ud, dt)
    got = M.unpack(X.cpu().numpy())
    J = ores.jacobian(geom, oph, U)
    x = np.linalg.solve(np.eye(J.shape[0]) - dt * J, ores.flatten(U))
    want = ores.unflatten(geom, x, 1)
    linf, _ = gu.rel_errors(got, want)
    assert linf < 1e-8, linf
    # linear: the first Newton step solves to the GMRES tolerance, a second one
    # at most to reach the Newton tolerance
    assert len(info["gmres_iterations"]) <= 2


def test_backward_euler_euler_equations_solve_the_implicit_equation(ctx):
    from paper_2105_08632_gb300 import implicit
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 2, "euler", "rusanov", "fp64")
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 62, 0.02)
    dt = 2e-3
    Ud = torch.from_numpy(M.pack(U)).cuda()
    X, info = implicit.backward_euler_step(M, Ud, dt, newton_tol=1e-11)
    Xb = M.unpack(X.cpu().numpy())
    R = ores.residual(geom, oph, Xb)
    F = [x - u - dt * r for x, u, r in zip(Xb, U, R)]
    fn = np.sqrt(sum(float(np.sum(f * f)) for f in F)) / np.sqrt(sum(float(np.sum(u * u)) for u in U))
    assert fn < 1e-10, fn
    h = info["residual_history"]
    assert len(h) <= 6 and h[-1] <= 1e-11, h
    if len(h) >= 3 and h[2] > 1e-13:
        assert h[2] < 10 * h[1] ** 1.5, h              # super-linear (Newton) convergence
