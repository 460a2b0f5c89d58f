"""The small benchmark configurations run end to end on the CUDA path against
the oracle.

Linear advection, 2D (paper Sec. 5.1 setting): 16 x 16 squares split into 512
triangles, p = 2, FP64, a = (1, 0.5), upwind flux, u0 = sin(2 pi x) sin(2 pi y),
RK4 with dt = 0.1 x the CFL limit (tau_max = 0.198 for triangle SDRT2 with
RK4, tau = |a| dt / h, h = 1/16: dt = 1.107e-3) for 100 steps; the free
stream u = 1.

Differentiation (paper Sec. 4 setting): 6^3 cubes split into 1,296
tetrahedra or 432 prisms, p = 1..4, linear advection along
a = (cos t0 cos t1, sin t0, cos t0 sin t1), t0 = pi/6, t1 = pi/4, and the Euler
equations linearised about a uniform state.  The JVP (FP32 and FP64) is
checked against central differences of the library's FP64 residual
(h = 1e-6) and against the oracle's complex-step JVP; the VJP through the
adjoint identity with the oracle's JVP, <w, J_oracle v> = <J^T w, v>."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import fields  # noqa: E402
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


def _to_dev(M, blocks):
    return torch.from_numpy(M.pack(blocks)).to("cuda")


def _call(M, fn, *blocks):
    dt = torch.float32 if M.dtype_np == np.float32 else torch.float64
    out = torch.zeros(M.state_len, dtype=dt, device="cuda")
    getattr(M, fn)(*[_to_dev(M, b) for b in blocks], out)
    M.sync()
    return M.unpack(out.cpu().numpy())


def test_advection_2d_rk4_100_steps(ctx):
    M, geom, oph, _ = gu.build_pair(ctx, "tri", (16, 16), 2, "advection", "upwind", "fp64", a=(1.0, 0.5))
    assert sum(g.nelem for g in geom.blocks) == 512
    U = gu.oracle_state(geom, fields.sine_product, 1)
    dt = 0.1 * 0.198 * (1 / 16) / np.hypot(1.0, 0.5)
    want = U
    for _ in range(100):
        want = ores.rk4_step(geom, oph, want, dt)
    Ud = _to_dev(M, U)
    M.rk4_step(Ud, dt, 100)
    M.sync()
    got = M.unpack(Ud.cpu().numpy())
    linf, l2 = gu.rel_errors(got, want)
    assert linf < 1e-10, linf


def test_advection_2d_free_stream(ctx):
    M, geom, oph, _ = gu.build_pair(ctx, "tri", (16, 16), 2, "advection", "upwind", "fp64", a=(1.0, 0.5))
    U = [np.ones((g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    R = _call(M, "residual", U)
    # |f| = |a| |u| ~ 1.1, h = 1/16
    assert max(np.abs(r).max() for r in R) < 1e-13 * 1.2 * 16


THETA0, THETA1 = np.pi / 6, np.pi / 4
A_DIFF = (np.cos(THETA0) * np.cos(THETA1), np.sin(THETA0), np.cos(THETA0) * np.sin(THETA1))


def _uniform_gas(X):
    """The uniform state the Euler equations are linearised about.  There
    u_L = u_R at every face, so the non-smooth wave speed of the Rusanov flux
    multiplies a zero jump and the linearisation is unique; near (not at) a
    uniform state the jumps are small and the wave speed's max() sits within
    a finite-difference step of its kink at some face points."""
    rho = np.full(len(X), 1.2)
    vel = np.tile([0.3, -0.2, 0.1], (len(X), 1))
    return fields.primitive_to_conserved(rho, vel, np.full(len(X), 2.0), 1.4)


def _state(geom, system, nvar, seed):
    if system == "euler":
        return gu.oracle_state(geom, _uniform_gas, nvar)
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]


DIFF_CASES = [(k, p, s) for k in ("tet", "pri") for p in (1, 2, 3, 4) for s in ("advection", "euler")]


@pytest.mark.parametrize("kind,p,system", DIFF_CASES)
def test_jvp_against_finite_differences_and_oracle(ctx, kind, p, system):
    riem = "rusanov" if system == "euler" else "upwind"
    n = (6, 6, 6)
    M64, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riem, "fp64", lo=0.0, hi=1.0, a=A_DIFF)
    M32, _, _, _ = gu.build_pair(ctx, kind, n, p, system, riem, "fp32", lo=0.0, hi=1.0, a=A_DIFF)
    U = _state(geom, system, oph.nvar, 41)
    rng = np.random.default_rng(42)
    V = [rng.normal(size=u.shape) for u in U]
    h = 1e-6
    Rp = _call(M64, "residual", [u + h * v for u, v in zip(U, V)])
    Rm = _call(M64, "residual", [u - h * v for u, v in zip(U, V)])
    fd = [(a - b) / (2 * h) for a, b in zip(Rp, Rm)]
    j64 = _call(M64, "jvp", U, V)
    j32 = _call(M32, "jvp", U, V)
    want = ores.jvp(geom, oph, U, V)
    assert gu.rel_errors(j64, fd)[0] < 1e-6
    assert gu.rel_errors(j64, want)[0] < 1e-10
    linf, l2 = gu.rel_errors(j32, want)
    assert linf < 2e-4 and l2 < 2e-5, (linf, l2)


@pytest.mark.parametrize("kind,p,system", [("tet", 2, "euler"), ("tet", 4, "advection"), ("pri", 3, "euler"),
                                           ("pri", 1, "advection")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vjp_adjoint_of_the_oracle_jvp(ctx, kind, p, system, precision):
    riem = "rusanov" if system == "euler" else "upwind"
    M, geom, oph, _ = gu.build_pair(ctx, kind, (6, 6, 6), p, system, riem, precision, a=A_DIFF)
    U = _state(geom, system, oph.nvar, 43)
    rng = np.random.default_rng(44)
    V = [rng.normal(size=u.shape) for u in U]
    W = [rng.normal(size=u.shape) for u in U]
    JV = ores.jvp(geom, oph, U, V)
    JTW = _call(M, "vjp", U, W)
    lhs = sum(float(np.sum(w * j)) for w, j in zip(W, JV))
    rhs = sum(float(np.sum(a.astype(np.float64) * v)) for a, v in zip(JTW, V))
    scale = np.sqrt(sum(float(np.sum(w * w)) for w in W) * sum(float(np.sum(j * j)) for j in JV))
    assert abs(lhs - rhs) <= (1e-11 if precision == "fp64" else 1e-4) * scale, (lhs, rhs, scale)
