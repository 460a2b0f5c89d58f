"""Parity of the viscous systems (advection-diffusion, Navier-Stokes) on the
CUDA path with the FP64 oracle: residual, RK4 and JVP, through the C ABI.

The LDG parameters are varied (beta = 0.5, 0, -0.3; eta > 0) so that both
orientations of every face enter the common value and the viscous flux, and
each case first checks that the viscous terms change the residual by a
sizable fraction, so that the comparison exercises them.  Tolerances as in
test_gpu_parity (relative to max |oracle|): FP64 1e-10, FP32 2e-4 (L-inf) and
2e-5 (L2)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import residual as ores  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

TOL64 = 1e-10
TOL32 = (2e-4, 2e-5)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    c = sdrt.Context(0)
    yield c
    c.close()


def _gpu_residual(M, U_blocks):
    dt = torch.float32 if M.dtype_np == np.float32 else torch.float64
    U = torch.from_numpy(M.pack(U_blocks)).to("cuda")
    R = torch.zeros(M.state_len, dtype=dt, device="cuda")
    M.residual(U, R)
    M.sync()
    return M.unpack(R.cpu().numpy())


def _check(got, want, precision):
    linf, l2 = gu.rel_errors(got, want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


def _viscous_share(geom, oph, U):
    """max |R - R_inviscid| / max |R| of the oracle residual."""
    import dataclasses
    inv = dataclasses.replace(oph, system="euler" if oph.system == "ns" else "advection")
    r = np.concatenate([x.ravel() for x in ores.residual(geom, oph, U)])
    r0 = np.concatenate([x.ravel() for x in ores.residual(geom, inv, U)])
    return np.abs(r - r0).max() / np.abs(r).max()


NS_CASES = [("tet", (3, 3, 2), p) for p in (1, 2, 3, 4)] + \
           [("hex", (3, 3, 2), 2), ("pri", (3, 2, 3), 3), ("tri", (7, 5), 3), ("quad", (6, 5), 2)]


@pytest.mark.parametrize("kind,n,p", NS_CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ns_residual(ctx, kind, n, p, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "ns", "rusanov", precision, mu=0.02, beta=0.5, eta=0.1)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, oph.nvar), 21, 0.02)
    assert _viscous_share(geom, oph, U) > 1e-2
    _check(_gpu_residual(M, U), ores.residual(geom, oph, U), precision)


@pytest.mark.parametrize("beta,eta", [(0.0, 0.0), (-0.3, 0.2), (0.5, 0.0)])
@pytest.mark.parametrize("riemann", ["rusanov", "roe"])
def test_ns_ldg_parameters(ctx, beta, eta, riemann):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 2, 3), 3, "ns", riemann, "fp64", mu=0.05, prandtl=0.7,
                                    beta=beta, eta=eta)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, oph.nvar), 22, 0.02)
    _check(_gpu_residual(M, U), ores.residual(geom, oph, U), "fp64")


@pytest.mark.parametrize("kind,n,p", [("tri", (9, 7), 3), ("quad", (6, 7), 2), ("tet", (3, 3, 3), 3),
                                      ("hex", (3, 3, 2), 3), ("pri", (3, 3, 2), 2)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_advdiff_residual(ctx, kind, n, p, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "advdiff", "upwind", precision, a=(1.0, 0.5, 0.25), mu=0.05,
                                    beta=-0.2, eta=0.3)
    rng = np.random.default_rng(23)
    U = [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    assert _viscous_share(geom, oph, U) > 1e-2
    _check(_gpu_residual(M, U), ores.residual(geom, oph, U), precision)


def test_ns_mixed_mesh(ctx):
    from inputs import meshes
    from oracle import mesh as omesh
    from oracle import physics as ophx
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh(["tet", "tet", "pri"], (3, 2, 3), [0, 0, 0], [1, 1, 1])
    degs = {"tet": 2, "pri": 2}
    M = sdrt.Mesh(ctx, mesh, degs, sdrt.make_physics("ns", 3, "rusanov", "fp64", mu=0.03, beta=0.25, eta=0.1))
    geom = omesh.build(mesh, degs)
    oph = ophx.Physics("ns", 3, "rusanov", mu=0.03, beta=0.25, eta=0.1)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 24, 0.02)
    _check(_gpu_residual(M, U), ores.residual(geom, oph, U), "fp64")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ns_rk4_steps(ctx, precision):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 3, "ns", "rusanov", precision, mu=0.02)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 25, 0.01)
    dt = 1e-3
    want = U
    for _ in range(3):
        want = ores.rk4_step(geom, oph, want, dt)
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    M.rk4_step(Ud, dt, 3)
    M.sync()
    got = M.unpack(Ud.cpu().numpy())
    d_got = [g - u for g, u in zip(got, U)]
    d_want = [w - u for w, u in zip(want, U)]
    linf, _ = gu.rel_errors(d_got, d_want)
    assert linf < (1e-9 if precision == "fp64" else 5e-3), linf


@pytest.mark.parametrize("kind,p,system", [("tet", 3, "ns"), ("hex", 2, "ns"), ("tri", 3, "ns"),
                                           ("tet", 2, "advdiff")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_viscous_jvp(ctx, kind, p, system, precision):
    riem = "rusanov" if system == "ns" else "upwind"
    n = (5, 4) if kind == "tri" else (3, 3, 2)
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riem, precision, mu=0.03, beta=0.3, eta=0.1)
    rng = np.random.default_rng(26)
    if system == "ns":
        U = gu.oracle_state(geom, gu.smooth_gas, oph.nvar)
    else:
        U = [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    V = [rng.normal(size=u.shape) for u in U]
    want = ores.jvp(geom, oph, U, V)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    Vd = torch.from_numpy(M.pack(V)).to("cuda")
    JV = torch.zeros(M.state_len, dtype=dt, device="cuda")
    M.jvp(Ud, Vd, JV)
    M.sync()
    _check(M.unpack(JV.cpu().numpy()), want, precision)


def test_viscous_noalloc_rejected(ctx):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 2, "ns", "rusanov", "fp64", mu=0.01)
    U = torch.zeros(M.state_len, dtype=torch.float64, device="cuda")
    R = torch.zeros_like(U)
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_residual_noalloc(ctx.ptr, M.id, U, R)
    assert ei.value.code == -2
