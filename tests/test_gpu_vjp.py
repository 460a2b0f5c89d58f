"""Vector-Jacobian product of the residual on the CUDA path (inviscid and
viscous: LDG advection-diffusion and Navier-Stokes).

1. Against the oracle's W^T J built from its dense Jacobian (complex-step
   columns) on small periodic meshes.
2. The adjoint identity <W, J V> = <J^T W, V> with the library's own JVP at
   sizes past the oracle's dense reach: several tiles with a ragged tail, the
   register-blocked tetrahedron path and a mixed mesh.
Tolerances relative to max |oracle| as in test_gpu_parity (FP64 1e-10, FP32
2e-4 / 2e-5); the identity to 1e-11 (FP64) / 1e-4 (FP32) of |W| |J V|."""
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


def _dev(M, blocks):
    return torch.from_numpy(M.pack(blocks)).to("cuda")


def _vjp(M, U, W):
    dt = torch.float32 if M.dtype_np == np.float32 else torch.float64
    out = torch.zeros(M.state_len, dtype=dt, device="cuda")
    M.vjp(_dev(M, U), _dev(M, W), out)
    M.sync()
    return M.unpack(out.cpu().numpy())


def _jvp(M, U, V):
    dt = torch.float32 if M.dtype_np == np.float32 else torch.float64
    out = torch.zeros(M.state_len, dtype=dt, device="cuda")
    M.jvp(_dev(M, U), _dev(M, V), out)
    M.sync()
    return M.unpack(out.cpu().numpy())


def _shifted_gas(X):
    # smooth_gas has a zero momentum component on planes through Gauss points
    # of the 2-cell boxes (x = 0.75), where |v.n| has a kink and the
    # derivative is not unique; the shift moves those planes off the points.
    return gu.smooth_gas(X + 0.1234)


def _state(geom, oph, seed):
    if oph.system == "euler":
        return gu.perturb(gu.oracle_state(geom, _shifted_gas, oph.nvar), seed, 0.02)
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]


SMALL = [("tri", (4, 4), 2, "euler", "rusanov"), ("tet", (2, 2, 2), 1, "euler", "rusanov"),
         ("hex", (2, 2, 2), 2, "euler", "roe"), ("tet", (2, 2, 2), 3, "advection", "upwind"),
         ("quad", (4, 3), 3, "euler", "roe")]


@pytest.mark.parametrize("kind,n,p,system,riemann", SMALL)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vjp_matches_oracle_dense_jacobian(ctx, kind, n, p, system, riemann, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riemann, precision)
    U = _state(geom, oph, 31)
    rng = np.random.default_rng(32)
    W = [rng.normal(size=u.shape) for u in U]
    want = ores.vjp(geom, oph, U, W)
    linf, l2 = gu.rel_errors(_vjp(M, U, W), want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


def _dot(a, b):
    return float(sum(np.vdot(x.astype(np.float64), y.astype(np.float64)) for x, y in zip(a, b)))


@pytest.mark.parametrize("kind,n,p,system,riemann", [("tet", (5, 4, 4), 3, "euler", "rusanov"),
                                                     ("tet", (4, 4, 3), 4, "euler", "rusanov"),
                                                     ("pri", (5, 4, 3), 2, "euler", "roe"),
                                                     ("hex", (5, 4, 3), 3, "advection", "upwind"),
                                                     ("tri", (21, 17), 4, "euler", "rusanov")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_identity(ctx, kind, n, p, system, riemann, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riemann, precision)
    U = _state(geom, oph, 33)
    rng = np.random.default_rng(34)
    V = [rng.normal(size=u.shape) for u in U]
    W = [rng.normal(size=u.shape) for u in U]
    JV = _jvp(M, U, V)
    JTW = _vjp(M, U, W)
    lhs, rhs = _dot(W, JV), _dot(JTW, V)
    scale = np.sqrt(_dot(W, W) * _dot(JV, JV))
    tol = 1e-11 if precision == "fp64" else 1e-4
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)


def test_adjoint_identity_mixed_mesh(ctx):
    from inputs import meshes
    from oracle import mesh as omesh
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh(["tet", "tet", "pri"], (3, 3, 3), [0, 0, 0], [1, 1, 1])
    degs = {"tet": 3, "pri": 3}
    M = sdrt.Mesh(ctx, mesh, degs, sdrt.make_physics("euler", 3, "rusanov", "fp64"))
    geom = omesh.build(mesh, degs)
    U = gu.perturb(gu.oracle_state(geom, _shifted_gas, 5), 35, 0.02)
    rng = np.random.default_rng(36)
    V = [rng.normal(size=u.shape) for u in U]
    W = [rng.normal(size=u.shape) for u in U]
    JV, JTW = _jvp(M, U, V), _vjp(M, U, W)
    lhs, rhs = _dot(W, JV), _dot(JTW, V)
    assert abs(lhs - rhs) <= 1e-11 * np.sqrt(_dot(W, W) * _dot(JV, JV)), (lhs, rhs)


# Viscous systems with non-symmetric LDG weights (beta != 0) and a penalty, so
# that the face orientation and every term of the common value / flux enter.
VISC = [("hex", (2, 2, 2), 1, "ns", "rusanov"), ("quad", (3, 3), 2, "ns", "roe"),
        ("tet", (2, 2, 1), 1, "ns", "rusanov"), ("tet", (2, 2, 2), 2, "advdiff", "upwind"),
        ("tri", (4, 4), 3, "advdiff", "upwind")]
VISC_KW = {"mu": 0.03, "beta": 0.3, "eta": 0.1, "prandtl": 0.71}


@pytest.mark.parametrize("kind,n,p,system,riemann", VISC)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_viscous_vjp_matches_oracle_dense_jacobian(ctx, kind, n, p, system, riemann, precision):
    a = (0.8, -0.4, 0.3) if system == "advdiff" else (1.0, 0.5, 0.25)
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riemann, precision, a=a, **VISC_KW)
    if system == "ns":
        U = gu.perturb(gu.oracle_state(geom, _shifted_gas, oph.nvar), 41, 0.02)
    else:
        U = _state(geom, oph, 41)
    rng = np.random.default_rng(42)
    W = [rng.normal(size=u.shape) for u in U]
    want = ores.vjp(geom, oph, U, W)
    linf, l2 = gu.rel_errors(_vjp(M, U, W), want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


@pytest.mark.parametrize("kind,n,p,system", [("tet", (4, 3, 3), 3, "ns"), ("pri", (3, 3, 3), 2, "ns"),
                                             ("hex", (4, 3, 2), 2, "advdiff"), ("tet", (3, 3, 2), 4, "ns")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_viscous_adjoint_identity(ctx, kind, n, p, system, precision):
    riem = "upwind" if system == "advdiff" else "rusanov"
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riem, precision, **VISC_KW)
    if system == "ns":
        U = gu.perturb(gu.oracle_state(geom, _shifted_gas, oph.nvar), 43, 0.02)
    else:
        U = _state(geom, oph, 43)
    rng = np.random.default_rng(44)
    V = [rng.normal(size=u.shape) for u in U]
    W = [rng.normal(size=u.shape) for u in U]
    JV = _jvp(M, U, V)
    JTW = _vjp(M, U, W)
    lhs, rhs = _dot(W, JV), _dot(JTW, V)
    scale = np.sqrt(_dot(W, W) * _dot(JV, JV))
    tol = 1e-11 if precision == "fp64" else 1e-4
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)


def test_autograd_backward_navier_stokes(ctx):
    from paper_2105_08632_gb300 import autograd
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 2, "ns", "rusanov", "fp64", **VISC_KW)
    U = _dev(M, gu.perturb(gu.oracle_state(geom, _shifted_gas, 5), 45, 0.02))
    rng = np.random.default_rng(46)
    W = _dev(M, [rng.normal(size=(g.ops.n_sol, 5, g.nelem)) for g in geom.blocks])
    Ug = U.clone().requires_grad_(True)
    (g,) = torch.autograd.grad((autograd.residual(Ug, M) * W).sum(), Ug)
    g_ref = torch.zeros_like(U)
    M.vjp(U, W, g_ref)
    assert torch.equal(g, g_ref)


def test_autograd_function_matches_the_c_abi(ctx):
    from paper_2105_08632_gb300 import autograd
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 3, "euler", "rusanov", "fp64")
    U = _dev(M, _state(geom, oph, 37))
    rng = np.random.default_rng(38)
    V = _dev(M, [rng.normal(size=(g.ops.n_sol, 5, g.nelem)) for g in geom.blocks])
    W = _dev(M, [rng.normal(size=(g.ops.n_sol, 5, g.nelem)) for g in geom.blocks])
    # forward
    R = autograd.residual(U, M)
    R_ref = torch.zeros_like(U)
    M.residual(U, R_ref)
    assert torch.equal(R, R_ref)
    # reverse mode = VJP
    Ug = U.clone().requires_grad_(True)
    (g,) = torch.autograd.grad((autograd.residual(Ug, M) * W).sum(), Ug)
    g_ref = torch.zeros_like(U)
    M.vjp(U, W, g_ref)
    assert torch.equal(g, g_ref)
    # forward mode = JVP
    import torch.autograd.forward_ad as fwAD
    with fwAD.dual_level():
        out = autograd.residual(fwAD.make_dual(U, V), M)
        tangent = fwAD.unpack_dual(out).tangent
    j_ref = torch.zeros_like(U)
    M.jvp(U, V, j_ref)
    assert torch.equal(tangent, j_ref)


def test_binding_rejects_bad_state_arrays(ctx):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 2, "euler", "rusanov", "fp32")
    good = torch.zeros(M.state_len, dtype=torch.float32, device="cuda")
    for bad in (torch.zeros(M.state_len - 1, dtype=torch.float32, device="cuda"),
                torch.zeros(M.state_len, dtype=torch.float64, device="cuda"),
                torch.zeros(M.state_len, dtype=torch.float32)):
        with pytest.raises(ValueError):
            M.residual(bad, good)
