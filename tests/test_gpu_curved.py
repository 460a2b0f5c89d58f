"""Curved (quadratic isoparametric) elements on the CUDA path against the
oracle (oracle/mapping.py, oracle/mesh.py: metrics at every point the method
evaluates them, paper Sec. 2 and 2.1), through sdrt_setup_mesh_curved:

* residuals element by element, every element type, Euler (Rusanov / Roe),
  advection, advection-diffusion and Navier-Stokes (LDG), FP64 (1e-10 of max
  |oracle|) and FP32 (2e-4 / 2e-5 as the affine parity tests), on meshes of
  several tiles with a ragged last tile;
* free-stream preservation on curved tetrahedra of degree 2 and 3;
* discrete conservation with the per-point det J;
* RK4 steps, the JVP (oracle complex step), the VJP (oracle dense Jacobian)
  and the adjoint identity;
* the allocation-free residual; the Taylor-Green diagnostics refuse curved
  meshes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import residual as ores  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

TOL64 = 1e-10
TOL32 = (2e-4, 2e-5)
AMP = 0.04


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


def _call(M, fn, *arrays):
    dt = torch.float32 if M.dtype_np == np.float32 else torch.float64
    out = torch.zeros(M.state_len, dtype=dt, device="cuda")
    fn(*[_dev(M, a) for a in arrays], out)
    M.sync()
    return M.unpack(out.cpu().numpy())


def _state(geom, oph, seed):
    if oph.system in ("euler", "ns"):
        return gu.perturb(gu.oracle_state(geom, lambda X: gu.smooth_gas(X + 0.1234), oph.nvar), seed, 0.02)
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]


CASES = [("tet", (3, 3, 3), 2, "euler", "rusanov"), ("tet", (3, 3, 2), 3, "euler", "roe"),
         ("hex", (4, 3, 3), 2, "euler", "rusanov"), ("pri", (3, 3, 3), 2, "advection", "upwind"),
         ("tri", (9, 7), 3, "euler", "rusanov"), ("quad", (7, 5), 3, "euler", "roe"),
         ("tet", (3, 3, 2), 2, "ns", "rusanov"), ("hex", (3, 3, 2), 2, "advdiff", "upwind"),
         ("tri", (7, 6), 2, "ns", "roe")]
VISC_KW = {"mu": 0.03, "beta": 0.3, "eta": 0.1, "prandtl": 0.71}


@pytest.mark.parametrize("kind,n,p,system,riemann", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_curved_residual_matches_oracle(ctx, kind, n, p, system, riemann, precision):
    kw = VISC_KW if system in ("ns", "advdiff") else {}
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riemann, precision, curve=AMP, curve_seed=5, **kw)
    assert M.info["curved"] == 1 and M.info["path"] == 0
    assert geom.blocks[0].curved
    U = _state(geom, oph, 21)
    linf, l2 = gu.rel_errors(_call(M, M.residual, U), ores.residual(geom, oph, U))
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_curved_free_stream(ctx, p, precision):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 3), p, "euler", "rusanov", precision, curve=AMP, curve_seed=2)
    state = np.array([1.2, 0.3, -0.2, 0.1, 3.0])
    U = [np.repeat(state[None, :, None], g.nelem, 2).repeat(g.ops.n_sol, 0) for g in geom.blocks]
    R = _call(M, M.residual, U)
    # zero up to rounding, in units of u S, S the magnitude of the divergence's
    # terms: FP32 arithmetic within 128 u S (u = 2^-24); in FP64 (u = 2^-53) the
    # operators' own construction error (Vandermonde inverses, condition ~1e3)
    # dominates: the oracle's FP64 residual of a uniform state reaches 270 u S on
    # affine degree-3 tetrahedra, so the bound is 4096 u S (~5e-13 S)
    _, S = ores.residual(geom, oph, U, terms=True)
    u, bound = (gu.U32, 128) if precision == "fp32" else (2.0 ** -53, 4096)
    ratio = max(float(np.max(np.abs(r) / (u * s + 1e-300))) for r, s in zip(R, S))
    assert ratio < bound, ratio


def test_curved_conservation(ctx):
    from tests.test_oracle_curved import _weights
    M, geom, oph, _ = gu.build_pair(ctx, "pri", (3, 3, 2), 3, "euler", "rusanov", "fp64", curve=AMP, curve_seed=8)
    U = _state(geom, oph, 23)
    R = _call(M, M.residual, U)
    tot = sum(np.einsum("s,sve,es->v", _weights(g), r, g.dets) for g, r in zip(geom.blocks, R))
    assert np.abs(tot).max() < 1e-11 * max(np.abs(r).max() for r in R)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_curved_rk4_steps(ctx, precision):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 3, "euler", "rusanov", precision, curve=AMP, curve_seed=6)
    U = _state(geom, oph, 25)
    dt = 1e-3
    W = U
    for _ in range(3):
        W = ores.rk4_step(geom, oph, W, dt)
    Ud = _dev(M, U)
    M.rk4_step(Ud, dt, 3)
    M.sync()
    got = M.unpack(Ud.cpu().numpy())
    linf, _ = gu.rel_errors([g - u for g, u in zip(got, U)], [w - u for w, u in zip(W, U)])
    assert linf < (1e-9 if precision == "fp64" else 5e-3), linf


@pytest.mark.parametrize("kind,n,p,system", [("tet", (2, 2, 1), 2, "euler"), ("hex", (2, 2, 1), 2, "ns"),
                                             ("tri", (4, 3), 2, "advdiff")])
def test_curved_jvp_and_vjp_match_oracle(ctx, kind, n, p, system):
    riem = "upwind" if system == "advdiff" else "rusanov"
    kw = VISC_KW if system in ("ns", "advdiff") else {}
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riem, "fp64", curve=AMP, curve_seed=9, **kw)
    U = _state(geom, oph, 27)
    rng = np.random.default_rng(28)
    V = [rng.normal(size=u.shape) for u in U]
    W = [rng.normal(size=u.shape) for u in U]
    linf, _ = gu.rel_errors(_call(M, M.jvp, U, V), ores.jvp(geom, oph, U, V))
    assert linf < TOL64, linf
    linf, _ = gu.rel_errors(_call(M, M.vjp, U, W), ores.vjp(geom, oph, U, W))
    assert linf < TOL64, linf


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_curved_adjoint_identity(ctx, precision):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (4, 4, 3), 3, "ns", "rusanov", precision, curve=AMP,
                                    curve_seed=3, **VISC_KW)
    U = _state(geom, oph, 29)
    rng = np.random.default_rng(30)
    V = [rng.normal(size=u.shape) for u in U]
    W = [rng.normal(size=u.shape) for u in U]
    JV, JTW = _call(M, M.jvp, U, V), _call(M, M.vjp, U, W)
    dot = lambda a, b: float(sum(np.vdot(x.astype(np.float64), y.astype(np.float64)) for x, y in zip(a, b)))  # noqa: E731
    lhs, rhs = dot(W, JV), dot(JTW, V)
    tol = 1e-11 if precision == "fp64" else 1e-4
    assert abs(lhs - rhs) <= tol * np.sqrt(dot(W, W) * dot(JV, JV)), (lhs, rhs)


def test_curved_noalloc_and_diagnostics_refusal(ctx):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 2, "euler", "rusanov", "fp32", curve=AMP, curve_seed=4)
    U = _dev(M, _state(geom, oph, 31))
    R1, R2 = torch.zeros_like(U), torch.zeros_like(U)
    M.residual(U, R1)
    sdrt.sdrt_residual_noalloc(ctx.ptr, M.id, U, R2)
    M.sync()
    assert torch.equal(R1, R2)
    Mn, geom_n, oph_n, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 2, "ns", "rusanov", "fp64", curve=AMP, **VISC_KW)
    with pytest.raises(sdrt.SdrtError) as ei:
        Mn.tgv_diagnostics(_dev(Mn, _state(geom_n, oph_n, 32)))
    assert ei.value.code == -2
