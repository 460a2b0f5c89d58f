"""FR-SDRT (Sec. 2.3) on the GPU: element types with the FR scheme run the
generic kernels with the FR operators; the residual is compared element by
element with the oracle's FR-SDRT residual (flux at the solution points,
differentiated there, plus the M14 correction; its own differentiation
matrices), and for linear advection with the GPU's SDRT residual (the two
schemes coincide for linear fluxes on affine meshes, Sec. 2.3)."""
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


def _res(M, U):
    Ud = torch.from_numpy(M.pack(U)).cuda()
    R = torch.zeros_like(Ud)
    M.residual(Ud, R)
    M.sync()
    return M.unpack(R.cpu().numpy())


CASES = [
    ("tet", (2, 2, 2), 3, "euler", "rusanov", "fp64", {}),
    ("tet", (3, 2, 2), 2, "euler", "roe", "fp64", {}),
    ("hex", (2, 2, 2), 2, "euler", "rusanov", "fp64", {}),
    ("pri", (2, 2, 2), 3, "advection", "upwind", "fp64", {}),
    ("tri", (4, 3), 4, "euler", "rusanov", "fp64", {}),
    ("quad", (3, 3), 3, "ns", "rusanov", "fp64", {"mu": 0.03, "prandtl": 0.72, "beta": 0.5, "eta": 0.1}),
    ("tet", (2, 2, 2), 2, "ns", "rusanov", "fp64", {"mu": 0.02, "prandtl": 0.72, "beta": 0.25, "eta": 0.2}),
    ("tet", (3, 3, 2), 3, "euler", "rusanov", "fp32", {}),
]


@pytest.mark.parametrize("kind,n,p,system,riemann,precision,kw", CASES)
def test_fr_residual_matches_oracle(ctx, kind, n, p, system, riemann, precision, kw):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, system, riemann, precision, scheme="fr", **kw)
    nv = M.nvar
    if system == "advection":
        U = [np.random.default_rng(41).uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    else:
        U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, nv), 42, 0.02)
    want = ores.residual(geom, oph, U, fr=True)
    linf, l2 = gu.rel_errors(_res(M, U), want)
    tol = (1e-10, 1e-11) if precision == "fp64" else (2e-4, 2e-5)
    assert linf < tol[0] and l2 < tol[1], (linf, l2)


@pytest.mark.parametrize("kind,n,p", [("tet", (2, 2, 2), 3), ("hex", (2, 2, 2), 2), ("tri", (4, 4), 3)])
def test_fr_equals_sdrt_for_linear_advection(ctx, kind, n, p):
    Mf, geom, _, _ = gu.build_pair(ctx, kind, n, p, "advection", "upwind", "fp64", scheme="fr")
    Ms, _, _, _ = gu.build_pair(ctx, kind, n, p, "advection", "upwind", "fp64")
    U = [np.random.default_rng(43).uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    linf, _ = gu.rel_errors(_res(Mf, U), _res(Ms, U))
    assert linf < 1e-11, linf
