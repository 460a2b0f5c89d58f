"""Fourier stability analysis on the GPU against the paper's CFL_MAX tables
for SDRT with RK schemes (Sec. 4, Tables "quad_sdrt_cfl_theta=pi/6" and
"hex_sdrt_cfl_theta0=pi/6_theta1=pi/4"): quadrilaterals with the advection
angle theta0 = pi/6 and hexahedra with theta0 = pi/6, theta1 = pi/4; the
tensor-product point sets (Gauss-Legendre) are fully specified by the paper,
so these values pin the whole operator chain (operators, metrics, face map,
upwind flux, JVP) to the paper's numbers.  The tables are reproduced with the
wavenumber along the advection direction (as the paper states), kappa h in
[0, 2 pi]; the range and sampling are not stated, hence a 5 % tolerance (the
quadrilateral RK4 column agrees to 0.4 %).  Over the whole wavenumber zone
degree 2 is more restrictive (0.266 on quadrilaterals).
The reduced Jacobians are assembled from the library's FP64 JVPs; eigenvalues
in FP64 on the GPU.  The whole-zone 32^3 grid of the differentiation
configuration is exercised for tetrahedra and prisms (stable operator,
finite CFL).  The pure-diffusion table for quadrilateral SDRT (Sec.
"Von-Neumann analysis with diffusion", Table "diff_quad_sdrt_cfl") pins the
library's LDG path the same way."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# The paper states neither the kappa h range nor its sampling: with kappa
# parallel to a and kappa h in [0, 2 pi] the RK4 column of the quadrilateral
# table agrees within 0.4 % (asserted to 0.6 %), the other entries within 4.3 %.
TOL = 0.05

# (RK3, RK4, RK54) per degree, as printed in the paper
QUAD = {1: (0.459, 0.509, 0.695), 2: (0.235, 0.281, 0.392), 3: (0.149, 0.165, 0.247), 4: (0.102, 0.119, 0.173)}
HEX = {1: (0.345, 0.403, 0.552), 2: (0.187, 0.222, 0.304), 3: (0.117, 0.131, 0.196), 4: (0.081, 0.094, 0.136)}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    c = sdrt.Context(0)
    yield c
    c.close()


def _advection(ctx, kind, p, a, kappas, schemes):
    from inputs import meshes
    from paper_2105_08632_gb300 import sdrt
    from paper_2105_08632_gb300 import stability as st
    nd = len(a)
    mesh = meshes.box_mesh(kind, (3,) * nd, [0.0] * nd, [3.0] * nd)
    phys = sdrt.make_physics("advection", nd, "upwind", "fp64", a=a)
    return st.cfl_table(ctx, mesh, 3, [p], phys, kappas, schemes)[p]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_quadrilateral_cfl_table(ctx, p):
    from paper_2105_08632_gb300 import stability as st
    a = st.advection_direction(np.pi / 6)
    got = _advection(ctx, "quad", p, a, st.kappa_line(a, 721), ("rk3", "rk4", "rk54"))
    assert got["max_real"] < 1e-10                 # the semi-discrete operator is stable
    for s, want in zip(("rk3", "rk4", "rk54"), QUAD[p]):
        assert abs(got[s] - want) <= TOL * want, (p, s, got[s], want)
    assert abs(got["rk4"] - QUAD[p][1]) <= 0.006 * QUAD[p][1] + 5e-4, (p, got["rk4"])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_hexahedron_cfl_table(ctx, p):
    from paper_2105_08632_gb300 import stability as st
    a = st.advection_direction(np.pi / 6, np.pi / 4)
    got = _advection(ctx, "hex", p, a, st.kappa_line(a, 361), ("rk4",))
    assert got["max_real"] < 1e-10
    assert abs(got["rk4"] - HEX[p][1]) <= TOL * HEX[p][1], (p, got["rk4"], HEX[p][1])


@pytest.mark.parametrize("kind,p", [("tet", 2), ("pri", 2)])
def test_simplex_whole_zone_grid(ctx, kind, p):
    from paper_2105_08632_gb300 import stability as st
    a = st.advection_direction(np.pi / 6, np.pi / 4)
    got = _advection(ctx, kind, p, a, st.kappa_grid(3, 32), ("rk4",))
    # stable up to the eigen-solver's rounding on a non-normal G
    assert got["max_real"] < 1e-8 * got["max_abs"], got
    assert 0.02 < got["rk4"] < 1.0, got


# Table "diff_quad_sdrt_cfl" (pure diffusion, BR1 beta = 0, eta = 0): (RK3,
# RK4, RK54) per degree, as printed; the printed values are the CFL_MAX
# truncated to 4 decimals, with kappa along a mesh axis, kappa h in [0, 2 pi].
DIFF_QUAD = {1: (0.2791, 0.3094, 0.5174), 2: (0.0348, 0.0386, 0.0646), 3: (0.0157, 0.0174, 0.0291),
             4: (0.0055, 0.0061, 0.0103)}


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_quadrilateral_diffusion_cfl_table(ctx, p):
    """The library's LDG path (common value, lifting, gradient interpolation,
    common viscous flux) through its FP64 JVP reproduces the paper's diffusion
    table exactly (4-decimal truncation), like the oracle does."""
    from inputs import meshes
    from paper_2105_08632_gb300 import sdrt
    from paper_2105_08632_gb300 import stability as st
    mesh = meshes.box_mesh("quad", (5, 5), [0.0, 0.0], [5.0, 5.0])
    phys = sdrt.make_physics("advdiff", 2, "upwind", "fp64", a=(0.0, 0.0), mu=1.0, beta=0.0, eta=0.0)
    got = st.cfl_table(ctx, mesh, 5, [p], phys, st.kappa_line((1.0, 0.0), 361), ("rk3", "rk4", "rk54"))[p]
    assert got["max_real"] < 1e-10 * got["max_abs"]
    for s, want in zip(("rk3", "rk4", "rk54"), DIFF_QUAD[p]):
        assert np.floor(got[s] * 1e4 + 1e-9) == round(want * 1e4), (p, s, got[s], want)
