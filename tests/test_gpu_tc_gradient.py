"""The Navier-Stokes gradient chain on the tensor cores (k_grad_tc, 3xTF32,
SDRT_OPT_TC_GRADIENT, on by default) against the oracle and against the
CUDA-core gradient kernel: every instantiated element type (tetrahedra p3 /
p4, hexahedra p2, prisms p2), FP32, meshes of two 128-element tiles with a
ragged second one, non-symmetric LDG weights (beta != 1/2) so that the face
orientation enters; residuals within the FP32 parity bounds (2e-4 / 2e-5 of
max |oracle|) and within 1e-4 of the CUDA-core path; two RK4 steps within
the RK4 parity bound; a mesh with a block of another kind keeps the CUDA-core
kernel (bit-identical with the option off)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import residual as ores  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

TOL32 = (2e-4, 2e-5)
KW = {"mu": 0.02, "beta": 0.3, "eta": 0.1, "prandtl": 0.71}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    c = sdrt.Context(0)
    yield c
    c.close()


def _state(geom, seed):
    return gu.perturb(gu.oracle_state(geom, lambda X: gu.smooth_gas(X + 0.1234), 5), seed, 0.02)


def _residual(M, U):
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    R = torch.zeros_like(Ud)
    M.residual(Ud, R)
    M.sync()
    return M.unpack(R.cpu().numpy())


CASES = [("tet", (3, 3, 3), 4), ("tet", (3, 3, 3), 3), ("hex", (6, 5, 5), 2), ("pri", (5, 4, 4), 2)]


@pytest.mark.parametrize("kind,n,p", CASES)
def test_tensor_core_gradient_residual(ctx, kind, n, p):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "ns", "rusanov", "fp32", **KW)
    assert 128 < M.layouts[0]["nelem"] < 256
    U = _state(geom, 61)
    try:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_GRADIENT, 1)
        r_tc = _residual(M, U)
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_GRADIENT, 0)
        r_cc = _residual(M, U)
    finally:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_GRADIENT, 1)
    want = ores.residual(geom, oph, U)
    linf, l2 = gu.rel_errors(r_tc, want)
    assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)
    linf_cc, _ = gu.rel_errors(r_tc, r_cc)
    assert linf_cc < 1e-4, linf_cc
    assert not all(np.array_equal(a, b) for a, b in zip(r_tc, r_cc))      # the tensor-core path ran


def test_tensor_core_gradient_rk4_steps(ctx):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 3), 4, "ns", "rusanov", "fp32", **KW)
    U = _state(geom, 62)
    dt = 2e-4
    W = U
    for _ in range(2):
        W = ores.rk4_step(geom, oph, W, dt)
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    M.rk4_step(Ud, dt, 2)
    M.sync()
    got = M.unpack(Ud.cpu().numpy())
    linf, _ = gu.rel_errors([g - u for g, u in zip(got, U)], [w - u for w, u in zip(W, U)])
    assert linf < 5e-3, linf


def test_other_element_types_keep_the_cuda_core_kernel(ctx):
    """Tetrahedra of degree 2 have no tensor-core gradient: with them in the mesh
    (beside prisms of degree 2, which have one) every block keeps the CUDA-core
    kernel."""
    from inputs import meshes
    from oracle import mesh as omesh
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh(["tet", "tet", "pri"], (3, 3, 3), [0, 0, 0], [1, 1, 1])
    M = sdrt.Mesh(ctx, mesh, {"tet": 2, "pri": 2}, sdrt.make_physics("ns", 3, "rusanov", "fp32", **KW))
    geom = omesh.build(mesh, {"tet": 2, "pri": 2})
    U = _state(geom, 63)
    try:
        r_on = _residual(M, U)
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_GRADIENT, 0)
        r_off = _residual(M, U)
    finally:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_GRADIENT, 1)
    assert all(np.array_equal(a, b) for a, b in zip(r_on, r_off))
