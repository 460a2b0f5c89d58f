"""Parity at the benchmark's size and launch configuration, and agreement of the
tensor-core (tcgen05, 3xTF32) and CUDA-core interpolation paths.

The full-size case is the benchmark workload: Euler on the periodic cube
[-5, 5]^3 split into 24^3 x 6 = 82,944 tetrahedra of degree 3, isentropic
vortex (Ma 0.5) times (1 + 1e-3 U(-1, 1)), FP32 -- compared element by element
with the FP64 oracle evaluated on the same state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import fields, meshes  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from oracle import physics as ophx  # noqa: E402
from oracle import residual as ores  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

TOL32 = (2e-4, 2e-5)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    stream = torch.cuda.Stream(0)
    torch.cuda.set_stream(stream)
    c = sdrt.Context(0, stream.cuda_stream)
    yield c
    c.close()


def _residual(M, U_blocks):
    U = torch.from_numpy(M.pack(U_blocks)).to("cuda")
    R = torch.zeros_like(U)
    M.residual(U, R)
    M.sync()
    return M.unpack(R.cpu().numpy())


@pytest.mark.parametrize("use_tc", [1, 0])
def test_tensor_core_and_fma_interpolation(ctx, use_tc):
    from paper_2105_08632_gb300 import sdrt
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TENSOR_CORES, use_tc)
    try:
        # 5 x 5 x 5 x 6 = 750 tets: 5 tensor-core tiles of 128, the last one ragged
        M, geom, oph, _ = gu.build_pair(ctx, "tet", (5, 5, 5), 3, "euler", "rusanov", "fp32")
        U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 31, 0.02)
        linf, l2 = gu.rel_errors(_residual(M, U), ores.residual(geom, oph, U))
        assert linf < TOL32[0] and l2 < TOL32[1], (use_tc, linf, l2)
    finally:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TENSOR_CORES, 1)


def test_full_size_benchmark_workload(ctx):
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh("tet", (24, 24, 24), [-5.0] * 3, [5.0] * 3)
    M = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
    geom = omesh.build(mesh, 3)
    g = geom.blocks[0]
    X = g.xsol.reshape(-1, 3)
    u = fields.isentropic_vortex(X, gamma=1.4, mach=0.5)
    u = u * (1 + fields.uniform_noise(u.shape, 20210518, 1e-3))
    U = [np.ascontiguousarray(u.reshape(g.nelem, g.ops.n_sol, 5).transpose(1, 2, 0))]
    want, scale = ores.residual(geom, ophx.Physics("euler", 3, "rusanov", gamma=1.4), U, terms=True)
    got = _residual(M, U)
    linf, l2 = gu.rel_errors(got, want)
    # The vortex is close to a free stream: dU/dt is a small difference of large
    # flux terms, so the FP32 error is bounded elementwise by the forward-error
    # scale u * S (S = sum of |operator| |flux| terms / det J, u = 2^-24) rather
    # than by max |dU/dt|: 70 summed terms, ~20-operation fluxes and 20-term
    # interpolations give a worst case of ~110 u S; the bound asserted is 128 u S.
    ratio = gu.fp32_bound_ratio(got, want, scale)
    assert ratio < 128 and l2 < TOL32[1], (ratio, linf, l2)
    # the face map at full size is the oracle's, bit for bit
    part, left = M.face_map()
    assert np.array_equal(part.astype(np.int64), geom.partner)
    assert np.array_equal(left.astype(bool), geom.is_left)
