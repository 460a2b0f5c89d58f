"""Parity at the benchmark's size and launch configuration, and agreement of the
tensor-core (tcgen05, 3xTF32) and CUDA-core interpolation and divergence paths.

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


def _options(ctx, interp_tc, div_tc):
    from paper_2105_08632_gb300 import sdrt
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TENSOR_CORES, interp_tc)
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_DIVERGENCE, div_tc)


@pytest.mark.parametrize("interp_tc,div_tc", [(1, 0), (0, 0), (0, 1), (1, 1)])
def test_tensor_core_and_fma_paths(ctx, interp_tc, div_tc):
    _options(ctx, interp_tc, div_tc)
    try:
        # 5 x 5 x 5 x 6 = 750 tets: 6 interpolation tiles of 128 and 32
        # divergence tiles of 24, the last ones ragged
        M, geom, oph, _ = gu.build_pair(ctx, "tet", (5, 5, 5), 3, "euler", "rusanov", "fp32")
        U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 31, 0.02)
        linf, l2 = gu.rel_errors(_residual(M, U), ores.residual(geom, oph, U))
        assert linf < TOL32[0] and l2 < TOL32[1], (interp_tc, div_tc, linf, l2)
    finally:
        _options(ctx, 0, 0)


@pytest.mark.parametrize("div_tc", [1, 0])
def test_rk4_stages_on_tensor_core_divergence(ctx, div_tc):
    """Every epilogue mode (RK stages 1..4) of the tensor-core divergence
    against the FMA kernel over three RK4 steps on 4 x 4 x 3 x 6 tets."""
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (4, 4, 3), 3, "euler", "rusanov", "fp32")
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 32, 0.01)
    dt = 2e-3
    want = U
    for _ in range(3):
        want = ores.rk4_step(geom, oph, want, dt)
    _options(ctx, 0, div_tc)
    try:
        Ud = torch.from_numpy(M.pack(U)).to("cuda")
        M.rk4_step(Ud, dt, 3)
        M.sync()
        got = M.unpack(Ud.cpu().numpy())
    finally:
        _options(ctx, 0, 0)
    d_got = [g - u for g, u in zip(got, U)]
    d_want = [w - u for w, u in zip(want, U)]
    linf, _ = gu.rel_errors(d_got, d_want)
    assert linf < 5e-3, (div_tc, linf)


@pytest.mark.parametrize("div_tc", [1, 0])
def test_full_size_benchmark_workload(ctx, div_tc):
    from paper_2105_08632_gb300 import sdrt
    _options(ctx, 0, div_tc)
    mesh = meshes.box_mesh("tet", (24, 24, 24), [-5.0] * 3, [5.0] * 3)
    M = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
    geom = omesh.build(mesh, 3)
    g = geom.blocks[0]
    X = g.xsol.reshape(-1, 3)
    u = fields.isentropic_vortex(X, gamma=1.4, mach=0.5)
    u = u * (1 + fields.uniform_noise(u.shape, 20210518, 1e-3))
    U = [np.ascontiguousarray(u.reshape(g.nelem, g.ops.n_sol, 5).transpose(1, 2, 0))]
    want, scale = ores.residual(geom, ophx.Physics("euler", 3, "rusanov", gamma=1.4), U, terms=True)
    try:
        got = _residual(M, U)
    finally:
        _options(ctx, 0, 0)
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


@pytest.mark.parametrize("ncell", [(3, 3, 3), (24, 24, 24)])
def test_fused_rk_stages_match_the_unfused_sequence(ctx, ncell):
    """RK4 with the next stage's interpolation in the stage update
    (SDRT_OPT_FUSED_RK, one interpolation and four flux kernels per step)
    against one interpolation kernel per stage: the same FP32 operations in
    the same order, so the states after three steps agree bit for bit.
    162 tetrahedra: five full tiles of 32 and a ragged one of 2; 82,944: the
    benchmark workload."""
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh("tet", ncell, [-5.0] * 3, [5.0] * 3)
    M = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
    X = M.sol_points()[0]
    u = fields.isentropic_vortex(X.reshape(-1, 3), gamma=1.4, mach=0.5).reshape(X.shape[0], X.shape[1], 5)
    u = u * (1 + fields.uniform_noise(u.shape, 7, 1e-2))
    U0 = M.pack([np.ascontiguousarray(u.transpose(1, 2, 0))])
    out = {}
    try:
        for fused in (1, 0):
            sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_FUSED_RK, fused)
            Ud = torch.from_numpy(U0.copy()).to("cuda")
            M.rk4_step(Ud, 1e-3, 3)
            M.sync()
            out[fused] = Ud.cpu().numpy()
    finally:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_FUSED_RK, 1)
    assert np.isfinite(out[1]).all()
    assert not np.array_equal(out[1], U0)
    assert np.array_equal(out[1], out[0])


def test_tf32x3_precision_routes_to_the_tensor_cores(ctx):
    """SDRT_TF32X3 through the boundary: FP32 states, the record path's
    interpolation and divergence on the tensor cores -- the same results, bit
    for bit, as an FP32 mesh with both tensor-core options on, and within the
    FP32 parity bounds of the oracle (2e-4 / 2e-5)."""
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh("tet", (3, 3, 3), [-5.0] * 3, [5.0] * 3)
    geom = omesh.build(mesh, 3)
    g = geom.blocks[0]
    u = fields.isentropic_vortex(g.xsol.reshape(-1, 3), gamma=1.4, mach=0.5)
    u = u * (1 + fields.uniform_noise(u.shape, 11, 1e-2))
    U = [np.ascontiguousarray(u.reshape(g.nelem, g.ops.n_sol, 5).transpose(1, 2, 0))]
    M3 = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "tf32x3", gamma=1.4))
    assert M3.info["precision"] == 2 and M3.dtype_np == np.float32 and M3.info["path"] == 1
    r3 = _residual(M3, U)
    M1 = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
    _options(ctx, 1, 1)
    try:
        r_tc = _residual(M1, U)
    finally:
        _options(ctx, 0, 0)
    r_fma = _residual(M1, U)
    assert all(np.array_equal(a, b) for a, b in zip(r3, r_tc))
    assert not all(np.array_equal(a, b) for a, b in zip(r3, r_fma))      # a different product split
    linf, l2 = gu.rel_errors(r3, ores.residual(geom, ophx.Physics("euler", 3, "rusanov", gamma=1.4), U))
    assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)
