"""Per-launch event timing of the library (used by bench.py's roofline): the
counts match the launches of an RK4 step, with and without the captured graph."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests import gpu_util as gu  # noqa: E402


@pytest.mark.parametrize("generated", [0, 1])
def test_profile_counts_rk4_steps(generated):
    """Generic kernels: one interpolation and one residual launch per stage.
    Operator-specialised kernels: one interpolation per step (later stages
    write the next stage's face records), one stage launch per stage."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    stream = torch.cuda.Stream(0)
    with torch.cuda.stream(stream):
        ctx = sdrt.Context(0, stream.cuda_stream)
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_GENERATED, generated)
        M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 2, "euler", "rusanov", "fp32")
        assert sdrt.sdrt_get_mesh_info(ctx.ptr, M.id)["path"] == (2 if generated else 0)
        n_interp = 1 if generated else 4
        U = torch.from_numpy(M.pack(gu.oracle_state(geom, gu.smooth_gas, 5))).to("cuda")
        M.rk4_step(U, 1e-3, 1)                 # eager warm-up step
        sdrt.sdrt_profile_enable(ctx.ptr, True)
        for _ in range(3):                     # graph captured on the first, replayed after
            M.rk4_step(U, 1e-3, 1)
            prof = sdrt.sdrt_profile_collect(ctx.ptr)
            assert prof["interp_ext"][1] == n_interp and prof["residual"][1] == 4
            assert prof["residual"][0] > 0 and prof["interp_ext"][0] > 0
        R = torch.zeros_like(U)
        M.residual(U, R)
        prof = sdrt.sdrt_profile_collect(ctx.ptr)
        assert prof["interp_ext"][1] == 1 and prof["residual"][1] == 1
        sdrt.sdrt_profile_enable(ctx.ptr, False)
        M.sync()
        ctx.close()


def test_nvtx_ranges_leave_results_unchanged():
    """SDRT_OPT_NVTX: host-side markers only; the residual and RK4 steps are
    bit-identical with and without them."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    ctx = sdrt.Context(0)
    try:
        M, geom, oph, _ = gu.build_pair(ctx, "hex", (3, 3, 2), 2, "ns", "rusanov", "fp32", mu=0.02)
        U0 = torch.from_numpy(M.pack(gu.oracle_state(geom, gu.smooth_gas, 5))).to("cuda")
        out = []
        for nvtx in (0, 1):
            sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_NVTX, nvtx)
            U = U0.clone()
            R = torch.zeros_like(U)
            M.residual(U, R)
            M.rk4_step(U, 1e-3, 2)
            M.sync()
            out.append((R, U))
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_NVTX, 0)
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    finally:
        ctx.close()
