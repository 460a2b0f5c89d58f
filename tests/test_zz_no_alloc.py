"""sdrt_residual_noalloc: the residual for callers that cannot allocate device
memory (plugins inside another framework's memory pool, loops that cannot take
cudaMalloc's implicit synchronisation).  It must give the same result as
sdrt_residual, on consecutive calls (its scratch buffer is shared and keeps the
previous call's contents), allocate no device memory, and reject meshes whose
face states exceed its fixed buffer.

Kept in a file that pytest collects last; it is self-contained, so it passes
alone in a fresh process and after the other tests."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests import gpu_util as gu  # noqa: E402

TOL32 = (2e-4, 2e-5)     # the FP32 tolerances of the parity tests
TOL64 = 1e-10


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    c = sdrt.Context(0)
    yield c
    c.close()


def _states(geom, seeds):
    return [gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), s, 0.02) for s in seeds]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_residual_on_two_calls(ctx, precision):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (4, 3, 3), 3, "euler", "rusanov", precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    U1, U2 = (torch.from_numpy(M.pack(u)).to("cuda") for u in _states(geom, (21, 22)))
    ref1, ref2, out1, out2 = (torch.zeros(M.state_len, dtype=dt, device="cuda") for _ in range(4))
    M.residual(U1, ref1)
    M.residual(U2, ref2)
    M.sync()
    sdrt.sdrt_residual_noalloc(ctx.ptr, M.id, U1, out1)      # first call: buffer set-up
    M.sync()
    free_before, _ = torch.cuda.mem_get_info()
    sdrt.sdrt_residual_noalloc(ctx.ptr, M.id, U2, out2)      # second call, buffer holds call 1's data
    M.sync()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    for out, ref in ((out1, ref1), (out2, ref2)):
        linf, l2 = gu.rel_errors(M.unpack(out.cpu().numpy()), M.unpack(ref.cpu().numpy()))
        if precision == "fp64":
            assert linf < TOL64, linf
        else:
            assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


def test_first_noalloc_call_allocates_nothing():
    """A fresh context: the static buffer is resolved when the context is
    created, so free device memory is unchanged across the first
    allocation-free call (kernel code loaded beforehand by sdrt_residual on
    the same generic-path mesh)."""
    from paper_2105_08632_gb300 import sdrt
    c = sdrt.Context(0)
    try:
        # the generic kernels for sdrt_residual too (the operator-specialised
        # ones would otherwise take this mesh), so that their code is loaded
        sdrt.sdrt_set_option(c.ptr, sdrt.SDRT_OPT_GENERATED, 0)
        M, geom, oph, _ = gu.build_pair(c, "hex", (3, 3, 2), 2, "euler", "rusanov", "fp32")
        U = torch.from_numpy(M.pack(_states(geom, (31,))[0])).to("cuda")
        ref, out = torch.zeros_like(U), torch.zeros_like(U)
        M.residual(U, ref)
        M.sync()
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        sdrt.sdrt_residual_noalloc(c.ptr, M.id, U, out)
        M.sync()
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after == free_before, (free_before, free_after)
        # generic path on both sides: the same kernels on the same data
        assert torch.equal(out, ref)
    finally:
        c.close()


def test_noalloc_rejects_meshes_beyond_its_buffer(ctx):
    from inputs import meshes
    from paper_2105_08632_gb300 import sdrt
    # 16^3 x 6 = 24,576 tets of degree 4 in FP64: 5 x 60 x 24,576 x 8 B = 59 MB > 32 MiB
    mesh = meshes.box_mesh("tet", (16, 16, 16), [0.0] * 3, [1.0] * 3)
    M = sdrt.Mesh(ctx, mesh, 4, sdrt.make_physics("euler", 3, "rusanov", "fp64"))
    U = torch.zeros(M.state_len, dtype=torch.float64, device="cuda")
    R = torch.zeros_like(U)
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_residual_noalloc(ctx.ptr, M.id, U, R)
    assert ei.value.code == -2
    assert "33554432" in str(ei.value)
