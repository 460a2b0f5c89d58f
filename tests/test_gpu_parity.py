"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (normalised by max |oracle|):
  FP64 path  rel L-inf <= 1e-10 (operators built in a different basis: the
             difference is the rounding of two FP64 evaluations);
  FP32 path  rel L-inf <= 2e-4, rel L2 <= 2e-5 (single-precision storage of
             the state, operators and metrics; sums of up to ~500 terms of
             mixed sign in the divergence).
Meshes span several 32-element tiles with a ragged last tile."""
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


EULER_CASES = [("tet", (3, 3, 3), p) for p in (1, 2, 3, 4)] + \
              [("pri", (3, 3, 3), p) for p in (1, 2, 3, 4)] + \
              [("hex", (3, 3, 3), p) for p in (1, 2, 3, 4)] + \
              [("tri", (7, 5), 2), ("quad", (6, 7), 3)]


@pytest.mark.parametrize("kind,n,p", EULER_CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_euler_rusanov_residual(ctx, kind, n, p, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "euler", "rusanov", precision)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, oph.nvar), 11, 0.02)
    want = ores.residual(geom, oph, U)
    got = _gpu_residual(M, U)
    linf, l2 = gu.rel_errors(got, want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


@pytest.mark.parametrize("kind,n,p", [("tet", (3, 3, 3), 3), ("hex", (3, 3, 3), 2), ("pri", (3, 2, 3), 2),
                                      ("quad", (5, 5), 2)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_euler_roe_residual(ctx, kind, n, p, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "euler", "roe", precision)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, oph.nvar), 12, 0.02)
    want = ores.residual(geom, oph, U)
    got = _gpu_residual(M, U)
    linf, l2 = gu.rel_errors(got, want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


@pytest.mark.parametrize("kind,n,p", [("tri", (16, 16), 2), ("tet", (3, 3, 3), 3), ("hex", (3, 3, 2), 3),
                                      ("pri", (3, 3, 3), 4)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_advection_residual(ctx, kind, n, p, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "advection", "upwind", precision, a=(1.0, 0.5, 0.25))
    rng = np.random.default_rng(13)
    U = [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    want = ores.residual(geom, oph, U)
    got = _gpu_residual(M, U)
    linf, l2 = gu.rel_errors(got, want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


@pytest.mark.parametrize("kinds,degs", [(["tet", "tet", "pri"], {"tet": 3, "pri": 3}),
                                        (["hex", "pri_x", "pri_x"], {"hex": 2, "pri": 2})])
def test_mixed_mesh_residual(ctx, kinds, degs):
    from inputs import meshes
    from oracle import mesh as omesh
    from oracle import physics as ophx
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh(kinds, (3, 2, 3), [0, 0, 0], [1, 1, 1])
    M = sdrt.Mesh(ctx, mesh, degs, sdrt.make_physics("euler", 3, "rusanov", "fp64"))
    geom = omesh.build(mesh, degs)
    oph = ophx.Physics("euler", 3, "rusanov")
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 14, 0.02)
    linf, _ = gu.rel_errors(_gpu_residual(M, U), ores.residual(geom, oph, U))
    assert linf < TOL64, linf


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rk4_steps(ctx, precision):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 3, "euler", "rusanov", precision)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 15, 0.01)
    dt = 2e-3
    want = U
    for _ in range(3):
        want = ores.rk4_step(geom, oph, want, dt)
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    M.rk4_step(Ud, dt, 3)
    M.sync()
    got = M.unpack(Ud.cpu().numpy())
    # compare the change over the steps (the state itself is O(1))
    d_got = [g - u for g, u in zip(got, U)]
    d_want = [w - u for w, u in zip(want, U)]
    linf, l2 = gu.rel_errors(d_got, d_want)
    assert linf < (1e-9 if precision == "fp64" else 5e-3), linf


def test_rk4_host_entry_point_matches_device(ctx):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 2, "euler", "rusanov", "fp32")
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 16, 0.01)
    host = M.pack(U)
    out = np.zeros_like(host)
    M.rk4_step_host(host, out, 1e-3, 2)
    Ud = torch.from_numpy(host).to("cuda")
    M.rk4_step(Ud, 1e-3, 2)
    M.sync()
    assert np.array_equal(out, Ud.cpu().numpy())


@pytest.mark.parametrize("kind,p,system", [("tet", 3, "euler"), ("tet", 4, "euler"), ("pri", 2, "euler"),
                                           ("hex", 2, "euler"), ("tet", 4, "advection")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_jvp(ctx, kind, p, system, precision):
    riem = "rusanov" if system == "euler" else "upwind"
    M, geom, oph, _ = gu.build_pair(ctx, kind, (3, 3, 2), p, system, riem, precision)
    rng = np.random.default_rng(17)
    if system == "euler":
        U = gu.oracle_state(geom, gu.smooth_gas, 5)
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
    linf, l2 = gu.rel_errors(M.unpack(JV.cpu().numpy()), want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_free_stream_and_conservation_on_gpu(ctx, precision):
    from tests import quadrature
    from oracle import operators
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (4, 3, 3), 3, "euler", "rusanov", precision)
    const = [np.tile(np.array([1.2, 0.3, -0.2, 0.1, 3.0])[None, :, None], (g.ops.n_sol, 1, g.nelem))
             for g in geom.blocks]
    R = _gpu_residual(M, const)
    fmag = 3.0 / 0.25
    assert max(np.abs(r).max() for r in R) < (1e-9 if precision == "fp64" else 2e-5) * fmag
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 18, 0.05)
    R = _gpu_residual(M, U)
    tot = 0.0
    for g, r in zip(geom.blocks, R):
        Xq, Wq = quadrature.rule(g.shape, 10)
        w = Wq @ operators.nodal_sol(g.shape, g.p, g.ops.xs, Xq)
        tot = tot + np.einsum("s,sve,e->v", w, r.astype(np.float64), g.detJ)
    scale = max(np.abs(r).max() for r in R) * sum(g.detJ.sum() for g in geom.blocks)
    assert np.abs(tot).max() < (1e-12 if precision == "fp64" else 1e-5) * scale


def test_nonfinite_flag(ctx):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 1, "euler", "rusanov", "fp32")
    U = gu.oracle_state(geom, gu.smooth_gas, 5)
    U[0][:, 0, 3] = -1.0          # negative density: the sound speed becomes NaN
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    R = torch.zeros_like(Ud)
    M.residual(Ud, R)
    with pytest.raises(sdrt.SdrtError) as ei:
        M.sync()
    assert ei.value.code == -5
    M.sync()                      # the flag was cleared


def test_face_map_matches_oracle_on_device_context(ctx):
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 2, 2), 3, "euler", "rusanov", "fp32")
    part, left = M.face_map()
    assert np.array_equal(part.astype(np.int64), geom.partner)
    assert np.array_equal(left.astype(bool), geom.is_left)


def test_wait_timeout_reported_and_results_intact(ctx):
    """A bounded device wait that runs out is reported as SDRT_ERR_TIMEOUT by
    sdrt_sync (SDRT_OPT_WAIT_POLLS makes the record flux kernel's first copy
    wait a single non-blocking check); the kernel then waits for its own
    copies with the normal bound, so the residual is still the right one, and
    with the option reset the next call reports nothing."""
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 3, "euler", "rusanov", "fp32")
    assert sdrt.PATHS[sdrt.sdrt_get_mesh_info(ctx.ptr, M.id)["path"]] == "record"
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 19, 0.02)
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    R1, R2 = torch.zeros_like(Ud), torch.zeros_like(Ud)
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_WAIT_POLLS, 1)
    try:
        M.residual(Ud, R1)
        with pytest.raises(sdrt.SdrtError) as ei:
            M.sync()
        assert ei.value.code == -6
    finally:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_WAIT_POLLS, 0)
    M.residual(Ud, R2)
    M.sync()
    assert torch.equal(R1, R2)
    linf, l2 = gu.rel_errors(M.unpack(R2.cpu().numpy()), ores.residual(geom, oph, U))
    assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)
