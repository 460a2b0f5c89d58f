"""Operator-specialised kernels (generated per element type at build time,
SDRT_OPT_GENERATED) against the FP64 oracle and against the generic kernels:

* the FP32 Euler / Rusanov residual of every generated element type (hexahedra
  of degree 1-3, prisms and tetrahedra of degree 1-4) on periodic meshes of
  several 32-element tiles with a ragged last tile, within the FP32
  tolerances of the parity tests (rel L-inf 2e-4, rel L2 2e-5 of max |R|);
* mixed tet/prism and hex/prism meshes (face records read across blocks,
  concurrent per-block branches), residual and RK4 steps;
* the batched configuration: four independent periodic meshes at degrees
  1, 2, 3 and 4 (hexahedra / x-extruded prisms and tetrahedra / z-extruded
  prisms) in one mesh, residual and two RK4 steps against the oracle in FP32
  (generated kernels) and FP64 (generic kernels, after autotuning their
  tiles);
* the generated and generic kernels agree to FP32 rounding; RK4 steps
  captured in a graph equal eagerly launched ones bit for bit.
"""
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
    stream = torch.cuda.Stream(0)
    torch.cuda.set_stream(stream)
    c = sdrt.Context(0, stream.cuda_stream)
    yield c
    c.close()


def _residual(M, U_blocks):
    dt = torch.float32 if M.dtype_np == np.float32 else torch.float64
    U = torch.from_numpy(M.pack(U_blocks)).to("cuda")
    R = torch.zeros(M.state_len, dtype=dt, device="cuda")
    M.residual(U, R)
    M.sync()
    return M.unpack(R.cpu().numpy())


def _path(ctx, M):
    from paper_2105_08632_gb300 import sdrt
    return sdrt.PATHS[sdrt.sdrt_get_mesh_info(ctx.ptr, M.id)["path"]]


# (kind, cells, degree): every generated element type, > 1 tile, ragged tail
GEN_CASES = [("hex", (4, 3, 3), 1), ("hex", (4, 3, 3), 2), ("hex", (4, 3, 3), 3),
             ("pri", (3, 3, 3), 1), ("pri", (3, 3, 3), 2), ("pri", (3, 3, 3), 3), ("pri", (3, 3, 2), 4),
             ("tet", (3, 3, 2), 1), ("tet", (3, 3, 2), 2)]


@pytest.mark.parametrize("kind,n,p", GEN_CASES)
def test_generated_residual_matches_oracle(ctx, kind, n, p):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "euler", "rusanov", "fp32")
    assert _path(ctx, M) == "generated"
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 61, 0.02)
    linf, l2 = gu.rel_errors(_residual(M, U), ores.residual(geom, oph, U))
    assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


def test_generated_degree4_tetrahedra_in_a_mixed_mesh(ctx):
    """Degree-4 (and 3) tetrahedra alone take the record path; next to prisms
    they take the generated kernels."""
    from inputs import meshes
    from oracle import mesh as omesh
    from oracle import physics as ophx
    from paper_2105_08632_gb300 import sdrt
    for p in (3, 4):
        mesh = meshes.box_mesh(["tet", "pri", "tet"], (3, 2, 3), [0, 0, 0], [1, 1, 1])
        M = sdrt.Mesh(ctx, mesh, p, sdrt.make_physics("euler", 3, "rusanov", "fp32"))
        assert _path(ctx, M) == "generated"
        geom = omesh.build(mesh, p)
        oph = ophx.Physics("euler", 3, "rusanov")
        U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 62 + p, 0.02)
        linf, l2 = gu.rel_errors(_residual(M, U), ores.residual(geom, oph, U))
        assert linf < TOL32[0] and l2 < TOL32[1], (p, linf, l2)


@pytest.mark.parametrize("kinds,degs", [(["tet", "tet", "pri"], {"tet": 3, "pri": 3}),
                                        (["hex", "pri_x", "pri_x"], {"hex": 2, "pri": 2}),
                                        (["pri_x", "hex", "pri_x", "hex"], {"hex": 1, "pri": 1})])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_mixed_mesh_residual(ctx, kinds, degs, precision):
    from inputs import meshes
    from oracle import mesh as omesh
    from oracle import physics as ophx
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh(kinds, (3, 2, len(kinds)), [0, 0, 0], [1, 1, 1])
    M = sdrt.Mesh(ctx, mesh, degs, sdrt.make_physics("euler", 3, "rusanov", precision))
    assert _path(ctx, M) == ("generated" if precision == "fp32" else "generic")
    geom = omesh.build(mesh, degs)
    oph = ophx.Physics("euler", 3, "rusanov")
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 64, 0.02)
    linf, l2 = gu.rel_errors(_residual(M, U), ores.residual(geom, oph, U))
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)


def _batched_mesh(scale=1):
    """Four independent periodic meshes, degrees 1..4 (the batched
    configuration's structure at a reduced size)."""
    from inputs import meshes
    parts = [meshes.box_mesh(["hex", "pri_x", "hex", "pri_x"], (4 * scale, 3, 4), [-5.0] * 3, [5.0] * 3),
             meshes.box_mesh(["tet", "pri", "tet"], (3, 2, 3), [-5.0] * 3, [5.0] * 3),
             meshes.box_mesh(["pri_x", "hex", "hex"], (3, 3, 3), [-5.0] * 3, [5.0] * 3),
             meshes.box_mesh(["pri", "tet"], (2, 2, 2), [-5.0] * 3, [5.0] * 3)]
    degs = []
    for part, p in zip(parts, (1, 2, 3, 4)):
        degs += [p] * len(part["blocks"])
    return meshes.merge_meshes(parts), degs


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_four_meshes_degrees_1_to_4(ctx, precision):
    from oracle import mesh as omesh
    from oracle import physics as ophx
    from paper_2105_08632_gb300 import sdrt
    mesh, degs = _batched_mesh()
    M = sdrt.Mesh(ctx, mesh, degs, sdrt.make_physics("euler", 3, "rusanov", precision))
    assert _path(ctx, M) == ("generated" if precision == "fp32" else "generic")
    geom = omesh.build(mesh, degs)
    oph = ophx.Physics("euler", 3, "rusanov")
    U = gu.perturb(gu.oracle_state(geom, lambda X: gu.smooth_gas(X / 10.0), 5), 65, 0.02)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    if precision == "fp64":
        tiles = {t["residual"] for t in M.tiles()}
        assert len(tiles) >= 2, tiles            # several tile widths across the blocks
    M.autotune(Ud, reps=1)
    R = torch.zeros(M.state_len, dtype=dtype, device="cuda")
    M.residual(Ud, R)
    M.sync()
    want = ores.residual(geom, oph, U)
    linf, l2 = gu.rel_errors(M.unpack(R.cpu().numpy()), want)
    if precision == "fp64":
        assert linf < TOL64, linf
    else:
        assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)
    dt = 1e-3
    W = U
    for _ in range(2):
        W = ores.rk4_step(geom, oph, W, dt)
    M.rk4_step(Ud, dt, 2)
    M.sync()
    got = M.unpack(Ud.cpu().numpy())
    d_got = [g - u for g, u in zip(got, U)]
    d_want = [w - u for w, u in zip(W, U)]
    linf, _ = gu.rel_errors(d_got, d_want)
    assert linf < (1e-9 if precision == "fp64" else 5e-3), linf


def test_generated_and_generic_kernels_agree(ctx):
    from paper_2105_08632_gb300 import sdrt
    mesh, degs = _batched_mesh()
    from oracle import mesh as omesh
    geom = omesh.build(mesh, degs)
    U = gu.perturb(gu.oracle_state(geom, lambda X: gu.smooth_gas(X / 10.0), 5), 66, 0.02)
    M = sdrt.Mesh(ctx, mesh, degs, sdrt.make_physics("euler", 3, "rusanov", "fp32"))
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    out = {}
    for gen in (1, 0):
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_GENERATED, gen)
        R = torch.zeros_like(Ud)
        M.residual(Ud, R)
        V = Ud.clone()
        M.rk4_step(V, 1e-3, 3)
        M.sync()
        out[gen] = (M.unpack(R.cpu().numpy()), M.unpack(V.cpu().numpy()))
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_GENERATED, 1)
    linf, l2 = gu.rel_errors(out[1][0], out[0][0])
    assert linf < TOL32[0] and l2 < TOL32[1], (linf, l2)
    linf, _ = gu.rel_errors([a - u for a, u in zip(out[1][1], U)], [b - u for b, u in zip(out[0][1], U)])
    assert linf < 1e-3, linf


def test_graph_steps_equal_eager_steps(ctx):
    """The first RK4 step of a mesh runs eagerly, later ones replay a captured
    graph with the per-block branches: both give the same bits."""
    from paper_2105_08632_gb300 import sdrt
    mesh, degs = _batched_mesh()
    from oracle import mesh as omesh
    geom = omesh.build(mesh, degs)
    U = gu.perturb(gu.oracle_state(geom, lambda X: gu.smooth_gas(X / 10.0), 5), 67, 0.02)
    phys = sdrt.make_physics("euler", 3, "rusanov", "fp32")
    A = sdrt.Mesh(ctx, mesh, degs, phys)
    B = sdrt.Mesh(ctx, mesh, degs, phys)
    Ua = torch.from_numpy(A.pack(U)).to("cuda")
    Ub = Ua.clone()
    A.rk4_step(Ua, 1e-3, 3)                     # eager, then two graph replays
    for _ in range(3):
        B.rk4_step(Ub, 1e-3, 1)                 # eager, then replays of its own graph
    A.sync()
    assert torch.equal(Ua, Ub)


def test_generated_nonfinite_flag(ctx):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "hex", (3, 2, 2), 2, "euler", "rusanov", "fp32")
    assert _path(ctx, M) == "generated"
    U = gu.oracle_state(geom, gu.smooth_gas, 5)
    U[0][:, 0, 5] = -1.0
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    R = torch.zeros_like(Ud)
    M.residual(Ud, R)
    with pytest.raises(sdrt.SdrtError) as ei:
        M.sync()
    assert ei.value.code == -5
    M.sync()
