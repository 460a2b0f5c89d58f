"""Partitioned residual on the GPU: the mesh split into virtual partitions
held by one process, each with ghost copies of its neighbours' elements; the
face records of the partition-boundary faces are packed, exchanged by device
copies and unpacked (sdrt_residual_begin / sdrt_residual_end).  Every owned
element's residual equals the whole-mesh residual bit for bit: the same
kernels on the same face states, element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import meshes  # noqa: E402
from tests import gpu_util as gu  # noqa: E402


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


def _owners(n, scheme, nparts):
    if scheme == "slabs":
        return (np.arange(n) * nparts) // n
    return np.random.default_rng(9).integers(0, nparts, n)


@pytest.mark.parametrize("kinds,n,system,precision,p,scheme,nparts", [
    # record path (tetrahedra of degree 3 / 4)
    ("tet", (4, 4, 3), "euler", "fp32", 3, "slabs", 3),
    ("tet", (4, 4, 3), "euler", "fp32", 3, "random", 4),
    ("tet", (4, 4, 3), "euler", "fp64", 3, "random", 3),
    ("tet", (4, 4, 3), "euler", "fp32", 4, "random", 2),
    ("tet", (4, 4, 3), "advection", "fp32", 3, "random", 3),
    ("tet", (4, 4, 3), "advection", "fp64", 4, "slabs", 2),
    # generic path: other degrees and element types, mixed meshes, 2D
    ("tet", (3, 3, 3), "euler", "fp32", 2, "random", 3),
    ("hex", (3, 3, 3), "euler", "fp64", 2, "random", 4),
    (["tet", "pri", "pri"], (3, 3, 3), "euler", "fp32", 2, "random", 3),
    ("tri", (6, 5), "advection", "fp64", 3, "random", 3),
    ("quad", (5, 4), "euler", "fp32", 3, "slabs", 2),
    # viscous systems: face states, then flux-point gradients exchanged
    ("tet", (3, 3, 3), "ns", "fp64", 2, "random", 3),
    ("hex", (3, 3, 3), "ns", "fp32", 2, "random", 3),
    ("tet", (3, 3, 3), "ns", "fp32", 3, "slabs", 2),
    ("quad", (5, 4), "advdiff", "fp64", 3, "random", 3),
])
def test_partitioned_residual_equals_whole_mesh(ctx, kinds, n, system, precision, p, scheme, nparts):
    from paper_2105_08632_gb300 import partition as pt
    from paper_2105_08632_gb300 import sdrt
    nd = len(n)
    mesh = meshes.box_mesh(kinds, n, [-1.0] * nd, [1.0] * nd)
    kw = {"euler": {"gamma": 1.4}, "ns": {"gamma": 1.4, "mu": 0.02, "beta": 0.5, "eta": 0.1},
          "advection": {"a": (1.0, 0.5, 0.25)[:nd]},
          "advdiff": {"a": (1.0, 0.5, 0.25)[:nd], "mu": 0.05, "beta": 0.3, "eta": 0.2}}[system]
    riemann = "rusanov" if system in ("euler", "ns") else "upwind"
    phys = sdrt.make_physics(system, nd, riemann, precision, **kw)
    M = sdrt.Mesh(ctx, mesh, p, phys)
    nv = M.nvar
    Ug = []
    for b, X in enumerate(M.sol_points()):
        if system in ("euler", "ns"):
            u = gu.smooth_gas(X.reshape(-1, nd)).reshape(X.shape[0], X.shape[1], nv)
        else:
            u = np.sin(2 * X[..., :1]) * np.cos(X[..., 1:2] + (0.5 * X[..., 2:3] if nd == 3 else 0.0))
        u = u * (1 + 0.01 * np.random.default_rng(3 + b).uniform(-1, 1, u.shape))
        Ug.append(np.ascontiguousarray(u.transpose(1, 2, 0)))
    dt = torch.float32 if precision == "fp32" else torch.float64
    U = torch.from_numpy(M.pack(Ug)).to("cuda")
    R = torch.zeros_like(U)
    # partitions run the generic or record kernels: the whole mesh too (not
    # the operator-specialised ones nor the tensor-core gradient chain), so
    # that the two agree bit for bit
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_GENERATED, 0)
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_GRADIENT, 0)
    try:
        M.residual(U, R)
        M.sync()
    finally:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_GENERATED, 1)
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_GRADIENT, 1)
    want = M.unpack(R.cpu().numpy())

    owner = _owners(sum(len(b["verts"]) for b in mesh["blocks"]), scheme, nparts)
    plans = pt.split(mesh, owner, nparts)
    parts = [pt.PartitionMesh(ctx, pl, p, phys) for pl in plans]
    Us = [torch.from_numpy(pm.pack(pt.scatter_state(pl, Ug))).to("cuda") for pm, pl in zip(parts, plans)]
    Rs = [torch.full_like(x, float("nan")) for x in Us]
    assert all(x.dtype == dt for x in Us)
    pt.residual_local(parts, Us, Rs)
    parts[0].sync()
    got = pt.gather_state(plans, [pm.unpack(r.cpu().numpy()) for pm, r in zip(parts, Rs)], want)
    assert sum(pm.xinfo["nrecv"] for pm in parts) > 0
    for g, w in zip(got, want):
        assert np.array_equal(g, w), float(np.abs(g - w).max())


def test_whole_mesh_calls_refuse_a_partition(ctx):
    from paper_2105_08632_gb300 import partition as pt
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh("tet", (2, 2, 2), [0.0] * 3, [1.0] * 3)
    plans = pt.split(mesh, _owners(48, "slabs", 2), 2)
    pm = pt.PartitionMesh(ctx, plans[0], 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
    U = torch.zeros(pm.state_len, dtype=torch.float32, device="cuda")
    R = torch.zeros_like(U)
    with pytest.raises(sdrt.SdrtError):
        pm.residual(U, R)
    with pytest.raises(sdrt.SdrtError):
        pm.rk4_step(U, 1e-3, 1)


@pytest.mark.parametrize("kinds,p,precision,tol", [("tet", 3, "fp64", 1e-13), ("hex", 2, "fp32", 1e-6)])
def test_partitioned_rk4_step(ctx, kinds, p, precision, tol):
    """Two RK4 steps of virtual partitions (four exchanges per step) against
    the whole mesh's RK4 steps: the same residuals; the stage combinations
    differ only in rounding (separate multiply-adds vs fused epilogue)."""
    from paper_2105_08632_gb300 import partition as pt
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh(kinds, (3, 3, 3), [-1.0] * 3, [1.0] * 3)
    phys = sdrt.make_physics("euler", 3, "rusanov", precision, gamma=1.4)
    M = sdrt.Mesh(ctx, mesh, p, phys)
    Ug = []
    for b, X in enumerate(M.sol_points()):
        u = gu.smooth_gas(X.reshape(-1, 3)).reshape(X.shape[0], X.shape[1], 5)
        Ug.append(np.ascontiguousarray(u.transpose(1, 2, 0)))
    U = torch.from_numpy(M.pack(Ug)).to("cuda")
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_GENERATED, 0)      # the partitions' kernels
    try:
        M.rk4_step(U, 1e-3, 2)
        M.sync()
    finally:
        sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_GENERATED, 1)
    want = M.unpack(U.cpu().numpy())
    owner = _owners(sum(len(b["verts"]) for b in mesh["blocks"]), "random", 3)
    plans = pt.split(mesh, owner, 3)
    parts = [pt.PartitionMesh(ctx, pl, p, phys) for pl in plans]
    Us = [torch.from_numpy(pm.pack(pt.scatter_state(pl, Ug))).to("cuda") for pm, pl in zip(parts, plans)]
    for _ in range(2):
        pt.rk4_step_local(parts, Us, 1e-3)
    parts[0].sync()
    got = pt.gather_state(plans, [pm.unpack(u.cpu().numpy()) for pm, u in zip(parts, Us)], want)
    for g, w in zip(got, want):
        assert np.abs(g - w).max() <= tol * np.abs(w).max(), float(np.abs(g - w).max())
