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


@pytest.mark.parametrize("system,precision,p,scheme,nparts", [
    ("euler", "fp32", 3, "slabs", 3),
    ("euler", "fp32", 3, "random", 4),
    ("euler", "fp64", 3, "random", 3),
    ("euler", "fp32", 4, "random", 2),
    ("advection", "fp32", 3, "random", 3),
    ("advection", "fp64", 4, "slabs", 2),
])
def test_partitioned_residual_equals_whole_mesh(ctx, system, precision, p, scheme, nparts):
    from paper_2105_08632_gb300 import partition as pt
    from paper_2105_08632_gb300 import sdrt
    mesh = meshes.box_mesh("tet", (4, 4, 3), [-1.0] * 3, [1.0] * 3)
    kw = {"gamma": 1.4} if system == "euler" else {"a": (1.0, 0.5, 0.25)}
    riemann = "rusanov" if system == "euler" else "upwind"
    phys = sdrt.make_physics(system, 3, riemann, precision, **kw)
    M = sdrt.Mesh(ctx, mesh, p, phys)
    X = M.sol_points()[0]
    nv = M.nvar
    if system == "euler":
        u = gu.smooth_gas(X.reshape(-1, 3)).reshape(X.shape[0], X.shape[1], nv)
    else:
        u = np.sin(2 * X[..., :1]) * np.cos(X[..., 1:2] + 0.5 * X[..., 2:3])
    u = u * (1 + 0.01 * np.random.default_rng(3).uniform(-1, 1, u.shape))
    Ug = [np.ascontiguousarray(u.transpose(1, 2, 0))]
    dt = torch.float32 if precision == "fp32" else torch.float64
    U = torch.from_numpy(M.pack(Ug)).to("cuda")
    R = torch.zeros_like(U)
    M.residual(U, R)
    M.sync()
    want = M.unpack(R.cpu().numpy())

    owner = _owners(len(X), scheme, nparts)
    plans = pt.split(mesh, owner, nparts)
    parts = [pt.PartitionMesh(ctx, pl, p, phys) for pl in plans]
    Us = [torch.from_numpy(pm.pack(pt.scatter_state(pl, Ug))).to("cuda") for pm, pl in zip(parts, plans)]
    Rs = [torch.full_like(x, float("nan")) for x in Us]
    assert all(x.dtype == dt for x in Us)
    pt.residual_local(parts, Us, Rs)
    parts[0].sync()
    got = pt.gather_state(plans, [pm.unpack(r.cpu().numpy()) for pm, r in zip(parts, Rs)], want)
    assert sum(pm.xinfo["nrecv"] for pm in parts) > 0
    assert np.array_equal(got[0], want[0]), float(np.abs(got[0] - want[0]).max())


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
