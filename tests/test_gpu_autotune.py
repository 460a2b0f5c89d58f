"""Tile autotuner of the generic kernels: the chosen tiles are valid, the
residual is bit-for-bit unchanged (tiles only partition the elements), and
the RK4 graph re-captured afterwards gives the same steps."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _batch():
    from inputs import meshes
    a = meshes.box_mesh(["hex", "pri_x", "hex"], (4, 3, 3), [0, 0, 0], [1, 1, 1])
    b = meshes.box_mesh(["tet", "pri", "pri"], (3, 3, 3), [0, 0, 0], [1, 1, 1])
    m = meshes.merge_meshes([a, b])
    degs = [2] * len(a["blocks"]) + [3] * len(b["blocks"])
    return m, degs


@pytest.mark.parametrize("system", ["euler", "ns"])
def test_autotune_keeps_results_and_picks_valid_tiles(ctx, system):
    from oracle import mesh as omesh
    from paper_2105_08632_gb300 import sdrt
    mesh, degs = _batch()
    kw = {"mu": 0.02} if system == "ns" else {}
    M = sdrt.Mesh(ctx, mesh, degs, sdrt.make_physics(system, 3, "rusanov", "fp32", **kw))
    geom = omesh.build(mesh, degs)
    U = torch.from_numpy(M.pack(gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 51, 0.02))).cuda()
    R0, R1 = torch.zeros_like(U), torch.zeros_like(U)
    M.residual(U, R0)
    V0 = U.clone()
    M.rk4_step(V0, 1e-3, 2)
    M.sync()
    before = M.tiles()
    M.autotune(U, reps=2)
    after = M.tiles()
    M.residual(U, R1)
    V1 = U.clone()
    M.rk4_step(V1, 1e-3, 2)
    M.sync()
    assert torch.equal(R0, R1)
    assert torch.equal(V0, V1)
    for t0, t1 in zip(before, after):
        assert t1["residual"] in (4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64)
        if system == "ns":
            assert t1["gradient"] in (4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64)
        assert t1["residual_jvp"] == t0["residual_jvp"]


def test_autotune_is_a_no_op_on_the_record_path(ctx):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (3, 3, 2), 3, "euler", "rusanov", "fp32")
    U = torch.from_numpy(M.pack(gu.oracle_state(geom, gu.smooth_gas, 5))).cuda()
    before = M.tiles()
    M.autotune(U)
    assert M.tiles() == before
