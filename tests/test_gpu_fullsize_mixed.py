"""The batched mixed-element benchmark workload at full size (four periodic
meshes, hexahedra / prisms / tetrahedra of degrees 1-4, 489,664 elements),
FP32, on the kernels and launch configuration the benchmark times (the
operator-specialised path):

* the smallest of the four independent meshes (tetrahedra and prisms of
  degree 4) against the oracle, element by element, within the FP32
  forward-error scale 128 u S (u = 2^-24, S = the magnitudes of the
  divergence's terms, computed by the oracle);
* properties that hold at any size on the whole batch: a uniform state has a
  zero residual up to FP32 rounding of its flux terms (affine elements,
  Sec. 2), bounded per block by 128 u S with S the largest over the elements
  of a small box of the same cells, computed by the oracle (in a uniform box
  the elements of a cell differ only by orientation); discrete conservation
  of every variable over every mesh (Sec. 2.1) within 4 u times the sum of
  the flux terms' scale (the FP32-rounded operator entries).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import meshes  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from oracle import operators  # noqa: E402
from oracle import physics as ophx  # noqa: E402
from oracle import residual as ores  # noqa: E402
from tests import gpu_util as gu  # noqa: E402
from tests import quadrature  # noqa: E402

STATE = np.array([1.2, 0.3, -0.2, 0.1, 3.0])


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    ctx = sdrt.Context(0)
    spec = bench.Workload("mixed")
    M = sdrt.Mesh(ctx, spec.mesh, list(spec.degrees), spec.physics(sdrt, "fp32"))
    assert spec.nelem == 489664
    assert sdrt.PATHS[M.info["path"]] == "generated"
    yield spec, M
    ctx.close()


def _residual(M, blocks):
    U = torch.from_numpy(M.pack(blocks)).to("cuda")
    R = torch.zeros_like(U)
    M.residual(U, R)
    M.sync()
    return M.unpack(R.cpu().numpy())


def _part_blocks(spec, k):
    b0 = sum(len(m["blocks"]) for m, _ in spec.parts[:k])
    return list(range(b0, b0 + len(spec.parts[k][0]["blocks"])))


def test_degree4_mesh_of_the_batch_matches_oracle(setup):
    spec, M = setup
    k = 3                                                   # tetrahedra / prisms of degree 4
    mesh_k, degs_k = spec.parts[k]
    geom = omesh.build(mesh_k, degs_k)
    blocks = _part_blocks(spec, k)
    sol = M.sol_points()
    U_all = spec.state(sol)
    for j, b in enumerate(blocks):
        np.testing.assert_allclose(sol[b], geom.blocks[j].xsol, atol=1e-12)
    R = _residual(M, U_all)
    U_k = [U_all[b].astype(np.float64) for b in blocks]
    want, scale = ores.residual(geom, ophx.Physics("euler", 3, "rusanov", gamma=1.4), U_k, terms=True)
    got = [R[b] for b in blocks]
    ratio = gu.fp32_bound_ratio(got, want, scale)
    assert ratio < 128, ratio


def _uniform_scale(kind, p, cell):
    """S of a uniform state, per shape the largest over the elements of a
    2 x 2 x 2 box of the same cells (dimensions `cell`) and degree p: an upper
    bound of every element's S in a uniform box of those cells (the elements
    of a cell differ only by orientation)."""
    m = meshes.box_mesh(kind, (2, 2, 2), [0.0] * 3, [2 * c for c in cell])
    geom = omesh.build(m, p)
    U = [np.repeat(STATE[None, :, None], g.nelem, 2).repeat(g.ops.n_sol, 0) for g in geom.blocks]
    _, S = ores.residual(geom, ophx.Physics("euler", 3, "rusanov", gamma=1.4), U, terms=True)
    return {g.shape: s.max(axis=2) for g, s in zip(geom.blocks, S)}       # (N_s, V) per shape


def test_uniform_state_and_conservation_at_full_size(setup):
    import bench
    spec, M = setup
    const = [np.tile(STATE.astype(np.float32)[None, :, None], (l["nsol"], 1, l["nelem"])) for l in M.layouts]
    R = _residual(M, const)
    checked = 0
    part_scales = []
    for k, (kind, p, nc, n1, n2) in enumerate(bench.MIXED_PARTS):
        cell = (10.0 / nc, 10.0 / nc, 10.0 / (n1 + n2))          # the part's box [-5, 5]^3 in (nc, nc, slabs) cells
        scales = _uniform_scale(kind, p, cell)
        scales.update(_uniform_scale("pri_x" if kind == "hex" else "pri", p, cell))
        part_scales.append(scales)
        for b in _part_blocks(spec, k):
            shape = spec.mesh["blocks"][b]["shape"]
            S = scales[shape][:, :, None]
            ratio = float(np.max(np.abs(R[b]) / (gu.U32 * S)))
            assert ratio < 128, (k, shape, ratio)
            checked += 1
    assert checked == len(spec.mesh["blocks"])
    # conservation: sum over each independent mesh of w_s det J dU/dt_s = 0.  In
    # FP32 the operators' entries are rounded (relative u each), so the sum is
    # off by a few u times the flux terms' magnitudes, not by u |dU/dt| (the
    # near free-stream state cancels its terms): the bound is 4 u sum |w_s| det J S
    # with S the terms' scale of the uniform state above (same magnitudes);
    # a face flux missing on one side would be off by whole flux terms.
    U = spec.state(M.sol_points())
    R = _residual(M, U)
    for k in range(len(bench.MIXED_PARTS)):
        tot = np.zeros(5)
        bound = np.zeros(5)
        for b in _part_blocks(spec, k):
            blk = spec.mesh["blocks"][b]
            shape, p = blk["shape"], spec.degrees[b]
            xs = operators.get(shape, p).xs
            Xq, Wq = quadrature.rule(shape, 10)
            w = Wq @ operators.nodal_sol(shape, p, xs, Xq)
            det = np.abs(np.linalg.det(0.5 * np.stack([blk["verts"][:, c] - blk["verts"][:, 0] for c in
                                                       {"tet": (1, 2, 3), "pri": (1, 2, 3),
                                                        "hex": (1, 3, 4)}[shape]], axis=2)))
            r = R[b].astype(np.float64)
            tot += np.einsum("s,sve,e->v", w, r, det)
            smax = part_scales[k][shape].max(axis=0)                 # (V,)
            bound += 4 * gu.U32 * np.abs(w).sum() * det.sum() * smax
        assert (np.abs(tot) < bound).all(), (k, tot, bound)
