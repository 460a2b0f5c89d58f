"""Host-side checks of libsdrt (no GPU needed): the library loads and exports
every entry point of include/sdrt.h; its FP64 operators (built from a
Legendre-product basis) equal the oracle's (monomial basis); its face maps
equal the oracle's bit for bit; bad arguments give error codes."""
import os
import re

import numpy as np
import pytest

from inputs import meshes
from oracle import mesh as omesh
from oracle import operators as oops

sdrt = pytest.importorskip("paper_2105_08632_gb300.sdrt")

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "sdrt.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(sdrt.LIB_PATH):
        from paper_2105_08632_gb300 import build
        build.build()
    return sdrt.lib()


@pytest.fixture(scope="module")
def hctx(lib):
    c = sdrt.sdrt_create(-1)
    yield c
    sdrt.sdrt_destroy(c)


def test_exports_every_declared_symbol(lib):
    text = open(HEADER).read()
    declared = set(re.findall(r"^\s*(?:int|void|int64_t|const char\*)\s+(sdrt_\w+)\s*\(", text, re.M))
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(sdrt.EXPORTED) | declared


CASES = [(s, p) for s in ("tri", "quad", "tet", "pri", "hex") for p in (1, 2, 3, 4)]


@pytest.mark.parametrize("shape,p", CASES)
def test_operators_match_oracle(hctx, shape, p):
    et = sdrt.sdrt_setup_element_type(hctx, shape, p)
    info = sdrt.sdrt_get_etype_info(hctx, et)
    ref = oops.get(shape, p)
    assert (info["nsol"], info["nfe"], info["nfi"], info["nfiu"]) == (ref.n_sol, ref.n_fe, ref.n_fi, ref.n_fiu)
    np.testing.assert_allclose(sdrt.sdrt_get_operator(hctx, et, "xs"), ref.xs, atol=1e-14)
    np.testing.assert_allclose(sdrt.sdrt_get_operator(hctx, et, "xfe"), ref.xfe, atol=1e-14)
    for name in ("M0", "M12", "M13", "M14", "M15", "M16"):
        got = sdrt.sdrt_get_operator(hctx, et, name)
        want = getattr(ref, name)
        tol = 1e-12 * max(1.0, np.abs(want).max()) * max(1.0, ref.cond_flux / 1e3)
        assert np.abs(got - want).max() < tol, (name, np.abs(got - want).max())


@pytest.mark.parametrize("shape,p", CASES)
def test_fr_scheme_operators(hctx, shape, p):
    """FR-SDRT element types (Sec. 2.3): internal DOFs (r, d) at the solution
    points, M12 = I, and a divergence operator equal to the oracle's FR form
    written out with its own differentiation matrices (from the Vandermonde
    derivatives):  M13_FR[s, (r, d)] = D_d[s, r] - sum_j M14[s, j] M0[j, r] n~_jd."""
    et = sdrt.sdrt_setup_element_type(hctx, shape, p, "fr")
    info = sdrt.sdrt_get_etype_info(hctx, et)
    ref = oops.get(shape, p)
    nd, ns = ref.nd, ref.n_sol
    assert (info["nsol"], info["nfe"], info["nfi"], info["nfiu"]) == (ns, ref.n_fe, nd * ns, ns)
    np.testing.assert_array_equal(sdrt.sdrt_get_operator(hctx, et, "M12"), np.eye(ns))
    want = np.zeros((ns, ns, nd))
    for d in range(nd):
        want[:, :, d] = ref.Dsol[d] - np.einsum("sj,jr,j->sr", ref.M14, ref.M0, ref.nrm_fe[:, d])
    got = sdrt.sdrt_get_operator(hctx, et, "M13")
    tol = 1e-11 * max(1.0, np.abs(want).max()) * max(1.0, ref.cond_flux / 1e3)
    assert np.abs(got - want.reshape(ns, ns * nd)).max() < tol
    # the viscous gradient operator M15 P M12 is SDRT's
    sd = sdrt.sdrt_setup_element_type(hctx, shape, p)
    def grad_op(e, nfi, fi_point):
        M15 = sdrt.sdrt_get_operator(hctx, e, "M15")
        M12 = sdrt.sdrt_get_operator(hctx, e, "M12")
        return M15 @ M12[fi_point]
    fr_pt = np.repeat(np.arange(ns), nd)
    np.testing.assert_allclose(grad_op(et, nd * ns, fr_pt), grad_op(sd, ref.n_fi, ref.fi_point), atol=tol)


MESHES = [("tri", (5, 3), 2), ("quad", (3, 4), 3), ("tet", (3, 2, 2), 3), ("pri", (2, 3, 2), 2),
          ("hex", (2, 2, 3), 2), ("tet", (2, 2, 2), 4)]


def _lib_mesh(ctx, mesh, p, system="euler", precision="fp64"):
    nd = mesh["blocks"][0]["verts"].shape[2]
    phys = sdrt.make_physics(system, nd, "rusanov" if system == "euler" else "upwind", precision)
    blocks = [(sdrt.sdrt_setup_element_type(ctx, b["shape"], p), b["verts"]) for b in mesh["blocks"]]
    mid = sdrt.sdrt_setup_mesh(ctx, phys, blocks, (mesh["faces"], mesh["shift"]))
    return mid


@pytest.mark.parametrize("kind,n,p", MESHES)
def test_face_map_bit_exact(hctx, kind, n, p):
    mesh = meshes.box_mesh(kind, n, [0.0] * len(n), [1.0] * len(n))
    mid = _lib_mesh(hctx, mesh, p)
    info = sdrt.sdrt_get_mesh_info(hctx, mid)
    part, left = sdrt.sdrt_get_face_map(hctx, mid, info["nfe_total"])
    geom = omesh.build(mesh, p)
    assert np.array_equal(part.astype(np.int64), geom.partner)
    assert np.array_equal(left.astype(bool), geom.is_left)


def test_mixed_mesh_face_map(hctx):
    """Tetrahedra glued to z-extruded prisms, prisms (x-extruded) glued to hexahedra."""
    for kinds, degs in ((["tet", "tet", "pri"], {"tet": 2, "pri": 2}),
                        (["hex", "pri_x", "pri_x"], {"hex": 2, "pri": 2})):
        mesh = meshes.box_mesh(kinds, (2, 2, 3), [0, 0, 0], [1, 1, 1])
        phys = sdrt.make_physics("euler", 3, "rusanov", "fp64")
        blocks = [(sdrt.sdrt_setup_element_type(hctx, b["shape"], degs[b["shape"]]), b["verts"])
                  for b in mesh["blocks"]]
        mid = sdrt.sdrt_setup_mesh(hctx, phys, blocks, (mesh["faces"], mesh["shift"]))
        info = sdrt.sdrt_get_mesh_info(hctx, mid)
        part, left = sdrt.sdrt_get_face_map(hctx, mid, info["nfe_total"])
        geom = omesh.build(mesh, degs)
        assert np.array_equal(part.astype(np.int64), geom.partner)
        assert np.array_equal(left.astype(bool), geom.is_left)


def test_sol_points_match_oracle(hctx):
    mesh = meshes.box_mesh("tet", (2, 3, 2), [-1.0, 0.0, 2.0], [1.0, 3.0, 3.0])
    mid = _lib_mesh(hctx, mesh, 3)
    info = sdrt.sdrt_get_mesh_info(hctx, mid)
    lay = sdrt.sdrt_get_block_layout(hctx, mid, 0)
    n = lay["nelem"] * lay["nsol"] * 3
    got = sdrt.sdrt_get_sol_points(hctx, mid, n).reshape(lay["nelem"], lay["nsol"], 3)
    geom = omesh.build(mesh, 3)
    np.testing.assert_allclose(got, geom.blocks[0].xsol, atol=1e-13)
    assert lay["ld"] % 32 == 0 and lay["ld"] >= lay["nelem"]
    assert info["ndof"] == lay["nelem"] * lay["nsol"] * 5


def test_error_codes(hctx):
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_element_type(hctx, 7, 2)
    assert ei.value.code == -1
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_get_mesh_info(hctx, 12345)
    assert ei.value.code == -1
    # a mesh with a missing face is rejected
    mesh = meshes.box_mesh("tet", (2, 2, 2), [0, 0, 0], [1, 1, 1])
    phys = sdrt.make_physics("euler", 3, "rusanov", "fp64")
    et = sdrt.sdrt_setup_element_type(hctx, "tet", 2)
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_mesh(hctx, phys, [(et, mesh["blocks"][0]["verts"])], (mesh["faces"][1:], mesh["shift"][1:]))
    assert ei.value.code == -7
    # mismatched faces (wrong local face index) are rejected
    bad = mesh["faces"].copy()
    bad[0, 2] = (bad[0, 2] + 1) % 4
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_mesh(hctx, phys, [(et, mesh["blocks"][0]["verts"])], (bad, mesh["shift"]))
    assert ei.value.code == -7
    # device computation is refused on a host-only context
    mid = sdrt.sdrt_setup_mesh(hctx, phys, [(et, mesh["blocks"][0]["verts"])], (mesh["faces"], mesh["shift"]))
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_residual(hctx, mid, 1, 2)
    assert ei.value.code == -4


def test_viscous_mesh_setup_on_host(hctx):
    """Advection-diffusion and Navier-Stokes meshes set up (host side); the
    Roe flux is refused for the scalar systems."""
    mesh = meshes.box_mesh("tet", (2, 2, 2), [0, 0, 0], [1, 1, 1])
    et = sdrt.sdrt_setup_element_type(hctx, "tet", 3)
    blocks = [(et, mesh["blocks"][0]["verts"])]
    faces = (mesh["faces"], mesh["shift"])
    for system, riem, nvar in (("ns", "roe", 5), ("ns", "rusanov", 5), ("advdiff", "upwind", 1)):
        phys = sdrt.make_physics(system, 3, riem, "fp32", mu=0.01)
        mid = sdrt.sdrt_setup_mesh(hctx, phys, blocks, faces)
        assert sdrt.sdrt_get_mesh_info(hctx, mid)["nvar"] == nvar
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_mesh(hctx, sdrt.make_physics("advdiff", 3, "roe", "fp32", mu=0.01), blocks, faces)
    assert ei.value.code == -1


@pytest.mark.parametrize("kind,n,p", [("tet", (2, 2, 2), 2), ("hex", (2, 2, 2), 2), ("pri", (2, 2, 2), 3),
                                      ("tri", (3, 3), 2), ("quad", (3, 2), 3)])
def test_curved_mesh_on_host(hctx, kind, n, p):
    """Curved elements (quadratic map): solution points at the oracle's mapped
    points, the oracle's face map bit for bit, the curved flag."""
    mesh = meshes.curved_mesh(meshes.box_mesh(kind, n, [0.0] * len(n), [1.0] * len(n)), 0.04, seed=7)
    nd = len(n)
    phys = sdrt.make_physics("euler", nd, "rusanov", "fp64")
    blocks = [(sdrt.sdrt_setup_element_type(hctx, b["shape"], p), b["verts"]) for b in mesh["blocks"]]
    mid = sdrt.sdrt_setup_mesh(hctx, phys, blocks, (mesh["faces"], mesh["shift"]),
                               nodes=[b["nodes"] for b in mesh["blocks"]])
    info = sdrt.sdrt_get_mesh_info(hctx, mid)
    assert info["curved"] == 1 and info["path"] == 0
    geom = omesh.build(mesh, p)
    part, left = sdrt.sdrt_get_face_map(hctx, mid, info["nfe_total"])
    assert np.array_equal(part.astype(np.int64), geom.partner)
    assert np.array_equal(left.astype(bool), geom.is_left)
    off = 0
    flat = sdrt.sdrt_get_sol_points(hctx, mid, sum(g.nelem * g.ops.n_sol * nd for g in geom.blocks))
    for g in geom.blocks:
        k = g.nelem * g.ops.n_sol * nd
        np.testing.assert_allclose(flat[off:off + k].reshape(g.xsol.shape), g.xsol, atol=1e-13)
        off += k
    # the straight mesh's info says affine
    m0 = meshes.box_mesh(kind, n, [0.0] * nd, [1.0] * nd)
    assert sdrt.sdrt_get_mesh_info(hctx, _lib_mesh(hctx, m0, p))["curved"] == 0


def test_curved_mesh_errors(hctx):
    mesh = meshes.curved_mesh(meshes.box_mesh("tet", (2, 2, 2), [0.0] * 3, [1.0] * 3), 0.04)
    phys = sdrt.make_physics("euler", 3, "rusanov", "fp64")
    et = sdrt.sdrt_setup_element_type(hctx, "tet", 2)
    X = mesh["blocks"][0]["nodes"]
    # an inverted element (two vertices swapped) is rejected
    bad = X.copy()
    bad[0, [0, 2]] = bad[0, [2, 0]]
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_mesh(hctx, phys, [(et, mesh["blocks"][0]["verts"])], (mesh["faces"], mesh["shift"]),
                             nodes=[bad])
    assert ei.value.code == -7
    # displaced hexahedron vertices given to the affine entry: not affine
    hm = meshes.curved_mesh(meshes.box_mesh("hex", (2, 2, 2), [0.0] * 3, [1.0] * 3), 0.04, seed=3)
    eh = sdrt.sdrt_setup_element_type(hctx, "hex", 2)
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_mesh(hctx, phys, [(eh, hm["blocks"][0]["verts"])], (hm["faces"], hm["shift"]))
    assert ei.value.code == -2
    # FR-SDRT on curved elements is refused
    efr = sdrt.sdrt_setup_element_type(hctx, "tet", 2, "fr")
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_mesh(hctx, phys, [(efr, mesh["blocks"][0]["verts"])], (mesh["faces"], mesh["shift"]),
                             nodes=[X])
    assert ei.value.code == -2


def test_tf32x3_precision_on_host(hctx):
    """SDRT_TF32X3 meshes hold FP32 states (state length and layout of an FP32
    mesh) and report their precision; other precision values are refused."""
    mesh = meshes.box_mesh("tet", (2, 2, 2), [0.0] * 3, [1.0] * 3)
    et = sdrt.sdrt_setup_element_type(hctx, "tet", 3)
    blocks = [(et, mesh["blocks"][0]["verts"])]
    infos = {}
    for prec in ("fp32", "tf32x3"):
        mid = sdrt.sdrt_setup_mesh(hctx, sdrt.make_physics("euler", 3, "rusanov", prec), blocks,
                                   (mesh["faces"], mesh["shift"]))
        infos[prec] = sdrt.sdrt_get_mesh_info(hctx, mid)
    assert infos["tf32x3"]["precision"] == 2 and infos["fp32"]["precision"] == 1
    assert infos["tf32x3"]["state_len"] == infos["fp32"]["state_len"]
    bad = sdrt.make_physics("euler", 3, "rusanov", "fp32")
    bad.precision = 3
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_setup_mesh(hctx, bad, blocks, (mesh["faces"], mesh["shift"]))
    assert ei.value.code == -1


def test_options_on_host_context(hctx):
    for opt, default in ((sdrt.SDRT_OPT_NVTX, 0), (sdrt.SDRT_OPT_WAIT_POLLS, 0), (sdrt.SDRT_OPT_GENERATED, 1)):
        sdrt.sdrt_set_option(hctx, opt, 1 - default)
        sdrt.sdrt_set_option(hctx, opt, default)
    with pytest.raises(sdrt.SdrtError) as ei:
        sdrt.sdrt_set_option(hctx, 99, 1)
    assert ei.value.code == -1
