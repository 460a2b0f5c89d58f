"""Partitions of a mesh for a distributed residual, host side (no GPU): the
partition plans (owned and ghost elements, faces, exchange lists), their
set-up in a host-only library context, the error codes, and the exchange of
packed face records between two processes with torch.distributed (gloo),
each record tagged with the (global element, face) it carries."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from inputs import meshes  # noqa: E402

sdrt = pytest.importorskip("paper_2105_08632_gb300.sdrt")
from paper_2105_08632_gb300 import partition as pt  # noqa: E402


def _owners(mesh, scheme, nparts):
    n = sum(len(b["verts"]) for b in mesh["blocks"])
    if scheme == "slabs":                        # contiguous runs of elements: z slabs of the box
        return (np.arange(n) * nparts) // n
    return np.random.default_rng(5).integers(0, nparts, n)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(sdrt.LIB_PATH):
        from paper_2105_08632_gb300 import build
        build.build()
    return sdrt.lib()


@pytest.mark.parametrize("kinds,scheme,nparts", [("tet", "slabs", 3), ("tet", "random", 4),
                                                 (["tet", "pri", "tet"], "random", 3), (["hex", "pri_x"], "slabs", 2)])
def test_plan_invariants(kinds, scheme, nparts):
    n = (3, 3, 3) if isinstance(kinds, str) else (3, 2, len(kinds))
    mesh = meshes.box_mesh(kinds, n, [0.0] * 3, [1.0] * 3)
    owner = _owners(mesh, scheme, nparts)
    plans = pt.split(mesh, owner, nparts)
    nglob = len(owner)
    seen = np.zeros(nglob, int)
    faces = np.asarray(mesh["faces"]).reshape(-1, 6)
    off = pt.global_offsets(mesh)
    gl = off[faces[:, 0]] + faces[:, 1]
    gr = off[faces[:, 3]] + faces[:, 4]
    for p, pl in enumerate(plans):
        for b, ids in pl["owned"]:
            seen[ids] += 1
            assert (owner[ids] == p).all()
        for b, ids in pl["ghosts"]:
            assert (owner[ids] != p).all()
        # owned blocks first, then ghosts
        g = pl["ghost"]
        assert (np.diff(g.astype(int)) >= 0).all() and g[0] == 0
        # the partition's faces are the global faces touching its elements, L / R order kept
        touch = (owner[gl] == p) | (owner[gr] == p)
        assert len(pl["mesh"]["faces"]) == int(touch.sum())
        inv = {v: k for k, v in pl["local"].items()}
        for row, fi in zip(pl["mesh"]["faces"], np.nonzero(touch)[0]):
            assert inv[(row[0], row[1])] == gl[fi] and inv[(row[3], row[4])] == gr[fi]
            assert row[2] == faces[fi, 2] and row[5] == faces[fi, 5]
        # exchange lists agree pairwise and name ghost faces glued to owned elements
        for q, keys in pl["keys_recv"].items():
            assert np.array_equal(keys, plans[q]["keys_send"][p])
            assert (owner[keys[:, 0]] == q).all()
            for (G, f), (b, e, f2) in zip(keys, pl["recv"][q]):
                assert g[b] == 1 and inv[(b, e)] == G and f2 == f
            for (G, f), (b, e, f2) in zip(keys, plans[q]["send"][p]):
                assert plans[q]["ghost"][b] == 0 and {v: k for k, v in plans[q]["local"].items()}[(b, e)] == G
        # every face between p and another partition appears once in p's receive keys
        cross = set()
        for fi in range(len(faces)):
            for G, f, H in ((gl[fi], faces[fi, 2], gr[fi]), (gr[fi], faces[fi, 5], gl[fi])):
                if owner[H] == p and owner[G] != p:
                    cross.add((int(G), int(f)))
        got = {tuple(k) for keys in pl["keys_recv"].values() for k in keys.tolist()}
        assert got == cross
    assert (seen == 1).all()


def test_partition_setup_in_host_context(lib):
    mesh = meshes.box_mesh("tet", (3, 3, 3), [0.0] * 3, [1.0] * 3)
    owner = _owners(mesh, "random", 3)
    plans = pt.split(mesh, owner, 3)
    ctx = sdrt.Context(-1)
    try:
        phys = sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4)
        total = 0
        for pl in plans:
            pm = pt.PartitionMesh(ctx, pl, 3, phys)
            nown = sum(len(ids) for _, ids in pl["owned"])
            total += nown
            assert pm.info["ndof"] == 20 * 5 * nown
            assert pm.info["nblocks"] == len(pl["owned"])
            assert pm.state_len == sum(20 * 5 * ((len(ids) + 31) // 32 * 32) for _, ids in pl["owned"])
            x = pm.xinfo
            assert x["nsend"] == sum(len(a) for a in pl["send"].values())
            assert x["nrecv"] == sum(len(a) for a in pl["recv"].values())
            assert x["face_record"] == 52                     # 10 points x 5 variables, padded to 4
            with pytest.raises(sdrt.SdrtError):                # no device work in a host-only context
                pm.residual_begin(1)                           # (a raw pointer reaches the library)
        assert total == len(owner)
    finally:
        ctx.close()


def test_partition_errors(lib):
    ctx = sdrt.sdrt_create(-1)
    try:
        mesh = meshes.box_mesh("tet", (2, 2, 2), [0.0] * 3, [1.0] * 3)
        pl = pt.split(mesh, _owners(mesh, "slabs", 2), 2)[0]
        phys = sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4)
        et = sdrt.sdrt_setup_element_type(ctx, "tet", 3)
        blocks = [(et, b["verts"]) for b in pl["mesh"]["blocks"]]
        faces = (pl["mesh"]["faces"], pl["mesh"]["shift"])
        with pytest.raises(sdrt.SdrtError):                    # ghost block before an owned one
            sdrt.sdrt_setup_partition(ctx, phys, blocks[::-1], pl["ghost"][::-1].copy(), faces)
        mid = sdrt.sdrt_setup_partition(ctx, phys, blocks, pl["ghost"], faces)
        with pytest.raises(sdrt.SdrtError):                    # a ghost face in the send list
            sdrt.sdrt_set_exchange(ctx, mid, pt.concat(pl["recv"]), pt.concat(pl["recv"]))
        with pytest.raises(sdrt.SdrtError):                    # element out of range
            sdrt.sdrt_set_exchange(ctx, mid, np.array([[0, 10 ** 6, 0]]), np.zeros((0, 3)))
        with pytest.raises(sdrt.SdrtError):                    # unglued face on an owned element
            sdrt.sdrt_setup_partition(ctx, phys, blocks, pl["ghost"],
                                      (pl["mesh"]["faces"][1:], pl["mesh"]["shift"][1:]))
        # mismatched ghost flags (one per block)
        with pytest.raises(ValueError):
            sdrt.sdrt_setup_partition(ctx, phys, blocks, pl["ghost"][:-1].copy(), faces)
    finally:
        sdrt.sdrt_destroy(ctx)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tag(keys, fr):
    """Record values carrying (G, f): value k of the record of (G, f) is (8 G + f) * 64 + k."""
    k = np.arange(fr)
    return ((8 * keys[:, 0:1] + keys[:, 1:2]) * 64 + k[None, :]).astype(np.float64)


def _exchange_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh = meshes.box_mesh("tet", (3, 3, 4), [0.0] * 3, [1.0] * 3)
        n = sum(len(b["verts"]) for b in mesh["blocks"])
        owner = np.random.default_rng(11).integers(0, world, n)
        plan = pt.split(mesh, owner, world)[rank]
        fr = 52
        send = {q: torch.from_numpy(_tag(k, fr).reshape(-1)) for q, k in plan["keys_send"].items()}
        recv = {q: torch.zeros(len(k) * fr, dtype=torch.float64) for q, k in plan["keys_recv"].items()}
        pt.exchange(send, recv)
        ok = all(np.array_equal(recv[q].numpy(), _tag(k, fr).reshape(-1)) for q, k in plan["keys_recv"].items())
        nrec = sum(len(k) for k in plan["keys_recv"].values())
        gathered = [None] * world
        dist.all_gather_object(gathered, (ok, nrec))
        if rank == 0:
            out.put(gathered)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_face_record_exchange_between_two_processes():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for ok, _ in res), res
    assert all(n > 0 for _, n in res)


@pytest.mark.parametrize("kinds,p,scheme,nparts", [("tet", 3, "slabs", 2), ("tet", 3, "random", 3),
                                                   (["tet", "pri"], 2, "random", 3), ("hex", 2, "random", 2)])
def test_partition_face_maps_match_the_whole_mesh(lib, kinds, p, scheme, nparts):
    """The face pairing of every partition (owned points glued to owned or ghost
    points), mapped back to global (element, point) ids, is the whole mesh's
    face map bit for bit, L / R sides included (record and generic paths)."""
    mesh = meshes.box_mesh(kinds, (3, 3, 2), [0.0] * 3, [1.0] * 3)
    owner = _owners(mesh, scheme, nparts)
    plans = pt.split(mesh, owner, nparts)
    off = pt.global_offsets(mesh)
    ctx = sdrt.Context(-1)
    try:
        phys = sdrt.make_physics("euler", 3, "rusanov", "fp64", gamma=1.4)
        W = sdrt.Mesh(ctx, mesh, p, phys)
        wpart, wleft = W.face_map()
        nfe_of = [l["nfe"] for l in W.layouts]
        wbase = np.concatenate([[0], np.cumsum([len(b["verts"]) * n for b, n in zip(mesh["blocks"], nfe_of)])])

        def wcanon(G, s):                      # global element, local point -> whole-mesh canonical index
            b = int(np.searchsorted(off, G, side="right") - 1)
            return int(wbase[b] + (G - off[b]) * nfe_of[b] + s)

        for pl in plans:
            pm = pt.PartitionMesh(ctx, pl, p, phys)
            part, left = pm.face_map()
            blocks = pl["owned"] + pl["ghosts"]
            nfe_l = [nfe_of[b] for b, _ in blocks]
            base = np.concatenate([[0], np.cumsum([len(ids) * n for (_, ids), n in zip(blocks, nfe_l)])])
            for lb in range(len(pl["owned"])):
                ids = blocks[lb][1]
                for e, G in enumerate(ids):
                    for s in range(nfe_l[lb]):
                        g = int(base[lb] + e * nfe_l[lb] + s)
                        q = int(part[g])
                        qb = int(np.searchsorted(base, q, side="right") - 1)
                        qe, qs = divmod(q - int(base[qb]), nfe_l[qb])
                        assert wcanon(int(blocks[qb][1][qe]), qs) == int(wpart[wcanon(int(G), s)])
                        assert left[g] == wleft[wcanon(int(G), s)]
    finally:
        ctx.close()


@pytest.mark.parametrize("kinds,p,frec", [(["tet", "pri"], 2, 48), ("hex", 2, 48), ("tet", 2, 32)])
def test_generic_partition_setup_in_host_context(lib, kinds, p, frec):
    """Partitions on the generic path (any element type): face records of the
    largest face's points x nvar, padded to 4 (prisms: 9-point quadrilateral and
    6-point triangular faces at p = 2)."""
    n = (2, 2, 2)
    mesh = meshes.box_mesh(kinds if isinstance(kinds, str) else kinds, n, [0.0] * 3, [1.0] * 3)
    owner = _owners(mesh, "random", 3)
    plans = pt.split(mesh, owner, 3)
    ctx = sdrt.Context(-1)
    try:
        phys = sdrt.make_physics("euler", 3, "rusanov", "fp64", gamma=1.4)
        for pl in plans:
            pm = pt.PartitionMesh(ctx, pl, p, phys)
            assert pm.xinfo["face_record"] == frec
            assert pm.xinfo["nsend"] == sum(len(a) for a in pl["send"].values())
    finally:
        ctx.close()


@pytest.mark.parametrize("kinds,n,system,p,frec,grec", [("tet", (3, 3, 3), "ns", 2, 32, 92),
                                                        ("hex", (2, 2, 3), "ns", 2, 48, 136),
                                                        ("quad", (4, 4), "advdiff", 3, 4, 8)])
def test_viscous_partition_records(lib, kinds, n, system, p, frec, grec):
    """Viscous partitions exchange face states and then the face points'
    gradients: records of (points per face) x nvar and x ndim x nvar values."""
    nd = len(n)
    mesh = meshes.box_mesh(kinds, n, [0.0] * nd, [1.0] * nd)
    plans = pt.split(mesh, _owners(mesh, "random", 3), 3)
    kw = {"gamma": 1.4, "mu": 0.02} if system == "ns" else {"a": (1.0, 0.5, 0.25)[:nd], "mu": 0.05}
    phys = sdrt.make_physics(system, nd, "rusanov" if system == "ns" else "upwind", "fp64", **kw)
    ctx = sdrt.Context(-1)
    try:
        for pl in plans:
            pm = pt.PartitionMesh(ctx, pl, p, phys)
            assert pm.viscous and pm.xinfo["face_record"] == frec and pm.xinfo["grad_record"] == grec
    finally:
        ctx.close()


def test_single_partition_has_no_exchange(lib):
    mesh = meshes.box_mesh("tet", (2, 2, 2), [0.0] * 3, [1.0] * 3)
    plans = pt.split(mesh, np.zeros(48, int), 1)
    pl = plans[0]
    assert not pl["recv"] and not pl["send"] and not pl["ghosts"]
    assert len(pl["mesh"]["faces"]) == len(mesh["faces"])
    ctx = sdrt.Context(-1)
    try:
        pm = pt.PartitionMesh(ctx, pl, 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
        assert pm.xinfo["nsend"] == 0 and pm.xinfo["nrecv"] == 0
        W = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
        assert pm.state_len == W.state_len
    finally:
        ctx.close()


def test_split_rejects_bad_owners():
    mesh = meshes.box_mesh("tet", (2, 2, 2), [0.0] * 3, [1.0] * 3)
    with pytest.raises(ValueError):
        pt.split(mesh, np.zeros(47, int))
    with pytest.raises(ValueError):
        pt.split(mesh, np.full(48, 3), 2)


@pytest.mark.parametrize("kinds,p", [("tet", 3), (["tet", "pri"], 2)])
def test_partition_solution_points_are_the_owned_elements(lib, kinds, p):
    mesh = meshes.box_mesh(kinds, (3, 2, 2), [0.0] * 3, [1.0] * 3)
    plans = pt.split(mesh, _owners(mesh, "random", 3), 3)
    ctx = sdrt.Context(-1)
    try:
        phys = sdrt.make_physics("euler", 3, "rusanov", "fp64", gamma=1.4)
        W = sdrt.Mesh(ctx, mesh, p, phys)
        wx = W.sol_points()
        off = pt.global_offsets(mesh)
        for pl in plans:
            pm = pt.PartitionMesh(ctx, pl, p, phys)
            for (b, ids), x in zip(pl["owned"], pm.sol_points()):
                np.testing.assert_array_equal(x, wx[b][ids - off[b]])
    finally:
        ctx.close()


@pytest.mark.parametrize("kinds,n,nparts", [("tet", (4, 4, 4), 4), ("tet", (4, 4, 4), 3), (["tet", "pri"], (3, 3, 2), 5)])
def test_bisection_owners_balance_and_cut(kinds, n, nparts):
    """Recursive coordinate bisection: every partition within one element of the
    mean size, and fewer exchanged faces than a random assignment (planar cuts)."""
    mesh = meshes.box_mesh(kinds, n, [0.0] * 3, [1.0] * 3)
    owner = pt.bisection_owners(mesh, nparts)
    counts = np.bincount(owner, minlength=nparts)
    assert counts.min() > 0 and counts.max() - counts.min() <= 1
    def cut_faces(own):
        return sum(len(k) for pl in pt.split(mesh, own, nparts) for k in pl["keys_recv"].values())
    rnd = np.random.default_rng(1).integers(0, nparts, len(owner))
    assert cut_faces(owner) < 0.5 * cut_faces(rnd)
    assert np.array_equal(owner, pt.bisection_owners(mesh, nparts))     # deterministic


@pytest.mark.parametrize("nparts", [2, 5, 8])
def test_bisection_owners_skewed_weights_leave_no_partition_empty(nparts):
    """One element carrying almost all the weight: the weighted quantile alone
    would put every other element on one side; the cut keeps at least one
    element per partition on each side, and every element has an owner."""
    mesh = meshes.box_mesh("tet", (2, 2, 1), [0.0] * 3, [1.0] * 3)       # 24 elements
    n = sum(len(b["verts"]) for b in mesh["blocks"])
    for heavy in (0, n // 2, n - 1):
        w = np.ones(n)
        w[heavy] = 1e6
        owner = pt.bisection_owners(mesh, nparts, weights=w)
        counts = np.bincount(owner, minlength=nparts)
        assert len(counts) == nparts and counts.min() >= 1, counts
        plans = pt.split(mesh, owner, nparts)                            # plans build for every partition
        assert sum(len(ids) for pl in plans for _, ids in pl["owned"]) == n
    # exactly as many elements as parts: one element each
    owner = pt.bisection_owners(mesh, n, weights=np.arange(1.0, n + 1) ** 4)
    assert sorted(owner.tolist()) == list(range(n))


class _FakePart:
    """A partition of a 1D periodic upwind operator (du_i/dt = u_{i-1} - u_i)
    with the interface of PartitionMesh used by rk4_step_distributed: each rank
    owns a contiguous half and receives its left neighbour's last value."""

    def __init__(self, rank, world, n):
        self.rank, self.world, self.n = rank, world, n
        self.viscous = False
        self.left, self.right = (rank - 1) % world, (rank + 1) % world
        self.send_seg = {self.right: (0, 1)}
        self.recv_seg = {self.left: (0, 1)}
        self.send_buf = torch.zeros(1, dtype=torch.float64)
        self.recv_buf = torch.zeros(1, dtype=torch.float64)
        self.X = None

    def residual_begin(self, X):
        self.X = X
        self.send_buf[0] = X[-1]

    def residual_end(self, R):
        up = torch.cat([self.recv_buf, self.X[:-1]])
        R.copy_(up - self.X)

    def send_view(self, q, grad=False):
        return self.send_buf

    def recv_view(self, q, grad=False):
        return self.recv_buf


def _rk4_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 8
        x = np.arange(world * n)
        u = np.sin(2 * np.pi * x / (world * n))
        part = _FakePart(rank, world, n)
        U = torch.from_numpy(u[rank * n:(rank + 1) * n].copy())
        for _ in range(3):
            pt.rk4_step_distributed(part, U, 0.1)
        got = [None] * world
        dist.all_gather_object(got, U.numpy().tolist())
        if rank == 0:
            out.put(np.concatenate(got))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_distributed_rk4_orchestration_with_gloo():
    """rk4_step_distributed: one exchange per stage, stage combinations of
    classical RK4 -- two gloo processes give the serial RK4 of the whole array."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rk4_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u = np.sin(2 * np.pi * np.arange(16) / 16)
    f = lambda v: np.roll(v, 1) - v
    for _ in range(3):
        k1 = f(u)
        k2 = f(u + 0.05 * k1)
        k3 = f(u + 0.05 * k2)
        k4 = f(u + 0.1 * k3)
        u = u + 0.1 / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    np.testing.assert_allclose(got, u, rtol=0, atol=1e-14)
