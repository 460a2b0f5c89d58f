"""Partitions of a mesh for a distributed residual.

Elements couple only through the common flux at the faces they share (paper
Sec. 2.1), so a partition of the elements needs, once per residual
evaluation, the external-point states of its partition-boundary faces from
the partitions that own the elements on the other side -- one exchange step
of packed face records, then the usual flux and divergence kernels.

`split` is the host-side plan: every partition's mesh (its owned elements,
then ghost copies of the other partitions' elements that share a face with
them), and the exchange lists: partition p receives from q the face records
of the faces (G, f) -- G a global element owned by q glued to an element of
p, f its local face -- in ascending (G, f) order, and q sends them in the
same order.  `PartitionMesh` sets one partition up in a Context;
`residual_local` runs the residual of partitions held by one process (device
copies between the buffers), `exchange` moves the buffers between processes
with torch.distributed point-to-point calls (NCCL between GPUs, gloo on CPU).
"""
import numpy as np

from . import sdrt


def global_offsets(mesh):
    """First global element id of every block (blocks in order, elements in order)."""
    n = [len(b["verts"]) for b in mesh["blocks"]]
    return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)


def bisection_owners(mesh, nparts, weights=None):
    """Owner array by recursive coordinate bisection of the element centroids:
    each step cuts the element set across its longest centroid extent, at the
    weighted quantile that gives the two sides parts in proportion to the
    partitions they will hold (weights: work per element, e.g. nsol x nvar per
    block; default 1).  Balanced to one element's weight for equal weights;
    the cuts are planes, so the exchanged faces are those of ~nparts^(1/d)
    planes across the box.  With at least nparts elements no partition is
    empty, however skewed the weights."""
    cents = np.concatenate([np.asarray(b["verts"], float).mean(axis=1) for b in mesh["blocks"]])
    n = len(cents)
    w = np.ones(n) if weights is None else np.asarray(weights, float)
    owner = np.zeros(n, np.int64)

    def cut(idx, first, count):
        if count == 1 or len(idx) == 0:
            owner[idx] = first
            return
        left = count // 2
        c = cents[idx]
        axis = int(np.argmax(c.max(axis=0) - c.min(axis=0)))
        order = idx[np.lexsort((idx, c[:, axis]))]           # ties broken by element id
        cw = np.cumsum(w[order])
        k = int(np.searchsorted(cw, cw[-1] * left / count, side="right"))
        if len(idx) >= count:
            # skewed weights: each side keeps at least one element per partition
            k = min(max(k, left), len(idx) - (count - left))
        cut(order[:k], first, left)
        cut(order[k:], first + left, count - left)

    cut(np.arange(n), 0, int(nparts))
    return owner


def split(mesh, owner, nparts=None):
    """Plans of the partitions of `mesh` (dict of inputs.meshes) by owner[G]
    (partition of every global element).  Returns one dict per partition:
      mesh   : the partition's mesh dict (owned blocks first, then ghost blocks)
      ghost  : uint8 flag per block
      owned  : per owned block, (original block, global ids of its elements)
      ghosts : per ghost block, (original block, global ids)
      recv   : {q: int32 (n, 3) ghost (block, element, face) triplets}
      send   : {q: int32 (n, 3) owned triplets, in the order of q's recv[p]}
      keys_recv / keys_send : {q: int64 (n, 2) (G, f) of those records}
    """
    owner = np.asarray(owner, np.int64)
    off = global_offsets(mesh)
    nglob = int(off[-1])
    if owner.shape != (nglob,):
        raise ValueError(f"owner needs one entry per element ({nglob})")
    if nparts is None:
        nparts = int(owner.max()) + 1
    if owner.min() < 0 or owner.max() >= nparts:
        raise ValueError("owner out of range")
    faces = np.asarray(mesh["faces"], np.int64).reshape(-1, 6)
    shift = np.asarray(mesh["shift"], float).reshape(len(faces), -1)
    gl = off[faces[:, 0]] + faces[:, 1]
    gr = off[faces[:, 3]] + faces[:, 4]
    blk_of = np.repeat(np.arange(len(mesh["blocks"])), np.diff(off))
    plans = []
    for p in range(nparts):
        mine = owner == p
        touch = mine[gl] | mine[gr]
        ghost_ids = np.unique(np.concatenate([gr[touch & mine[gl] & ~mine[gr]], gl[touch & mine[gr] & ~mine[gl]]]))
        blocks, ghost, owned, ghosts = [], [], [], []
        local = {}                                   # global id -> (local block, local element)
        for b, blk in enumerate(mesh["blocks"]):
            ids = np.nonzero(mine[off[b]:off[b + 1]])[0] + off[b]
            if len(ids):
                for k, G in enumerate(ids):
                    local[int(G)] = (len(blocks), k)
                blocks.append({"shape": blk["shape"], "verts": np.asarray(blk["verts"])[ids - off[b]]})
                ghost.append(0)
                owned.append((b, ids))
        for b, blk in enumerate(mesh["blocks"]):
            ids = ghost_ids[blk_of[ghost_ids] == b] if len(ghost_ids) else ghost_ids
            if len(ids):
                for k, G in enumerate(ids):
                    local[int(G)] = (len(blocks), k)
                blocks.append({"shape": blk["shape"], "verts": np.asarray(blk["verts"])[ids - off[b]]})
                ghost.append(1)
                ghosts.append((b, ids))
        sel = np.nonzero(touch)[0]
        pf = np.zeros((len(sel), 6), np.int64)
        for i, fi in enumerate(sel):
            bl, el = local[int(gl[fi])]
            br, er = local[int(gr[fi])]
            pf[i] = (bl, el, faces[fi, 2], br, er, faces[fi, 5])
        plans.append({"mesh": {"blocks": blocks, "faces": pf, "shift": shift[sel]},
                      "ghost": np.array(ghost, np.uint8), "owned": owned, "ghosts": ghosts,
                      "recv": {}, "send": {}, "keys_recv": {}, "keys_send": {}, "local": local, "part": p,
                      "offsets": off})
    # Exchange lists: faces (G, f) with G owned by q and glued to an element of p != q.
    for fi in range(len(faces)):
        for (G, f, H) in ((gl[fi], faces[fi, 2], gr[fi]), (gr[fi], faces[fi, 5], gl[fi])):
            q, p = int(owner[G]), int(owner[H])
            if q != p:
                plans[p]["keys_recv"].setdefault(q, []).append((int(G), int(f)))
    for p in range(nparts):
        for q, keys in list(plans[p]["keys_recv"].items()):
            keys = np.array(sorted(set(keys)), np.int64).reshape(-1, 2)
            plans[p]["keys_recv"][q] = keys
            plans[q]["keys_send"][p] = keys
            plans[p]["recv"][q] = np.array([(*plans[p]["local"][int(G)], f) for G, f in keys], np.int32).reshape(-1, 3)
            plans[q]["send"][p] = np.array([(*plans[q]["local"][int(G)], f) for G, f in keys], np.int32).reshape(-1, 3)
    for pl in plans:
        pl["recv"] = dict(sorted(pl["recv"].items()))
        pl["send"] = dict(sorted(pl["send"].items()))
        pl["keys_recv"] = dict(sorted(pl["keys_recv"].items()))
        pl["keys_send"] = dict(sorted(pl["keys_send"].items()))
    return plans


def segments(lists):
    """{peer: (start, count)} of the peers' lists concatenated in peer order."""
    out, s = {}, 0
    for q, a in lists.items():
        out[q] = (s, len(a))
        s += len(a)
    return out


def concat(lists):
    return np.concatenate([a for a in lists.values()]).astype(np.int32) if lists else np.zeros((0, 3), np.int32)


def scatter_state(plan, U_global):
    """Owned blocks' states (N_s, V, E_local) from the whole mesh's per-block
    states (N_s, V, E)."""
    off = plan["offsets"]
    return [np.ascontiguousarray(U_global[b][:, :, ids - off[b]]) for b, ids in plan["owned"]]


def gather_state(plans, parts_blocks, like):
    """Whole-mesh per-block arrays from every partition's owned-block arrays
    (`like`: the whole mesh's per-block arrays, for shapes and dtype)."""
    out = [np.zeros_like(a) for a in like]
    for plan, blocks in zip(plans, parts_blocks):
        off = plan["offsets"]
        for (b, ids), a in zip(plan["owned"], blocks):
            out[b][:, :, ids - off[b]] = a
    return out


class PartitionMesh(sdrt.Mesh):
    """One partition set up in a Context, with its exchange lists and device
    send / receive buffers."""

    def __init__(self, ctx, plan, degree, physics):
        import torch
        self.plan = plan
        degrees = degree
        if isinstance(degree, (list, tuple)):         # per original block
            degrees = [degree[b] for b, _ in plan["owned"]] + [degree[b] for b, _ in plan["ghosts"]]
        super().__init__(ctx, plan["mesh"], degrees, physics, ghost=plan["ghost"])
        self.send_seg = segments(plan["send"])
        self.recv_seg = segments(plan["recv"])
        sdrt.sdrt_set_exchange(ctx.ptr, self.id, concat(plan["send"]), concat(plan["recv"]))
        self.xinfo = sdrt.sdrt_get_exchange_info(ctx.ptr, self.id)
        fr = self.xinfo["face_record"]
        gr = self.xinfo["grad_record"]
        self.viscous = gr > 0
        dt = torch.float32 if self.dtype_np == np.float32 else torch.float64
        dev = torch.device("cuda", ctx.device) if ctx.device >= 0 else torch.device("cpu")
        self.send_buf = torch.zeros(max(self.xinfo["nsend"], 1) * fr, dtype=dt, device=dev)
        self.recv_buf = torch.zeros(max(self.xinfo["nrecv"], 1) * fr, dtype=dt, device=dev)
        if self.viscous:
            self.send_gbuf = torch.zeros(max(self.xinfo["nsend"], 1) * gr, dtype=dt, device=dev)
            self.recv_gbuf = torch.zeros(max(self.xinfo["nrecv"], 1) * gr, dtype=dt, device=dev)

    def residual_begin(self, U):
        self._check(U)
        sdrt.sdrt_residual_begin(self.ctx.ptr, self.id, U, self.send_buf)

    def residual_gradients(self):
        sdrt.sdrt_residual_gradients(self.ctx.ptr, self.id, self.recv_buf, self.send_gbuf)

    def residual_end(self, R):
        self._check(R)
        sdrt.sdrt_residual_end(self.ctx.ptr, self.id, self.recv_gbuf if self.viscous else self.recv_buf, R)

    def _view(self, buf, seg, rec, q):
        s, n = seg[q]
        return buf[s * rec:(s + n) * rec]

    def send_view(self, q, grad=False):
        if grad:
            return self._view(self.send_gbuf, self.send_seg, self.xinfo["grad_record"], q)
        return self._view(self.send_buf, self.send_seg, self.xinfo["face_record"], q)

    def recv_view(self, q, grad=False):
        if grad:
            return self._view(self.recv_gbuf, self.recv_seg, self.xinfo["grad_record"], q)
        return self._view(self.recv_buf, self.recv_seg, self.xinfo["face_record"], q)


def copy_local(parts, grad=False):
    """Exchange between partitions held by one process (same stream): every
    receive segment from its sender's send segment (face states, or the
    gradient records of the viscous systems)."""
    by_part = {pm.plan["part"]: pm for pm in parts}
    for pm in parts:
        p = pm.plan["part"]
        for q in pm.recv_seg:
            pm.recv_view(q, grad).copy_(by_part[q].send_view(p, grad))


def residual_local(parts, Us, Rs):
    """Residual of partitions held by one process on one device: interpolate and
    pack every partition, exchange by device copies (viscous systems: then the
    flux-point gradients and a second exchange), then fluxes and divergence."""
    for pm, U in zip(parts, Us):
        pm.residual_begin(U)
    copy_local(parts)
    if parts and parts[0].viscous:
        for pm in parts:
            pm.residual_gradients()
        copy_local(parts, grad=True)
    for pm, R in zip(parts, Rs):
        pm.residual_end(R)


def exchange(send_views, recv_views, group=None):
    """Point-to-point exchange between processes: send_views / recv_views map
    peer rank -> contiguous tensor (the segments of this rank's buffers).
    torch.distributed with NCCL (device tensors) or gloo (CPU tensors)."""
    import torch.distributed as dist
    ops = []
    for q, t in recv_views.items():
        ops.append(dist.P2POp(dist.irecv, t, q, group))
    for q, t in send_views.items():
        ops.append(dist.P2POp(dist.isend, t, q, group))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


def _rk4(residual, Us, dt):
    """Classical RK4 (Sec. 2.1 explicit RK) over per-partition state tensors,
    `residual(Xs, Rs)` filling Rs with dU/dt of every partition."""
    import torch
    k = [torch.zeros_like(u) for u in Us]
    acc = [u.clone() for u in Us]
    X = [u.clone() for u in Us]
    for c_next, c_acc in ((0.5, 1.0 / 6.0), (0.5, 1.0 / 3.0), (1.0, 1.0 / 3.0), (None, 1.0 / 6.0)):
        residual(X, k)
        for i, u in enumerate(Us):
            acc[i].add_(k[i], alpha=dt * c_acc)
            if c_next is not None:
                torch.add(u, k[i], alpha=dt * c_next, out=X[i])
    for u, a in zip(Us, acc):
        u.copy_(a)


def rk4_step_local(parts, Us, dt):
    """One RK4 step of partitions held by one process (in place on Us): four
    partitioned residuals with device-copy exchanges, stage combinations on
    the padded state arrays (their padding stays zero)."""
    _rk4(lambda X, R: residual_local(parts, X, R), Us, dt)


def rk4_step_distributed(part, U, dt, group=None):
    """One RK4 step of this process's partition (in place on U), the face
    records exchanged with the peers by `exchange` once per stage."""
    def residual(X, R):
        part.residual_begin(X[0])
        exchange({q: part.send_view(q) for q in part.send_seg}, {q: part.recv_view(q) for q in part.recv_seg},
                 group)
        if part.viscous:
            part.residual_gradients()
            exchange({q: part.send_view(q, True) for q in part.send_seg},
                     {q: part.recv_view(q, True) for q in part.recv_seg}, group)
        part.residual_end(R[0])
    _rk4(residual, [U], dt)
