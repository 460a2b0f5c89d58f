"""Helpers for the GPU parity tests: build the same seeded mesh in the library
and in the oracle, pack / unpack states, seeded smooth states."""
import numpy as np

from inputs import fields, meshes
from oracle import mesh as omesh
from oracle import physics as ophx


def smooth_gas(X, amp=0.1):
    """Smooth gas state with independently varying rho, v, p (no flux ties)."""
    nd = X.shape[1]
    s = np.sin(2 * np.pi * X[:, 0])
    c = np.cos(2 * np.pi * X[:, 1])
    t = np.sin(2 * np.pi * (X[:, -1] + 0.3 * X[:, 0]))
    rho = 1.2 + amp * s * c
    vel = [0.3 + 2 * amp * c, -0.2 + 1.5 * amp * t, 0.1 + amp * s][:nd]
    p = 2.0 + 3 * amp * t * c
    return fields.primitive_to_conserved(rho, np.column_stack(vel), p, 1.4)


def oracle_state(geom, fn, nvar):
    out = []
    for g in geom.blocks:
        X = g.xsol.reshape(-1, g.xsol.shape[-1])
        v = fn(X).reshape(g.nelem, g.ops.n_sol, nvar)
        out.append(np.ascontiguousarray(np.transpose(v, (1, 2, 0))))
    return out


def perturb(U, seed, amp):
    return [u * (1 + fields.uniform_noise(u.shape, seed + i, amp)) for i, u in enumerate(U)]


def build_pair(ctx, kind, n, degree, system="euler", riemann="rusanov", precision="fp64", lo=0.0, hi=1.0,
               a=(1.0, 0.5, 0.25), scheme="sdrt", curve=0.0, curve_seed=None, **kw):
    """Library Mesh and oracle (geom, physics) for the same seeded box mesh;
    curve > 0: curved elements, the box displaced by meshes.curved_mesh."""
    from paper_2105_08632_gb300 import sdrt
    nd = len(n)
    mesh = meshes.box_mesh(kind, n, [lo] * nd, [hi] * nd)
    if curve:
        mesh = meshes.curved_mesh(mesh, curve, curve_seed)
    phys = sdrt.make_physics(system, nd, riemann, precision, a=a, **kw)
    M = sdrt.Mesh(ctx, mesh, degree, phys, scheme=scheme)
    geom = omesh.build(mesh, degree)
    oph = ophx.Physics(system, nd, riemann, a=tuple(a), mu=kw.get("mu", 0.0), gamma=kw.get("gamma", 1.4),
                       Pr=kw.get("prandtl", 0.72), beta=kw.get("beta", 0.5), eta=kw.get("eta", 0.1))
    return M, geom, oph, mesh


def rel_errors(got, want):
    """(relative L-inf, relative L2) over all blocks, normalised by max |want|."""
    g = np.concatenate([x.ravel() for x in got])
    w = np.concatenate([x.ravel() for x in want])
    scale = np.abs(w).max()
    return np.abs(g - w).max() / scale, np.sqrt(np.mean((g - w) ** 2)) / scale


U32 = 2.0 ** -24


def fp32_bound_ratio(got, want, scale):
    """max over all values of |got - want| / (u S): the observed error in units
    of the FP32 forward-error scale u * S (u = 2^-24, S = oracle term magnitudes)."""
    g = np.concatenate([x.ravel() for x in got])
    w = np.concatenate([x.ravel() for x in want])
    S = np.concatenate([x.ravel() for x in scale])
    return float(np.max(np.abs(g - w) / (U32 * S + 1e-300)))
