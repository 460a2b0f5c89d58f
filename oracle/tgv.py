"""Taylor-Green vortex diagnostics (paper Sec. 5.3): the ensemble average of
the non-dimensional kinetic energy and the dissipation terms eps1, eps2, eps3.

Oracle (test infrastructure only).
  <.> = (1/|Omega|) int_Omega . dOmega, with an element quadrature exact for
  polynomials of degree 10 (the paper's choice of degree): the Gauss-Legendre
  tensor rule of 7 points per direction, collapsed (Duffy) onto the simplex
  directions;
  E*   = (1/2) rho v.v / (rho_inf v_inf^2)  (the printed formula drops the 1/2;
         with it eps1 = eps2 + eps3 is the kinetic-energy balance, the reading
         recorded in the design notes);
  eps1 = -d<E*>/dt*, t* = t / t_c, t_c = L / v_inf, evaluated from the
         residual: d(rho v.v / 2)/dt = v . R_m - (v.v / 2) R_rho;
  eps2 = 2 mu t_c <S^d : S^d> / (rho_inf v_inf^2), S^d the deviatoric strain rate;
  eps3 = -t_c <p div v> / (rho_inf v_inf^2);
velocity gradients from the scheme's LDG gradients q at the solution points
(the paper computes eps3 from the LDG gradients), interpolated with the
solution nodal basis.

Parity: pinned by the Taylor-Green initial state's closed forms (<E*> = 1/8
up to the O(Ma^2) density variation, eps2 = 3 mu / 4 (t_c = 1), eps3 = 0 for
the divergence-free initial field, eps1 = eps2 + eps3 for a resolved mesh) and
by exact integration of monomials (tests/test_oracle_tgv.py).
"""
import numpy as np

from . import operators
from . import residual as ores


def quadrature(shape, n=7):
    """Points (nq, ND) and weights of the tensor Gauss-Legendre rule on the
    reference element (collapsed onto simplices: triangle x_i >= -1, x + y <= 0;
    tetrahedron x_i >= -1, x + y + z <= -1; prism = triangle x [-1, 1])."""
    g, w = np.polynomial.legendre.leggauss(n)
    if shape == "quad":
        A, B = np.meshgrid(g, g, indexing="xy")
        WA, WB = np.meshgrid(w, w, indexing="xy")
        return np.column_stack([A.ravel(), B.ravel()]), (WA * WB).ravel()
    if shape == "hex":
        X, W = [], []
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    X.append((g[i], g[j], g[k]))
                    W.append(w[i] * w[j] * w[k])
        return np.array(X), np.array(W)

    def tri():
        X, W = [], []
        for j in range(n):
            for i in range(n):
                X.append(((1 + g[i]) * (1 - g[j]) / 2 - 1, g[j]))
                W.append(w[i] * w[j] * (1 - g[j]) / 2)
        return np.array(X), np.array(W)
    if shape == "tri":
        return tri()
    if shape == "pri":
        Xt, Wt = tri()
        X = np.array([(x[0], x[1], z) for z in g for x in Xt])
        W = np.array([wt * wz for wz in w for wt in Wt])
        return X, W
    X, W = [], []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                z = g[k]
                y = (1 + g[j]) * (1 - z) / 2 - 1
                x = (1 + g[i]) * (-y - z) / 2 - 1
                X.append((x, y, z))
                W.append(w[i] * w[j] * w[k] * (1 - z) / 2 * (-y - z) / 2)
    return np.array(X), np.array(W)


def diagnostics(geom, phys, U, rho_inf=1.0, v_inf=1.0, length=1.0):
    """Dict E (<E*>), eps1, eps2, eps3 of the state U (3D Navier-Stokes)."""
    R = ores.residual(geom, phys, U)
    Q = ores.solution_gradients(geom, phys, U)           # (ND, N_s, V, E) per block
    s = np.zeros(5)
    for g, u, r, q in zip(geom.blocks, U, R, Q):
        if g.curved:
            raise ValueError("diagnostics take affine elements (one det J per element)")
        Xq, Wq = quadrature(g.shape)
        L = operators.nodal_sol(g.shape, g.p, g.ops.xs, Xq)   # (nq, N_s)
        uq = np.einsum("qs,sve->qve", L, u)
        rq = np.einsum("qs,sve->qve", L, r)
        gq = np.einsum("qs,dsve->qdve", L, q)
        w = Wq[:, None] * g.detJ[None, :]
        rho = uq[:, 0]
        m = uq[:, 1:4]
        vel = m / rho[:, None]
        ke = np.einsum("qie,qie->qe", m, vel)              # rho v.v
        p = (phys.gamma - 1) * (uq[:, 4] - 0.5 * ke)
        dke = np.einsum("qie,qie->qe", vel, rq[:, 1:4]) - 0.5 * (ke / rho) * rq[:, 0]
        gv = (gq[:, :, 1:4] - vel[:, None, :, :] * gq[:, :, 0:1]) / rho[:, None, None, :]   # (q, d, i, e)
        div = gv[:, 0, 0] + gv[:, 1, 1] + gv[:, 2, 2]
        Sd = 0.5 * (gv + np.swapaxes(gv, 1, 2)) - (div / 3.0)[:, None, None, :] * np.eye(3)[None, :, :, None]
        ss = np.einsum("qije,qije->qe", Sd, Sd)
        s += [w.sum(), (w * 0.5 * ke).sum(), (w * dke).sum(), (w * ss).sum(), (w * p * div).sum()]
    scale, tc, vol = rho_inf * v_inf ** 2, length / v_inf, s[0]
    return {"E": s[1] / vol / scale, "eps1": -tc * s[2] / vol / scale,
            "eps2": 2 * phys.mu * tc * s[3] / vol / scale, "eps3": -tc * s[4] / vol / scale}
