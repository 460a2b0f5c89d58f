"""SDRT and FR-SDRT semi-discrete residuals, RK4, complex-step JVP, Jacobians.

Oracle (test infrastructure only).  State layout per block: U[b] of shape
(N_s, V, E) (solution point, variable, element), the paper's state matrix
(App. B, Eq. "state_matrices") with the element index fastest.

SDRT residual, in the paper's order (Sec. 2.1):
  1. u_fe = M0 U, u_fiu = M12 U, u_fi = P u_fiu    (Eqs. "interpolate_sol_to_flux",
                                                   "interpolate_sol_to_fluxint", App. B)
  2. viscous only: common value C at external points (Eq. "common_var_for_grad"),
     transformed gradient q~ = M16 C + M15 u_fi (Eq. for q~ at solution points,
     App. B), physical q = J^{-T} q~ with J at each solution point,
     interpolated with M0 / M12
  3. internal DOFs: F~_nu = [det J J^{-1} f(u, q)] . n~_nu, J at the internal
     point (Eq. "normal_transformed_flux")
  4. external points: F~ = det J |J^{-T} n~| F(uL, uR, qL, qR, n), J at the
     external point (common flux, Sec. 2.1)
  5. div = M14 F~_fe + M13 F~_fi                   (Eq. "divergence_sdrt", "residual_sdrt_matrices")
  6. dU/dt = -div / det J, J at each solution point (semi-discrete form, Sec. 2.1)
FR-SDRT (Sec. 2.3, Eq. "divergence_fr" with grad.g = grad.l^fe):
  div = sum_d D_d f~_d + M14 (F~_fe - (M0 f~) . n~_fe),  f~ at solution points;
  viscous gradient with the same correction: q~ = D u + M16 (C - M0 u).

Parity: pinned by free-stream preservation, discrete conservation, FR-SDRT
equivalence, the p+1 convergence order against the analytic advected solution,
and (for the JVP) central finite differences and linearity
(tests/test_oracle_residual.py).
"""
import numpy as np

from . import physics as phx


def _gather_partner(geom, vals):
    """vals: list per block of (N_fe, ..., E) arrays -> (u_face_L, u_face_R) each a
    list of (E, N_fe, ...) arrays: the values of the face's L and R sides seen
    from each external point (own value on its own side)."""
    flat = []
    for g, v in zip(geom.blocks, vals):
        t = np.moveaxis(v, -1, 0)                 # (E, N_fe, ...)
        flat.append(t.reshape((-1,) + t.shape[2:]))
    flat = np.concatenate(flat, axis=0)
    other = flat[geom.partner]
    left = geom.is_left.reshape((-1,) + (1,) * (flat.ndim - 1))
    fL = np.where(left, flat, other)
    fR = np.where(left, other, flat)
    outL, outR = [], []
    for b, g in enumerate(geom.blocks):
        n = g.nelem * g.ops.n_fe
        s = geom.fe_base[b]
        shp = (g.nelem, g.ops.n_fe) + flat.shape[1:]
        outL.append(fL[s:s + n].reshape(shp))
        outR.append(fR[s:s + n].reshape(shp))
    return outL, outR


def _face_sign(geom, b):
    """+1 on the L side of each point's face, -1 on the R side: (E, N_fe)."""
    g = geom.blocks[b]
    s = geom.fe_base[b]
    n = g.nelem * g.ops.n_fe
    return np.where(geom.is_left[s:s + n], 1.0, -1.0).reshape(g.nelem, g.ops.n_fe)


def _to_phys_grad(Jinvs, qt):
    """q_i = sum_d Jinv[d, i] q~_d at every solution point.  Jinvs: (E, N_s, ND, ND),
    qt: (ND, N_s, V, E) -> (ND, N_s, V, E)."""
    return np.einsum("endi,dnve->inve", Jinvs, qt)


def solution_gradients(geom, phys, U, fr=False):
    """Physical gradients q at the solution points, per block (ND, N_s, V, E):
    q~ = M16 C + M15 u_fi with the common value C at the external points
    (Sec. 2.1, Eq. "common_var_for_grad" and the transformed auxiliary
    gradient), q = J^{-T} q~."""
    ufe = [np.einsum("sr,rve->sve", g.ops.M0, u) for g, u in zip(geom.blocks, U)]
    ufiu = [np.einsum("kr,rve->kve", g.ops.M12, u) for g, u in zip(geom.blocks, U)]
    return _sol_gradients(geom, phys, U, ufe, ufiu, fr)


def _sol_gradients(geom, phys, U, ufe, ufiu, fr=False):
    uL, uR = _gather_partner(geom, ufe)
    out = []
    for b, g in enumerate(geom.blocks):
        ops = g.ops
        C = phx.common_value(phys, uL[b], uR[b])            # (E, N_fe, V)
        C = np.moveaxis(C, 0, -1)                           # (N_fe, V, E)
        nd, ns = g.ops.nd, ops.n_sol
        if not fr:
            ufi = np.einsum("ik,kve->ive", ops.P, ufiu[b])
            qt = (np.einsum("sr,rve->sve", ops.M16, C) + np.einsum("si,ive->sve", ops.M15, ufi))
        else:
            Du = np.einsum("dsr,rve->dsve", ops.Dsol, U[b]).reshape(nd * ns, *U[b].shape[1:])
            qt = Du + np.einsum("sr,rve->sve", ops.M16, C - ufe[b])
        qt = qt.reshape(nd, ns, *qt.shape[1:])
        out.append(_to_phys_grad(g.Jinvs, qt))               # (ND, N_s, V, E)
    return out


def _gradients(geom, phys, U, ufe, ufiu, fr=False):
    """Physical gradients at external and unique internal points (viscous only)."""
    qfe, qfiu = [], []
    for g, q in zip(geom.blocks, _sol_gradients(geom, phys, U, ufe, ufiu, fr)):
        qfe.append(np.einsum("fs,dsve->fdve", g.ops.M0, q))   # (N_fe, ND, V, E)
        qfiu.append(np.einsum("ks,dsve->kdve", g.ops.M12, q))
    return qfe, qfiu


def residual(geom, phys, U, fr=False, terms=False):
    """dU/dt for every block.  U: list of (N_s, V, E) arrays (real or complex).

    terms=True also returns, per block, the magnitude of the divergence's terms
    S = (|M14| |F~_fe| + |M13| |F~_fi|) / det J (same shape as dU/dt): the scale
    of the rounding errors of a finite-precision evaluation (forward error
    bound |dR| <= gamma S)."""
    scales = []
    ufe = [np.einsum("sr,rve->sve", g.ops.M0, u) for g, u in zip(geom.blocks, U)]
    ufiu = [np.einsum("kr,rve->kve", g.ops.M12, u) for g, u in zip(geom.blocks, U)]
    if phys.viscous:
        qfe, qfiu = _gradients(geom, phys, U, ufe, ufiu, fr=fr)
    uL, uR = _gather_partner(geom, ufe)
    if phys.viscous:
        qL, qR = _gather_partner(geom, qfe)                 # (E, N_fe, ND, V)
    out = []
    for b, g in enumerate(geom.blocks):
        ops = g.ops
        # Common flux of each face along its L normal, transformed with det J |n|
        # and signed for the point's own side.
        sgn = _face_sign(geom, b)
        nL = sgn[:, :, None] * g.nunit
        F = phx.common_convective(phys, uL[b], uR[b], nL)
        if phys.viscous:
            F = F + phx.common_viscous(phys, uL[b], uR[b], qL[b], qR[b], nL)
        Ft_fe = np.moveaxis((sgn * g.nmag)[:, :, None] * F, 0, -1)  # (N_fe, V, E)
        if not fr:
            # Internal flux at unique points: (E, N_fiu, ND, V).
            u_in = np.moveaxis(ufiu[b], -1, 0)
            q_in = np.moveaxis(qfiu[b], -1, 0) if phys.viscous else None
            f = phx.flux(phys, u_in, q_in)
            ft = g.detf[:, :, None, None] * np.einsum("ekdi,ekiv->ekdv", g.Jinvf, f)
            ftp = ft[:, ops.fi_point]                          # (E, N_fi, ND, V)
            Ft_fi = np.einsum("nd,endv->nve", ops.fi_dir, ftp)  # (N_fi, V, E)
            div = np.einsum("sf,fve->sve", ops.M14, Ft_fe) + np.einsum("sn,nve->sve", ops.M13, Ft_fi)
            if terms:
                scales.append((np.einsum("sf,fve->sve", np.abs(ops.M14), np.abs(Ft_fe)) +
                               np.einsum("sn,nve->sve", np.abs(ops.M13), np.abs(Ft_fi))) / g.dets.T[:, None, :])
        else:
            u_s = np.moveaxis(U[b], -1, 0)                      # (E, N_s, V)
            if phys.viscous:
                # gradient at solution points, recomputed from the FR correction
                q_s = _fr_sol_grad(g, phys, U[b], ufe[b], uL[b], uR[b])
            else:
                q_s = None
            f = phx.flux(phys, u_s, q_s)                        # (E, N_s, ND, V)
            ft = g.dets[:, :, None, None] * np.einsum("esdi,esiv->esdv", g.Jinvs, f)
            div = np.einsum("dsr,erdv->sve", ops.Dsol, ft)
            ft_fe = np.einsum("fs,esdv->efdv", ops.M0, ft)
            jump = Ft_fe - np.moveaxis(np.einsum("efdv,fd->efv", ft_fe, ops.nrm_fe), 0, -1)
            div = div + np.einsum("sf,fve->sve", ops.M14, jump)
        out.append(-div / g.dets.T[:, None, :])
    return (out, scales) if terms else out


def _fr_sol_grad(g, phys, U, ufe, uL, uR):
    ops = g.ops
    nd, ns = ops.nd, ops.n_sol
    C = np.moveaxis(phx.common_value(phys, uL, uR), 0, -1)
    qt = np.einsum("dsr,rve->dsve", ops.Dsol, U) + \
        np.einsum("sr,rve->sve", ops.M16, C - ufe).reshape(nd, ns, *U.shape[1:])
    q = _to_phys_grad(g.Jinvs, qt)                          # (ND, N_s, V, E)
    return np.transpose(q, (3, 1, 0, 2))                   # (E, N_s, ND, V)


def rk4_step(geom, phys, U, dt, fr=False):
    """Classical RK4 (paper Sec. 2.1 uses explicit RK; RK4 polynomial Eq. "rk_exponential")."""
    k1 = residual(geom, phys, U, fr)
    k2 = residual(geom, phys, [u + 0.5 * dt * k for u, k in zip(U, k1)], fr)
    k3 = residual(geom, phys, [u + 0.5 * dt * k for u, k in zip(U, k2)], fr)
    k4 = residual(geom, phys, [u + dt * k for u, k in zip(U, k3)], fr)
    return [u + dt / 6 * (a + 2 * b + 2 * c + d) for u, a, b, c, d in zip(U, k1, k2, k3, k4)]


def jvp(geom, phys, U, V, h=1e-30):
    """Exact directional derivative dR/dU . V by the complex step (Im R(U + i h V) / h)."""
    Uc = [u.astype(complex) + 1j * h * v for u, v in zip(U, V)]
    return [r.imag / h for r in residual(geom, phys, Uc)]


def flatten(U):
    return np.concatenate([u.ravel() for u in U])


def unflatten(geom, x, nvar):
    out, s = [], 0
    for g in geom.blocks:
        n = g.ops.n_sol * nvar * g.nelem
        out.append(x[s:s + n].reshape(g.ops.n_sol, nvar, g.nelem))
        s += n
    return out


def jacobian(geom, phys, U):
    """Dense RHS Jacobian (small meshes only), column j = JVP with unit vector j."""
    x0 = flatten(U)
    n = x0.size
    Jm = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Jm[:, j] = flatten(jvp(geom, phys, U, unflatten(geom, e, phys.nvar)))
    return Jm


def vjp(geom, phys, U, W):
    """W^T J via the dense Jacobian (small meshes only)."""
    Jm = jacobian(geom, phys, U)
    return unflatten(geom, Jm.T @ flatten(W), phys.nvar)
