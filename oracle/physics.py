"""Physical fluxes and common fluxes.

Oracle (test infrastructure only).  Arrays carry arbitrary leading dimensions:
u (..., V), physical gradient q (..., ND, V), unit normal n (..., ND), flux
f (..., ND, V).  All functions also accept complex arrays (complex-step JVP):
|.| and max() then branch on the real part, ties taking the left/first operand.

Systems (paper Sec. 3, 5):
  advection        f = a u                                     (Eq. "linear_advection")
  advdiff          f = a u - mu grad u                         (Sec. 5.1)
  euler            f = (rho v, rho v v + p I, (rho E + p) v)   (Eq. "fluxOperatorEuler")
  ns               euler + (0, -tau, -tau.v - mu gamma/Pr grad e)   (Eq. "fluxOperatorNavierStokes";
                   mu c_p/Pr grad T = mu gamma/Pr grad e with e = c_v T, mu dynamic)
Common fluxes (Sec. 2.1):
  upwind   F = (a.n)/2 (uL+uR) + |a.n|/2 (uL-uR)               (Eq. "flux_advection")
  rusanov  F = n.(fL+fR)/2 + phi/2 (uL-uR); phi = max(|vL.n|+cL, |vR.n|+cR) for gas
           dynamics, |a.n| for advection (reading: the paper leaves the estimator open)
  roe      textbook Roe average with a Harten entropy fix (delta = 0.1 c~) on the
           acoustic waves (not in the paper)
  ldg      F_v = n.[(1/2+beta) f_v,L + (1/2-beta) f_v,R] + eta (uL - uR)
           (Eq. for the common viscous flux with the repeated f_L read as f_R)
  common value for gradients  C = (1/2-beta) uL + (1/2+beta) uR   (Eq. "common_var_for_grad")

Parity: pinned by free-stream preservation, conservation, exactness of the
upwind flux for linear advection, the Roe flux's Rankine-Hugoniot property on a
single shock / exactness on a contact, and finite differences of the JVP
(tests/test_oracle_residual.py, tests/test_oracle_physics.py).
"""
from dataclasses import dataclass

import numpy as np


def rabs(z):
    if np.iscomplexobj(z):
        return np.where(z.real >= 0, z, -z)
    return np.abs(z)


def rmax(a, b):
    if np.iscomplexobj(a) or np.iscomplexobj(b):
        return np.where(a.real >= b.real, a, b)
    return np.where(a >= b, a, b)


@dataclass
class Physics:
    system: str                    # advection | advdiff | euler | ns
    nd: int
    riemann: str = "rusanov"       # upwind | rusanov | roe
    a: tuple = (1.0, 0.0, 0.0)
    mu: float = 0.0
    gamma: float = 1.4
    Pr: float = 0.72
    beta: float = 0.5
    eta: float = 0.1

    @property
    def nvar(self):
        return 1 if self.system in ("advection", "advdiff") else self.nd + 2

    @property
    def viscous(self):
        return self.system in ("advdiff", "ns")

    @property
    def avec(self):
        return np.asarray(self.a[: self.nd], float)


def euler_flux(u, gamma):
    nd = u.shape[-1] - 2
    rho = u[..., 0]
    m = u[..., 1:1 + nd]
    E = u[..., -1]
    v = m / rho[..., None]
    p = (gamma - 1) * (E - 0.5 * (m * v).sum(axis=-1))
    f = np.zeros(u.shape[:-1] + (nd, nd + 2), dtype=u.dtype)
    for d in range(nd):
        f[..., d, 0] = m[..., d]
        for i in range(nd):
            f[..., d, 1 + i] = m[..., d] * v[..., i]
        f[..., d, 1 + d] += p
        f[..., d, -1] = (E + p) * v[..., d]
    return f


def ns_viscous_flux(u, q, mu, gamma, Pr):
    """Viscous part f_v (..., ND, V) of the Navier-Stokes flux, q = physical gradient."""
    nd = u.shape[-1] - 2
    rho = u[..., 0]
    m = u[..., 1:1 + nd]
    E = u[..., -1]
    v = m / rho[..., None]
    grho = q[..., :, 0]                                  # (..., ND)
    gv = (q[..., :, 1:1 + nd] - grho[..., :, None] * v[..., None, :]) / rho[..., None, None]
    # gv[..., d, i] = d v_i / d x_d
    div = sum(gv[..., i, i] for i in range(nd))
    tau = np.zeros(u.shape[:-1] + (nd, nd), dtype=u.dtype)
    for i in range(nd):
        for j in range(nd):
            tau[..., i, j] = mu * (gv[..., j, i] + gv[..., i, j])
        tau[..., i, i] -= mu * 2.0 / 3.0 * div
    ge = (q[..., :, -1] - (E / rho)[..., None] * grho) / rho[..., None] \
        - (v[..., None, :] * gv).sum(axis=-1)             # grad of e = E/rho - |v|^2/2
    fv = np.zeros(u.shape[:-1] + (nd, nd + 2), dtype=u.dtype)
    for d in range(nd):
        for i in range(nd):
            fv[..., d, 1 + i] = -tau[..., i, d]
        fv[..., d, -1] = -(tau[..., d, :] * v).sum(axis=-1) - mu * gamma / Pr * ge[..., d]
    return fv


def flux(phys, u, q=None):
    """Total physical flux (..., ND, V)."""
    if phys.system in ("advection", "advdiff"):
        f = phys.avec[:, None] * u[..., None, :]
        if phys.system == "advdiff":
            f = f - phys.mu * q
        return f
    f = euler_flux(u, phys.gamma)
    if phys.system == "ns":
        f = f + ns_viscous_flux(u, q, phys.mu, phys.gamma, phys.Pr)
    return f


def viscous_flux(phys, u, q):
    if phys.system == "advdiff":
        return -phys.mu * q
    return ns_viscous_flux(u, q, phys.mu, phys.gamma, phys.Pr)


def _normal(f, n):
    return (f * n[..., :, None]).sum(axis=-2)


def sound_speed_and_vn(u, n, gamma):
    nd = u.shape[-1] - 2
    rho = u[..., 0]
    m = u[..., 1:1 + nd]
    v = m / rho[..., None]
    p = (gamma - 1) * (u[..., -1] - 0.5 * (m * v).sum(axis=-1))
    c = np.sqrt(gamma * p / rho)
    vn = (v * n).sum(axis=-1)
    return c, vn


def roe_flux(uL, uR, n, gamma):
    """Roe flux for the Euler equations, Harten entropy fix (delta = 0.1 c~) on the
    two acoustic waves only (the contact and shear waves stay exact)."""
    nd = uL.shape[-1] - 2
    fL = _normal(euler_flux(uL, gamma), n)
    fR = _normal(euler_flux(uR, gamma), n)

    def prim(u):
        rho = u[..., 0]
        v = u[..., 1:1 + nd] / rho[..., None]
        p = (gamma - 1) * (u[..., -1] - 0.5 * rho * (v * v).sum(axis=-1))
        H = (u[..., -1] + p) / rho
        return rho, v, p, H

    rL, vL, pL, HL = prim(uL)
    rR, vR, pR, HR = prim(uR)
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    w = sL + sR
    vt = (sL[..., None] * vL + sR[..., None] * vR) / w[..., None]
    Ht = (sL * HL + sR * HR) / w
    rt = sL * sR
    q2 = (vt * vt).sum(axis=-1)
    ct = np.sqrt((gamma - 1) * (Ht - 0.5 * q2))
    vnt = (vt * n).sum(axis=-1)
    dr = rR - rL
    dp = pR - pL
    dv = vR - vL
    dvn = (dv * n).sum(axis=-1)

    def fix(lam):
        a = rabs(lam)
        d = 0.1 * ct
        return np.where(a.real < d.real, (a * a + d * d) / (2 * d), a)

    l1, l2, l5 = fix(vnt - ct), rabs(vnt), fix(vnt + ct)
    a1 = (dp - rt * ct * dvn) / (2 * ct * ct)
    a5 = (dp + rt * ct * dvn) / (2 * ct * ct)
    a2 = dr - dp / (ct * ct)
    V = nd + 2
    diss = np.zeros(uL.shape, dtype=np.result_type(uL, uR, n))
    # acoustic waves
    for a, l, sgn in ((a1, l1, -1.0), (a5, l5, 1.0)):
        k = np.zeros_like(diss)
        k[..., 0] = 1
        k[..., 1:1 + nd] = vt + sgn * ct[..., None] * n
        k[..., -1] = Ht + sgn * ct * vnt
        diss = diss + (l * a)[..., None] * k
    # entropy wave
    k = np.zeros_like(diss)
    k[..., 0] = 1
    k[..., 1:1 + nd] = vt
    k[..., -1] = 0.5 * q2
    diss = diss + (l2 * a2)[..., None] * k
    # shear waves
    dvt = dv - dvn[..., None] * n
    k = np.zeros_like(diss)
    k[..., 1:1 + nd] = dvt
    k[..., -1] = (vt * dvt).sum(axis=-1)
    diss = diss + (l2 * rt)[..., None] * k
    assert diss.shape[-1] == V
    return 0.5 * (fL + fR) - 0.5 * diss


def common_convective(phys, uL, uR, n):
    if phys.system in ("advection", "advdiff"):
        an = (phys.avec * n).sum(axis=-1)[..., None]
        if phys.riemann not in ("upwind", "rusanov"):
            raise ValueError("advection supports upwind / rusanov")
        return 0.5 * an * (uL + uR) + 0.5 * rabs(an) * (uL - uR)
    if phys.riemann == "roe":
        return roe_flux(uL, uR, n, phys.gamma)
    if phys.riemann != "rusanov":
        raise ValueError(phys.riemann)
    fL = _normal(euler_flux(uL, phys.gamma), n)
    fR = _normal(euler_flux(uR, phys.gamma), n)
    cL, vnL = sound_speed_and_vn(uL, n, phys.gamma)
    cR, vnR = sound_speed_and_vn(uR, n, phys.gamma)
    phi = rmax(rabs(vnL) + cL, rabs(vnR) + cR)
    return 0.5 * (fL + fR) + 0.5 * phi[..., None] * (uL - uR)


def common_viscous(phys, uL, uR, qL, qR, n):
    fvL = _normal(viscous_flux(phys, uL, qL), n)
    fvR = _normal(viscous_flux(phys, uR, qR), n)
    return (0.5 + phys.beta) * fvL + (0.5 - phys.beta) * fvR + phys.eta * (uL - uR)


def common_value(phys, uL, uR):
    return (0.5 - phys.beta) * uL + (0.5 + phys.beta) * uR
