"""Pins of the oracle's residual against what the paper and the mathematics fix.

  * free-stream preservation on affine meshes (Sec. 2: analytical metrics on
    uniform grids);
  * discrete conservation on periodic meshes (common flux antisymmetry, Sec. 2.1);
  * FR-SDRT == SDRT for linear fluxes on constant-metric elements (Sec. 2.3,
    Tables "linadvecdiff_linfty_diff_sdrt_fr_sdrt*": differences at roundoff);
  * order p+1 against the exact advected solution (Sec. 5.1, "order of accuracy");
  * closed-form viscous rates: shear / longitudinal / heat-conduction waves;
  * the isentropic vortex's exact time derivative (translation, Eq. "eulerVortexWitherden");
  * Taylor-Green initial kinetic-energy decay d<E_k>/dt = -(3/4) mu;
  * complex-step JVP against central differences; linearity for advection.
"""
import numpy as np
import pytest

from inputs import fields, meshes
from oracle import mesh as omesh
from oracle import operators
from oracle import physics as phx
from oracle import residual as ores
from tests import quadrature

KIND = {"tri": "tri", "quad": "quad", "tet": "tet", "pri": "pri", "hex": "hex"}
N2 = {"tri": (3, 3), "quad": (3, 3), "tet": (2, 2, 2), "pri": (2, 2, 2), "hex": (2, 2, 2)}


def _geom(shape, p, n=None, lo=0.0, hi=1.0):
    n = n or N2[shape]
    nd = len(n)
    m = meshes.box_mesh(KIND[shape], n, [lo] * nd, [hi] * nd)
    return omesh.build(m, p), m


def _eval(geom, fn, nvar):
    out = []
    for g in geom.blocks:
        X = g.xsol.reshape(-1, g.xsol.shape[-1])
        v = fn(X).reshape(g.nelem, g.ops.n_sol, nvar)
        out.append(np.ascontiguousarray(np.transpose(v, (1, 2, 0))))
    return out


def _weights(g):
    Xq, Wq = quadrature.rule(g.shape, 10)
    return Wq @ operators.nodal_sol(g.shape, g.p, g.ops.xs, Xq)


def _integral(geom, R):
    tot = 0.0
    for g, r in zip(geom.blocks, R):
        tot = tot + np.einsum("s,sve,e->v", _weights(g), r, g.detJ)
    return tot


EULER_STATE = {2: [1.2, 0.3, -0.2, 3.0], 3: [1.2, 0.3, -0.2, 0.1, 3.0]}
CASES = [(s, p) for s in ("tri", "quad", "tet", "pri", "hex") for p in (1, 2, 3, 4)]


@pytest.mark.parametrize("shape,p", CASES)
def test_free_stream(shape, p):
    geom, _ = _geom(shape, p)
    nd = geom.nd
    for phys, state in (
            (phx.Physics("advection", nd, "upwind", a=(1.0, 0.5, 0.25)), [1.0]),
            (phx.Physics("euler", nd, "rusanov"), EULER_STATE[nd]),
            (phx.Physics("euler", nd, "roe"), EULER_STATE[nd]),
            (phx.Physics("ns", nd, "rusanov", mu=0.01, Pr=0.71), EULER_STATE[nd])):
        U = _eval(geom, lambda X: fields.constant(X, state), phys.nvar)
        R = ores.residual(geom, phys, U)
        fmag = 3.0 / 0.5                      # |f| / h
        assert max(np.abs(r).max() for r in R) < 1e-9 * fmag, phys.system


@pytest.mark.parametrize("shape,p", CASES)
def test_conservation(shape, p):
    geom, _ = _geom(shape, p)
    nd = geom.nd
    rng = np.random.default_rng(5)
    for phys in (phx.Physics("euler", nd, "rusanov"), phx.Physics("euler", nd, "roe"),
                 phx.Physics("ns", nd, "rusanov", mu=0.05, Pr=0.71, beta=0.5, eta=0.1)):
        U = _eval(geom, lambda X: fields.constant(X, EULER_STATE[nd]), phys.nvar)
        U = [u * (1 + 0.05 * rng.uniform(-1, 1, u.shape)) for u in U]
        R = ores.residual(geom, phys, U)
        scale = max(np.abs(r).max() for r in R)
        assert np.abs(_integral(geom, R)).max() < 1e-12 * scale * 10


@pytest.mark.parametrize("shape,p", CASES)
def test_fr_sdrt_free_stream_and_conservation(shape, p):
    """FR-SDRT (Sec. 2.3) with the nonlinear fluxes: a constant state gives a zero
    residual, and the discrete integral of dU/dt vanishes on periodic meshes
    (the correction carries the common flux through the faces, Sec. 2.3), for
    Euler with Rusanov and Roe fluxes and for Navier-Stokes."""
    geom, _ = _geom(shape, p)
    nd = geom.nd
    rng = np.random.default_rng(7)
    for phys in (phx.Physics("euler", nd, "rusanov"), phx.Physics("euler", nd, "roe"),
                 phx.Physics("ns", nd, "rusanov", mu=0.05, Pr=0.71, beta=0.5, eta=0.1)):
        U = _eval(geom, lambda X: fields.constant(X, EULER_STATE[nd]), phys.nvar)
        R = ores.residual(geom, phys, U, fr=True)
        assert max(np.abs(r).max() for r in R) < 1e-9 * 3.0 / 0.5, phys.system
        U = [u * (1 + 0.05 * rng.uniform(-1, 1, u.shape)) for u in U]
        R = ores.residual(geom, phys, U, fr=True)
        scale = max(np.abs(r).max() for r in R)
        assert np.abs(_integral(geom, R)).max() < 1e-12 * scale * 10, phys.system


@pytest.mark.parametrize("shape,p", CASES)
def test_fr_sdrt_equivalence(shape, p):
    """Sec. 2.3: with constant metrics and a linear flux, SDRT and FR-SDRT give the
    same residual for any state (also with the LDG gradient, remark of Sec. 2.3)."""
    geom, _ = _geom(shape, p)
    nd = geom.nd
    rng = np.random.default_rng(6)
    for phys in (phx.Physics("advection", nd, "upwind", a=(1.0, 0.5, 0.25)),
                 phx.Physics("advdiff", nd, "upwind", a=(1.0, 0.5, 0.25), mu=0.1, beta=0.3, eta=0.2)):
        U = [rng.uniform(-1, 1, (g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
        R = ores.residual(geom, phys, U)
        Rfr = ores.residual(geom, phys, U, fr=True)
        scale = max(np.abs(r).max() for r in R)
        assert max(np.abs(a - b).max() for a, b in zip(R, Rfr)) < 1e-12 * scale


def _advect_error(shape, p, n, T=0.25):
    a = (1.0, 0.5)
    phys = phx.Physics("advection", 2, "upwind", a=a)
    geom, _ = _geom(shape, p, (n, n))
    U = _eval(geom, fields.sine_product, 1)
    h = 1.0 / n
    steps = int(np.ceil(T / (0.1 * h)))
    dt = T / steps
    for _ in range(steps):
        U = ores.rk4_step(geom, phys, U, dt)
    exact = _eval(geom, lambda X: fields.sine_product(X - np.array(a) * T), 1)
    return max(np.abs(u - e).max() for u, e in zip(U, exact))


@pytest.mark.parametrize("shape,p", [("tri", 1), ("tri", 2), ("quad", 2), ("quad", 3)])
def test_convergence_order(shape, p):
    e1 = _advect_error(shape, p, 8)
    e2 = _advect_error(shape, p, 16)
    order = np.log2(e1 / e2)
    assert order > p + 1 - 0.5, (e1, e2, order)


def _wave_residual(phys, geom, prim_fn):
    def cons(X):
        rho, vel, p = prim_fn(X)
        return fields.primitive_to_conserved(rho, vel, p, phys.gamma)
    U = _eval(geom, cons, phys.nvar)
    return U, ores.residual(geom, phys, U)


@pytest.mark.parametrize("shape,p", [("hex", 3), ("tet", 3), ("pri", 3)])
def test_viscous_rates_closed_form(shape, p):
    """With eps = 1e-3 waves of wavenumber k = 2 pi, R(mu) - R(0) projected on
    sin(kx) (the decay rate of the mode) equals
      shear  v = (0, eps sin kx, 0):        d(rho v)/dt = -mu k^2 eps sin kx
      long.  v = (eps sin kx, 0, 0):        d(rho u)/dt = -(4/3) mu k^2 eps sin kx
      heat   p = p0 + eps sin kx, v = 0:    d(rho E)/dt = -mu gamma/(Pr (gamma-1)) k^2 eps sin kx
    up to O(eps^2 mu) and the discretisation error (LDG, beta = 1/2, eta = 0.1)."""
    geom, _ = _geom(shape, p, (4, 4, 4))
    k, eps, mu, Pr, gam = 2 * np.pi, 1e-3, 0.02, 0.71, 1.4
    visc = phx.Physics("ns", 3, "rusanov", mu=mu, Pr=Pr, beta=0.5, eta=0.1)
    invisc = phx.Physics("euler", 3, "rusanov")
    cases = [
        (lambda X: (np.ones(len(X)), np.column_stack([0 * X[:, 0], eps * np.sin(k * X[:, 0]), 0 * X[:, 0]]),
                    np.full(len(X), 10.0)), 2, mu),
        (lambda X: (np.ones(len(X)), np.column_stack([eps * np.sin(k * X[:, 0]), 0 * X[:, 0], 0 * X[:, 0]]),
                    np.full(len(X), 10.0)), 1, 4.0 / 3.0 * mu),
        (lambda X: (np.ones(len(X)), np.zeros((len(X), 3)), 10.0 + eps * np.sin(k * X[:, 0])), 4,
         mu * gam / (Pr * (gam - 1))),
    ]
    for prim, var, coef in cases:
        _, Rv = _wave_residual(visc, geom, prim)
        _, Ri = _wave_residual(invisc, geom, prim)
        num, den = 0.0, 0.0
        for g, rv, ri in zip(geom.blocks, Rv, Ri):
            w = _weights(g)
            s = np.sin(k * g.xsol[:, :, 0].T)
            num += np.einsum("s,se,e->", w, (rv - ri)[:, var, :] * s, g.detJ)
            den += np.einsum("s,se,e->", w, s * s, g.detJ)
        rate = num / den
        assert abs(rate / (-coef * k * k * eps) - 1) < 0.02, (var, rate)


@pytest.mark.parametrize("shape,p", [("tet", 3), ("hex", 3)])
def test_vortex_time_derivative(shape, p):
    """dU/dt of the translating isentropic vortex (S = 13.5, R = 1.5, Ma = 0.5)
    equals the exact time derivative of Eq. "eulerVortexWitherden"; the discrete
    residual's pointwise error falls at least like h^2 (SD truncation error is
    O(h^p) pointwise) on [-7.5, 7.5]^2 x one periodic layer."""
    phys = phx.Physics("euler", 3, "rusanov")
    errs = []
    for n in (12, 24):
        geom, _ = _geom(shape, p, (n, n, 1), lo=-7.5, hi=7.5)
        def at(t):
            return _eval(geom, lambda X: fields.isentropic_vortex(X, mach=0.5, t=t), 5)
        R = ores.residual(geom, phys, at(0.0))
        dt = 1e-6
        exact = [(a - b) / (2 * dt) for a, b in zip(at(dt), at(-dt))]
        errs.append(max(np.abs(r - e).max() for r, e in zip(R, exact)) /
                    max(np.abs(e).max() for e in exact))
    assert errs[1] < 0.25 * errs[0], errs
    assert errs[1] < 0.2, errs


def test_taylor_green_initial_dissipation():
    """d<E_k>/dt at t = 0 equals -mu <|grad v|^2> = -(3/4) mu for the TGV
    (Eq. "tgvInitCondition": div v = 0, convective terms conserve E_k)."""
    mu = 1.0 / 100.0
    phys = phx.Physics("ns", 3, "rusanov", mu=mu, Pr=0.71, beta=0.5, eta=0.1)
    geom, _ = _geom("hex", 3, (6, 6, 6), lo=0.0, hi=2 * np.pi)
    U = _eval(geom, lambda X: fields.taylor_green(X, mach=0.1), 5)
    R = ores.residual(geom, phys, U)
    tot, vol = 0.0, 0.0
    for g, u, r in zip(geom.blocks, U, R):
        w = _weights(g)
        v = u[:, 1:4, :] / u[:, 0:1, :]
        dEk = (v * r[:, 1:4, :]).sum(1) - 0.5 * (v * v).sum(1) * r[:, 0, :]
        tot += np.einsum("s,se,e->", w, dEk, g.detJ)
        vol += w.sum() * g.detJ.sum()
    rate = tot / vol
    assert abs(rate / (-0.75 * mu) - 1) < 0.05, rate


@pytest.mark.parametrize("riemann", ["rusanov", "roe"])
def test_common_flux_properties(riemann):
    rng = np.random.default_rng(7)
    phys = phx.Physics("euler", 3, riemann)
    uL = np.array([1.0, 0.2, -0.1, 0.3, 2.5]) * (1 + 0.1 * rng.uniform(-1, 1, (50, 5)))
    uR = np.array([0.9, -0.1, 0.2, 0.1, 2.2]) * (1 + 0.1 * rng.uniform(-1, 1, (50, 5)))
    n = rng.normal(size=(50, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    F = phx.common_convective(phys, uL, uR, n)
    Fr = phx.common_convective(phys, uR, uL, -n)
    assert np.abs(F + Fr).max() < 1e-13            # conservation property (Sec. 2.1)
    fn = (phx.euler_flux(uL, 1.4) * n[:, :, None]).sum(1)
    assert np.abs(phx.common_convective(phys, uL, uL, n) - fn).max() < 1e-13   # consistency


def test_roe_exact_for_stationary_contact():
    """A stationary contact (equal p, zero velocity, different rho) is an exact
    Roe-linearised discontinuity: the flux is the pressure only."""
    phys = phx.Physics("euler", 3, "roe")
    p = 2.0
    uL = fields.primitive_to_conserved(np.array([1.0]), np.zeros((1, 3)), np.array([p]), 1.4)
    uR = fields.primitive_to_conserved(np.array([0.3]), np.zeros((1, 3)), np.array([p]), 1.4)
    F = phx.common_convective(phys, uL, uR, np.array([[1.0, 0.0, 0.0]]))
    assert np.allclose(F, [[0, p, 0, 0, 0]], atol=1e-14)


def test_upwind_flux_takes_upwind_state():
    phys = phx.Physics("advection", 2, "upwind", a=(1.0, 0.5))
    F = phx.common_convective(phys, np.array([[2.0]]), np.array([[5.0]]), np.array([[1.0, 0.0]]))
    assert F[0, 0] == 2.0
    F = phx.common_convective(phys, np.array([[2.0]]), np.array([[5.0]]), np.array([[-1.0, 0.0]]))
    assert F[0, 0] == -5.0


def _smooth_gas_state(X):
    """Smooth gas state whose density, velocity and pressure vary independently
    (no ties in the Rusanov wave-speed estimate)."""
    s = np.sin(2 * np.pi * X[:, 0])
    c = np.cos(2 * np.pi * X[:, 1])
    t = np.sin(2 * np.pi * (X[:, 2] + 0.3 * X[:, 0]))
    rho = 1.2 + 0.1 * s * c
    vel = np.column_stack([0.3 + 0.2 * c, -0.2 + 0.15 * t, 0.1 + 0.1 * s])
    p = 2.0 + 0.3 * t * c
    return fields.primitive_to_conserved(rho, vel, p, 1.4)


@pytest.mark.parametrize("shape,p", [("tet", 2), ("pri", 2), ("hex", 1)])
def test_jvp_matches_finite_differences(shape, p):
    geom, _ = _geom(shape, p)
    phys = phx.Physics("euler", 3, "rusanov")
    rng = np.random.default_rng(8)
    U = _eval(geom, _smooth_gas_state, 5)
    V = [rng.normal(size=u.shape) for u in U]
    Jv = ores.jvp(geom, phys, U, V)
    h = 1e-6
    Rp = ores.residual(geom, phys, [u + h * v for u, v in zip(U, V)])
    Rm = ores.residual(geom, phys, [u - h * v for u, v in zip(U, V)])
    fd = [(a - b) / (2 * h) for a, b in zip(Rp, Rm)]
    scale = max(np.abs(x).max() for x in Jv)
    assert max(np.abs(a - b).max() for a, b in zip(Jv, fd)) < 1e-6 * scale


def test_jvp_of_linear_advection_is_the_residual():
    geom, _ = _geom("tet", 2)
    phys = phx.Physics("advection", 3, "upwind", a=(1.0, 0.5, 0.25))
    rng = np.random.default_rng(9)
    U = [rng.normal(size=(g.ops.n_sol, 1, g.nelem)) for g in geom.blocks]
    V = [rng.normal(size=u.shape) for u in U]
    Jv = ores.jvp(geom, phys, U, V)
    Rv = ores.residual(geom, phys, V)
    assert max(np.abs(a - b).max() for a, b in zip(Jv, Rv)) < 1e-13


def test_vjp_is_the_gradient_of_the_weighted_residual():
    """W^T J is the gradient of phi(U) = <W, R(U)>: checked by central
    differences of phi along random directions (independent of the JVP)."""
    geom, _ = _geom("tet", 1)
    phys = phx.Physics("euler", 3, "rusanov")
    rng = np.random.default_rng(10)
    U = _eval(geom, _smooth_gas_state, 5)
    W = [rng.normal(size=u.shape) for u in U]
    g = ores.vjp(geom, phys, U, W)

    def phi(X):
        return sum(float(np.sum(w * r)) for w, r in zip(W, ores.residual(geom, phys, X)))

    h = 1e-6
    for _ in range(3):
        d = [rng.normal(size=u.shape) for u in U]
        fd = (phi([u + h * x for u, x in zip(U, d)]) - phi([u - h * x for u, x in zip(U, d)])) / (2 * h)
        ad = sum(float(np.sum(a * x)) for a, x in zip(g, d))
        assert abs(fd - ad) < 1e-6 * max(1.0, abs(ad)), (fd, ad)


def test_face_map_is_an_involution_pairing_coincident_points():
    for shape in ("tri", "tet", "pri", "hex", "quad"):
        geom, m = _geom(shape, 2)
        part = geom.partner
        assert np.array_equal(part[part], np.arange(len(part)))
        assert np.all(part != np.arange(len(part)))
