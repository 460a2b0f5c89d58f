"""Host-side pins of the stability tools (no GPU): the RK stability
polynomials and the CFL search against textbook stability limits, and the
Fourier-mode bookkeeping (wavenumber sets, reduced-Jacobian assembly) on a
case with a closed-form spectrum."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2105_08632_gb300 import stability as st  # noqa: E402


def test_rk_polynomials_are_the_truncated_exponential():
    """P(z) - exp(z) = O(z^{order+1}) for RK3 / RK4 (and RK54, 4th order)."""
    z = torch.tensor([0.3 + 0.2j, -1.1 + 0.7j], dtype=torch.complex128)
    for scheme, order in (("rk3", 3), ("rk4", 4), ("rk54", 4)):
        err = (st.rk_polynomial(z * 1e-2, scheme) - torch.exp(z * 1e-2)).abs().max()
        assert err < 1e-2 ** (order + 1), (scheme, float(err))


@pytest.mark.parametrize("scheme,real,imag", [("rk3", 2.5127453266, 1.7320508076),
                                              ("rk4", 2.7852935634, 2.8284271247)])
def test_cfl_search_matches_textbook_limits(scheme, real, imag):
    """Stability limits of RK3 / RK4 on the negative real axis and the imaginary
    axis (textbook values: RK3 sqrt(3) on the imaginary axis, RK4 2 sqrt(2))."""
    lam = torch.tensor([-1.0 + 0.0j], dtype=torch.complex128)
    assert st.cfl_max(lam, scheme) == pytest.approx(real, rel=1e-8)
    lam = torch.tensor([1.0j, -1.0j], dtype=torch.complex128)
    assert st.cfl_max(lam, scheme) == pytest.approx(imag, rel=1e-8)


def test_reduced_eigenvalues_of_a_periodic_difference_operator():
    """G(kappa) = sum_c J_c e^{-i kappa dx_c} for the first-order upwind operator
    on a 1-cell pattern: J_0 = -1, J_{-1} = +1 (the upstream cell), so
    lambda(kappa) = -1 + e^{i kappa}: the wavenumber bookkeeping and the sign of
    the phase, pinned by the closed form."""
    blocks = torch.tensor([[[-1.0]], [[1.0]]], dtype=torch.float64)        # cells 0 and -1
    offsets = torch.tensor([[0.0], [-1.0]], dtype=torch.float64)
    kap = st.kappa_line((1.0,), 9)
    lam = st.reduced_eigenvalues(blocks, offsets, kap)[:, 0]
    want = -1.0 + torch.exp(1j * kap[:, 0].to(torch.complex128))
    assert torch.allclose(lam, want, atol=1e-14)
    # and its RK4 CFL limit: the disc |1 + lambda| = 1 scaled, tau_max = 1.3925...
    tau = st.cfl_max(lam, "rk4")
    assert 1.0 < tau < 2.0


def test_kappa_sets():
    g = st.kappa_grid(2, 4)
    assert g.shape == (16, 2) and float(g.min()) == pytest.approx(-np.pi) and float(g.max()) < np.pi
    line = st.kappa_line((3.0, 4.0), 5)
    assert line.shape == (5, 2)
    assert torch.allclose(line[-1], torch.tensor([0.6, 0.8], dtype=torch.float64) * 2 * np.pi)
    a = st.advection_direction(np.pi / 6, np.pi / 4)
    assert np.linalg.norm(a) == pytest.approx(1.0)
