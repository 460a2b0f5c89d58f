"""RK54 (Carpenter-Kennedy two-register scheme) and its PI step-size
controller on the GPU against the oracle (oracle/timestep.py, which is pinned
by the paper's stability polynomial and the order conditions):

* fixed RK54 steps equal the oracle's steps (FP64 1e-9 of the change of the
  state, FP32 5e-3 as for the RK4 parity test);
* one adaptive step: the same error norm (L-infinity of the embedded
  estimate over atol + rtol max(|U_start|, |U|)), acceptance and next step
  size as the oracle's; a rejected step leaves the state unchanged;
* an adaptive integration over a span takes the oracle's accepted /
  rejected steps and ends at its state.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import residual as ores  # noqa: E402
from oracle import timestep as ots  # noqa: E402
from tests import gpu_util as gu  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    c = sdrt.Context(0)
    yield c
    c.close()


def _case(ctx, precision, kind="tet", n=(2, 2, 2), p=2):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "euler", "rusanov", precision)
    U = gu.perturb(gu.oracle_state(geom, gu.smooth_gas, 5), 71, 0.01)
    rhs = lambda X: ores.residual(geom, oph, X)          # noqa: E731
    return M, U, rhs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rk54_steps_match_oracle(ctx, precision):
    M, U, rhs = _case(ctx, precision)
    dt = 2e-3
    W = U
    for _ in range(3):
        W = ots.rk54_step(rhs, W, dt)
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    M.rk54_step(Ud, dt, 3)
    M.sync()
    got = M.unpack(Ud.cpu().numpy())
    linf, _ = gu.rel_errors([g - u for g, u in zip(got, U)], [w - u for w, u in zip(W, U)])
    assert linf < (1e-9 if precision == "fp64" else 5e-3), linf


def test_adaptive_step_matches_oracle(ctx):
    M, U, rhs = _case(ctx, "fp64")
    atol = rtol = 1e-7
    for dt in (5e-4, 5e-3):                                # an accepted and a rejected attempt
        Ud = torch.from_numpy(M.pack(U)).to("cuda")
        before = Ud.clone()
        acc, err, dtn = M.rk54_adaptive_step(Ud, dt, atol, rtol)
        Un, acc_o, err_o, dtn_o, _ = ots.adaptive_step(rhs, U, dt, atol, rtol, 1.0)
        assert acc == acc_o, (dt, err, err_o)
        assert err == pytest.approx(err_o, rel=1e-6), (dt, err, err_o)
        assert dtn == pytest.approx(dtn_o, rel=1e-6)
        if acc:
            linf, _ = gu.rel_errors([g - u for g, u in zip(M.unpack(Ud.cpu().numpy()), U)],
                                    [w - u for w, u in zip(Un, U)])
            assert linf < 1e-9, linf
        else:
            assert torch.equal(Ud, before)
    assert dt == 5e-3 and not acc


def test_adaptive_integration_matches_oracle(ctx):
    M, U, rhs = _case(ctx, "fp64")
    atol = rtol = 1e-6
    span, dt0 = 0.02, 0.05
    W, dt_o, na_o, nr_o = ots.integrate(rhs, U, span, dt0, atol, rtol)
    Ud = torch.from_numpy(M.pack(U)).to("cuda")
    dt_n, na, nr = M.rk54_integrate(Ud, span, dt0, atol, rtol)
    assert (na, nr) == (na_o, nr_o)
    assert nr >= 1
    assert dt_n == pytest.approx(dt_o, rel=1e-5)
    got = M.unpack(Ud.cpu().numpy())
    linf, _ = gu.rel_errors([g - u for g, u in zip(got, U)], [w - u for w, u in zip(W, U)])
    assert linf < 1e-8, linf
