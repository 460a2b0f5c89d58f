"""Taylor-Green diagnostics of the library (sdrt_tgv_diagnostics, paper Sec.
5.3) against the oracle's (pinned in tests/test_oracle_tgv.py): the same
ensemble averages of the kinetic energy and of eps1, eps2, eps3 at the
initial state and after RK4 steps, FP64 to 1e-9 relative (eps3, which is
~0 at t = 0, to 1e-9 of eps2), FP32 to the FP32 tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import fields  # noqa: E402
from oracle import residual as ores  # noqa: E402
from oracle import tgv  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

KW = {"mu": 1 / 1600, "prandtl": 0.71, "beta": 0.5, "eta": 0.1}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08632_gb300 import build, sdrt
    build.build()
    c = sdrt.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kind,n,p", [("tet", (3, 3, 3), 3), ("hex", (3, 3, 3), 2), ("pri", (3, 3, 2), 3)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diagnostics_match_oracle(ctx, kind, n, p, precision):
    M, geom, oph, _ = gu.build_pair(ctx, kind, n, p, "ns", "rusanov", precision, lo=0.0, hi=2 * np.pi, **KW)
    U = gu.oracle_state(geom, lambda X: fields.taylor_green(X, gamma=1.4, mach=0.1), 5)
    for step in range(2):
        want = tgv.diagnostics(geom, oph, U)
        got = M.tgv_diagnostics(torch.from_numpy(M.pack(U)).to("cuda"))
        tol = 1e-9 if precision == "fp64" else 1e-4
        for k in ("E", "eps1", "eps2"):
            assert got[k] == pytest.approx(want[k], rel=tol if k != "eps1" or precision == "fp64" else 2e-2), \
                (step, k, got[k], want[k])
        assert abs(got["eps3"] - want["eps3"]) <= (1e-9 if precision == "fp64" else 1e-2) * abs(want["eps2"]), \
            (step, got["eps3"], want["eps3"])
        U = ores.rk4_step(geom, oph, U, 5e-4)


def test_diagnostics_reject_other_systems(ctx):
    from paper_2105_08632_gb300 import sdrt
    M, geom, oph, _ = gu.build_pair(ctx, "tet", (2, 2, 2), 2, "euler", "rusanov", "fp64")
    U = torch.ones(M.state_len, dtype=torch.float64, device="cuda")
    with pytest.raises(sdrt.SdrtError) as ei:
        M.tgv_diagnostics(U)
    assert ei.value.code == -2
