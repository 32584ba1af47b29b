"""The bifurcation at full size: parent R = 0.5 cm with a 0.06 cm wall, a
4 cm parent and two 4 cm daughters at +-35 degrees, 40 x 40 core cells, 24
lumen rings (the last 3 graded by 0.6 towards the wall) and 5 wall rings,
633 layers (about 4M nodes, 16M unknowns).  Eight
right-hand sides -R at inflow peaks drawn U(0, 60) cm/s on one Jacobian
(the nominal 30 cm/s), solved as one 8-column block solve in mixed
precision with the FP64 outer FGMRES.  At this size the oracle checks
properties: every column's FP64 residual, recomputed with the oracle's
block operator, meets 1e-8.  Collected after every other test (the
longest case: the other files run first in a run that stops at the first
failure)."""
import numpy as np
import pytest

import fsi_inputs as F
from oracle.sparse import BlockOperator, rel_residual

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2206_06996_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def test_bifurcation_full_size_eight_inflow_peaks():
    s = F.tube_system("bifurcation")
    assert s.n > 15_000_000
    peaks = np.random.default_rng(2206).uniform(0.0, 60.0, 8)
    rhs = [torch.as_tensor(F.rhs_only("bifurcation", u_max=float(u)), device="cuda") for u in peaks]
    Ad, Bd, Cd, Dd = (pkg.DeviceBSR.from_host(M) for M in (s.A, s.B, s.C, s.D))
    with pkg.BlockSolver(nrhs=8, precision=pkg.SCR_MIXED) as sol:
        sol.setup(Ad, Bd, Cd, Dd)
        xs, rel = sol.solve_multi(rhs)
    assert np.all(rel <= 1e-8)
    op = BlockOperator.from_system(s)
    for b, x in zip(rhs, xs):
        assert rel_residual(op, x.cpu().numpy(), b.cpu().numpy()) <= 1e-8
