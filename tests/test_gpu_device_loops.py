"""Inner GMRES solves as device loops inside one CUDA graph per
preconditioner application (option graph_krylov), against the host-driven
loops (needs a GB300).

The recorded graph runs the same kernels on the same data as the host loop
(Gmres::solve): the convergence tests (residual estimate against the
tolerance, breakdown, restart length, iteration cap) are the same
comparisons, taken on the device.  So every solution below is required to be
bit-identical between the two modes, with the same iteration counts, and
the device-loop answer is checked against the oracle's direct solve like
any other.
"""
import numpy as np
import pytest

import fsi_inputs as F
from oracle import direct
from oracle.sparse import BlockOperator, rel_residual

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2206_06996_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)

COUNTS = ("outer_iters", "a_solves", "a_iters", "s_iters", "i_iters", "vcycles_A", "vcycles_S")


@pytest.fixture(scope="module")
def small():
    return F.tube_system("tube_small", keep_mesh=True)


@pytest.fixture(scope="module")
def small_direct(small):
    return direct.solve_block(small)


def _both_modes(system, **opts):
    out = {}
    for g in (0, 1):
        with pkg.BlockSolver(graph_krylov=g, **opts) as sol:
            sol.setup(system.A, system.B, system.C, system.D)
            l0 = sol.stats()["kernel_launches"]
            x = sol.solve(system.b.copy())
            st = sol.stats()
            out[g] = (x, st, st["kernel_launches"] - l0, sol.iters())
    return out


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
@pytest.mark.parametrize("precond", [pkg.SCR_PC_SCR, pkg.SCR_PC_SIMPLE, pkg.SCR_PC_SIMPLEC])
def test_device_loops_equal_host_loops(small, small_direct, precision, precond):
    res = _both_modes(small, precision=precision, precond=precond)
    (x0, s0, l0, it0), (x1, s1, l1, it1) = res[0], res[1]
    np.testing.assert_array_equal(x0, x1)
    assert it0 == it1
    for k in COUNTS:
        assert s0[k] == s1[k], k
    # every preconditioner application of the solve came from the graph,
    # none in host mode
    assert s0["pc_graph_runs"] == 0
    assert s1["pc_graph_runs"] == s1["outer_iters"] > 0
    # the host waits once per outer iteration (plus the final checks), not
    # once per inner step
    assert s1["syncs"] < s0["syncs"]
    assert s1["syncs"] <= s1["outer_iters"] + 4
    # the replayed kernels are counted: the same work plus the loop control
    assert l1 >= l0
    assert rel_residual(BlockOperator.from_system(small), x1, small.b) <= 1e-8
    err = np.linalg.norm(x1 - small_direct) / np.linalg.norm(small_direct)
    assert err <= 1e-6


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_device_loops_restart_and_iteration_cap(small, precision):
    """Inner restart length 3 and tight inner tolerances make every inner
    solve restart (the IF node of the recorded loop) and some stop at their
    iteration cap (max 7 steps): still bit-identical to the host loops."""
    opts = dict(precision=precision, restart_inner=3, rtol_A=1e-6, rtol_I=1e-6, rtol_S=1e-5,
                max_A=7, max_I=7, max_S=7)
    res = _both_modes(small, **opts)
    (x0, s0, _, it0), (x1, s1, _, it1) = res[0], res[1]
    np.testing.assert_array_equal(x0, x1)
    assert it0 == it1
    for k in COUNTS:
        assert s0[k] == s1[k], k
    # more steps than one cycle of 3 holds: the A solves restarted
    assert s1["a_iters"] > 3 * s1["a_solves"]
    assert s1["pc_graph_runs"] == s1["outer_iters"]
    assert rel_residual(BlockOperator.from_system(small), x1, small.b) <= 1e-8


def test_device_loops_fixed_count_and_outlets():
    """The fixed-count inner solve (two V-cycle Richardson steps, recorded
    as straight-line launches) and the outlets' rank-1 terms inside the
    recorded operator: bit-identical to the host loops."""
    s = F.tube_system("tube_small", outlet_resistance=2.7e4)
    res = {}
    for g in (0, 1):
        with pkg.BlockSolver(graph_krylov=g, inner_vcycles=2) as sol:
            sol.set_outlets(s.a_out, s.c_out)
            sol.setup(s.A, s.B, s.C, s.D)
            x = sol.solve(s.b.copy())
            res[g] = (x, sol.stats(), sol.iters())
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][2] == res[1][2]
    for k in COUNTS:
        assert res[0][1][k] == res[1][1][k], k
    assert res[1][1]["pc_graph_runs"] > 0


def test_device_loops_repeat_and_resetup(small):
    """The graph recorded at the first application after a set-up is
    replayed by later solves and recorded again after scr_setup and after
    scr_update_values (new values on the same pattern): each solve equals the
    host-driven one on the same values."""
    A2 = F.BSR(small.A.br, small.A.bc, small.A.nb_rows, small.A.nb_cols, small.A.row_ptr, small.A.col,
               small.A.val * 1.01)
    xs = {}
    for g in (0, 1):
        with pkg.BlockSolver(graph_krylov=g) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            first = sol.solve(small.b.copy())
            again = sol.solve(small.b.copy())
            sol.update_values(A2, small.B, small.C, small.D)
            upd = sol.solve(small.b.copy())
            sol.setup(small.A, small.B, small.C, small.D)
            fresh = sol.solve(small.b.copy())
            xs[g] = (first, again, upd, fresh, sol.stats()["pc_graph_runs"])
    for a, b in zip(xs[0][:4], xs[1][:4]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(xs[1][0], xs[1][1])
    np.testing.assert_array_equal(xs[1][0], xs[1][3])
    assert xs[1][4] > 0


def test_device_loops_multi_rhs(small):
    """Eight interleaved right-hand sides (block products, one FGMRES):
    bit-identical with and without device loops."""
    rng = np.random.default_rng(8)
    rhs = [small.b * rng.uniform(0.1, 2.0) for _ in range(8)]
    out = {}
    for g in (0, 1):
        with pkg.BlockSolver(graph_krylov=g, precision=pkg.SCR_MIXED, nrhs=8) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            xs, _ = sol.solve_multi([b.copy() for b in rhs])
            out[g] = (xs, sol.stats())
    for a, b in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(a, b)
    for k in COUNTS:
        assert out[0][1][k] == out[1][1][k], k
    assert out[1][1]["pc_graph_runs"] > 0
    for x in out[1][0]:
        assert np.all(np.isfinite(x))


def test_device_loops_single_preconditioner_application(small):
    """scr_apply_pc (Algorithm 1 once) from the recorded graph equals the
    direct application, twice in a row (record, then replay)."""
    r = np.random.default_rng(5).standard_normal(small.n)
    ys = {}
    for g in (0, 1):
        with pkg.BlockSolver(graph_krylov=g) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            y1 = sol.apply_pc(_dev(r)).cpu().numpy()
            st1 = sol.stats()
            y2 = sol.apply_pc(_dev(r)).cpu().numpy()
            ys[g] = (y1, y2, st1)
    for a, b in zip(ys[0][:2], ys[1][:2]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ys[1][0], ys[1][1])
    for k in ("a_solves", "a_iters", "s_iters", "i_iters"):
        assert ys[0][2][k] == ys[1][2][k], k
    assert ys[1][2]["pc_graph_runs"] == 1


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_device_loops_handle_reused_across_member_shapes(precision):
    """One handle set up and solved on members of uneven sizes in turn (the
    one-by-one form of the batched workload): the graph recorded for each
    member's set-up is used for that member only, and every member's answer
    and counts equal the host-driven ones."""
    members = [F.tube_system("batch", **F.batch_member_params(i)) for i in (0, 21, 42, 63)]
    out = {}
    for g in (0, 1):
        res = []
        with pkg.BlockSolver(graph_krylov=g, precision=precision) as sol:
            for m in members + members[:1]:
                sol.setup(m.A, m.B, m.C, m.D)
                x = sol.solve(m.b.copy())
                st = sol.stats()
                res.append((x, tuple(st[k] for k in COUNTS), st["pc_graph_runs"]))
        out[g] = res
    for (x0, c0, p0), (x1, c1, p1) in zip(out[0], out[1]):
        np.testing.assert_array_equal(x0, x1)
        assert c0 == c1
        assert p0 == 0 and p1 == c1[0]
    np.testing.assert_array_equal(out[1][0][0], out[1][-1][0])


def test_default_runs_device_loops_on_small_systems(small):
    """graph_krylov = 2 (the default) runs the device loops on a system of
    24,764 unknowns (below 1,000,000) and gives the same answer as either
    forced mode."""
    with pkg.BlockSolver() as sol:
        assert sol.opts.graph_krylov == 2
        sol.setup(small.A, small.B, small.C, small.D)
        x = sol.solve(small.b.copy())
        st = sol.stats()
    assert st["pc_graph_runs"] == st["outer_iters"] > 0
    with pkg.BlockSolver(graph_krylov=0) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        np.testing.assert_array_equal(sol.solve(small.b.copy()), x)


def test_graph_krylov_option_is_checked():
    with pytest.raises(Exception):
        pkg.BlockSolver(graph_krylov=3)


def test_device_loops_zero_and_nonfinite_inner_right_hand_sides(small):
    """Algorithm 1 applied to a zero vector, and to one with a NaN in its
    velocity part: the intermediate A solves then start from b = 0 (x = 0, no
    step) or from a non-finite b (x = 0, stopped at once), the S solve runs
    as usual, and the recorded loops give what the host loops give."""
    nv3 = 3 * small.n_v
    r_nan = np.random.default_rng(9).standard_normal(small.n)
    r_nan[7] = np.nan
    out = {}
    for g in (0, 1):
        with pkg.BlockSolver(graph_krylov=g) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            y0 = sol.apply_pc(_dev(np.zeros(small.n))).cpu().numpy()
            st0 = sol.stats()
            y1 = sol.apply_pc(_dev(r_nan)).cpu().numpy()
            st1 = sol.stats()
            out[g] = (y0, y1, st0, st1)
    for g in (0, 1):
        assert np.all(out[g][0] == 0.0)
        assert np.all(out[g][1][:nv3] == 0.0)
    np.testing.assert_array_equal(out[0][1], out[1][1])
    for k in ("a_iters", "s_iters", "i_iters"):
        assert out[0][2][k] == out[1][2][k] == 0, k
        assert out[0][3][k] == out[1][3][k], k
    assert out[1][3]["a_iters"] == 0
