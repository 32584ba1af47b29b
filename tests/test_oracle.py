"""Pins of the CPU oracle against brute force, closed forms and invariants
(no GPU).  A few tests plant a mistake in an oracle function (on the CPU)
and check that the pins catch it."""
import numpy as np
import pytest
import scipy.sparse as sp

import fsi_inputs as F
from oracle import amg, direct, krylov, schur, scr
from oracle.sparse import BlockOperator, bsr_matvec_by_definition, rel_residual, to_csr


def _random_bsr(rng, nbr, nbc, br, bc, density=0.3):
    rp = [0]
    cols = []
    for i in range(nbr):
        c = np.nonzero(rng.random(nbc) < density)[0]
        cols.extend(c.tolist())
        rp.append(len(cols))
    rp = np.array(rp, dtype=np.int32)
    col = np.array(cols, dtype=np.int32)
    val = rng.standard_normal(len(cols) * br * bc)
    return F.BSR(br, bc, nbr, nbc, rp, col, val)


# ------------------------------------------------------------- sparse
@pytest.mark.parametrize("br,bc", [(3, 3), (3, 1), (1, 3), (1, 1)])
def test_block_matvec_definition_vs_dense(br, bc):
    rng = np.random.default_rng(br * 10 + bc)
    M = _random_bsr(rng, 17, 13, br, bc)
    dense = np.zeros((17 * br, 13 * bc))
    blocks = M.val.reshape(-1, br, bc)
    for i in range(17):
        for t in range(M.row_ptr[i], M.row_ptr[i + 1]):
            j = M.col[t]
            dense[i * br:(i + 1) * br, j * bc:(j + 1) * bc] += blocks[t]
    x = rng.standard_normal(13 * bc)
    assert np.allclose(bsr_matvec_by_definition(M, x), dense @ x, rtol=1e-13, atol=1e-13)
    assert np.allclose(to_csr(M).toarray(), dense)


# ------------------------------------------------------------- direct
def test_direct_solution_residual(mini_system, mini_direct):
    op = BlockOperator.from_system(mini_system)
    assert rel_residual(op, mini_direct, mini_system.b) < 1e-12


def test_direct_matches_dense_on_tiny(tiny_system):
    op = BlockOperator.from_system(tiny_system)
    x = direct.solve_block(tiny_system)
    xd = np.linalg.solve(op.full().toarray(), tiny_system.b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_mesh_direct(mini_system):
    u = direct.solve_mesh(mini_system)
    L = to_csr(mini_system.L)
    g = mini_system.mesh_b.reshape(-1, 3)
    assert np.linalg.norm(L @ u.reshape(-1, 3) - g) < 1e-12 * np.linalg.norm(g)


# ------------------------------------------------------------- schur
def test_ldu_factorisation(tiny_system):
    op = BlockOperator.from_system(tiny_system)
    Lf, Df, Uf = schur.ldu_factors_dense(op)
    K = op.full().toarray()
    assert np.allclose(Lf @ Df @ Uf, K, rtol=1e-10, atol=1e-12 * np.abs(K).max())


def test_exact_scr_is_inverse(tiny_system):
    op = BlockOperator.from_system(tiny_system)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(op.n)
    y = schur.scr_exact_apply(op, r)
    yd = np.linalg.solve(op.full().toarray(), r)
    assert np.linalg.norm(y - yd) <= 1e-9 * np.linalg.norm(yd)


def test_exact_scr_catches_planted_mistake(tiny_system, monkeypatch):
    """Algorithm 1 with step 2 dropped (r_p not updated) must miss A^{-1}."""
    op = BlockOperator.from_system(tiny_system)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(op.n)
    yd = np.linalg.solve(op.full().toarray(), r)

    def broken(op, r):
        A = op.A.toarray()
        S = schur.schur_exact_dense(op)
        rv, rp = op.split(r)
        yp = np.linalg.solve(S, rp)
        yv = np.linalg.solve(A, rv - op.B @ yp)
        return np.concatenate([yv, yp])

    monkeypatch.setattr(schur, "scr_exact_apply", broken)
    y = schur.scr_exact_apply(op, r)
    # the pin above holds to 1e-9; the planted mistake misses by far more
    assert np.linalg.norm(y - yd) > 1e-6 * np.linalg.norm(yd)


def test_schur_hat_definition(tiny_system):
    op = BlockOperator.from_system(tiny_system)
    A, B, C, D = (M.toarray() for M in (op.A, op.B, op.C, op.D))
    Sh = D - C @ np.diag(1.0 / np.diag(A)) @ B
    assert np.allclose(schur.schur_hat(op).toarray(), Sh, rtol=1e-12, atol=1e-14 * np.abs(Sh).max())
    # Shat equals the exact S when A is diagonal
    Adiag = sp.diags(op.A.diagonal()).tocsr()
    op2 = BlockOperator.__new__(BlockOperator)
    op2.A, op2.B, op2.C, op2.D = Adiag, op.B, op.C, op.D
    op2.nv, op2.np, op2.n = op.nv, op.np, op.n
    assert np.allclose(schur.schur_hat(op2).toarray(), schur.schur_exact_dense(op2), rtol=1e-10,
                       atol=1e-14 * np.abs(Sh).max())


def test_simple_identity(tiny_system):
    op = BlockOperator.from_system(tiny_system)
    P1 = schur.simple_matrix_dense(op)
    P2 = schur.simple_factored_dense(op)
    assert np.allclose(P1, P2, rtol=1e-9, atol=1e-12 * np.abs(P1).max())


def test_simple_inverse_is_inverse_of_simple_matrix(tiny_system):
    op = BlockOperator.from_system(tiny_system)
    rng = np.random.default_rng(8)
    r = rng.standard_normal(op.n)
    y = schur.simple_inverse_apply_dense(op, r)
    P = schur.simple_matrix_dense(op)
    assert np.linalg.norm(P @ y - r) <= 1e-9 * np.linalg.norm(r)


def test_simple_apply_with_tight_solves(tiny_system):
    opts = scr.SolverOptions(rtol_A=1e-13, rtol_S=1e-13, max_A=400, max_S=400, restart_inner=80,
                             precond="simple")
    s = scr.SCRSolver(tiny_system, opts)
    rng = np.random.default_rng(9)
    r = rng.standard_normal(s.op.n)
    y = s.apply_simple(r)
    yd = schur.simple_inverse_apply_dense(s.op, r)
    assert np.linalg.norm(y - yd) <= 1e-8 * np.linalg.norm(yd)


def test_simple_full_solve_matches_direct(mini_system, mini_direct):
    s = scr.SCRSolver(mini_system, scr.SolverOptions(precond="simple"))
    x, info = s.solve(mini_system.b)
    assert info.converged
    assert s.rel_residual(x, mini_system.b) <= 1e-8
    assert np.linalg.norm(x - mini_direct) <= 1e-6 * np.linalg.norm(mini_direct)


# ------------------------------------------------------------- krylov
def _nonsym(rng, n):
    return np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)


def test_gmres_finite_termination():
    rng = np.random.default_rng(1)
    n = 25
    A = _nonsym(rng, n)
    b = rng.standard_normal(n)
    x, info = krylov.fgmres(lambda v: A @ v, b, tol=1e-13, restart=n, maxit=n)
    assert info.iters <= n
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)


def test_gmres_restarted_converges():
    rng = np.random.default_rng(2)
    n = 60
    A = _nonsym(rng, n)
    b = rng.standard_normal(n)
    x, info = krylov.fgmres(lambda v: A @ v, b, tol=1e-10, restart=7, maxit=400)
    assert info.converged and info.restarts > 1
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)


def test_fgmres_exact_preconditioner_one_iteration(tiny_system):
    op = BlockOperator.from_system(tiny_system)
    x, info = krylov.fgmres(op.matvec, tiny_system.b, lambda r: schur.scr_exact_apply(op, r),
                            tol=1e-8)
    assert info.iters == 1
    assert rel_residual(op, x, tiny_system.b) < 1e-8


def test_fgmres_residual_estimate_matches_true_residual():
    # the Givens recurrence value |g_{k+1}| equals ||b - A x_k||
    rng = np.random.default_rng(3)
    n = 40
    A = _nonsym(rng, n)
    b = rng.standard_normal(n)
    for k in (3, 6, 9):
        x, info = krylov.fgmres(lambda v: A @ v, b, tol=1e-300, restart=k, maxit=k,
                                true_residual_check=False)
        est = info.rel_res
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert abs(est - true) < 1e-10


def test_pcg():
    rng = np.random.default_rng(4)
    n = 30
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    x, info = krylov.pcg(lambda v: A @ v, b, lambda r: r / np.diag(A), tol=1e-12, maxit=n + 5)
    assert info.converged and info.iters <= n
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9)


def test_zero_rhs():
    x, info = krylov.fgmres(lambda v: 2 * v, np.zeros(5))
    assert info.converged and np.all(x == 0)
    x, info = krylov.pcg(lambda v: 2 * v, np.zeros(5))
    assert info.converged and np.all(x == 0)


# ------------------------------------------------------------- amg
def test_tentative_prolongator_orthonormal():
    agg = np.array([0, 0, 1, -1, 1, 1, 2, 0])
    for bs in (1, 3):
        Pt = amg.tentative_prolongator(agg, bs).toarray()
        assert np.allclose(Pt.T @ Pt, np.eye(3 * bs))
        # constants on each aggregate are reproduced
        assert np.allclose((Pt @ (Pt.T @ np.ones(8 * bs)))[np.repeat(agg >= 0, bs)], 1.0)


def test_aggregation_covers_strong_nodes(mini_system):
    A = to_csr(mini_system.A)
    S = amg.strength_graph(A, 3, 0.08)
    agg = amg.aggregate_greedy(S)
    has_nb = np.diff(S.indptr) > 0
    assert np.all(agg[has_nb] >= 0) and np.all(agg[~has_nb] == -1)
    # every aggregate is connected in the strength graph
    for a in range(agg.max() + 1):
        nodes = np.nonzero(agg == a)[0]
        sub = S[nodes][:, nodes]
        ncomp = sp.csgraph.connected_components(sub, directed=False)[0]
        assert ncomp == 1


def test_vcycle_contracts_on_spd(mini_system):
    L = to_csr(mini_system.L)
    H = amg.setup(L, 1, 0.08, 10, 16, 2, 2)
    assert H.n_levels >= 2
    rng = np.random.default_rng(5)
    Ld = L.toarray()
    # error propagation E = I - M^{-1} L; its energy norm must be < 1
    n = L.shape[0]
    E = np.eye(n) - np.column_stack([amg.vcycle(H, Ld[:, j]) for j in range(n)])
    w, V = np.linalg.eigh(Ld)
    Lh = V @ np.diag(np.sqrt(w)) @ V.T
    Lhi = V @ np.diag(1 / np.sqrt(w)) @ V.T
    rho = np.linalg.norm(Lh @ E @ Lhi, 2)
    assert rho < 0.9, rho
    # the V-cycle is a symmetric operator (usable in CG)
    M = np.column_stack([amg.vcycle(H, np.eye(n)[:, j]) for j in range(n)])
    assert np.allclose(M, M.T, atol=1e-10 * np.abs(M).max())


def test_galerkin_operator(mini_system):
    L = to_csr(mini_system.L)
    H = amg.setup(L, 1, 0.08, 10, 16, 1, 1)
    l0, l1 = H.levels[0], H.levels[1]
    Ac = (l0.P.T @ l0.A @ l0.P).toarray()
    assert np.allclose(l1.A.toarray(), Ac, rtol=1e-12, atol=1e-14 * np.abs(Ac).max())
    # smoothed prolongator definition
    lam = np.max(np.abs(L).sum(axis=1).A1 / np.abs(L.diagonal()))
    Pt = amg.tentative_prolongator(l0.agg, 1)
    P = Pt - (4 / (3 * lam)) * sp.diags(1 / L.diagonal()) @ L @ Pt
    assert np.allclose(l0.P.toarray(), P.toarray(), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("bs", [1, 3])
def test_prolongator_truncation_definition(bs):
    """Vectorised truncation = the per-row definition (keep blocks with
    norm >= 0.3 of the row maximum, at most 4, largest first with ties to
    the smaller column; rescale each scalar row to its old sum)."""
    rng = np.random.default_rng(bs)
    nbr, nbc = 150, 50
    P = sp.random(nbr * bs, nbc * bs, density=0.15, random_state=bs, format="csr")
    P.data = np.abs(rng.standard_normal(P.data.size)) + 0.1
    T = amg.truncate_prolongator(P, bs, 0.3, 4).toarray()
    Pd = P.toarray()
    R = np.zeros_like(Pd)
    for i in range(nbr):
        rows = slice(i * bs, (i + 1) * bs)
        blocks = [(j, Pd[rows, j * bs:(j + 1) * bs]) for j in range(nbc)]
        blocks = [(j, b) for j, b in blocks if np.any(b != 0)]
        if not blocks:
            continue
        m = max(np.linalg.norm(b) for _, b in blocks)
        cand = sorted(((np.linalg.norm(b), j, b) for j, b in blocks if np.linalg.norm(b) >= 0.3 * m),
                      key=lambda t: (-t[0], t[1]))[:4]
        skept = sum(b.sum(axis=1) for _, _, b in cand)
        # a scalar row whose kept part sums to zero keeps its values
        sc = np.ones(bs)
        nzk = skept != 0
        sc[nzk] = Pd[rows].sum(axis=1)[nzk] / skept[nzk]
        for _, j, b in cand:
            R[rows, j * bs:(j + 1) * bs] = b * sc[:, None]
    assert np.allclose(T, R, rtol=1e-13, atol=1e-15)
    # row sums are preserved wherever a kept entry carries them
    keep_rows = np.abs(T).sum(axis=1) > 0
    assert np.allclose(T.sum(axis=1)[keep_rows], Pd.sum(axis=1)[keep_rows])


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_chebyshev_smoother_is_the_chebyshev_polynomial(degree):
    """With b = 0 the smoother maps an eigenvector of D^{-1}A with eigenvalue
    mu to p(mu) times itself, p(mu) = T_k((theta - mu)/delta) / T_k(theta/delta)
    on [lam/30, lam] (closed form of Chebyshev acceleration)."""
    n = 40
    L = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    dinv = 1.0 / L.diagonal()
    lam = 2.2
    j = np.arange(1, n + 1)
    for k in (1, 7, 23, 40):
        v = np.sin(np.pi * k * j / (n + 1))
        mu = 1.0 - np.cos(np.pi * k / (n + 1))
        x = amg.cheb_smooth(L, dinv, lam, degree, v.copy(), np.zeros(n), False)
        lo, hi = lam / 30, lam
        theta, delta = (hi + lo) / 2, (hi - lo) / 2
        Tk = lambda t: np.polynomial.chebyshev.chebval(t, [0] * degree + [1])
        p = Tk((theta - mu) / delta) / Tk(theta / delta)
        assert np.allclose(x, p * v, rtol=1e-10, atol=1e-12)


def test_power_lambda_converges_to_spectral_radius():
    n = 20
    L = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    rho = 1.0 - np.cos(np.pi * n / (n + 1))   # largest eigenvalue of D^{-1} L
    est = amg.power_lambda(L, 1.0 / L.diagonal(), iters=400) / 1.1
    assert abs(est - rho) < 1e-3
    assert amg.power_lambda(L, 1.0 / L.diagonal()) / 1.1 <= rho + 1e-12


def test_vcycle_chebyshev_contracts_on_spd(mini_system):
    L = to_csr(mini_system.L)
    H = amg.setup(L, 1, 0.08, 10, 16, 1, 1, 0.3, 5, "cheb", 3)
    n = L.shape[0]
    Ld = L.toarray()
    M = np.column_stack([amg.vcycle(H, np.eye(n)[:, j]) for j in range(n)])
    E = np.eye(n) - M @ Ld
    w, V = np.linalg.eigh(Ld)
    Lh = V @ np.diag(np.sqrt(w)) @ V.T
    Lhi = V @ np.diag(1 / np.sqrt(w)) @ V.T
    assert np.linalg.norm(Lh @ E @ Lhi, 2) < 0.5
    assert np.allclose(M, M.T, atol=1e-10 * np.abs(M).max())


def test_two_level_exact_on_constant_near_nullspace():
    # 1-D Laplacian: the V-cycle reduces a smooth error far better than one
    # Jacobi sweep (checks the coarse-grid correction is wired in)
    n = 200
    L = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    H = amg.setup(L, 1, 0.08, 10, 8, 1, 1)
    x = np.sin(np.pi * np.arange(1, n + 1) / (n + 1))
    b = L @ x
    e_v = np.linalg.norm(x - amg.vcycle(H, b)) / np.linalg.norm(x)
    e_j = np.linalg.norm(x - b / np.abs(L).sum(axis=1).A1) / np.linalg.norm(x)
    assert e_v < 0.5 * e_j


# ------------------------------------------------------------- scr
def test_algorithm2_matches_schur_definition(tiny_system):
    opts = scr.SolverOptions(rtol_I=1e-13, max_I=400, restart_inner=60)
    s = scr.SCRSolver(tiny_system, opts)
    S = schur.schur_exact_dense(s.op)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(s.op.np)
    assert np.allclose(s.apply_S(x), S @ x, rtol=1e-8, atol=1e-9 * np.abs(S @ x).max())


def test_algorithm1_with_tight_inner_is_inverse(tiny_system):
    opts = scr.SolverOptions(rtol_A=1e-13, rtol_S=1e-13, rtol_I=1e-14, max_A=400, max_S=400,
                             max_I=400, restart_inner=80)
    s = scr.SCRSolver(tiny_system, opts)
    rng = np.random.default_rng(7)
    r = rng.standard_normal(s.op.n)
    y = s.apply_pc(r)
    yd = np.linalg.solve(s.op.full().toarray(), r)
    assert np.linalg.norm(y - yd) <= 1e-7 * np.linalg.norm(yd)


def test_full_solve_matches_direct(mini_system, mini_direct):
    s = scr.SCRSolver(mini_system)
    x, info = s.solve(mini_system.b)
    assert info.converged
    assert s.rel_residual(x, mini_system.b) <= 1e-8
    assert np.linalg.norm(x - mini_direct) <= 1e-6 * np.linalg.norm(mini_direct)
    assert 1 <= info.iters <= 10


def test_mesh_cg_matches_direct(mini_system):
    m = scr.MeshSolver(mini_system, scr.SolverOptions(mm_rtol=1e-12))
    u, info = m.solve(mini_system.mesh_b)
    assert info.converged
    ud = direct.solve_mesh(mini_system)
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)


# ---------------------------------------------------------------- storage formats
def test_bf16_rounding_special_values():
    from oracle.precision import round_bf16
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    x = np.array([1.0, 1.0 + 2.0**-8, 1.0 + 3 * 2.0**-8, -2.5, 0.0, 1.0 + 2.0**-9, 65280.0 + 128.0])
    want = np.array([1.0, 1.0, 1.0 + 2.0**-6, -2.5, 0.0, 1.0, 65536.0])
    np.testing.assert_array_equal(round_bf16(x), want)


def test_bf16_rounding_matches_torch_and_error_bound():
    """Against an independent implementation (PyTorch's binary32 -> bfloat16
    cast, round to nearest even) and the format's error bound 2^-8."""
    torch = pytest.importorskip("torch")
    from oracle.precision import round_bf16, round_f32
    rng = np.random.default_rng(7)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(round_bf16(x), ref)
    assert np.all(np.abs(round_bf16(x) - x) <= 2.0**-8 * np.abs(x) * (1 + 2.0**-20))
    assert np.all(np.abs(round_f32(x) - x) <= 2.0**-24 * np.abs(x))


# ------------------------------------------------------------- SIMPLEC
def test_simplec_identity(tiny_system):
    """P_SIMPLEC in factored form equals its closed form [[A, A D_c^{-1} B], [C, D]]."""
    op = BlockOperator.from_system(tiny_system)
    P1 = schur.simple_matrix_dense(op, lumped=True)
    P2 = schur.simple_factored_dense(op, lumped=True)
    assert np.allclose(P1, P2, rtol=1e-9, atol=1e-12 * np.abs(P1).max())
    # the lumped diagonal dominates |diag(A)| and differs from it on this system
    d, dl = schur.simple_diagonal(op), schur.simple_diagonal(op, lumped=True)
    assert np.all(dl >= np.abs(d)) and np.any(dl > np.abs(d) * (1 + 1e-6))


def test_simplec_reduces_to_simple_for_a_diagonal_A(tiny_system):
    """With a diagonal A (positive entries) the lumped diagonal is diag(A):
    SIMPLEC and SIMPLE coincide, including P^{-1} r."""
    op = BlockOperator.from_system(tiny_system)
    opd = BlockOperator.from_system(tiny_system)
    opd.A = sp.diags(np.abs(op.A.diagonal()) + 1.0).tocsr()
    assert np.array_equal(schur.simple_diagonal(opd, lumped=True), schur.simple_diagonal(opd))
    r = np.random.default_rng(3).standard_normal(opd.n)
    y1 = schur.simple_inverse_apply_dense(opd, r)
    y2 = schur.simple_inverse_apply_dense(opd, r, lumped=True)
    assert np.allclose(y1, y2, rtol=1e-12, atol=1e-12 * np.abs(y1).max())


def test_simplec_apply_with_tight_solves(tiny_system):
    opts = scr.SolverOptions(rtol_A=1e-13, rtol_S=1e-13, max_A=400, max_S=400, restart_inner=80,
                             precond="simplec")
    s = scr.SCRSolver(tiny_system, opts)
    r = np.random.default_rng(10).standard_normal(s.op.n)
    y = s.apply_simple(r)
    yd = schur.simple_inverse_apply_dense(s.op, r, lumped=True)
    assert np.linalg.norm(y - yd) <= 1e-8 * np.linalg.norm(yd)
    P = schur.simple_matrix_dense(s.op, lumped=True)
    assert np.linalg.norm(P @ yd - r) <= 1e-9 * np.linalg.norm(r)


def test_simplec_full_solve_matches_direct(mini_system, mini_direct):
    s = scr.SCRSolver(mini_system, scr.SolverOptions(precond="simplec"))
    x, info = s.solve(mini_system.b)
    assert info.converged
    assert s.rel_residual(x, mini_system.b) <= 1e-8
    assert np.linalg.norm(x - mini_direct) <= 1e-6 * np.linalg.norm(mini_direct)


# ------------------------------------------------------------- Chebyshev guard
def test_cheb_guard_keeps_chebyshev_on_spd_and_switches_on_rotation():
    """The guard's test (5 homogeneous Chebyshev sweeps from the fixed start
    vector) contracts for a 1D Laplacian and blows up for a matrix whose
    D^{-1} A has complex eigenvalues 1 +- a i (2x2 rotation blocks), far off
    the real interval the polynomial damps."""
    n = 200
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    d = 1.0 / T.diagonal()
    assert amg.cheb_guard_growth(T, d, amg.power_lambda(T, d), 3) <= 1.0
    for a in (0.5, 3.0):
        R = sp.block_diag([sp.csr_matrix(np.array([[1.0, a], [-a, 1.0]]))] * (n // 2)).tocsr()
        d = 1.0 / R.diagonal()
        assert amg.cheb_guard_growth(R, d, amg.power_lambda(R, d), 3) > amg.CHEB_GUARD_GROWTH


def test_cheb_guard_decisions_on_the_tube(tiny_system):
    """Default tube: every level of every hierarchy keeps Chebyshev; a stiff,
    heavy wall (rho_s = 100) makes level 1 of the Shat hierarchy switch to
    l1-Jacobi, and the preconditioned GMRES on Shat then converges."""
    s = F.tube_system("tube_small")
    op = BlockOperator.from_system(s)
    for M, bs in ((op.A, 3), (schur.schur_hat(op), 1), (to_csr(s.L), 1)):
        H = amg.setup(M, bs, 0.08, 10, 64, 1, 1, 0.3, 5, "cheb", 3)
        assert all(lv.cheb for lv in H.levels[:-1])
    s = F.tube_system("tube_small", rho_s=100.0)
    Sh = schur.schur_hat(BlockOperator.from_system(s))
    H = amg.setup(Sh, 1, 0.08, 10, 64, 1, 1, 0.3, 5, "cheb", 3)
    assert [lv.cheb for lv in H.levels[:-1]] == [True, False, True]
    b = np.random.default_rng(0).standard_normal(Sh.shape[0])
    _, info = krylov.gmres(lambda v: Sh @ v, b, lambda v: amg.vcycle(H, v), tol=1e-3, maxit=200, restart=30)
    assert info.converged
    del tiny_system


def test_direct_solve_of_several_right_hand_sides(mini_system, mini_direct):
    op = BlockOperator.from_system(mini_system)
    rng = np.random.default_rng(21)
    rhs = [mini_system.b, rng.standard_normal(op.n), 2.0 * mini_system.b]
    xs = direct.solve_block_many(mini_system, rhs)
    assert np.allclose(xs[0], mini_direct, rtol=0, atol=1e-12 * np.abs(mini_direct).max())
    assert np.allclose(xs[2], 2.0 * mini_direct, rtol=0, atol=1e-11 * np.abs(mini_direct).max())
    assert rel_residual(op, xs[1], rhs[1]) <= 1e-10


# ---------------------------------------------------------------- resistance outlet
def test_outlet_term_in_the_block_operator():
    """calA with a resistance outlet: the momentum block acts as
    A v + c a (a^T v) (checked against that expression), its diagonal gains
    c a_i^2 (enters Shat), and the SCR-FGMRES solve of the oracle matches the
    direct solve of the full system."""
    s = F.tube_system("tube_mini", outlet_resistance=2.7e4)
    op = BlockOperator.from_system(s)
    a, c = s.a_out[0], s.c_out[0]
    v = np.random.default_rng(5).standard_normal(op.nv)
    assert np.allclose(op.A @ v, op.A_sparse @ v + c * a * (a @ v), rtol=1e-13, atol=1e-13 * np.abs(op.A @ v).max())
    assert np.allclose(op.A.diagonal(), op.A_sparse.diagonal() + c * a * a, rtol=1e-14)
    assert np.any(c * a * a > 1e-3 * np.abs(op.A_sparse.diagonal()))
    x_ref = direct.solve_block(s)
    sol = scr.SCRSolver(s)
    x, info = sol.solve(s.b)
    assert info.converged and rel_residual(op, x, s.b) <= 1e-8
    assert np.linalg.norm(x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)


# ---------------------------------------------------------------- multi-corrector
def test_corrector_starts_from_the_system_rhs_and_contracts():
    """The oracle's corrector evaluates b = -R at the assembly state, which is
    the block system's right-hand side; with the consistent tangent
    (alpha_m dR/dvdot + alpha_f gamma dt dR/dy, frozen tau) and the matching
    generalized-alpha updates the residual drops by orders of magnitude per
    iteration (a wrong weight or sign in the update would stall it)."""
    from oracle import corrector
    s = F.tube_system("tube_mini", keep_mesh=True)
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_mini"]))
    v, p = asm.initial_state()
    nn = s.mesh.n_nodes
    *_, norms = corrector.corrector(s, asm, v, p, np.zeros(3 * nn), np.zeros(3 * nn), 3)
    assert norms[0] == pytest.approx(np.linalg.norm(s.b), rel=1e-13)
    assert norms[1] < 1e-3 * norms[0] and norms[2] < 1e-2 * norms[1] and norms[3] < norms[2]
    am, cf, cu = corrector.genalpha_weights(0.5, 1e-4)
    assert am == pytest.approx(5.0 / 6.0) and cf == pytest.approx(4.0 / 9.0 * 1e-4)
    assert cu == pytest.approx(cf * cf / am)


def test_corrector_with_a_resistance_outlet_contracts():
    """With the outlet traction in the residual and its rank-1 derivative in
    the tangent, the corrector starts from the system's right-hand side and
    contracts as fast as without outlets."""
    from oracle import corrector
    s = F.tube_system("tube_mini", keep_mesh=True, outlet_resistance=2.7e4)
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_mini"]))
    v, p = asm.initial_state()
    nn = s.mesh.n_nodes
    *_, norms = corrector.corrector(s, asm, v, p, np.zeros(3 * nn), np.zeros(3 * nn), 2)
    assert norms[0] == pytest.approx(np.linalg.norm(s.b), rel=1e-12)
    assert norms[1] < 1e-3 * norms[0] and norms[2] < 1e-2 * norms[1]


# ------------------------------------------------- mesh motion inside the corrector
def _ale_case(name="tube_mini"):
    s = F.tube_system(name, keep_mesh=True)
    asm = F.Assembler(F.make_params(**F.PRESETS[name]))
    return s, asm, to_csr(asm.mesh_laplacian()), F.interface_follow(s.mesh)


def test_mesh_displacement_reproduces_linear_fields():
    """Linear finite elements reproduce linear functions, so the harmonic
    extension (Sec. 5.2.2) of linear Dirichlet data is that linear field at
    every fluid node: a wrong sign in the lift, a swapped free/Dirichlet
    block or a component mix-up breaks it."""
    from oracle import corrector
    s, asm, L, _ = _ale_case()
    m = s.mesh
    nodes = np.flatnonzero(m.fluid_id >= 0)
    X = np.zeros((m.n_fluid, 3))
    X[m.fluid_id[nodes]] = m.xyz[nodes]
    G = np.array([[0.3, -1.1, 0.2], [0.5, 0.7, -0.4], [-0.2, 0.1, 0.9]])
    want = X @ G.T + np.array([1e-3, -2e-3, 5e-4])
    g = np.where(m.dir_m[:, None], want, 123.0).ravel()  # free entries must be ignored
    uh = corrector.mesh_displacement(L, m.dir_m, g)
    np.testing.assert_allclose(uh, want.ravel(), rtol=0, atol=1e-12 * np.abs(want).max())


def test_mesh_velocity_keeps_a_constant_rate_and_drops_the_old_rate():
    """Step 4 with the generalized-alpha update (Sec. 3.4): a mesh moving at
    a constant rate w keeps vhat = w at t_{n+1} and t_{n+alpha_f}; with
    alpha_f = gamma the intermediate mesh velocity is (uhat_{n+1} - uhat_n) / dt
    whatever vhat_n is."""
    from oracle import corrector
    rng = np.random.default_rng(5)
    dt, t = 1e-4, 0.37
    w = rng.standard_normal(30)
    for rho in (0.0, 0.5, 1.0):
        v1, va = corrector.mesh_velocity(w * (t + dt), w * t, w, rho, dt)
        np.testing.assert_allclose(v1, w, rtol=1e-9)
        np.testing.assert_allclose(va, w, rtol=1e-9)
        u1, u0, vn = (rng.standard_normal(30) for _ in range(3))
        _, va = corrector.mesh_velocity(u1, u0, vn, rho, dt)
        np.testing.assert_allclose(va, (u1 - u0) / dt, rtol=1e-9)


def test_corrector_ale_without_interface_motion_is_the_fixed_mesh_loop():
    """No node follows the wall and uhat_n = 0: the mesh stays put, the mesh
    velocity is zero and the loop is the fixed-mesh corrector."""
    from oracle import corrector
    s, asm, L, follow = _ale_case()
    m = s.mesh
    v, p = asm.initial_state()
    z, zf = np.zeros(3 * m.n_nodes), np.zeros(3 * m.n_fluid)
    ref = corrector.corrector(s, asm, v, p, z, z, 2)
    got = corrector.corrector_ale(s, asm, v, p, z, z, 2, L, m.fluid_id, m.dir_m, 0 * follow, zf,
                                  np.random.default_rng(1).standard_normal(3 * m.n_fluid))
    for a, b in zip(ref[:4], got[:4]):  # zero vhat vs none: rounding of near-zero entries only
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13 * np.abs(a).max())
    np.testing.assert_allclose(ref[4], got[5], rtol=1e-13, atol=1e-13 * ref[4][0])
    assert not got[4].any()


def test_corrector_ale_moves_the_mesh_with_the_wall_and_contracts():
    """With the interface following the wall the corrector still starts from
    the system's right-hand side and contracts by orders of magnitude per
    iteration (the tangent leaves out only the weak mesh-velocity coupling);
    the final mesh displacement equals u_{n+1} = u_n + (u - u_n) / alpha_f on
    the interface and zero on the other Dirichlet nodes, the wall moved, and
    vhat_n drops out (alpha_f = gamma)."""
    from oracle import corrector
    s, asm, L, follow = _ale_case()
    m = s.mesh
    v, p = asm.initial_state()
    z, zf = np.zeros(3 * m.n_nodes), np.zeros(3 * m.n_fluid)
    vn = np.random.default_rng(2).standard_normal(3 * m.n_fluid)
    vr, pr, vdr, ur, uh, norms = corrector.corrector_ale(s, asm, v, p, z, z, 3, L, m.fluid_id, m.dir_m,
                                                         follow, zf, vn)
    assert norms[0] == pytest.approx(np.linalg.norm(s.b), rel=1e-12)
    assert norms[1] < 1e-2 * norms[0] and norms[2] < 1e-2 * norms[1] and norms[3] < 1e-2 * norms[2]
    af = 1.0 / (1.0 + s.params["rho_inf"])
    nodes = np.flatnonzero(m.fluid_id >= 0)
    U = uh.reshape(-1, 3)
    u1 = ur.reshape(-1, 3)[nodes] / af
    f = m.fluid_id[nodes]
    on = follow[f].astype(bool)
    np.testing.assert_allclose(U[f[on]], u1[on], rtol=0, atol=1e-15)
    assert not U[m.dir_m & ~follow.astype(bool)].any()
    assert np.abs(U[f[on]]).max() > 1e-6
    *_, norms0 = corrector.corrector_ale(s, asm, v, p, z, z, 3, L, m.fluid_id, m.dir_m, follow, zf, zf)
    np.testing.assert_allclose(norms, norms0, rtol=1e-9, atol=1e-13 * norms[0])


# ------------------------------------------------- AMG building blocks, one by one
def test_chebyshev_residual_polynomial_is_the_scaled_chebyshev_polynomial():
    """Chebyshev smoothing of degree k from a zero iterate leaves the residual
    T_k((theta - lambda) / delta) / T_k(theta / delta) b for an operator with
    eigenvalue lambda (theta, delta: centre and half-width of [lam/30, lam]):
    checked on a diagonal operator against numpy's Chebyshev series, with
    D = I and with a general diagonal scaling (the smoother works on D^-1 A)."""
    from numpy.polynomial import chebyshev as npc
    from oracle import amg
    lam = 3.7
    lo, hi = lam / 30.0, lam
    theta, delta = (hi + lo) / 2.0, (hi - lo) / 2.0
    mu = np.concatenate([np.linspace(lo, hi, 9), [0.3 * lo, 1.2 * hi]])  # eigenvalues of D^-1 A
    for degree in (1, 2, 3, 4):
        Tk = npc.Chebyshev.basis(degree)
        want = Tk((theta - mu) / delta) / Tk(theta / delta)
        for d in (np.ones(mu.size), np.linspace(0.5, 2.0, mu.size)):
            A = sp.diags(mu * d).tocsr()          # D^-1 A = diag(mu) with D = diag(d)
            b = np.linspace(1.0, 2.0, mu.size)
            x = amg.cheb_smooth(A, 1.0 / d, lam, degree, np.zeros_like(b), b, True)
            np.testing.assert_allclose((b - A @ x) / b, want, rtol=1e-10, atol=1e-13)
            # from a nonzero iterate the error contracts by the same polynomial
            x0 = np.cos(np.arange(mu.size))
            xs = b / A.diagonal()
            x1 = amg.cheb_smooth(A, 1.0 / d, lam, degree, x0, b, False)
            np.testing.assert_allclose((x1 - xs) / (x0 - xs), want, rtol=1e-9, atol=1e-12)


def test_l1_jacobi_diagonal_dominates_an_spd_matrix():
    """d_i = sum_j |a_ij| (row sums of absolute values, diagonal included) on a
    hand example, and for SPD A the l1-Jacobi iteration converges: D_l1 - A
    is weakly diagonally dominant, so every eigenvalue of D_l1^-1 A lies in
    (0, 1]."""
    from oracle import amg
    M = sp.csr_matrix(np.array([[4.0, -1.0, 2.0], [0.0, 3.0, -3.0], [1.0, 1.0, -5.0]]))
    np.testing.assert_array_equal(amg.l1_diag(M), [7.0, 6.0, 7.0])
    rng = np.random.default_rng(11)
    Q = rng.standard_normal((30, 30))
    A = Q @ Q.T + 0.1 * np.eye(30)
    A[np.abs(A) < 2.0] = 0.0
    w = np.linalg.eigvalsh(A)
    if w.min() <= 0:
        A += (1e-3 - w.min()) * np.eye(30)
    d = amg.l1_diag(sp.csr_matrix(A))
    ev = np.linalg.eigvals(A / d[:, None])
    assert ev.real.min() > 0 and ev.real.max() <= 1.0 + 1e-12 and np.abs(ev.imag).max() < 1e-10


def test_gershgorin_bound_holds_and_is_tight_on_a_singular_laplacian():
    """max_i sum_j |a_ij| / |a_ii| bounds the spectral radius of D^-1 A (random
    nonsymmetric matrices) and equals it for the 1-D Neumann Laplacian, whose
    D^-1 A has the eigenvalue 2 (the alternating vector)."""
    from oracle import amg
    rng = np.random.default_rng(12)
    for _ in range(5):
        A = rng.standard_normal((25, 25)) * (rng.random((25, 25)) < 0.2) + np.diag(rng.uniform(1, 3, 25))
        rho = np.abs(np.linalg.eigvals(A / np.diag(A)[:, None])).max()
        assert amg.gershgorin_dinv_a(sp.csr_matrix(A)) >= rho - 1e-12
    n = 12
    L = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil()
    L[0, 0] = L[n - 1, n - 1] = 1.0
    L = L.tocsr()
    rho = np.abs(np.linalg.eigvals(L.toarray() / L.diagonal()[:, None])).max()
    assert amg.gershgorin_dinv_a(L) == pytest.approx(2.0) and rho == pytest.approx(2.0)


def test_smoothed_prolongator_keeps_the_near_nullspace_and_lowers_the_energy():
    """Prolongator smoothing (Sec. 7: smoothed aggregation): where A
    annihilates the near-nullspace (constants of the Neumann Laplacian),
    P B_c = P_tent B_c = 1; omega = 4 / (3 lambda) with lambda = 2 there; and
    damped Jacobi lowers the energy p^T A p of every coarse basis function
    (a wrong sign raises it)."""
    from oracle import amg
    n = 30
    L = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil()
    L[0, 0] = L[n - 1, n - 1] = 1.0
    L = L.tocsr()
    agg = np.arange(n) // 3
    Pt = amg.tentative_prolongator(agg, 1)
    Bc = np.sqrt(np.bincount(agg).astype(float))
    np.testing.assert_allclose(Pt @ Bc, np.ones(n), rtol=1e-14)
    P, omega = amg.smoothed_prolongator(L, Pt)
    assert omega == pytest.approx(2.0 / 3.0)
    np.testing.assert_allclose(P @ Bc, np.ones(n), rtol=1e-13)
    e_t = np.asarray((Pt.T @ (L @ Pt)).diagonal()).ravel()
    e_s = np.asarray((P.T @ (L @ P)).diagonal()).ravel()
    assert np.all(e_s < e_t)


def test_strength_graph_by_brute_force():
    """Block rows i != j are strongly connected when ||A_ij||_F >= theta
    sqrt(||A_ii||_F ||A_jj||_F) in either direction (the graph is
    symmetrised), checked pair by pair with dense blocks on a random
    3x3-block matrix; the edge weight is the larger block norm of the pair."""
    from oracle import amg
    rng = np.random.default_rng(13)
    n, bs, theta = 40, 3, 0.3
    mask = rng.random((n, n)) < 0.15
    np.fill_diagonal(mask, True)
    D = np.zeros((n * bs, n * bs))
    for i, j in zip(*np.nonzero(mask)):
        blk = rng.standard_normal((bs, bs)) * (3.0 if i == j else rng.uniform(0.05, 1.5))
        D[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = blk
    S = amg.strength_graph(sp.csr_matrix(D), bs, theta).toarray()
    nrm = np.array([[np.linalg.norm(D[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]) for j in range(n)]
                    for i in range(n)])
    want = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            strong_ij = nrm[i, j] > 0 and nrm[i, j] >= theta * np.sqrt(nrm[i, i] * nrm[j, j])
            strong_ji = nrm[j, i] > 0 and nrm[j, i] >= theta * np.sqrt(nrm[i, i] * nrm[j, j])
            w = max(nrm[i, j] if strong_ij else 0.0, nrm[j, i] if strong_ji else 0.0)
            want[i, j] = w
    np.testing.assert_allclose(S, want, rtol=1e-14)
    assert (want > 0).sum() > n  # the case has strong and weak pairs
    assert ((nrm > 0) & (want == 0) & ~np.eye(n, dtype=bool)).any()


# ------------------------------------------------------------- bifurcation
def test_bifurcation_scr_and_mesh_cg_match_direct():
    """On the bifurcation (parent, carina tip, two sheared half-disk
    daughters) the oracle's SCR-FGMRES meets 1e-8 and matches the direct
    solve, and the mesh CG + AMG matches the direct mesh solve."""
    s = F.tube_system("bif_mini", keep_mesh=True)
    assert np.isfinite(s.b).all() and np.isfinite(s.mesh_b).all()
    xd = direct.solve_block(s)
    sol = scr.SCRSolver(s)
    x, info = sol.solve(s.b)
    assert info.converged and sol.rel_residual(x, s.b) <= 1e-8
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    assert 1 <= info.iters <= 10
    m = scr.MeshSolver(s, scr.SolverOptions(mm_rtol=1e-12))
    u, minfo = m.solve(s.mesh_b)
    ud = direct.solve_mesh(s)
    assert minfo.converged and np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)


# ---------------------------------------------------------------- fixed-count A solves
def test_richardson_closed_form():
    """k Richardson steps with a linear preconditioner M = omega I equal the
    closed form x_k = V diag((1 - (1 - omega lam)^k) / lam) V^T b from the
    eigen-decomposition of an SPD A (the truncated Neumann series of A^{-1})."""
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.linspace(0.5, 3.0, 12)
    A = (Q * lam) @ Q.T
    b = rng.standard_normal(12)
    omega = 0.4
    for k in (1, 2, 5):
        x = krylov.richardson(lambda v: A @ v, b, lambda v: omega * v, k)
        ref = Q @ (((1.0 - (1.0 - omega * lam) ** k) / lam) * (Q.T @ b))
        assert np.allclose(x, ref, rtol=1e-12, atol=1e-14)
    # an exact preconditioner solves in one step, and further steps keep it
    Ainv = np.linalg.inv(A)
    for k in (1, 3):
        x = krylov.richardson(lambda v: A @ v, b, lambda v: Ainv @ v, k)
        assert np.allclose(A @ x, b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("inner,inter", [(2, 0), (3, 2), (1, 1)])
def test_scr_with_fixed_count_a_solves_matches_direct(mini_system, mini_direct, inner, inter):
    """With Algorithm 2's inner A solve (and Algorithm 1's A solves) replaced
    by a few V-cycle Richardson steps, the flexible outer FGMRES still meets
    1e-8 and the direct solution to 1e-6."""
    s = mini_system
    out = scr.solve_system(s, scr.SolverOptions(inner_vcycles=inner, inter_vcycles=inter))
    op = BlockOperator.from_system(s)
    assert out["info"].converged
    assert rel_residual(op, out["x"], s.b) <= 1e-8
    assert np.linalg.norm(out["x"] - mini_direct) <= 1e-6 * np.linalg.norm(mini_direct)
    assert out["counters"].i_iters % inner == 0


# ---------------------------------------------------------------- tangent at a state
def test_tangent_at_the_initial_state_is_the_input_system():
    """The oracle's Jacobian at a state, at the generator's assembly state,
    equals the block system the input module builds (the same element loop
    and the same Dirichlet convention: identity rows of A, rows of B and
    columns of A and C removed at Dirichlet velocity nodes)."""
    from oracle import corrector
    s = F.tube_system("tube_mini", keep_mesh=True)
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_mini"]))
    v, p = asm.initial_state()
    A, B, C, D = corrector.tangent(s, asm, v, p)
    for got, want in ((A, s.A), (B, s.B), (C, s.C), (D, s.D)):
        w = to_csr(want)
        assert abs(got - w).max() <= 1e-14 * abs(w).max()
    dv = np.repeat(s.mesh.dir_v, 3)
    assert np.all(A.diagonal()[dv] == 1.0)
    assert abs(A[dv][:, ~dv]).max() == 0 and abs(A[~dv][:, dv]).max() == 0
    assert abs(B[dv]).max() == 0 and abs(C[:, dv]).max() == 0


def test_tangent_is_the_derivative_of_the_residual_at_a_moved_state():
    """At a state away from the assembly state (perturbed velocity, pressure,
    mesh velocity, rates and solid displacement), the tangent's action on an
    increment equals the central difference of the residual along the
    generalized-alpha update of that increment (rates by alpha_m, values by
    alpha_f gamma dt, the displacement by (alpha_f gamma dt)^2 / alpha_m),
    with tau frozen at the state: free rows of the momentum and mass
    residuals."""
    from oracle import corrector
    s = F.tube_system("tube_mini", keep_mesh=True)
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_mini"]))
    v0, p0 = asm.initial_state()
    rng = np.random.default_rng(11)
    nn = s.mesh.n_nodes
    v = v0 + 2.0 * rng.standard_normal(v0.size)
    p = p0 + 10.0 * rng.standard_normal(p0.size)
    vd = 50.0 * rng.standard_normal(3 * nn)
    vh = 1.0 * rng.standard_normal(3 * nn)
    A, B, C, D = corrector.tangent(s, asm, v, p, vd, vh)
    am, cf, cu = corrector.genalpha_weights(s.params["rho_inf"], s.params["dt"])
    dv = np.repeat(s.mesh.dir_v, 3)
    xv = rng.standard_normal(3 * nn)
    xv[dv] = 0.0
    xp = rng.standard_normal(p.size)
    tau = np.zeros(8 * s.mesh.n_elem)
    asm.evaluate(v, p, vd=vd, vhat=vh, tau=tau, tau_mode=1, want_mat=False)
    h = 1e-4  # the increments are scaled by alpha_f gamma dt: the state moves by about 1e-8
    u = 1e-3 * rng.standard_normal(3 * nn)
    R = [asm.evaluate(v + sg * h * cf * xv, p + sg * h * cf * xp, vd=vd + sg * h * am * xv,
                      u=u + sg * h * cu * xv, vhat=vh, tau=tau, tau_mode=2, want_mat=False) for sg in (1.0, -1.0)]
    dRm = (R[0]["Rm"] - R[1]["Rm"]) / (2 * h)
    dRp = (R[0]["Rp"] - R[1]["Rp"]) / (2 * h)
    Km = A @ xv + B @ xp
    Kp = C @ xv + D @ xp
    assert np.linalg.norm(Km[~dv] - dRm[~dv]) <= 1e-6 * np.linalg.norm(dRm[~dv])
    assert np.linalg.norm(Kp - dRp) <= 1e-6 * np.linalg.norm(dRp)


def test_newton_corrector_first_step_is_the_frozen_one_and_it_contracts():
    """Re-assembling the tangent at every iteration: the first iteration
    uses the tangent at the initial state, so it matches the frozen-tangent
    loop; later iterations keep contracting the residual."""
    from oracle import corrector
    s = F.tube_system("tube_mini", keep_mesh=True)
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_mini"]))
    v, p = asm.initial_state()
    z = np.zeros(3 * s.mesh.n_nodes)
    *_, nf = corrector.corrector(s, asm, v, p, z, z, 1)
    *_, nn_ = corrector.corrector(s, asm, v, p, z, z, 3, newton=True)
    assert nn_[0] == pytest.approx(nf[0], rel=1e-14) and nn_[1] == pytest.approx(nf[1], rel=1e-9)
    assert nn_[2] < 1e-2 * nn_[1] and nn_[3] < nn_[2]


def test_truncation_to_a_given_pattern():
    """Truncating to the pattern the truncation itself selects reproduces
    it exactly; on another matrix with the same block pattern it keeps those
    positions and every scalar row sum (the rescaling of step 4)."""
    s = F.tube_system("tube_mini")
    A = to_csr(s.A)
    S = amg.strength_graph(A, 3, 0.08)
    agg = amg.aggregate_greedy(S)
    Pt = amg.tentative_prolongator(agg, 3)
    P, _ = amg.smoothed_prolongator(A, Pt)
    Pk = amg.truncate_prolongator(P, 3, 0.3, 5)
    Bk = sp.bsr_matrix(Pk, blocksize=(3, 3))
    Bk.sort_indices()
    got = amg.truncate_to_pattern(P, 3, Bk.indptr, Bk.indices)
    assert abs(got - Pk).max() <= 1e-15 * abs(Pk).max()
    A2 = (A + sp.diags(0.1 * np.abs(A.diagonal()))).tocsr()
    P2, _ = amg.smoothed_prolongator(A2, Pt)
    got2 = amg.truncate_to_pattern(P2, 3, Bk.indptr, Bk.indices)
    B2 = sp.bsr_matrix(got2, blocksize=(3, 3))
    B2.sort_indices()
    assert np.array_equal(B2.indptr, Bk.indptr) and np.array_equal(B2.indices, Bk.indices)
    assert np.allclose(np.asarray(got2.sum(axis=1)).ravel(), np.asarray(P2.sum(axis=1)).ravel(), rtol=1e-12, atol=1e-14)

