"""Parity of the CUDA path with the CPU oracle (needs a GB300).

Every call goes through the C ABI (the thin binding).  Tolerances:
- block products, Shat, prolongators, Galerkin operators, V-cycles: FP64
  rounding with a different summation order, 1e-12 relative (1e-5 for the
  FP32 preconditioner copies);
- the block solve (the paper's method reaches x* = calA^{-1} b only up to
  the outer tolerance): ||x - x*|| / ||x*|| <= 1e-6 and
  ||b - calA x|| / ||b|| <= 1e-8, recomputed by the oracle;
- the mesh CG: relative residual <= 1e-8, error vs the direct solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import fsi_inputs as F
from mis2_check import check_mis2_aggregation
from oracle import amg, direct, schur, scr
from oracle.sparse import BlockOperator, bsr_matvec_by_definition, rel_residual, to_csr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2206_06996_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _random_bsr(rng, nbr, nbc, br, bc, max_per_row=20, empty_every=7):
    rp = [0]
    cols = []
    for i in range(nbr):
        k = 0 if (empty_every and i % empty_every == 3) else int(rng.integers(1, max_per_row + 1))
        c = np.sort(rng.choice(nbc, size=min(k, nbc), replace=False))
        cols.extend(c.tolist())
        rp.append(len(cols))
    return F.BSR(br, bc, nbr, nbc, np.array(rp, np.int32), np.array(cols, np.int32),
                 rng.standard_normal(len(cols) * br * bc))


@pytest.fixture(scope="module")
def small():
    return F.tube_system("tube_small", keep_mesh=True)


@pytest.fixture(scope="module")
def small_direct(small):
    return direct.solve_block(small)


@pytest.fixture(scope="module")
def mini():
    return F.tube_system("tube_mini", keep_mesh=True)


@pytest.fixture(scope="module")
def mini_x(mini):
    return direct.solve_block(mini)


# ---------------------------------------------------------------- K1 SpMV
@pytest.mark.parametrize("br,bc", [(3, 3), (3, 1), (1, 3), (1, 1)])
@pytest.mark.parametrize("nbr", [1, 37, 1000, 4099])
def test_bsr_spmv_random(br, bc, nbr):
    rng = np.random.default_rng(nbr * 7 + br * 3 + bc)
    M = _random_bsr(rng, nbr, max(nbr // 2, 3), br, bc)
    x = rng.standard_normal(M.nb_cols * bc)
    y = pkg.bsr_spmv(pkg.DeviceBSR.from_host(M), _dev(x)).cpu().numpy()
    ref = bsr_matvec_by_definition(M, x)
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_bsr_spmv_empty_matrix():
    M = F.BSR(3, 3, 5, 5, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    y = pkg.bsr_spmv(pkg.DeviceBSR.from_host(M), _dev(np.ones(15))).cpu().numpy()
    assert np.all(y == 0.0)


def test_bsr_spmv_rejects_bad_columns():
    M = F.BSR(1, 1, 2, 2, np.array([0, 2, 3], np.int32), np.array([1, 0, 5], np.int32), np.ones(3))
    with pytest.raises(pkg.ScrError) as e:
        pkg.bsr_spmv(pkg.DeviceBSR.from_host(M), _dev(np.ones(2)))
    assert e.value.status == 1


# ---------------------------------------------------------------- K2 calA
@pytest.mark.parametrize("name", ["tube_mini", "tube_small"])
def test_block_operator(name):
    s = F.tube_system(name)
    op = BlockOperator.from_system(s)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(s.n)
    with pkg.BlockSolver() as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        y = sol.apply_op(_dev(x)).cpu().numpy()
    ref = op.matvec(x)
    assert _rel(y, ref) < 1e-13


# ---------------------------------------------------------------- K4/K5 set-up
def test_schur_hat(small):
    op = BlockOperator.from_system(small)
    ref = schur.schur_hat(op).toarray() if small.n_p < 3000 else None
    with pkg.BlockSolver() as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        Sh = sol.export(pkg.SCR_HIER_SHAT, 0, pkg.SCR_EXPORT_OPERATOR)
    got = to_csr(Sh)
    want = schur.schur_hat(op)
    diff = abs(got - want).max()
    assert diff <= 1e-12 * abs(want).max()
    # same sparsity (no structural zeros dropped or added beyond the union)
    assert got.nnz >= want.nnz - 0
    del ref


def test_schur_hat_simplec(small):
    """SIMPLEC builds Shat with the lumped diagonal (oracle: schur_hat(lumped=True))."""
    op = BlockOperator.from_system(small)
    with pkg.BlockSolver(precond=pkg.SCR_PC_SIMPLEC) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        got = to_csr(sol.export(pkg.SCR_HIER_SHAT, 0, pkg.SCR_EXPORT_OPERATOR))
    want = schur.schur_hat(op, lumped=True)
    assert abs(got - want).max() <= 1e-12 * abs(want).max()
    assert abs(got - schur.schur_hat(op)).max() > 1e-6 * abs(want).max()


def _strength_pattern(A, bs, theta):
    return amg.strength_graph(A, bs, theta)


@pytest.mark.parametrize("which,bs", [(0, 3), (1, 1), (2, 1)])
def test_aggregates_are_a_valid_mis2_aggregation(small, which, bs):
    """The GPU's MIS-2 aggregation on the first two levels of each hierarchy
    (A, Shat, the mesh Laplacian) of the small tube meets every property of
    a distance-2 maximal independent set aggregation, checked completely."""
    with pkg.BlockSolver() as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        sol.mesh_setup(small.L)
        nl = sol.amg_levels(which)
        cases = []
        for l in range(min(2, nl - 1)):
            A = to_csr(sol.export(which, l, pkg.SCR_EXPORT_OPERATOR))
            agg = sol.export(which, l, pkg.SCR_EXPORT_AGGREGATES)
            roots = sol.export(which, l, pkg.SCR_EXPORT_ROOTS)
            cases.append((A, agg, roots))
    assert cases
    for A, agg, roots in cases:
        check_mis2_aggregation(_strength_pattern(A, bs, 0.08), agg, roots)


@pytest.mark.parametrize("which,bs", [(0, 3), (1, 1), (2, 1)])
def test_prolongator_and_galerkin_operator(small, which, bs):
    with pkg.BlockSolver() as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        sol.mesh_setup(small.L)
        nl = sol.amg_levels(which)
        assert nl >= 2
        for l in range(nl - 1):
            A = to_csr(sol.export(which, l, pkg.SCR_EXPORT_OPERATOR))
            P = to_csr(sol.export(which, l, pkg.SCR_EXPORT_PROLONGATOR))
            agg = sol.export(which, l, pkg.SCR_EXPORT_AGGREGATES)
            Ac = to_csr(sol.export(which, l + 1, pkg.SCR_EXPORT_OPERATOR))
            Pt = amg.tentative_prolongator(agg.astype(np.int64), bs)
            Pref, _ = amg.smoothed_prolongator(A, Pt)
            Pref = amg.truncate_prolongator(Pref, bs, 0.3, 5)
            assert abs(P - Pref).max() <= 1e-12 * abs(Pref).max()
            Aref = (Pref.T @ A @ Pref).tocsr()
            assert abs(Ac - Aref).max() <= 1e-11 * abs(Aref).max()


@pytest.mark.parametrize("which,bs,nrhs", [(0, 3, 1), (1, 1, 1), (2, 1, 3)])
@pytest.mark.parametrize("smoother,nu,degree", [("l1", 1, 3), ("l1", 2, 3), ("cheb", 1, 3), ("cheb", 1, 2)])
def test_vcycle_matches_oracle_on_exported_hierarchy(small, which, bs, nrhs, smoother, nu, degree):
    code = 1 if smoother == "cheb" else 0
    with pkg.BlockSolver(amg_nu=nu, amg_smoother=code, amg_degree=degree) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        sol.mesh_setup(small.L)
        nl = sol.amg_levels(which)
        As = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_OPERATOR)) for l in range(nl)]
        Ps = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_PROLONGATOR)) for l in range(nl - 1)]
        H = amg.hierarchy_from_matrices(As, Ps, bs, nu, nu, smoother, degree)
        rng = np.random.default_rng(3)
        b = rng.standard_normal(As[0].shape[0] * nrhs)
        x = sol.amg_apply(which, _dev(b)).cpu().numpy()
    ref = amg.vcycle(H, b.reshape(-1, nrhs) if nrhs > 1 else b).reshape(-1)
    assert _rel(x, ref) < 1e-11


def _round_csr(M, rnd):
    M = sp.csr_matrix(M, copy=True)
    M.data = rnd(M.data)
    return M


@pytest.mark.parametrize("which,bs", [(pkg.SCR_HIER_A, 3), (pkg.SCR_HIER_SHAT, 1)])
def test_mixed_vcycle_with_bf16_coarse_levels_matches_oracle(small, which, bs):
    """Mixed form: level 0 stored in FP32, the operators and transfers of the
    coarser levels in BF16 (FP32 vectors and sums).  The oracle V-cycle with
    its matrices rounded the same way (oracle.precision) agrees to FP32
    rounding of the vectors; the unrounded FP64 V-cycle is much farther off,
    so the BF16 values are the ones the GPU used."""
    from oracle import precision
    with pkg.BlockSolver(precision=pkg.SCR_MIXED) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        nl = sol.amg_levels(which)
        assert nl >= 3
        As = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_OPERATOR)) for l in range(nl)]
        Ps = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_PROLONGATOR)) for l in range(nl - 1)]
        b = np.random.default_rng(12).standard_normal(As[0].shape[0])
        x = sol.amg_apply(which, _dev(b)).cpu().numpy()
    H = amg.hierarchy_from_matrices(As, Ps, bs, 1, 1, "cheb", 3)
    exact = amg.vcycle(H, b)
    for l, lev in enumerate(H.levels[:-1]):
        rnd = precision.round_f32 if l == 0 else precision.round_bf16
        lev.A = _round_csr(lev.A, rnd)
        lev.P = _round_csr(lev.P, rnd)
        lev.R = _round_csr(lev.R, rnd)
    ref = amg.vcycle(H, b)
    err = _rel(x, ref)
    assert err < 1e-5
    assert _rel(x, exact) > 10 * err


def test_mixed_solve_with_fp32_coarse_levels(small, small_direct):
    op = BlockOperator.from_system(small)
    with pkg.BlockSolver(precision=pkg.SCR_MIXED, amg_coarse_bf16=0) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        x = sol.solve(small.b.copy())
    assert rel_residual(op, x, small.b) <= 1e-8 and _rel(x, small_direct) <= 1e-6
    with pytest.raises(pkg.ScrError):
        pkg.BlockSolver(amg_coarse_bf16=2)


def test_vcycle_with_chebyshev_guard_matches_oracle():
    """Heavy, stiff wall (rho_s = 100): a Galerkin level of the Shat hierarchy
    fails the Chebyshev guard on both sides and is smoothed by l1-Jacobi; the
    GPU V-cycle equals the oracle's on the exported hierarchy (whose guard
    takes the same per-level decisions) and a Shat solve converges."""
    s = F.tube_system("tube_small", rho_s=100.0)
    with pkg.BlockSolver() as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        which = pkg.SCR_HIER_SHAT
        nl = sol.amg_levels(which)
        As = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_OPERATOR)) for l in range(nl)]
        Ps = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_PROLONGATOR)) for l in range(nl - 1)]
        b = np.random.default_rng(4).standard_normal(As[0].shape[0])
        x = sol.amg_apply(which, _dev(b)).cpu().numpy()
    H = amg.hierarchy_from_matrices(As, Ps, 1, 1, 1, "cheb", 3)
    assert not all(lv.cheb for lv in H.levels[:-1])
    assert _rel(x, amg.vcycle(H, b)) < 1e-11


@pytest.mark.parametrize("br,bc", [(3, 3), (1, 1)])
@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_vector_kernel_random_matrices(br, bc, G):
    """The 16-byte kernels on the padded copy (forced with spmv_group = 300 +
    G) equal the block product's definition on random matrices with empty
    rows, one-block rows and ragged row lengths (the last chunk of a row
    partly filled), over sizes spanning many CTAs."""
    with pkg.BlockSolver(spmv_group=300 + G, autotune=0):
        for nbr in (1, 37, 4099):
            rng = np.random.default_rng(nbr * 11 + G + br)
            M = _random_bsr(rng, nbr, max(nbr // 2, 3), br, bc, max_per_row=23)
            x = rng.standard_normal(M.nb_cols * bc)
            y = pkg.bsr_spmv(pkg.DeviceBSR.from_host(M), _dev(x)).cpu().numpy()
            ref = bsr_matvec_by_definition(M, x)
            assert np.allclose(y, ref, rtol=1e-13, atol=1e-13 * max(1.0, np.abs(ref).max()))
            assert np.all(y[np.repeat(np.diff(M.row_ptr) == 0, br)] == 0.0)


@pytest.mark.parametrize("which,bs", [(pkg.SCR_HIER_A, 3), (pkg.SCR_HIER_SHAT, 1)])
@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_vector_kernel_vcycle_matches_oracle(small, which, bs, G):
    """V-cycles whose level-0 products run the 16-byte kernels (A 3x3, Shat
    1x1, every smoother epilogue) equal the oracle's V-cycle on the exported
    hierarchy (FP64)."""
    with pkg.BlockSolver(spmv_group=300 + G, autotune=0) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        nl = sol.amg_levels(which)
        As = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_OPERATOR)) for l in range(nl)]
        Ps = [to_csr(sol.export(which, l, pkg.SCR_EXPORT_PROLONGATOR)) for l in range(nl - 1)]
        b = np.random.default_rng(31 + G).standard_normal(As[0].shape[0])
        x = sol.amg_apply(which, _dev(b)).cpu().numpy()
    H = amg.hierarchy_from_matrices(As, Ps, bs, 1, 1, "cheb", 3)
    assert _rel(x, amg.vcycle(H, b)) < 1e-11


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
@pytest.mark.parametrize("G", [2, 4])
def test_block_solve_with_vector_kernels_matches_direct(small, small_direct, precision, G):
    """Whole solves with the 16-byte kernels forced (FP64 and mixed) meet the
    direct solve; without the padded copy (vec = 0) the same forced code runs
    the scalar-row kernel and the two answers agree to the solve tolerance."""
    op = BlockOperator.from_system(small)
    xs = []
    for vec in (1, 0):
        with pkg.BlockSolver(precision=precision, spmv_group=300 + G, autotune=0, vec=vec) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            x = sol.solve(small.b.copy())
            st = sol.stats()
        assert st["rel_res"] <= 1e-8 and rel_residual(op, x, small.b) <= 1e-8
        assert _rel(x, small_direct) <= 1e-6
        xs.append(x)
    assert _rel(xs[0], xs[1]) <= 1e-6


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_sliced_ell_products_match_slab_products(small, precision):
    """The sliced block-ELL copies of A, Shat and L give the same V-cycles as
    the slab layout (same arithmetic per row, same order of terms)."""
    rng = np.random.default_rng(5)
    outs = []
    for sell in (0, 32, 512):
        with pkg.BlockSolver(sell=sell, precision=precision) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            sol.mesh_setup(small.L)
            r = []
            for which, n in ((pkg.SCR_HIER_A, 3 * small.n_v), (pkg.SCR_HIER_SHAT, small.n_p),
                             (pkg.SCR_HIER_MESH, 3 * small.L.nb_rows)):
                b = _dev(np.random.default_rng(which).standard_normal(n))
                r.append(sol.amg_apply(which, b).cpu().numpy())
            outs.append(r)
    tol = 1e-12 if precision == pkg.SCR_FP64 else 1e-5
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert _rel(a, b) < tol
    del rng


def _three_vcycles(sol, small):
    out = []
    for which, n in ((pkg.SCR_HIER_A, 3 * small.n_v), (pkg.SCR_HIER_SHAT, small.n_p),
                     (pkg.SCR_HIER_MESH, 3 * small.L.nb_rows)):
        b = _dev(np.random.default_rng(which + 11).standard_normal(n))
        out.append(sol.amg_apply(which, b).cpu().numpy())
    return out


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_cuda_graph_vcycles_equal_eager_vcycles(small, precision):
    """A V-cycle replayed from its CUDA graph launches the same kernels with
    the same arguments as the eager V-cycle: V-cycles of A, Shat and L (each
    applied twice, so the second runs from the graph) and a whole solve are
    bit-identical with and without graphs, and the launch counter still
    counts the replayed kernels."""
    res = {}
    for graphs in (0, 1):
        with pkg.BlockSolver(cuda_graphs=graphs, precision=precision) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            sol.mesh_setup(small.L)
            first = _three_vcycles(sol, small)
            l0 = sol.stats()["kernel_launches"]
            second = _three_vcycles(sol, small)
            launched = sol.stats()["kernel_launches"] - l0
            x = sol.solve(small.b.copy())
            res[graphs] = (first, second, x, launched, sol.iters())
    for a, b in zip(res[0][0] + res[0][1], res[1][0] + res[1][1]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(res[0][2], res[1][2])
    assert res[0][4] == res[1][4]
    # three replayed V-cycles: the eager kernels plus one copy in and one out each
    assert res[1][3] == res[0][3] + 2 * 3


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
@pytest.mark.parametrize("graphs", [0, 1])
def test_programmatic_dependent_launch_changes_no_result(small, precision, graphs):
    """With the product kernels launched under programmatic stream
    serialization (each waits for its predecessor before reading a vector,
    after prefetching its own matrix rows), V-cycles of A, Shat and L and a
    whole solve are bit-identical to ordinary launches, eager and from CUDA
    graphs, with the scalar-row and the 16-byte kernels."""
    for code in (0, 304):
        res = []
        for pdl in (0, 1):
            with pkg.BlockSolver(pdl=pdl, cuda_graphs=graphs, precision=precision, spmv_group=code,
                                 autotune=0) as sol:
                sol.setup(small.A, small.B, small.C, small.D)
                sol.mesh_setup(small.L)
                out = _three_vcycles(sol, small) + _three_vcycles(sol, small)
                x = sol.solve(small.b.copy())
                res.append((out, x, sol.iters()))
        for a, b in zip(res[0][0], res[1][0]):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(res[0][1], res[1][1])
        assert res[0][2] == res[1][2]


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_l2_prefetch_changes_no_result(small, precision):
    """The bulk L2 prefetch of the scalar-row products only moves data into
    L2: V-cycles are bit-identical with it off, 1 CTA ahead and 192 ahead
    (the last CTAs of every product prefetch nothing past the arrays)."""
    ref = None
    for pf in (0, 1, 192):
        with pkg.BlockSolver(l2_prefetch=pf, autotune=0, spmv_group=102, precision=precision) as sol:
            sol.setup(small.A, small.B, small.C, small.D)
            sol.mesh_setup(small.L)
            out = _three_vcycles(sol, small)
        if ref is None:
            ref = out
            continue
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b)


def test_prefetch_option_is_validated():
    with pytest.raises(pkg.ScrError):
        pkg.BlockSolver(l2_prefetch=-1)


# ---------------------------------------------------------------- Alg. 1 / 2
def test_algorithm2_tight_inner_equals_schur(mini):
    op = BlockOperator.from_system(mini)
    S = schur.schur_exact_dense(op)
    rng = np.random.default_rng(4)
    xp = rng.standard_normal(op.np)
    with pkg.BlockSolver(rtol_I=1e-13, max_I=2000, restart_inner=60) as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        y = sol.apply_schur(_dev(xp)).cpu().numpy()
    assert _rel(y, S @ xp) < 1e-8


@pytest.mark.parametrize("k", [1, 2, 4])
def test_algorithm2_fixed_count_inner_matches_oracle(small, k):
    """Algorithm 2 with the inner A solve as k V-cycle Richardson steps: the
    GPU's S x_p equals D x_p - C R_k B x_p with R_k the oracle's Richardson
    map on the exported hierarchy of A (FP64)."""
    op = BlockOperator.from_system(small)
    xp = np.random.default_rng(40 + k).standard_normal(op.np)
    with pkg.BlockSolver(inner_vcycles=k) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        y = sol.apply_schur(_dev(xp)).cpu().numpy()
        nl = sol.amg_levels(pkg.SCR_HIER_A)
        As = [to_csr(sol.export(pkg.SCR_HIER_A, l, pkg.SCR_EXPORT_OPERATOR)) for l in range(nl)]
        Ps = [to_csr(sol.export(pkg.SCR_HIER_A, l, pkg.SCR_EXPORT_PROLONGATOR)) for l in range(nl - 1)]
    from oracle import krylov
    H = amg.hierarchy_from_matrices(As, Ps, 3, 1, 1, "cheb", 3)
    A = to_csr(small.A)
    xt = krylov.richardson(lambda v: A @ v, op.B @ xp, lambda v: amg.vcycle(H, v), k)
    ref = op.D @ xp - op.C @ xt
    assert _rel(y, ref) < 1e-11


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
@pytest.mark.parametrize("inner,inter", [(2, 0), (3, 2)])
def test_block_solve_with_fixed_count_a_solves_matches_direct(small, small_direct, precision, inner, inter):
    """Whole SCR solves with fixed-count inner (and intermediate) A solves
    meet 1e-8 and the direct solution to 1e-6; the inner count is exactly k
    per application of S."""
    op = BlockOperator.from_system(small)
    with pkg.BlockSolver(precision=precision, inner_vcycles=inner, inter_vcycles=inter) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        x = sol.solve(small.b.copy())
        st = sol.stats()
    assert st["rel_res"] <= 1e-8 and rel_residual(op, x, small.b) <= 1e-8
    assert _rel(x, small_direct) <= 1e-6
    assert st["i_iters"] == inner * st["s_iters"] or st["i_iters"] % inner == 0
    if inter:
        assert st["a_iters"] == inter * st["a_solves"]


def test_fixed_count_options_are_validated():
    for bad in ({"inner_vcycles": -1}, {"inter_vcycles": 65}):
        with pytest.raises(pkg.ScrError):
            pkg.BlockSolver(**bad)


def test_algorithm1_tight_solves_equals_inverse(mini, mini_x):
    op = BlockOperator.from_system(mini)
    with pkg.BlockSolver(rtol_A=1e-13, rtol_S=1e-12, rtol_I=1e-14, max_A=2000, max_S=2000, max_I=2000,
                         restart_inner=60) as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        y = sol.apply_pc(_dev(mini.b)).cpu().numpy()
    assert _rel(y, mini_x) < 1e-6
    assert rel_residual(op, y, mini.b) < 1e-6


# ---------------------------------------------------------------- full solve
@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_block_solve_matches_direct(small, small_direct, precision):
    op = BlockOperator.from_system(small)
    with pkg.BlockSolver(precision=precision) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        x = sol.solve(small.b.copy())
        st = sol.stats()
    assert st["rel_res"] <= 1e-8
    assert rel_residual(op, x, small.b) <= 1e-8
    assert _rel(x, small_direct) <= 1e-6
    assert 1 <= st["outer_iters"] <= 30


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_simple_preconditioned_solve_matches_direct(small, small_direct, precision):
    op = BlockOperator.from_system(small)
    with pkg.BlockSolver(precond=pkg.SCR_PC_SIMPLE, precision=precision) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        x = sol.solve(small.b.copy())
        st = sol.stats()
    assert st["rel_res"] <= 1e-8 and rel_residual(op, x, small.b) <= 1e-8
    assert _rel(x, small_direct) <= 1e-6
    assert st["i_iters"] == 0  # SIMPLE never invokes the inner level


def test_simple_apply_with_tight_solves(mini):
    op = BlockOperator.from_system(mini)
    rng = np.random.default_rng(12)
    r = rng.standard_normal(op.n)
    with pkg.BlockSolver(precond=pkg.SCR_PC_SIMPLE, rtol_A=1e-13, rtol_S=1e-13, max_A=2000, max_S=2000,
                         restart_inner=60) as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        y = sol.apply_pc(_dev(r)).cpu().numpy()
    yd = schur.simple_inverse_apply_dense(op, r)
    assert _rel(y, yd) < 1e-7


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_simplec_preconditioned_solve_matches_direct(small, small_direct, precision):
    op = BlockOperator.from_system(small)
    with pkg.BlockSolver(precond=pkg.SCR_PC_SIMPLEC, precision=precision) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        x = sol.solve(small.b.copy())
        st = sol.stats()
    assert st["rel_res"] <= 1e-8 and rel_residual(op, x, small.b) <= 1e-8
    assert _rel(x, small_direct) <= 1e-6
    assert st["i_iters"] == 0


def test_simplec_apply_with_tight_solves(mini):
    """P_SIMPLEC^{-1} r with tight intermediate solves equals the oracle's
    dense P_SIMPLEC^{-1} r, and differs from P_SIMPLE^{-1} r (the lumped
    diagonal is in effect)."""
    op = BlockOperator.from_system(mini)
    r = np.random.default_rng(13).standard_normal(op.n)
    with pkg.BlockSolver(precond=pkg.SCR_PC_SIMPLEC, rtol_A=1e-13, rtol_S=1e-13, max_A=2000, max_S=2000,
                         restart_inner=60) as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        y = sol.apply_pc(_dev(r)).cpu().numpy()
    yd = schur.simple_inverse_apply_dense(op, r, lumped=True)
    assert _rel(y, yd) < 1e-7
    assert _rel(y, schur.simple_inverse_apply_dense(op, r)) > 1e-4


def test_block_solve_device_pointers(mini, mini_x):
    with pkg.BlockSolver() as sol:
        sol.setup(pkg.DeviceBSR.from_host(mini.A), pkg.DeviceBSR.from_host(mini.B),
                  pkg.DeviceBSR.from_host(mini.C), pkg.DeviceBSR.from_host(mini.D))
        x = sol.solve(_dev(mini.b)).cpu().numpy()
        assert sol.residual() <= 1e-8
    assert _rel(x, mini_x) <= 1e-6


def test_block_solve_is_deterministic(mini):
    with pkg.BlockSolver() as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        x1 = sol.solve(mini.b.copy())
        x2 = sol.solve(mini.b.copy())
    with pkg.BlockSolver() as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        x3 = sol.solve(mini.b.copy())
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)


def test_mesh_cg_matches_direct(small):
    ud = direct.solve_mesh(small)
    L = to_csr(small.L)
    g = small.mesh_b.reshape(-1, 3)
    with pkg.BlockSolver(mm_rtol=1e-12) as sol:
        sol.mesh_setup(small.L)
        u = sol.mesh_solve(small.mesh_b.copy())
        it, rel = sol.mesh_iters()
    assert rel <= 1e-12  # the reported residual is the true one, g - L u
    assert np.linalg.norm(L @ u.reshape(-1, 3) - g) / np.linalg.norm(g) <= 1e-12
    assert _rel(u, ud) <= 1e-9
    assert 1 <= it <= 100


# ---------------------------------------------------------------- edge cases
def test_zero_rhs_gives_zero(mini):
    with pkg.BlockSolver() as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        x = sol.solve(np.zeros(mini.n))
        assert np.all(x == 0.0)
        assert sol.iters()[0] == 0
        sol.mesh_setup(mini.L)
        u = sol.mesh_solve(np.zeros(3 * mini.L.nb_rows))
        assert np.all(u == 0.0)


def test_not_converged_status(mini):
    with pkg.BlockSolver(max_it=1, rtol_A=0.5, rtol_S=0.5, rtol_I=0.5) as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        with pytest.raises(pkg.ScrError) as e:
            sol.solve(mini.b.copy())
        assert e.value.status == 3
        x = sol.solve(mini.b.copy(), raise_on_nonconvergence=False)
        assert sol.iters()[0] == 1
        assert np.all(np.isfinite(x))


def test_invalid_shapes_rejected(mini):
    with pkg.BlockSolver() as sol:
        with pytest.raises(pkg.ScrError) as e:
            sol.setup(mini.A, mini.C, mini.B, mini.D)  # B and C swapped
        assert e.value.status == 1
        bad = F.BSR(1, 1, mini.D.nb_rows, mini.D.nb_cols, mini.D.row_ptr.copy(), mini.D.col[::-1].copy(),
                    mini.D.val.copy())
        with pytest.raises(pkg.ScrError) as e:
            sol.setup(mini.A, mini.B, mini.C, bad)
        assert e.value.status == 1
        with pytest.raises(pkg.ScrError):
            sol.solve(np.zeros(mini.n))  # no successful set-up yet


def test_zero_diagonal_rejected(mini):
    A = F.BSR(3, 3, mini.A.nb_rows, mini.A.nb_cols, mini.A.row_ptr.copy(), mini.A.col.copy(), mini.A.val.copy())
    r = 5
    t = np.searchsorted(A.col[A.row_ptr[r]:A.row_ptr[r + 1]], r) + A.row_ptr[r]
    A.val[9 * t + 4] = 0.0
    with pkg.BlockSolver() as sol:
        with pytest.raises(pkg.ScrError) as e:
            sol.setup(A, mini.B, mini.C, mini.D)
        assert e.value.status == 1


def test_tiny_system_single_level(tiny_system):
    # smaller than the coarse size: the hierarchy is one dense level
    x_ref = direct.solve_block(tiny_system)
    with pkg.BlockSolver() as sol:
        sol.setup(tiny_system.A, tiny_system.B, tiny_system.C, tiny_system.D)
        assert sol.amg_levels(pkg.SCR_HIER_A) == 1
        x = sol.solve(tiny_system.b.copy())
    assert _rel(x, x_ref) <= 1e-6


# ---------------------------------------------------------------- full size
@pytest.mark.slow
def test_large_tube_solve_properties():
    """The benchmark workload (616,337 nodes, 2.5M unknowns): the oracle
    recomputes the FP64 residual of the GPU answer; sampled rows of calA
    are checked one by one against the oracle's block definition."""
    s = F.tube_system("tube_large")
    op = BlockOperator.from_system(s)
    with pkg.BlockSolver() as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        rng = np.random.default_rng(9)
        xr = rng.standard_normal(s.n)
        y = sol.apply_op(_dev(xr)).cpu().numpy()
        rows = rng.choice(s.n, 2000, replace=False)
        K = op.full()
        assert np.allclose(y[rows], K[rows] @ xr, rtol=1e-12, atol=1e-12 * np.abs(y).max())
        x = sol.solve(s.b.copy())
        st = sol.stats()
        sol.mesh_setup(s.L)
        u = sol.mesh_solve(s.mesh_b.copy())
        assert sol.mesh_iters()[1] <= 1e-8
    assert st["rel_res"] <= 1e-8
    assert rel_residual(op, x, s.b) <= 1e-8
    L = to_csr(s.L)
    g = s.mesh_b.reshape(-1, 3)
    assert np.linalg.norm(L @ u.reshape(-1, 3) - g) / np.linalg.norm(g) <= 1e-8


@pytest.mark.slow
def test_stenosis_mixed_precision_solve():
    """Stenosed tube (1,923,801 nodes, 7,791,364 unknowns), FP32 preconditioner
    with FP64 outer iteration: the oracle recomputes the FP64 residual of the
    mixed and the FP64 GPU answers; the two agree to the accuracy the
    1e-8 residual allows."""
    s = F.tube_system("stenosis")
    op = BlockOperator.from_system(s)
    xs = {}
    for prec in (pkg.SCR_MIXED, pkg.SCR_FP64):
        with pkg.BlockSolver(precision=prec) as sol:
            sol.setup(s.A, s.B, s.C, s.D)
            xs[prec] = sol.solve(s.b.copy())
            assert sol.residual() <= 1e-8
        assert rel_residual(op, xs[prec], s.b) <= 1e-8
    assert _rel(xs[pkg.SCR_MIXED], xs[pkg.SCR_FP64]) <= 1e-5


# ---------------------------------------------------------------- batched form
def _member(i, **kw):
    p = F.batch_member_params(i)
    p.update(kw)
    return F.tube_system("batch", **p)


def test_batched_small_members_match_direct():
    """Several independent tubes of different sizes solved as one batch:
    every member meets the tolerance on its own and matches its direct
    solution."""
    members = [_member(i, n_ax=6 + 3 * i) for i in range(5)]
    with pkg.BlockSolver() as sol:
        sol.setup_batch([(m.A, m.B, m.C, m.D) for m in members])
        xs = sol.solve_batch([m.b.copy() for m in members])
        rel = sol.batch_residuals()
    for m, x, r in zip(members, xs, rel):
        op = BlockOperator.from_system(m)
        assert r <= 1e-8
        assert rel_residual(op, x, m.b) <= 1e-8
        xd = direct.solve_block(m)
        assert _rel(x, xd) <= 1e-6


def test_batched_single_member_equals_plain_solve(mini):
    with pkg.BlockSolver() as sol:
        sol.setup_batch([(mini.A, mini.B, mini.C, mini.D)])
        xb = sol.solve_batch([mini.b.copy()])[0]
    with pkg.BlockSolver() as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        x = sol.solve(mini.b.copy())
    assert np.array_equal(xb, x)


@pytest.mark.slow
def test_batched_64_tubes_mixed():
    """The batched workload: 64 straight / stenosed tubes (radius
    0.15-0.5 cm, 5k-80k nodes) in one block-diagonal solve, FP32
    preconditioner with FP64 outer iteration; the oracle recomputes every
    member's FP64 residual."""
    members = [_member(i) for i in range(64)]
    with pkg.BlockSolver(precision=pkg.SCR_MIXED) as sol:
        sol.setup_batch([(m.A, m.B, m.C, m.D) for m in members])
        xs = sol.solve_batch([m.b.copy() for m in members])
        rel = sol.batch_residuals()
    assert np.all(rel <= 1e-8)
    for m, x in zip(members, xs):
        assert rel_residual(BlockOperator.from_system(m), x, m.b) <= 1e-8
    smallest = int(np.argmin([m.n for m in members]))
    assert _rel(xs[smallest], direct.solve_block(members[smallest])) <= 1e-6


def test_time_step_trends_scr_versus_simple():
    """Robustness trends of Sec. 6 (SCR needs far fewer outer iterations
    than SIMPLE; inner work grows with dt): on the small tube at dt = 1e-4
    and 1e-3 both preconditioners meet the tolerance, SCR with fewer outer
    iterations than SIMPLE, and SCR's inner iterations grow with dt."""
    outer, inner = {}, {}
    for dt in (1e-4, 1e-3):
        s = F.tube_system("tube_small", dt=dt)
        op = BlockOperator.from_system(s)
        for pc in (pkg.SCR_PC_SCR, pkg.SCR_PC_SIMPLE):
            with pkg.BlockSolver(precond=pc) as sol:
                sol.setup(s.A, s.B, s.C, s.D)
                x = sol.solve(s.b.copy())
                outer[(dt, pc)], inner[(dt, pc)] = sol.iters()
            assert rel_residual(op, x, s.b) <= 1e-8
        assert outer[(dt, pkg.SCR_PC_SCR)] < outer[(dt, pkg.SCR_PC_SIMPLE)], outer
        assert outer[(dt, pkg.SCR_PC_SCR)] <= 10, outer
    assert inner[(1e-3, pkg.SCR_PC_SCR)] > inner[(1e-4, pkg.SCR_PC_SCR)], inner


def test_smallest_time_step_converges_with_the_guard():
    """dt = 1e-5 (the smallest step of Sec. 6's time-step study): the Galerkin
    levels of the Shat hierarchy fail the Chebyshev guard and are smoothed by
    l1-Jacobi; SCR and SIMPLEC then reach the tolerance (CPU oracle: 13 and
    18 outer iterations; SIMPLE still stalls, as every Shat solve hits its
    iteration cap)."""
    s = F.tube_system("tube_small", dt=1e-5)
    op = BlockOperator.from_system(s)
    for pc in (pkg.SCR_PC_SCR, pkg.SCR_PC_SIMPLEC):
        with pkg.BlockSolver(precond=pc) as sol:
            sol.setup(s.A, s.B, s.C, s.D)
            x = sol.solve(s.b.copy())
            assert sol.iters()[0] <= 40
        assert rel_residual(op, x, s.b) <= 1e-8


@pytest.mark.parametrize("rho_s,E_s", [(1e-2, 4e6), (1e2, 4e6), (1.0, 1e6), (1.0, 1e8)])
def test_wall_parameter_robustness(rho_s, E_s):
    """Robustness over the wall density and Young's modulus (Sec. 6, table of
    rho_s in [1e-2, 1e2] and E in [1e6, 1e8]: SCR's outer iteration count
    barely moves, SIMPLE needs several times more).  On the small tube every
    solve meets the tolerance, SCR stays within 1 to 5 outer iterations
    (the CPU oracle: 3 in every case) and below SIMPLE's count."""
    s = F.tube_system("tube_small", rho_s=rho_s, E_s=E_s)
    op = BlockOperator.from_system(s)
    outer = {}
    for pc in (pkg.SCR_PC_SCR, pkg.SCR_PC_SIMPLE, pkg.SCR_PC_SIMPLEC):
        with pkg.BlockSolver(precond=pc) as sol:
            sol.setup(s.A, s.B, s.C, s.D)
            x = sol.solve(s.b.copy())
            outer[pc] = sol.iters()[0]
        assert rel_residual(op, x, s.b) <= 1e-8
    assert 1 <= outer[pkg.SCR_PC_SCR] <= 5, outer
    assert outer[pkg.SCR_PC_SCR] < outer[pkg.SCR_PC_SIMPLE], outer
    assert outer[pkg.SCR_PC_SCR] < outer[pkg.SCR_PC_SIMPLEC], outer


def _inflow_rhs(name, n_rhs=8, seed=2206):
    """Right-hand sides -R at states whose inflow peaks are drawn U(0, 60)
    cm/s (one Jacobian, at the nominal 30 cm/s, solves all of them)."""
    peaks = np.random.default_rng(seed).uniform(0.0, 60.0, n_rhs)
    return [F.rhs_only(name, u_max=float(u)) for u in peaks]


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_multi_rhs_solve_matches_direct(small, precision):
    """Eight right-hand sides with one set-up: interleaved vectors, every
    product with eight columns at once, one FGMRES on the interleaved system;
    every column meets the tolerance (recomputed by the oracle) and matches
    the direct solve of its own right-hand side."""
    op = BlockOperator.from_system(small)
    rhs = _inflow_rhs("tube_small")
    ref = direct.solve_block_many(small, rhs)
    with pkg.BlockSolver(nrhs=8, precision=precision) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        xs, rel = sol.solve_multi([b.copy() for b in rhs])
        xd, reld = sol.solve_multi([_dev(b) for b in rhs])
        with pytest.raises(pkg.ScrError):
            sol.solve(rhs[0].copy())
    assert np.all(rel <= 1e-8) and np.all(reld <= 1e-8)
    for b, x, x2, xr in zip(rhs, xs, xd, ref):
        assert rel_residual(op, x, b) <= 1e-8
        assert _rel(x, xr) <= 1e-6
        np.testing.assert_array_equal(x, x2.cpu().numpy())


def test_multi_rhs_equal_columns_give_the_single_solution(small, small_direct):
    """Eight copies of one right-hand side: each column equals the direct
    solution; zero columns stay zero."""
    b = small.b
    with pkg.BlockSolver(nrhs=8) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        xs, rel = sol.solve_multi([b.copy() for _ in range(7)] + [np.zeros_like(b)])
    for x in xs[:7]:
        assert _rel(x, small_direct) <= 1e-6
    assert np.all(xs[7] == 0.0)
    assert np.all(rel[:7] <= 1e-8)


@pytest.fixture(scope="module")
def outlet_small():
    return F.tube_system("tube_small", outlet_resistance=2.7e4)


def test_outlet_terms_in_calA_and_shat(outlet_small):
    """Resistance outlet: calA x and Shat with the rank-1 outlet term equal
    the oracle's (explicit) operator."""
    s = outlet_small
    op = BlockOperator.from_system(s)
    x = np.random.default_rng(6).standard_normal(op.n)
    with pkg.BlockSolver() as sol:
        sol.set_outlets(s.a_out, s.c_out)
        sol.setup(s.A, s.B, s.C, s.D)
        y = sol.apply_op(_dev(x)).cpu().numpy()
        Sh = to_csr(sol.export(pkg.SCR_HIER_SHAT, 0, pkg.SCR_EXPORT_OPERATOR))
    assert _rel(y, op.matvec(x)) < 1e-13
    want = schur.schur_hat(op)
    assert abs(Sh - want).max() <= 1e-12 * abs(want).max()


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
@pytest.mark.parametrize("precond", [pkg.SCR_PC_SCR, pkg.SCR_PC_SIMPLE])
def test_outlet_solve_matches_direct(outlet_small, precision, precond):
    s = outlet_small
    op = BlockOperator.from_system(s)
    x_ref = direct.solve_block(s)
    with pkg.BlockSolver(precision=precision, precond=precond) as sol:
        sol.set_outlets(s.a_out, s.c_out)
        sol.setup(s.A, s.B, s.C, s.D)
        x = sol.solve(s.b.copy())
        assert sol.residual() <= 1e-8
    assert rel_residual(op, x, s.b) <= 1e-8
    assert _rel(x, x_ref) <= 1e-6


def test_outlet_option_checks(outlet_small):
    s = outlet_small
    with pkg.BlockSolver(precond=pkg.SCR_PC_SIMPLEC) as sol:
        sol.set_outlets(s.a_out, s.c_out)
        with pytest.raises(pkg.ScrError):
            sol.setup(s.A, s.B, s.C, s.D)
    with pkg.BlockSolver(nrhs=8) as sol:
        sol.set_outlets(s.a_out, s.c_out)
        with pytest.raises(pkg.ScrError):
            sol.setup(s.A, s.B, s.C, s.D)
    with pkg.BlockSolver() as sol:  # removing the outlets gives the sparse operator back
        sol.set_outlets(s.a_out, s.c_out)
        sol.set_outlets([], [])
        sol.setup(s.A, s.B, s.C, s.D)
        x = np.random.default_rng(7).standard_normal(3 * s.n_v + s.n_p)
        y = sol.apply_op(_dev(x)).cpu().numpy()
    op0 = BlockOperator(s.A, s.B, s.C, s.D)
    assert _rel(y, op0.matvec(x)) < 1e-13


# ---------------------------------------------------------------- residual assembly
def _residual_case(name, **kw):
    s = F.tube_system(name, keep_mesh=True, **kw)
    asm = F.Assembler(F.make_params(**{**F.PRESETS[name], **kw}))
    v, p = asm.initial_state()
    rng = np.random.default_rng(17)
    nn = s.mesh.n_nodes
    vd = 0.1 * rng.standard_normal(3 * nn)
    u = 1e-4 * rng.standard_normal(3 * nn)
    vhat = 0.01 * rng.standard_normal(3 * nn)
    return s, asm, v, p, vd, u, vhat


@pytest.mark.parametrize("name", ["tube_mini", "tube_small"])
def test_gpu_residual_matches_the_element_loop(name):
    """R = [R_m | R_p] from the GPU element loop equals the generator's
    element loop (the fluid VMS residual with tau at the state, the solid
    residual) at a state with rates, solid displacement and mesh velocity,
    and every evaluation adds the same terms in the same order."""
    s, asm, v, p, vd, u, vhat = _residual_case(name)
    ref = asm.evaluate(v, p, vd=vd, u=u, vhat=vhat, want_mat=False)
    want = np.concatenate([ref["Rm"], ref["Rp"]])
    with pkg.BlockSolver() as sol:
        sol.assembly_setup(s.mesh, s.params)
        R = sol.assemble_residual(v, p, vhat=vhat, vdot=vd, u=u)
        Rd = sol.assemble_residual(_dev(v), _dev(p), vhat=_dev(vhat), vdot=_dev(vd), u=_dev(u)).cpu().numpy()
    assert _rel(R, want) < 1e-12
    np.testing.assert_array_equal(R, Rd)
    # the momentum and mass parts separately (different scales)
    nv3 = 3 * s.mesh.n_nodes
    assert _rel(R[:nv3], want[:nv3]) < 1e-12 and _rel(R[nv3:], want[nv3:]) < 1e-12


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_gpu_corrector_matches_the_oracle_loop(small, precision):
    """Three multi-corrector iterations on the GPU (assembled residual,
    SCR-FGMRES + AMG solve, generalized-alpha updates, tangent and mesh fixed)
    follow the oracle's loop (the generator's residual, direct solves): same
    starting residual, the same contraction, the same final state up to the
    solves' tolerance; host and device state give the same result."""
    from oracle import corrector
    s = small
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
    v0, p0 = asm.initial_state()
    nn = s.mesh.n_nodes
    z = np.zeros(3 * nn)
    vr, pr, vdr, ur, nr = corrector.corrector(s, asm, v0, p0, z, z, 3)
    with pkg.BlockSolver(precision=precision) as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        sol.assembly_setup(s.mesh, s.params)
        v, p, vd, u = v0.copy(), p0.copy(), z.copy(), z.copy()
        norms = sol.corrector(v, p, vd, u, 3)
        dv, dp, dvd, du = (_dev(a) for a in (v0, p0, z, z))
        norms_d = sol.corrector(dv, dp, dvd, du, 3)
    assert norms[0] == pytest.approx(nr[0], rel=1e-12)
    assert norms[1] == pytest.approx(nr[1], rel=1e-3)
    assert norms[2] < 1e-2 * norms[1] and norms[3] < 1e-4 * norms[1]
    for a, b in ((v, vr), (p, pr), (vd, vdr), (u, ur)):
        assert _rel(a, b) < 1e-7
    np.testing.assert_array_equal(norms, norms_d)
    np.testing.assert_array_equal(v, dv.cpu().numpy())


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_gpu_corrector_ale_matches_the_oracle_loop(small, precision):
    """Multi-corrector with the mesh moving inside the loop (Sec. 3.5, steps
    3-4): the GPU's mesh CG + AMG on the eliminated Laplacian with the lifted
    interface displacement, its mesh velocity and the residual at that mesh
    velocity follow the oracle's loop (direct mesh and block solves): same
    starting residual, the same contraction, the same state and mesh
    displacement up to the solves' tolerances; host and device paths agree
    bit for bit."""
    from oracle import corrector
    from oracle.sparse import to_csr
    s = small
    m = s.mesh
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
    L_raw = asm.mesh_laplacian()
    follow = F.interface_follow(m)
    v0, p0 = asm.initial_state()
    z, zf = np.zeros(3 * m.n_nodes), np.zeros(3 * m.n_fluid)
    vn = 0.01 * np.random.default_rng(4).standard_normal(3 * m.n_fluid)
    vr, pr, vdr, ur, uhr, nr = corrector.corrector_ale(s, asm, v0, p0, z, z, 3, to_csr(L_raw), m.fluid_id,
                                                       m.dir_m, follow, zf, vn)
    with pkg.BlockSolver(precision=precision) as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        sol.assembly_setup(m, s.params)
        sol.mesh_setup(s.L)
        sol.mesh_coupling(L_raw, m.fluid_id, m.dir_m, follow)
        v, p, vd, u = v0.copy(), p0.copy(), z.copy(), z.copy()
        norms, uh = sol.corrector_ale(v, p, vd, u, zf, 3, vhat_n=vn)
        dv, dp, dvd, du = (_dev(a) for a in (v0, p0, z, z))
        norms_d, uh_d = sol.corrector_ale(dv, dp, dvd, du, _dev(zf), 3, vhat_n=_dev(vn))
    assert norms[0] == pytest.approx(nr[0], rel=1e-12)
    assert norms[1] == pytest.approx(nr[1], rel=1e-3)
    assert norms[2] < 1e-2 * norms[1] and norms[3] < 1e-2 * norms[2]
    for a, b in ((v, vr), (p, pr), (vd, vdr), (u, ur), (uh, uhr)):
        assert _rel(a, b) < 1e-7
    assert np.abs(uh).max() > 1e-6
    np.testing.assert_array_equal(norms, norms_d)
    np.testing.assert_array_equal(uh, uh_d.cpu().numpy())


def _gpu_blocks(sol):
    A = to_csr(sol.export(pkg.SCR_HIER_A, 0, pkg.SCR_EXPORT_OPERATOR))
    B, C, D = (to_csr(sol.export(pkg.SCR_HIER_A, 0, k))
               for k in (pkg.SCR_EXPORT_BLOCK_B, pkg.SCR_EXPORT_BLOCK_C, pkg.SCR_EXPORT_BLOCK_D))
    return A, B, C, D


def _moved_state(s, asm, seed):
    v0, p0 = asm.initial_state()
    rng = np.random.default_rng(seed)
    nn = s.mesh.n_nodes
    v = v0 + 2.0 * rng.standard_normal(v0.size)
    p = p0 + 10.0 * rng.standard_normal(p0.size)
    vd = 50.0 * rng.standard_normal(3 * nn)
    vh = rng.standard_normal(3 * nn)
    return v, p, vd, vh


@pytest.mark.parametrize("preset", ["tube_mini", "tube_small", "bif_mini"])
def test_gpu_tangent_matches_the_oracle_at_a_moved_state(preset):
    """The GPU's tangent assembly (one thread per element column, summed per
    stored block in element order) at a state away from the assembly state
    (perturbed velocity, pressure, mesh velocity and rates) equals the
    oracle's Jacobian there (the generator's element tangent with tau frozen,
    the Dirichlet convention applied) to FP64 rounding, block by block; the
    solve on it meets the direct solve of that Jacobian."""
    from oracle import corrector
    s = F.tube_system(preset, keep_mesh=True)
    asm = F.Assembler(F.make_params(**F.PRESETS[preset]))
    v, p, vd, vh = _moved_state(s, asm, 17)
    want = corrector.tangent(s, asm, v, p, vd, vh)
    with pkg.BlockSolver() as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        sol.assembly_setup(s.mesh, s.params)
        sol.assemble_tangent(v, p, vhat=vh, vdot=vd)
        got = _gpu_blocks(sol)
        x = sol.solve(s.b.copy())
        # the same from device pointers
        sol.assemble_tangent(_dev(v), _dev(p), vhat=_dev(vh), vdot=_dev(vd))
        got_d = _gpu_blocks(sol)
    for g, w, gd in zip(got, want, got_d):
        assert g.shape == w.shape
        assert abs(g - w).max() <= 1e-12 * abs(w).max()
        assert abs(g - gd).max() == 0
    K = sp.bmat([[want[0], want[1]], [want[2], want[3]]], format="csc")
    xd = spl.spsolve(K, s.b)
    assert np.linalg.norm(K @ x - s.b) <= 1e-8 * np.linalg.norm(s.b)
    assert _rel(x, xd) <= 1e-6


def test_gpu_tangent_at_the_assembly_state_is_the_input_system(small):
    """At the generator's assembly state the GPU's tangent is the input block
    system itself (the patterns kept, Dirichlet rows identity)."""
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
    v0, p0 = asm.initial_state()
    with pkg.BlockSolver() as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        sol.assembly_setup(small.mesh, small.params)
        sol.assemble_tangent(v0, p0)
        got = _gpu_blocks(sol)
    for g, w in zip(got, (small.A, small.B, small.C, small.D)):
        w = to_csr(w)
        assert abs(g - w).max() <= 1e-12 * abs(w).max()


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
@pytest.mark.parametrize("resetup", [0, 1])
def test_gpu_newton_corrector_matches_the_oracle_loop(small, precision, resetup):
    """The multi-corrector with the tangent re-assembled on the GPU at every
    iteration (option newton) follows the oracle's loop that re-assembles
    the generator's tangent and solves directly: same starting residual, same
    residuals up to the solves' tolerance, the same final state."""
    from oracle import corrector
    s = small
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
    v0, p0 = asm.initial_state()
    z = np.zeros(3 * s.mesh.n_nodes)
    vr, pr, vdr, ur, nr = corrector.corrector(s, asm, v0, p0, z, z, 3, newton=True)
    with pkg.BlockSolver(precision=precision, newton=1, tangent_resetup=resetup) as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        sol.assembly_setup(s.mesh, s.params)
        v, p, vd, u = v0.copy(), p0.copy(), z.copy(), z.copy()
        norms = sol.corrector(v, p, vd, u, 3)
        dv, dp, dvd, du = (_dev(a) for a in (v0, p0, z, z))
        norms_d = sol.corrector(dv, dp, dvd, du, 3)
    assert norms[0] == pytest.approx(nr[0], rel=1e-12)
    assert norms[1] == pytest.approx(nr[1], rel=1e-3)
    assert norms[2] < 1e-2 * norms[1]
    for a, b in ((v, vr), (p, pr), (vd, vdr), (u, ur)):
        assert _rel(a, b) < 1e-7
    np.testing.assert_array_equal(norms, norms_d)


@pytest.mark.parametrize("precision", [pkg.SCR_FP64])
def test_gpu_newton_corrector_ale_matches_the_oracle_loop(small, precision):
    """The same with the mesh moving inside the loop: the tangent at each
    iteration sees that iteration's mesh velocity."""
    from oracle import corrector
    from oracle.sparse import to_csr as tc
    s = small
    m = s.mesh
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
    L_raw = asm.mesh_laplacian()
    follow = F.interface_follow(m)
    v0, p0 = asm.initial_state()
    z, zf = np.zeros(3 * m.n_nodes), np.zeros(3 * m.n_fluid)
    vn = 0.01 * np.random.default_rng(4).standard_normal(3 * m.n_fluid)
    vr, pr, vdr, ur, uhr, nr = corrector.corrector_ale(s, asm, v0, p0, z, z, 3, tc(L_raw), m.fluid_id,
                                                       m.dir_m, follow, zf, vn, newton=True)
    with pkg.BlockSolver(precision=precision, newton=1) as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        sol.assembly_setup(m, s.params)
        sol.mesh_setup(s.L)
        sol.mesh_coupling(L_raw, m.fluid_id, m.dir_m, follow)
        v, p, vd, u = v0.copy(), p0.copy(), z.copy(), z.copy()
        norms, uh = sol.corrector_ale(v, p, vd, u, zf, 3, vhat_n=vn)
    assert norms[0] == pytest.approx(nr[0], rel=1e-12)
    assert norms[1] == pytest.approx(nr[1], rel=1e-3)
    for a, b in ((v, vr), (p, pr), (vd, vdr), (u, ur), (uh, uhr)):
        assert _rel(a, b) < 1e-7


def test_gpu_tangent_needs_both_set_ups(small):
    with pkg.BlockSolver() as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        v, p = np.zeros(3 * small.n_v), np.zeros(small.n_p)
        with pytest.raises(pkg.ScrError, match="scr_assembly_setup"):
            sol.assemble_tangent(v, p)
    with pytest.raises(pkg.ScrError):
        pkg.BlockSolver(newton=2)


def _exported_blocks(sol):
    """The solver's A, B, C, D as block matrices in the set-up's patterns."""
    return (sol.export(pkg.SCR_HIER_A, 0, pkg.SCR_EXPORT_OPERATOR),
            *(sol.export(pkg.SCR_HIER_A, 0, k) for k in (pkg.SCR_EXPORT_BLOCK_B, pkg.SCR_EXPORT_BLOCK_C,
                                                         pkg.SCR_EXPORT_BLOCK_D)))


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_numeric_resetup_with_the_same_values_changes_nothing(small, precision):
    """scr_update_values with the set-up's own values reproduces the set-up:
    V-cycles of both hierarchies and a whole solve are bit-identical."""
    with pkg.BlockSolver(precision=precision) as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        sol.mesh_setup(small.L)
        v0 = _three_vcycles(sol, small)
        x0 = sol.solve(small.b.copy())
        sol.update_values(small.A, small.B, small.C, small.D)
        v1 = _three_vcycles(sol, small)
        x1 = sol.solve(small.b.copy())
    for a, b in zip(v0, v1):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(x0, x1)


def test_numeric_resetup_matches_the_oracle_on_the_kept_patterns(small):
    """New values on the set-up's patterns (the Jacobian at a moved state,
    assembled on the GPU): the solver's A, B, C, D are the new ones, Shat is
    the oracle's D - C diag(A)^{-1} B of them, the aggregates are the set-up's,
    every prolongator is the oracle's smoothed prolongator of the new level
    operator truncated to the set-up's kept positions, every coarse operator
    is P^T A P, and the solve meets the direct solve of the new system."""
    s = small
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
    v, p, vd, vh = _moved_state(s, asm, 23)
    with pkg.BlockSolver(tangent_resetup=0) as tsol:
        tsol.setup(s.A, s.B, s.C, s.D)
        tsol.assembly_setup(s.mesh, s.params)
        tsol.assemble_tangent(v, p, vhat=vh, vdot=vd)
        new = _exported_blocks(tsol)
    with pkg.BlockSolver() as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        before = {}
        for which in (pkg.SCR_HIER_A, pkg.SCR_HIER_SHAT):
            nl = sol.amg_levels(which)
            before[which] = [(sol.export(which, l, pkg.SCR_EXPORT_AGGREGATES),
                              sol.export(which, l, pkg.SCR_EXPORT_PROLONGATOR)) for l in range(nl - 1)]
        sol.update_values(*new)
        got = _exported_blocks(sol)
        after = {}
        for which in (pkg.SCR_HIER_A, pkg.SCR_HIER_SHAT):
            nl = sol.amg_levels(which)
            after[which] = ([to_csr(sol.export(which, l, pkg.SCR_EXPORT_OPERATOR)) for l in range(nl)],
                            [sol.export(which, l, pkg.SCR_EXPORT_PROLONGATOR) for l in range(nl - 1)],
                            [sol.export(which, l, pkg.SCR_EXPORT_AGGREGATES) for l in range(nl - 1)])
        b = np.random.default_rng(5).standard_normal(s.n)
        x = sol.solve(b.copy())
    for g, w in zip(got, new):
        assert np.array_equal(g.row_ptr, w.row_ptr) and np.array_equal(g.col, w.col)
        assert np.array_equal(g.val, w.val)
    op = BlockOperator(*new)
    Shat = schur.schur_hat(op)
    As, Ps, aggs = after[pkg.SCR_HIER_SHAT]
    assert abs(As[0] - Shat).max() <= 1e-12 * abs(Shat).max()
    for which, bs in ((pkg.SCR_HIER_A, 3), (pkg.SCR_HIER_SHAT, 1)):
        As, Ps, aggs = after[which]
        for l, ((agg0, P0), P, agg) in enumerate(zip(before[which], Ps, aggs)):
            np.testing.assert_array_equal(agg, agg0)
            assert np.array_equal(P.row_ptr, P0.row_ptr) and np.array_equal(P.col, P0.col)
            Pt = amg.tentative_prolongator(agg.astype(np.int64), bs)
            Psm, _ = amg.smoothed_prolongator(As[l], Pt)
            Pref = amg.truncate_to_pattern(Psm, bs, P0.row_ptr, P0.col)
            Pg = to_csr(P)
            assert abs(Pg - Pref).max() <= 1e-12 * abs(Pref).max()
            Aref = (Pref.T @ As[l] @ Pref).tocsr()
            assert abs(As[l + 1] - Aref).max() <= 1e-11 * abs(Aref).max()
    K = op.full().tocsc()
    xd = spl.spsolve(K, b)
    assert np.linalg.norm(K @ x - b) <= 1e-8 * np.linalg.norm(b)
    assert _rel(x, xd) <= 1e-6


def test_numeric_resetup_rejects_another_pattern(small, mini):
    """Other sizes, or the same sizes with other column indices, are argument
    errors (checked on the device before any value is written)."""
    with pkg.BlockSolver() as sol:
        sol.setup(small.A, small.B, small.C, small.D)
        with pytest.raises(pkg.ScrError, match="differ"):
            sol.update_values(mini.A, mini.B, mini.C, mini.D)
        A = F.BSR(small.A.br, small.A.bc, small.A.nb_rows, small.A.nb_cols, small.A.row_ptr.copy(),
                  small.A.col.copy(), small.A.val.copy())
        r = int(np.nonzero(np.diff(A.row_ptr) >= 3)[0][0])
        a, b = A.row_ptr[r], A.row_ptr[r + 1]
        A.col[a:b] = np.roll(A.col[a:b], 1)  # same sizes, another pattern
        with pytest.raises(pkg.ScrError, match="pattern"):
            sol.update_values(A, small.B, small.C, small.D)


def test_gpu_corrector_ale_rejects_a_missing_coupling(small):
    """scr_corrector_ale without scr_mesh_coupling, and a coupling whose
    follow flag sits on a free mesh node, are argument errors."""
    s = small
    m = s.mesh
    z, zf = np.zeros(3 * m.n_nodes), np.zeros(3 * m.n_fluid)
    with pkg.BlockSolver() as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        sol.assembly_setup(m, s.params)
        sol.mesh_setup(s.L)
        sol.n_fluid = m.n_fluid
        v, p = np.zeros(3 * m.n_nodes), np.zeros(m.n_p)
        with pytest.raises(pkg.ScrError, match="scr_mesh_coupling"):
            sol.corrector_ale(v, p, z.copy(), z.copy(), zf, 1)
        bad = F.interface_follow(m).copy()
        bad[np.flatnonzero(~m.dir_m)[0]] = 1
        asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
        with pytest.raises(pkg.ScrError, match="follow"):
            sol.mesh_coupling(asm.mesh_laplacian(), m.fluid_id, m.dir_m, bad)


def test_gpu_corrector_with_a_resistance_outlet(outlet_small):
    """Corrector with the outlet traction in the residual and the rank-1 term
    in the tangent: follows the oracle's loop and contracts."""
    from oracle import corrector
    s = F.tube_system("tube_small", keep_mesh=True, outlet_resistance=2.7e4)
    asm = F.Assembler(F.make_params(**F.PRESETS["tube_small"]))
    v0, p0 = asm.initial_state()
    z = np.zeros(3 * s.mesh.n_nodes)
    vr, pr, _, _, nr = corrector.corrector(s, asm, v0, p0, z, z, 2)
    with pkg.BlockSolver() as sol:
        sol.set_outlets(s.a_out, s.c_out)
        sol.setup(s.A, s.B, s.C, s.D)
        sol.assembly_setup(s.mesh, s.params)
        v, p, vd, u = v0.copy(), p0.copy(), z.copy(), z.copy()
        norms = sol.corrector(v, p, vd, u, 2)
    assert norms[0] == pytest.approx(nr[0], rel=1e-12)
    assert norms[1] == pytest.approx(nr[1], rel=1e-3) and norms[2] < 1e-2 * norms[1]
    assert _rel(v, vr) < 1e-7 and _rel(p, pr) < 1e-7
    del outlet_small


# ---------------------------------------------------------------- bifurcation
@pytest.fixture(scope="module")
def bif_mini():
    s = F.tube_system("bif_mini", keep_mesh=True)
    return s, direct.solve_block(s)


@pytest.mark.parametrize("precision", [pkg.SCR_FP64, pkg.SCR_MIXED])
def test_gpu_bifurcation_matches_direct(bif_mini, precision):
    """The bifurcation (parent, solid carina tip, two sheared half-disk
    daughters): the GPU's SCR-FGMRES answer matches the direct solve and its
    FP64 residual, recomputed by the oracle, meets 1e-8; the mesh CG + AMG
    meets 1e-8 on the bifurcation's mesh system."""
    s, xd = bif_mini
    op = BlockOperator.from_system(s)
    with pkg.BlockSolver(precision=precision) as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        x = sol.solve(s.b.copy())
        sol.mesh_setup(s.L)
        u = sol.mesh_solve(s.mesh_b.copy())
        assert sol.mesh_iters()[1] <= 1e-8
    assert rel_residual(op, x, s.b) <= 1e-8 and _rel(x, xd) <= 1e-6
    L = to_csr(s.L)
    g = s.mesh_b.reshape(-1, 3)
    assert np.linalg.norm(L @ u.reshape(-1, 3) - g) <= 1e-8 * np.linalg.norm(g)


def test_gpu_bifurcation_eight_inflow_peaks():
    """Eight right-hand sides -R at inflow peaks drawn U(0, 60) cm/s on one
    bifurcation Jacobian, solved as one 8-column mixed-precision block solve:
    every column meets 1e-8 (recomputed by the oracle), and the first column
    matches the oracle's own SCR-FGMRES driven to 1e-12."""
    s = F.tube_system("bif_small")
    op = BlockOperator.from_system(s)
    peaks = np.random.default_rng(2206).uniform(0.0, 60.0, 8)
    rhs = [F.rhs_only("bif_small", u_max=float(u)) for u in peaks]
    with pkg.BlockSolver(nrhs=8, precision=pkg.SCR_MIXED) as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        xs, rel = sol.solve_multi([b.copy() for b in rhs])
    assert np.all(rel <= 1e-8)
    for b, x in zip(rhs, xs):
        assert rel_residual(op, x, b) <= 1e-8
    ref, info = scr.SCRSolver(s, scr.SolverOptions(rtol=1e-12)).solve(rhs[0])
    assert info.converged and _rel(xs[0], ref) <= 1e-6


# ---------------------------------------------------------------- non-finite input
def test_nan_right_hand_side_is_reported_and_the_handle_stays_usable(mini):
    """A NaN in the right-hand side of the block solve or of the mesh solve
    is reported as SCR_NOT_CONVERGED (never as a converged zero), and the
    same handle then solves a clean system to 1e-8."""
    with pkg.BlockSolver() as sol:
        sol.setup(mini.A, mini.B, mini.C, mini.D)
        b = mini.b.copy()
        b[7] = np.nan
        with pytest.raises(pkg.ScrError) as e:
            sol.solve(b)
        assert e.value.status == 3
        sol.mesh_setup(mini.L)
        g = mini.mesh_b.copy()
        g[5] = np.nan
        with pytest.raises(pkg.ScrError) as e:
            sol.mesh_solve(g)
        assert e.value.status == 3
        sol.solve(mini.b.copy())
        assert sol.residual() <= 1e-8
        sol.mesh_solve(mini.mesh_b.copy())
        assert sol.mesh_iters()[1] <= 1e-8  # the true residual, confirmed before the CG stops
