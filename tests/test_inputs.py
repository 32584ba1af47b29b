"""Pins of the seeded input generator (mesh + element loop) against closed
forms, invariants and textbook special cases."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import fsi_inputs as F
from oracle.sparse import to_csr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(path):
    out = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


# ---------------------------------------------------------------- constants
def test_genalpha_golden():
    for r in _rows(os.path.join(GOLDEN, "genalpha.txt")):
        rho, am, af, ga = map(float, r)
        got = F.genalpha(rho)
        assert np.allclose(got, (am, af, ga), rtol=0, atol=1e-15)


@pytest.mark.parametrize("rho", [0.0, 0.1, 0.5, 0.9, 1.0])
def test_genalpha_gamma_identity(rho):
    # gamma = 1/2 + alpha_m - alpha_f holds for the first-order family
    am, af, ga = F.genalpha(rho)
    assert abs(ga - (0.5 + am - af)) < 1e-15


# ---------------------------------------------------------------- geometry
def test_counts_golden():
    for r in _rows(os.path.join(GOLDEN, "tube_counts.txt")):
        name = r[0]
        nodes, tets, iface, unk, fl, free = map(int, r[1:])
        p = F.make_params(**F.PRESETS[name])
        if nodes > 100000:
            nr = p.n_rad_f + p.n_rad_s
            assert (1 + p.n_circ * nr) * (p.n_ax + 1) == nodes
            continue
        m = F.build_mesh(p)
        assert (m.n_nodes, m.n_elem, m.n_iface, m.n_fluid) == (nodes, tets, iface, fl)
        assert 3 * m.n_nodes + m.n_p == unk
        assert int((~m.dir_m).sum()) == free


def test_gauss_rule_integrates_quadratics():
    # int lambda_a lambda_b dV = V (1 + delta_ab) / 20, int lambda_a = V / 4
    N = F.gauss_points()
    w = 0.25
    assert np.allclose(N.sum(axis=1), 1.0)
    M = w * N.T @ N
    assert np.allclose(M, (np.ones((4, 4)) + np.eye(4)) / 20.0, atol=1e-15)
    assert np.allclose(w * N.sum(axis=0), 0.25)


def test_mesh_conforming_and_volume():
    p = F.make_params(**F.PRESETS["tube_mini"])
    m = F.build_mesh(p)
    faces = {}
    for t in m.ien:
        for f in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
            key = tuple(sorted(t[list(f)]))
            faces[key] = faces.get(key, 0) + 1
    counts = np.array(list(faces.values()))
    assert counts.max() == 2
    # boundary triangles: 2 end caps of the section + lateral outer surface
    nc, nr, na = p.n_circ, p.n_rad_f + p.n_rad_s, p.n_ax
    tri_sec = nc + 2 * nc * (nr - 1)
    assert int((counts == 1).sum()) == 2 * tri_sec + 2 * nc * na
    # volumes: the mesh fills the polygonal prism exactly
    x = m.xyz[m.ien]
    vol = np.abs(np.einsum("ni,ni->n", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))) / 6
    Ro = p.R + p.wall
    poly = 0.5 * nc * Ro * Ro * math.sin(2 * math.pi / nc)
    assert abs(vol.sum() - poly * p.L) < 1e-12 * poly * p.L
    assert vol.min() > 0


def test_mesh_laplacian_reproduces_linear_fields():
    p = F.make_params(**F.PRESETS["tube_mini"])
    asm = F.Assembler(p)
    L = to_csr(asm.mesh_laplacian())
    m = asm.mesh
    fl = np.nonzero(m.fluid_id >= 0)[0]
    X = m.xyz[fl]
    assert np.allclose(L @ np.ones(L.shape[0]), 0.0, atol=1e-13)
    # x^T L x = int |grad x|^2 = volume of the lumen polygon prism
    poly = 0.5 * p.n_circ * p.R ** 2 * math.sin(2 * math.pi / p.n_circ)
    for c in range(3):
        assert abs(X[:, c] @ (L @ X[:, c]) - poly * p.L) < 1e-10 * poly * p.L
    # rows of interior nodes annihilate linear fields
    interior = (m.ring[fl] < p.n_rad_f) & (m.layer[fl] > 0) & (m.layer[fl] < p.n_ax)
    for c in range(3):
        assert np.abs((L @ X[:, c])[interior]).max() < 1e-12
    assert abs(L - L.T).max() < 1e-15


def test_interface_pressure_duplication(mini_system):
    s, m = mini_system, mini_system.mesh
    assert m.n_p == m.n_nodes + m.n_iface
    assert s.D.nb_rows == m.n_p and s.A.nb_rows == m.n_nodes
    # fluid elements use the node index, solid elements the duplicate
    iface = m.iface_of >= 0
    for e in range(m.n_elem):
        for a in range(4):
            n = m.ien[e, a]
            if iface[n]:
                expect = n if m.etype[e] == 0 else m.n_nodes + m.iface_of[n]
                assert m.pien[e, a] == expect
    # the fluid pressure of an interface node couples only to fluid-element nodes
    C = s.C
    fluid_node = m.fluid_id >= 0
    for n in np.nonzero(iface)[0][:50]:
        cols = C.col[C.row_ptr[n]:C.row_ptr[n + 1]]
        assert fluid_node[cols].all()
        dup = m.n_nodes + m.iface_of[n]
        cols = C.col[C.row_ptr[dup]:C.row_ptr[dup + 1]]
        assert (m.ring[cols] >= F.PRESETS["tube_mini"]["n_rad_f"]).all()


def test_mesh_matrix_spd(mini_system):
    L = to_csr(mini_system.L).toarray()
    assert np.abs(L - L.T).max() <= 1e-14 * np.abs(L).max()
    np.linalg.cholesky(L)


# ---------------------------------------------------------------- element
def _random_tet(rng, scale=1.0):
    while True:
        x = rng.standard_normal((4, 3)) * scale
        v = np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]]))
        if abs(v) > 0.05 * scale ** 3:
            return x


def _grads(x):
    J = np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]], axis=1)
    Ji = np.linalg.inv(J)
    g = np.zeros((4, 3))
    g[1:] = Ji
    g[0] = -Ji.sum(axis=0)
    return g, abs(np.linalg.det(J)) / 6


def test_metric_invariant_under_node_permutation():
    rng = np.random.default_rng(1)
    for _ in range(5):
        x = _random_tet(rng)
        Gs = []
        for perm in ([0, 1, 2, 3], [1, 2, 3, 0], [3, 0, 2, 1], [2, 3, 1, 0]):
            g, _ = _grads(x[perm])
            Gs.append(F.metric_G(g[1:]))
        for G in Gs[1:]:
            assert np.allclose(G, Gs[0], rtol=1e-12)


def test_metric_reference_element_and_scaling():
    c = 2 ** (1 / 3) / 2
    M = c * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]])
    assert np.allclose(F.metric_G(np.eye(3)), M)
    # G scales like 1/h^2
    assert np.allclose(F.metric_G(np.eye(3) / 0.1), M / 0.01)


def test_tau_limits():
    G = F.metric_G(np.eye(3) * 20.0)
    rho, mu = 1.06, 0.04
    # small dt: tau_M -> dt / (2 rho)   (sqrt(C_T) = 2)
    tm, tc = F.tau_fluid(G, np.zeros(3), rho, mu, 1e-9)
    assert abs(tm - 1e-9 / (2 * rho)) < 1e-6 * tm
    assert abs(tc * tm * np.trace(G) - 1.0) < 1e-12
    # diffusion limit: tau_M -> 1 / (rho * 6 nu ||G||_F)   (sqrt(C_I) = 6)
    tm, _ = F.tau_fluid(G, np.zeros(3), rho, 1e3, 1e12)
    nu = 1e3 / rho
    assert abs(tm - 1.0 / (rho * 6 * nu * np.linalg.norm(G))) < 1e-9 * tm
    # advection limit: tau_M -> 1 / (rho sqrt(u G u))
    u = np.array([1e6, -2e6, 3e5])
    tm, _ = F.tau_fluid(G, u, rho, 1e-12, 1e12)
    assert abs(tm - 1.0 / (rho * math.sqrt(u @ G @ u))) < 1e-9 * tm


def test_circumsphere_diameter():
    rng = np.random.default_rng(2)
    x = _random_tet(rng)
    d = F.circum_diameter(x)
    c = None
    # centre equidistant from the four vertices
    A = 2 * (x[1:] - x[0])
    b = (x[1:] ** 2).sum(1) - (x[0] ** 2).sum()
    c = np.linalg.solve(A, b)
    r = np.linalg.norm(x - c, axis=1)
    assert np.allclose(r, d / 2)
    # regular tet of edge 1: circumradius sqrt(6)/4
    reg = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]]) / (2 * math.sqrt(2))
    assert abs(F.circum_diameter(reg) - math.sqrt(6) / 2) < 1e-14


def test_fluid_element_mass_block():
    # at rest (v = 0, p = 0) with only the rate coefficient the tangent is the
    # consistent mass matrix rho * V (1 + delta_ab) / 20 * I3
    rng = np.random.default_rng(3)
    x = _random_tet(rng)
    _, V = _grads(x)
    rho = 1.06
    out = F.fluid_element(x, np.zeros((4, 3)), np.zeros(4), rho=rho, cm=0.7, cf=0.0)
    Mab = V * (np.ones((4, 4)) + np.eye(4)) / 20
    expect = 0.7 * rho * np.einsum("ab,ik->abik", Mab, np.eye(3))
    assert np.allclose(out["Ae"], expect, rtol=1e-13, atol=1e-16)


def test_fluid_element_viscous_block_kernel():
    # rates off, at rest: translations and rigid rotations are in the kernel
    rng = np.random.default_rng(4)
    x = _random_tet(rng)
    out = F.fluid_element(x, np.zeros((4, 3)), np.zeros(4), mu=0.04, cm=0.0, cf=1.0, dt=1e-4)
    A = out["Ae"].transpose(0, 2, 1, 3).reshape(12, 12)
    for k in range(3):
        t = np.zeros((4, 3)); t[:, k] = 1.0
        assert np.abs(A @ t.ravel()).max() < 1e-12 * np.abs(A).max()
    # a rotation has zero rate of deformation and zero divergence
    w = np.array([0.3, -1.2, 0.7])
    rot = np.cross(w, x)
    assert np.abs(A @ rot.ravel()).max() < 1e-12 * np.abs(A).max() * np.abs(rot).max()
    assert np.allclose(A, A.T, rtol=1e-12, atol=1e-16)


def test_fluid_element_gradient_divergence_pair():
    # at rest with cm = 0 the stabilisation drops out of B and C:
    # C_ab,k = cf V/4 dN_b,k and B = -C^T (discrete gradient = -divergence^T)
    rng = np.random.default_rng(5)
    x = _random_tet(rng)
    g, V = _grads(x)
    cf = 0.37
    out = F.fluid_element(x, np.zeros((4, 3)), np.zeros(4), cm=0.0, cf=cf, tau_mode=1)
    C = out["Ce"]
    expect = cf * V / 4 * np.broadcast_to(g[None, :, :], (4, 4, 3))
    assert np.allclose(C, expect, rtol=1e-12)
    assert np.allclose(out["Be"], -C.transpose(1, 0, 2), rtol=1e-12)
    # D = cf tau_M V gradN_a . gradN_b
    tm = out["tau"][0]
    assert np.allclose(out["De"], cf * tm * V * g @ g.T, rtol=1e-12)


def test_fluid_residual_vanishes_for_rest_state():
    rng = np.random.default_rng(6)
    x = _random_tet(rng)
    g, V = _grads(x)
    out = F.fluid_element(x, np.zeros((4, 3)), np.full(4, 3.5), want_mat=False)
    # constant pressure, no flow: only the weak pressure gradient remains,
    # -int dN_a/dx_i p = -p V dN_a/dx_i, which sums to zero over the nodes
    assert np.allclose(out["Rm"], -3.5 * V * g, rtol=1e-12, atol=1e-14)
    assert np.abs(out["Rm"].sum(axis=0)).max() < 1e-12
    assert np.abs(out["Rp"]).max() < 1e-15


def test_solid_element_blocks():
    rng = np.random.default_rng(7)
    x = _random_tet(rng)
    g, V = _grads(x)
    z = np.zeros((4, 3))
    cm, cf, cu, rho, mu = 0.8, 0.3, 0.11, 1.0, 2.0
    out = F.solid_element(x, z, z, np.zeros(4), z, rho, mu, 0.05, 0.0, cm, cf, cu)
    A = out["Ae"].transpose(0, 2, 1, 3).reshape(12, 12)
    Mab = V * (np.ones((4, 4)) + np.eye(4)) / 20
    # mass + elasticity; elasticity annihilates translations and rotations
    mass = cm * rho * np.kron(Mab, np.eye(3))
    K = (A - mass) / cu
    for k in range(3):
        t = np.zeros((4, 3)); t[:, k] = 1.0
        assert np.abs(K @ t.ravel()).max() < 1e-10 * np.abs(K).max()
    rot = np.cross(np.array([0.2, 0.5, -0.9]), x)
    assert np.abs(K @ rot.ravel()).max() < 1e-10 * np.abs(K).max() * np.abs(rot).max()
    assert np.allclose(K, K.T, rtol=1e-12)
    assert np.allclose(out["Be"], -cf * V / 4 * np.broadcast_to(g[:, None, :], (4, 4, 3)), rtol=1e-12)
    expectC = cf * V / 4 * g[None, :, :] + cm * 0.05 * rho * V / 4 * g[:, None, :]
    assert np.allclose(out["Ce"], expectC, rtol=1e-12)
    assert np.allclose(out["De"], cf * 0.05 * V * g @ g.T, rtol=1e-12)


# ---------------------------------------------------------------- tangent
def _bsr_dense(M):
    return to_csr(M)


@pytest.mark.parametrize("preset", ["tube_tiny", "tube_mini"])
def test_tangent_matches_central_differences(preset):
    """K dy = (R(y + e dy) - R(y - e dy)) / (2e) with tau frozen, where the
    increment moves vdot by alpha_m, v and p by alpha_f gamma dt and the
    solid displacement by (alpha_f gamma dt)^2 / alpha_m (Sec. 3.5)."""
    p = F.make_params(**F.PRESETS[preset])
    asm = F.Assembler(p)
    v, pr = asm.initial_state()
    m = asm.mesh
    rng = np.random.default_rng(11)
    nn, np_ = m.n_nodes, m.n_p
    vd = 50.0 * rng.standard_normal(3 * nn)      # exercise the rate terms
    u = 1e-3 * rng.standard_normal(3 * nn)
    vhat = 2.0 * rng.standard_normal(3 * nn)
    am, af, ga = F.genalpha(p.rho_inf)
    cf = af * ga * p.dt
    cu = cf * cf / am
    tau = np.zeros(8 * m.n_elem)
    base = asm.evaluate(v, pr, vd, u, vhat, am, cf, cu, tau=tau, tau_mode=1, want_mat=True)
    dv = rng.standard_normal(3 * nn) * 5.0
    dp = rng.standard_normal(np_) * 500.0
    K = sp.bmat([[_bsr_dense(base["A"]), _bsr_dense(base["B"])],
                 [_bsr_dense(base["C"]), _bsr_dense(base["D"])]]).tocsr()
    lin = K @ np.concatenate([dv, dp])
    eps = 1e-3
    def res(s):
        o = asm.evaluate(v + s * cf * dv, pr + s * cf * dp, vd + s * am * dv, u + s * cu * dv, vhat,
                         am, cf, cu, tau=tau, tau_mode=2, want_mat=False)
        return np.concatenate([o["Rm"], o["Rp"]])
    fd = (res(eps) - res(-eps)) / (2 * eps)
    err = np.linalg.norm(fd - lin) / np.linalg.norm(lin)
    assert err < 1e-6, err


# ---------------------------------------------------------------- physics
def _steady_poiseuille(n_circ, n_rad, n_ax, L=2.0):
    """Steady rigid-wall tube (dt -> infinity, rates off) solved by Newton on
    the generator's residual and tangent."""
    import scipy.sparse.linalg as spl
    p = F.make_params(n_circ=n_circ, n_rad_f=n_rad, n_rad_s=1, n_ax=n_ax, fluid_only=1,
                      L=L, dt=1e12, pert_amp=0.0)
    asm = F.Assembler(p)
    v, pr = asm.initial_state()
    pr[:] = 0.0
    m = asm.mesh
    dirv = np.repeat(m.dir_v, 3)
    for _ in range(8):
        o = asm.evaluate(v, pr, cm=0.0, cf=1.0, want_mat=True)
        K = sp.bmat([[to_csr(o["A"]), to_csr(o["B"])], [to_csr(o["C"]), to_csr(o["D"])]]).tolil()
        R = np.concatenate([o["Rm"], o["Rp"]])
        nv = 3 * m.n_nodes
        idx = np.nonzero(dirv)[0]
        K[idx, :] = 0.0
        K[idx, idx] = 1.0
        R[idx] = 0.0
        d = spl.spsolve(K.tocsc(), -R)
        v += d[:nv]
        pr += d[nv:]
        if np.linalg.norm(d[:nv]) < 1e-10 * np.linalg.norm(v):
            break
    return p, m, v, pr


def test_poiseuille_steady_flow():
    """A rigid tube with a parabolic inflow keeps the Poiseuille profile
    u = u_max (1 - r^2/R^2) and dp/dz = -4 mu u_max / R^2 (= -53.33 dyn/cm^3
    for mu = 0.04, u_max = 30, R = 0.3) away from the outlet, converging
    under refinement."""
    errs, slope_errs = [], []
    G = -4 * 0.04 * 30.0 / 0.3 ** 2
    assert abs(G + 53.333333333) < 1e-6
    for (nc, nr, na) in [(12, 3, 8), (24, 6, 16)]:
        p, m, v, pr = _steady_poiseuille(nc, nr, na)
        mid = m.layer == na // 2
        r2 = (m.xyz[:, 0] ** 2 + m.xyz[:, 1] ** 2) / p.R ** 2
        vz = v.reshape(-1, 3)[:, 2]
        exact = p.u_max * (1 - r2)
        errs.append(np.abs(vz[mid] - exact[mid]).max() / p.u_max)
        # pressure gradient on the axis between 1/4 and 1/2 of the length
        ax = m.ring == 0
        z = m.xyz[ax, 2]
        pa = pr[: m.n_nodes][ax]
        sel = (z >= 0.25 * p.L) & (z <= 0.5 * p.L)
        slope_errs.append(abs(np.polyfit(z[sel], pa[sel], 1)[0] - G) / abs(G))
    # second-order convergence (halving h divides the errors by ~4; the
    # polygonal lumen adds an O(h^2) geometric error of the same order)
    assert errs[1] < 0.02 and errs[1] < errs[0] / 2.5, errs
    assert slope_errs[1] < 0.05 and slope_errs[1] < slope_errs[0] / 2.5, slope_errs


def test_system_rhs_zero_on_dirichlet(mini_system):
    s, m = mini_system, mini_system.mesh
    bv = s.b[: 3 * s.n_v].reshape(-1, 3)
    assert np.all(bv[m.dir_v] == 0.0)
    A = to_csr(s.A)
    idx = np.nonzero(np.repeat(m.dir_v, 3))[0]
    Ad = A[idx][:, idx].toarray()
    assert np.allclose(Ad, np.eye(idx.size))
    assert abs(A[:, idx]).sum() == idx.size       # only the identity entries
    assert abs(to_csr(s.C)[:, idx]).sum() == 0.0
    assert abs(to_csr(s.B)[idx]).sum() == 0.0


def test_generator_deterministic_across_threads():
    a = F.tube_system("tube_mini", threads=1)
    b = F.tube_system("tube_mini", threads=3)
    for M, N in ((a.A, b.A), (a.B, b.B), (a.C, b.C), (a.D, b.D), (a.L, b.L)):
        assert np.array_equal(M.row_ptr, N.row_ptr) and np.array_equal(M.col, N.col)
        assert np.array_equal(M.val, N.val)
    assert np.array_equal(a.b, b.b)
    F.lib().tg_set_threads(os.cpu_count() or 1)


# ---------------------------------------------------------------- resistance outlet
def test_outlet_vector_integrates_the_outlet_section():
    """a_{A,z} = int_outlet N_A dGamma sums to the area of the outlet's lumen
    polygon (n_circ vertices on the lumen radius: n/2 R^2 sin(2 pi / n)),
    only z components are nonzero, and a^T v is the discrete Poiseuille flux
    pi R^2 u_max / 2 up to the O(h^2) interpolation error."""
    s = F.tube_system("tube_small", keep_mesh=True)
    p = s.params
    a = F.outlet_vector(s.mesh, p["n_ax"], zero_dirichlet=False)
    nc, R = p["n_circ"], p["R"]
    assert abs(a.sum() - 0.5 * nc * R * R * np.sin(2 * np.pi / nc)) <= 1e-12 * a.sum()
    assert np.all(a.reshape(-1, 3)[:, :2] == 0.0)
    z_nodes = np.nonzero(a.reshape(-1, 3)[:, 2])[0]
    assert np.all(s.mesh.layer[z_nodes] == p["n_ax"]) and np.all(s.mesh.fluid_id[z_nodes] >= 0)
    v = np.zeros(3 * s.mesh.n_nodes)
    r2 = s.mesh.xyz[:, 0] ** 2 + s.mesh.xyz[:, 1] ** 2
    v[2::3] = np.where(s.mesh.fluid_id >= 0, p["u_max"] * np.clip(1 - r2 / R ** 2, 0, None), 0.0)
    q = a @ v
    assert abs(q - np.pi * R * R * p["u_max"] / 2) <= 0.1 * q


def test_resistance_outlet_terms():
    """c = alpha_f gamma dt R_out (closed form); a is zero on Dirichlet rows;
    zero resistance gives the zero-traction system unchanged."""
    r_out = 2.7e4
    s = F.tube_system("tube_mini", outlet_resistance=r_out, keep_mesh=True)
    am, af, ga = F.genalpha(s.params["rho_inf"])
    assert s.c_out[0] == pytest.approx(af * ga * s.params["dt"] * r_out, rel=1e-15)
    a = s.a_out[0]
    assert np.all(a[np.repeat(s.mesh.dir_v, 3)] == 0.0) and a.sum() > 0
    s0 = F.tube_system("tube_mini")
    s1 = F.tube_system("tube_mini", outlet_resistance=0.0)
    assert s1.a_out is None and np.array_equal(s0.b, s1.b)


# ------------------------------------------------------------- bifurcation
def _faces(m):
    FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
    f = np.sort(m.ien[:, FACES].reshape(-1, 3), axis=1)
    key, inv, cnt = np.unique(f, axis=0, return_inverse=True, return_counts=True)
    return key, inv.ravel(), cnt


def test_bifurcation_mesh_is_conforming_sealed_and_splits_in_two():
    """The bifurcation (one extruded O-grid section whose septum band is lumen
    in the parent, solid at the carina tip and removed between the sheared
    daughters): every face is shared by at most two tets, every tet has a
    positive volume, the lumen touches the outside only at the inlet and
    outlet planes, the fluid of a parent layer is one connected piece and
    that of a daughter layer two, and every daughter layer has the same
    volume (the shear keeps volumes)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    p = F.make_params(**F.PRESETS["bif_mini"])
    m = F.build_mesh(p)
    key, inv, cnt = _faces(m)
    assert cnt.max() == 2
    x = m.xyz[m.ien]
    vol = np.abs(np.einsum("ni,ni->n", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))) / 6
    assert vol.min() > 0.05 * vol.max()
    owner = np.repeat(np.arange(m.n_elem), 4)
    fl = m.etype[owner] == 0
    kf = np.bincount(inv[fl], minlength=len(key))
    ks = np.bincount(inv[~fl], minlength=len(key))
    z = m.xyz[key[(kf == 1) & (ks == 0)]][:, :, 2]
    zmax = m.xyz[:, 2].max()
    assert np.all(np.all(z == 0.0, axis=1) | np.all(np.abs(z - zmax) < 1e-12, axis=1))
    # fluid components per element layer
    dz = zmax / p.n_ax
    lay = np.floor(x[:, :, 2].mean(axis=1) / dz).astype(int)
    both = np.nonzero((kf == 2))[0]
    fi = np.full(len(key), -1)
    fj = np.full(len(key), -1)
    for e, k in zip(owner[fl], inv[fl]):
        if fi[k] < 0:
            fi[k] = e
        else:
            fj[k] = e
    adj = sp.coo_matrix((np.ones(both.size), (fi[both], fj[both])), shape=(m.n_elem, m.n_elem)).tocsr()
    comps = []
    for k in range(p.n_ax):
        sel = np.nonzero((lay == k) & (m.etype == 0))[0]
        comps.append(csg.connected_components(adj[sel][:, sel], directed=False)[0])
    assert comps[0] == 1 and comps[-1] == 2
    assert sorted(set(comps)) == [1, 2] and comps == sorted(comps)
    # the solid carina tip already splits the lumen; the void cells go after it
    first_dau = comps.index(2) + p.bif_tip_layers
    vl = np.bincount(lay, weights=vol, minlength=p.n_ax)
    assert np.allclose(vl[first_dau:], vl[-1], rtol=1e-10) and vl[first_dau - 1] > vl[-1]
    # the daughters diverge: at the outlet the two lumens lie on either side
    out = (np.abs(m.xyz[:, 2] - zmax) < 1e-12) & (m.fluid_id >= 0)
    xs = m.xyz[out, 0]
    gap = np.sort(xs)
    assert gap.min() < -p.R and gap.max() > p.R and np.diff(gap).max() > 0.5 * p.R


def test_bifurcation_interface_and_pressure_duplication():
    """Interface nodes are exactly the nodes of both fluid and solid tets;
    solid tets read the duplicated pressure there, fluid tets the node's;
    the mesh-motion Laplacian annihilates linear fields in its interior rows
    and is symmetric positive definite once the Dirichlet rows are
    eliminated."""
    p = F.make_params(**F.PRESETS["bif_mini"])
    asm = F.Assembler(p)
    m = asm.mesh
    hf = np.zeros(m.n_nodes, bool)
    hs = np.zeros(m.n_nodes, bool)
    hf[m.ien[m.etype == 0].ravel()] = True
    hs[m.ien[m.etype == 1].ravel()] = True
    np.testing.assert_array_equal(m.iface_of >= 0, hf & hs)
    assert m.n_p == m.n_nodes + int((hf & hs).sum())
    solid = m.etype == 1
    dup = m.iface_of[m.ien] >= 0
    np.testing.assert_array_equal(m.pien[solid & dup.any(axis=1)] >= m.n_nodes,
                                  dup[solid & dup.any(axis=1)])
    np.testing.assert_array_equal(m.pien[~solid], m.ien[~solid])
    L = to_csr(asm.mesh_laplacian())
    fl = np.nonzero(m.fluid_id >= 0)[0]
    X = m.xyz[fl]
    free = ~m.dir_m
    for c in range(3):
        assert np.allclose((L @ X[:, c])[free], 0.0, atol=1e-12 * np.abs(L).max())
    Lf = L[free][:, free].toarray()
    assert np.allclose(Lf, Lf.T) and np.linalg.eigvalsh(Lf).min() > 0


def test_rhs_only_matches_the_full_build():
    """The residual-only right-hand side equals the full build's, bit for
    bit, for a tube and for the bifurcation at another inflow peak."""
    for name, u in (("bif_mini", 17.0), ("tube_mini", 44.0)):
        np.testing.assert_array_equal(F.rhs_only(name, u_max=u), F.tube_system(name, u_max=u).b)


def test_system_file_round_trip(tmp_path):
    """save_system / load_system keep every array bit for bit (the layout the
    C client reads), and a truncated file is rejected."""
    s = F.tube_system("tube_mini")
    path = str(tmp_path / "sys.bin")
    F.save_system(s, path)
    t = F.load_system(path)
    for a, b in ((s.A, t.A), (s.B, t.B), (s.C, t.C), (s.D, t.D)):
        assert (a.br, a.bc, a.nb_rows, a.nb_cols) == (b.br, b.bc, b.nb_rows, b.nb_cols)
        np.testing.assert_array_equal(a.row_ptr, b.row_ptr)
        np.testing.assert_array_equal(a.col, b.col)
        np.testing.assert_array_equal(a.val, b.val)
    np.testing.assert_array_equal(s.b, t.b)
    with open(path, "rb") as f:
        data = f.read()
    with open(path, "wb") as f:
        f.write(data[:-8])
    with pytest.raises(ValueError):
        F.load_system(path)


def test_bifurcation_boundary_layers_are_graded():
    """With n boundary layers of ratio r the last n lumen-ring intervals along
    a ray shrink by r each towards the wall, the inner ones stay uniform, and
    the graded mesh is still conforming with positive volumes."""
    kw = dict(F.PRESETS["bif_mini"], bif_bl_layers=3, bif_bl_ratio=0.6)
    p = F.make_params(**kw)
    m = F.build_mesh(p)
    nc, nrf = p.n_circ, p.n_rad_f
    ncore = (nc + 1) ** 2
    # the ray through the core corner (0, 0): node layer 0 keeps every section node
    ids = [0] + [ncore + (q - 1) * 4 * nc for q in range(1, nrf + 1)]
    r = np.linalg.norm(m.xyz[ids, :2], axis=1)
    w = np.diff(r)
    np.testing.assert_allclose(w[-3:] / w[-4:-1], 0.6, rtol=1e-9)
    np.testing.assert_allclose(r[-1], p.R, rtol=1e-12)
    key, inv, cnt = _faces(m)
    assert cnt.max() == 2
    x = m.xyz[m.ien]
    vol = np.abs(np.einsum("ni,ni->n", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0])))
    assert vol.min() > 0.01 * vol.max()


# ------------------------------------------------- first-order generalized-alpha
def _sdof_step(rho_inf, Om):
    """One step of the first-order generalized-alpha scheme (Sec. 3.4) on
    the single-degree-of-freedom oscillator d' = v, v' = -w^2 d written as a
    first-order system (dt = 1, w = Om): unknowns (d, v, d', v') at t_{n+1};
    returns the 4 x 4 amplification matrix built from the scheme's four
    defining relations and the constants of the generator."""
    am, af, ga = F.genalpha(rho_inf)
    w2 = Om * Om
    M = np.array([[1, 0, -ga, 0], [0, 1, 0, -ga], [0, -af, am, 0], [w2 * af, 0, 0, am]], dtype=float)
    N = np.array([[1, 0, 1 - ga, 0], [0, 1, 0, 1 - ga], [0, 1 - af, -(1 - am), 0],
                  [-w2 * (1 - af), 0, 0, -(1 - am)]], dtype=float)
    return np.linalg.solve(M, N), (am, af, ga)


def test_first_order_generalized_alpha_limits_and_order():
    """The constants alpha_m = (3 - rho) / (2 (1 + rho)), alpha_f = gamma =
    1 / (1 + rho) make the scheme what the appendix's analysis states: the
    spectral radius of the amplification matrix tends to 1 as Omega = w dt ->
    0 and to rho_inf as Omega -> infinity; the first step's displacement at
    Omega -> infinity is (1 - alpha_m / (alpha_f gamma)) d_0 (the appendix's
    printed limit); the global error at a fixed time falls four-fold when dt
    halves (second order).  A wrong constant breaks one of them."""
    from oracle import corrector
    for rho in (0.0, 0.25, 0.5, 1.0):
        A, (am, af, ga) = _sdof_step(rho, 1e9)
        assert abs(np.abs(np.linalg.eigvals(A)).max() - rho) < 1e-3
        A0, _ = _sdof_step(rho, 1e-4)
        assert abs(np.abs(np.linalg.eigvals(A0)).max() - 1.0) < 1e-6
        d0 = 0.7
        x1 = A @ np.array([d0, 1.3, 1.3, -1e18 * d0])  # compatible start: d'(0) = v(0), v'(0) = -w^2 d(0)
        assert x1[0] == pytest.approx((1.0 - am / (af * ga)) * d0, rel=1e-6)
        # the oracle's corrector weights come from the same constants
        amo, cf, cu = corrector.genalpha_weights(rho, 1e-4)
        assert amo == pytest.approx(am, rel=1e-15) and cf == pytest.approx(af * ga * 1e-4, rel=1e-15)
        assert cu == pytest.approx(cf * cf / am, rel=1e-15)
    for rho in (0.0, 0.5):
        errs = []
        for n in (200, 400):
            A, _ = _sdof_step(rho, 1.0 / n)
            x = np.array([1.0, 0.0, 0.0, -1.0 / n ** 2])
            for _ in range(n):
                x = A @ x
            errs.append(abs(x[0] - np.cos(1.0)))
        assert 3.8 < errs[0] / errs[1] < 4.2


def test_bifurcation_state_inlet_is_poiseuille_and_walls_rest():
    """The bifurcation's state: at the inlet section the axial velocity is
    u_max (1 - r^2 / R^2) exactly (the perturbation vanishes there) with no
    transverse part; interface and solid nodes are at rest; the fluid
    pressure falls along the arc length (parent z, then each daughter's
    axis), the same in both daughters by symmetry of the draw's profile."""
    p = F.make_params(**F.PRESETS["bif_mini"])
    asm = F.Assembler(p)
    m = asm.mesh
    v, pr = asm.initial_state()
    V = v.reshape(-1, 3)
    inlet = (m.layer == 0) & (m.fluid_id >= 0) & (m.iface_of < 0)
    r2 = (m.xyz[inlet, :2] ** 2).sum(axis=1)
    np.testing.assert_allclose(V[inlet, 2], p.u_max * np.clip(1 - r2 / p.R ** 2, 0, None), rtol=1e-12, atol=1e-12)
    assert np.all(V[inlet, :2] == 0.0)
    rest = (m.fluid_id < 0) | (m.iface_of >= 0)
    assert np.all(V[rest] == 0.0)
    fl = m.fluid_id >= 0
    z = m.xyz[fl, 2]
    order = np.argsort(z)
    assert np.all(np.diff(pr[:m.n_nodes][fl][order]) <= 1e-12)
    # the two daughters: mirror pressures at the outlet
    out = fl & (m.layer == p.n_ax)
    xo = m.xyz[out, 0]
    assert np.allclose(np.sort(pr[:m.n_nodes][out][xo < 0]), np.sort(pr[:m.n_nodes][out][xo > 0]))
