"""Seeded synthetic inputs for the vascular FSI block solver.

This package builds the linear systems that both the CUDA solver and the
CPU oracle consume.  It holds no solver arithmetic: it generates meshes,
evaluates the paper's element loop (unified-continuum VMS on linear tets,
Sec. 3.1-3.2, tangent of the first-order generalized-alpha scheme,
Sec. 3.4-3.5) and returns the block Jacobian [[A, B], [C, D]], its
right-hand side and the mesh-motion Laplacian (harmonic extension, Sec. 2.2)
as plain numpy arrays.

The C source sits in ``csrc/tubegen.c`` and is compiled on first use with
gcc (OpenMP) into ``_tubegen.so`` beside this file.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "tubegen.c")
_SO = os.path.join(_HERE, "_tubegen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library (gcc, -O2, OpenMP) if it is stale."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                   "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("n_circ", C.c_int), ("n_rad_f", C.c_int), ("n_rad_s", C.c_int),
        ("n_ax", C.c_int), ("fluid_only", C.c_int),
        ("R", C.c_double), ("wall", C.c_double), ("L", C.c_double),
        ("sten_sigma", C.c_double), ("sten_frac", C.c_double),
        ("rho_f", C.c_double), ("mu_f", C.c_double), ("rho_s", C.c_double),
        ("E_s", C.c_double), ("nu_s", C.c_double),
        ("dt", C.c_double), ("rho_inf", C.c_double),
        ("u_max", C.c_double), ("pert_amp", C.c_double), ("mesh_amp", C.c_double),
        ("c_m_solid", C.c_double), ("c_c_solid", C.c_double),
        ("seed", C.c_uint64),
        ("bif_angle_deg", C.c_double), ("bif_daughter_len", C.c_double), ("bif_tip_layers", C.c_int),
        ("bif_bl_layers", C.c_int), ("bif_bl_ratio", C.c_double),
    ]


class _Mesh(C.Structure):
    _fields_ = [
        ("n_sec", C.c_int), ("n_nodes", C.c_int), ("n_elem", C.c_int), ("n_iface", C.c_int),
        ("n_p", C.c_int), ("n_fluid", C.c_int),
        ("xyz", C.POINTER(C.c_double)), ("ring", C.POINTER(C.c_int)),
        ("layer", C.POINTER(C.c_int)), ("sec", C.POINTER(C.c_int)),
        ("ien", C.POINTER(C.c_int)), ("pien", C.POINTER(C.c_int)),
        ("etype", C.POINTER(C.c_ubyte)), ("iface_of", C.POINTER(C.c_int)),
        ("fluid_id", C.POINTER(C.c_int)), ("dir_v", C.POINTER(C.c_ubyte)),
        ("dir_m", C.POINTER(C.c_ubyte)),
    ]


class _Bsr(C.Structure):
    _fields_ = [
        ("nb_rows", C.c_int), ("nb_cols", C.c_int), ("br", C.c_int), ("bc", C.c_int),
        ("nnzb", C.c_int), ("row_ptr", C.POINTER(C.c_int)), ("col", C.POINTER(C.c_int)),
        ("val", C.POINTER(C.c_double)),
    ]


class _Raw(C.Structure):
    _fields_ = [("A", _Bsr), ("B", _Bsr), ("C", _Bsr), ("D", _Bsr), ("L", _Bsr),
                ("Rm", C.POINTER(C.c_double)), ("Rp", C.POINTER(C.c_double))]


class _System(C.Structure):
    _fields_ = [("A", _Bsr), ("B", _Bsr), ("C", _Bsr), ("D", _Bsr),
                ("b", C.POINTER(C.c_double)), ("L", _Bsr),
                ("mesh_b", C.POINTER(C.c_double)), ("mesh_g", C.POINTER(C.c_double))]


class ElemOut(C.Structure):
    _fields_ = [("Ae", C.c_double * 144), ("Be", C.c_double * 48), ("Ce", C.c_double * 48),
                ("De", C.c_double * 16), ("Rm", C.c_double * 12), ("Rp", C.c_double * 4)]

    def arrays(self):
        return dict(
            Ae=np.array(self.Ae).reshape(4, 4, 3, 3), Be=np.array(self.Be).reshape(4, 4, 3),
            Ce=np.array(self.Ce).reshape(4, 4, 3), De=np.array(self.De).reshape(4, 4),
            Rm=np.array(self.Rm).reshape(4, 3), Rp=np.array(self.Rp).reshape(4))


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.POINTER
        L.tg_default_params.argtypes = [P(Params)]
        L.tg_genalpha.argtypes = [C.c_double, P(C.c_double), P(C.c_double), P(C.c_double)]
        L.tg_mesh_build.argtypes = [P(Params)]
        L.tg_mesh_build.restype = P(_Mesh)
        L.tg_mesh_free.argtypes = [P(_Mesh)]
        L.tg_state_init.argtypes = [P(Params), P(_Mesh), P(C.c_double), P(C.c_double)]
        L.tg_assemble.argtypes = [P(Params), P(_Mesh)] + [P(C.c_double)] * 5 + \
            [C.c_double] * 3 + [C.c_int, P(C.c_double), C.c_int]
        L.tg_assemble.restype = P(_Raw)
        L.tg_raw_free.argtypes = [P(_Raw)]
        L.tg_mesh_laplacian_raw.argtypes = [P(_Mesh)]
        L.tg_mesh_laplacian_raw.restype = P(_Bsr)
        L.tg_bsr_free.argtypes = [P(_Bsr)]
        L.tg_finalize.argtypes = [P(_Mesh), P(_Raw), P(_Bsr), P(Params)]
        L.tg_finalize.restype = P(_System)
        L.tg_system_free.argtypes = [P(_System)]
        L.tg_set_threads.argtypes = [C.c_int]
        L.tg_metric.argtypes = [P(C.c_double), P(C.c_double)]
        L.tg_tau_fluid.argtypes = [P(C.c_double), P(C.c_double)] + [C.c_double] * 3 + \
            [P(C.c_double), P(C.c_double)]
        L.tg_circum_diameter.argtypes = [P(C.c_double)]
        L.tg_circum_diameter.restype = C.c_double
        L.tg_gauss_points.argtypes = [P(C.c_double)]
        L.tg_fluid_element.argtypes = [P(C.c_double)] * 5 + [C.c_double] * 5 + \
            [C.c_int, P(C.c_double), C.c_int, P(ElemOut)]
        L.tg_solid_element.argtypes = [P(C.c_double)] * 5 + [C.c_double] * 7 + \
            [C.c_int, P(ElemOut)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclasses.dataclass
class BSR:
    """Block compressed sparse rows: ``nb_rows`` block rows of ``br`` x ``bc``
    blocks, 0-based int32 ``row_ptr``/``col``, values block by block, each
    block row-major."""
    br: int
    bc: int
    nb_rows: int
    nb_cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnzb(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def shape(self):
        return (self.nb_rows * self.br, self.nb_cols * self.bc)

    def blocks(self) -> np.ndarray:
        return self.val.reshape(-1, self.br, self.bc)


def _bsr_from_c(b: _Bsr) -> BSR:
    nr, nnz = b.nb_rows, b.nnzb
    rp = np.ctypeslib.as_array(b.row_ptr, shape=(nr + 1,)).astype(np.int32, copy=True)
    col = np.ctypeslib.as_array(b.col, shape=(max(nnz, 1),))[:nnz].astype(np.int32, copy=True)
    val = np.ctypeslib.as_array(b.val, shape=(max(nnz * b.br * b.bc, 1),))[:nnz * b.br * b.bc].copy()
    return BSR(b.br, b.bc, nr, b.nb_cols, rp, col, val)


@dataclasses.dataclass
class Mesh:
    n_nodes: int
    n_elem: int
    n_iface: int
    n_p: int
    n_fluid: int
    xyz: np.ndarray
    ring: np.ndarray
    layer: np.ndarray
    ien: np.ndarray
    pien: np.ndarray
    etype: np.ndarray
    iface_of: np.ndarray
    fluid_id: np.ndarray
    dir_v: np.ndarray
    dir_m: np.ndarray


def _mesh_from_c(m: _Mesh) -> Mesh:
    nn, ne, nf = m.n_nodes, m.n_elem, m.n_fluid
    a = np.ctypeslib.as_array
    return Mesh(
        n_nodes=nn, n_elem=ne, n_iface=m.n_iface, n_p=m.n_p, n_fluid=nf,
        xyz=a(m.xyz, shape=(nn, 3)).copy(), ring=a(m.ring, shape=(nn,)).copy(),
        layer=a(m.layer, shape=(nn,)).copy(), ien=a(m.ien, shape=(ne, 4)).copy(),
        pien=a(m.pien, shape=(ne, 4)).copy(), etype=a(m.etype, shape=(ne,)).copy(),
        iface_of=a(m.iface_of, shape=(nn,)).copy(), fluid_id=a(m.fluid_id, shape=(nn,)).copy(),
        dir_v=a(m.dir_v, shape=(nn,)).astype(bool), dir_m=a(m.dir_m, shape=(max(nf, 1),))[:nf].astype(bool))


@dataclasses.dataclass
class BlockSystem:
    """The 2x2 block system [[A, B], [C, D]] x = b of one Newton step
    (Sec. 3.5) plus the mesh-motion system L U = g (Sec. 5.2.2).

    Vector order: all velocity nodes interleaved (x, y, z), then all
    pressures (node pressures first, then the interface duplicates).
    ``mesh_b`` is n_fluid x 3 interleaved."""
    name: str
    A: BSR
    B: BSR
    C: BSR
    D: BSR
    b: np.ndarray
    L: BSR | None
    mesh_b: np.ndarray | None
    mesh: Mesh | None
    params: dict
    # resistance outlet (optional): the momentum block's consistent tangent
    # gains alpha_f gamma dt sum_k m_k a_k a_k^T (Sec. 3.5, outlet coupling
    # matrix); a_out[k] has the 3 n_v entries int_{outlet k} N_A n_i dGamma
    # (zero on Dirichlet rows), c_out[k] = alpha_f gamma dt m_k
    a_out: list | None = None
    c_out: list | None = None

    @property
    def n_v(self) -> int:
        return self.A.nb_rows

    @property
    def n_p(self) -> int:
        return self.D.nb_rows

    @property
    def n(self) -> int:
        return 3 * self.n_v + self.n_p


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------
def default_params() -> Params:
    p = Params()
    lib().tg_default_params(C.byref(p))
    return p


def make_params(**kw) -> Params:
    p = default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


PRESETS = {
    # straight tube, 24 circ x (4 fluid + 2 wall) x 40 axial: ~6k nodes
    "tube_small": dict(n_circ=24, n_rad_f=4, n_rad_s=2, n_ax=40),
    # refined tube 96 x (11 + 5) x 400: 616,337 nodes, 2,503,844 unknowns
    "tube_large": dict(n_circ=96, n_rad_f=11, n_rad_s=5, n_ax=400),
    # stenosed tube, 50% area at mid-length, 160 x (13 + 7) x 600
    "stenosis": dict(kind=1, n_circ=160, n_rad_f=13, n_rad_s=7, n_ax=600),
    # tiny tube for dense brute force: 4 circ x (1 + 1) x 2 axial
    "tube_tiny": dict(n_circ=4, n_rad_f=1, n_rad_s=1, n_ax=2),
    # a few thousand unknowns: several GPU tiles, seconds on the CPU
    "tube_mini": dict(n_circ=12, n_rad_f=3, n_rad_s=2, n_ax=12),
    # bifurcation (kind 2): parent R = 0.5 cm, wall 0.06 cm (12% of R), 4 cm
    # parent and 4 cm daughters at +-35 degrees; n_circ = core cells per
    # side of the O-grid's square, n_rad_f lumen rings, n_rad_s wall rings;
    # the full size has 3 boundary layers (ratio 0.6) next to the lumen wall
    "bifurcation": dict(kind=2, R=0.5, wall=0.06, L=4.0, n_circ=40, n_rad_f=24, n_rad_s=5, n_ax=633,
                        bif_bl_layers=3, bif_bl_ratio=0.6),
    "bif_small": dict(kind=2, R=0.5, wall=0.06, L=4.0, n_circ=16, n_rad_f=8, n_rad_s=2, n_ax=16),
    "bif_mini": dict(kind=2, R=0.5, wall=0.06, L=4.0, n_circ=10, n_rad_f=4, n_rad_s=1, n_ax=10),
}


def genalpha(rho_inf: float):
    am, af, ga = C.c_double(), C.c_double(), C.c_double()
    lib().tg_genalpha(rho_inf, C.byref(am), C.byref(af), C.byref(ga))
    return am.value, af.value, ga.value


def build_mesh(params: Params) -> Mesh:
    L = lib()
    pm = L.tg_mesh_build(C.byref(params))
    if not pm:
        raise ValueError("no mesh: parameters out of range")
    try:
        return _mesh_from_c(pm.contents)
    finally:
        L.tg_mesh_free(pm)


def tube_system(name: str = "tube_small", threads: int = 0, keep_mesh: bool = False,
                **overrides) -> BlockSystem:
    """Build the block system of a preset (``PRESETS``) with overrides."""
    kw = dict(PRESETS[name]) if name in PRESETS else {}
    kw.update(overrides)
    r_out = float(kw.pop("outlet_resistance", 0.0))
    params = make_params(**kw)
    L = lib()
    if threads:
        L.tg_set_threads(threads)
    pm = L.tg_mesh_build(C.byref(params))
    if not pm:
        raise ValueError(f"no mesh for {name}: parameters out of range")
    try:
        m = pm.contents
        nn, np_ = m.n_nodes, m.n_p
        v = np.zeros(3 * nn)
        p = np.zeros(np_)
        L.tg_state_init(C.byref(params), pm, _dp(v), _dp(p))
        am, af, ga = genalpha(params.rho_inf)
        cf = af * ga * params.dt
        cu = cf * cf / am
        raw = L.tg_assemble(C.byref(params), pm, _dp(v), None, _dp(p), None, None,
                            am, cf, cu, 0, None, 1)
        Lraw = L.tg_mesh_laplacian_raw(pm) if not params.fluid_only else None
        sysp = L.tg_finalize(pm, raw, Lraw, C.byref(params))
        s = sysp.contents
        n = 3 * nn + np_
        out = BlockSystem(
            name=name, A=_bsr_from_c(s.A), B=_bsr_from_c(s.B), C=_bsr_from_c(s.C), D=_bsr_from_c(s.D),
            b=np.ctypeslib.as_array(s.b, shape=(n,)).copy(),
            L=_bsr_from_c(s.L) if Lraw else None,
            mesh_b=(np.ctypeslib.as_array(s.mesh_b, shape=(3 * m.n_fluid,)).copy() if Lraw else None),
            mesh=_mesh_from_c(m) if keep_mesh else None,
            params={f: getattr(params, f) for f, _ in Params._fields_})
        if r_out > 0.0:
            a = outlet_vector(_mesh_from_c(m), params.n_ax)
            # resistance outlet: pressure P = r_out Q with Q = a^T v, so the
            # momentum residual gains P a and its tangent alpha_f gamma dt
            # r_out a a^T; b = -R
            out.b[: 3 * nn] -= r_out * float(a @ v) * a
            out.a_out, out.c_out = [a], [cf * r_out]
            out.params["outlet_resistance"] = r_out
        L.tg_system_free(sysp)
        L.tg_raw_free(raw)
        if Lraw:
            L.tg_bsr_free(Lraw)
        return out
    finally:
        L.tg_mesh_free(pm)


def interface_follow(mesh: Mesh) -> np.ndarray:
    """Per fluid node: 1 where the node is a Dirichlet mesh node on the
    fluid-solid interface (its mesh displacement is the wall's), 0 on the
    other fluid nodes (inlet and outlet sections, the interior)."""
    follow = np.zeros(mesh.n_fluid, dtype=np.uint8)
    nodes = np.flatnonzero(mesh.fluid_id >= 0)
    follow[mesh.fluid_id[nodes]] = mesh.iface_of[nodes] >= 0
    return follow & mesh.dir_m.astype(np.uint8)


# --------------------------------------------------------------------------
# system files (the layout tests/c_abi_client.c reads)
# --------------------------------------------------------------------------
def save_system(s: BlockSystem, path: str) -> None:
    """Write A, B, C, D and b in native byte order: per matrix int32
    nb_rows, nb_cols, br, bc, nnzb, then int32 row_ptr[nb_rows + 1], int32
    col[nnzb], float64 val[nnzb * br * bc] (blocks row-major); then float64
    b[3 n_v + n_p].  A run can restart from the file without the generator."""
    with open(path, "wb") as f:
        for M in (s.A, s.B, s.C, s.D):
            col = np.ascontiguousarray(M.col, dtype=np.int32)
            np.array([M.nb_rows, M.nb_cols, M.br, M.bc, col.size], dtype=np.int32).tofile(f)
            np.ascontiguousarray(M.row_ptr, dtype=np.int32).tofile(f)
            col.tofile(f)
            np.ascontiguousarray(M.val, dtype=np.float64).tofile(f)
        np.ascontiguousarray(s.b, dtype=np.float64).tofile(f)


def load_system(path: str, name: str = "") -> BlockSystem:
    """Read a file of ``save_system``; the mesh system and the mesh are not
    part of it (L, mesh_b and mesh are None)."""
    with open(path, "rb") as f:
        mats = []
        for _ in range(4):
            nbr, nbc, br, bc, nnzb = (int(v) for v in np.fromfile(f, dtype=np.int32, count=5))
            rp = np.fromfile(f, dtype=np.int32, count=nbr + 1)
            col = np.fromfile(f, dtype=np.int32, count=nnzb)
            val = np.fromfile(f, dtype=np.float64, count=nnzb * br * bc)
            if rp.size != nbr + 1 or col.size != nnzb or val.size != nnzb * br * bc:
                raise ValueError(f"{path}: truncated matrix")
            mats.append(BSR(br, bc, nbr, nbc, rp, col, val))
        n = 3 * mats[0].nb_rows + mats[3].nb_rows
        b = np.fromfile(f, dtype=np.float64, count=n)
        if b.size != n or f.read(1):
            raise ValueError(f"{path}: wrong right-hand side length")
    return BlockSystem(name=name, A=mats[0], B=mats[1], C=mats[2], D=mats[3], b=b, L=None, mesh_b=None,
                       mesh=None, params={})


def rhs_only(name: str, **overrides) -> np.ndarray:
    """The right-hand side b = -[R_m; R_p] (Dirichlet velocity rows zero) of
    ``tube_system(name, **overrides)`` without assembling the matrices: the
    same state, the same generalized-alpha coefficients, the same element
    loop with the tangent switched off (for several right-hand sides on one
    Jacobian, e.g. inflow peaks)."""
    kw = dict(PRESETS[name]) if name in PRESETS else {}
    kw.update(overrides)
    params = make_params(**kw)
    L = lib()
    pm = L.tg_mesh_build(C.byref(params))
    if not pm:
        raise ValueError(f"no mesh for {name}")
    try:
        m = pm.contents
        nn, np_ = m.n_nodes, m.n_p
        v = np.zeros(3 * nn)
        p = np.zeros(np_)
        L.tg_state_init(C.byref(params), pm, _dp(v), _dp(p))
        am, af, ga = genalpha(params.rho_inf)
        cf = af * ga * params.dt
        raw = L.tg_assemble(C.byref(params), pm, _dp(v), None, _dp(p), None, None,
                            am, cf, cf * cf / am, 0, None, 0)
        r = raw.contents
        b = -np.concatenate([np.ctypeslib.as_array(r.Rm, shape=(3 * nn,)),
                             np.ctypeslib.as_array(r.Rp, shape=(np_,))])
        dv = np.ctypeslib.as_array(m.dir_v, shape=(nn,)).astype(bool)
        b[:3 * nn][np.repeat(dv, 3)] = 0.0
        L.tg_raw_free(raw)
        return b
    finally:
        L.tg_mesh_free(pm)


def outlet_vector(mesh: Mesh, n_ax: int, zero_dirichlet: bool = True) -> np.ndarray:
    """a_{A,i} = int_{outlet} N_A n_i dGamma over the fluid outlet section
    (the faces of fluid tets with all three vertices on the last axial
    layer; outward normal +z, so only the z components are nonzero); a
    linear shape function integrates to a third of the triangle's area.
    Entries on Dirichlet velocity rows are zero."""
    a = np.zeros(3 * mesh.n_nodes)
    on = mesh.layer == n_ax
    for e in np.nonzero(mesh.etype == 0)[0]:
        v = mesh.ien[e]
        for drop in range(4):
            f = [v[q] for q in range(4) if q != drop]
            if not all(on[f]):
                continue
            x = mesh.xyz[f]
            area = 0.5 * np.linalg.norm(np.cross(x[1] - x[0], x[2] - x[0]))
            for node in f:
                a[3 * node + 2] += area / 3.0
    if zero_dirichlet:
        a[np.repeat(mesh.dir_v, 3)] = 0.0
    return a


class Assembler:
    """Raw (pre-boundary-condition) residual/tangent evaluation at arbitrary
    states, for the finite-difference and steady-flow checks."""

    def __init__(self, params: Params):
        self.params = params
        self.L = lib()
        self.pm = self.L.tg_mesh_build(C.byref(params))
        if not self.pm:
            raise ValueError("no mesh: parameters out of range")
        self.mesh = _mesh_from_c(self.pm.contents)

    def close(self):
        if self.pm:
            self.L.tg_mesh_free(self.pm)
            self.pm = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def initial_state(self):
        nn, np_ = self.mesh.n_nodes, self.mesh.n_p
        v = np.zeros(3 * nn)
        p = np.zeros(np_)
        self.L.tg_state_init(C.byref(self.params), self.pm, _dp(v), _dp(p))
        return v, p

    def evaluate(self, v, p, vd=None, u=None, vhat=None, cm=0.0, cf=1.0, cu=0.0,
                 tau=None, tau_mode=0, want_mat=True):
        nn = self.mesh.n_nodes
        z = lambda a: None if a is None else _dp(np.ascontiguousarray(a, dtype=np.float64))
        keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
                for a in (v, vhat, p, vd, u)]
        ptrs = [None if a is None else _dp(a) for a in keep]
        raw = self.L.tg_assemble(C.byref(self.params), self.pm, ptrs[0], ptrs[1], ptrs[2],
                                 ptrs[3], ptrs[4], cm, cf, cu, tau_mode,
                                 _dp(tau) if tau is not None else None, int(want_mat))
        r = raw.contents
        out = dict(Rm=np.ctypeslib.as_array(r.Rm, shape=(3 * nn,)).copy(),
                   Rp=np.ctypeslib.as_array(r.Rp, shape=(self.mesh.n_p,)).copy())
        if want_mat:
            out.update(A=_bsr_from_c(r.A), B=_bsr_from_c(r.B), C=_bsr_from_c(r.C), D=_bsr_from_c(r.D))
        self.L.tg_raw_free(raw)
        del z
        return out

    def mesh_laplacian(self) -> BSR:
        b = self.L.tg_mesh_laplacian_raw(self.pm)
        out = _bsr_from_c(b.contents)
        self.L.tg_bsr_free(b)
        return out


def fluid_element(x, v, p, vd=None, vhat=None, rho=1.06, mu=0.04, dt=1e-4, cm=1.0, cf=1.0,
                  tau=None, tau_mode=0, want_mat=True):
    """Evaluate one fluid element (tests): returns the element arrays."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(4, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(4, 3)
    vd = np.zeros((4, 3)) if vd is None else np.ascontiguousarray(vd, dtype=np.float64).reshape(4, 3)
    vh = np.zeros((4, 3)) if vhat is None else np.ascontiguousarray(vhat, dtype=np.float64).reshape(4, 3)
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(4)
    t = np.zeros(8) if tau is None else np.ascontiguousarray(tau, dtype=np.float64)
    out = ElemOut()
    lib().tg_fluid_element(_dp(x), _dp(v), _dp(vh), _dp(p), _dp(vd), rho, mu, dt, cm, cf,
                           tau_mode, _dp(t), int(want_mat), C.byref(out))
    res = out.arrays()
    res["tau"] = t
    return res


def solid_element(x, u, v, p, vd, rho, mu_s, tauM, tauC, cm, cf, cu, want_mat=True):
    arr = [np.ascontiguousarray(a, dtype=np.float64).reshape(4, 3) for a in (x, u, v)]
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(4)
    vd = np.ascontiguousarray(vd, dtype=np.float64).reshape(4, 3)
    out = ElemOut()
    lib().tg_solid_element(_dp(arr[0]), _dp(arr[1]), _dp(arr[2]), _dp(p), _dp(vd), rho, mu_s,
                           tauM, tauC, cm, cf, cu, int(want_mat), C.byref(out))
    return out.arrays()


def metric_G(dxi) -> np.ndarray:
    d = np.ascontiguousarray(dxi, dtype=np.float64).reshape(3, 3)
    G = np.zeros((3, 3))
    lib().tg_metric(_dp(d), _dp(G))
    return G


def tau_fluid(G, u, rho, mu, dt):
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(3, 3)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(3)
    tm, tc = C.c_double(), C.c_double()
    lib().tg_tau_fluid(_dp(G), _dp(u), rho, mu, dt, C.byref(tm), C.byref(tc))
    return tm.value, tc.value


def circum_diameter(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(4, 3)
    return lib().tg_circum_diameter(_dp(x))


def gauss_points() -> np.ndarray:
    N = np.zeros((4, 4))
    lib().tg_gauss_points(_dp(N))
    return N


def batch_member_params(i: int, seed: int = 2206) -> dict:
    """Member i of the batched workload: radius U(0.15, 0.5), wall
    U(0.10, 0.20) R, node target log-uniform in [5k, 80k], 6 radial rings
    (4 lumen + 2 wall), n_circ = 4 * 6, odd members stenosed.  Draws come
    from splitmix64 seeded with seed + i (same generator as the C side)."""
    st = [(seed + i) & 0xFFFFFFFFFFFFFFFF]

    def nxt():
        st[0] = (st[0] + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = st[0]
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return (z ^ (z >> 31)) & 0xFFFFFFFFFFFFFFFF

    u = lambda: (nxt() >> 11) * (1.0 / 9007199254740992.0)
    R = 0.15 + 0.35 * u()
    wall = (0.10 + 0.10 * u()) * R
    target = math.exp(math.log(5e3) + (math.log(8e4) - math.log(5e3)) * u())
    n_rad = 6
    n_circ = 4 * n_rad
    n_sec = 1 + n_circ * n_rad
    n_ax = max(4, int(round(target / n_sec)) - 1)
    return dict(kind=i % 2, R=R, wall=wall, n_circ=n_circ, n_rad_f=4, n_rad_s=2, n_ax=n_ax,
                sten_sigma=2.0 * R, seed=seed + i)
