"""Python face of the C ABI: argument marshalling only."""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from .abi import (BsrOut, Bsr, KProf, Mesh, Opts, Physics, SCR_NOT_CONVERGED, SCR_OK, Stats,
                  check, load_library)


def _torch():
    import torch
    return torch


@dataclasses.dataclass
class DeviceBSR:
    """Block CSR with its arrays in device memory (torch CUDA tensors)."""
    br: int
    bc: int
    nb_rows: int
    nb_cols: int
    row_ptr: object  # torch.int32
    col: object      # torch.int32
    val: object      # torch.float64

    @classmethod
    def pinned(cls, M):
        """Host copy in page-locked memory (fast host-to-device copies)."""
        torch = _torch()
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).pin_memory()
        return cls(M.br, M.bc, M.nb_rows, M.nb_cols, t(M.row_ptr, np.int32), t(M.col, np.int32),
                   t(M.val, np.float64))

    def nbytes(self) -> int:
        return sum(int(a.numel() * a.element_size()) for a in (self.row_ptr, self.col, self.val))

    @classmethod
    def from_host(cls, M, device="cuda"):
        torch = _torch()
        return cls(M.br, M.bc, M.nb_rows, M.nb_cols,
                   torch.as_tensor(np.ascontiguousarray(M.row_ptr, dtype=np.int32), device=device),
                   torch.as_tensor(np.ascontiguousarray(M.col, dtype=np.int32), device=device),
                   torch.as_tensor(np.ascontiguousarray(M.val, dtype=np.float64), device=device))

    @property
    def nnzb(self) -> int:
        return int(self.col.numel())


def _as_bsr(M, keep: list) -> tuple[Bsr, int]:
    """(C struct, ptr_is_device) for a host (numpy), pinned-host or device
    (torch) matrix."""
    if isinstance(M, DeviceBSR):
        s = Bsr(M.nb_rows, M.nb_cols, M.br, M.bc, M.nnzb, M.row_ptr.data_ptr(), M.col.data_ptr(),
                M.val.data_ptr())
        keep.append(M)
        return s, int(M.row_ptr.is_cuda)
    rp = np.ascontiguousarray(M.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(M.col, dtype=np.int32)
    val = np.ascontiguousarray(M.val, dtype=np.float64)
    keep.extend([rp, col, val])
    s = Bsr(M.nb_rows, M.nb_cols, M.br, M.bc, int(col.size), rp.ctypes.data, col.ctypes.data, val.ctypes.data)
    return s, 0


def _ptr(x, keep: list) -> tuple[int, int]:
    """(address, ptr_is_device) of a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(x)
        return x.ctypes.data, 0
    torch = _torch()
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("vectors must be contiguous float64 tensors")
        keep.append(x)
        return x.data_ptr(), int(x.is_cuda)
    raise TypeError(f"unsupported vector type {type(x)}")


class BlockSolver:
    """One solver context (scr_handle) on the current CUDA device."""

    def __init__(self, stream=None, **opts):
        self.lib = load_library()
        o = Opts()
        self.lib.scr_default_opts(C.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise KeyError(f"unknown option {k}")
            setattr(o, k, v)
        self.opts = o
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = C.c_void_p()
        check(self.lib.scr_create(C.byref(h), C.byref(o), C.c_void_p(stream)))
        self.h = h
        self.n_v = self.n_p = self.n_m = 0
        self.n_fluid = 0  # fluid nodes of the mesh coupling (mesh_coupling)

    # -------------------------------------------------------------- life
    def close(self):
        if getattr(self, "h", None):
            self.lib.scr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- block system
    def setup(self, A, B, Cm, D):
        keep: list = []
        sa, da = _as_bsr(A, keep)
        sb, db = _as_bsr(B, keep)
        sc, dc = _as_bsr(Cm, keep)
        sd, dd = _as_bsr(D, keep)
        if len({da, db, dc, dd}) != 1:
            raise ValueError("A, B, C, D must all be on the host or all on the device")
        check(self.lib.scr_setup(self.h, C.byref(sa), C.byref(sb), C.byref(sc), C.byref(sd), da))
        self.n_v, self.n_p = A.nb_rows, D.nb_rows
        return self

    def update_values(self, A, B, Cm, D):
        """New values for the set-up's block system (same patterns):
        scr_update_values, the numeric re-set-up."""
        keep: list = []
        sa, da = _as_bsr(A, keep)
        sb, db = _as_bsr(B, keep)
        sc, dc = _as_bsr(Cm, keep)
        sd, dd = _as_bsr(D, keep)
        if len({da, db, dc, dd}) != 1:
            raise ValueError("A, B, C, D must all be on the host or all on the device")
        check(self.lib.scr_update_values(self.h, C.byref(sa), C.byref(sb), C.byref(sc), C.byref(sd), da))
        return self

    def solve(self, b, x=None, raise_on_nonconvergence: bool = True):
        """x with calA x = b.  numpy in -> numpy out (host pointers);
        CUDA tensor in -> CUDA tensor out (device pointers)."""
        n = 3 * self.n_v + self.n_p
        keep: list = []
        pb, dev = _ptr(b, keep)
        if x is None:
            if dev:
                x = _torch().empty(n, dtype=_torch().float64, device=b.device)
            else:
                x = np.empty(n)
        px, dx = _ptr(x, keep)
        if dx != dev:
            raise ValueError("b and x must both be host or both device")
        st = self.lib.scr_solve(self.h, C.c_void_p(pb), C.c_void_p(px), dev)
        check(st, (SCR_OK,) if raise_on_nonconvergence else (SCR_OK, SCR_NOT_CONVERGED))
        return x

    def iters(self):
        o, i = C.c_int(), C.c_int()
        check(self.lib.scr_iters(self.h, C.byref(o), C.byref(i)))
        return o.value, i.value

    def residual(self) -> float:
        r = C.c_double()
        check(self.lib.scr_residual(self.h, C.byref(r)))
        return r.value

    def stats(self) -> dict:
        s = Stats()
        check(self.lib.scr_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    # -------------------------------------------------------------- batched form
    def setup_batch(self, systems):
        """systems: list of (A, B, C, D), all host (numpy) or all device."""
        keep: list = []
        nb = len(systems)
        arrs = [(Bsr * nb)() for _ in range(4)]
        devs = set()
        for i, sysm in enumerate(systems):
            for j in range(4):
                st, d = _as_bsr(sysm[j], keep)
                arrs[j][i] = st
                devs.add(d)
        if len(devs) != 1:
            raise ValueError("all members must be on the host or all on the device")
        check(self.lib.scr_setup_batch(self.h, nb, arrs[0], arrs[1], arrs[2], arrs[3], devs.pop()))
        self.batch_sizes = [(sysm[0].nb_rows, sysm[3].nb_rows) for sysm in systems]
        return self

    def solve_batch(self, bs, xs=None, raise_on_nonconvergence: bool = True):
        nb = len(bs)
        keep: list = []
        if xs is None:
            xs = [np.empty_like(np.asarray(b, dtype=np.float64)) if isinstance(b, np.ndarray)
                  else _torch().empty_like(b) for b in bs]
        pb = (C.c_void_p * nb)()
        px = (C.c_void_p * nb)()
        devs = set()
        for i in range(nb):
            a, d = _ptr(bs[i], keep)
            c, e = _ptr(xs[i], keep)
            pb[i], px[i] = a, c
            devs.update((d, e))
        if len(devs) != 1:
            raise ValueError("vectors must all be host or all device")
        st = self.lib.scr_solve_batch(self.h, pb, px, devs.pop())
        check(st, (SCR_OK,) if raise_on_nonconvergence else (SCR_OK, SCR_NOT_CONVERGED))
        return xs

    def assembly_setup(self, mesh, params: dict):
        """Upload a mesh (arrays xyz, ien, pien, etype, dir_v, sizes
        n_nodes, n_elem, n_p) and the physical parameters for scr_residual."""
        keep = [np.ascontiguousarray(mesh.xyz, dtype=np.float64), np.ascontiguousarray(mesh.ien, dtype=np.int32),
                np.ascontiguousarray(mesh.pien, dtype=np.int32), np.ascontiguousarray(mesh.etype, dtype=np.uint8),
                np.ascontiguousarray(mesh.dir_v, dtype=np.uint8)]
        m = Mesh(mesh.n_nodes, mesh.n_elem, mesh.n_p, *(k.ctypes.data_as(C.c_void_p) for k in keep))
        ph = Physics(*(float(params[f]) for f, _ in Physics._fields_))
        check(self.lib.scr_assembly_setup(self.h, C.byref(m), C.byref(ph)))
        self._res_sizes = (mesh.n_nodes, mesh.n_p)

    def assemble_residual(self, v, p, vhat=None, vdot=None, u=None):
        """R = [R_m | R_p] at the state (numpy in -> numpy out, CUDA tensors
        in -> CUDA tensor out)."""
        nn, np_ = self._res_sizes
        keep: list = []
        pv, dev = _ptr(v, keep)
        pp, _ = _ptr(p, keep)
        opt = [(_ptr(a, keep)[0] if a is not None else None) for a in (vhat, vdot, u)]
        if dev:
            R = _torch().empty(3 * nn + np_, dtype=_torch().float64, device=v.device)
        else:
            R = np.empty(3 * nn + np_)
        pr, _ = _ptr(R, keep)
        vp = lambda a: None if a is None else C.c_void_p(a)
        check(self.lib.scr_assemble_residual(self.h, vp(pv), vp(opt[0]), vp(pp), vp(opt[1]), vp(opt[2]), vp(pr), dev))
        return R

    def assemble_tangent(self, v, p, vhat=None, vdot=None):
        """Assemble the tangent blocks A, B, C, D on the GPU at the state and
        set the block solve up on them (scr_assemble_tangent); numpy arrays or
        CUDA tensors."""
        keep: list = []
        pv, dev = _ptr(v, keep)
        pp, _ = _ptr(p, keep)
        opt = [(_ptr(a, keep)[0] if a is not None else None) for a in (vhat, vdot)]
        vp = lambda a: None if a is None else C.c_void_p(a)
        check(self.lib.scr_assemble_tangent(self.h, vp(pv), vp(opt[0]), vp(pp), vp(opt[1]), dev))

    def corrector(self, v, p, vdot, u, n_iter: int):
        """n_iter multi-corrector iterations on the state (updated in place:
        numpy arrays or CUDA tensors); returns the residual norms."""
        keep: list = []
        ptrs = [_ptr(a, keep) for a in (v, p, vdot, u)]
        devs = {d for _, d in ptrs}
        if len(devs) != 1:
            raise ValueError("state vectors must all be host or all device")
        if not devs.pop() and any(k is not a for k, a in zip(keep, (v, p, vdot, u))):
            raise TypeError("host state vectors must be contiguous float64 arrays (updated in place)")
        norms = np.zeros(n_iter + 1)
        st = self.lib.scr_corrector(self.h, *(C.c_void_p(q) for q, _ in ptrs), int(n_iter),
                                    norms.ctypes.data_as(C.c_void_p), ptrs[0][1])
        check(st, (SCR_OK, SCR_NOT_CONVERGED))
        return norms

    def mesh_coupling(self, L_raw, fluid_id, dir_m, follow):
        """Mesh motion for ``corrector_ale``: the fluid nodes' mesh Laplacian
        without boundary conditions (host BSR), the node -> fluid ordinal
        map (-1 off the fluid), the Dirichlet mesh flags and the flags of
        the Dirichlet nodes that follow the solid displacement."""
        keep: list = []
        sl, dl = _as_bsr(L_raw, keep)
        if dl:
            raise TypeError("L_raw must be a host matrix")
        fid = np.ascontiguousarray(fluid_id, dtype=np.int32)
        dm = np.ascontiguousarray(dir_m, dtype=np.uint8)
        fo = np.ascontiguousarray(follow, dtype=np.uint8)
        nf = int(L_raw.nb_rows)
        if dm.size != nf or fo.size != nf:
            raise ValueError("dir_m and follow need one flag per fluid node")
        check(self.lib.scr_mesh_coupling(self.h, nf, fid.ctypes.data_as(C.c_void_p), dm.ctypes.data_as(C.c_void_p),
                                         fo.ctypes.data_as(C.c_void_p), C.byref(sl)))
        self.n_fluid = nf

    def corrector_ale(self, v, p, vdot, u, uhat_n, n_iter: int, vhat_n=None):
        """``corrector`` with the mesh moving inside the loop; the state
        (entering at the same-Y predictor) is updated in place.  Returns
        (residual norms, uhat_{n+1})."""
        keep: list = []
        ptrs = [_ptr(a, keep) for a in (v, p, vdot, u)]
        devs = {d for _, d in ptrs}
        if len(devs) != 1:
            raise ValueError("state vectors must all be host or all device")
        dev = devs.pop()
        if not dev and any(k is not a for k, a in zip(keep, (v, p, vdot, u))):
            raise TypeError("host state vectors must be contiguous float64 arrays (updated in place)")
        n3 = 3 * self.n_fluid
        if dev:
            uhat = _torch().empty(n3, dtype=_torch().float64, device=v.device)
        else:
            uhat = np.empty(n3)
        extra = [_ptr(a, keep) for a in (uhat_n, uhat)]
        pvn = None
        if vhat_n is not None:
            pvn, dvn = _ptr(vhat_n, keep)
            extra.append((pvn, dvn))
        if any(d != dev for _, d in extra):
            raise ValueError("uhat_n and vhat_n must live where the state does")
        norms = np.zeros(n_iter + 1)
        st = self.lib.scr_corrector_ale(self.h, *(C.c_void_p(q) for q, _ in ptrs), C.c_void_p(extra[0][0]),
                                        None if pvn is None else C.c_void_p(pvn), C.c_void_p(extra[1][0]),
                                        int(n_iter), norms.ctypes.data_as(C.c_void_p), dev)
        check(st, (SCR_OK, SCR_NOT_CONVERGED))
        return norms, uhat

    def set_outlets(self, a_out, c_out):
        """Rank-1 outlet terms for the next setup: vectors a_j (3 n_v each)
        and coefficients c_j; empty lists remove them."""
        a_out = [np.ascontiguousarray(a, dtype=np.float64) for a in (a_out or [])]
        c = np.ascontiguousarray(c_out or [], dtype=np.float64)
        n = len(a_out)
        if n != c.size:
            raise ValueError("one coefficient per outlet vector")
        a = np.concatenate(a_out) if n else np.zeros(1)
        ln = a_out[0].size if n else 0
        check(self.lib.scr_set_outlets(self.h, n, ln, a.ctypes.data_as(C.c_void_p), c.ctypes.data_as(C.c_void_p)))

    def solve_multi(self, bs, xs=None, raise_on_nonconvergence: bool = True):
        """x_c with calA x_c = b_c for the opts.nrhs right-hand sides bs (all
        numpy or all CUDA tensors); returns (xs, per-column FP64 relative
        residuals)."""
        k = self.opts.nrhs
        if len(bs) != k:
            raise ValueError(f"the handle solves {k} right-hand sides at once")
        keep: list = []
        if xs is None:
            xs = [np.empty_like(np.asarray(b, dtype=np.float64)) if isinstance(b, np.ndarray)
                  else _torch().empty_like(b) for b in bs]
        pb = (C.c_void_p * k)()
        px = (C.c_void_p * k)()
        devs = set()
        for i in range(k):
            a, d = _ptr(bs[i], keep)
            c, e = _ptr(xs[i], keep)
            pb[i], px[i] = a, c
            devs.update((d, e))
        if len(devs) != 1:
            raise ValueError("vectors must all be host or all device")
        rel = np.zeros(k)
        st = self.lib.scr_solve_multi(self.h, pb, px, devs.pop(), rel.ctypes.data_as(C.c_void_p))
        check(st, (SCR_OK,) if raise_on_nonconvergence else (SCR_OK, SCR_NOT_CONVERGED))
        return xs, rel

    def batch_residuals(self):
        n = len(self.batch_sizes)
        r = (C.c_double * n)()
        check(self.lib.scr_batch_residuals(self.h, r))
        return np.array(r[:])

    # -------------------------------------------------------------- mesh
    def mesh_setup(self, L):
        keep: list = []
        sl, dl = _as_bsr(L, keep)
        check(self.lib.mm_setup(self.h, C.byref(sl), dl))
        self.n_m = L.nb_rows
        return self

    def mesh_solve(self, g, u=None, raise_on_nonconvergence: bool = True):
        n = 3 * self.n_m
        keep: list = []
        pg, dev = _ptr(g, keep)
        if u is None:
            u = _torch().empty(n, dtype=_torch().float64, device=g.device) if dev else np.empty(n)
        pu, du = _ptr(u, keep)
        st = self.lib.mm_solve(self.h, C.c_void_p(pg), C.c_void_p(pu), dev)
        check(st, (SCR_OK,) if raise_on_nonconvergence else (SCR_OK, SCR_NOT_CONVERGED))
        return u

    def mesh_iters(self):
        i, r = C.c_int(), C.c_double()
        check(self.lib.mm_iters(self.h, C.byref(i), C.byref(r)))
        return i.value, r.value

    # -------------------------------------------------------------- single steps
    def _dev2(self, fn, x, n_out):
        torch = _torch()
        y = torch.empty(n_out, dtype=torch.float64, device=x.device)
        check(fn(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def profile_begin(self, kernel_class: int = 0, capacity: int = 20000):
        check(self.lib.scr_profile_begin(self.h, kernel_class, capacity))

    def profile_end(self) -> dict:
        p = KProf()
        check(self.lib.scr_profile_end(self.h, C.byref(p)))
        return {f: getattr(p, f) for f, _ in KProf._fields_}

    def apply_op(self, x):
        return self._dev2(self.lib.scr_apply_op, x, 3 * self.n_v + self.n_p)

    def apply_pc(self, r):
        return self._dev2(self.lib.scr_apply_pc, r, 3 * self.n_v + self.n_p)

    def apply_schur(self, xp):
        return self._dev2(self.lib.scr_apply_schur, xp, self.n_p)

    def amg_apply(self, which: int, b):
        torch = _torch()
        x = torch.empty_like(b)
        check(self.lib.scr_amg_apply(self.h, which, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr())))
        return x

    def amg_levels(self, which: int) -> int:
        n = C.c_int()
        check(self.lib.scr_amg_levels(self.h, which, C.byref(n)))
        return n.value

    def export(self, which: int, level: int, kind: int):
        """Copy a hierarchy operator / prolongator (block CSR, numpy), the
        aggregates or the aggregates' roots (int arrays) to the host."""
        from .abi import SCR_EXPORT_AGGREGATES, SCR_EXPORT_ROOTS  # noqa: F401
        o = BsrOut()
        check(self.lib.scr_export(self.h, which, level, kind, C.byref(o)))
        if kind in (SCR_EXPORT_AGGREGATES, SCR_EXPORT_ROOTS):
            agg = np.empty(max(o.nb_rows, 1), dtype=np.int32)
            o2 = BsrOut()
            o2.col_idx = agg.ctypes.data
            check(self.lib.scr_export(self.h, which, level, kind, C.byref(o2)))
            return agg[: o.nb_rows] if o.nnzb else None
        rp = np.empty(o.nb_rows + 1, dtype=np.int32)
        col = np.empty(max(o.nnzb, 1), dtype=np.int32)
        val = np.empty(max(o.nnzb * o.br * o.bc, 1))
        o2 = BsrOut()
        o2.row_ptr, o2.col_idx, o2.val = rp.ctypes.data, col.ctypes.data, val.ctypes.data
        check(self.lib.scr_export(self.h, which, level, kind, C.byref(o2)))
        from types import SimpleNamespace
        return SimpleNamespace(br=o.br, bc=o.bc, nb_rows=o.nb_rows, nb_cols=o.nb_cols, row_ptr=rp,
                               col=col[: o.nnzb], val=val[: o.nnzb * o.br * o.bc])


def bsr_spmv(M: DeviceBSR, x, y=None, stream=None):
    """y = M x for a device block matrix, through scr_bsr_spmv."""
    torch = _torch()
    lib = load_library()
    if y is None:
        y = torch.empty(M.nb_rows * M.br, dtype=torch.float64, device=x.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    s = Bsr(M.nb_rows, M.nb_cols, M.br, M.bc, M.nnzb, M.row_ptr.data_ptr(), M.col.data_ptr(), M.val.data_ptr())
    check(lib.scr_bsr_spmv(C.byref(s), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), C.c_void_p(stream)))
    return y


def bsr_spmv_noalloc(M: DeviceBSR, x, y, stream=None):
    """y = M x through scr_bsr_spmv_noalloc (no device allocation inside the
    call; y must be preallocated)."""
    torch = _torch()
    lib = load_library()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    s = Bsr(M.nb_rows, M.nb_cols, M.br, M.bc, M.nnzb, M.row_ptr.data_ptr(), M.col.data_ptr(), M.val.data_ptr())
    check(lib.scr_bsr_spmv_noalloc(C.byref(s), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                   C.c_void_p(stream)))
    return y


def tune_save(path: str) -> None:
    """Write the autotuner's cached kernel choices to a text file."""
    check(load_library().scr_tune_save(os.fsencode(path)))


def tune_load(path: str) -> None:
    """Add the kernel choices of a file written by tune_save to the cache."""
    check(load_library().scr_tune_load(os.fsencode(path)))
