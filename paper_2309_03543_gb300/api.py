"""Thin Python binding of libcps.so (argument marshalling only).

Tensors are torch tensors; device tensors are passed straight through as
device pointers on the current torch stream.  Host (CPU) tensors are copied to
the device first and results copied back, so the same calls serve callers
that hold their data in host memory.  Every step of the computation runs in
the CUDA library; nothing here computes.
"""
from __future__ import annotations

import ctypes
import weakref
from dataclasses import dataclass

import torch

from . import _cps

P = ctypes.c_void_p


class CpsError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_cps.ERROR_NAMES.get(code, code)}: {message}")
        self.code = code


@dataclass
class SolveStats:
    iters: int
    rel_res: float
    status: int
    refinements: int
    launches: int


def _stats(s: _cps.Stats) -> SolveStats:
    return SolveStats(int(s.iters), float(s.rel_res), int(s.status), int(s.refinements),
                      int(s.launches))


def _stream(device: torch.device) -> P:
    return P(torch.cuda.current_stream(device).cuda_stream)


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device: int | torch.device = 0):
        self.lib = _cps.load()
        self.device = torch.device("cuda", device if isinstance(device, int) else device.index or 0)
        h = P()
        rc = self.lib.cps_create(ctypes.byref(h), self.device.index)
        if rc != _cps.OK:
            raise CpsError(rc, "cps_create failed")
        self.handle = h
        self._systems = weakref.WeakSet()

    def last_error(self) -> str:
        m = self.lib.cps_last_error(self.handle)
        return m.decode() if m else ""

    def check(self, rc: int, what: str):
        if rc != _cps.OK:
            raise CpsError(rc, f"{what}: {self.last_error()}")

    def dev(self, t, dtype) -> torch.Tensor:
        """The tensor on this device, contiguous, of dtype (copied if needed)."""
        t = torch.as_tensor(t)
        return t.to(device=self.device, dtype=dtype).contiguous()

    def set_batch_path(self, path: int):
        """BATCH_ONE_LAUNCH (default) or BATCH_GRAPH: how solve_batch runs FP64
        ensembles on this context."""
        self.check(self.lib.cps_set_batch_path(self.handle, path), "cps_set_batch_path")

    def close(self):
        if getattr(self, "handle", None):
            for s in list(self._systems):
                s.handle = None          # freed by cps_destroy with the context
            self.lib.cps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ assembly
    def assemble(self, xy, tri, dirichlet, eps, kinv, field_loc: int = _cps.PER_VERTEX,
                 kind: int = _cps.KIND_CP2, nu: float = 1.5e-5, dt: float = 0.225) -> "System":
        xy_d = self.dev(xy, torch.float64)
        tri_d = self.dev(tri, torch.int32)
        dir_d = self.dev(dirichlet, torch.int32)
        eps_d = self.dev(eps, torch.float64)
        kinv_d = self.dev(kinv, torch.float64)
        nv = xy_d.numel() // 2
        nt = tri_d.numel() // 3
        h = P()
        rc = self.lib.cps_assemble(self.handle, P(xy_d.data_ptr()), nv, P(tri_d.data_ptr()), nt,
                                   P(dir_d.data_ptr()) if dir_d.numel() else None, dir_d.numel(),
                                   P(eps_d.data_ptr()), P(kinv_d.data_ptr()), field_loc, kind,
                                   nu, dt, ctypes.byref(h), _stream(self.device))
        self.check(rc, "cps_assemble")
        s = System(self, h, nt)
        self._systems.add(s)
        return s


class System:
    """One assembled corrector system (matrix, preconditioner, workspace)."""

    def __init__(self, ctx: Context, handle: P, nt: int):
        self.ctx = ctx
        self.handle = handle
        self.nt = nt

    def free(self):
        if self.handle and self.ctx.handle:
            self.ctx.lib.cps_sys_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        nt, ne, sl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        dmin, mm = ctypes.c_double(), ctypes.c_int()
        self.ctx.check(self.ctx.lib.cps_sys_info(self.handle, ctypes.byref(nt), ctypes.byref(ne),
                                                 ctypes.byref(dmin), ctypes.byref(mm),
                                                 ctypes.byref(sl)),
                       "cps_sys_info")
        return {"nt": nt.value, "n_interior_sides": ne.value, "diag_min": dmin.value,
                "is_mmatrix": bool(mm.value), "setup_launches": sl.value}

    def tuning(self, precision: int = _cps.FP64) -> dict:
        """Autotuned (unroll, grid) of the iteration kernels for a precision,
        and which way of running the loop the tuner chose (with the measured
        microseconds per iteration of each candidate; 0 where not tried)."""
        u = (ctypes.c_int32 * 3)()
        g = (ctypes.c_int32 * 3)()
        bl = (ctypes.c_int32 * 3)()
        f = (ctypes.c_int32 * 8)()
        pr = (ctypes.c_double * 18)()
        self.ctx.check(self.ctx.lib.cps_get_tuning(self.handle, precision, u, g, bl, f, pr),
                       "cps_get_tuning")
        gu, gg, gb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self.ctx.check(self.ctx.lib.cps_get_gear_shape(self.handle, ctypes.byref(gu),
                                                      ctypes.byref(gg), ctypes.byref(gb)),
                       "cps_get_gear_shape")
        return {"unroll": list(u), "grid": list(g), "block": list(bl),
                "cluster": bool(f[0]),
                "cluster_recurrence": (None, "textbook", "single_reduction", "pipelined", "s_step2",
                                       "s_step3")[f[0]],
                "l2_window": ("none", "matrix", "vectors", "vectors5")[f[1]],
                "persistent": bool(f[2]), "reduced_persistent": bool(f[3]),
                "reduced_single_reduction": f[3] == 2,
                "reduced_l2_window": ("none", "matrix", "vectors", "vectors5")[f[4]],
                "stream_single_reduction": bool(f[5]),
                "persistent_single_reduction": bool(f[6]),
                "ic0_persistent": bool(f[7]),
                "ic0_l2_window": ("none", "none", "vectors5", "vectors6")[f[7]],
                "update_1red": [gu.value, gg.value, gb.value],
                "probe_us_per_iter": {
                    "stream": pr[0], "cluster": pr[1], "stream_l2_matrix": pr[2],
                    "persistent": pr[3], "stream_l2_vectors": pr[4], "persistent_l2_vectors": pr[5],
                    "reduced_stream": pr[6], "reduced_persistent": pr[7],
                    "reduced_stream_l2_vectors": pr[8], "reduced_persistent_l2_vectors": pr[9],
                    "stream_1red": pr[10], "stream_1red_l2_vectors": pr[11],
                    "persistent_1red": pr[12], "persistent_1red_l2_vectors": pr[13],
                    "ic0_stream": pr[14], "ic0_persistent": pr[15],
                    "reduced_persistent_1red": pr[16],
                    "reduced_persistent_1red_l2_vectors": pr[17]}}

    def set_solver_path(self, path: int):
        """PATH_AUTO, PATH_STREAM, PATH_CLUSTER, PATH_CLUSTER_1RED, PATH_CLUSTER_PIPE,
        PATH_CLUSTER_SSTEP2, PATH_CLUSTER_SSTEP3, PATH_PERSISTENT, PATH_STREAM_L2, PATH_PERSISTENT_L2, PATH_STREAM_1RED,
        PATH_STREAM_1RED_L2, PATH_PERSISTENT_1RED or PATH_PERSISTENT_1RED_L2 for
        FP64 Jacobi (and reduced-system) solves."""
        self.ctx.check(self.ctx.lib.cps_set_solver_path(self.handle, path), "cps_set_solver_path")

    def set_kernel_shapes(self, precision: int, unroll, grid, block):
        """Pin (unroll, grid, block) of the iteration kernels of a precision
        (3 entries each) instead of autotuning them."""
        arr = lambda v: (ctypes.c_int32 * 3)(*[int(t) for t in v])
        self.ctx.check(self.ctx.lib.cps_set_kernel_shapes(self.handle, precision, arr(unroll),
                                                          arr(grid), arr(block)),
                       "cps_set_kernel_shapes")

    def set_precond(self, precond: int):
        self.ctx.check(self.ctx.lib.cps_set_precond(self.handle, precond,
                                                    _stream(self.ctx.device)), "cps_set_precond")

    def export_matrix(self):
        """(diag [nt], col [3, nt], val [3, nt]) on the device."""
        d = torch.empty(self.nt, dtype=torch.float64, device=self.ctx.device)
        c = torch.empty(3 * self.nt, dtype=torch.int32, device=self.ctx.device)
        v = torch.empty(3 * self.nt, dtype=torch.float64, device=self.ctx.device)
        self.ctx.check(self.ctx.lib.cps_export_matrix(self.handle, P(d.data_ptr()), P(c.data_ptr()),
                                                      P(v.data_ptr()), _stream(self.ctx.device)),
                       "cps_export_matrix")
        return d, c.view(3, self.nt), v.view(3, self.nt)

    def matvec(self, x) -> torch.Tensor:
        xd = self.ctx.dev(x, torch.float64)
        y = torch.empty_like(xd)
        self.ctx.check(self.ctx.lib.cps_matvec(self.handle, P(xd.data_ptr()), P(y.data_ptr()),
                                               _stream(self.ctx.device)), "cps_matvec")
        return y

    def solve(self, b, x=None, rtol: float = 1e-10, max_iter: int = 1_000_000,
              precision: int = _cps.FP64, check: bool = True):
        """Solve A x = b.  x (if given, a device tensor) is the initial guess
        and is overwritten in place.  Host inputs are copied in and the result
        copied back to the host.  Returns (x, SolveStats)."""
        host = not (isinstance(b, torch.Tensor) and b.is_cuda)
        bd = self.ctx.dev(b, torch.float64)
        if x is None:
            xd = torch.zeros_like(bd)
        elif isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 \
                and x.is_contiguous():
            xd = x
        else:
            xd = self.ctx.dev(x, torch.float64)
        st = _cps.Stats()
        rc = self.ctx.lib.cps_solve(self.handle, P(bd.data_ptr()), P(xd.data_ptr()), rtol,
                                    max_iter, precision, ctypes.byref(st),
                                    _stream(self.ctx.device))
        if check:
            self.ctx.check(rc, "cps_solve")
        out = xd.cpu() if host else xd
        return out, _stats(st)

    def cp2_setup(self, xy, tri, eps, kinv):
        """Prepare the CP2 step on this (CP2) system from the mesh and fields it
        was assembled from (kinv holds theta for log-permeability systems)."""
        d = self.ctx.dev
        xy_d, tri_d = d(xy, torch.float64), d(tri, torch.int32)
        eps_d, kinv_d = d(eps, torch.float64), d(kinv, torch.float64)
        rc = self.ctx.lib.cps_cp2_setup(self.handle, P(xy_d.data_ptr()), P(tri_d.data_ptr()),
                                        P(eps_d.data_ptr()), P(kinv_d.data_ptr()),
                                        _stream(self.ctx.device))
        self.ctx.check(rc, "cps_cp2_setup")

    def cp2_step(self, u23, g_k, rtol: float = 1e-10, max_iter: int = 1_000_000,
                 precision: int = _cps.FP64, check: bool = True) -> dict:
        """One CP2 step (Sec. 3.2.3) from the cell velocity u23 [2, nt] and the
        cell field g_k = eps grad(Psi^k) [2, nt].  Returns device tensors
        eta_tilde, eta [nt], u_next, g_next [2, nt], flux [3, nt] (outward
        side fluxes of u_next) and the stats of the two solves."""
        u = self.ctx.dev(u23, torch.float64).reshape(2, self.nt)
        g = self.ctx.dev(g_k, torch.float64).reshape(2, self.nt)
        z = lambda *shape: torch.empty(*shape, dtype=torch.float64, device=self.ctx.device)
        out = {"eta_tilde": z(self.nt), "eta": z(self.nt), "u_next": z(2, self.nt),
               "g_next": z(2, self.nt), "flux": z(3, self.nt)}
        st = (_cps.Stats * 2)()
        rc = self.ctx.lib.cps_cp2_step(self.handle, P(u.data_ptr()), P(g.data_ptr()),
                                       P(out["eta_tilde"].data_ptr()), P(out["eta"].data_ptr()),
                                       P(out["u_next"].data_ptr()), P(out["g_next"].data_ptr()),
                                       P(out["flux"].data_ptr()), rtol, max_iter, precision, st,
                                       _stream(self.ctx.device))
        if check:
            self.ctx.check(rc, "cps_cp2_step")
        out["stats"] = (_stats(st[0]), _stats(st[1]))
        out["status"] = rc
        return out

    def cp2_kernel_times(self) -> list:
        """Device milliseconds of the last CP2 step's kernels: mean flux,
        tangential flux, update."""
        ms = (ctypes.c_float * 3)()
        self.ctx.check(self.ctx.lib.cps_cp2_kernel_times(self.handle, ms), "cps_cp2_kernel_times")
        return list(ms)

    def adjoint(self, x, g, lam=None, dT=None, dtheta=None, rtol: float = 1e-12,
                max_iter: int = 1_000_000):
        """lambda = A^-1 g; accumulates dL/dT into dT [3, nt] and dL/dtheta
        into dtheta [nt] when those device tensors are given."""
        xd = self.ctx.dev(x, torch.float64)
        gd = self.ctx.dev(g, torch.float64)
        lam = torch.zeros_like(gd) if lam is None else lam
        st = _cps.Stats()
        rc = self.ctx.lib.cps_adjoint(self.handle, P(xd.data_ptr()), P(gd.data_ptr()),
                                      P(lam.data_ptr()),
                                      P(dT.data_ptr()) if dT is not None else None,
                                      P(dtheta.data_ptr()) if dtheta is not None else None,
                                      rtol, max_iter, ctypes.byref(st), _stream(self.ctx.device))
        self.ctx.check(rc, "cps_adjoint")
        return lam, _stats(st)


def cp1_setup(sys_x: System, sys_y: System, xy, tri, eps, kinv):
    """Prepare the CP1 step on a CP1_X / CP1_Y pair assembled from the same
    mesh, fields and Dirichlet sides (the data lives on sys_x)."""
    d = sys_x.ctx.dev
    xy_d, tri_d = d(xy, torch.float64), d(tri, torch.int32)
    eps_d, kinv_d = d(eps, torch.float64), d(kinv, torch.float64)
    rc = sys_x.ctx.lib.cps_cp1_setup(sys_x.handle, sys_y.handle, P(xy_d.data_ptr()),
                                     P(tri_d.data_ptr()), P(eps_d.data_ptr()),
                                     P(kinv_d.data_ptr()), _stream(sys_x.ctx.device))
    sys_x.ctx.check(rc, "cps_cp1_setup")


def set_cp1_path(sys_x: System, path: int):
    """CP1_ONE_LAUNCH (default: the whole outer iteration in one launch for
    Jacobi systems) or CP1_HOST (a cps_solve per solve, the change sums read
    back per sweep), for the pair prepared on sys_x."""
    sys_x.ctx.check(sys_x.ctx.lib.cps_set_cp1_path(sys_x.handle, path), "cps_set_cp1_path")


def cp1_step(sys_x: System, sys_y: System, du_breve, du=None, toll: float = 1e-4,
             max_outer: int = 1000, rtol: float = 1e-10, max_iter: int = 1_000_000,
             precision: int = _cps.FP64, check: bool = True):
    """The CP1 solves of one step (Sec. 3.2.2) with the outer iteration of
    App. B.  du_breve [2, nt] is the predictor increment; du (device [2, nt],
    optional) is the initial guess and is overwritten.  Returns (du, stats
    dict with outer, solve_iters, err, rel_res_max, status)."""
    ctx = sys_x.ctx
    nt = sys_x.nt
    b = ctx.dev(du_breve, torch.float64).reshape(2, nt)
    if du is None:
        du = torch.zeros(2, nt, dtype=torch.float64, device=ctx.device)
    st = _cps.Cp1Stats()
    rc = ctx.lib.cps_cp1_step(sys_x.handle, sys_y.handle, P(b.data_ptr()), P(du.data_ptr()),
                              toll, max_outer, rtol, max_iter, precision, ctypes.byref(st),
                              _stream(ctx.device))
    if check:
        ctx.check(rc, "cps_cp1_step")
    return du, {"outer": int(st.outer), "solve_iters": int(st.solve_iters), "err": float(st.err),
                "rel_res_max": float(st.rel_res_max), "status": rc}


def solve_batch(systems, bs, xs, rtol: float = 1e-10, max_iter: int = 1_000_000,
                precision: int = _cps.FP64, check: bool = True):
    """Solve several systems (device tensors b, x per system) in one call."""
    ctx = systems[0].ctx
    n = len(systems)
    hs = (P * n)(*[s.handle for s in systems])
    bp = (P * n)(*[P(b.data_ptr()) for b in bs])
    xp = (P * n)(*[P(x.data_ptr()) for x in xs])
    st = (_cps.Stats * n)()
    rc = ctx.lib.cps_solve_batch(hs, n, bp, xp, rtol, max_iter, precision, st,
                                 _stream(ctx.device))
    if check:
        ctx.check(rc, "cps_solve_batch")
    return [_stats(s) for s in st]
