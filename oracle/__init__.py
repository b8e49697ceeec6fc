"""CPU oracle for the corrector-step solves (arXiv 2309.03543).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  The CUDA library never imports it and
shares no code with it.  All arithmetic is in ``cps_oracle.c`` (plain FP64,
single-threaded); this module compiles it with gcc on first use and marshals
numpy arrays through ctypes.

Each function names the passage of the paper it follows:

* ``topology`` / ``geometry`` -- Sec. 3.1 (Delaunay mesh, circumcentres,
  sides), Eq. cs1_discr (signed circumcentre distance d_{e,ep}).
* ``xi`` -- Eq. Cs2_4 (Xi = eps M^-1) with M = M0/dt, M0 = I + nu eps Kinv dt.
* ``side_coefficients`` / ``assemble`` -- Eq. CS2_sys_coeff and Eq. Cs2_5
  (CP2 transmissibility l_j d_{j,n}/d_{e,ep}), Eq. CS1_sys_coeff (CP1).
* ``pcg`` -- PCG with Jacobi or incomplete Cholesky IC(0) in natural or a
  given (colour) order, Sec. 3.2.2 / 3.2.3.
* ``pcg_jacobi_omp`` -- the same Jacobi-PCG with OpenMP parallel loops on
  all host cores (``cps_oracle_omp.c``): a timing variant for the CPU
  baseline, checked against ``pcg`` in the tests; never a parity reference.
* ``dense_cholesky_solve`` -- textbook Cholesky, for tiny meshes.
* ``side_gradient`` / ``theta_gradient`` -- adjoint of one solve with respect
  to the side coefficients and the log-permeability (derived from
  Eq. CS2_sys_coeff).
* ``cp2_mean_flux`` / ``cp2_tangential_flux`` / ``cp2_update`` /
  ``cp2_step`` -- the CP2 step around the two solves: the area-weighted mean
  side flux (Eq. flux_k_+_2/3), the co-normal tangential flux of Xi grad eta
  (Eq. Cs2_6, Eq. eta_flux, App. C), the two systems of Eq. Cs2_7, the RT0
  cell velocity (Eq. RT0) and the eps grad Psi update (Eq. grad_PSI).
* ``cp1_mass`` / ``cp1_laplacian`` / ``cp1_step`` -- the two CP1 systems
  (Eq. cs1_sys2, Eq. CS1_sys_coeff) coupled through Mbar_12 and solved by the
  outer iteration of App. B (Eq. A1).

Parity status: every function is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cps_oracle.c")
_LIB = os.path.join(_HERE, "libcps_oracle.so")
_SRC_OMP = os.path.join(_HERE, "cps_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "libcps_oracle_omp.so")

OK = 0
ERR_ARG = -1
ERR_NONMANIFOLD = -2
ERR_NONDELAUNAY = -3
ERR_ORIENTATION = -4
ERR_NOT_SPD = -5
ERR_NOT_CONVERGED = -6
ERR_SINGULAR = -7

CP2, CP1_X, CP1_Y = 0, 1, 2
PER_VERTEX, PER_CELL = 0, 1
PC_NONE, PC_JACOBI, PC_IC0 = 0, 1, 2

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C11, -O2), and its
    multi-threaded timing variant (``build_omp``)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    build_omp(force)
    return _LIB


def build_omp(force: bool = False) -> str:
    """Compile cps_oracle_omp.c (the oracle's Jacobi-PCG with OpenMP parallel
    loops, the benchmark's CPU baseline) with -fopenmp; where the compiler
    has no OpenMP the same source builds single-threaded."""
    if force or not os.path.exists(_LIB_OMP) or \
            os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC_OMP):
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC_OMP, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            D = ctypes.c_double
            lib.or_topology.argtypes = [I64, P, P]
            lib.or_geometry.argtypes = [I64, P, I64, P, P, P, P, P, P, P]
            lib.or_xi.argtypes = [I64, P, P, D, D, P]
            lib.or_xi.restype = None
            lib.or_side_coefficients.argtypes = [I64, P, I64, P, P, P, I64, P, P, I, I, D, D,
                                                 P, P, P]
            lib.or_assemble_csr.argtypes = [I64, P, I64, P, P, I64, P, P, I, I, D, D, P, P, P, P]
            lib.or_pcg.argtypes = [I64, P, P, P, P, P, D, I64, I, P, P]
            lib.or_matvec.argtypes = [I64, P, P, P, P, P]
            lib.or_matvec.restype = None
            lib.or_dense_cholesky_solve.argtypes = [I64, P, P]
            lib.or_side_gradient.argtypes = [I64, P, P, P, P, P]
            lib.or_side_gradient.restype = None
            lib.or_theta_gradient.argtypes = [I64, P, I64, P, P, P, P, P, D, D, P, P]
            lib.or_cp2_mean_flux.argtypes = [I64, P, I64, P, P, P, P, P]
            lib.or_cp1_mass.argtypes = [I64, P, I64, P, P, P, I, D, D, P]
            lib.or_cp2_tangential_flux.argtypes = [I64, P, I64, P, P, P, P, P, I, D, D, P, P]
            lib.or_cp2_update.argtypes = [I64, P, I64, P, P, P, P, P, I, D, D, P, P, P, P,
                                          P, P, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


# ------------------------------------------------------------------ mesh

def topology(tri) -> np.ndarray:
    """nbr[e, j]: cell across local side j of e (side j joins vertices
    (j+1)%3 and (j+2)%3), -1 on the boundary."""
    tri = _i32(tri)
    nt = tri.shape[0]
    nbr = np.empty((nt, 3), dtype=np.int32)
    _check(_load().or_topology(nt, _p(tri), _p(nbr)), "topology")
    return nbr


@dataclass
class Geometry:
    nbr: np.ndarray      # [nt, 3]
    area: np.ndarray     # [nt]
    cc: np.ndarray       # [nt, 2] circumcentres
    length: np.ndarray   # [nt, 3]
    normal: np.ndarray   # [nt, 3, 2] outward unit normals
    dist: np.ndarray     # [nt, 3] d_{e,ep} (interior) or delta (boundary)


def geometry(xy, tri) -> Geometry:
    xy = _f64(xy)
    tri = _i32(tri)
    nt = tri.shape[0]
    nbr = topology(tri)
    area = np.empty(nt)
    cc = np.empty((nt, 2))
    ln = np.empty((nt, 3))
    nrm = np.empty((nt, 3, 2))
    dist = np.empty((nt, 3))
    _check(_load().or_geometry(xy.shape[0], _p(xy), nt, _p(tri), _p(nbr), _p(area), _p(cc),
                               _p(ln), _p(nrm), _p(dist)), "geometry")
    return Geometry(nbr, area, cc, ln, nrm, dist)


def xi(eps, kinv, nu: float, dt: float) -> np.ndarray:
    """Xi = eps dt (I + nu eps dt Kinv)^-1 as (xx, xy, yy) per point."""
    eps = _f64(eps)
    kinv = _f64(kinv).reshape(-1, 3)
    out = np.empty((eps.shape[0], 3))
    _load().or_xi(eps.shape[0], _p(eps), _p(kinv), nu, dt, _p(out))
    return out


def side_coefficients(xy, tri, dirichlet, eps, kinv, field_loc: int, kind: int,
                      nu: float, dt: float):
    """(T [nt,3], sigma [nt], is_dirichlet [nt,3], nbr [nt,3])."""
    xy = _f64(xy)
    tri = _i32(tri)
    dirichlet = _i32(dirichlet)
    eps = _f64(eps)
    kinv = _f64(kinv).reshape(-1, 3)
    nt = tri.shape[0]
    nbr = topology(tri)
    T = np.empty((nt, 3))
    sigma = np.empty(nt)
    isd = np.empty((nt, 3), dtype=np.int32)
    _check(_load().or_side_coefficients(xy.shape[0], _p(xy), nt, _p(tri), _p(nbr),
                                        _p(dirichlet), dirichlet.shape[0], _p(eps), _p(kinv),
                                        field_loc, kind, nu, dt, _p(T), _p(sigma), _p(isd)),
           "side_coefficients")
    return T, sigma, isd, nbr


@dataclass
class CSR:
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def n(self) -> int:
        return self.rowptr.shape[0] - 1

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            for k in range(self.rowptr[i], self.rowptr[i + 1]):
                A[i, self.col[k]] += self.val[k]
        return A

    def matvec(self, x) -> np.ndarray:
        x = _f64(x)
        y = np.empty(self.n)
        _load().or_matvec(self.n, _p(self.rowptr), _p(self.col), _p(self.val), _p(x), _p(y))
        return y

    def diagonal(self) -> np.ndarray:
        d = np.zeros(self.n)
        for i in range(self.n):
            for k in range(self.rowptr[i], self.rowptr[i + 1]):
                if self.col[k] == i:
                    d[i] += self.val[k]
        return d


def assemble(xy, tri, dirichlet, eps, kinv, field_loc: int = PER_VERTEX, kind: int = CP2,
             nu: float = 1.5e-5, dt: float = 0.225) -> CSR:
    """Corrector matrix in CSR (diagonal first in each row)."""
    xy = _f64(xy)
    tri = _i32(tri)
    dirichlet = _i32(dirichlet)
    eps = _f64(eps)
    kinv = _f64(kinv).reshape(-1, 3)
    nt = tri.shape[0]
    rowptr = np.empty(nt + 1, dtype=np.int64)
    col = np.empty(max(4 * nt, 1), dtype=np.int32)
    val = np.empty(max(4 * nt, 1))
    nnz = ctypes.c_int64(0)
    _check(_load().or_assemble_csr(xy.shape[0], _p(xy), nt, _p(tri), _p(dirichlet),
                                   dirichlet.shape[0], _p(eps), _p(kinv), field_loc, kind, nu,
                                   dt, _p(rowptr), _p(col), _p(val), ctypes.byref(nnz)),
           "assemble")
    k = nnz.value
    return CSR(rowptr, col[:k].copy(), val[:k].copy())


def assemble_problem(problem, kind: int = CP2) -> CSR:
    m = problem.mesh
    return assemble(m.xy, m.tri, m.dirichlet, problem.eps, problem.kinv, problem.field_loc,
                    kind, problem.nu, problem.dt)


# ------------------------------------------------------------------ solves

@dataclass
class SolveStats:
    iters: int
    rel_res: float        # true ||b - A x|| / ||b||
    rec_res: float        # recursively updated residual at exit
    status: int


def pcg(A: CSR, b, x0=None, rtol: float = 1e-10, maxit: int = 100000,
        precond: int = PC_JACOBI, perm=None, raise_on_error: bool = True):
    """Textbook PCG; returns (x, SolveStats).  perm[new] = old gives the IC(0)
    elimination order (None: natural)."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    st = np.zeros(3)
    pp = None if perm is None else _i32(perm)
    rc = _load().or_pcg(A.n, _p(A.rowptr), _p(A.col), _p(A.val), _p(b), _p(x), rtol, maxit,
                        precond, None if pp is None else _p(pp), _p(st))
    if raise_on_error and rc not in (OK,):
        raise OracleError(rc, "pcg")
    return x, SolveStats(int(st[0]), float(st[1]), float(st[2]), rc)


_lib_omp = None


def _load_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            build_omp()
            lib = ctypes.CDLL(_LIB_OMP)
            P = ctypes.c_void_p
            lib.oro_threads.argtypes = []
            lib.oro_threads.restype = ctypes.c_int
            lib.oro_pcg_jacobi.argtypes = [ctypes.c_int64, P, P, P, P, P, ctypes.c_double,
                                           ctypes.c_int64, P]
            _lib_omp = lib
    return _lib_omp


def omp_threads() -> int:
    """Threads of the multi-threaded timing variant (OMP_NUM_THREADS, else
    every core the process may run on)."""
    return int(_load_omp().oro_threads())


def pcg_jacobi_omp(A: CSR, b, x0=None, rtol: float = 1e-10, maxit: int = 100000):
    """The textbook Jacobi-PCG of ``pcg`` with OpenMP parallel row loops and
    reductions on all host cores (cps_oracle_omp.c): the benchmark's CPU
    baseline.  Returns (x, SolveStats); the iterates equal ``pcg``'s up to
    the summation order of the inner products."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    st = np.zeros(3)
    rc = _load_omp().oro_pcg_jacobi(A.n, _p(A.rowptr), _p(A.col), _p(A.val), _p(b), _p(x),
                                    rtol, maxit, _p(st))
    return x, SolveStats(int(st[0]), float(st[1]), float(st[2]), rc)


def dense_cholesky_solve(A, b) -> np.ndarray:
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    x = _f64(b).copy()
    _check(_load().or_dense_cholesky_solve(A.shape[0], _p(A), _p(x)), "dense_cholesky")
    return x


def red_black_order(nt: int) -> np.ndarray:
    """perm[new] = old: even cells (up triangles of the lattice) first, then
    odd ones -- a two-colouring of the lattice's cell graph."""
    return np.concatenate([np.arange(0, nt, 2), np.arange(1, nt, 2)]).astype(np.int32)


# ------------------------------------------------------------------ adjoint

def side_gradient(nbr, is_dirichlet, lam, x) -> np.ndarray:
    """dL/dT per local side for one solve with adjoint lam = A^-1 dL/dx."""
    nbr = _i32(nbr)
    isd = _i32(is_dirichlet)
    lam = _f64(lam)
    x = _f64(x)
    nt = nbr.shape[0]
    dT = np.empty((nt, 3))
    _load().or_side_gradient(nt, _p(nbr), _p(isd), _p(lam), _p(x), _p(dT))
    return dT


def theta_gradient(xy, tri, nbr, is_dirichlet, eps, theta, nu, dt, dT) -> np.ndarray:
    """Chain dL/dT to the cell log-permeability theta (Kinv = exp(-theta) I)."""
    xy = _f64(xy)
    tri = _i32(tri)
    nbr = _i32(nbr)
    isd = _i32(is_dirichlet)
    eps = _f64(eps)
    theta = _f64(theta)
    dT = _f64(dT)
    nt = tri.shape[0]
    out = np.empty(nt)
    _check(_load().or_theta_gradient(xy.shape[0], _p(xy), nt, _p(tri), _p(nbr), _p(isd),
                                     _p(eps), _p(theta), nu, dt, _p(dT), _p(out)),
           "theta_gradient")
    return out


def solve_problem(problem, b, rtol: float = 1e-13, precond: int = PC_JACOBI, x0=None,
                  maxit: int = 1000000, kind: int = CP2):
    """Assemble and solve one corrector system; returns (x, stats, A)."""
    A = assemble_problem(problem, kind)
    x, st = pcg(A, b, x0=x0, rtol=rtol, maxit=maxit, precond=precond,
                raise_on_error=False)
    if st.status not in (OK, ERR_NOT_CONVERGED):
        raise OracleError(st.status, "pcg")
    return x, st, A


# ------------------------------------------------------------------ CP2 step

def _mesh_args(xy, tri, nbr, is_dirichlet):
    return _f64(xy), _i32(tri), _i32(nbr), _i32(is_dirichlet)


def cp2_mean_flux(xy, tri, nbr, is_dirichlet, u) -> np.ndarray:
    """Fbar [nt, 3]: outward area-weighted mean flux per local side
    (Eq. flux_k_+_2/3).  u is [2, nt] (x row, y row)."""
    xy, tri, nbr, isd = _mesh_args(xy, tri, nbr, is_dirichlet)
    u = _f64(u).reshape(2, -1)
    nt = tri.shape[0]
    out = np.empty((nt, 3))
    _check(_load().or_cp2_mean_flux(xy.shape[0], _p(xy), nt, _p(tri), _p(nbr), _p(isd),
                                    _p(u), _p(out)), "cp2_mean_flux")
    return out


def cp2_tangential_flux(xy, tri, nbr, is_dirichlet, eps, kinv, field_loc, nu, dt,
                        eta) -> np.ndarray:
    """tau [nt, 3]: tangential (co-normal) part of the outward flux of
    Xi grad(eta) per local side (Eq. Cs2_6, Eq. eta_flux, App. C)."""
    xy, tri, nbr, isd = _mesh_args(xy, tri, nbr, is_dirichlet)
    eps = _f64(eps)
    kinv = _f64(kinv).reshape(-1, 3)
    eta = _f64(eta)
    nt = tri.shape[0]
    out = np.empty((nt, 3))
    _check(_load().or_cp2_tangential_flux(xy.shape[0], _p(xy), nt, _p(tri), _p(nbr), _p(isd),
                                          _p(eps), _p(kinv), field_loc, nu, dt, _p(eta),
                                          _p(out)), "cp2_tangential_flux")
    return out


def cp2_update(xy, tri, nbr, is_dirichlet, eps, kinv, field_loc, nu, dt, fbar, T, tau, eta,
               u23, g_k):
    """(Q [nt,3], u_next [2,nt], g_next [2,nt]): outward side fluxes of the
    new velocity, its RT0 cell value at the centroid (Eq. RT0) and the
    eps grad Psi update (Eq. grad_PSI)."""
    xy, tri, nbr, isd = _mesh_args(xy, tri, nbr, is_dirichlet)
    eps = _f64(eps)
    kinv = _f64(kinv).reshape(-1, 3)
    fbar, T, tau, eta = _f64(fbar), _f64(T), _f64(tau), _f64(eta)
    u23 = _f64(u23).reshape(2, -1)
    g_k = _f64(g_k).reshape(2, -1)
    nt = tri.shape[0]
    Q = np.empty((nt, 3))
    u_next = np.empty((2, nt))
    g_next = np.empty((2, nt))
    _check(_load().or_cp2_update(xy.shape[0], _p(xy), nt, _p(tri), _p(nbr), _p(isd), _p(eps),
                                 _p(kinv), field_loc, nu, dt, _p(fbar), _p(T), _p(tau),
                                 _p(eta), _p(u23), _p(g_k), _p(Q), _p(u_next), _p(g_next)),
           "cp2_update")
    return Q, u_next, g_next


@dataclass
class CP2Step:
    fbar: np.ndarray     # [nt, 3]
    eta_tilde: np.ndarray
    tau: np.ndarray      # [nt, 3], from eta_tilde
    eta: np.ndarray
    Q: np.ndarray        # [nt, 3]
    u_next: np.ndarray   # [2, nt]
    g_next: np.ndarray   # [2, nt]
    A: CSR


def cp2_step(problem, u23, g_k, rtol: float = 1e-13, dense: bool | None = None) -> CP2Step:
    """One CP2 step (Sec. 3.2.3): Fbar -> solve A eta~ = sum Fbar
    (Eq. Cs2_7_1) -> tau(eta~) -> solve A eta = sum Fbar + sum tau
    (Eq. Cs2_7_2, warm start eta~) -> fluxes, RT0 velocity, eps grad Psi.
    Solves by dense Cholesky for nt <= 2000 (or ``dense=True``), else PCG
    (Jacobi) to ``rtol``."""
    m = problem.mesh
    if problem.field_loc not in (PER_VERTEX, PER_CELL):
        raise ValueError("cp2_step takes vertex or cell fields (Xi from eps, Kinv)")
    A = assemble_problem(problem, CP2)
    T, _, isd, nbr = side_coefficients(m.xy, m.tri, m.dirichlet, problem.eps, problem.kinv,
                                       problem.field_loc, CP2, problem.nu, problem.dt)
    nt = m.tri.shape[0]
    if dense is None:
        dense = nt <= 2000
    D = A.dense() if dense else None

    def solve(b, x0):
        if dense:
            return dense_cholesky_solve(D, b)
        x, st = pcg(A, b, x0=x0, rtol=rtol, raise_on_error=False)
        if st.status not in (OK, ERR_NOT_CONVERGED):
            raise OracleError(st.status, "pcg")
        return x

    args = (m.xy, m.tri, nbr, isd)
    fields = (problem.eps, problem.kinv, problem.field_loc, problem.nu, problem.dt)
    fbar = cp2_mean_flux(*args, u23)
    eta_t = solve(fbar.sum(axis=1), None)
    tau = cp2_tangential_flux(*args, *fields, eta_t)
    eta = solve(fbar.sum(axis=1) + tau.sum(axis=1), eta_t)
    Q, u_next, g_next = cp2_update(*args, *fields, fbar, T, tau, eta, u23, g_k)
    return CP2Step(fbar, eta_t, tau, eta, Q, u_next, g_next, A)


# ------------------------------------------------------------------ CP1 step

def cp1_mass(xy, tri, eps, kinv, field_loc, nu, dt) -> np.ndarray:
    """[nt, 3]: (Mbar_11 A_e, Mbar_12 A_e, Mbar_22 A_e) per cell."""
    xy, tri = _f64(xy), _i32(tri)
    eps = _f64(eps)
    kinv = _f64(kinv).reshape(-1, 3)
    nt = tri.shape[0]
    out = np.empty((nt, 3))
    _check(_load().or_cp1_mass(xy.shape[0], _p(xy), nt, _p(tri), _p(eps), _p(kinv), field_loc,
                               nu, dt, _p(out)), "cp1_mass")
    return out


def cp1_laplacian(T, nbr, is_dirichlet, u) -> np.ndarray:
    """(nu L u)_e = sum_j T_j (u_e - u_ep), T_j = nu l_j / d_{e,ep}; a Dirichlet
    side (zero increment at its midpoint) adds T_j u_e, a no-flux side
    nothing -- the off-diagonal part of Eq. CS1_sys_coeff as an operator."""
    u = _f64(u)
    across = np.where(nbr >= 0, u[np.maximum(nbr, 0)], 0.0)
    open_side = (nbr >= 0) | (is_dirichlet != 0)
    return np.where(open_side, T * (u[:, None] - across), 0.0).sum(axis=1)


@dataclass
class CP1Step:
    du: np.ndarray          # [2, nt] the converged increments (x row, y row)
    outer: int              # outer iterations after the uncoupled start
    err: float              # last err = min(err_x, err_y)
    history: list           # err per outer iteration


def cp1_step(problem, du_breve, toll: float = 1e-4, max_outer: int = 1000, rtol: float = 1e-13,
             dense: bool | None = None, criterion: str = "min") -> CP1Step:
    """The CP1 solves of one time step (Sec. 3.2.2, App. B).

    Per component k (x, y) the system (Eq. cs1_sys2 with the coefficients of
    Eq. CS1_sys_coeff) is
        (Mbar_kk A_e + nu L) du_k = -nu L du_breve_k - Mbar_12 A_e du_other,
    the right-hand side with the sign of Eq. CS1_new / CS1_2 written with the
    outward normal derivative (a backward-Euler viscous update of the
    predictor increment).  Eq. A1: i = 0 solves both with the coupling left
    out; then both are solved again, each with the other's previous iterate,
    until err = min(err_x, err_y) <= toll, err_k = ||du_k^{i+1} - du_k^i|| /
    ||du_k^i|| (2-norms; 0/0 = 0).  ``criterion="max"`` stops on the larger
    of the two instead (used by the pins to reach the coupled solution)."""
    m = problem.mesh
    if problem.field_loc not in (PER_VERTEX, PER_CELL):
        raise ValueError("cp1_step takes vertex or cell fields")
    f = (problem.eps, problem.kinv, problem.field_loc, problem.nu, problem.dt)
    Ax = assemble(m.xy, m.tri, m.dirichlet, problem.eps, problem.kinv, problem.field_loc, CP1_X,
                  problem.nu, problem.dt)
    Ay = assemble(m.xy, m.tri, m.dirichlet, problem.eps, problem.kinv, problem.field_loc, CP1_Y,
                  problem.nu, problem.dt)
    T, _, isd, nbr = side_coefficients(m.xy, m.tri, m.dirichlet, *f[:3], CP1_X, f[3], f[4])
    mass = cp1_mass(m.xy, m.tri, *f)
    nt = m.tri.shape[0]
    if dense is None:
        dense = nt <= 2000
    Dx, Dy = (Ax.dense(), Ay.dense()) if dense else (None, None)

    def solve(A, D, b, x0):
        if dense:
            return dense_cholesky_solve(D, b)
        x, st = pcg(A, b, x0=x0, rtol=rtol, raise_on_error=False)
        if st.status not in (OK, ERR_NOT_CONVERGED):
            raise OracleError(st.status, "pcg")
        return x

    du_breve = _f64(du_breve).reshape(2, nt)
    lap = np.stack([-cp1_laplacian(T, nbr, isd, du_breve[0]),
                    -cp1_laplacian(T, nbr, isd, du_breve[1])])
    u = solve(Ax, Dx, lap[0], None)
    v = solve(Ay, Dy, lap[1], None)

    def rel(new, old):
        d, o = np.linalg.norm(new - old), np.linalg.norm(old)
        return 0.0 if d == 0.0 else (d / o if o > 0.0 else np.inf)

    hist = []
    it = 0
    err = np.inf
    while it < max_outer:
        un = solve(Ax, Dx, lap[0] - mass[:, 1] * v, u)
        vn = solve(Ay, Dy, lap[1] - mass[:, 1] * u, v)
        ex, ey = rel(un, u), rel(vn, v)
        err = min(ex, ey) if criterion == "min" else max(ex, ey)
        u, v = un, vn
        it += 1
        hist.append(err)
        if err <= toll:
            break
    return CP1Step(np.stack([u, v]), it, err, hist)
