"""ctypes front end of the plain FP64 CPU oracle (test infrastructure).

The oracle is ``sdc_oracle.cpp`` compiled with the host C++ compiler into
``liboracle.so`` next to this file.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package; the CUDA library and its
Python binding never do.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdc_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MAX_SWEEPS = 64
MAX_M = 8
OK, INVALID, CG_NOCONV, NONFINITE, DOMAIN = 0, -1, -4, -6, -7


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no OpenMP, no BLAS)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Ionic(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("ga", "gs", "a", "eps", "mu1", "mu2", "cw")]


class _Opts(C.Structure):
    _fields_ = [("alpha", C.c_double), ("cg_rtol", C.c_double), ("cg_maxit", C.c_int),
                ("reaction_implicit", C.c_int), ("w_frozen", C.c_int),
                ("energy_stop", C.c_int), ("rho", C.c_double), ("qhat", C.c_int),
                ("drop_rule", C.c_int), ("coarse_min_rows", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("sweeps_run", C.c_int), ("n_active", C.c_int * MAX_SWEEPS),
                ("cg_iters", C.c_int * (MAX_SWEEPS * MAX_M)), ("cg_relres_max", C.c_double),
                ("min_margin", C.c_double), ("energy", C.c_double * MAX_SWEEPS),
                ("tol_drop", C.c_double)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.ora_collocation.argtypes = [C.c_int, _dp, _dp, _dp]
        L.ora_ionic_eval.argtypes = [C.POINTER(_Ionic), C.c_double, C.c_double, _dp]
        L.ora_create_fem.argtypes = [C.c_int, C.c_int, _dp, C.c_int, _ip, _dp, _dp, _dp]
        L.ora_create_fem.restype = C.c_void_p
        L.ora_create_matrix.argtypes = [C.c_int, _ip, _ip, _dp, _dp]
        L.ora_create_matrix.restype = C.c_void_p
        L.ora_n.argtypes = [C.c_void_p]
        L.ora_nnz.argtypes = [C.c_void_p]
        L.ora_get_matrix.argtypes = [C.c_void_p, _ip, _ip, _dp, _dp]
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_step.argtypes = [C.c_void_p, C.POINTER(_Ionic), C.c_int, _dp, _dp, _dp, C.c_double,
                               C.c_int, C.c_double, C.POINTER(_Opts), C.POINTER(Stats), _ip, _dp, _dp]
        L.ora_step_forced.argtypes = [C.c_void_p, C.POINTER(_Ionic), C.c_int, _dp, _dp, _dp,
                                      C.c_double, C.c_int, C.c_double, C.POINTER(_Opts),
                                      C.POINTER(Stats), _ip, _dp, _dp, _ip, _ip]
        L.ora_step_tangent.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(_Ionic),
                                       C.POINTER(_Ionic), C.c_int, _dp, _dp, _dp, _dp, _dp,
                                       C.c_double, C.c_int, C.POINTER(_Opts), _ip, _ip, _ip]
        L.ora_step_emi.argtypes = [C.c_void_p, C.POINTER(_Ionic), C.c_double, C.c_double, C.c_int,
                                   C.c_int, _ip, _ip, _dp, _ip, _dp, _dp, _dp, C.c_double, C.c_int,
                                   C.c_double, C.POINTER(_Opts), C.POINTER(Stats), _ip, _ip]
        L.ora_pcg_csr.argtypes = [C.c_int, _ip, _ip, _dp, C.c_int, _ip, _ip, _dp, _dp, C.c_double,
                                  C.c_int, _ip]
        L.ora_two_level_apply.argtypes = [C.c_int, _ip, _ip, _dp, C.c_int, _ip, _ip, _dp, _dp]
        L.ora_collocation_solve.argtypes = [C.c_void_p, C.POINTER(_Ionic), C.c_int, _dp, _dp, _dp,
                                            C.c_double, _dp, _dp, _ip]
        _lib = L
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _i(a):
    return None if a is None else a.ctypes.data_as(_ip)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def collocation(M: int):
    """Radau-IIA nodes tau, cumulative quadrature Q and LU-trick Qhat (Sec. 3.1)."""
    tau, Q, Qh = np.zeros(M), np.zeros((M, M)), np.zeros((M, M))
    rc = lib().ora_collocation(M, _d(tau), _d(Q), _d(Qh))
    if rc != OK:
        raise ValueError("ora_collocation(M=%d) failed: %d" % (M, rc))
    return tau, Q, Qh


def pcg_csr(ptr, col, val, b, act=None, dom=None, rtol=1e-10, maxit=100000):
    """PCG on an explicit CSR matrix restricted to `act` (all rows when None):
    Jacobi, plus the two-level coarse part over the labels `dom` when given.
    Returns (x, iterations, status)."""
    ptr, col, val, b = _i32(ptr), _i32(col), _f64(val), _f64(b)
    n = len(b)
    act = _i32(np.arange(n) if act is None else act)
    x = np.zeros(n)
    it = C.c_int(0)
    rc = lib().ora_pcg_csr(n, _i(ptr), _i(col), _d(val), len(act), _i(act), _i(_i32(dom)), _d(b),
                           _d(x), rtol, maxit, C.byref(it))
    return x, it.value, rc


def two_level_apply(ptr, col, val, r, dom, act=None):
    """z = D^-1 r + Z E^-1 Z' r of the two-level preconditioner (Sec. 6) on an explicit
    CSR matrix restricted to `act`, Z the indicator vectors of the labels `dom`."""
    ptr, col, val, r = _i32(ptr), _i32(col), _f64(val), _f64(r)
    n = len(r)
    act = _i32(np.arange(n) if act is None else act)
    z = np.zeros(n)
    rc = lib().ora_two_level_apply(n, _i(ptr), _i(col), _d(val), len(act), _i(act),
                                   _i(_i32(dom)), _d(r), _d(z))
    if rc != OK:
        raise ValueError("ora_two_level_apply failed: %d" % rc)
    return z


def _ionic(p: dict) -> _Ionic:
    return _Ionic(*(float(p[k]) for k in ("ga", "gs", "a", "eps", "mu1", "mu2", "cw")))


def ionic_eval(p: dict, v: float, w: float):
    """(I_ion, dI/dv, dI/dw, R, dR/dv, dR/dw) of the Aliev-Panfilov model (Sec. 5.1.1)."""
    out = np.zeros(6)
    lib().ora_ionic_eval(C.byref(_ionic(p)), float(v), float(w), _d(out))
    return out


class System:
    """Assembled P1 system (stiffness K, lumped mass m) held by the oracle."""

    def __init__(self, handle):
        if not handle:
            raise ValueError("oracle system creation failed")
        self._h = C.c_void_p(handle)

    @classmethod
    def from_mesh(cls, mesh, sigma=None, dof_scale=None):
        sigma9 = _f64(np.eye(3) if sigma is None else np.asarray(sigma).reshape(3, 3))
        es = None if mesh.elem_sigma is None else _f64(mesh.elem_sigma.reshape(-1, 9))
        xyz = _f64(mesh.xyz)
        el = _i32(mesh.elems)
        ds = _f64(dof_scale)
        h = lib().ora_create_fem(mesh.dim, mesh.n_nodes, _d(xyz), mesh.n_elems, _i(el),
                                 _d(sigma9), _d(es), _d(ds))
        return cls(h)

    @classmethod
    def from_matrix(cls, ptr, col, val, mass):
        ptr, col, val, mass = _i32(ptr), _i32(col), _f64(val), _f64(mass)
        return cls(lib().ora_create_matrix(len(mass), _i(ptr), _i(col), _d(val), _d(mass)))

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.ora_destroy(self._h)
            self._h = None

    @property
    def n(self) -> int:
        return lib().ora_n(self._h)

    def matrix(self):
        n, nnz = self.n, lib().ora_nnz(self._h)
        ptr, col = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32)
        val, mass = np.zeros(nnz), np.zeros(n)
        lib().ora_get_matrix(self._h, _i(ptr), _i(col), _d(val), _d(mass))
        return ptr, col, val, mass

    def dense(self):
        ptr, col, val, mass = self.matrix()
        K = np.zeros((self.n, self.n))
        for i in range(self.n):
            K[i, col[ptr[i]:ptr[i + 1]]] += val[ptr[i]:ptr[i + 1]]
        return K, mass

    def step(self, ionic: dict, M: int, v, w, dt: float, sweeps: int, tol: float,
             alpha: float = 0.1, cg_rtol: float = 1e-10, cg_maxit: int = 10000,
             istim=None, reaction_implicit: bool = True, w_frozen: bool = False,
             want_log: bool = False, want_nodes: bool = False, energy_stop: bool = False,
             rho: float = 0.0, qhat: str = "lu", drop_rule: int = 0):
        """One SDC step.  Returns dict(v, w, status, stats, active[, V, W]).
        energy_stop ends the sweeps by the energy-norm test of Sec. 3.2 with SDC
        contraction rho (0: estimated from successive sweeps); `sweeps` is then
        the largest number of sweeps.  qhat: "lu" (LU trick) or "ie" (implicit
        Euler) preconditioner of the sweep.  drop_rule 1 selects with the a
        priori drop tolerance of Sec. 4.1 (rho > 0 given, c from the first sweep)
        instead of alpha TOL; stats.tol_drop is the value used."""
        n = self.n
        v = np.array(v, dtype=np.float64, copy=True)
        w = np.array(w, dtype=np.float64, copy=True)
        st = Stats()
        opts = _Opts(alpha, cg_rtol, cg_maxit, int(reaction_implicit), int(w_frozen),
                     int(energy_stop), float(rho), {"lu": 0, "ie": 1}[qhat], int(drop_rule))
        log = np.zeros(max(1, sweeps) * n, np.int32) if want_log else None
        Vn = np.zeros((M, n)) if want_nodes else None
        Wn = np.zeros((M, n)) if want_nodes else None
        rc = lib().ora_step(self._h, C.byref(_ionic(ionic)), M, _d(_f64(istim)), _d(v), _d(w),
                            dt, sweeps, tol, C.byref(opts), C.byref(st), _i(log), _d(Vn), _d(Wn))
        out = dict(v=v, w=w, status=rc, stats=st)
        if want_log:
            lists, pos = [], 0
            for k in range(st.sweeps_run):
                c = st.n_active[k]
                lists.append(log[pos:pos + c].copy())
                pos += c
            out["active"] = lists
        if want_nodes:
            out["V"], out["W"] = Vn, Wn
        return out

    def step_forced(self, ionic: dict, M: int, v, w, dt: float, sweeps: int, active_lists,
                    cg_rtol: float = 1e-10, cg_maxit: int = 10000, istim=None,
                    reaction_implicit: bool = True, w_frozen: bool = False):
        """One SDC step whose active sets are given (active_lists[k] for sweeps
        k >= 1; the first sweep covers every dof) instead of selected."""
        n = self.n
        v = np.array(v, dtype=np.float64, copy=True)
        w = np.array(w, dtype=np.float64, copy=True)
        counts = np.zeros(max(1, sweeps), np.int32)
        counts[0] = n
        lists = []
        for k in range(1, sweeps):
            lk = np.ascontiguousarray(active_lists[k], dtype=np.int32)
            counts[k] = lk.size
            lists.append(lk)
        flat = np.concatenate(lists) if lists else np.zeros(1, np.int32)
        flat = np.ascontiguousarray(flat, dtype=np.int32)
        st = Stats()
        opts = _Opts(0.1, cg_rtol, cg_maxit, int(reaction_implicit), int(w_frozen))
        rc = lib().ora_step_forced(self._h, C.byref(_ionic(ionic)), M, _d(_f64(istim)), _d(v),
                                   _d(w), dt, sweeps, 0.0, C.byref(opts), C.byref(st), None, None,
                                   None, _i(counts), _i(flat))
        return dict(v=v, w=w, status=rc, stats=st)

    def step_tangent(self, ionic: dict, M: int, v, dv, w, dw, dt: float, sweeps: int,
                     active_lists, dionic: dict = None, dscale_system=None,
                     cg_rtol: float = 1e-13, cg_maxit: int = 10000, istim=None,
                     reaction_implicit: bool = True, w_frozen: bool = False):
        """Forward-mode derivative of step_forced along a direction: (dv, dw) of
        the initial state, dionic of the ionic parameters, and a conductivity
        scale direction given as the system assembled with that direction as its
        scale (dscale_system; K is linear in the scale).  Returns dict(v, dv, w,
        dw, status); v, w equal step_forced's result bitwise."""
        n = self.n
        v = np.array(v, dtype=np.float64, copy=True)
        w = np.array(w, dtype=np.float64, copy=True)
        dv = np.array(dv, dtype=np.float64, copy=True)
        dw = np.array(dw, dtype=np.float64, copy=True)
        counts = np.zeros(max(1, sweeps), np.int32)
        counts[0] = n
        lists = []
        for k in range(1, sweeps):
            lk = np.ascontiguousarray(active_lists[k], dtype=np.int32)
            counts[k] = lk.size
            lists.append(lk)
        flat = np.concatenate(lists) if lists else np.zeros(1, np.int32)
        flat = np.ascontiguousarray(flat, dtype=np.int32)
        opts = _Opts(0.1, cg_rtol, cg_maxit, int(reaction_implicit), int(w_frozen))
        di = C.byref(_ionic(dionic)) if dionic is not None else None
        hd = dscale_system._h if dscale_system is not None else None
        iters = np.zeros(MAX_SWEEPS * MAX_M, np.int32)
        rc = lib().ora_step_tangent(self._h, hd, C.byref(_ionic(ionic)), di, M, _d(_f64(istim)),
                                    _d(v), _d(dv), _d(w), _d(dw), dt, sweeps, C.byref(opts),
                                    _i(counts), _i(flat), _i(iters))
        return dict(v=v, dv=dv, w=w, dw=dw, status=rc, iters=iters)

    def step_emi(self, wl, u, w, sweeps=None, tol=None, cg_rtol=None, w_frozen=False,
                 want_log=False, energy_stop=False, rho=0.0, alpha=None, drop_rule=0,
                 coarse=False, coarse_min_rows=0):
        """One SDC step of a cell-by-cell workload (K of this system = the
        subdomain stiffness; pairs, Robin and membrane data from `wl`).
        `energy_stop` ends the sweeps by the energy-norm test of Sec. 3.2
        (`rho` given, or estimated from successive sweep energies when 0).
        `coarse` solves the node systems with the two-level preconditioner (Sec. 6)
        instead of Jacobi alone, over the workload's subdomain labels (True) or the
        block labels given as an array; sweeps with fewer than `coarse_min_rows`
        active dofs keep Jacobi alone."""
        n = self.n
        sweeps = wl.sweeps if sweeps is None else sweeps
        tol = wl.tol if tol is None else tol
        cg_rtol = wl.cg_rtol if cg_rtol is None else cg_rtol
        u = np.array(u, dtype=np.float64, copy=True)
        w = np.array(w, dtype=np.float64, copy=True)
        st = Stats()
        opts = _Opts(wl.alpha if alpha is None else alpha, cg_rtol, 100000, 1, int(w_frozen),
                     int(energy_stop), rho, 0, int(drop_rule), int(coarse_min_rows))
        log = np.zeros(max(1, sweeps) * n, np.int32) if want_log else None
        rob = _f64(wl.robin)
        dom = None
        if coarse is not None and coarse is not False:
            dom = _i32(wl.labels if coarse is True else coarse)
        pk, pl, pa, pkd = _i32(wl.pair_k), _i32(wl.pair_l), _f64(wl.pair_area), _i32(wl.pair_kind)
        rc = lib().ora_step_emi(self._h, C.byref(_ionic(wl.ionic)), wl.Cm, wl.g_gap, wl.M,
                                wl.n_pairs, _i(pk), _i(pl), _d(pa), _i(pkd), _d(rob), _d(u),
                                _d(w), wl.dt, sweeps, tol, C.byref(opts), C.byref(st), _i(log),
                                _i(dom))
        out = dict(u=u, w=w, status=rc, stats=st)
        if want_log:
            lists, pos = [], 0
            for k in range(st.sweeps_run):
                c = st.n_active[k]
                lists.append(log[pos:pos + c].copy())
                pos += c
            out["active"] = lists
        return out

    def collocation_solve(self, ionic: dict, M: int, v, w, dt: float, istim=None):
        """Dense Newton solution of the full collocation system (tiny meshes)."""
        n = self.n
        v = np.array(v, dtype=np.float64, copy=True)
        w = np.array(w, dtype=np.float64, copy=True)
        Vn, Wn = np.zeros((M, n)), np.zeros((M, n))
        it = C.c_int(0)
        rc = lib().ora_collocation_solve(self._h, C.byref(_ionic(ionic)), M, _d(_f64(istim)),
                                         _d(v), _d(w), dt, _d(Vn), _d(Wn), C.byref(it))
        return dict(v=v, w=w, V=Vn, W=Wn, status=rc, newton_iters=it.value)
