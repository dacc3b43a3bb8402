"""ctypes binding of libsdc_gb300.so: the C ABI of include/sdc.h, same names.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no fallback: if the shared library is missing, every
call raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SDC_GB300_LIB selects another build of the library, e.g. the checked build
# libsdc_gb300_checked.so (every kernel gather tested against its bound)
LIB_PATH = os.environ.get("SDC_GB300_LIB") or os.path.join(HERE, "libsdc_gb300.so")

SDC_MAX_M = 8
SDC_MAX_SWEEPS = 64
SDC_N_PHASES = 5
SDC_PCG_NOALLOC_MAX_ROWS = 65536
SDC_MAX_COARSE_BLOCKS = 1024
PHASES = ("residual", "pcg", "update", "select", "extract")
SDC_OK, SDC_E_INVALID, SDC_E_CUDA, SDC_E_NOMEM = 0, -1, -2, -3
SDC_E_CG_NOCONV, SDC_E_TIMEOUT, SDC_E_NONFINITE, SDC_E_DOMAIN = -4, -5, -6, -7


class sdc_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int), ("xyz", C.POINTER(C.c_double)),
                ("n_elems", C.c_int), ("elem_ptr", C.POINTER(C.c_int)),
                ("elem_node", C.POINTER(C.c_int)), ("sigma", C.POINTER(C.c_double)),
                ("elem_sigma", C.POINTER(C.c_double)), ("dof_scale", C.POINTER(C.c_double))]


class sdc_ionic(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("ga", "gs", "a", "eps", "mu1", "mu2", "cw")]


class sdc_options(C.Structure):
    _fields_ = [("alpha", C.c_double), ("cg_rtol", C.c_double), ("cg_maxit", C.c_int),
                ("reaction_implicit", C.c_int), ("w_frozen", C.c_int), ("drop_rel", C.c_double),
                ("spin_budget", C.c_longlong), ("cg_block_size", C.c_int),
                ("cg_smem_block_size", C.c_int), ("cg_cluster_max", C.c_int),
                ("cg_max_blocks", C.c_int), ("cg_variant", C.c_int),
                ("cg_rows_per_block", C.c_int), ("cg_cluster_rows", C.c_int),
                ("profile", C.c_int), ("inject_fault", C.c_int), ("cg_pipelined", C.c_int),
                ("energy_stop", C.c_int), ("sdc_rho", C.c_double), ("sdc_qhat", C.c_int),
                ("reorder", C.c_int), ("drop_rule", C.c_int), ("cg_scaled", C.c_int),
                ("batch_graph", C.c_int), ("coarse_min_rows", C.c_int)]


class sdc_stats(C.Structure):
    _fields_ = [("sweeps_run", C.c_int), ("n_active", C.c_int * SDC_MAX_SWEEPS),
                ("nnz_active", C.c_longlong * SDC_MAX_SWEEPS),
                ("cg_iters", (C.c_int * SDC_MAX_M) * SDC_MAX_SWEEPS),
                ("cg_relres_max", C.c_double), ("min_margin", C.c_double),
                ("kernel_launches", C.c_int), ("phase_launches", C.c_int * SDC_N_PHASES),
                ("phase_ms", C.c_double * SDC_N_PHASES),
                ("cg_ms", (C.c_double * SDC_MAX_M) * SDC_MAX_SWEEPS),
                ("energy", C.c_double * SDC_MAX_SWEEPS), ("tol_drop", C.c_double),
                ("captured", C.c_int)]


class sdc_tune_report(C.Structure):
    _fields_ = [("trials", C.c_int), ("base_ms", C.c_double), ("best_ms", C.c_double),
                ("cg_pipelined", C.c_int), ("cg_scaled", C.c_int), ("smem_block", C.c_int),
                ("big_rows", C.c_int), ("general_block", C.c_int), ("cluster_rows", C.c_int),
                ("batch_pipelined", C.c_int), ("batch_block", C.c_int),
                ("batch_rows_per_block", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class sdc_tape(C.Structure):
    _fields_ = [("mode", C.c_int), ("sweeps", C.c_int), ("d_V", C.c_void_p), ("d_W", C.c_void_p),
                ("d_act", C.c_void_p), ("n_active", C.c_int * SDC_MAX_SWEEPS)]


class sdc_emi(C.Structure):
    _fields_ = [("n_pairs", C.c_int), ("pair_k", C.POINTER(C.c_int)),
                ("pair_l", C.POINTER(C.c_int)), ("pair_area", C.POINTER(C.c_double)),
                ("pair_kind", C.POINTER(C.c_int)), ("robin", C.POINTER(C.c_double)),
                ("Cm", C.c_double), ("g_gap", C.c_double)]


SDC_TAPE_OFF, SDC_TAPE_RECORD, SDC_TAPE_REPLAY = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p

# name -> (restype, argtypes)
SIGNATURES = {
    "sdc_default_options": (None, [C.POINTER(sdc_options)]),
    "sdc_default_ionic": (None, [C.POINTER(sdc_ionic)]),
    "sdc_radau": (C.c_int, [C.c_int, _dp, _dp, _dp]),
    "sdc_create": (C.c_int, [C.POINTER(_vp), C.POINTER(sdc_mesh), C.POINTER(sdc_ionic), C.c_int,
                             C.POINTER(sdc_options), _vp]),
    "sdc_create_emi": (C.c_int, [C.POINTER(_vp), C.POINTER(sdc_mesh), C.POINTER(sdc_emi),
                                 C.POINTER(sdc_ionic), C.c_int, C.POINTER(sdc_options), _vp]),
    "sdc_set_stimulus": (C.c_int, [_vp, _ip, C.c_int, C.c_double, C.c_double, C.c_double]),
    "sdc_step": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_double, C.c_int, C.c_double,
                           C.POINTER(sdc_stats)]),
    "sdc_step_host": (C.c_int, [_vp, _dp, _dp, C.c_double, C.c_double, C.c_int, C.c_double,
                                C.POINTER(sdc_stats)]),
    "sdc_get_nodes": (C.c_int, [_vp, _vp, _vp]),
    "sdc_get_active": (C.c_int, [_vp, C.c_int, _ip, _ip]),
    "sdc_get_info": (C.c_int, [_vp, _ip, C.POINTER(C.c_longlong), _ip]),
    "sdc_get_matrix": (C.c_int, [_vp, _ip, _ip, _dp, _dp]),
    "sdc_pcg_solve": (C.c_int, [C.c_int, _vp, _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp,
                                C.c_double, _vp, _vp, C.c_double, C.c_int, _ip, _dp, _vp]),
    "sdc_pcg_solve_noalloc": (C.c_int, [C.c_int, _vp, _vp, _vp, C.c_int, C.c_int, _vp, _vp,
                                        _vp, C.c_double, _vp, _vp, C.c_double, C.c_int, _ip, _dp,
                                        _vp]),
    "sdc_batch_create": (C.c_int, [C.POINTER(_vp), _vp, C.c_int, C.POINTER(sdc_ionic), C.c_int,
                                   C.POINTER(sdc_options), _vp]),
    "sdc_batch_info": (C.c_int, [_vp, _ip, _ip]),
    "sdc_batch_set_stimulus": (C.c_int, [_vp, C.c_int, _ip, C.c_int, C.c_double, C.c_double,
                                         C.c_double]),
    "sdc_autotune": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_double, C.c_int, C.c_double,
                               C.c_int, C.POINTER(sdc_tune_report)]),
    "sdc_batch_autotune": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_double, C.c_int,
                                     C.c_double, C.c_int, C.POINTER(sdc_tune_report)]),
    "sdc_batch_step": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_double, C.c_int, C.c_double,
                                 C.POINTER(sdc_stats)]),
    "sdc_batch_instance_stats": (C.c_int, [_vp, C.c_int, _ip, _ip]),
    "sdc_batch_context": (_vp, [_vp]),
    "sdc_batch_destroy": (None, [_vp]),
    "sdc_tape_bytes": (C.c_size_t, [_vp, C.c_int]),
    "sdc_step_taped": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_double, C.c_int, C.c_double,
                                 C.POINTER(sdc_stats), C.POINTER(sdc_tape)]),
    "sdc_step_adjoint": (C.c_int, [_vp, C.POINTER(sdc_tape), _vp, _vp, C.c_double, _vp, _vp, _vp,
                                   _vp, _vp, _dp]),
    "sdc_set_dof_scale": (C.c_int, [_vp, _dp]),
    "sdc_set_ionic": (C.c_int, [_vp, C.POINTER(sdc_ionic)]),
    "sdc_set_coarse_blocks": (C.c_int, [_vp, _ip, C.c_int]),
    "sdc_last_error": (C.c_char_p, [_vp]),
    "sdc_status_string": (C.c_char_p, [C.c_int]),
    "sdc_destroy": (None, [_vp]),
}

_lib = None


def load():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsdc_gb300.so is not built (%s); run __graft_entry__.build()"
                               % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class SdcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (load().sdc_status_string(status).decode(), status, message))
        self.status = status


def _check(status, ctx=None):
    if status != SDC_OK:
        msg = load().sdc_last_error(ctx).decode()
        raise SdcError(status, msg)


def default_options(**kw) -> sdc_options:
    o = sdc_options()
    load().sdc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ionic_struct(p: dict) -> sdc_ionic:
    return sdc_ionic(*(float(p[k]) for k in ("ga", "gs", "a", "eps", "mu1", "mu2", "cw")))


def radau(M: int):
    tau, Q, Qh = np.zeros(M), np.zeros((M, M)), np.zeros((M, M))
    _check(load().sdc_radau(M, tau.ctypes.data_as(_dp), Q.ctypes.data_as(_dp),
                            Qh.ctypes.data_as(_dp)))
    return tau, Q, Qh


def _ptr(t):
    """Device pointer of a torch tensor (or an int address)."""
    if isinstance(t, int):
        return t
    return t.data_ptr()


class Context:
    """One sdc_ctx.  Mesh arrays are copied by the library at creation."""

    def __init__(self, dim, xyz, elems, sigma=None, elem_sigma=None, dof_scale=None,
                 ionic=None, M=3, options=None, stream=0, emi=None):
        L = load()
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        elems = np.ascontiguousarray(elems, dtype=np.int32)
        ne, nv = elems.shape
        eptr = np.arange(0, (ne + 1) * nv, nv, dtype=np.int32)
        sig = None if sigma is None else np.ascontiguousarray(np.asarray(sigma).reshape(9), np.float64)
        es = None if elem_sigma is None else np.ascontiguousarray(
            np.asarray(elem_sigma).reshape(-1, 9), np.float64)
        ds = None if dof_scale is None else np.ascontiguousarray(dof_scale, np.float64)
        self._keep = (xyz, elems, eptr, sig, es, ds)
        dp = lambda a: None if a is None else a.ctypes.data_as(_dp)
        mesh = sdc_mesh(dim, xyz.shape[0], dp(xyz), ne, eptr.ctypes.data_as(_ip),
                        elems.ctypes.data_as(_ip), dp(sig), dp(es), dp(ds))
        ion = sdc_ionic()
        if ionic is None:
            L.sdc_default_ionic(C.byref(ion))
        else:
            ion = ionic_struct(ionic)
        opts = options if options is not None else default_options()
        h = _vp()
        self.n_pairs = 0
        if emi is None:
            _check(L.sdc_create(C.byref(h), C.byref(mesh), C.byref(ion), int(M), C.byref(opts),
                                _vp(stream)))
        else:
            pk = np.ascontiguousarray(emi["pair_k"], np.int32)
            pl = np.ascontiguousarray(emi["pair_l"], np.int32)
            pa = np.ascontiguousarray(emi["pair_area"], np.float64)
            pkind = np.ascontiguousarray(emi["pair_kind"], np.int32)
            rb = emi.get("robin")
            rb = None if rb is None else np.ascontiguousarray(rb, np.float64)
            self._keep_emi = (pk, pl, pa, pkind, rb)
            e = sdc_emi(pk.size, pk.ctypes.data_as(_ip), pl.ctypes.data_as(_ip),
                        pa.ctypes.data_as(_dp), pkind.ctypes.data_as(_ip), dp(rb),
                        float(emi["Cm"]), float(emi["g_gap"]))
            _check(L.sdc_create_emi(C.byref(h), C.byref(mesh), C.byref(e), C.byref(ion), int(M),
                                    C.byref(opts), _vp(stream)))
            self.n_pairs = int(pk.size)
        self._h = h
        self.M = int(M)
        self.n = int(xyz.shape[0])
        # the parameters last handed to the library (read back by the autograd
        # driver, which must restore them around its recomputation)
        self.dof_scale = None if ds is None else ds.copy()
        self.ionic = {k: getattr(ion, k) for k, _ in sdc_ionic._fields_}

    @classmethod
    def from_workload(cls, wl, options=None, stream=0):
        ctx = cls(wl.mesh.dim, wl.mesh.xyz, wl.mesh.elems, sigma=wl.sigma,
                  elem_sigma=wl.mesh.elem_sigma, dof_scale=wl.dof_scale, ionic=wl.ionic, M=wl.M,
                  options=options, stream=stream)
        if wl.stim_nodes.size:
            ctx.set_stimulus(wl.stim_nodes, wl.stim_amp, wl.stim_t_on, wl.stim_t_off)
        return ctx

    @classmethod
    def from_emi(cls, wl, options=None, stream=0):
        """Cell-by-cell context of an EMI workload (state: n potentials, n_pairs gating)."""
        emi = dict(pair_k=wl.pair_k, pair_l=wl.pair_l, pair_area=wl.pair_area,
                   pair_kind=wl.pair_kind, robin=wl.robin, Cm=wl.Cm, g_gap=wl.g_gap)
        return cls(wl.mesh.dim, wl.mesh.xyz, wl.mesh.elems, sigma=np.eye(3),
                   elem_sigma=wl.mesh.elem_sigma, ionic=wl.ionic, M=wl.M, options=options,
                   stream=stream, emi=emi)

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.sdc_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stimulus(self, nodes, amp, t_on, t_off):
        nodes = np.ascontiguousarray(nodes, dtype=np.int32)
        _check(load().sdc_set_stimulus(self._h, nodes.ctypes.data_as(_ip), nodes.size, amp,
                                       t_on, t_off), self._h)

    def step(self, v, w, t, dt, sweeps, tol, want_stats=True):
        """One step on device tensors v, w (FP64, n entries each, updated in place)."""
        st = sdc_stats() if want_stats else None
        _check(load().sdc_step(self._h, _vp(_ptr(v)), _vp(_ptr(w)), float(t), float(dt),
                               int(sweeps), float(tol), C.byref(st) if st is not None else None),
               self._h)
        return st

    def autotune(self, v, w, t, dt, sweeps, tol, trial_steps=3):
        """Pick the node solves' launch shape by timing steps from (v, w) (restored)."""
        rep = sdc_tune_report()
        _check(load().sdc_autotune(self._h, _vp(_ptr(v)), _vp(_ptr(w)), float(t), float(dt),
                                   int(sweeps), float(tol), int(trial_steps), C.byref(rep)),
               self._h)
        return rep.as_dict()

    def step_host(self, v, w, t, dt, sweeps, tol, want_stats=False):
        """One step on host numpy arrays v, w (updated in place)."""
        assert v.dtype == np.float64 and w.dtype == np.float64
        assert v.flags.c_contiguous and w.flags.c_contiguous
        st = sdc_stats() if want_stats else None
        _check(load().sdc_step_host(self._h, v.ctypes.data_as(_dp), w.ctypes.data_as(_dp),
                                    float(t), float(dt), int(sweeps), float(tol),
                                    C.byref(st) if st is not None else None), self._h)
        return st

    # ---- differentiation ----------------------------------------------------
    def new_tape(self, sweeps, device):
        """A tape (device buffers owned by torch tensors kept on the object)."""
        import torch
        tp = sdc_tape()
        tp.mode = SDC_TAPE_RECORD
        tp.sweeps = 0
        tp._V = torch.empty(sweeps * self.n * self.M, dtype=torch.float64, device=device)
        tp._W = torch.empty_like(tp._V)
        tp._act = torch.zeros(max(1, sweeps * self.n), dtype=torch.int32, device=device)
        tp.d_V, tp.d_W, tp.d_act = tp._V.data_ptr(), tp._W.data_ptr(), tp._act.data_ptr()
        return tp

    def step_taped(self, v, w, t, dt, sweeps, tol, tape, mode=SDC_TAPE_RECORD, want_stats=False):
        tape.mode = mode
        st = sdc_stats() if want_stats else None
        _check(load().sdc_step_taped(self._h, _vp(_ptr(v)), _vp(_ptr(w)), float(t), float(dt),
                                     int(sweeps), float(tol),
                                     C.byref(st) if st is not None else None, C.byref(tape)),
               self._h)
        return st

    def adjoint(self, tape, v0, w0, dt, lam_v, lam_w, lam_v0, lam_w0, grad_scale=None,
                grad_ionic=None):
        """Adjoint of the step on `tape`; grad_ionic: numpy float64[3] accumulated."""
        gi = grad_ionic.ctypes.data_as(_dp) if grad_ionic is not None else None
        _check(load().sdc_step_adjoint(self._h, C.byref(tape), _vp(_ptr(v0)), _vp(_ptr(w0)),
                                       float(dt), _vp(_ptr(lam_v)), _vp(_ptr(lam_w)),
                                       _vp(_ptr(lam_v0)), _vp(_ptr(lam_w0)),
                                       _vp(_ptr(grad_scale)) if grad_scale is not None else None,
                                       gi), self._h)

    def set_dof_scale(self, scale):
        sc = None if scale is None else np.array(scale, dtype=np.float64, copy=True)
        _check(load().sdc_set_dof_scale(self._h, None if sc is None else sc.ctypes.data_as(_dp)),
               self._h)
        self.dof_scale = sc

    def set_coarse_blocks(self, labels, n_blocks=None):
        """Two-level preconditioner of the cell-by-cell node solves over the given
        block of each dof (None: back to Jacobi)."""
        if labels is None:
            _check(load().sdc_set_coarse_blocks(self._h, None, 0), self._h)
            return
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        nb = int(lab.max()) + 1 if n_blocks is None else int(n_blocks)
        _check(load().sdc_set_coarse_blocks(self._h, lab.ctypes.data_as(_ip), nb), self._h)

    def set_ionic(self, ionic):
        _check(load().sdc_set_ionic(self._h, C.byref(ionic_struct(ionic))), self._h)
        self.ionic = dict(ionic)

    def nodes(self, V, W):
        _check(load().sdc_get_nodes(self._h, _vp(_ptr(V)), _vp(_ptr(W))), self._h)

    def active(self, sweep):
        n = C.c_int(0)
        _check(load().sdc_get_active(self._h, sweep, None, C.byref(n)), self._h)
        out = np.zeros(max(1, n.value), np.int32)
        _check(load().sdc_get_active(self._h, sweep, out.ctypes.data_as(_ip), C.byref(n)), self._h)
        return out[:n.value]

    def info(self):
        n, nnz, w = C.c_int(0), C.c_longlong(0), C.c_int(0)
        _check(load().sdc_get_info(self._h, C.byref(n), C.byref(nnz), C.byref(w)), self._h)
        return n.value, nnz.value, w.value

    def matrix(self):
        n, nnz, _ = self.info()
        rp, ci = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32)
        val, mass = np.zeros(nnz), np.zeros(n)
        _check(load().sdc_get_matrix(self._h, rp.ctypes.data_as(_ip), ci.ctypes.data_as(_ip),
                                     val.ctypes.data_as(_dp), mass.ctypes.data_as(_dp)), self._h)
        return rp, ci, val, mass


def csr_to_ell(rp, ci, val, n):
    """Split a CSR matrix into its diagonal and column-major ELL off-diagonal
    slots (marshalling for sdc_pcg_solve).  Returns kdiag, ell_val, ell_col,
    ell_len, ld, width."""
    rp = np.asarray(rp)
    ci = np.asarray(ci)
    val = np.asarray(val, dtype=np.float64)
    kdiag = np.zeros(n)
    rows = []
    width = 0
    for i in range(n):
        cols = ci[rp[i]:rp[i + 1]]
        vals = val[rp[i]:rp[i + 1]]
        off = cols != i
        kdiag[i] = vals[~off].sum()
        rows.append((cols[off], vals[off]))
        width = max(width, int(off.sum()))
    ld = (n + 31) // 32 * 32
    ev = np.zeros((max(width, 1), ld))
    ec = np.zeros((max(width, 1), ld), dtype=np.int32)
    el = np.zeros(n, dtype=np.int32)
    for i, (cols, vals) in enumerate(rows):
        el[i] = len(cols)
        ev[:len(cols), i] = vals
        ec[:len(cols), i] = cols
    return kdiag, ev, ec, el, ld, width


def pcg_solve(n, ell_val, ell_col, ell_len, ld, width, kdiag, mass, J, c, b, x, rtol=1e-10,
              maxit=10000, stream=0):
    """sdc_pcg_solve on device tensors (or integer device addresses)."""
    it = C.c_int(0)
    rr = C.c_double(0.0)
    _check(load().sdc_pcg_solve(int(n), _vp(_ptr(ell_val)), _vp(_ptr(ell_col)), _vp(_ptr(ell_len)),
                                int(ld), int(width), _vp(_ptr(kdiag)), _vp(_ptr(mass)),
                                _vp(_ptr(J)), float(c), _vp(_ptr(b)), _vp(_ptr(x)), float(rtol),
                                int(maxit), C.byref(it), C.byref(rr), _vp(stream)))
    return it.value, rr.value


def pcg_solve_noalloc(n, ell_val, ell_col, ell_len, ld, width, kdiag, mass, J, c, b, x,
                      rtol=1e-10, maxit=10000, stream=0):
    """sdc_pcg_solve_noalloc: the same solve, workspace in the library's static
    device array (no device allocation; n <= SDC_PCG_NOALLOC_MAX_ROWS; calls
    that overlap on the GPU race)."""
    it = C.c_int(0)
    rr = C.c_double(0.0)
    _check(load().sdc_pcg_solve_noalloc(int(n), _vp(_ptr(ell_val)), _vp(_ptr(ell_col)),
                                        _vp(_ptr(ell_len)), int(ld), int(width), _vp(_ptr(kdiag)),
                                        _vp(_ptr(mass)), _vp(_ptr(J)), float(c), _vp(_ptr(b)),
                                        _vp(_ptr(x)), float(rtol), int(maxit), C.byref(it),
                                        C.byref(rr), _vp(stream)))
    return it.value, rr.value


class Batch:
    """One sdc_batch: instances stacked as disjoint diagonal blocks."""

    def __init__(self, workloads, options=None, stream=0):
        L = load()
        wl0 = workloads[0]
        keep = []
        meshes = (sdc_mesh * len(workloads))()
        for b, wl in enumerate(workloads):
            if wl.M != wl0.M or wl.ionic != wl0.ionic:
                raise ValueError("batch instances share M and the ionic parameters")
            xyz = np.ascontiguousarray(wl.mesh.xyz, dtype=np.float64)
            el = np.ascontiguousarray(wl.mesh.elems, dtype=np.int32)
            ne, nv = el.shape
            ep = np.arange(0, (ne + 1) * nv, nv, dtype=np.int32)
            sig = np.ascontiguousarray(np.asarray(wl.sigma).reshape(9), np.float64)
            es = None if wl.mesh.elem_sigma is None else np.ascontiguousarray(
                wl.mesh.elem_sigma.reshape(-1, 9), np.float64)
            ds = None if wl.dof_scale is None else np.ascontiguousarray(wl.dof_scale, np.float64)
            keep.append((xyz, el, ep, sig, es, ds))
            dp = lambda a: None if a is None else a.ctypes.data_as(_dp)
            meshes[b] = sdc_mesh(wl.mesh.dim, xyz.shape[0], dp(xyz), ne, ep.ctypes.data_as(_ip),
                                 el.ctypes.data_as(_ip), dp(sig), dp(es), dp(ds))
        opts = options if options is not None else default_options()
        h = _vp()
        _check(L.sdc_batch_create(C.byref(h), meshes, len(workloads), C.byref(ionic_struct(wl0.ionic)),
                                  wl0.M, C.byref(opts), _vp(stream)))
        self._h = h
        self.M = wl0.M
        self.count = len(workloads)
        off = np.zeros(self.count + 1, np.int32)
        _check(L.sdc_batch_info(self._h, None, off.ctypes.data_as(_ip)))
        self.offsets = off
        self.n = int(off[-1])
        for b, wl in enumerate(workloads):
            if wl.stim_nodes.size:
                nodes = np.ascontiguousarray(wl.stim_nodes, np.int32)
                _check(L.sdc_batch_set_stimulus(self._h, b, nodes.ctypes.data_as(_ip), nodes.size,
                                                wl.stim_amp, wl.stim_t_on, wl.stim_t_off),
                       L.sdc_batch_context(self._h))

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.sdc_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, v, w, t, dt, sweeps, tol):
        st = sdc_stats()
        _check(load().sdc_batch_step(self._h, _vp(_ptr(v)), _vp(_ptr(w)), float(t), float(dt),
                                     int(sweeps), float(tol), C.byref(st)),
               load().sdc_batch_context(self._h))
        return st

    def autotune(self, v, w, t, dt, sweeps, tol, trial_steps=3):
        """Pick the batched solves' launch shape by timing steps from (v, w) (restored)."""
        rep = sdc_tune_report()
        _check(load().sdc_batch_autotune(self._h, _vp(_ptr(v)), _vp(_ptr(w)), float(t),
                                         float(dt), int(sweeps), float(tol), int(trial_steps),
                                         C.byref(rep)),
               load().sdc_batch_context(self._h))
        return rep.as_dict()

    def instance_stats(self, sweep):
        na = np.zeros(self.count, np.int32)
        it = np.zeros((self.M, self.count), np.int32)
        _check(load().sdc_batch_instance_stats(self._h, sweep, na.ctypes.data_as(_ip),
                                               it.ctypes.data_as(_ip)),
               load().sdc_batch_context(self._h))
        return na, it

    def active(self, sweep):
        """Active list of the stacked system for a sweep of the last step."""
        ctx = load().sdc_batch_context(self._h)
        n = C.c_int(0)
        _check(load().sdc_get_active(ctx, sweep, None, C.byref(n)), ctx)
        out = np.zeros(max(1, n.value), np.int32)
        _check(load().sdc_get_active(ctx, sweep, out.ctypes.data_as(_ip), C.byref(n)), ctx)
        return out[:n.value]
