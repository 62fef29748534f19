"""Thin ctypes binding of the C ABI in include/richards.h (argument marshalling only).

Device buffers are torch CUDA tensors (float64, contiguous); the binding passes
their data pointers and the current torch CUDA stream.  Every numerical step
runs in the CUDA library; when the library is missing the binding raises.
"""
import ctypes
import os

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librichards_gb300.so")

RICH_OK = 0
KRYLOV_FCG, KRYLOV_FGMRES = 0, 1
AMG_REFRESH, AMG_SETUP_ONCE, AMG_REBUILD_STEP = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
AGG_MIS2, AGG_MATCHING = 0, 1
SMOOTH_L1JACOBI, SMOOTH_HYBRID_GS = 0, 1
PRECOND_AMG, PRECOND_AS = 0, 1
BC_NOFLUX, BC_DIRICHLET, BC_INTERFACE = 0, 1, 2
LAYOUT_AUTO, LAYOUT_CSR, LAYOUT_SELL, LAYOUT_SELL8, LAYOUT_SELL2, LAYOUT_SELLP = 0, 1, 2, 3, 4, 5
UNROLL, SELL_VARIANT, SELL_VARIANT8, SELL_VARIANT2, SELL_VARIANTP = 0x100, 0x200, 0x201, 0x202, 0x203

ERRORS = {-1: "RICH_EINVAL", -2: "RICH_ENOMEM", -3: "RICH_ECUDA", -4: "RICH_ENOTCONV_LIN",
          -5: "RICH_ENOTCONV_NEWTON", -6: "RICH_ELINESEARCH", -7: "RICH_ENONFINITE", -8: "RICH_ESTATE",
          -9: "RICH_ELIMIT", -10: "RICH_EBUSY"}
RICH_EBUSY = -10


class RichError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (%d)%s" % (what, ERRORS.get(status, "?"), status,
                                                   (" [" + _last_cuda() + "]") if status == -3 else ""))


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("h", ctypes.c_double * 3)]


def _grid_struct(grid):
    """ctypes Grid of a synth.Grid (its explicit spacing, if it has one)."""
    sp = getattr(grid, "spacing", None)
    return Grid(grid.nx, grid.ny, grid.nz, grid.lx, grid.ly, grid.lz, (ctypes.c_double * 3)(*(sp or (0.0, 0.0, 0.0))))


class Soil(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("theta_s", ctypes.c_double),
                ("theta_r", ctypes.c_double), ("a", ctypes.c_double), ("gamma", ctypes.c_double),
                ("ks_const", ctypes.c_double), ("rho_phi", ctypes.c_double), ("ks_field_dev", ctypes.c_void_p)]


class BC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 6), ("value", ctypes.c_double * 6), ("value_field_dev", ctypes.c_void_p * 6),
                ("ghost_ks_dev", ctypes.c_void_p * 6)]


def _bc_struct(bc, keep):
    """ctypes BC; per-face value arrays (and the ghost K_s of interface faces) are
    uploaded to device tensors kept in `keep`."""
    import torch

    def upload(arr):
        if arr is None:
            return None
        t = torch.as_tensor(arr, dtype=torch.float64).reshape(-1).cuda().contiguous()
        keep.append(t)
        return t.data_ptr()

    ptrs = [upload(bc.field(f) if hasattr(bc, "field") else None) for f in range(6)]
    gks = [upload(bc.ghost_ks_field(f) if hasattr(bc, "ghost_ks_field") else None) for f in range(6)]
    return BC((ctypes.c_int * 6)(*bc.kind), (ctypes.c_double * 6)(*bc.value), (ctypes.c_void_p * 6)(*ptrs),
              (ctypes.c_void_p * 6)(*gks))


class AmgOpts(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("seed", ctypes.c_uint64), ("coarse_max", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("smooth_levels", ctypes.c_int), ("product_lists", ctypes.c_int), ("aggregation", ctypes.c_int),
                ("max_agg_size", ctypes.c_int), ("smoother", ctypes.c_int), ("hgs_seg", ctypes.c_int),
                ("hgs_block", ctypes.c_int), ("precond", ctypes.c_int), ("as_block", ctypes.c_int),
                ("as_overlap", ctypes.c_int), ("autotune", ctypes.c_int), ("isolated_join", ctypes.c_int),
                ("csr_layout", ctypes.c_int), ("graph", ctypes.c_int)]


class KrylovOpts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("restart", ctypes.c_int), ("eta", ctypes.c_double),
                ("maxit", ctypes.c_int), ("stall", ctypes.c_double)]


class KrylovStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double)]


class NewtonOpts(ctypes.Structure):
    _fields_ = [("krylov", KrylovOpts), ("amg", AmgOpts), ("amg_policy", ctypes.c_int), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("max_newton", ctypes.c_int), ("armijo_c", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("fcg_fallback_restart", ctypes.c_int),
                ("max_dt_halvings", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("linear_its", ctypes.c_int), ("line_search_evals", ctypes.c_int),
                ("fallbacks", ctypes.c_int), ("amg_setups", ctypes.c_int), ("amg_refreshes", ctypes.c_int),
                ("converged", ctypes.c_int), ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("min_lambda", ctypes.c_double), ("ms_feval", ctypes.c_double), ("ms_jacobian", ctypes.c_double),
                ("ms_setup", ctypes.c_double), ("ms_linsol", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("substeps", ctypes.c_int), ("dt_failures", ctypes.c_int), ("dt_min", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("mem_budget_bytes", ctypes.c_double), ("max_sessions", ctypes.c_int),
                ("batch_max", ctypes.c_int), ("batch_min_cells", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("grid", Grid), ("soil", Soil), ("ks_field_host", ctypes.c_void_p), ("kmean", ctypes.c_int),
                ("bc", BC), ("precision", ctypes.c_int), ("dt", ctypes.c_double), ("opts", NewtonOpts),
                ("p0_host", ctypes.c_void_p), ("p_out_host", ctypes.c_void_p), ("session", ctypes.c_longlong)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("stats", StepStats), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("slot", ctypes.c_int),
                ("mem_estimate", ctypes.c_double), ("mem_in_flight", ctypes.c_double), ("batch_size", ctypes.c_int),
                ("batch_rerun", ctypes.c_int)]


class AmgInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("n", ctypes.c_int * 16), ("nnz", ctypes.c_longlong * 16),
                ("mis_rounds", ctypes.c_int * 16), ("omega", ctypes.c_double * 16),
                ("operator_complexity", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
EXPORTS = {
    "rich_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Soil), ctypes.c_int, ctypes.POINTER(BC),
                                   ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "rich_destroy": (ctypes.c_int, [_P]),
    "rich_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rich_last_cuda_error": (ctypes.c_char_p, []),
    "rich_num_cells": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "rich_saturation": (ctypes.c_int, [_P, _P, _P]),
    "rich_residual": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_double)]),
    "rich_residual3": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_double)]),
    "rich_residual_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Soil), ctypes.c_int,
                                             ctypes.POINTER(BC), _P, _P, ctypes.c_double, _P,
                                             ctypes.POINTER(ctypes.c_double), _P]),
    "rich_kernel_launches": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong)]),
    "rich_measure_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "rich_autotune_table": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int]),
    "rich_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "rich_set_face_values": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "rich_pack_face": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "rich_face_apply": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "rich_vec_dot": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "rich_vec_axpby": (ctypes.c_int, [_P, ctypes.c_double, _P, ctypes.c_double, _P]),
    "rich_sell_layout": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_longlong)]),
    "rich_profile_kernel": (ctypes.c_int, [ctypes.c_char_p]),
    "rich_profile_result": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "rich_profile_table": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int]),
    "rich_profile_stride": (ctypes.c_int, [ctypes.c_int]),
    "rich_memory_peak": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.c_int]),
    "rich_jacobian": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P]),
    "rich_jacobian_apply": (ctypes.c_int, [_P, _P, _P]),
    "amg_setup": (ctypes.c_int, [_P, ctypes.POINTER(AmgOpts), ctypes.POINTER(AmgInfo)]),
    "amg_update": (ctypes.c_int, [_P, ctypes.c_int]),
    "amg_vcycle": (ctypes.c_int, [_P, _P, _P]),
    "amg_export_level": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "amg_export_prolongator": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _P, _P, _P]),
    "krylov_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(KrylovOpts), ctypes.POINTER(KrylovStats)]),
    "rich_step": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.POINTER(NewtonOpts), ctypes.POINTER(StepStats)]),
    "rich_step_host": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.POINTER(NewtonOpts),
                                      ctypes.POINTER(StepStats)]),
    "rich_create_batch": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(Soil), ctypes.c_int,
                                         ctypes.POINTER(BC), ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "rich_step_batch": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.POINTER(NewtonOpts), ctypes.POINTER(StepStats),
                                       ctypes.POINTER(ctypes.c_int)]),
    "rich_default_newton_opts": (None, [ctypes.POINTER(NewtonOpts)]),
    "rich_default_amg_opts": (None, [ctypes.POINTER(AmgOpts)]),
    "rich_default_server_opts": (None, [ctypes.POINTER(ServerOpts)]),
    "rich_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(_P)]),
    "rich_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]),
    "rich_server_poll": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.POINTER(RequestResult)]),
    "rich_server_wait": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.POINTER(RequestResult)]),
    "rich_server_drain": (ctypes.c_int, [_P]),
    "rich_server_counters": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_double)]),
    "rich_server_destroy": (ctypes.c_int, [_P]),
}


def load():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librichards_gb300.so is missing: run __graft_entry__.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _last_cuda():
    try:
        return load().rich_last_cuda_error().decode()
    except Exception:  # pragma: no cover
        return ""


def check(status, what):
    if status != RICH_OK:
        raise RichError(status, what)


def _ptr(t):
    if t is None:
        return None
    assert t.is_contiguous(), "tensor must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_newton_opts(**kw):
    o = NewtonOpts()
    load().rich_default_newton_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("kind", "restart", "eta", "maxit", "stall"):
            setattr(o.krylov, k, v)
        elif k in ("theta", "seed", "coarse_max", "max_levels", "nu1", "nu2", "smooth_levels", "product_lists",
                   "aggregation", "max_agg_size", "isolated_join", "smoother", "hgs_seg", "hgs_block",
                   "autotune", "precond", "as_block", "as_overlap", "csr_layout", "graph"):
            setattr(o.amg, k, v)
        else:
            setattr(o, k, v)
    return o


def default_amg_opts(**kw):
    o = AmgOpts()
    load().rich_default_amg_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def residual_noalloc(grid, soil, bc, kmean, p, s_old, dt, F, ks=None, norms=True):
    """Phi(p) through rich_residual_noalloc (no context, no device allocation by the library).

    ks, if given, must be a contiguous float64 CUDA tensor of n cells (read in place).
    Returns the status code and (||Phi||_2, ||Phi||_inf) or None.
    """
    g = _grid_struct(grid)
    s = Soil(soil.alpha, soil.beta, soil.theta_s, soil.theta_r, soil.a, soil.gamma, soil.ks, soil.rho_phi,
             _ptr(ks) if ks is not None else None)
    keep = []
    b = _bc_struct(bc, keep)
    arr = (ctypes.c_double * 2)() if norms else None
    st = load().rich_residual_noalloc(ctypes.byref(g), ctypes.byref(s), kmean, ctypes.byref(b), _ptr(p),
                                      _ptr(s_old), dt, _ptr(F), arr, _stream())
    return st, ((arr[0], arr[1]) if norms else None)


def profile_table():
    """Per-kernel totals recorded under the "*" profiling target: {name: (launches, ms, bytes, flops)}."""
    buf = ctypes.create_string_buffer(1 << 16)
    check(load().rich_profile_table(buf, len(buf)), "rich_profile_table")
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms, b, f = line.split()
        out[name] = (int(n), float(ms), float(b), float(f))
    return out


class Context:
    """A solver context on the current CUDA device (wraps rich_create/rich_destroy)."""

    def __init__(self, grid: synth.Grid, soil: synth.Soil, bc: synth.BC, kmean: int, ks=None,
                 precision=PREC_FP64):
        import torch
        lib = load()
        g = _grid_struct(grid)
        self._ks = None
        if ks is not None:
            self._ks = torch.as_tensor(ks, dtype=torch.float64).reshape(-1).cuda().contiguous()
        s = Soil(soil.alpha, soil.beta, soil.theta_s, soil.theta_r, soil.a, soil.gamma, soil.ks, soil.rho_phi,
                 _ptr(self._ks) if self._ks is not None else None)
        self._bc_keep = []
        b = _bc_struct(bc, self._bc_keep)
        h = ctypes.c_void_p()
        check(lib.rich_create(ctypes.byref(g), ctypes.byref(s), kmean, ctypes.byref(b), precision, _stream(),
                              ctypes.byref(h)), "rich_create")
        self.h = h
        self.n = grid.n
        self.grid = grid

    def close(self):
        if getattr(self, "h", None):
            load().rich_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def saturation(self, p, s):
        check(load().rich_saturation(self.h, _ptr(p), _ptr(s)), "rich_saturation")

    def pack_face(self, face, field, out):
        """out = the cells of `field` next to face `face`, in the face layout (device)."""
        check(load().rich_pack_face(self.h, face, _ptr(field), _ptr(out)), "rich_pack_face")

    def dot(self, x, y):
        """x . y over the context's cells (device vectors)."""
        out = ctypes.c_double()
        check(load().rich_vec_dot(self.h, _ptr(x), _ptr(y), ctypes.byref(out)), "rich_vec_dot")
        return out.value

    def axpby(self, a, x, b, y):
        """y = a x + b y (y = a x when b == 0)."""
        check(load().rich_vec_axpby(self.h, a, _ptr(x), b, _ptr(y)), "rich_vec_axpby")

    def face_apply(self, face, which, ghost, y):
        """y += (J if which == 0 else A_aux) coupling of interface face `face` times ghost."""
        check(load().rich_face_apply(self.h, face, which, _ptr(ghost), _ptr(y)), "rich_face_apply")

    def set_face_values(self, face, values):
        """Per-cell values of a face created with a field (Dirichlet values, or the
        ghost pressures of an interface face), from a float64 CUDA tensor."""
        check(load().rich_set_face_values(self.h, face, _ptr(values)), "rich_set_face_values")

    def residual(self, p, s_old, dt, F, norms=True):
        arr = (ctypes.c_double * 2)() if norms else None
        check(load().rich_residual(self.h, _ptr(p), _ptr(s_old), dt, _ptr(F), arr), "rich_residual")
        return (arr[0], arr[1]) if norms else None

    def residual3(self, p, s_old, dt, F):
        """Phi into F; returns (||Phi||_2, ||Phi||_inf, ||m||_2), eps ||m||_2 being the
        accuracy of Phi (the Newton test's round-off floor)."""
        arr = (ctypes.c_double * 3)()
        check(load().rich_residual3(self.h, _ptr(p), _ptr(s_old), dt, _ptr(F), arr), "rich_residual3")
        return arr[0], arr[1], arr[2]

    def jacobian(self, p, dt, J7=None, A7=None):
        check(load().rich_jacobian(self.h, _ptr(p), dt, _ptr(J7), _ptr(A7)), "rich_jacobian")

    def jacobian_apply(self, x, y):
        check(load().rich_jacobian_apply(self.h, _ptr(x), _ptr(y)), "rich_jacobian_apply")

    def amg_setup(self, opts=None):
        info = AmgInfo()
        check(load().amg_setup(self.h, ctypes.byref(opts) if opts is not None else None, ctypes.byref(info)),
              "amg_setup")
        return info

    def amg_update(self, policy=AMG_REFRESH):
        check(load().amg_update(self.h, policy), "amg_update")

    def vcycle(self, r, z):
        check(load().amg_vcycle(self.h, _ptr(r), _ptr(z)), "amg_vcycle")

    def export_level(self, level, info):
        import numpy as np
        n = info.n[level]
        nnz = info.nnz[level]
        agg = np.zeros(n, dtype=np.int32) if level < info.levels - 1 else None
        rp = np.zeros(n + 1, dtype=np.int32)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz, dtype=np.float64)
        cp = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
        check(load().amg_export_level(self.h, level, cp(agg), cp(rp), cp(col), cp(val)), "amg_export_level")
        return agg, rp, col, val

    def export_prolongator(self, level, info):
        import numpy as np
        nnz = ctypes.c_longlong()
        check(load().amg_export_prolongator(self.h, level, ctypes.byref(nnz), None, None, None),
              "amg_export_prolongator")
        rp = np.zeros(info.n[level] + 1, dtype=np.int32)
        col = np.zeros(nnz.value, dtype=np.int32)
        val = np.zeros(nnz.value, dtype=np.float64)
        cp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        check(load().amg_export_prolongator(self.h, level, ctypes.byref(nnz), cp(rp), cp(col), cp(val)),
              "amg_export_prolongator")
        return rp, col, val

    def krylov_solve(self, b, x, kind=KRYLOV_FCG, restart=30, eta=1e-7, maxit=200, check_status=True, stall=0.0):
        o = KrylovOpts(kind, restart, eta, maxit, stall)
        st = KrylovStats()
        s = load().krylov_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(st))
        if check_status:
            check(s, "krylov_solve")
        return s, st

    def step(self, p, dt, opts=None, check_status=True):
        """One backward-Euler step; returns the step statistics (and, with
        check_status=False, the status code first instead of raising on failure)."""
        st = StepStats()
        s = load().rich_step(self.h, _ptr(p), dt, ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
        if not check_status:
            return s, st
        check(s, "rich_step")
        return st

    def step_host(self, p_host, dt, opts=None):
        """p_host: numpy float64 array or pinned CPU tensor (updated in place)."""
        st = StepStats()
        if hasattr(p_host, "data_ptr"):
            ptr = ctypes.c_void_p(p_host.data_ptr())
        else:
            ptr = p_host.ctypes.data_as(ctypes.c_void_p)
        check(load().rich_step_host(self.h, ptr, dt, ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(st)), "rich_step_host")
        return st


class BatchContext(Context):
    """nbatch problems of one grid stacked along z (rich_create_batch / rich_step_batch).

    ks: None or an (nbatch * n) array of K_s values, problem b at [b n, (b+1) n)."""

    def __init__(self, grid: synth.Grid, nbatch: int, soil: synth.Soil, bc: synth.BC, kmean: int, ks=None,
                 precision=PREC_MIXED):
        import torch
        lib = load()
        g = _grid_struct(grid)
        self._ks = None
        if ks is not None:
            self._ks = torch.as_tensor(ks, dtype=torch.float64).reshape(-1).cuda().contiguous()
        s = Soil(soil.alpha, soil.beta, soil.theta_s, soil.theta_r, soil.a, soil.gamma, soil.ks, soil.rho_phi,
                 _ptr(self._ks) if self._ks is not None else None)
        self._bc_keep = []
        b = _bc_struct(bc, self._bc_keep)
        h = ctypes.c_void_p()
        check(lib.rich_create_batch(ctypes.byref(g), nbatch, ctypes.byref(s), kmean, ctypes.byref(b), precision,
                                    _stream(), ctypes.byref(h)), "rich_create_batch")
        self.h = h
        self.nbatch = nbatch
        self.n = grid.n * nbatch
        self.grid = grid

    def step_batch(self, p, dt, opts=None):
        """Returns ([status per problem], [StepStats per problem])."""
        st = (StepStats * self.nbatch)()
        status = (ctypes.c_int * self.nbatch)()
        check(load().rich_step_batch(self.h, _ptr(p), dt, ctypes.byref(opts) if opts is not None else None, st,
                                     status), "rich_step_batch")
        return list(status), list(st)


def default_server_opts(**kw):
    o = ServerOpts()
    load().rich_default_server_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Server:
    """Request server (rich_server_*): time-step solves of any size, several in flight at once.

    submit() takes host numpy arrays (float64); they stay referenced until the
    request's result has been collected with wait() or poll().  A result holds
    the step's status and statistics, host timestamps (seconds since the server
    started) and the output pressure (after a failed step: the last accepted
    Newton iterate).
    """

    def __init__(self, slots=8, mem_budget_bytes=0.0, max_sessions=64, batch_max=1):
        self._lib = load()
        self.h = ctypes.c_void_p()
        o = default_server_opts(slots=slots, mem_budget_bytes=float(mem_budget_bytes), max_sessions=max_sessions,
                                batch_max=batch_max)
        check(self._lib.rich_server_create(ctypes.byref(o), ctypes.byref(self.h)), "rich_server_create")
        self._keep = {}

    def submit(self, grid, soil, bc, kmean, dt, p0=None, ks=None, precision=PREC_MIXED, opts=None, session=0,
               want_output=True):
        import numpy as np
        if any(bc.field(f) is not None for f in range(6)):
            raise ValueError("the request server takes constant boundary values only")
        r = Request()
        r.grid = _grid_struct(grid)
        r.soil = Soil(soil.alpha, soil.beta, soil.theta_s, soil.theta_r, soil.a, soil.gamma, soil.ks, soil.rho_phi,
                      None)
        keep = []
        if ks is not None:
            ks = np.ascontiguousarray(ks, dtype=np.float64)
            keep.append(ks)
            r.ks_field_host = ks.ctypes.data
        r.kmean = kmean
        r.bc = BC((ctypes.c_int * 6)(*bc.kind), (ctypes.c_double * 6)(*bc.value), (ctypes.c_void_p * 6)())
        r.precision = precision
        r.dt = dt
        r.opts = opts if opts is not None else default_newton_opts()
        if p0 is not None:
            p0 = np.ascontiguousarray(p0, dtype=np.float64)
            keep.append(p0)
            r.p0_host = p0.ctypes.data
        out = None
        if want_output:
            out = np.full(grid.n, np.nan)
            keep.append(out)
            r.p_out_host = out.ctypes.data
        r.session = session
        rid = ctypes.c_longlong()
        check(self._lib.rich_server_submit(self.h, ctypes.byref(r), ctypes.byref(rid)), "rich_server_submit")
        self._keep[rid.value] = (keep, out)
        return rid.value

    def _result(self, rid, res):
        keep, out = self._keep.pop(rid)
        return {"status": res.status, "stats": res.stats.as_dict(), "t_submit": res.t_submit,
                "t_admit": res.t_admit, "t_done": res.t_done, "slot": res.slot, "mem_estimate": res.mem_estimate,
                "mem_in_flight": res.mem_in_flight, "batch_size": res.batch_size, "batch_rerun": res.batch_rerun,
                "p": out}

    def wait(self, rid):
        res = RequestResult()
        check(self._lib.rich_server_wait(self.h, rid, ctypes.byref(res)), "rich_server_wait")
        return self._result(rid, res)

    def poll(self, rid):
        res = RequestResult()
        st = self._lib.rich_server_poll(self.h, rid, ctypes.byref(res))
        if st == RICH_EBUSY:
            return None
        check(st, "rich_server_poll")
        return self._result(rid, res)

    def drain(self):
        check(self._lib.rich_server_drain(self.h), "rich_server_drain")

    def counters(self):
        a = ctypes.c_longlong()
        m = ctypes.c_int()
        b = ctypes.c_double()
        check(self._lib.rich_server_counters(self.h, ctypes.byref(a), ctypes.byref(m), ctypes.byref(b)),
              "rich_server_counters")
        return {"admitted": a.value, "max_in_flight": m.value, "reserved_bytes": b.value}

    def close(self):
        if self.h:
            self._lib.rich_server_destroy(self.h)
            self.h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def memory_peak(reset=False):
    """(bytes in use, bytes reserved) high-water marks of the library's device memory pool."""
    u = ctypes.c_longlong()
    r = ctypes.c_longlong()
    check(load().rich_memory_peak(ctypes.byref(u), ctypes.byref(r), 1 if reset else 0), "rich_memory_peak")
    return u.value, r.value


def fma_peak_tflops(fp64=True):
    """Measured FP64 (or FP32) FMA peak of the current device, TFLOP/s."""
    v = ctypes.c_double()
    check(load().rich_measure_fma_peak(1 if fp64 else 0, ctypes.byref(v)), "rich_measure_fma_peak")
    return v.value


def autotune_table():
    """The row-operation autotuner's choices:
    [(mode, value_bytes, rows_bin, mean_row_length, sell_offered, variant, best_us)],
    variant = lanes per row (+ UNROLL for four-way unrolled rows) or SELL_VARIANT."""
    out = []
    for line in autotune_text().splitlines():
        m, t, n, z, so, g, us, _ = line.split()
        out.append((int(m), int(t), int(n), int(z), int(so), int(g), float(us)))
    return out


def sell_layout(rowptr):
    """The SELL-C-sigma layout of a CSR row pointer (host): (perm, sptr, slots)."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    n = len(rp) - 1
    ns = (n + 31) // 32
    perm = np.empty(32 * ns, dtype=np.int32)
    sptr = np.empty(ns + 1, dtype=np.int32)
    slots = ctypes.c_longlong()
    cp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    check(load().rich_sell_layout(cp(rp), n, cp(perm), cp(sptr), ctypes.byref(slots)), "rich_sell_layout")
    return perm, sptr, slots.value


def autotune_text():
    """The autotuner's table as text (rich_autotune_table), for saving."""
    buf = ctypes.create_string_buffer(1 << 16)
    check(load().rich_autotune_table(buf, len(buf)), "rich_autotune_table")
    return buf.value.decode()


def autotune_load(text):
    """Adds a saved table (autotune_text) to the process's autotuner."""
    check(load().rich_autotune_load(text.encode()), "rich_autotune_load")
