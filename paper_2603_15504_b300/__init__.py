"""Python binding of the PDCS C ABI (include/pdcs.h): argument marshalling only.

Every computation runs in libpdcs.so (hand-written CUDA for sm_103a).  Arrays
may be NumPy arrays (host) or CUDA torch tensors (device); the library detects
the pointer kind.  There is no CPU fallback: if the library or a GPU is missing
the calls raise.
"""
import ctypes
import os

import numpy as np

from .build import LIB, build  # noqa: F401

CONE_ZERO, CONE_NONNEG, CONE_SOC, CONE_RSOC, CONE_EXP, CONE_DUAL_EXP = 0, 1, 2, 3, 4, 5
TRACE_FIELDS = 13
TRACE_NAMES = ("iter", "kbar", "period", "eta", "eta_hat", "beta", "omega", "max_err", "check",
               "cand_avg", "restart", "rho_c", "fallback")
EXIT_NAMES = {0: "optimal", 1: "max_iter", 2: "primal_infeasible_low_acc",
              3: "primal_infeasible_high_acc", 4: "dual_infeasible_low_acc",
              5: "dual_infeasible_high_acc", 6: "time_limit", 7: "continue",
              8: "numerical_error"}


class PdcsCone(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("pad", ctypes.c_int32), ("dim", ctypes.c_int64)]


class PdcsOptions(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("time_limit", ctypes.c_double), ("max_iter", ctypes.c_int64),
                ("use_preconditioner", ctypes.c_int32), ("ruiz_iters", ctypes.c_int32),
                ("pc_alpha", ctypes.c_double), ("method", ctypes.c_int32),
                ("use_adaptive_restart", ctypes.c_int32), ("check_freq", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("require_abs", ctypes.c_int32),
                ("bisect_rel_tol", ctypes.c_double), ("verbose", ctypes.c_int32),
                ("trace_capacity", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("eager", ctypes.c_int32), ("use_adaptive_step_size_weight", ctypes.c_int32),
                ("use_duality_gap_restart", ctypes.c_int32), ("use_kkt_restart", ctypes.c_int32),
                ("overlap_launches", ctypes.c_int32), ("kkt_restart_freq", ctypes.c_int64),
                ("print_freq", ctypes.c_int64),
                ("eps_primal_infeasible_low_acc", ctypes.c_double),
                ("eps_dual_infeasible_low_acc", ctypes.c_double),
                ("eps_primal_infeasible_high_acc", ctypes.c_double),
                ("eps_dual_infeasible_high_acc", ctypes.c_double)]


class PdcsResult(ctypes.Structure):
    _fields_ = [("exit_code", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("pobj", ctypes.c_double), ("dobj", ctypes.c_double),
                ("err_rel_p", ctypes.c_double), ("err_rel_d", ctypes.c_double),
                ("err_rel_gap", ctypes.c_double), ("err_abs_p", ctypes.c_double),
                ("err_abs_d", ctypes.c_double), ("err_abs_gap", ctypes.c_double),
                ("solve_time_s", ctypes.c_double), ("iters", ctypes.c_int64),
                ("attempts", ctypes.c_int64), ("restarts", ctypes.c_int64)]


class PdcsInstance(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("h", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("nb", ctypes.c_int64), ("lb", ctypes.c_void_p),
                ("ub", ctypes.c_void_p), ("row_cones", ctypes.c_void_p),
                ("n_row_cones", ctypes.c_int64), ("col_cones", ctypes.c_void_p),
                ("n_col_cones", ctypes.c_int64)]


class PdcsMlpConfig(ctypes.Structure):
    _fields_ = [("in_dim", ctypes.c_int64), ("hidden", ctypes.c_int64),
                ("n_hidden", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("out_dim", ctypes.c_int64), ("max_batch", ctypes.c_int64),
                ("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("seed", ctypes.c_uint64)]


class PdcsState(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int64), ("kbar", ctypes.c_int64), ("k", ctypes.c_int64),
                ("period", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("eta_hat", ctypes.c_double), ("eta_last", ctypes.c_double),
                ("omega", ctypes.c_double), ("wsum", ctypes.c_double),
                ("has_ref", ctypes.c_int32), ("has_prev", ctypes.c_int32),
                ("ref_rho", ctypes.c_double), ("ref_abs_p", ctypes.c_double),
                ("ref_abs_d", ctypes.c_double), ("ref_abs_gap", ctypes.c_double),
                ("prev_rho", ctypes.c_double), ("prev_abs_p", ctypes.c_double),
                ("prev_abs_d", ctypes.c_double), ("prev_abs_gap", ctypes.c_double)]


class PdcsProfile(ctypes.Structure):
    _fields_ = [("g_launches", ctypes.c_int64), ("g_seconds", ctypes.c_double),
                ("g_bytes", ctypes.c_double), ("gt_launches", ctypes.c_int64),
                ("gt_seconds", ctypes.c_double), ("gt_bytes", ctypes.c_double),
                ("nnz_flops", ctypes.c_double), ("graph_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64)]


KERNEL_CLASSES = ("spmv_g", "spmv_gt", "spmv_check", "soc_grid", "soc_cta", "exp", "primal", "dual",
                  "step", "res_prep", "stats_attempt", "stats_check", "halpern", "probe_prep",
                  "probe_reduce", "check_misc")

EXPORTS = ("pdcs_default_options", "pdcs_setup", "pdcs_solve", "pdcs_resume", "pdcs_get_state",
           "pdcs_set_state", "pdcs_get_iterate", "pdcs_get_trace", "pdcs_get_profile",
           "pdcs_get_kernel_times", "pdcs_get_sizes", "pdcs_free", "pdcs_last_error",
           "pdcs_mlp_default_config", "pdcs_mlp_create", "pdcs_mlp_train_step",
           "pdcs_mlp_gradients", "pdcs_mlp_predict", "pdcs_mlp_get_layer", "pdcs_mlp_set_layer",
           "pdcs_mlp_free", "pdcs_kkt", "pdcs_setup_batch", "pdcs_solve_batch",
           "pdcs_spmv_noalloc", "pdcs_spmv_noalloc_status")

_LIB = None


def lib():
    """Load libpdcs.so (building it first if it is missing or stale, unless
    PDCS_AUTOBUILD=0)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if os.environ.get("PDCS_AUTOBUILD", "1") == "1" or not os.path.exists(LIB):
        try:
            build()
        except Exception as e:  # noqa: BLE001
            if not os.path.exists(LIB):
                raise RuntimeError("libpdcs.so is missing and could not be built: %s" % e)
    L = ctypes.CDLL(LIB)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.pdcs_default_options.argtypes = [ctypes.POINTER(PdcsOptions)]
    L.pdcs_default_options.restype = None
    L.pdcs_setup.argtypes = [ctypes.POINTER(vp), i64, i64, vp, vp, vp, vp, vp, i64, vp, vp,
                             ctypes.POINTER(PdcsCone), i64, ctypes.POINTER(PdcsCone), i64,
                             ctypes.POINTER(PdcsOptions), vp]
    L.pdcs_setup.restype = ctypes.c_int
    L.pdcs_solve.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(PdcsResult)]
    L.pdcs_solve.restype = ctypes.c_int
    L.pdcs_resume.argtypes = [vp, i64, vp, vp, vp, ctypes.POINTER(PdcsResult)]
    L.pdcs_resume.restype = ctypes.c_int
    L.pdcs_get_state.argtypes = [vp, ctypes.POINTER(PdcsState), vp, vp, vp, vp, vp, vp]
    L.pdcs_get_state.restype = ctypes.c_int
    L.pdcs_set_state.argtypes = [vp, ctypes.POINTER(PdcsState), vp, vp, vp, vp, vp, vp]
    L.pdcs_set_state.restype = ctypes.c_int
    L.pdcs_get_iterate.argtypes = [vp, i32, vp, vp]
    L.pdcs_get_iterate.restype = ctypes.c_int
    L.pdcs_get_trace.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    L.pdcs_get_trace.restype = ctypes.c_int
    L.pdcs_get_profile.argtypes = [vp, ctypes.POINTER(PdcsProfile)]
    L.pdcs_get_profile.restype = ctypes.c_int
    L.pdcs_get_kernel_times.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i32)]
    L.pdcs_get_kernel_times.restype = ctypes.c_int
    L.pdcs_get_sizes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.pdcs_get_sizes.restype = ctypes.c_int
    L.pdcs_free.argtypes = [vp]
    L.pdcs_free.restype = None
    L.pdcs_last_error.argtypes = []
    L.pdcs_last_error.restype = ctypes.c_char_p
    L.pdcs_spmv_noalloc.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp]
    L.pdcs_spmv_noalloc.restype = ctypes.c_int
    L.pdcs_spmv_noalloc_status.argtypes = [vp, ctypes.POINTER(i64)]
    L.pdcs_spmv_noalloc_status.restype = ctypes.c_int
    L.pdcs_setup_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PdcsInstance), i64,
                                   ctypes.POINTER(PdcsOptions), vp]
    L.pdcs_setup_batch.restype = ctypes.c_int
    L.pdcs_solve_batch.argtypes = [vp, vp, vp, vp, ctypes.POINTER(PdcsResult), vp]
    L.pdcs_solve_batch.restype = ctypes.c_int
    L.pdcs_kkt.argtypes = [vp, vp, vp, ctypes.POINTER(PdcsResult)]
    L.pdcs_kkt.restype = ctypes.c_int
    L.pdcs_mlp_default_config.argtypes = [ctypes.POINTER(PdcsMlpConfig)]
    L.pdcs_mlp_default_config.restype = None
    L.pdcs_mlp_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PdcsMlpConfig), vp]
    L.pdcs_mlp_create.restype = ctypes.c_int
    L.pdcs_mlp_train_step.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctypes.c_double)]
    L.pdcs_mlp_train_step.restype = ctypes.c_int
    L.pdcs_mlp_gradients.argtypes = [vp, vp, vp, i64, i32, vp, vp, ctypes.POINTER(ctypes.c_double)]
    L.pdcs_mlp_gradients.restype = ctypes.c_int
    L.pdcs_mlp_predict.argtypes = [vp, vp, i64, vp]
    L.pdcs_mlp_predict.restype = ctypes.c_int
    L.pdcs_mlp_get_layer.argtypes = [vp, i32, vp, vp]
    L.pdcs_mlp_get_layer.restype = ctypes.c_int
    L.pdcs_mlp_set_layer.argtypes = [vp, i32, vp, vp]
    L.pdcs_mlp_set_layer.restype = ctypes.c_int
    L.pdcs_mlp_free.argtypes = [vp]
    L.pdcs_mlp_free.restype = None
    _LIB = L
    return L


class PdcsError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise PdcsError("pdcs error %d: %s" % (rc, lib().pdcs_last_error().decode()))


def _ptr(a):
    """Address of a contiguous NumPy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def default_options(**kw):
    o = PdcsOptions()
    lib().pdcs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "method" and isinstance(v, str):
            v = {"average": 0, "halpern": 1}[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp64": 0, "fp32": 1}[v]
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _cones(lst):
    arr = (PdcsCone * max(1, len(lst)))()
    for i, (t, d) in enumerate(lst):
        arr[i].type = int(t)
        arr[i].dim = int(d)
    return arr


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


class Solver:
    """One problem set up on the GPU (pdcs_setup); solve() may be called repeatedly.

    `problem` is a dict with m, n, row_ptr, col_idx, val, h, c, nb, lo, hi,
    row_cones, col_cones (NumPy arrays or CUDA tensors of the C ABI's dtypes)."""

    def __init__(self, problem, stream=None, **options):
        self._h = ctypes.c_void_p()
        keep = []
        L = lib()
        p = problem

        def arr(key, dtype):
            a = p[key]
            if not hasattr(a, "data_ptr"):
                a = np.ascontiguousarray(a, dtype=dtype)
            keep.append(a)
            return a

        self.m, self.n, self.nb = int(p["m"]), int(p["n"]), int(p["nb"])
        rp = arr("row_ptr", np.int64)
        ci = arr("col_idx", np.int32)
        vv = arr("val", np.float64)
        h = arr("h", np.float64)
        c = arr("c", np.float64)
        lo = arr("lo", np.float64) if self.nb else None
        hi = arr("hi", np.float64) if self.nb else None
        rc = _cones(p["row_cones"])
        cc = _cones(p["col_cones"])
        self.options = default_options(**options)
        st = stream if stream is not None else _current_stream()
        _check(L.pdcs_setup(ctypes.byref(self._h), self.m, self.n, _ptr(rp), _ptr(ci), _ptr(vv),
                            _ptr(h), _ptr(c), self.nb, _ptr(lo), _ptr(hi), rc,
                            len(p["row_cones"]), cc, len(p["col_cones"]),
                            ctypes.byref(self.options), st))
        mm, nn, nz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(L.pdcs_get_sizes(self._h, ctypes.byref(mm), ctypes.byref(nn), ctypes.byref(nz)))
        self.nnz = nz.value

    def _result(self, res, x, y, s):
        d = {k: getattr(res, k) for k, _ in PdcsResult._fields_ if k != "pad"}
        d.update(x=x, y=y, s=s, status=EXIT_NAMES.get(res.exit_code, "?"))
        return d

    def kkt(self, x=None, y=None):
        """KKT errors of a point in the original variables (pdcs_kkt); replaces
        the handle's iterate.  Returns the pdcs_result fields."""
        res = PdcsResult()
        if x is not None and not hasattr(x, "data_ptr"):
            x = np.ascontiguousarray(x, dtype=np.float64)
        if y is not None and not hasattr(y, "data_ptr"):
            y = np.ascontiguousarray(y, dtype=np.float64)
        _check(lib().pdcs_kkt(self._h, _ptr(x), _ptr(y), ctypes.byref(res)))
        d = {k: getattr(res, k) for k, _ in PdcsResult._fields_ if k != "pad"}
        d["max_rel"] = max(res.err_rel_p, res.err_rel_d, res.err_rel_gap)
        return d

    def solve(self, x0=None, y0=None, out=None):
        """Run one solve.  Returns a dict with x, y, s (NumPy, or the arrays in
        `out` = (x, y, s) when given) and the pdcs_result fields."""
        res = PdcsResult()
        if out is None:
            x, y, s = np.empty(self.n), np.empty(self.m), np.empty(self.m)
        else:
            x, y, s = out
        if x0 is not None and not hasattr(x0, "data_ptr"):
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
        if y0 is not None and not hasattr(y0, "data_ptr"):
            y0 = np.ascontiguousarray(y0, dtype=np.float64)
        _check(lib().pdcs_solve(self._h, _ptr(x0), _ptr(y0), _ptr(x), _ptr(y), _ptr(s),
                                ctypes.byref(res)))
        return self._result(res, x, y, s)

    def resume(self, max_iter=0):
        """Continue from the current state (pdcs_resume)."""
        res = PdcsResult()
        x, y, s = np.empty(self.n), np.empty(self.m), np.empty(self.m)
        _check(lib().pdcs_resume(self._h, int(max_iter), _ptr(x), _ptr(y), _ptr(s),
                                 ctypes.byref(res)))
        return self._result(res, x, y, s)

    def get_state(self):
        """Solver state: the pdcs_state scalars plus x, y, x0, y0, xs, ys
        (scaled, reformulated variables)."""
        st = PdcsState()
        v = {k: np.empty(self.n if k in ("x", "x0", "xs") else self.m)
             for k in ("x", "y", "x0", "y0", "xs", "ys")}
        _check(lib().pdcs_get_state(self._h, ctypes.byref(st),
                                    *[_ptr(v[k]) for k in ("x", "y", "x0", "y0", "xs", "ys")]))
        d = {k: getattr(st, k) for k, _ in PdcsState._fields_}
        d.update(v)
        return d

    def set_state(self, state):
        """Replace the solver state (keys as returned by get_state)."""
        st = PdcsState()
        for k, _ in PdcsState._fields_:
            setattr(st, k, state[k])
        vec = [np.ascontiguousarray(state[k], dtype=np.float64)
               for k in ("x", "y", "x0", "y0", "xs", "ys")]
        _check(lib().pdcs_set_state(self._h, ctypes.byref(st), *[_ptr(a) for a in vec]))

    def get_iterate(self, which=0):
        """Internal iterate (scaled, reformulated variables) as NumPy arrays."""
        x, y = np.empty(self.n), np.empty(self.m)
        _check(lib().pdcs_get_iterate(self._h, int(which), _ptr(x), _ptr(y)))
        return x, y

    def profile(self):
        """Device-timed SpMV statistics of the last solve / resume."""
        pr = PdcsProfile()
        _check(lib().pdcs_get_profile(self._h, ctypes.byref(pr)))
        return {k: getattr(pr, k) for k, _ in PdcsProfile._fields_}

    def kernel_times(self):
        """{kernel class: (seconds, launches)} of the last solve / resume."""
        k = len(KERNEL_CLASSES)
        sec = np.zeros(k)
        la = np.zeros(k, dtype=np.int64)
        cnt = ctypes.c_int32()
        _check(lib().pdcs_get_kernel_times(self._h, _ptr(sec), _ptr(la), k, ctypes.byref(cnt)))
        return {KERNEL_CLASSES[i]: (float(sec[i]), int(la[i])) for i in range(cnt.value)}

    def trace(self):
        cap = int(self.options.trace_capacity)
        out = np.zeros((max(cap, 1), TRACE_FIELDS))
        cnt = ctypes.c_int64()
        _check(lib().pdcs_get_trace(self._h, _ptr(out), cap, ctypes.byref(cnt)))
        return out[:cnt.value]

    def close(self):
        if self._h:
            lib().pdcs_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def spmv_noalloc(row_ptr, col_idx, val, x, y, n=None, stream=None):
    """y = G x through pdcs_spmv_noalloc (no allocation, no synchronisation in
    the call).  All arrays are CUDA tensors on the current device (int64,
    int32, float64, float64, float64); stream: a torch.cuda.Stream (default:
    the current one).  A matrix beyond the scratch's limits is rejected on the
    device, leaving y as it was: spmv_noalloc_status() counts such calls."""
    import torch
    m = row_ptr.numel() - 1
    n = x.numel() if n is None else int(n)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().pdcs_spmv_noalloc(int(m), n, _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(x),
                                   _ptr(y), ctypes.c_void_p(st.cuda_stream)))
    return y


def spmv_noalloc_status(stream=None):
    """Number of spmv_noalloc calls rejected on the device since the previous
    query (then reset); synchronises `stream` (default: the current one)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_int64(0)
    _check(lib().pdcs_spmv_noalloc_status(ctypes.c_void_p(st.cuda_stream), ctypes.byref(out)))
    return int(out.value)


class Batch:
    """Many independent problems solved in one persistent kernel launch
    (pdcs_setup_batch / pdcs_solve_batch).  `problems` is a list of problem
    dicts as for Solver (host arrays)."""

    def __init__(self, problems, stream=None, **options):
        self._h = ctypes.c_void_p()
        self.count = len(problems)
        keep = []
        inst = (PdcsInstance * self.count)()
        self.sizes = []
        for k, p in enumerate(problems):
            def arr(key, dtype):
                a = np.ascontiguousarray(p[key], dtype=dtype)
                keep.append(a)
                return a.ctypes.data
            m, n, nb = int(p["m"]), int(p["n"]), int(p["nb"])
            rc, cc = _cones(p["row_cones"]), _cones(p["col_cones"])
            keep += [rc, cc]
            inst[k] = PdcsInstance(m, n, arr("row_ptr", np.int64), arr("col_idx", np.int32),
                                   arr("val", np.float64), arr("h", np.float64),
                                   arr("c", np.float64), nb,
                                   arr("lo", np.float64) if nb else None,
                                   arr("hi", np.float64) if nb else None,
                                   ctypes.cast(rc, ctypes.c_void_p), len(p["row_cones"]),
                                   ctypes.cast(cc, ctypes.c_void_p), len(p["col_cones"]))
            self.sizes.append((m, n))
        self.options = default_options(**options)
        st = stream if stream is not None else _current_stream()
        _check(lib().pdcs_setup_batch(ctypes.byref(self._h), inst, self.count,
                                      ctypes.byref(self.options), st))

    def solve(self):
        """Returns (list of per-problem result dicts with x, y, s, finish time
        from the first start)."""
        nt = sum(n for _, n in self.sizes)
        mt = sum(m for m, _ in self.sizes)
        x, y, s = np.empty(nt), np.empty(mt), np.empty(mt)
        res = (PdcsResult * self.count)()
        fin = np.empty(self.count)
        _check(lib().pdcs_solve_batch(self._h, _ptr(x), _ptr(y), _ptr(s), res, _ptr(fin)))
        out, r0, c0 = [], 0, 0
        for k, (m, n) in enumerate(self.sizes):
            d = {f: getattr(res[k], f) for f, _ in PdcsResult._fields_ if f != "pad"}
            d.update(x=x[c0:c0 + n], y=y[r0:r0 + m], s=s[r0:r0 + m], finish_s=fin[k],
                     status=EXIT_NAMES.get(res[k].exit_code, "?"))
            out.append(d)
            r0 += m
            c0 += n
        return out

    def close(self):
        if self._h:
            lib().pdcs_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Mlp:
    """The warm-start network (pdcs_mlp_*).  Arrays are FP32 NumPy arrays or
    CUDA tensors, row-major (batch x features)."""

    def __init__(self, in_dim, out_dim, hidden=512, n_hidden=3, max_batch=256, lr=1e-3,
                 beta1=0.9, beta2=0.999, eps=1e-8, seed=20260105, stream=None):
        cfg = PdcsMlpConfig()
        lib().pdcs_mlp_default_config(ctypes.byref(cfg))
        cfg.in_dim, cfg.out_dim, cfg.hidden, cfg.n_hidden = in_dim, out_dim, hidden, n_hidden
        cfg.max_batch, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, cfg.seed = (
            max_batch, lr, beta1, beta2, eps, seed)
        self.cfg = cfg
        self.dims = [in_dim] + [hidden] * n_hidden + [out_dim]
        self._h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(lib().pdcs_mlp_create(ctypes.byref(self._h), ctypes.byref(cfg), st))

    @staticmethod
    def _f32(a):
        if a is None or hasattr(a, "data_ptr"):
            return a
        return np.ascontiguousarray(a, dtype=np.float32)

    def train_step(self, X, T):
        X, T = self._f32(X), self._f32(T)
        loss = ctypes.c_double()
        _check(lib().pdcs_mlp_train_step(self._h, _ptr(X), _ptr(T), int(X.shape[0]),
                                         ctypes.byref(loss)))
        return loss.value

    def gradients(self, X, T, layer):
        X, T = self._f32(X), self._f32(T)
        dW = np.empty((self.dims[layer + 1], self.dims[layer]), np.float32)
        db = np.empty(self.dims[layer + 1], np.float32)
        loss = ctypes.c_double()
        _check(lib().pdcs_mlp_gradients(self._h, _ptr(X), _ptr(T), int(X.shape[0]), int(layer),
                                        _ptr(dW), _ptr(db), ctypes.byref(loss)))
        return loss.value, dW, db

    def predict(self, X, out=None):
        X = self._f32(X)
        Y = out if out is not None else np.empty((X.shape[0], self.dims[-1]), np.float32)
        _check(lib().pdcs_mlp_predict(self._h, _ptr(X), int(X.shape[0]), _ptr(Y)))
        return Y

    def get_layer(self, layer):
        W = np.empty((self.dims[layer + 1], self.dims[layer]), np.float32)
        b = np.empty(self.dims[layer + 1], np.float32)
        _check(lib().pdcs_mlp_get_layer(self._h, int(layer), _ptr(W), _ptr(b)))
        return W, b

    def set_layer(self, layer, W, b):
        W, b = self._f32(W), self._f32(b)
        _check(lib().pdcs_mlp_set_layer(self._h, int(layer), _ptr(W), _ptr(b)))

    def close(self):
        if self._h:
            lib().pdcs_mlp_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve(problem, x0=None, y0=None, **options):
    """Set up, solve once, free."""
    with Solver(problem, **options) as s:
        return s.solve(x0, y0)
