"""ctypes binding of libabsorber.so (include/absorber.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python values and
torch tensors (used for device memory and streams) to the C ABI's plain pointers and
structs.  It raises if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libabsorber.so")

ABS_OK = 0
STATUS = {0: "ok", -1: "arg", -2: "cuda", -3: "oom", -4: "inertia", -5: "linesearch", -6: "maxiter",
          -7: "numeric", -8: "timeout", -9: "infeasible"}
PREC_FP64, PREC_FP32, PREC_FP32_TC, PREC_FP64_LDL = 0, 1, 3, 4
NSC = 220
N_FEED = 18


class AbsParams(C.Structure):
    _fields_ = [("R", C.c_double), ("u_max", C.c_double), ("d_lo", C.c_double), ("d_hi", C.c_double),
                ("T_lo", C.c_double), ("T_hi", C.c_double), ("T_ref", C.c_double),
                ("sx", C.c_double * 9), ("sy", C.c_double * 4), ("sT", C.c_double),
                ("KE_A", C.c_double * 5), ("KE_B", C.c_double * 5), ("KE_C", C.c_double * 5),
                ("KE_D", C.c_double * 5),
                ("psat_a", C.c_double), ("psat_b", C.c_double), ("psat_c", C.c_double),
                ("henry_a", C.c_double), ("henry_b", C.c_double), ("henry_m", C.c_double),
                ("henry_w", C.c_double), ("rho_L", C.c_double),
                ("hL_ref", C.c_double * 9), ("hL_cpa", C.c_double * 9), ("hL_cpb", C.c_double * 9),
                ("hL_dh", C.c_double * 9),
                ("hV_ref", C.c_double * 4), ("hV_cpa", C.c_double * 4), ("hV_cpb", C.c_double * 4),
                ("hV_dh", C.c_double * 4), ("n_sections", C.c_int32), ("dp_stage", C.c_double)]


class AbsSizes(C.Structure):
    _fields_ = [("S", C.c_int64), ("ld", C.c_int64), ("n_var_paper", C.c_int64), ("n_mesh", C.c_int64),
                ("n_fix", C.c_int64), ("n_hyd", C.c_int64), ("n_unknowns", C.c_int64),
                ("n_rows", C.c_int64), ("nnzJ_scen", C.c_int32), ("nnzH_scen", C.c_int32)]


class AbsKKTDiag(C.Structure):
    _fields_ = [("sigma", C.c_void_p), ("delta_w", C.c_double), ("delta_c", C.c_double)]


class AbsInertia(C.Structure):
    _fields_ = [("n_pos", C.c_int64), ("n_neg", C.c_int64), ("n_zero", C.c_int64), ("schur_d", C.c_double),
                ("n_singular", C.c_int64)]


class AbsSolveInfo(C.Structure):
    _fields_ = [("refine_steps", C.c_int32), ("residual", C.c_double)]


class AbsOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("max_refine", C.c_int32), ("refine_tol", C.c_double),
                ("mu_init", C.c_double), ("kappa_eps", C.c_double), ("kappa_mu", C.c_double),
                ("theta_mu", C.c_double), ("tau_min", C.c_double), ("s_max", C.c_double),
                ("kappa_sigma", C.c_double), ("bound_push", C.c_double), ("bound_frac", C.c_double),
                ("gamma_theta", C.c_double), ("gamma_phi", C.c_double), ("delta", C.c_double),
                ("s_theta", C.c_double), ("s_phi", C.c_double), ("eta_phi", C.c_double),
                ("gamma_alpha", C.c_double), ("lam_init_max", C.c_double),
                ("dw0", C.c_double), ("dw_min", C.c_double), ("dw_max", C.c_double),
                ("kw_minus", C.c_double), ("kw_plus", C.c_double), ("kw_plus_bar", C.c_double),
                ("max_ls", C.c_int32), ("verbose", C.c_int32), ("profile", C.c_int32),
                ("init", C.c_int32), ("soc_max", C.c_int32), ("kappa_soc", C.c_double),
                ("obj_scaling", C.c_double), ("warm_mu_init", C.c_double), ("warm_bound_push", C.c_double),
                ("warm_multipliers", C.c_int32), ("autotune", C.c_int32), ("graphs", C.c_int32),
                ("factor_tile", C.c_int32), ("resto_max", C.c_int32), ("factor_kernel", C.c_int32),
                ("kkt", C.c_int32)]


class AbsResult(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int32), ("ls_trials", C.c_int32),
                ("inertia_corrections", C.c_int32), ("refine_steps", C.c_int32),
                ("d", C.c_double), ("obj", C.c_double), ("E0", C.c_double), ("mu", C.c_double),
                ("inf_pr", C.c_double), ("inf_du", C.c_double), ("solve_ms", C.c_double),
                ("phase_ms", C.c_double * 6), ("kernel_ms", C.c_double * 5),
                ("kernel_launches", C.c_int32 * 5), ("launches", C.c_int64),
                ("base_iters", C.c_int32), ("soc_steps", C.c_int32), ("fp64_fallbacks", C.c_int32),
                ("base_ms", C.c_double), ("warm_status", C.c_int32), ("fp64_scenarios", C.c_int32),
                ("warm_ms", C.c_double), ("warm_E0", C.c_double), ("cold_E0", C.c_double),
                ("warm_theta", C.c_double), ("cold_theta", C.c_double), ("tiles", C.c_int32 * 4),
                ("graph_replays", C.c_int32), ("resto_phases", C.c_int32),
                ("kind_launches", C.c_int64 * 16), ("d_sec", C.c_double * 2)]


class AbsTrainOptions(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double), ("lr_final", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double), ("seed", C.c_uint64)]


MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS = 3, 256, 440, 245688

KERNELS = ("eval", "eval_trial", "factor", "solve", "solve_t")
KINDS = ("eval", "eval_trial", "factor", "solve", "solve_t", "residual", "schur", "dual", "reduce_planes", "rhs",
         "dz", "step", "accept", "vector", "control", "eval_jac")
PHASES = ("eval", "factor", "solve", "linesearch", "step", "other")


EXPORTS = {
    "absorber_create": (C.c_int, [C.POINTER(AbsParams), C.c_void_p, C.c_void_p, C.c_int64,
                                  C.POINTER(C.c_void_p)]),
    "absorber_destroy": (None, [C.c_void_p]),
    "absorber_set_feeds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "abs_last_error": (C.c_char_p, [C.c_void_p]),
    "absorber_sizes": (C.c_int, [C.c_void_p, C.POINTER(AbsSizes)]),
    "absorber_pattern": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "abs_scenario_pattern": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    "abs_struct_size": (C.c_int64, [C.c_int]),
    "abs_measure_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "eval_grad_jac_hess": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(C.c_double),
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "kkt_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(AbsKKTDiag), C.c_int,
                             C.POINTER(AbsInertia), C.c_void_p]),
    "kkt_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                            C.POINTER(AbsSolveInfo), C.c_void_p]),
    "abs_default_options": (None, [C.POINTER(AbsOptions)]),
    "kkt_newton_noalloc": (C.c_int, [C.POINTER(AbsParams), C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "ipm_solve": (C.c_int, [C.c_void_p, C.POINTER(AbsOptions), C.c_void_p, C.c_void_p, C.POINTER(AbsResult),
                            C.c_void_p, C.c_void_p, C.c_void_p]),
    "absorber_bound_multipliers": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ipm_solve_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(AbsOptions), C.POINTER(AbsResult),
                                    C.POINTER(C.c_void_p), C.c_void_p]),
    "absorber_create_batched": (C.c_int, [C.POINTER(AbsParams), C.c_void_p, C.POINTER(C.c_int64), C.c_int32,
                                          C.POINTER(C.c_void_p)]),
    "absorber_num_problems": (C.c_int32, [C.c_void_p]),
    "ipm_solve_batch": (C.c_int, [C.c_void_p, C.POINTER(AbsOptions), C.POINTER(AbsResult), C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "absorber_scenario_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "absorber_paper_layout": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "abs_mlp_create": (C.c_int, [C.c_uint64, C.POINTER(C.c_void_p)]),
    "abs_mlp_destroy": (None, [C.c_void_p]),
    "abs_mlp_last_error": (C.c_char_p, [C.c_void_p]),
    "abs_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "abs_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "abs_mlp_set_normalization": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "abs_mlp_get_normalization": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "abs_mlp_fit_normalization": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "abs_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "abs_mlp_set_tensor_cores": (C.c_int, [C.c_void_p, C.c_int32]),
    "abs_mlp_device_fault": (C.c_int32, [C.c_void_p]),
    "abs_mlp_selftest_wait": (C.c_int, [C.c_void_p, C.c_void_p]),
    "abs_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double),
                                    C.c_void_p, C.c_void_p]),
    "abs_default_train_options": (None, [C.POINTER(AbsTrainOptions)]),
    "abs_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(AbsTrainOptions),
                                C.c_void_p, C.c_void_p]),
    "abs_mlp_make_dataset": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                                       C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "ipm_solve_learned": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(AbsOptions), C.POINTER(AbsResult),
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
}

_lib = None


def lib():
    """Load libabsorber.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2607_15420_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class AbsorberError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def make_params(P: dict) -> AbsParams:
    p = AbsParams()
    for name, _ in AbsParams._fields_:
        if name == "n_sections":
            p.n_sections = int(P.get("n_sections", 1))
            continue
        if name == "dp_stage":
            p.dp_stage = float(P.get("dp_stage", 0.0))
            continue
        v = P[name]
        if isinstance(v, (tuple, list)):
            arr = getattr(p, name)
            for i, e in enumerate(v):
                arr[i] = float(e)
        else:
            setattr(p, name, float(v))
    return p


def default_options(**kw) -> AbsOptions:
    o = AbsOptions()
    lib().abs_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def measure_fma_peak(kind):
    """Measured FMA throughput of the current device in GFLOP/s (kind 0 FP64, 1 FP32)."""
    v = C.c_double(0.0)
    st = lib().abs_measure_fma_peak(int(kind), C.byref(v))
    if st != ABS_OK:
        raise AbsorberError(st, lib().abs_last_error(None).decode())
    return v.value


NOALLOC_MAX_SCENARIOS = 128


def kkt_newton_noalloc(params, S, ld, x, jac, hess, sigma, rhs_x, rhs_c, sol_x, sol_c, delta_w=0.0,
                       stream=None):
    """The allocation-free Newton direction (kkt_newton_noalloc); returns the Schur scalar."""
    p = make_params(params) if isinstance(params, dict) else params
    sd = C.c_double(0.0)
    st = lib().kkt_newton_noalloc(C.byref(p), int(S), int(ld), _ptr(x), _ptr(jac), _ptr(hess), _ptr(sigma),
                                  float(delta_w), _ptr(rhs_x), _ptr(rhs_c), _ptr(sol_x), _ptr(sol_c),
                                  C.byref(sd), _stream(stream))
    if st != ABS_OK:
        raise AbsorberError(st, lib().abs_last_error(None).decode())
    return sd.value


STRUCTS = [AbsParams, AbsSizes, AbsKKTDiag, AbsInertia, AbsSolveInfo, AbsOptions, AbsResult, AbsTrainOptions]


def scenario_pattern():
    """Per-scenario CSR patterns (jrow, jcol, hrow, hcol) from the library; no device needed."""
    nj, nh = C.c_int32(), C.c_int32()
    st = lib().abs_scenario_pattern(C.byref(nj), C.byref(nh), None, None, None, None)
    if st != ABS_OK:
        raise AbsorberError(st, lib().abs_last_error(None).decode())
    jr, jc = np.zeros(nj.value, np.int32), np.zeros(nj.value, np.int32)
    hr, hc = np.zeros(nh.value, np.int32), np.zeros(nh.value, np.int32)
    lib().abs_scenario_pattern(None, None, jr.ctypes.data, jc.ctypes.data, hr.ctypes.data, hc.ctypes.data)
    return jr, jc, hr, hc


class Problem:
    """One instance of problem (10) held by the library (absorber_create)."""

    def __init__(self, params: dict, feeds: np.ndarray, prob=None):
        feeds = np.ascontiguousarray(feeds, dtype=np.float64)
        if feeds.ndim != 2 or feeds.shape[0] != N_FEED:
            raise ValueError("feeds must be (18, S)")
        self.params = make_params(params)
        h = C.c_void_p()
        pr = None
        if prob is not None:
            prob = np.ascontiguousarray(prob, dtype=np.float64)
            pr = prob.ctypes.data
        st = lib().absorber_create(C.byref(self.params), feeds.ctypes.data, pr, feeds.shape[1], C.byref(h))
        if st != ABS_OK:
            raise AbsorberError(st, lib().abs_last_error(None).decode())
        self.h = h
        self.sizes = AbsSizes()
        self._check(lib().absorber_sizes(self.h, C.byref(self.sizes)))
        self.S = self.sizes.S
        self.ld = self.sizes.ld

    def _check(self, st):
        if st != ABS_OK:
            raise AbsorberError(st, lib().abs_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            lib().absorber_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def K(self):
        """Design entries (column sections with their own diameter)."""
        return int(self.params.n_sections)

    @property
    def n_primal(self):
        return NSC * self.ld + self.K

    @property
    def n_row(self):
        return NSC * self.ld

    def pattern(self):
        nj, nh = self.sizes.nnzJ_scen, self.sizes.nnzH_scen
        jr, jc = np.zeros(nj, np.int32), np.zeros(nj, np.int32)
        hr, hc = np.zeros(nh, np.int32), np.zeros(nh, np.int32)
        self._check(lib().absorber_pattern(self.h, jr.ctypes.data, jc.ctypes.data, hr.ctypes.data, hc.ctypes.data))
        return jr, jc, hr, hc

    def eval_grad_jac_hess(self, x, lam=None, obj_factor=1.0, grad=None, c=None, jac=None, hess=None,
                           want_f=False, stream=None):
        f = C.c_double(0.0)
        self._check(lib().eval_grad_jac_hess(self.h, _ptr(x), _ptr(lam), float(obj_factor),
                                             C.byref(f) if want_f else None, _ptr(grad), _ptr(c), _ptr(jac),
                                             _ptr(hess), _stream(stream)))
        return f.value if want_f else None

    def kkt_factor(self, x, jac, hess, sigma, delta_w=0.0, delta_c=0.0, precision=PREC_FP64, stream=None,
                   check=True):
        diag = AbsKKTDiag(_ptr(sigma), float(delta_w), float(delta_c))
        inert = AbsInertia()
        st = lib().kkt_factor(self.h, _ptr(x), _ptr(jac), _ptr(hess), C.byref(diag), int(precision),
                              C.byref(inert), _stream(stream))
        if check:
            self._check(st)
        return inert

    def kkt_solve(self, rhs_x, rhs_c, sol_x, sol_c, max_refine=2, refine_tol=1e-14, stream=None):
        info = AbsSolveInfo()
        self._check(lib().kkt_solve(self.h, _ptr(rhs_x), _ptr(rhs_c), _ptr(sol_x), _ptr(sol_c), int(max_refine),
                                    float(refine_tol), C.byref(info), _stream(stream)))
        return info

    def ipm_solve(self, options=None, warm_x=None, warm_y=None, x_out=None, y_out=None, stream=None,
                  check=False):
        res = AbsResult()
        st = lib().ipm_solve(self.h, C.byref(options) if options is not None else None, _ptr(warm_x),
                             _ptr(warm_y), C.byref(res), _ptr(x_out), _ptr(y_out), _stream(stream))
        if st != ABS_OK and res.status == ABS_OK:
            res.status = st
        if check:
            self._check(st)
        return res

    def bound_multipliers(self, zl_out=None, zu_out=None, stream=None):
        """Bound multipliers of the last solve (unscaled problem min d) into the device
        vectors zl_out, zu_out; returns the host array [z_L(d) per problem, z_U(d) per
        problem]."""
        nprob = int(lib().absorber_num_problems(self.h))
        zd = np.zeros(2 * self.K * nprob)
        self._check(lib().absorber_bound_multipliers(self.h, _ptr(zl_out), _ptr(zu_out), zd.ctypes.data,
                                                     _stream(stream)))
        return zd

    def last_error(self):
        msg = lib().abs_last_error(self.h)
        return msg.decode() if msg else ""

    def scenario_status(self):
        out = np.zeros(self.S, dtype=np.int32)
        self._check(lib().absorber_scenario_status(self.h, out.ctypes.data))
        return out

    def paper_layout(self, x, out, stream=None):
        """Device primal vector -> device [d, z_1..z_S] (300 per scenario, paper's layout)."""
        self._check(lib().absorber_paper_layout(self.h, _ptr(x), _ptr(out), _stream(stream)))

    def set_feeds(self, feeds, stream=None):
        """Replace the scenario feeds (host numpy array or device tensor, (18, S))."""
        if isinstance(feeds, np.ndarray):
            feeds = np.ascontiguousarray(feeds, dtype=np.float64)
            ptr = feeds.ctypes.data
        else:
            ptr = _ptr(feeds)
        self._check(lib().absorber_set_feeds(self.h, ptr, _stream(stream)))

    # ---- layout helpers (host-side reshaping only) ----------------------------------
    def to_soa(self, Z, d=None):
        """(S, 220) per-scenario rows -> flat primal (or row) vector with leading dim ld."""
        S = self.S
        out = np.zeros(self.n_primal if d is not None else self.n_row)
        out[:NSC * self.ld].reshape(NSC, self.ld)[:, :S] = np.asarray(Z).T
        if d is not None:
            out[NSC * self.ld:NSC * self.ld + self.K] = np.atleast_1d(d)
        return out

    def from_soa(self, v):
        """flat primal/row vector -> ((S, 220), d or None)."""
        v = np.asarray(v)
        Z = v[:NSC * self.ld].reshape(NSC, self.ld)[:, :self.S].T.copy()
        d = None
        if v.shape[0] > NSC * self.ld:
            d = float(v[NSC * self.ld]) if self.K == 1 else v[NSC * self.ld:NSC * self.ld + self.K].copy()
        return Z, d

    def values_to_scen(self, vals, nnz):
        """value array [nnz * ld] -> (S, nnz)."""
        return np.asarray(vals)[:nnz * self.ld].reshape(nnz, self.ld)[:, :self.S].T.copy()


class Batch(Problem):
    """P independent problems in one handle (absorber_create_batched)."""

    def __init__(self, params: dict, feeds_list):
        sizes = np.array([np.asarray(F).shape[1] for F in feeds_list], dtype=np.int64)
        feeds = np.ascontiguousarray(np.concatenate([np.asarray(F, dtype=np.float64) for F in feeds_list], axis=1))
        if feeds.shape[0] != N_FEED:
            raise ValueError("feeds must be (18, S_q)")
        self.params = make_params(params)
        h = C.c_void_p()
        st = lib().absorber_create_batched(C.byref(self.params), feeds.ctypes.data,
                                           sizes.ctypes.data_as(C.POINTER(C.c_int64)), len(sizes), C.byref(h))
        if st != ABS_OK:
            raise AbsorberError(st, lib().abs_last_error(None).decode())
        self.h = h
        self.sizes = AbsSizes()
        self._check(lib().absorber_sizes(self.h, C.byref(self.sizes)))
        self.S = self.sizes.S
        self.ld = self.sizes.ld
        self.P = int(lib().absorber_num_problems(self.h))
        self.problem_sizes = sizes
        self.off = np.concatenate([[0], np.cumsum(sizes)])

    @property
    def n_primal(self):
        return NSC * self.ld + self.K * self.ld

    def ipm_solve(self, options=None, x_out=None, y_out=None, stream=None):
        res = (AbsResult * self.P)()
        self._check(lib().ipm_solve_batch(self.h, C.byref(options) if options is not None else None, res,
                                          _ptr(x_out), _ptr(y_out), _stream(stream)))
        return list(res)

    def split(self, v):
        """flat batch vector -> list of ((S_q, 220), d_q or None) per problem."""
        v = np.asarray(v)
        Z = v[:NSC * self.ld].reshape(NSC, self.ld)
        out = []
        for q in range(self.P):
            Zq = Z[:, self.off[q]:self.off[q + 1]].T.copy()
            dq = None
            if v.shape[0] > NSC * self.ld:
                dv = v[NSC * self.ld + q + self.P * np.arange(self.K)]
                dq = float(dv[0]) if self.K == 1 else dv.copy()
            out.append((Zq, dq))
        return out


def ipm_solve_batched(problems, options=None, x_out=None, stream=None):
    """Solve independent problems as one batch; returns one AbsResult per problem.

    problems: list of Problem; x_out: None or a list of device primal vectors (or None
    entries), one per problem, each in its own problem's layout."""
    P = len(problems)
    if P < 1:
        raise ValueError("empty batch")
    hs = (C.c_void_p * P)(*[p.h for p in problems])
    res = (AbsResult * P)()
    xo = None
    if x_out is not None:
        xo = (C.c_void_p * P)(*[_ptr(v) for v in x_out])
    st = lib().ipm_solve_batched(hs, P, C.byref(options) if options is not None else None, res, xo,
                                 _stream(stream))
    if st != ABS_OK:
        raise AbsorberError(st, lib().abs_last_error(problems[0].h).decode())
    return list(res)


def train_options(**kw) -> AbsTrainOptions:
    o = AbsTrainOptions()
    lib().abs_default_train_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class MLP:
    """The warm-start network held by the library (abs_mlp_*)."""

    def __init__(self, seed=1):
        h = C.c_void_p()
        st = lib().abs_mlp_create(int(seed), C.byref(h))
        if st != ABS_OK:
            raise AbsorberError(st, lib().abs_mlp_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != ABS_OK:
            raise AbsorberError(st, lib().abs_mlp_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            lib().abs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.shape == (MLP_PARAMS,)
        self._check(lib().abs_mlp_set_params(self.h, theta.ctypes.data))

    def get_params(self):
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(lib().abs_mlp_get_params(self.h, out.ctypes.data))
        return out

    def set_normalization(self, in_shift, in_scale, out_shift, out_scale):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (in_shift, in_scale, out_shift, out_scale)]
        self._check(lib().abs_mlp_set_normalization(self.h, *[a.ctypes.data for a in arrs]))

    def get_normalization(self):
        a = [np.zeros(n) for n in (MLP_IN, MLP_IN, MLP_OUT, MLP_OUT)]
        self._check(lib().abs_mlp_get_normalization(self.h, *[x.ctypes.data for x in a]))
        return dict(in_shift=a[0], in_scale=a[1], out_shift=a[2], out_scale=a[3])

    def fit_normalization(self, X, Y, stream=None):
        self._check(lib().abs_mlp_fit_normalization(self.h, _ptr(X), _ptr(Y), X.shape[0], _stream(stream)))

    def forward(self, X, Y, stream=None):
        self._check(lib().abs_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), _stream(stream)))

    def set_tensor_cores(self, on):
        self._check(lib().abs_mlp_set_tensor_cores(self.h, int(on)))

    def device_fault(self):
        return int(lib().abs_mlp_device_fault(self.h))

    def selftest_wait(self, stream=None):
        """Status of the tensor-core wait's self-test (ABS_ERR_TIMEOUT when the expiry was
        reported)."""
        return int(lib().abs_mlp_selftest_wait(self.h, _stream(stream)))

    def loss_grad(self, X, Y, grad=None, stream=None):
        loss = C.c_double()
        self._check(lib().abs_mlp_loss_grad(self.h, _ptr(X), _ptr(Y), X.shape[0], C.byref(loss), _ptr(grad),
                                            _stream(stream)))
        return loss.value

    def train(self, X, Y, options=None, stream=None):
        o = options if options is not None else train_options()
        hist = np.zeros(o.epochs)
        self._check(lib().abs_mlp_train(self.h, _ptr(X), _ptr(Y), X.shape[0], C.byref(o), hist.ctypes.data,
                                        _stream(stream)))
        return hist


def make_dataset(problem, x, y, keep=None, n_aug=1, d_spread=0.0, stream=None):
    """Training pairs of a solved handle as new device tensors (X [rows][3], Y [rows][440])."""
    import torch
    kp = None
    if keep is not None:
        keep = np.ascontiguousarray(keep, dtype=np.int32)
        kp = keep.ctypes.data
    rows = C.c_int64()
    problem._check(lib().abs_mlp_make_dataset(problem.h, _ptr(x), _ptr(y), kp, int(n_aug), float(d_spread), None,
                                              None, C.byref(rows), _stream(stream)))
    X = torch.zeros((rows.value, MLP_IN), dtype=torch.float32, device="cuda")
    Y = torch.zeros((rows.value, MLP_OUT), dtype=torch.float32, device="cuda")
    problem._check(lib().abs_mlp_make_dataset(problem.h, _ptr(x), _ptr(y), kp, int(n_aug), float(d_spread),
                                              _ptr(X), _ptr(Y), C.byref(rows), _stream(stream)))
    return X, Y


def ipm_solve_learned(problem, net, options=None, x_out=None, y_out=None, stream=None):
    res = AbsResult()
    st = lib().ipm_solve_learned(problem.h, net.h, C.byref(options) if options is not None else None, C.byref(res),
                                 _ptr(x_out), _ptr(y_out), _stream(stream))
    if st != ABS_OK and res.status == ABS_OK:
        res.status = st
    return res
