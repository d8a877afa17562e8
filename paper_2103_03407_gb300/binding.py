"""ctypes binding of the C ABI in ``include/mlqmc_evp.h`` (argument marshalling only).

Every function keeps the name of the C entry point it wraps.  Host arrays are numpy arrays;
device arrays are torch CUDA tensors (PyTorch provides device memory and streams only), passed
by their data pointer.  A non-OK status raises :class:`MQError` carrying the library message;
``MQ_ENOCONV`` raises :class:`MQNoConvergence` after the outputs are written.

Loading fails loudly when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmlqmc_evp.so")

MQ_OK, MQ_EINVAL, MQ_ENOMEM, MQ_ECUDA, MQ_ENOCONV, MQ_ETIMEOUT, MQ_ESTATE = range(7)
MQ_PREC_FP64, MQ_PREC_MIXED = 0, 1
MQ_QOI_EIGENVALUE, MQ_QOI_FUNCTIONAL = 0, 1
STATUS_NAMES = {0: "MQ_OK", 1: "MQ_EINVAL", 2: "MQ_ENOMEM", 3: "MQ_ECUDA", 4: "MQ_ENOCONV", 5: "MQ_ETIMEOUT",
                6: "MQ_ESTATE"}

# every symbol the header declares
EXPORTS = [
    "mq_create", "mq_destroy", "mq_set_coefficient", "mq_set_levels", "mq_set_lattice", "mq_set_shifts",
    "mq_set_precision", "mq_set_solver_options", "mq_set_eig_options", "mq_set_smoothing", "mq_set_tier", "mq_set_cta_threads", "mq_eval_level", "mq_eval_level_device", "mq_eval_levels_device", "mq_estimate", "mq_reset_sums",
    "mq_get_level_timing", "mq_get_kernel_timing", "mq_get_launch_count", "mq_eval_point",
    "mq_get_stats", "mq_last_error", "mq_cbc_lattice", "mq_lattice_points_device", "mq_coefficients_device",
    "mq_apply_operator_device", "mq_twogrid_samples_noalloc", "mq_set_lattice_embedded", "mq_set_reuse",
    "mq_cbc_embedded_lattice", "mq_get_sums", "mq_estimate_sums", "mq_run_adaptive", "mq_set_level_config",
    "mq_autotune_level", "mq_graph_capture", "mq_graph_launch", "mq_get_graph_info", "mq_set_kernel_probe",
    "mq_get_kernel_probe", "mq_measure_fp64_peak", "mq_set_islands", "mq_set_qoi", "mq_reaction_coefficients_device",
]


class MQError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class MQNoConvergence(MQError):
    pass


class mq_level(C.Structure):
    _fields_ = [("n_fine", C.c_int32), ("n_coarse", C.c_int32), ("s", C.c_int32), ("S", C.c_int32),
                ("N", C.c_uint32), ("R", C.c_int32)]


class mq_adaptive_result(C.Structure):
    _fields_ = [("L", C.c_int32), ("converged", C.c_int32), ("doublings", C.c_int32), ("levels_added", C.c_int32),
                ("N", C.c_uint32 * 32), ("mean", C.c_double), ("std_err", C.c_double),
                ("level_mean", C.c_double * 32), ("level_var", C.c_double * 32)]


class mq_tune_choice(C.Structure):
    _fields_ = [("tier", C.c_int32), ("threads", C.c_int32), ("nu", C.c_int32), ("ms", C.c_double),
                ("from_cache", C.c_int32), ("tried", C.c_int32)]


class mq_stats(C.Structure):
    _fields_ = [("samples", C.c_uint64), ("noconv", C.c_uint64), ("coarse_iters_mean", C.c_double),
                ("coarse_iters_max", C.c_int32), ("fine_iters_mean", C.c_double), ("fine_iters_max", C.c_int32),
                ("outer_iters_mean", C.c_double), ("outer_iters_max", C.c_int32), ("kernel_ms", C.c_double),
                ("coef_ms", C.c_double), ("sample_ms", C.c_double), ("blocks", C.c_int32), ("threads", C.c_int32),
                ("smem_bytes", C.c_int32), ("workspace_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it is missing: build it with paper_2103_03407_gb300.build."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run python -m paper_2103_03407_gb300.build)")
    lib = C.CDLL(path)
    P = C.c_void_p
    i32, u32, f64, sz = C.c_int32, C.c_uint32, C.c_double, C.c_size_t
    dp = C.POINTER(C.c_double)
    sig = {
        "mq_create": ([C.POINTER(P), C.c_int, P], C.c_int),
        "mq_destroy": ([P], C.c_int),
        "mq_set_coefficient": ([P, f64, i32, i32, f64], C.c_int),
        "mq_set_levels": ([P, i32, C.POINTER(mq_level)], C.c_int),
        "mq_set_lattice": ([P, i32, C.POINTER(u32), i32], C.c_int),
        "mq_set_shifts": ([P, i32, dp], C.c_int),
        "mq_set_lattice_embedded": ([P, i32, C.POINTER(u32), i32, i32], C.c_int),
        "mq_set_reuse": ([P, i32], C.c_int),
        "mq_cbc_embedded_lattice": ([i32, i32, i32, f64, C.POINTER(u32)], C.c_int),
        "mq_get_sums": ([P, i32, dp, C.POINTER(C.c_uint64)], C.c_int),
        "mq_run_adaptive": ([P, f64, f64, u32, C.POINTER(mq_adaptive_result)], C.c_int),
        "mq_set_level_config": ([P, i32, i32, i32, i32], C.c_int),
        "mq_graph_capture": ([P, i32, C.POINTER(i32), C.POINTER(u32), C.POINTER(u32), C.POINTER(C.c_void_p),
                              C.POINTER(C.c_void_p)], C.c_int),
        "mq_graph_launch": ([P, C.POINTER(u32)], C.c_int),
        "mq_get_graph_info": ([P, C.POINTER(i32), C.POINTER(C.c_uint64)], C.c_int),
        "mq_set_kernel_probe": ([P, i32], C.c_int),
        "mq_get_kernel_probe": ([P, dp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int),
        "mq_measure_fp64_peak": ([C.c_int, dp, dp], C.c_int),
        "mq_autotune_level": ([P, i32, u32, C.c_char_p, C.POINTER(mq_tune_choice)], C.c_int),
        "mq_estimate_sums": ([i32, C.POINTER(i32), dp, C.POINTER(C.c_uint64), i32, dp, dp, dp, dp], C.c_int),
        "mq_set_precision": ([P, C.c_int, f64], C.c_int),
        "mq_set_tier": ([P, i32], C.c_int),
        "mq_set_solver_options": ([P, f64, i32, i32], C.c_int),
        "mq_set_eig_options": ([P, f64, i32], C.c_int),
        "mq_set_smoothing": ([P, i32], C.c_int),
        "mq_set_cta_threads": ([P, i32, i32], C.c_int),
        "mq_eval_level": ([P, i32, u32, u32, dp, dp], C.c_int),
        "mq_eval_level_device": ([P, i32, u32, u32, P, P], C.c_int),
        "mq_eval_levels_device": ([P, i32, C.POINTER(C.c_int32), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)], C.c_int),
        "mq_estimate": ([P, dp, dp, dp, dp], C.c_int),
        "mq_reset_sums": ([P], C.c_int),
        "mq_get_level_timing": ([P, i32, dp, dp, C.POINTER(C.c_uint64)], C.c_int),
        "mq_get_kernel_timing": ([P, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
        "mq_get_launch_count": ([P, C.POINTER(C.c_uint64)], C.c_int),
        "mq_eval_point": ([P, i32, dp, dp, dp, dp, dp], C.c_int),
        "mq_get_stats": ([P, P, sz], C.c_int),
        "mq_last_error": ([P], C.c_char_p),
        "mq_cbc_lattice": ([u32, i32, f64, C.POINTER(u32)], C.c_int),
        "mq_lattice_points_device": ([P, i32, u32, u32, P], C.c_int),
        "mq_coefficients_device": ([P, i32, i32, P, i32, i32, P], C.c_int),
        "mq_reaction_coefficients_device": ([P, i32, i32, P, i32, i32, P], C.c_int),
        "mq_set_islands": ([P, i32, f64, f64, f64, f64], C.c_int),
        "mq_set_qoi": ([P, i32], C.c_int),
        "mq_apply_operator_device": ([P, i32, i32, P, i32, f64, P, P], C.c_int),
        "mq_twogrid_samples_noalloc": ([i32, i32, i32, i32, i32, P, P, P, f64, P, P, P, P], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _tptr(t):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arguments must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


class Context:
    """Owns one ``mq_ctx``.  Methods are the C entry points with the context argument bound."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.mq_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None)
        if st != MQ_OK:
            raise MQError(st, "mq_create failed (no CUDA device?)")
        self.h = h
        self.levels = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.mq_destroy(self.h)
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

    def _check(self, st):
        if st == MQ_OK:
            return
        msg = self.lib.mq_last_error(self.h).decode()
        if st == MQ_ENOCONV:
            raise MQNoConvergence(st, msg)
        raise MQError(st, msg)

    # --- configuration ---------------------------------------------------------------------
    def mq_set_coefficient(self, a0=1.0, s_max=16, family=0, decay=2.0):
        self._check(self.lib.mq_set_coefficient(self.h, float(a0), int(s_max), int(family), float(decay)))

    def mq_set_islands(self, s_max, p_a=2.0, p_a_prime=2.0, p_b=2.0, p_b_prime=2.0):
        self._check(self.lib.mq_set_islands(self.h, int(s_max), float(p_a), float(p_a_prime), float(p_b),
                                            float(p_b_prime)))

    def mq_set_qoi(self, qoi=MQ_QOI_EIGENVALUE):
        self._check(self.lib.mq_set_qoi(self.h, int(qoi)))

    def mq_set_levels(self, levels):
        arr = (mq_level * len(levels))()
        for i, lv in enumerate(levels):
            arr[i] = mq_level(lv.n_fine, lv.n_coarse, lv.s, lv.S, lv.N, lv.R)
        self._check(self.lib.mq_set_levels(self.h, len(levels), arr))
        self.levels = list(levels)

    def mq_set_lattice(self, level, z):
        z = np.ascontiguousarray(z, dtype=np.uint32)
        self._check(self.lib.mq_set_lattice(self.h, int(level), z.ctypes.data_as(C.POINTER(C.c_uint32)), z.size))

    def mq_set_lattice_embedded(self, level, z, m_max):
        z = np.ascontiguousarray(z, dtype=np.uint32)
        self._check(self.lib.mq_set_lattice_embedded(self.h, int(level), z.ctypes.data_as(C.POINTER(C.c_uint32)),
                                                     z.size, int(m_max)))

    def mq_set_reuse(self, on=1):
        self._check(self.lib.mq_set_reuse(self.h, int(on)))

    def mq_set_shifts(self, level, delta):
        d = np.ascontiguousarray(delta, dtype=np.float64)
        self._check(self.lib.mq_set_shifts(self.h, int(level), _dptr(d)))

    def mq_set_precision(self, prec=MQ_PREC_FP64, tol_linear=0.0):
        self._check(self.lib.mq_set_precision(self.h, int(prec), float(tol_linear)))

    def mq_set_solver_options(self, tol_inner=0.0, max_inner=0, max_outer=0):
        self._check(self.lib.mq_set_solver_options(self.h, float(tol_inner), int(max_inner), int(max_outer)))

    def mq_set_eig_options(self, tol_eig=0.0, max_eig=0):
        self._check(self.lib.mq_set_eig_options(self.h, float(tol_eig), int(max_eig)))

    def mq_set_smoothing(self, nu=0):
        self._check(self.lib.mq_set_smoothing(self.h, int(nu)))

    def mq_set_cta_threads(self, level, threads=0):
        self._check(self.lib.mq_set_cta_threads(self.h, int(level), int(threads)))

    def mq_set_level_config(self, level, tier=-1, threads=0, nu=0):
        self._check(self.lib.mq_set_level_config(self.h, int(level), int(tier), int(threads), int(nu)))

    def mq_autotune_level(self, level, points, cache_path=None):
        ch = mq_tune_choice()
        path = cache_path.encode() if cache_path else None
        self._check(self.lib.mq_autotune_level(self.h, int(level), int(points), path, C.byref(ch)))
        return {k: getattr(ch, k) for k, _ in ch._fields_}

    def mq_set_tier(self, stream_min_n=0):
        self._check(self.lib.mq_set_tier(self.h, int(stream_min_n)))

    # --- evaluation --------------------------------------------------------------------------
    def mq_eval_level(self, level, k0, k1, per_sample=True, shift_sums=None):
        """Returns (per_sample [R, k1-k0, 4] or None, shift_sums [R])."""
        R = self.levels[level].R
        ps = np.zeros((R, k1 - k0, 4)) if per_sample else None
        ss = np.zeros(R) if shift_sums is None else np.ascontiguousarray(shift_sums, dtype=np.float64)
        st = self.lib.mq_eval_level(self.h, int(level), int(k0), int(k1), _dptr(ps) if ps is not None else None,
                                    _dptr(ss))
        self._check(st)
        return ps, ss

    def mq_eval_level_device(self, level, k0, k1, d_per_sample=None, d_shift_sums=None):
        self._check(self.lib.mq_eval_level_device(self.h, int(level), int(k0), int(k1), _tptr(d_per_sample),
                                                  _tptr(d_shift_sums)))

    def mq_eval_levels_device(self, levels, d_per_sample=None, d_shift_sums=None):
        """Whole levels at once, each on its own internal context and stream; per-level device
        outputs as in mq_eval_level_device (lists of tensors or None)."""
        n = len(levels)
        lv = (C.c_int32 * n)(*[int(l) for l in levels])
        ps = (C.c_void_p * n)(*[_tptr(t) for t in d_per_sample]) if d_per_sample is not None else None
        ss = (C.c_void_p * n)(*[_tptr(t) for t in d_shift_sums]) if d_shift_sums is not None else None
        self._check(self.lib.mq_eval_levels_device(self.h, n, lv, ps, ss))

    def mq_graph_capture(self, ranges, d_per_sample=None, d_shift_sums=None):
        """ranges: list of (level, k0, k1) evaluated in order as one CUDA graph; device outputs as in
        mq_eval_level_device (lists of tensors or None)."""
        n = len(ranges)
        lv = (C.c_int32 * n)(*[int(r[0]) for r in ranges])
        k0 = (C.c_uint32 * n)(*[int(r[1]) for r in ranges])
        k1 = (C.c_uint32 * n)(*[int(r[2]) for r in ranges])
        ps = (C.c_void_p * n)(*[_tptr(t) for t in d_per_sample]) if d_per_sample is not None else None
        ss = (C.c_void_p * n)(*[_tptr(t) for t in d_shift_sums]) if d_shift_sums is not None else None
        self._check(self.lib.mq_graph_capture(self.h, n, lv, k0, k1, ps, ss))

    def mq_graph_launch(self, k0s=None):
        k = (C.c_uint32 * len(k0s))(*[int(x) for x in k0s]) if k0s is not None else None
        self._check(self.lib.mq_graph_launch(self.h, k))

    def mq_get_graph_info(self):
        cap, nodes = C.c_int32(), C.c_uint64()
        self._check(self.lib.mq_get_graph_info(self.h, C.byref(cap), C.byref(nodes)))
        return bool(cap.value), nodes.value

    def mq_set_kernel_probe(self, on=1):
        self._check(self.lib.mq_set_kernel_probe(self.h, int(on)))

    def mq_get_kernel_probe(self):
        """(ms, launches, algorithmic bytes) of the operator sweep since the probe was switched on."""
        ms, n, b = C.c_double(), C.c_uint64(), C.c_uint64()
        self._check(self.lib.mq_get_kernel_probe(self.h, C.byref(ms), C.byref(n), C.byref(b)))
        return ms.value, n.value, b.value

    def mq_estimate(self):
        L = len(self.levels)
        m, se = C.c_double(), C.c_double()
        lm, lv = np.zeros(L), np.zeros(L)
        self._check(self.lib.mq_estimate(self.h, C.byref(m), C.byref(se), _dptr(lm), _dptr(lv)))
        return m.value, se.value, lm, lv

    def mq_get_sums(self, level):
        """(sums [R], points) of one level's estimator state."""
        R = self.levels[level].R
        sums, n = np.zeros(R), C.c_uint64()
        self._check(self.lib.mq_get_sums(self.h, int(level), _dptr(sums), C.byref(n)))
        return sums, n.value

    def mq_run_adaptive(self, eps, alpha=2.0, n_init=8):
        """Adaptive N_l and L (see the header); returns the result as a dict."""
        r = mq_adaptive_result()
        self._check(self.lib.mq_run_adaptive(self.h, float(eps), float(alpha), int(n_init), C.byref(r)))
        L = r.L
        return {"L": L, "converged": bool(r.converged), "doublings": r.doublings, "levels_added": r.levels_added,
                "N": [int(r.N[l]) for l in range(L + 1)], "mean": r.mean, "std_err": r.std_err,
                "level_mean": [r.level_mean[l] for l in range(L + 1)],
                "level_var": [r.level_var[l] for l in range(L + 1)]}

    def mq_reset_sums(self):
        self._check(self.lib.mq_reset_sums(self.h))

    def mq_get_level_timing(self, level):
        """(coef_ms, sample_ms, launches) accumulated on a level since the last reset."""
        a, b, n = C.c_double(), C.c_double(), C.c_uint64()
        self._check(self.lib.mq_get_level_timing(self.h, int(level), C.byref(a), C.byref(b), C.byref(n)))
        return a.value, b.value, n.value

    def mq_get_kernel_timing(self, level):
        """(percta_ms, stream_ms): the per-sample kernel alone and the streaming solves."""
        a, b = C.c_double(), C.c_double()
        self._check(self.lib.mq_get_kernel_timing(self.h, int(level), C.byref(a), C.byref(b)))
        return a.value, b.value

    def mq_get_launch_count(self):
        n = C.c_uint64()
        self._check(self.lib.mq_get_launch_count(self.h, C.byref(n)))
        return n.value

    def mq_eval_point(self, level, y, want_u=False):
        y = np.ascontiguousarray(y, dtype=np.float64)
        lH, lh, lp = C.c_double(), C.c_double(), C.c_double()
        nc = self.levels[level].n_coarse
        u = np.zeros((nc - 1) ** 2) if want_u else None
        st = self.lib.mq_eval_point(self.h, int(level), _dptr(y), C.byref(lH), C.byref(lh), C.byref(lp),
                                    _dptr(u) if u is not None else None)
        self._check(st)
        return (lH.value, lh.value, lp.value, u) if want_u else (lH.value, lh.value, lp.value)

    def mq_get_stats(self):
        s = mq_stats()
        self._check(self.lib.mq_get_stats(self.h, C.byref(s), C.sizeof(s)))
        return s.as_dict()

    # --- building blocks ----------------------------------------------------------------------
    def mq_lattice_points_device(self, level, k0, k1, d_Y):
        self._check(self.lib.mq_lattice_points_device(self.h, int(level), int(k0), int(k1), _tptr(d_Y)))

    def mq_coefficients_device(self, n, s, d_Y, B, ldy, d_a):
        self._check(self.lib.mq_coefficients_device(self.h, int(n), int(s), _tptr(d_Y), int(B), int(ldy),
                                                    _tptr(d_a)))

    def mq_reaction_coefficients_device(self, n, s, d_Y, B, ldy, d_b):
        self._check(self.lib.mq_reaction_coefficients_device(self.h, int(n), int(s), _tptr(d_Y), int(B), int(ldy),
                                                             _tptr(d_b)))

    def mq_apply_operator_device(self, n, B, d_a, which, sigma, d_x, d_y):
        self._check(self.lib.mq_apply_operator_device(self.h, int(n), int(B), _tptr(d_a), int(which), float(sigma),
                                                      _tptr(d_x), _tptr(d_y)))


def mq_twogrid_samples_noalloc(n_fine, n_coarse, n_prev, precision, B, d_a_fine, d_a_coarse, d_a_prev, d_out,
                               d_stat, d_outer, tol_linear=0.0, stream=None):
    """The allocation-free per-sample entry point (see the header): device tensors in and out,
    asynchronous on ``stream`` (a cudaStream_t value or None for the default stream)."""
    lib = load()
    st = lib.mq_twogrid_samples_noalloc(int(n_fine), int(n_coarse), int(n_prev), int(precision), int(B),
                                        _tptr(d_a_fine), _tptr(d_a_coarse), _tptr(d_a_prev), float(tol_linear),
                                        _tptr(d_out), _tptr(d_stat), _tptr(d_outer),
                                        C.c_void_p(stream) if stream else None)
    if st != MQ_OK:
        raise MQError(st, "mq_twogrid_samples_noalloc failed")


def mq_measure_fp64_peak(device=0):
    """(TFLOP/s, ms) of the library's FP64 fused multiply-add throughput kernel on `device`."""
    lib = load()
    tf, ms = C.c_double(), C.c_double()
    st = lib.mq_measure_fp64_peak(int(device), C.byref(tf), C.byref(ms))
    if st != MQ_OK:
        raise MQError(st, "mq_measure_fp64_peak failed")
    return tf.value, ms.value


def mq_estimate_sums(level_sums, npoints, shared=False):
    """Estimate from per-level shift sums (list of arrays [R_l]) and points per level: returns
    (mean, std_err, level_mean [L+1], level_var [L+1])."""
    lib = load()
    L1 = len(level_sums)
    R = (C.c_int32 * L1)(*[len(x) for x in level_sums])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in level_sums]))
    n = (C.c_uint64 * L1)(*[int(v) for v in npoints])
    m, se = C.c_double(), C.c_double()
    lm, lv = np.zeros(L1), np.zeros(L1)
    st = lib.mq_estimate_sums(L1, R, _dptr(flat), n, int(bool(shared)), C.byref(m), C.byref(se), _dptr(lm), _dptr(lv))
    if st != MQ_OK:
        raise MQError(st, "mq_estimate_sums: bad arguments")
    return m.value, se.value, lm, lv


def mq_cbc_embedded_lattice(m_min: int, m_max: int, s: int, decay: float = 2.0) -> np.ndarray:
    lib = load()
    z = np.zeros(s, dtype=np.uint32)
    st = lib.mq_cbc_embedded_lattice(int(m_min), int(m_max), int(s), float(decay),
                                     z.ctypes.data_as(C.POINTER(C.c_uint32)))
    if st != MQ_OK:
        raise MQError(st, "mq_cbc_embedded_lattice: bad arguments")
    return z


def mq_cbc_lattice(N: int, s: int, decay: float = 2.0) -> np.ndarray:
    lib = load()
    z = np.zeros(s, dtype=np.uint32)
    st = lib.mq_cbc_lattice(int(N), int(s), float(decay), z.ctypes.data_as(C.POINTER(C.c_uint32)))
    if st != MQ_OK:
        raise MQError(st, "mq_cbc_lattice: bad arguments")
    return z
