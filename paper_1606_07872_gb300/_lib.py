"""ctypes declarations of the libasp C-ABI (include/asp.h), argument
marshalling only: every step of the computation runs in libasp's kernels."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libasp.so")

ASP_KMAX = 50
ASP_STATIC_KMAX = 8
ASP_STATIC_GRID_MAX = 32
ASP_STATIC_SCRATCH_BYTES = 5964032

ASP_OK = 0
STATUS_NAMES = {0: "ASP_OK", 1: "ASP_ERR_INVALID_ARG", 2: "ASP_ERR_CUDA", 3: "ASP_ERR_OOM", 4: "ASP_ERR_NAN",
                5: "ASP_ERR_TIMEOUT", 6: "ASP_ERR_NOT_CONVERGED", 7: "ASP_ERR_STATE", 8: "ASP_ERR_UNSUPPORTED",
                9: "ASP_ERR_CAPACITY"}
ASP_INIT_AUTO, ASP_INIT_SIMPLE, ASP_INIT_SMOOTH = 0, 1, 2
ASP_PEAK_SIMPLE, ASP_PEAK_SMOOTH = 0, 1
ASP_SUB_AUTO, ASP_SUB_DIRECT, ASP_SUB_FFT = 0, 1, 2
ASP_SUB_FFT_MIN_PIXELS = 512 * 512
ASP_ELL_KMAX = 33
ASP_LM_CONVERGED, ASP_LM_CAP, ASP_LM_STALLED = 0, 1, 2
ASP_STOP_NONE, ASP_STOP_ITER, ASP_STOP_NOISE, ASP_STOP_CAPACITY = 0, 1, 2, 3


class asp_gauss(C.Structure):
    _fields_ = [("amp", C.c_double), ("x", C.c_double), ("y", C.c_double), ("width", C.c_double)]


class asp_component(C.Structure):
    _fields_ = [("flux", C.c_double), ("amp", C.c_double), ("x", C.c_double), ("y", C.c_double),
                ("width", C.c_double), ("is_point", C.c_int32), ("reserved", C.c_int32)]


class asp_gauss_ell(C.Structure):
    _fields_ = [("amp", C.c_double), ("x", C.c_double), ("y", C.c_double), ("pxx", C.c_double),
                ("pxy", C.c_double), ("pyy", C.c_double)]


class asp_component_ell(C.Structure):
    _fields_ = [("flux", C.c_double), ("amp", C.c_double), ("x", C.c_double), ("y", C.c_double),
                ("sxx", C.c_double), ("sxy", C.c_double), ("syy", C.c_double), ("is_point", C.c_int32),
                ("reserved", C.c_int32)]


class asp_peak(C.Structure):
    _fields_ = [("index", C.c_int64), ("x", C.c_int32), ("y", C.c_int32), ("value", C.c_float),
                ("scale", C.c_float), ("mode", C.c_int32), ("scale_index", C.c_int32),
                ("a0", C.c_double), ("x0", C.c_double), ("y0", C.c_double), ("w0", C.c_double)]


class asp_fit_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("passes", C.c_int32), ("status", C.c_int32), ("k", C.c_int32),
                ("x0", C.c_int32), ("x1", C.c_int32), ("y0", C.c_int32), ("y1", C.c_int32),
                ("chi2_init", C.c_double), ("chi2_final", C.c_double), ("lambda_", C.c_double),
                ("pixel_evals", C.c_int64)]


class asp_params(C.Structure):
    _fields_ = [("gain", C.c_float), ("k_max", C.c_int32), ("lm_max_iter", C.c_int32),
                ("lm_lambda0", C.c_double), ("lm_rtol", C.c_double), ("lm_xtol", C.c_double),
                ("noise_sigma", C.c_float), ("stop_ksigma", C.c_float), ("n_scales", C.c_int32),
                ("area_frac", C.c_float), ("init_mode", C.c_int32), ("tau", C.c_double),
                ("retained_cap", C.c_int32), ("max_components", C.c_int32),
                ("fit_px_per_cta", C.c_int32), ("major_every", C.c_int32),
                ("sub_mode", C.c_int32)]


class asp_cycle_stats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("components", C.c_int64), ("pixel_evals", C.c_int64),
                ("lm_iters", C.c_int64), ("lm_passes", C.c_int64), ("peak_abs", C.c_double),
                ("stop_reason", C.c_int32), ("reserved", C.c_int32), ("fit_flops", C.c_double),
                ("sub_flops", C.c_double), ("sub_bytes", C.c_double), ("smooth_flops", C.c_double),
                ("fit_pass_ms", C.c_double), ("fit_reduce_ms", C.c_double), ("fit_solve_ms", C.c_double),
                ("fit_factor_ms", C.c_double), ("fit_subst_ms", C.c_double), ("fit_refinements", C.c_int64),
                ("fit_fallbacks", C.c_int64), ("learned_fits", C.c_int64), ("learned_refits", C.c_int64),
                ("learned_kept", C.c_int64), ("fit_ex2", C.c_double), ("smooth_iters", C.c_int64)]


class asp_iter_record(C.Structure):
    _fields_ = [("t", C.c_int32), ("mode", C.c_int32), ("k", C.c_int32), ("status", C.c_int32),
                ("iters", C.c_int32), ("passes", C.c_int32), ("x0", C.c_int32), ("x1", C.c_int32),
                ("y0", C.c_int32), ("y1", C.c_int32), ("new_index", C.c_int32), ("n_terms", C.c_int32),
                ("peak_value", C.c_float), ("init_scale", C.c_float), ("chi2_init", C.c_double),
                ("chi2_final", C.c_double), ("a0", C.c_double), ("x0_init", C.c_double),
                ("y0_init", C.c_double), ("w0", C.c_double)]


class asp_batch_tuning(C.Structure):
    _fields_ = [("px_per_cta", C.c_int32), ("share_policy", C.c_int32), ("n_candidates", C.c_int32),
                ("best_ms", C.c_double), ("default_ms", C.c_double)]


class asp_alu_peaks(C.Structure):
    _fields_ = [("sms", C.c_int32), ("reserved", C.c_int32), ("fp32_fma_tflops", C.c_double),
                ("fp32_fma2_tflops", C.c_double), ("ex2_gops", C.c_double), ("sm_mhz_fma", C.c_double),
                ("sm_mhz_fma2", C.c_double), ("sm_mhz_ex2", C.c_double), ("fma_per_sm_clk", C.c_double),
                ("fma2_per_sm_clk", C.c_double), ("ex2_per_sm_clk", C.c_double)]


class asp_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


_P = C.c_void_p
_I = C.c_int
# name -> argtypes (all return asp_status unless listed in _RESTYPES)
SIGNATURES = {
    "asp_status_string": [_I],
    "asp_default_params": [C.POINTER(asp_params)],
    "asp_init": [C.POINTER(asp_params), _I, _I, _P, _P, _P, C.POINTER(_P)],
    "asp_init_host": [C.POINTER(asp_params), _I, _I, _P, _P, _P, C.POINTER(_P)],
    "asp_destroy": [_P],
    "asp_last_error": [_P],
    "asp_get_beam": [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                     C.POINTER(C.c_double)],
    "asp_find_peak": [_P, _I, C.POINTER(asp_peak)],
    "asp_fit_active_set": [_P, C.POINTER(asp_gauss), _I, _I, C.POINTER(asp_gauss), C.POINTER(asp_fit_info)],
    "asp_fit_lm": [_P, C.POINTER(asp_gauss), _I, _I, C.POINTER(asp_gauss), C.c_double, _I, C.POINTER(asp_gauss),
                   C.POINTER(asp_fit_info), C.POINTER(asp_gauss), C.POINTER(C.c_double)],
    "asp_eval_normal_equations": [_P, C.POINTER(asp_gauss), _I, _I, _I, _I, _I, _I, _P, _P, _P],
    "asp_fit_2004": [_P, C.POINTER(asp_gauss), _I, _I, C.c_double, C.POINTER(asp_gauss), C.POINTER(asp_fit_info)],
    "asp_subtract": [_P, C.POINTER(asp_component), _I, C.c_float],
    "asp_subtract_beam": [_P, C.POINTER(asp_component), _I, C.c_float],
    "asp_fit_beam_elliptical": [_P, C.POINTER(asp_gauss_ell)],
    "asp_fit_elliptical": [_P, C.POINTER(asp_gauss_ell), _I, _I, C.POINTER(asp_gauss_ell), C.POINTER(asp_fit_info)],
    "asp_deconvolve_elliptical": [_P, C.POINTER(asp_gauss_ell), _I, C.POINTER(asp_gauss_ell),
                                  C.POINTER(asp_component_ell)],
    "asp_minor_cycle": [_P, _I, C.POINTER(asp_cycle_stats)],
    "asp_smooth": [_P, _I, _P],
    "asp_num_scales": [_P, C.POINTER(_I), _P],
    "asp_residual_ptr": [_P, C.POINTER(_P)],
    "asp_copy_residual": [_P, _P, _I],
    "asp_set_residual": [_P, _P, _I],
    "asp_refresh_peak": [_P],
    "asp_get_components": [_P, C.POINTER(asp_component), _I, C.POINTER(_I)],
    "asp_get_history": [_P, C.POINTER(asp_iter_record), _I, C.POINTER(_I)],
    "asp_get_stats": [_P, C.POINTER(asp_cycle_stats)],
    "asp_get_state": [_P, C.POINTER(asp_component), _I, C.POINTER(_I), C.POINTER(_I), _I, C.POINTER(_I),
                      C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "asp_set_state": [_P, C.POINTER(asp_component), _I, C.POINTER(_I), _I, C.c_int64, C.c_double, C.c_double],
    "asp_reset": [_P, _P, _I, _P, _I],
    "asp_get_last_fit": [_P, C.POINTER(asp_gauss), _I, C.POINTER(_I), C.POINTER(asp_fit_info)],
    "asp_set_profiling": [_P, _I],
    "asp_get_kernel_times": [_P, C.POINTER(asp_kernel_time), _I, C.POINTER(_I)],
    "asp_launch_count": [_P, C.POINTER(C.c_int64)],
    "asp_fit_static": [_P, _I, _I, C.POINTER(asp_gauss), _I, _I, C.c_double, C.POINTER(asp_params),
                       C.POINTER(asp_gauss), C.POINTER(asp_fit_info), _P],
    "asp_measure_alu_peaks": [C.POINTER(asp_alu_peaks)],
    "asp_save_state": [_P, C.c_char_p],
    "asp_load_state": [_P, C.c_char_p],
    "asp_batch_create": [C.POINTER(asp_params), _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(_P), C.POINTER(_P), _I,
                         _P, C.POINTER(_P)],
    "asp_batch_destroy": [_P],
    "asp_batch_reset": [_P],
    "asp_batch_minor_cycle": [_P, _I, C.POINTER(asp_cycle_stats)],
    "asp_batch_run_queue": [_P, _I, _I, _I, C.POINTER(asp_cycle_stats)],
    "asp_batch_autotune": [_P, _I, C.POINTER(asp_batch_tuning)],
    "asp_batch_image": [_P, _I, C.POINTER(_P)],
    "asp_batch_launch_count": [_P, C.POINTER(C.c_int64)],
    "asp_batch_fit_joint": [_P, _P, _I, _I, _P, _P, _P, C.POINTER(asp_fit_info)],
    "asp_batch_set_mlp": [_P, _P, _I],
    "asp_mlp_gemm": [_P, _I, _P, _I, _P, _I, _I, _I, _I, _P],
    "asp_mlp_num_params": [C.POINTER(C.c_longlong)],
    "asp_mlp_create": [_P, _I, _P, C.POINTER(_P)],
    "asp_mlp_destroy": [_P],
    "asp_mlp_set_data": [_P, _P, _P, C.c_longlong],
    "asp_mlp_step": [_P, C.POINTER(_I), _I, C.c_float, _I, C.POINTER(C.c_float), _P],
    "asp_mlp_predict": [_P, _P, _I, _P],
    "asp_mlp_get_params": [_P, _P],
    "asp_set_mlp": [_P, _P, _I],
    "asp_set_harvest": [_P, _P, _P, _I],
}
_RESTYPES = {"asp_status_string": C.c_char_p, "asp_default_params": None, "asp_last_error": C.c_char_p}


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libasp.so and declare every exported symbol; raises if missing."""
    if not os.path.exists(path):
        raise ImportError(f"libasp.so is not built ({path}); run `python -m paper_1606_07872_gb300.build` "
                          "(the CUDA library has no CPU fallback)")
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPES.get(name, C.c_int)
    return lib
