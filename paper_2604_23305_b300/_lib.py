"""ctypes declarations of the C ABI in include/gateau.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgateau_b300.so")

OK, EINVAL, ENOMEM, ECUDA, EORDER, ESTATE, EDEVICE, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7, -8
PREC_FP32, PREC_BF16X3 = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
SCAN_STARE, SCAN_DAISY, SCAN_RASTER, SCAN_CUSTOM = 0, 1, 2, 3
DISP_FILTERBANK, DISP_LORENTZIAN, DISP_CUSTOM = 0, 1, 2
STAGE_REFLECTIVE, STAGE_OHMIC, STAGE_REFRACTIVE = 0, 1, 2
T_SKY = -1.0
NOISE_WHITE, NOISE_PINK = 1, 2
STATUS_PWV_CLAMPED, STATUS_WAIT_TIMEOUT, STATUS_BAD_INDEX = 1, 2, 4
VEC_NU, VEC_WEIGHT, VEC_ETA_FILT, VEC_C0, VEC_C1, VEC_C2, VEC_PINK_A, VEC_PINK_R, VEC_PINK_D, VEC_TB_A, VEC_TB_B = range(11)
PHASE_ROWS, PHASE_SPECTRUM, PHASE_CONTRACT, PHASE_PINK, PHASE_COUNT = 0, 1, 2, 3, 4

_STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EORDER: "EORDER",
                 ESTATE: "ESTATE", EDEVICE: "EDEVICE", ETIMEOUT: "ETIMEOUT", EUNSUPPORTED: "EUNSUPPORTED"}

dp = C.POINTER(C.c_double)
fp = C.POINTER(C.c_float)


class PlanDesc(C.Structure):
    _fields_ = [("n_freq", C.c_int), ("f_lo_hz", C.c_double), ("f_hi_hz", C.c_double),
                ("f_sample_hz", C.c_double), ("n_pix", C.c_int), ("pix_offsets_rad", dp),
                ("T_atm_K", C.c_double), ("T_cmb_K", C.c_double), ("h_column_m", C.c_double),
                ("wind_mps", C.c_double), ("eta_taper", C.c_double), ("rho_surf_m", C.c_double),
                ("eta_pol", C.c_double), ("delta_al_J", C.c_double), ("eta_pb", C.c_double),
                ("seed", C.c_ulonglong), ("precision", C.c_int), ("noise_flags", C.c_int),
                ("pink_f_min_hz", C.c_double)]


class Stage(C.Structure):
    _fields_ = [("kind", C.c_int), ("T_K", C.c_double), ("eta", C.c_double), ("eta_nu", dp),
                ("eps_ref", C.c_double), ("nu_ref_hz", C.c_double), ("d_m", C.c_double),
                ("n_index", C.c_double), ("tan_delta", C.c_double), ("T_refl_K", C.c_double),
                ("ar_coated", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("n_freq", C.c_int), ("n_freq_padded", C.c_int), ("n_ch", C.c_int), ("n_pix", C.c_int),
                ("n_pole", C.c_int), ("next_t0", C.c_longlong), ("device_bytes", C.c_size_t),
                ("staged_inputs", C.c_int), ("tile_groups", C.c_int), ("tile_half", C.c_int),
                ("ring_a", C.c_int), ("ring_b", C.c_int), ("tune_ms", C.c_double)]


class TileChoice(C.Structure):
    _fields_ = [("n_groups", C.c_int), ("n_half", C.c_int), ("ring_b", C.c_int), ("ring_a", C.c_int),
                ("ms", C.c_double), ("default_ms", C.c_double), ("candidates", C.c_int)]


class ServerDesc(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_active", C.c_int), ("chunk_samples", C.c_longlong),
                ("max_chunk_bytes", C.c_size_t), ("n_streams", C.c_int), ("dry_run", C.c_int),
                ("dry_seconds_per_sample", C.c_double), ("n_builders", C.c_int), ("shared_launches", C.c_int)]


class Request(C.Structure):
    _fields_ = [("arrival_s", C.c_double), ("nt", C.c_longlong), ("n_pix", C.c_int), ("n_ch", C.c_int),
                ("device_bytes", C.c_size_t), ("host_out", C.c_void_p)]


class ServerStats(C.Structure):
    _fields_ = [("n_requests", C.c_int), ("n_done", C.c_int), ("n_failed", C.c_int),
                ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double), ("mean_latency_s", C.c_double),
                ("max_latency_s", C.c_double), ("makespan_s", C.c_double), ("detector_samples", C.c_double),
                ("throughput", C.c_double), ("peak_bytes", C.c_size_t), ("peak_active", C.c_int),
                ("overlap", C.c_double), ("rounds", C.c_longlong), ("mean_round", C.c_double)]


PlanP = C.c_void_p
ServerP = C.c_void_p
PLAN_FACTORY = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_int)
PLAN_RELEASE = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_void_p)

# name -> (restype, argtypes); mirrors include/gateau.h one to one.
SIGNATURES = {
    "gateau_version": (C.c_char_p, []),
    "gateau_last_error": (C.c_char_p, []),
    "gateau_device_count": (C.c_int, []),
    "gateau_plan_create": (C.c_int, [C.POINTER(PlanDesc), C.POINTER(PlanP)]),
    "gateau_plan_destroy": (None, [PlanP]),
    "gateau_set_source_cube": (C.c_int, [PlanP, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int]),
    "gateau_set_atmosphere_screen": (C.c_int, [PlanP, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                                               C.c_double, C.c_int]),
    "gateau_set_atmosphere_table": (C.c_int, [PlanP, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int,
                                              C.c_int]),
    "gateau_set_cascade": (C.c_int, [PlanP, C.c_int, C.POINTER(Stage)]),
    "gateau_set_dispersive_element": (C.c_int, [PlanP, C.c_int, C.c_int, dp, dp, dp, dp]),
    "gateau_set_pink_noise": (C.c_int, [PlanP, dp, dp]),
    "gateau_set_scan": (C.c_int, [PlanP, C.c_int, dp, C.c_int, C.c_double, C.c_double, C.c_void_p,
                                  C.c_longlong, C.c_int]),
    "gateau_plan_prepare": (C.c_int, [PlanP]),
    "gateau_set_output_kelvin": (C.c_int, [PlanP, C.c_int, C.c_double, C.c_double, C.c_int]),
    "gateau_set_pink_timmer_koenig": (C.c_int, [PlanP, C.c_longlong]),
    "gateau_mean_zenith_pwv": (C.c_int, [PlanP, C.c_longlong, C.POINTER(C.c_double)]),
    "gateau_beam_far_field": (C.c_int, [dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_void_p, C.c_void_p]),
    "gateau_convolve_source": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "gateau_smooth_screen": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                       C.c_void_p]),
    "gateau_common_mode": (C.c_int, [PlanP, C.c_longlong, C.c_longlong, C.c_void_p, C.c_void_p, C.c_double,
                                     C.c_double, C.c_void_p]),
    "gateau_run": (C.c_int, [PlanP, C.c_longlong, C.c_longlong, C.c_void_p, C.c_void_p]),
    "gateau_run_host": (C.c_int, [PlanP, C.c_longlong, C.c_longlong, C.c_void_p, C.c_void_p]),
    "gateau_run_batch": (C.c_int, [C.POINTER(PlanP), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "gateau_plan_status": (C.c_int, [PlanP, C.POINTER(C.c_uint)]),
    "gateau_plan_get_info": (C.c_int, [PlanP, C.POINTER(PlanInfo)]),
    "gateau_plan_get_vector": (C.c_int, [PlanP, C.c_int, dp, C.c_size_t]),
    "gateau_plan_get_state": (C.c_int, [PlanP, C.POINTER(C.c_longlong), dp]),
    "gateau_plan_set_state": (C.c_int, [PlanP, C.c_longlong, dp]),
    "gateau_hex_offsets": (C.c_int, [C.c_int, C.c_double, dp, C.c_int, C.POINTER(C.c_int)]),
    "gateau_plan_set_timing": (C.c_int, [PlanP, C.c_int]),
    "gateau_plan_set_wait_budget": (C.c_int, [PlanP, C.c_longlong]),
    "gateau_plan_set_tiles": (C.c_int, [PlanP, C.c_int, C.c_int]),
    "gateau_plan_autotune": (C.c_int, [PlanP, C.c_longlong, C.c_void_p, C.c_void_p]),
    "gateau_plan_get_timing": (C.c_int, [PlanP, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "gateau_plan_estimate_bytes": (C.c_int, [C.POINTER(PlanDesc), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_int, C.c_longlong, C.c_longlong, C.POINTER(C.c_size_t)]),
    "gateau_server_create": (C.c_int, [C.POINTER(ServerDesc), C.POINTER(ServerP)]),
    "gateau_server_destroy": (None, [ServerP]),
    "gateau_server_run": (C.c_int, [ServerP, C.POINTER(Request), C.c_int, PLAN_FACTORY, PLAN_RELEASE, C.c_void_p,
                                    C.POINTER(ServerStats)]),
    "gateau_server_request_result": (C.c_int, [ServerP, C.c_int, C.POINTER(C.c_int), dp, dp, dp]),
    "gateau_pink_noise_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                            C.c_ulonglong, C.c_longlong, C.c_longlong, C.c_void_p, C.c_void_p,
                                            C.c_void_p]),
}


class GateauError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")


_lib = None


def lib():
    """Load libgateau_b300.so (built in-tree); raises if it is missing -- there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2604_23305_b300.build` "
                              "(the simulator has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != OK:
        raise GateauError(status, lib().gateau_last_error().decode(errors="replace"))
