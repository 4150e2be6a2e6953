"""ctypes binding of libhf.so (include/hf.h).  Argument marshalling only:
every step of the path runs in the library's CUDA kernels.  Device buffers
are torch CUDA tensors (passed as raw pointers); streams are torch streams.

The library must be built (``paper_1711_05017_b300.build.build()``); there is
no fallback: a missing library or a missing GPU raises."""
import ctypes
import os

from .build import LIB

HF_OK, HF_EINVAL, HF_ENOMEM, HF_EBUDGET, HF_ECUDA, HF_ETIMEOUT, HF_ENOTREADY, HF_EUNSUPPORTED = range(8)
STATUS_NAMES = {0: "HF_OK", 1: "HF_EINVAL", 2: "HF_ENOMEM", 3: "HF_EBUDGET", 4: "HF_ECUDA",
                5: "HF_ETIMEOUT", 6: "HF_ENOTREADY", 7: "HF_EUNSUPPORTED"}
HF_STATIONARY, HF_MOVING = 0, 1
HF_E, HF_F, HF_T, HF_TORQUE_F64, HF_TORQUE_C = 0x1, 0x2, 0x4, 0x10, 0x200
HF_PREC_SPLIT_BF16, HF_PREC_SPLIT_F16, HF_SPECTRAL, HF_TA = 0x20, 0x40, 0x80, 0x100
HF_CKPT_PART, HF_CKPT_FIELDSET, HF_CKPT_SESSION = 1, 2, 3

_vp = ctypes.c_void_p
_i = ctypes.c_int
_u = ctypes.c_uint
_sz = ctypes.c_size_t
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); the ABI of include/hf.h
SIGNATURES = {
    "hf_version": (ctypes.c_char_p, []),
    "hf_last_error": (ctypes.c_char_p, []),
    "hf_inject_alloc_failure": (None, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "hf_arena_selftest": (ctypes.c_int64, [ctypes.c_uint64, _sz, _i]),
    "hf_ctx_create": (_i, [_i, _sz, ctypes.POINTER(_vp)]),
    "hf_ctx_destroy": (None, [_vp]),
    "hf_ctx_reserved_bytes": (_sz, [_vp]),
    "hf_ctx_preload": (_i, [_vp, ctypes.POINTER(_i)]),
    "hf_ctx_resident_queries": (_i, [_vp, _i]),
    "hf_density_build": (_i, [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp]),
    "hf_part_create": (_i, [_vp, _i, _vp, _i, ctypes.POINTER(_vp), _vp]),
    "hf_part_release": (None, [_vp]),
    "hf_part_update": (_i, [_vp, _vp, _vp]),
    "hf_profile_enable": (_i, [_vp, _i]),
    "hf_profile_read": (_i, [_vp]),
    "hf_profile_entry": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_double)]),
    "hf_profile_reset": (None, [_vp]),
    "hf_fieldset_create": (_i, [_vp, _i, _i, _u, ctypes.POINTER(_vp)]),
    "hf_fieldset_compute": (_i, [_vp, _vp, _vp, _fp, _i, _vp, _vp]),
    "hf_fieldset_build": (_i, [_vp, _vp, _vp, _fp, _i, _u, ctypes.POINTER(_vp), _vp]),
    "hf_fieldset_get": (_i, [_vp, _i, _i, _vp, _vp]),
    "hf_fieldset_field_ptr": (_i, [_vp, _i, _i, ctypes.POINTER(_vp)]),
    "hf_fieldset_n": (_i, [_vp]),
    "hf_fieldset_rotations": (_i, [_vp]),
    "hf_fieldset_flags": (_u, [_vp]),
    "hf_fieldset_release": (None, [_vp]),
    "hf_query": (_i, [_vp, _fp, _fp, _i, _fp]),
    "hf_query_batch": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "hf_resample": (_i, [_i, _vp, _fp, _vp, _vp]),
    "hf_rfft3d_scratch_bytes": (_sz, [_i]),
    "hf_rfft3d": (_i, [_i, _vp, _vp, _vp, _vp]),
    "hf_fields_scratch_bytes": (_sz, [_i]),
    "hf_fields": (_i, [_vp, _vp, _vp, _fp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hf_torque": (_i, [_vp, _i, _i, _fp, _vp, _vp, _u, _ip, _vp]),
    "hf_fields_noalloc": (_i, [_i, _vp, _vp, _fp, _vp, _vp, _vp, _vp, _vp]),
    "hf_ctx_budget_bytes": (_sz, [_vp]),
    "hf_part_n": (_i, [_vp]),
    "hf_fieldset_bytes": (_sz, [_i, _i, _u]),
    "hf_server_create": (_i, [_vp, _i, _i, ctypes.POINTER(_vp)]),
    "hf_server_destroy": (None, [_vp]),
    "hf_server_session_open": (_i, [_vp, _vp, _vp, _ip]),
    "hf_server_session_close": (_i, [_vp, _i]),
    "hf_server_submit": (_i, [_vp, _i, _fp, _i, _u, ctypes.POINTER(ctypes.c_int64)]),
    "hf_server_request_state": (_i, [_vp, ctypes.c_int64, _ip, ctypes.POINTER(ctypes.c_double)]),
    "hf_server_query": (_i, [_vp, _i, _fp, _fp, _i, _fp]),
    "hf_server_field_ptr": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_vp)]),
    "hf_server_field_get": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "hf_server_stats_get": (_i, [_vp, _vp]),
    "hf_server_log_open": (_i, [_vp, ctypes.c_char_p, _i]),
    "hf_server_log_close": (_i, [_vp]),
    "hf_server_query_latencies": (_i, [_vp, _fp, _i]),
    "hf_server_set_chunk_bytes": (_i, [_vp, _sz]),
    "hf_server_request_chunks": (_i, [_vp, ctypes.c_int64, _ip, _ip]),
    "hf_server_session_counts": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "hf_server_session_save": (_i, [_vp, _i, ctypes.c_char_p]),
    "hf_server_session_restore": (_i, [_vp, _i, ctypes.c_char_p]),
    "hf_part_save": (_i, [_vp, ctypes.c_char_p, _vp]),
    "hf_part_load": (_i, [_vp, ctypes.c_char_p, ctypes.POINTER(_vp), _vp]),
    "hf_fieldset_save": (_i, [_vp, ctypes.c_char_p, _vp]),
    "hf_fieldset_load": (_i, [_vp, ctypes.c_char_p, ctypes.POINTER(_vp), _vp]),
    "hf_checkpoint_info": (_i, [ctypes.c_char_p, _ip, _ip, _ip, ctypes.POINTER(_u)]),
    "hf_server_trace": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double), _i]),
    "hf_rotation_chunks": (_i, [_fp, _i, _i, _i, _ip, _ip, _ip, _i]),
    "hf_server_drive_queries": (_i, [_vp, _i, _ip, _fp, _i, ctypes.c_double, _i, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "hf_batch_create": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ip, _u, _i, ctypes.POINTER(_vp)]),
    "hf_batch_set_rotations": (_i, [_vp, _i, _fp]),
    "hf_batch_capture": (_i, [_vp, _i]),
    "hf_batch_launch": (_i, [_vp, _vp]),
    "hf_batch_capture_queue": (_i, [_vp, _i, ctypes.c_longlong, _i]),
    "hf_batch_status": (_i, [_vp, _vp, _ip, _ip]),
    "hf_batch_fieldset": (_i, [_vp, _i, ctypes.POINTER(_vp)]),
    "hf_batch_slots": (_i, [_vp]),
    "hf_batch_release": (None, [_vp]),
    "hf_autotune": (_i, [_vp, _i, ctypes.c_char_p, _ip, _ip, ctypes.POINTER(ctypes.c_double)]),
    "hf_tune_set": (_i, [_vp, _i, _i, _i]),
    "hf_tune_get": (_i, [_vp, _i, _ip, _ip, ctypes.POINTER(ctypes.c_double)]),
    "hf_tune_tiles": (_i, [_vp, _i, _i, _ip, _ip]),
    "hf_tune_lanes": (_i, [_vp, _i, _i, _ip]),
    "hf_tc_timeouts": (_i, [_i]),
    "hf_bulk_timeouts": (_i, [_i]),
    "hf_bulk_selftest": (_i, [_i, _i, _ip]),
    "hf_part_spectral": (_i, [_vp, _i, _vp]),
    "hf_part_spectral_os": (_i, [_vp]),
    "hf_lowpass_query": (_i, [_vp, _vp, _i, _fp, _fp, _fp]),
    "hf_lowpass_query_batch": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp]),
    "hf_part_moments": (_i, [_vp, _vp]),
    "hf_density_mesh": (_i, [_vp, _i, _vp, _i, _vp, _i, ctypes.c_double, ctypes.c_double, _i, _vp, _vp, _vp]),
}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("superseded", ctypes.c_int64), ("evicted", ctypes.c_int64),
                ("queries", ctypes.c_int64), ("rotations_completed", ctypes.c_int64), ("queued", ctypes.c_int),
                ("running", ctypes.c_int), ("sessions", ctypes.c_int), ("reserved_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("chunks_submitted", ctypes.c_int64),
                ("chunks_completed", ctypes.c_int64), ("chunks_resident", ctypes.c_int), ("chunk_bytes", ctypes.c_size_t),
                ("pool_reserved_bytes", ctypes.c_size_t), ("pool_reserved_high", ctypes.c_size_t),
                ("arena_bytes", ctypes.c_size_t), ("arena_free_bytes", ctypes.c_size_t),
                ("arena_largest_free", ctypes.c_size_t), ("arena_refusals", ctypes.c_int64),
                ("resident_queries", ctypes.c_int64), ("resident_timeouts", ctypes.c_int64),
                ("resident_live", ctypes.c_int)]

_lib = None


def lib():
    """The loaded libhf.so with every ABI signature set (raises if not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libhf.so is not built ({LIB}); run paper_1711_05017_b300.build.build()")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class HFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, allow=()):
    if status != HF_OK and status not in allow:
        raise HFError(status, lib().hf_last_error().decode(errors="replace"))
    return status


def fptr(arr):
    """float* of a contiguous float32 numpy array (host)."""
    return arr.ctypes.data_as(_fp)
