"""ctypes declarations of libsmgpu.so (include/smgpu.h, include/smgen.h).

Loading never falls back to anything: if the shared library has not been
built, every entry point raises.  Build it with ``python -c "import
__graft_entry__ as g; g.build()"`` (or ``python paper_1012_2547_gb300/build.py``).
"""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsmgpu.so")

SM_OK, SM_EINVAL, SM_ENOMEM, SM_ECUDA, SM_ETIMEOUT, SM_ETRUNC = range(6)
VARIANTS = {"auto": 0, "shiftor": 1, "qgram": 2, "linear": 3, "dfa": 4}
VARIANT_NAMES = {v: k for k, v in VARIANTS.items()}
TUNE_M_BUCKETS = 12
TUNE_S_BUCKETS = 9


class SmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _strerror(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


class sm_config(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("word_bits", ctypes.c_uint32), ("tile", ctypes.c_uint32)]


class sm_plan_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint32), ("variant", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("word_bits", ctypes.c_uint32), ("hist", ctypes.c_uint32),
                ("tile_starts", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64),
                ("kernel", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class sm_plan_layout(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in (
        "m", "variant", "kernel", "bytes", "q", "s", "word_bits", "hist", "entry_bytes", "tile_starts",
        "off_masks", "off_pattern", "off_border", "off_qgram_bitmap", "bitmap_bits", "off_qgram_slots",
        "slot_bits", "off_qgram_offsets", "off_classes_tab", "off_automaton", "classes", "reserved")]


class sm_query(ctypes.Structure):
    _fields_ = [("text", ctypes.c_void_p), ("n", ctypes.c_uint64), ("plan", ctypes.c_void_p),
                ("out_pos", ctypes.c_void_p), ("cap", ctypes.c_uint64),
                ("out_count", ctypes.c_void_p)]


_st = ctypes.c_int
_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64

# name -> (restype, argtypes); every function declared in include/*.h.
SIGNATURES = {
    "sm_prepare": (_st, [_vp, _u32, _u32, _vp, ctypes.POINTER(_vp)]),
    "sm_prepare_ex": (_st, [_vp, _u32, _u32, ctypes.POINTER(sm_config), _vp, ctypes.POINTER(_vp)]),
    "sm_prepare_many": (_st, [_vp, ctypes.POINTER(_u32), _u32, _u32, ctypes.POINTER(sm_config),
                              _vp, ctypes.POINTER(_vp)]),
    "sm_plan_free": (_st, [_vp]),
    "sm_plan_free_many": (_st, [ctypes.POINTER(_vp), _u32]),
    "sm_plan_info": (_st, [_vp, ctypes.POINTER(sm_plan_desc)]),
    "sm_selftest_wait": (_st, [_vp]),
    "sm_plan_image": (_st, [_vp, _u32, _u32, ctypes.POINTER(sm_config), _vp, ctypes.c_size_t,
                            ctypes.POINTER(sm_plan_layout)]),
    "sm_search": (_st, [_vp, _u64, _vp, _u32, _vp, _u64, _vp, _vp]),
    "sm_search_plan": (_st, [_vp, _vp, _u64, _vp, _u64, _vp, _vp]),
    "sm_search_noalloc": (_st, [_vp, _u64, _vp, _u32, _vp, _u64, _vp, _vp]),
    "sm_search_batch": (_st, [ctypes.POINTER(sm_query), _u32, _vp]),
    "sm_batch_workspace_size": (_st, [ctypes.POINTER(sm_query), _u32, ctypes.POINTER(ctypes.c_size_t)]),
    "sm_search_batch_async": (_st, [ctypes.POINTER(sm_query), _u32, _vp, ctypes.c_size_t, _vp]),
    "sm_batch_create": (_st, [ctypes.POINTER(sm_query), _u32, _u32, _vp, ctypes.POINTER(_vp)]),
    "sm_batch_launch": (_st, [_vp, _vp]),
    "sm_batch_free": (_st, [_vp]),
    "sm_tuning_set": (_st, [ctypes.POINTER(sm_config), _u32]),
    "sm_tuning_get": (_st, [ctypes.POINTER(sm_config), _u32]),
    "sm_tuning_reset": (_st, []),
    "sm_sync": (_st, [_vp]),
    "sm_kernel_launches": (_u64, []),
    "sm_shutdown": (_st, []),
    "sm_strerror": (ctypes.c_char_p, [_st]),
    "sm_gen_text": (_st, [_vp, _u64, _u64, _u64, _u32, _vp, _u32, _vp, _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libsmgpu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: the CUDA library must be built first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def _strerror(status: int) -> str:
    try:
        return load().sm_strerror(status).decode()
    except Exception:  # library missing while formatting an error
        return f"status {status}"


def check(status: int, what: str = "") -> None:
    if status != SM_OK:
        raise SmError(status, what)
