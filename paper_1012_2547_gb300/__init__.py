"""GB300-native exact string matching (Python binding of libsmgpu).

Every function here only marshals arguments for the C ABI of
``include/smgpu.h``; all matching work runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: if
``libsmgpu.so`` is missing or no GPU is present, calls raise.

The operation (Section 1 of the paper): all 0-based start positions i with
t[i..i+m-1] = p, strictly increasing, overlapping occurrences included.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib
from ._lib import SM_ETRUNC, SmError, VARIANTS, VARIANT_NAMES, check, sm_config, sm_query

__all__ = [
    "Plan", "PlanArray", "prepare", "prepare_many", "prepare_array", "plan_image", "search", "search_into", "search_plan", "search_batch",
    "batch_workspace_size", "search_batch_async", "query_array", "search_batch_async_array",
    "batch_workspace_size_array",
    "Batch", "sync", "gen_text", "tuning_get", "tuning_set", "tuning_reset", "kernel_launches",
    "SmError", "SM_ETRUNC", "lib_path",
]


def _torch():
    import torch
    return torch


def lib_path() -> str:
    return _lib.LIB_PATH


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _config(variant="auto", q=0, word_bits=0, tile=0):
    if isinstance(variant, str):
        variant = VARIANTS[variant]
    return sm_config(int(variant), int(q), int(word_bits), int(tile))


@dataclass
class PlanInfo:
    m: int
    variant: str
    q: int
    word_bits: int
    hist: bool
    tile_starts: int
    device_bytes: int
    kernel: int


class Plan:
    """A prepared pattern (library-owned device tables)."""

    def __init__(self, handle: int, pattern: bytes):
        self._h = handle
        self.pattern = pattern

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("plan was freed")
        return self._h

    @property
    def m(self) -> int:
        return len(self.pattern)

    def info(self) -> PlanInfo:
        d = _lib.sm_plan_desc()
        check(_lib.load().sm_plan_info(self.handle, ctypes.byref(d)), "sm_plan_info")
        return PlanInfo(d.m, VARIANT_NAMES.get(d.variant, str(d.variant)), d.q, d.word_bits,
                        bool(d.hist), d.tile_starts, d.device_bytes, d.kernel)

    def free(self):
        if self._h:
            _lib.load().sm_plan_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _as_bytes(pattern) -> bytes:
    if isinstance(pattern, (bytes, bytearray, memoryview)):
        return bytes(pattern)
    import numpy as np
    return np.ascontiguousarray(pattern, dtype=np.uint8).tobytes()


def prepare(pattern, sigma_hint: int = 0, variant="auto", q: int = 0, word_bits: int = 0,
            tile: int = 0, stream=None) -> Plan:
    """sm_prepare / sm_prepare_ex: preprocess one pattern."""
    p = _as_bytes(pattern)
    h = ctypes.c_void_p()
    lib = _lib.load()
    if variant == "auto" and not (q or word_bits or tile):
        st = lib.sm_prepare(p, len(p), sigma_hint, _stream_ptr(stream), ctypes.byref(h))
    else:
        cfg = _config(variant, q, word_bits, tile)
        st = lib.sm_prepare_ex(p, len(p), sigma_hint, ctypes.byref(cfg), _stream_ptr(stream),
                               ctypes.byref(h))
    check(st, "sm_prepare")
    return Plan(h.value, p)


def plan_image(pattern, sigma_hint: int = 0, variant="auto", q: int = 0, word_bits: int = 0,
               tile: int = 0):
    """sm_plan_image: the device image of a plan, built in host memory with
    no CUDA call.  Returns (image as a uint8 numpy array, layout dict)."""
    import numpy as np
    p = _as_bytes(pattern)
    lib = _lib.load()
    cfg = None if variant == "auto" and not (q or word_bits or tile) else _config(variant, q, word_bits, tile)
    cfgp = ctypes.byref(cfg) if cfg is not None else None
    lay = _lib.sm_plan_layout()
    check(lib.sm_plan_image(p, len(p), sigma_hint, cfgp, None, 0, ctypes.byref(lay)), "sm_plan_image")
    img = np.zeros(lay.bytes, dtype=np.uint8)
    check(lib.sm_plan_image(p, len(p), sigma_hint, cfgp, img.ctypes.data, img.nbytes, ctypes.byref(lay)),
          "sm_plan_image")
    d = {f: getattr(lay, f) for f, _ in lay._fields_}
    d["variant"] = VARIANT_NAMES.get(d["variant"], str(d["variant"]))
    return img, d


def prepare_many(patterns, sigma_hint: int = 0, variant="auto", q: int = 0, word_bits: int = 0,
                 tile: int = 0, stream=None) -> list[Plan]:
    """sm_prepare_many: preprocess many patterns with one device copy."""
    pats = [_as_bytes(p) for p in patterns]
    if not pats:
        return []
    blob = b"".join(pats)
    lens = (ctypes.c_uint32 * len(pats))(*[len(p) for p in pats])
    out = (ctypes.c_void_p * len(pats))()
    cfg = _config(variant, q, word_bits, tile)
    auto = variant == "auto" and not (q or word_bits or tile)
    check(_lib.load().sm_prepare_many(blob, lens, len(pats), sigma_hint,
                                      None if auto else ctypes.byref(cfg), _stream_ptr(stream), out),
          "sm_prepare_many")
    return [Plan(out[i], pats[i]) for i in range(len(pats))]


class PlanArray:
    """The plans of one sm_prepare_many call, kept as an array of handles
    (`handles`, uint64), without a Python object per plan, and released
    together (sm_plan_free_many).  query_array takes it in place of a list
    of Plan objects."""

    def __init__(self, handles, lengths):
        self.handles = handles
        self.lengths = lengths

    def __len__(self) -> int:
        return len(self.handles)

    def info(self, i: int) -> PlanInfo:
        d = _lib.sm_plan_desc()
        check(_lib.load().sm_plan_info(int(self.handles[i]), ctypes.byref(d)), "sm_plan_info")
        return PlanInfo(d.m, VARIANT_NAMES.get(d.variant, str(d.variant)), d.q, d.word_bits,
                        bool(d.hist), d.tile_starts, d.device_bytes, d.kernel)

    def free(self):
        h = self.handles
        if h is not None and len(h):
            _lib.load().sm_plan_free_many(h.ctypes.data_as(ctypes.POINTER(ctypes.c_void_p)), len(h))
        self.handles = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def prepare_array(patterns, sigma_hint: int = 0, variant="auto", q: int = 0, word_bits: int = 0,
                  tile: int = 0, stream=None) -> PlanArray:
    """sm_prepare_many over `patterns` (a list of bytes objects, or a pair
    (concatenated bytes, uint32 lengths)), returning a PlanArray: the same
    plans as prepare_many without a Python object per plan."""
    import numpy as np
    if isinstance(patterns, tuple):
        blob, lens = patterns
        lens = np.ascontiguousarray(lens, dtype=np.uint32)
    else:
        blob = b"".join(patterns)
        lens = np.fromiter(map(len, patterns), dtype=np.uint32, count=len(patterns))
    n = len(lens)
    handles = np.zeros(n, dtype=np.uint64)
    if n == 0:
        return PlanArray(handles, lens)
    cfg = _config(variant, q, word_bits, tile)
    auto = variant == "auto" and not (q or word_bits or tile)
    check(_lib.load().sm_prepare_many(blob, lens.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n,
                                      sigma_hint, None if auto else ctypes.byref(cfg),
                                      _stream_ptr(stream),
                                      handles.ctypes.data_as(ctypes.POINTER(ctypes.c_void_p))),
          "sm_prepare_many")
    return PlanArray(handles, lens)


def _ptr(t):
    return 0 if t is None else t.data_ptr()


def search_into(text, pattern_or_plan, out_pos, out_count, n: int | None = None, cap: int | None = None,
                stream=None) -> None:
    """Enqueue one search (sm_search / sm_search_plan); no host sync.

    text: CUDA uint8 tensor; out_pos: CUDA int64/uint64 tensor (or None);
    out_count: CUDA int64 tensor with at least one element.
    """
    n = text.numel() if n is None else n
    cap = (0 if out_pos is None else out_pos.numel()) if cap is None else cap
    lib = _lib.load()
    if isinstance(pattern_or_plan, Plan):
        st = lib.sm_search_plan(pattern_or_plan.handle, _ptr(text), n, _ptr(out_pos), cap,
                                _ptr(out_count), _stream_ptr(stream))
    else:
        p = _as_bytes(pattern_or_plan)
        st = lib.sm_search(_ptr(text), n, p, len(p), _ptr(out_pos), cap, _ptr(out_count),
                           _stream_ptr(stream))
    check(st, "sm_search")


def search(text, pattern_or_plan, cap: int | None = None, stream=None, retry: bool = True):
    """All occurrences as a sorted int64 CUDA tensor (synchronises).

    With ``cap`` None the first attempt allows min(n, 65536) positions and a
    second one exactly the reported count.  With an explicit ``cap`` and
    ``retry`` False, a truncated result raises SmError(SM_ETRUNC).
    """
    torch = _torch()
    dev = text.device
    n = text.numel()
    first = min(n, 1 << 16) if cap is None else cap
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    out = torch.empty(max(first, 1), dtype=torch.int64, device=dev)
    search_into(text, pattern_or_plan, out, count, n=n, cap=first, stream=stream)
    sync(stream)
    total = int(count.item())
    if total <= first:
        return out[:total]
    if not retry and cap is not None:
        raise SmError(SM_ETRUNC, f"{total} occurrences, cap {cap}")
    out = torch.empty(total, dtype=torch.int64, device=dev)
    search_into(text, pattern_or_plan, out, count, n=n, cap=total, stream=stream)
    sync(stream)
    return out


def search_plan(text, plan: Plan, **kw):
    return search(text, plan, **kw)


def _queries(items):
    arr = (sm_query * len(items))()
    for i, it in enumerate(items):
        text, plan, out_pos, out_count = it[:4]
        n = it[4] if len(it) > 4 and it[4] is not None else text.numel()
        cap = 0 if out_pos is None else out_pos.numel()
        arr[i] = sm_query(_ptr(text), n, plan.handle, _ptr(out_pos), cap, _ptr(out_count))
    return arr


def batch_workspace_size(items) -> int:
    """sm_batch_workspace_size for (text, plan, out_pos, out_count[, n]) tuples."""
    if not items:
        return 0
    arr = _queries(items)
    out = ctypes.c_size_t()
    check(_lib.load().sm_batch_workspace_size(arr, len(items), ctypes.byref(out)),
          "sm_batch_workspace_size")
    return int(out.value)


def search_batch_async(items, workspace, stream=None) -> None:
    """sm_search_batch_async: enqueue a batch in caller-provided device
    workspace (a CUDA uint8 tensor of at least batch_workspace_size bytes,
    256-byte aligned); no allocation, no host sync."""
    if not items:
        return
    arr = _queries(items)
    check(_lib.load().sm_search_batch_async(arr, len(items), workspace.data_ptr(), workspace.numel(),
                                            _stream_ptr(stream)), "sm_search_batch_async")


def query_array(text_ptrs, ns, plans, out_ptrs, caps, count_ptrs):
    """An sm_query array built from raw device pointers (uint64 arrays of
    equal length), without per-query Python objects.  `plans` is a list of
    Plan objects or a PlanArray."""
    import numpy as np
    nq = len(ns)
    a = np.empty((nq, 6), dtype=np.uint64)
    a[:, 0] = text_ptrs
    a[:, 1] = ns
    a[:, 2] = plans.handles if isinstance(plans, PlanArray) else [p.handle for p in plans]
    a[:, 3] = out_ptrs
    a[:, 4] = caps
    a[:, 5] = count_ptrs
    return a


def search_batch_async_array(qarr, workspace_ptr: int, workspace_bytes: int, stream=None) -> None:
    """sm_search_batch_async on an array from query_array."""
    if len(qarr) == 0:
        return
    ptr = ctypes.cast(qarr.ctypes.data, ctypes.POINTER(sm_query))
    check(_lib.load().sm_search_batch_async(ptr, len(qarr), workspace_ptr, workspace_bytes,
                                            _stream_ptr(stream)), "sm_search_batch_async")


def batch_workspace_size_array(qarr) -> int:
    if len(qarr) == 0:
        return 0
    out = ctypes.c_size_t()
    ptr = ctypes.cast(qarr.ctypes.data, ctypes.POINTER(sm_query))
    check(_lib.load().sm_batch_workspace_size(ptr, len(qarr), ctypes.byref(out)),
          "sm_batch_workspace_size")
    return int(out.value)


def search_batch_array(qarr, stream=None) -> None:
    """sm_search_batch on an array from query_array (library workspace)."""
    if len(qarr) == 0:
        return
    ptr = ctypes.cast(qarr.ctypes.data, ctypes.POINTER(sm_query))
    check(_lib.load().sm_search_batch(ptr, len(qarr), _stream_ptr(stream)), "sm_search_batch")


def search_batch(items, stream=None) -> None:
    """sm_search_batch over (text, plan, out_pos, out_count[, n]) tuples."""
    if not items:
        return
    arr = _queries(items)
    check(_lib.load().sm_search_batch(arr, len(items), _stream_ptr(stream)), "sm_search_batch")


class Batch:
    """sm_batch_create / sm_batch_launch: a reusable (graph-captured) batch.

    Keeps references to the tensors and plans it names so they outlive it.
    """

    def __init__(self, items, graph: bool = True, stream=None, pack: bool = True):
        self._keep = list(items)
        arr = _queries(self._keep)
        h = ctypes.c_void_p()
        flags = (0 if graph else 1) | (0 if pack else 2)
        check(_lib.load().sm_batch_create(arr, len(self._keep), flags,
                                          _stream_ptr(stream), ctypes.byref(h)), "sm_batch_create")
        self._h = h.value

    def launch(self, stream=None) -> None:
        check(_lib.load().sm_batch_launch(self._h, _stream_ptr(stream)), "sm_batch_launch")

    def free(self) -> None:
        if self._h:
            _lib.load().sm_batch_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sync(stream=None) -> None:
    """sm_sync: wait for the stream, raise on a device-side timeout."""
    check(_lib.load().sm_sync(_stream_ptr(stream)), "sm_sync")


def gen_text(out, start: int, key: int, sigma: int = 0, thresholds=None, byte_map=None,
             stream=None) -> None:
    """sm_gen_text: fill CUDA uint8 tensor ``out`` with text bytes
    [start, start + out.numel()) of the counter-based generator."""
    nthr = 0 if thresholds is None else thresholds.numel()
    check(_lib.load().sm_gen_text(_ptr(out), int(start), out.numel(), int(key), int(sigma),
                                  _ptr(thresholds), nthr, _ptr(byte_map), _stream_ptr(stream)),
          "sm_gen_text")


def tuning_get() -> list[dict]:
    n = _lib.TUNE_M_BUCKETS * _lib.TUNE_S_BUCKETS
    arr = (sm_config * n)()
    check(_lib.load().sm_tuning_get(arr, n), "sm_tuning_get")
    return [dict(variant=c.variant, q=c.q, word_bits=c.word_bits, tile=c.tile) for c in arr]


def tuning_set(cells) -> None:
    n = _lib.TUNE_M_BUCKETS * _lib.TUNE_S_BUCKETS
    if len(cells) != n:
        raise ValueError(f"need {n} cells")
    arr = (sm_config * n)(*[sm_config(c.get("variant", 0), c.get("q", 0), c.get("word_bits", 0),
                                      c.get("tile", 0)) for c in cells])
    check(_lib.load().sm_tuning_set(arr, n), "sm_tuning_set")


def tuning_reset() -> None:
    check(_lib.load().sm_tuning_reset(), "sm_tuning_reset")


def kernel_launches() -> int:
    return int(_lib.load().sm_kernel_launches())
