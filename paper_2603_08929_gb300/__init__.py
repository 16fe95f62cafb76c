"""GB300 (sm_103a) bsort: the bsort key order for 8..64-bit integers and IEEE
floats, computed by hand-written CUDA kernels behind a C ABI (``include/bsort.h``).

This package is a thin binding: it marshals arguments to the shared library
``_lib/libbsort.so`` and raises on error.  Every step of a sort runs in the
library's kernels; there is no CPU path.  Build the library with
``paper_2603_08929_gb300.build.build()`` (done by ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "DTYPES", "BsortError", "lib", "bsort_keys", "bsort_keys_ws", "bsort_keys_host", "bsort_keys_noalloc",
    "bsort_keys_segmented", "segmented_workspace_bytes", "Graph", "Server", "sort_", "sort_segmented_",
    "bsort_keys_partial_ws", "selftest_bounded_wait", "top_digit_counts",
    "workspace_bytes", "Handle", "sort_", "status_string",
]

BSORT_OK = 0
MODE_PINGPONG, MODE_INPLACE = 0, 1

# bsort_dtype codes, in the order of include/bsort.h
DTYPES = ["uint8", "int8", "uint16", "int16", "float16", "uint32", "int32", "float32",
          "uint64", "int64", "float64", "bfloat16", "uint128", "int128"]
KEY_BYTES = {"uint8": 1, "int8": 1, "uint16": 2, "int16": 2, "float16": 2, "bfloat16": 2, "uint32": 4, "int32": 4,
             "float32": 4, "uint64": 8, "int64": 8, "float64": 8, "uint128": 16, "int128": 16}
_CODE = {name: i for i, name in enumerate(DTYPES)}

KERNEL_KINDS = ["init", "hist", "scan", "classify", "scatter", "finish", "fill",
                "count_hist", "count_scan", "count_fill"]

_PROFILE_MAX = 1024


class _Record(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("call", ctypes.c_int32),
                ("ms", ctypes.c_float), ("keys", ctypes.c_uint64), ("counted_bytes", ctypes.c_uint64)]


class _Profile(ctypes.Structure):
    _fields_ = [("num_records", ctypes.c_int32), ("num_calls", ctypes.c_int32),
                ("num_launches", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("finish_units_counting", ctypes.c_uint64), ("finish_units_compare", ctypes.c_uint64),
                ("finish_units_lsd", ctypes.c_uint64), ("finish_units_counting_fast", ctypes.c_uint64),
                ("rec", _Record * _PROFILE_MAX)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("num_slots", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_request_keys", ctypes.c_size_t), ("batch_keys", ctypes.c_size_t), ("mode", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class _Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("lane", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_uint64), ("t_admit_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64)]


class _ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("in_flight_bytes", ctypes.c_size_t),
                ("peak_in_flight_bytes", ctypes.c_size_t), ("max_concurrent_slots", ctypes.c_int32),
                ("num_lanes", ctypes.c_int32), ("slot_workspace_bytes", ctypes.c_size_t),
                ("launches", ctypes.c_uint64), ("grouped_sorts", ctypes.c_uint64)]


class _LaneInfo(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("num_slots", ctypes.c_int32), ("budget_bytes", ctypes.c_size_t),
                ("in_flight_bytes", ctypes.c_size_t), ("peak_in_flight_bytes", ctypes.c_size_t),
                ("queued_bytes", ctypes.c_size_t), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64)]


class _Tuning(ctypes.Structure):
    _fields_ = [("radix_bits", ctypes.c_int32), ("unit_keys", ctypes.c_int32), ("merge_keys", ctypes.c_int32),
                ("chunk_tiles", ctypes.c_int32)]


class BsortError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__((what + ": " if what else "") + status_string(status))


_lib = None


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("the bsort CUDA library is not built (%s missing); run "
                              "paper_2603_08929_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        vp, sz, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        L.bsort_status_string.argtypes = [i]
        L.bsort_status_string.restype = ctypes.c_char_p
        L.bsort_keys.argtypes = [vp, sz, i, i, vp]
        L.bsort_keys.restype = i
        L.bsort_workspace_bytes.argtypes = [sz, i, i, ctypes.POINTER(sz)]
        L.bsort_workspace_bytes.restype = i
        L.bsort_handle_create.argtypes = [ctypes.POINTER(vp)]
        L.bsort_handle_create.restype = i
        L.bsort_handle_destroy.argtypes = [vp]
        L.bsort_handle_destroy.restype = i
        L.bsort_keys_ws.argtypes = [vp, vp, sz, i, i, i, vp, sz, vp]
        L.bsort_keys_ws.restype = i
        L.bsort_keys_host.argtypes = [vp, sz, i, i, vp]
        L.bsort_keys_host.restype = i
        L.bsort_get_error.argtypes = [vp, vp]
        L.bsort_get_error.restype = i
        L.bsort_handle_set_profiling.argtypes = [vp, i]
        L.bsort_handle_set_profiling.restype = i
        L.bsort_handle_get_profile.argtypes = [vp, ctypes.POINTER(_Profile)]
        L.bsort_handle_get_profile.restype = i
        L.bsort_last_launch_count.argtypes = [vp, ctypes.POINTER(i)]
        L.bsort_last_launch_count.restype = i
        L.bsort_keys_noalloc.argtypes = [vp, sz, i, i, vp]
        L.bsort_keys_noalloc.restype = i
        L.bsort_segmented_workspace_bytes.argtypes = [sz, sz, i, ctypes.POINTER(sz)]
        L.bsort_segmented_workspace_bytes.restype = i
        L.bsort_segmented_workspace_bytes_tuned.argtypes = [sz, sz, i, ctypes.POINTER(_Tuning), ctypes.POINTER(sz)]
        L.bsort_segmented_workspace_bytes_tuned.restype = i
        L.bsort_pairs_workspace_bytes.argtypes = [sz, i, ctypes.POINTER(sz)]
        L.bsort_pairs_workspace_bytes.restype = i
        L.bsort_pairs_workspace_bytes_tuned.argtypes = [sz, i, ctypes.POINTER(_Tuning), ctypes.POINTER(sz)]
        L.bsort_pairs_workspace_bytes_tuned.restype = i
        L.bsort_pairs_ws.argtypes = [vp, vp, vp, sz, vp, sz, i, i, vp, sz, vp]
        L.bsort_pairs_ws.restype = i
        L.bsort_keys_segmented_ws.argtypes = [vp, vp, sz, vp, sz, i, i, vp, sz, vp]
        L.bsort_keys_segmented_ws.restype = i
        L.bsort_keys_segmented.argtypes = [vp, sz, vp, sz, i, i, vp]
        L.bsort_keys_segmented.restype = i
        L.bsort_graph_create.argtypes = [vp, vp, sz, i, i, vp, sz, ctypes.POINTER(vp)]
        L.bsort_graph_create.restype = i
        L.bsort_graph_create_segmented.argtypes = [vp, vp, sz, vp, sz, i, i, vp, sz, ctypes.POINTER(vp)]
        L.bsort_graph_create_segmented.restype = i
        L.bsort_graph_launch.argtypes = [vp, vp]
        L.bsort_graph_launch.restype = i
        L.bsort_graph_error.argtypes = [vp, vp]
        L.bsort_graph_error.restype = i
        L.bsort_graph_destroy.argtypes = [vp]
        L.bsort_graph_destroy.restype = i
        L.bsort_handle_set_tuning.argtypes = [vp, i, ctypes.POINTER(_Tuning)]
        L.bsort_handle_set_tuning.restype = i
        L.bsort_workspace_bytes_tuned.argtypes = [sz, i, i, ctypes.POINTER(_Tuning), ctypes.POINTER(sz)]
        L.bsort_workspace_bytes_tuned.restype = i
        L.bsort_keys_partial_ws.argtypes = [vp, vp, sz, i, i, i, vp, sz, vp]
        L.bsort_keys_partial_ws.restype = i
        L.bsort_selftest_bounded_wait.argtypes = [vp]
        L.bsort_selftest_bounded_wait.restype = i
        L.bsort_top_digit_counts.argtypes = [vp, sz, i, i, i, vp, vp]
        L.bsort_top_digit_counts.restype = i
        L.bsort_last_aux_bytes.argtypes = [vp, ctypes.POINTER(sz)]
        L.bsort_last_aux_bytes.restype = i
        L.bsort_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(vp)]
        L.bsort_server_create.restype = i
        L.bsort_server_submit.argtypes = [vp, vp, sz, i, i, ctypes.c_uint64]
        L.bsort_server_submit.restype = i
        L.bsort_server_poll.argtypes = [vp, ctypes.POINTER(_Completion), sz, ctypes.POINTER(sz)]
        L.bsort_server_poll.restype = i
        L.bsort_server_stats.argtypes = [vp, ctypes.POINTER(_ServerInfo)]
        L.bsort_server_create_multi.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(ctypes.c_int32),
                                                ctypes.c_int32, ctypes.POINTER(vp)]
        L.bsort_server_create_multi.restype = i
        L.bsort_server_pick_device.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
        L.bsort_server_pick_device.restype = i
        L.bsort_server_lane_stats.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(_LaneInfo)]
        L.bsort_server_lane_stats.restype = i
        L.bsort_server_stats.restype = i
        L.bsort_server_drain.argtypes = [vp, ctypes.c_double]
        L.bsort_server_drain.restype = i
        L.bsort_server_pause.argtypes = [vp, i]
        L.bsort_server_pause.restype = i
        L.bsort_server_destroy.argtypes = [vp]
        L.bsort_server_destroy.restype = i
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().bsort_status_string(int(status)).decode()


def _check(status: int, what: str) -> None:
    if status != BSORT_OK:
        raise BsortError(status, what)


def _dtype_code(dtype) -> int:
    name = str(dtype).replace("torch.", "")
    if name not in _CODE:
        raise TypeError("bsort does not sort dtype %s" % name)
    return _CODE[name]


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _device_tensor(t):
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("bsort sorts contiguous tensors only")
    return t


def _keys(keys, dtype=None):
    """(pointer, key count, dtype code) of a contiguous CUDA tensor.  With
    ``dtype`` ("uint128" / "int128", which torch lacks, or any other name)
    the tensor's bytes are read as keys of that dtype: 16-byte keys, low
    64 bits first, e.g. an int64 tensor of shape (n, 2)."""
    _device_tensor(keys)
    if dtype is None:
        return ctypes.c_void_p(keys.data_ptr()), keys.numel(), _dtype_code(keys.dtype)
    name = str(dtype).replace("torch.", "")
    nbytes = keys.numel() * keys.element_size()
    kb = KEY_BYTES[name]
    if nbytes % kb:
        raise ValueError("%d bytes are not whole %s keys" % (nbytes, name))
    return ctypes.c_void_p(keys.data_ptr()), nbytes // kb, _dtype_code(name)


def bsort_keys(keys, descending: bool = False, stream=None, dtype=None) -> None:
    """Sorts a contiguous CUDA tensor in place (C ABI ``bsort_keys``);
    ``dtype`` reads its bytes as keys of another dtype (see ``_keys``)."""
    ptr, n, code = _keys(keys, dtype)
    _check(lib().bsort_keys(ptr, n, code, int(bool(descending)), _stream_ptr(stream)), "bsort_keys")


_inplace_handle = None


def sort_(keys, descending: bool = False, mode: str = "pingpong", stream=None):
    """Sorts a contiguous CUDA tensor in place and returns it.  mode
    "pingpong" (default: ``bsort_keys``, cached workspace) or "inplace" (a
    workspace of ``workspace_bytes(..., MODE_INPLACE)`` allocated by torch for
    the call, no alternate copy of the keys)."""
    global _inplace_handle
    if mode == "pingpong":
        bsort_keys(keys, descending=descending, stream=stream)
    elif mode == "inplace":
        import torch
        if _inplace_handle is None:
            _inplace_handle = Handle()
        ws = torch.empty(max(1, workspace_bytes(keys.numel(), keys.dtype, mode=MODE_INPLACE)), dtype=torch.uint8,
                         device=keys.device)
        bsort_keys_ws(_inplace_handle, keys, ws, descending=descending, stream=stream, mode=MODE_INPLACE)
    else:
        raise ValueError("mode must be 'pingpong' or 'inplace'")
    return keys


def _tuning(t):
    if t is None:
        return None
    return ctypes.byref(_Tuning(int(t.get("radix_bits", 0)), int(t.get("unit_keys", 0)),
                                int(t.get("merge_keys", 0)), int(t.get("chunk_tiles", 0))))


def workspace_bytes(n: int, dtype, mode: int = MODE_PINGPONG, tuning: dict = None) -> int:
    """Workspace bytes for bsort_keys_ws; ``tuning`` (a dict with radix_bits,
    unit_keys, merge_keys, chunk_tiles) sizes it for a handle tuned that way."""
    out = ctypes.c_size_t(0)
    if tuning is None:
        _check(lib().bsort_workspace_bytes(int(n), _dtype_code(dtype), int(mode), ctypes.byref(out)),
               "bsort_workspace_bytes")
    else:
        _check(lib().bsort_workspace_bytes_tuned(int(n), _dtype_code(dtype), int(mode), _tuning(tuning),
                                                 ctypes.byref(out)), "bsort_workspace_bytes_tuned")
    return int(out.value)


class Handle:
    """An explicit library handle (profiling state, error word, last-call stats)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().bsort_handle_create(ctypes.byref(h)), "bsort_handle_create")
        self._h = h

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            lib().bsort_handle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def set_profiling(self, enable: bool = True):
        _check(lib().bsort_handle_set_profiling(self._h, int(bool(enable))), "bsort_handle_set_profiling")

    def launch_count(self) -> int:
        v = ctypes.c_int(0)
        _check(lib().bsort_last_launch_count(self._h, ctypes.byref(v)), "bsort_last_launch_count")
        return int(v.value)

    def profile(self) -> dict:
        """Per-launch records of the calls since the last read (then cleared)."""
        p = _Profile()
        _check(lib().bsort_handle_get_profile(self._h, ctypes.byref(p)), "bsort_handle_get_profile")
        recs = []
        for r in p.rec[: p.num_records]:
            recs.append({"kind": KERNEL_KINDS[r.kind], "level": int(r.level), "call": int(r.call),
                         "ms": float(r.ms), "keys": int(r.keys),
                         "counted_bytes": int(r.counted_bytes)})
        return {"calls": int(p.num_calls), "launches": int(p.num_launches), "records": recs,
                "finish_units": {"counting": int(p.finish_units_counting), "compare": int(p.finish_units_compare),
                                 "lsd": int(p.finish_units_lsd),
                                 "counting_fast": int(p.finish_units_counting_fast)}}

    def set_tuning(self, key_bytes: int, tuning: dict = None) -> None:
        """MSD tuning for 4- or 8-byte keys (``bsort_handle_set_tuning``);
        None restores the defaults."""
        _check(lib().bsort_handle_set_tuning(self._h, int(key_bytes), _tuning(tuning)), "bsort_handle_set_tuning")

    def last_aux_bytes(self) -> int:
        """Auxiliary device bytes of the last call (``bsort_last_aux_bytes``)."""
        out = ctypes.c_size_t(0)
        _check(lib().bsort_last_aux_bytes(self._h, ctypes.byref(out)), "bsort_last_aux_bytes")
        return int(out.value)

    def get_error(self, stream=None) -> int:
        return int(lib().bsort_get_error(self._h, _stream_ptr(stream)))


def bsort_keys_ws(handle: Handle, keys, workspace, descending: bool = False, stream=None,
                  mode: int = MODE_PINGPONG, dtype=None) -> None:
    """Sorts with a caller-provided device workspace (a uint8 CUDA tensor);
    ``dtype`` as for ``bsort_keys``."""
    kp, kn, code = _keys(keys, dtype)
    _device_tensor(workspace)
    _check(lib().bsort_keys_ws(handle.ptr, kp, kn, code, int(bool(descending)), int(mode),
                               ctypes.c_void_p(workspace.data_ptr()),
                               workspace.numel() * workspace.element_size(), _stream_ptr(stream)),
           "bsort_keys_ws")


def pairs_workspace_bytes(n: int, dtype, tuning8: dict = None) -> int:
    """Workspace bytes of a key-value sort of n keys (``tuning8`` is
    validated and has no effect: the key-value levels have a fixed shape)."""
    out = ctypes.c_size_t(0)
    if tuning8 is None:
        _check(lib().bsort_pairs_workspace_bytes(int(n), _dtype_code(dtype), ctypes.byref(out)),
               "bsort_pairs_workspace_bytes")
    else:
        _check(lib().bsort_pairs_workspace_bytes_tuned(int(n), _dtype_code(dtype), _tuning(tuning8),
                                                       ctypes.byref(out)), "bsort_pairs_workspace_bytes_tuned")
    return int(out.value)


def bsort_pairs_ws(handle: Handle, keys, workspace, values=None, indices=None, descending: bool = False,
                   stream=None) -> None:
    """Stable key-value sort (C ABI ``bsort_pairs_ws``): ``keys`` sorted in
    place, ``values`` (None or a CUDA tensor of as many 1-, 2-, 4- or 8-byte
    elements) permuted in place with them, ``indices`` (None or an int64 CUDA
    tensor of as many elements) set to the input position of each output
    element.  Equal keys keep their input order."""
    _device_tensor(keys)
    _device_tensor(workspace)
    n = keys.numel()
    vptr, vbytes = None, 0
    if values is not None:
        _device_tensor(values)
        if values.numel() != n:
            raise ValueError("values must have as many elements as keys")
        vptr, vbytes = ctypes.c_void_p(values.data_ptr()), values.element_size()
    iptr = None
    if indices is not None:
        _device_tensor(indices)
        if indices.numel() != n or str(indices.dtype) != "torch.int64":
            raise ValueError("indices must be an int64 tensor with as many elements as keys")
        iptr = ctypes.c_void_p(indices.data_ptr())
    _check(lib().bsort_pairs_ws(handle.ptr, ctypes.c_void_p(keys.data_ptr()), vptr, vbytes, iptr, n,
                                _dtype_code(keys.dtype), int(bool(descending)), ctypes.c_void_p(workspace.data_ptr()),
                                workspace.numel() * workspace.element_size(), _stream_ptr(stream)),
           "bsort_pairs_ws")


_pairs_handle = None


def sort_pairs_(keys, values=None, descending: bool = False, return_indices: bool = False, stream=None):
    """Stable key-value sort in place with a workspace allocated by torch for
    the call.  Returns (keys, values, indices), indices an int64 tensor of
    input positions when ``return_indices`` (else None)."""
    import torch
    global _pairs_handle
    if _pairs_handle is None:
        _pairs_handle = Handle()
    ws = torch.empty(max(1, pairs_workspace_bytes(keys.numel(), keys.dtype)), dtype=torch.uint8, device=keys.device)
    idx = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device) if return_indices else None
    bsort_pairs_ws(_pairs_handle, keys, ws, values=values, indices=idx, descending=descending, stream=stream)
    return keys, values, idx


def argsort(keys, descending: bool = False, stream=None):
    """Stable argsort of a CUDA tensor: the int64 input positions in sorted
    order.  ``keys`` is left unchanged (a copy of it is sorted)."""
    return sort_pairs_(keys.clone(), descending=descending, return_indices=True, stream=stream)[2]


def bsort_keys_noalloc(keys, descending: bool = False, stream=None) -> None:
    """Sorts in place with no device allocation: the scratch is a fixed array
    inside the library (C ABI ``bsort_keys_noalloc``; see include/bsort.h for
    the size limit and the rule that overlapping calls must not run at once)."""
    _device_tensor(keys)
    _check(lib().bsort_keys_noalloc(ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                    _dtype_code(keys.dtype), int(bool(descending)), _stream_ptr(stream)),
           "bsort_keys_noalloc")


def segmented_workspace_bytes(n: int, num_segments: int, dtype, tuning: dict = None) -> int:
    """Workspace bytes of a segmented sort; ``tuning`` sizes it for a handle
    tuned that way."""
    out = ctypes.c_size_t(0)
    if tuning is None:
        _check(lib().bsort_segmented_workspace_bytes(int(n), int(num_segments), _dtype_code(dtype),
                                                     ctypes.byref(out)), "bsort_segmented_workspace_bytes")
    else:
        _check(lib().bsort_segmented_workspace_bytes_tuned(int(n), int(num_segments), _dtype_code(dtype),
                                                           _tuning(tuning), ctypes.byref(out)),
               "bsort_segmented_workspace_bytes_tuned")
    return int(out.value)


def _offsets(offsets):
    _device_tensor(offsets)
    if offsets.element_size() != 8:
        raise TypeError("segment offsets must be a 64-bit integer CUDA tensor")
    return ctypes.c_void_p(offsets.data_ptr()), offsets.numel() - 1


def bsort_keys_segmented(keys, offsets, descending: bool = False, stream=None, handle=None, workspace=None,
                         dtype=None) -> None:
    """Sorts every segment keys[offsets[s]:offsets[s+1]] in place (C ABI
    ``bsort_keys_segmented``; with ``handle`` and ``workspace``:
    ``bsort_keys_segmented_ws``).  ``offsets``: int64 CUDA tensor, S + 1
    entries, in keys; ``dtype`` as for ``bsort_keys``."""
    kp, kn, code = _keys(keys, dtype)
    op, nseg = _offsets(offsets)
    if handle is None:
        _check(lib().bsort_keys_segmented(kp, kn, op, nseg, code, int(bool(descending)), _stream_ptr(stream)),
               "bsort_keys_segmented")
    else:
        _device_tensor(workspace)
        _check(lib().bsort_keys_segmented_ws(handle.ptr, kp, kn, op, nseg, code, int(bool(descending)),
                                             ctypes.c_void_p(workspace.data_ptr()),
                                             workspace.numel() * workspace.element_size(), _stream_ptr(stream)),
               "bsort_keys_segmented_ws")


def sort_segmented_(keys, offsets, descending: bool = False, stream=None):
    """Sorts each segment [offsets[i], offsets[i+1]) of a CUDA tensor in place
    (``bsort_keys_segmented``) and returns the tensor."""
    bsort_keys_segmented(keys, offsets, descending=descending, stream=stream)
    return keys


class Graph:
    """A captured CUDA graph of one sort (plain or segmented) on fixed buffers."""

    def __init__(self, handle: Handle, keys, workspace, descending: bool = False, offsets=None):
        _device_tensor(keys)
        _device_tensor(workspace)
        g = ctypes.c_void_p()
        wsb = workspace.numel() * workspace.element_size()
        if offsets is None:
            _check(lib().bsort_graph_create(handle.ptr, ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                            _dtype_code(keys.dtype), int(bool(descending)),
                                            ctypes.c_void_p(workspace.data_ptr()), wsb, ctypes.byref(g)),
                   "bsort_graph_create")
        else:
            op, nseg = _offsets(offsets)
            _check(lib().bsort_graph_create_segmented(handle.ptr, ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                                      op, nseg, _dtype_code(keys.dtype), int(bool(descending)),
                                                      ctypes.c_void_p(workspace.data_ptr()), wsb, ctypes.byref(g)),
                   "bsort_graph_create_segmented")
        self._g = g
        self._keep = (keys, workspace, offsets)

    def launch(self, stream=None):
        _check(lib().bsort_graph_launch(self._g, _stream_ptr(stream)), "bsort_graph_launch")

    def error(self, stream=None) -> int:
        return int(lib().bsort_graph_error(self._g, _stream_ptr(stream)))

    def close(self):
        if self._g:
            lib().bsort_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Server:
    """Continuous-batching sort server (C ABI ``bsort_server_*``), one lane
    per entry of ``devices`` (default: the current device), each with
    ``num_slots`` slots and its own ``hbm_budget_bytes``.  ``submit`` keeps a
    reference to each request's tensor until its completion is polled."""

    def __init__(self, num_slots: int = 8, hbm_budget_bytes: int = 64 << 30, max_request_keys: int = 1 << 24,
                 max_batch: int = 8, batch_keys: int = 1 << 20, mode: int = MODE_PINGPONG, devices=None):
        cfg = _ServerConfig(num_slots, max_batch, hbm_budget_bytes, max_request_keys, batch_keys, int(mode), 0)
        srv = ctypes.c_void_p()
        if devices is None:
            _check(lib().bsort_server_create(ctypes.byref(cfg), ctypes.byref(srv)), "bsort_server_create")
        else:
            arr = (ctypes.c_int32 * len(devices))(*[int(d) for d in devices])
            _check(lib().bsort_server_create_multi(ctypes.byref(cfg), arr, len(devices), ctypes.byref(srv)),
                   "bsort_server_create_multi")
        self._s = srv
        self._live = {}
        self._buf = (_Completion * 4096)()

    def submit(self, keys, descending: bool = False, tag: int = 0) -> None:
        _device_tensor(keys)
        self._live[int(tag)] = keys
        _check(lib().bsort_server_submit(self._s, ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                         _dtype_code(keys.dtype), int(bool(descending)), int(tag)),
               "bsort_server_submit")

    def poll(self) -> list:
        out = []
        while True:
            cnt = ctypes.c_size_t(0)
            _check(lib().bsort_server_poll(self._s, self._buf, len(self._buf), ctypes.byref(cnt)),
                   "bsort_server_poll")
            for c in self._buf[: cnt.value]:
                self._live.pop(int(c.tag), None)
                out.append({"tag": int(c.tag), "status": int(c.status), "slot": int(c.slot), "lane": int(c.lane),
                            "t_submit_ns": int(c.t_submit_ns), "t_admit_ns": int(c.t_admit_ns),
                            "t_done_ns": int(c.t_done_ns)})
            if cnt.value < len(self._buf):
                return out

    def stats(self) -> dict:
        info = _ServerInfo()
        _check(lib().bsort_server_stats(self._s, ctypes.byref(info)), "bsort_server_stats")
        return {f: int(getattr(info, f)) for f, _ in _ServerInfo._fields_ if f != "pad"}

    def lane_stats(self, lane: int) -> dict:
        info = _LaneInfo()
        _check(lib().bsort_server_lane_stats(self._s, int(lane), ctypes.byref(info)), "bsort_server_lane_stats")
        return {f: int(getattr(info, f)) for f, _ in _LaneInfo._fields_}

    def pick_device(self) -> int:
        """Device of the least-loaded lane (``bsort_server_pick_device``)."""
        d = ctypes.c_int32(0)
        _check(lib().bsort_server_pick_device(self._s, ctypes.byref(d)), "bsort_server_pick_device")
        return int(d.value)

    def pause(self, paused: bool = True) -> None:
        _check(lib().bsort_server_pause(self._s, int(bool(paused))), "bsort_server_pause")

    def drain(self, timeout_s: float = 60.0) -> None:
        _check(lib().bsort_server_drain(self._s, float(timeout_s)), "bsort_server_drain")

    def close(self):
        if self._s:
            lib().bsort_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def bsort_keys_partial_ws(handle: Handle, keys, workspace, levels: int, descending: bool = False,
                          stream=None) -> None:
    """Intermediate state after `levels` MSD levels (``bsort_keys_partial_ws``)."""
    _device_tensor(keys)
    _device_tensor(workspace)
    _check(lib().bsort_keys_partial_ws(handle.ptr, ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                       _dtype_code(keys.dtype), int(bool(descending)), int(levels),
                                       ctypes.c_void_p(workspace.data_ptr()),
                                       workspace.numel() * workspace.element_size(), _stream_ptr(stream)),
           "bsort_keys_partial_ws")


def top_digit_counts(keys, bits: int, descending: bool = False, stream=None):
    """Keys per value of the top ``bits`` bits of their sort-order code
    (``bsort_top_digit_counts``): an int64 tensor of 2^bits counts on the
    keys' device; digit d's keys precede digit d + 1's in the sorted output."""
    import torch
    _device_tensor(keys)
    counts = torch.empty(1 << int(bits), dtype=torch.int64, device=keys.device)
    _check(lib().bsort_top_digit_counts(ctypes.c_void_p(keys.data_ptr()), keys.numel(), _dtype_code(keys.dtype),
                                        int(bool(descending)), int(bits), ctypes.c_void_p(counts.data_ptr()),
                                        _stream_ptr(stream)), "bsort_top_digit_counts")
    return counts


def selftest_bounded_wait(stream=None) -> int:
    """Status of ``bsort_selftest_bounded_wait`` (BSORT_ERR_TIMEOUT = 7 expected)."""
    return int(lib().bsort_selftest_bounded_wait(_stream_ptr(stream)))


def bsort_keys_host(keys, descending: bool = False, stream=None, dtype=None) -> None:
    """End-to-end sort of a host array (numpy array or CPU tensor), in place;
    ``dtype`` reads its bytes as keys of that dtype (e.g. "uint128")."""
    if isinstance(keys, np.ndarray):
        if not keys.flags.c_contiguous:
            raise ValueError("bsort sorts contiguous arrays only")
        ptr, n, code = keys.ctypes.data, keys.size, _dtype_code(keys.dtype.name)
        nbytes = keys.nbytes
    else:
        if keys.is_cuda or not keys.is_contiguous():
            raise TypeError("expected a contiguous CPU tensor")
        ptr, n, code = keys.data_ptr(), keys.numel(), _dtype_code(keys.dtype)
        nbytes = keys.numel() * keys.element_size()
    if dtype is not None:
        name = str(dtype).replace("torch.", "")
        n, code = nbytes // KEY_BYTES[name], _dtype_code(name)
    _check(lib().bsort_keys_host(ctypes.c_void_p(ptr), n, code, int(bool(descending)),
                                 _stream_ptr(stream)), "bsort_keys_host")
