"""GB300 Huskysort: stable argsort of byte strings on one GPU.

Thin ctypes binding over the C ABI in include/husky.h (libhusky.so, built
in-tree by ``paper_2012_00866_gb300.build``).  This module only marshals
arguments: every step of the sort runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.

Strings are passed as a uint8 byte tensor plus an int64 (bit-identical to
uint64) offsets tensor of n + 1 entries; string i is
bytes[offsets[i]:offsets[i+1]].
"""

from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhusky.so")

# hs_status
OK = 0
ERR_INVALID_ARG = -1
ERR_CODER_DOMAIN = -2
ERR_OOM = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_INTERNAL = -6
ERR_WORKSPACE = -7
# hs_coder
CODER_AUTO, CODER_ASCII7, CODER_BYTE8, CODER_ALPHA = 0, 1, 2, 3
# hs_mode
MODE_PLAIN, MODE_LEARNED, MODE_AUTO = 0, 1, 2
# hs_index_t
U32, U64 = 0, 1
# hs_numeric
NUM_U64, NUM_I64, NUM_I32, NUM_F64, NUM_F32, NUM_DATETIME = 0, 1, 2, 3, 4, 5

MAX_N = 0x7FFFFFFF

# Every symbol include/husky.h declares (checked by the export test).
EXPORTS = ("hs_encode", "hs_argsort", "hs_argsort_batched", "hs_workspace_size",
           "hs_batched_workspace_size", "hs_stats_enable", "hs_stats_read",
           "hs_argsort_noalloc", "hs_argsort_host", "hs_host_workspace_size", "hs_shutdown",
           "hs_last_error", "hs_version", "hs_encode_numeric", "hs_numeric_workspace_size", "hs_argsort_numeric",
           "hs_autotune", "hs_autotune_choice", "hs_bigint_workspace_size", "hs_argsort_bigint",
           "hs_bigdecimal_workspace_size", "hs_argsort_bigdecimal",
           "hs_rmi_grad", "hs_rmi_leaf_fit", "hs_rmi_sample_indices", "hs_learned_profile",
           "hs_learned_force_bucket_bits", "hs_test_bounded_waits")

NOALLOC_MAX_N = 262144


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double), ("algo_bytes", ctypes.c_double)]

_lib = None


class HuskyError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"hs_status {status}: {message}")
        self.status = status


def load(path: str | None = None):
    """Load libhusky.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        from . import build as _build
        _build.build()
    if not os.path.exists(p):
        raise RuntimeError(f"libhusky.so not found at {p}")
    lib = ctypes.CDLL(p)
    vp, u64, ci, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
    lib.hs_encode.restype = ci
    lib.hs_encode.argtypes = [vp, vp, u64, ci, vp, vp, vp, vp, sz, vp]
    lib.hs_argsort.restype = ci
    lib.hs_argsort.argtypes = [vp, vp, u64, ci, ci, ci, vp, vp, sz, vp]
    lib.hs_argsort_batched.restype = ci
    lib.hs_argsort_batched.argtypes = [vp, vp, vp, u64, u64, ci, vp, vp, sz, vp]
    lib.hs_workspace_size.restype = ci
    lib.hs_workspace_size.argtypes = [u64, u64, ci, ci, ctypes.POINTER(sz)]
    lib.hs_batched_workspace_size.restype = ci
    lib.hs_batched_workspace_size.argtypes = [u64, u64, ctypes.POINTER(sz)]
    lib.hs_rmi_grad.restype = ci
    lib.hs_rmi_grad.argtypes = [vp, vp, vp, ctypes.c_uint32, vp, vp, vp]
    lib.hs_rmi_leaf_fit.restype = ci
    lib.hs_rmi_leaf_fit.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp, vp, vp, vp, vp]
    lib.hs_rmi_sample_indices.restype = ci
    lib.hs_rmi_sample_indices.argtypes = [u64, u64, vp, vp]
    lib.hs_learned_profile.restype = ci
    lib.hs_learned_profile.argtypes = [vp, vp, u64, ci, vp, vp, vp, vp, sz, vp]
    lib.hs_learned_force_bucket_bits.restype = ci
    lib.hs_test_bounded_waits.restype = ci
    lib.hs_test_bounded_waits.argtypes = [ctypes.c_uint32, ctypes.c_int64]
    lib.hs_learned_force_bucket_bits.argtypes = [ci]
    lib.hs_argsort_host.restype = ci
    lib.hs_argsort_host.argtypes = [vp, vp, u64, ci, ci, ci, vp, vp, sz, vp]
    lib.hs_host_workspace_size.restype = ci
    lib.hs_host_workspace_size.argtypes = [u64, u64, ci, ci, ctypes.POINTER(sz)]
    lib.hs_shutdown.restype = ci
    lib.hs_shutdown.argtypes = []
    lib.hs_bigint_workspace_size.restype = ci
    lib.hs_bigint_workspace_size.argtypes = [u64, u64, ci, ctypes.POINTER(ctypes.c_size_t)]
    lib.hs_argsort_bigint.restype = ci
    lib.hs_argsort_bigint.argtypes = [vp, vp, u64, u64, ci, vp, vp, ctypes.c_size_t, vp]
    lib.hs_bigdecimal_workspace_size.restype = ci
    lib.hs_bigdecimal_workspace_size.argtypes = [u64, u64, ci, ctypes.POINTER(ctypes.c_size_t)]
    lib.hs_argsort_bigdecimal.restype = ci
    lib.hs_argsort_bigdecimal.argtypes = [vp, vp, u64, u64, ci, vp, vp, ctypes.c_size_t, vp]
    lib.hs_autotune.restype = ci
    lib.hs_autotune.argtypes = [ci]
    lib.hs_autotune_choice.restype = ci
    lib.hs_autotune_choice.argtypes = [ci, u64, ctypes.POINTER(ctypes.c_int)]
    lib.hs_encode_numeric.restype = ci
    lib.hs_encode_numeric.argtypes = [vp, u64, ci, vp, vp]
    lib.hs_numeric_workspace_size.restype = ci
    lib.hs_numeric_workspace_size.argtypes = [u64, ci, ctypes.POINTER(ctypes.c_size_t)]
    lib.hs_argsort_numeric.restype = ci
    lib.hs_argsort_numeric.argtypes = [vp, u64, ci, ci, vp, vp, ctypes.c_size_t, vp]
    lib.hs_argsort_noalloc.restype = ci
    lib.hs_argsort_noalloc.argtypes = [vp, vp, u64, ci, ci, vp, vp]
    lib.hs_stats_enable.restype = ci
    lib.hs_stats_enable.argtypes = [ci]
    lib.hs_stats_read.restype = ci
    lib.hs_stats_read.argtypes = [ctypes.POINTER(KernelStat), ci, ctypes.POINTER(ci)]
    lib.hs_last_error.restype = ctypes.c_char_p
    lib.hs_last_error.argtypes = []
    lib.hs_version.restype = ci
    lib.hs_version.argtypes = []
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        msg = load().hs_last_error().decode(errors="replace")
        raise HuskyError(status, msg)


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> int:
    return 0 if t is None else int(t.data_ptr())


def test_bounded_waits(spin_limit: int = 0, withhold_tile: int = -1):
    """Test support: the look-back poll budget (0: default) and a tile whose
    counts are never published (-1: none), on the current device."""
    _check(load().hs_test_bounded_waits(spin_limit, withhold_tile))


def learned_force_bucket_bits(bits: int):
    """Test support: force the learned path's bucket-id bits (1..24), or 0
    for its own choice."""
    _check(load().hs_learned_force_bucket_bits(bits))


def workspace_size(n: int, mode: int = MODE_PLAIN, out_t: int = U32,
                   total_bytes: int = 0) -> int:
    out = ctypes.c_size_t(0)
    _check(load().hs_workspace_size(n, total_bytes, mode, out_t, ctypes.byref(out)))
    return int(out.value)


def host_workspace_size(n: int, total_bytes: int, mode: int = MODE_PLAIN, out_t: int = U32) -> int:
    out = ctypes.c_size_t(0)
    _check(load().hs_host_workspace_size(n, total_bytes, mode, out_t, ctypes.byref(out)))
    return int(out.value)


def batched_workspace_size(n: int, num_segs: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().hs_batched_workspace_size(n, num_segs, ctypes.byref(out)))
    return int(out.value)


_ws_cache: dict = {}


def workspace(nbytes: int, device) -> torch.Tensor:
    """A cached device scratch buffer of at least nbytes (grown on demand)."""
    dev = torch.device(device)
    key = dev.index if dev.index is not None else torch.cuda.current_device()
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        _ws_cache.pop(key, None)
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        _ws_cache[key] = buf
    return buf


def free_workspace():
    _ws_cache.clear()


def _as_device_inputs(data: torch.Tensor, offsets: torch.Tensor):
    if data.dtype != torch.uint8:
        raise TypeError("bytes must be a uint8 tensor")
    if offsets.dtype not in (torch.int64, torch.uint64):
        raise TypeError("offsets must be an int64/uint64 tensor")
    if not data.is_cuda or not offsets.is_cuda:
        raise ValueError("device tensors expected")
    if data.numel() == 0:  # the library wants a valid pointer even for no bytes
        data = torch.zeros(16, dtype=torch.uint8, device=offsets.device)
    return data.contiguous(), offsets.contiguous()


def encode(data: torch.Tensor, offsets: torch.Tensor, coder: int = CODER_AUTO,
           stream=None):
    """Step 1: (codes int64 tensor holding the uint64 codes, all_exact bool,
    coder used)."""
    data, offsets = _as_device_inputs(data, offsets)
    n = offsets.numel() - 1
    codes = torch.empty(max(n, 0), dtype=torch.int64, device=offsets.device)
    ws = workspace(workspace_size(0), offsets.device)
    exact = ctypes.c_int(0)
    used = ctypes.c_int(0)
    _check(load().hs_encode(_ptr(data), _ptr(offsets), n, coder, _ptr(codes),
                            ctypes.byref(exact), ctypes.byref(used), _ptr(ws),
                            ws.numel(), _stream_handle(stream)))
    return codes, bool(exact.value), int(used.value)


_NUM_TYPES = {torch.int64: NUM_I64, torch.int32: NUM_I32, torch.float64: NUM_F64, torch.float32: NUM_F32}


def _numeric_input(values: torch.Tensor, type):
    if not values.is_cuda:
        raise ValueError("values must be a CUDA tensor")
    values = values.contiguous()
    if type is None:
        if values.dtype not in _NUM_TYPES:
            raise ValueError(f"no numeric coder for {values.dtype}; pass type=")
        type = _NUM_TYPES[values.dtype]
    width = 4 if type in (NUM_I32, NUM_F32) else 8
    if values.element_size() != width:
        raise ValueError(f"numeric type {type} needs {width}-byte elements")
    return values, type


def argsort_bigdecimal(data: torch.Tensor, offsets: torch.Tensor, index_u64: bool = False,
                       stream=None) -> torch.Tensor:
    """Stable argsort of decimal texts (the form Java's BigDecimal(String)
    accepts) by numeric value, in the strings' data model."""
    data, offsets = _as_device_inputs(data, offsets)
    n = offsets.numel() - 1
    out = torch.empty(max(n, 0), dtype=torch.int64 if index_u64 else torch.int32, device=offsets.device)
    need = ctypes.c_size_t(0)
    _check(load().hs_bigdecimal_workspace_size(n, data.numel(), U64 if index_u64 else U32, ctypes.byref(need)))
    ws = workspace(need.value, offsets.device)
    _check(load().hs_argsort_bigdecimal(_ptr(data), _ptr(offsets), n, data.numel(), U64 if index_u64 else U32,
                                        _ptr(out), _ptr(ws), ws.numel(), _stream_handle(stream)))
    return out


def argsort_bigint(data: torch.Tensor, offsets: torch.Tensor, index_u64: bool = False,
                   stream=None) -> torch.Tensor:
    """Stable argsort of big integers given as minimal two's complement
    big-endian bytes (Java's toByteArray) in the strings' data model."""
    data, offsets = _as_device_inputs(data, offsets)
    n = offsets.numel() - 1
    out = torch.empty(max(n, 0), dtype=torch.int64 if index_u64 else torch.int32, device=offsets.device)
    need = ctypes.c_size_t(0)
    _check(load().hs_bigint_workspace_size(n, data.numel(), U64 if index_u64 else U32, ctypes.byref(need)))
    ws = workspace(need.value, offsets.device)
    _check(load().hs_argsort_bigint(_ptr(data), _ptr(offsets), n, data.numel(), U64 if index_u64 else U32,
                                    _ptr(out), _ptr(ws), ws.numel(), _stream_handle(stream)))
    return out


def autotune(mode: int = 1):
    """Tile-shape tuner: 1 tune new size classes (default), 0 off, 2 forget and re-tune."""
    _check(load().hs_autotune(mode))


def autotune_choice(layout: int, n: int) -> int:
    """Keys per thread the tuner chose for layout (0 packed words, 1 pairs) at n, 0 if none."""
    v = ctypes.c_int(0)
    _check(load().hs_autotune_choice(layout, n, ctypes.byref(v)))
    return v.value


def encode_numeric(values: torch.Tensor, type: int | None = None, stream=None) -> torch.Tensor:
    """Order-preserving uint64 codes of numeric values (an int64 tensor holding
    the codes' bits).  type defaults from the dtype (int64, int32, float64,
    float32); NUM_U64 and NUM_DATETIME take int64 tensors."""
    values, type = _numeric_input(values, type)
    codes = torch.empty(values.numel(), dtype=torch.int64, device=values.device)
    _check(load().hs_encode_numeric(_ptr(values), values.numel(), type, _ptr(codes), _stream_handle(stream)))
    return codes


def argsort_numeric(values: torch.Tensor, type: int | None = None, index_u64: bool = False,
                    stream=None) -> torch.Tensor:
    """Stable argsort of device-resident numeric values in the order of their
    numeric coder (Java's compareTo order; see hs_numeric in husky.h)."""
    values, type = _numeric_input(values, type)
    n = values.numel()
    out = torch.empty(n, dtype=torch.int64 if index_u64 else torch.int32, device=values.device)
    need = ctypes.c_size_t(0)
    _check(load().hs_numeric_workspace_size(n, U64 if index_u64 else U32, ctypes.byref(need)))
    ws = workspace(need.value, values.device)
    _check(load().hs_argsort_numeric(_ptr(values), n, type, U64 if index_u64 else U32, _ptr(out), _ptr(ws),
                                     ws.numel(), _stream_handle(stream)))
    return out


def argsort_device(data: torch.Tensor, offsets: torch.Tensor,
                   mode: int = MODE_PLAIN, coder: int = CODER_AUTO,
                   index_u64: bool = False, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """Stable argsort of device-resident strings; returns a device tensor
    (int32 for uint32 indices, int64 for uint64)."""
    data, offsets = _as_device_inputs(data, offsets)
    n = offsets.numel() - 1
    dt = torch.int64 if index_u64 else torch.int32
    if out is None:
        out = torch.empty(max(n, 0), dtype=dt, device=offsets.device)
    elif out.dtype != dt or out.numel() != n or not out.is_cuda:
        raise ValueError("out has the wrong dtype, size or device")
    out_t = U64 if index_u64 else U32
    need = workspace_size(n, mode, out_t)
    ws = workspace(need, offsets.device)
    _check(load().hs_argsort(_ptr(data), _ptr(offsets), n, mode, coder, out_t,
                             _ptr(out), _ptr(ws), ws.numel(),
                             _stream_handle(stream)))
    return out


def argsort(data: torch.Tensor, offsets: torch.Tensor, mode: int = MODE_PLAIN,
            coder: int = CODER_AUTO, index_u64: bool = False,
            device="cuda", stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Stable argsort of strings held in host or device tensors.

    Device inputs are sorted on the device (hs_argsort) and the permutation
    stays there.  Host inputs go through hs_argsort_host: the library copies
    them in chunks (overlapped with the encoder), sorts on the device and
    copies the permutation back into a pinned host tensor, which is
    returned (`out`, when given: a pinned host tensor of n int32, or int64
    with index_u64, reused across calls).  Pinned inputs give the full
    transfer speed."""
    if data.is_cuda and offsets.is_cuda:
        return argsort_device(data, offsets, mode, coder, index_u64, out=out, stream=stream)
    if data.is_cuda or offsets.is_cuda:
        raise ValueError("bytes and offsets must both be on the host or both on the device")
    if data.dtype != torch.uint8:
        raise TypeError("bytes must be a uint8 tensor")
    if offsets.dtype not in (torch.int64, torch.uint64):
        raise TypeError("offsets must be an int64/uint64 tensor")
    data = data.contiguous()
    offsets = offsets.contiguous()
    n = offsets.numel() - 1
    dt = torch.int64 if index_u64 else torch.int32
    if out is None:
        out = torch.empty(max(n, 0), dtype=dt, pin_memory=True)
    elif out.dtype != dt or out.numel() != max(n, 0) or out.is_cuda or not out.is_pinned():
        raise ValueError("out must be a pinned host tensor of n indices of the output type")
    if n <= 0:
        return out
    lib = load()
    out_t = U64 if index_u64 else U32
    total = int(offsets[-1])
    if total > data.numel():
        raise ValueError("offsets[n] exceeds the byte buffer")
    dev = torch.device(device)
    with torch.cuda.device(dev):
        nbytes = host_workspace_size(n, total, mode, out_t)
        ws = workspace(nbytes, dev)
        _check(lib.hs_argsort_host(_ptr(data), _ptr(offsets), n, mode, coder, out_t, _ptr(out),
                                   _ptr(ws), nbytes, _stream_handle(stream)))
    return out


def argsort_batched(data: torch.Tensor, offsets: torch.Tensor,
                    seg_offsets: torch.Tensor, coder: int = CODER_AUTO,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Independent stable argsorts of the instances delimited by seg_offsets
    (string-index boundaries); returns local indices (int32) laid out like
    the strings (written into `out` when given)."""
    data, offsets = _as_device_inputs(data, offsets)
    if seg_offsets.dtype not in (torch.int64, torch.uint64) or not seg_offsets.is_cuda:
        raise TypeError("seg_offsets must be an int64 device tensor")
    seg_offsets = seg_offsets.contiguous()
    n = offsets.numel() - 1
    num_segs = seg_offsets.numel() - 1
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
    elif out.dtype != torch.int32 or out.numel() != n or not out.is_cuda:
        raise ValueError("out has the wrong dtype, size or device")
    ws = workspace(batched_workspace_size(n, num_segs), offsets.device)
    _check(load().hs_argsort_batched(_ptr(data), _ptr(offsets), _ptr(seg_offsets),
                                     num_segs, n, coder, _ptr(out), _ptr(ws),
                                     ws.numel(), _stream_handle(stream)))
    return out


def stats_enable(on: bool = True):
    """Start (and reset) or stop per-kernel event timing inside the library."""
    _check(load().hs_stats_enable(1 if on else 0))


def stats_read() -> dict:
    """{kernel kind: {"launches", "total_ms", "algo_bytes"}} since enabling."""
    rows = (KernelStat * 64)()
    count = ctypes.c_int(0)
    _check(load().hs_stats_read(rows, 64, ctypes.byref(count)))
    out = {}
    for r in rows[: min(count.value, 64)]:
        out[r.name.decode()] = dict(launches=int(r.launches), total_ms=float(r.total_ms),
                                    algo_bytes=float(r.algo_bytes))
    return out


def rmi_grad(params: torch.Tensor, x: torch.Tensor, t: torch.Tensor, stream=None):
    """(loss, grad) of the learned root network on device float32 tensors."""
    grad = torch.empty(1153, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(load().hs_rmi_grad(_ptr(params), _ptr(x), _ptr(t), x.numel(), _ptr(grad), _ptr(loss),
                              _stream_handle(stream)))
    return float(loss.item()), grad


def rmi_leaf_fit(x: torch.Tensor, t: torch.Tensor, leaf_start: torch.Tensor, stream=None):
    """Per-leaf (slope, intercept, band lo, band hi) float32 device tensors."""
    leaves = leaf_start.numel() - 1
    outs = [torch.empty(leaves, dtype=torch.float32, device=x.device) for _ in range(4)]
    _check(load().hs_rmi_leaf_fit(_ptr(x), _ptr(t), _ptr(leaf_start), x.numel(), leaves,
                                  *[_ptr(o) for o in outs], _stream_handle(stream)))
    return outs


def rmi_sample_indices(n: int, seed: int, device="cuda", stream=None) -> torch.Tensor:
    out = torch.empty(max(n // 100, 1), dtype=torch.int64, device=device)
    _check(load().hs_rmi_sample_indices(n, seed, _ptr(out), _stream_handle(stream)))
    return out[: n // 100]


def learned_profile(data: torch.Tensor, offsets: torch.Tensor, linear: bool = False, stream=None):
    """(sort keys int64, buckets int32, info dict) from the learned path's model."""
    data, offsets = _as_device_inputs(data, offsets)
    n = offsets.numel() - 1
    keys = torch.empty(n, dtype=torch.int64, device=offsets.device)
    buckets = torch.empty(n, dtype=torch.int32, device=offsets.device)
    info = (ctypes.c_double * 4)()
    ws = workspace(workspace_size(n, MODE_LEARNED), offsets.device)
    _check(load().hs_learned_profile(_ptr(data), _ptr(offsets), n, 1 if linear else 0, _ptr(keys),
                                     _ptr(buckets), info, _ptr(ws), ws.numel(), _stream_handle(stream)))
    return keys, buckets, dict(bits=int(info[0]), sample=int(info[1]), loss0=info[2], loss1=info[3])


def shutdown():
    """Release the library's cached streams, events and timing table, and
    the binding's cached workspaces."""
    free_workspace()
    _check(load().hs_shutdown())


def version() -> int:
    return int(load().hs_version())
