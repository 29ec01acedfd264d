"""Huskysort oracle -- TEST INFRASTRUCTURE ONLY.

Plain CPU reference implementations used to check the CUDA library.  Only the
test-suite, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline / reference
arm import this package; the product path never does.  It shares no code with
the CUDA library (``paper_2012_00866_gb300``) and imports nothing from it.

  husky_oracle.c  Algorithm 4 encoder, Algorithms 2/3 array encoding, stable
                  lexicographic argsort, sortedness/stability property check.
  rmi_oracle.py   FP64 learned-bucketer model (forward, gradient, SGD step,
                  least-squares leaf fit, bucket function).
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "husky_oracle.c")
_LIB = os.path.join(_HERE, "libhusky_oracle.so")
_lib = None

CODER_ASCII7 = 1
CODER_BYTE8 = 2


def build(force: bool = False) -> str:
    """Compile husky_oracle.c into libhusky_oracle.so beside it."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-pthread", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, vp, ci = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
        lib.oracle_string_to_long.restype = u64
        lib.oracle_string_to_long.argtypes = [vp, u64, ci, ci, u64]
        lib.oracle_encode.restype = ci
        lib.oracle_encode.argtypes = [vp, vp, u64, ci, vp, vp, vp]
        lib.oracle_string_compare.restype = ci
        lib.oracle_string_compare.argtypes = [vp, vp, u64, u64]
        lib.oracle_stable_argsort.restype = ci
        lib.oracle_stable_argsort.argtypes = [vp, vp, u64, vp, ci, ci]
        lib.oracle_check_sorted.restype = ctypes.c_int64
        lib.oracle_check_sorted.argtypes = [vp, vp, u64, vp, ci, ci]
        lib.oracle_stable_argsort_batched.restype = ci
        lib.oracle_stable_argsort_batched.argtypes = [vp, vp, vp, u64, vp, ci]
        lib.oracle_check_sorted_batched.restype = ctypes.c_int64
        lib.oracle_check_sorted_batched.argtypes = [vp, vp, vp, u64, vp, ci]
        lib.oracle_string_to_long_mapped.restype = u64
        lib.oracle_string_to_long_mapped.argtypes = [vp, u64, ci, ci, vp]
        lib.oracle_alpha_params_k.restype = ci
        lib.oracle_alpha_params_k.argtypes = [vp, vp, u64, ci, vp, vp, vp]
        lib.oracle_units_to_long.restype = u64
        lib.oracle_units_to_long.argtypes = [vp, u64, ci, ci, u64]
        lib.oracle_unicode_to_long.restype = u64
        lib.oracle_unicode_to_long.argtypes = [vp, u64]
        lib.oracle_encode_alpha_k.restype = ci
        lib.oracle_encode_alpha_k.argtypes = [vp, vp, u64, ci, vp, vp, vp, vp, vp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _threads(threads):
    return threads if threads else (os.cpu_count() or 1)


def string_to_long(s: bytes, max_length: int, bit_width: int, mask: int) -> int:
    """Algorithm 4 on one string."""
    buf = np.frombuffer(s, dtype=np.uint8) if s else np.zeros(1, np.uint8)
    return int(_load().oracle_string_to_long(_ptr(buf), len(s), max_length,
                                             bit_width, mask))


def ascii_to_long(s: bytes) -> int:
    """The ASCII coder: 7 bits x 64/7 = 9 chars, mask 0x7F."""
    return string_to_long(s, 64 // 7, 7, 0x7F)


def byte_to_long(s: bytes) -> int:
    """The byte coder: 8 bits x 8 chars, no mask."""
    return string_to_long(s, 8, 8, 0)


def unicode_to_long(units) -> int:
    """The paper's Unicode coder on one string of UTF-16 code units:
    Algorithm 4 with 16 bits x 4 units, mask 0xFFFF, then >>> 1."""
    buf = np.asarray(units, dtype=np.uint16) if len(units) else np.zeros(1, np.uint16)
    return int(_load().oracle_unicode_to_long(_ptr(np.ascontiguousarray(buf)), len(units)))


def units_to_long(units, max_length: int, bit_width: int, mask: int) -> int:
    """Algorithm 4 over 16-bit chars."""
    buf = np.asarray(units, dtype=np.uint16) if len(units) else np.zeros(1, np.uint16)
    return int(_load().oracle_units_to_long(_ptr(np.ascontiguousarray(buf)), len(units), max_length,
                                            bit_width, mask))


def encode(data: np.ndarray, offsets: np.ndarray, coder: int = CODER_ASCII7):
    """Algorithms 2/3: (codes uint64[n], exact uint8[n], perfect bool)."""
    n = offsets.shape[0] - 1
    codes = np.empty(n, dtype=np.uint64)
    exact = np.empty(n, dtype=np.uint8)
    perfect = ctypes.c_int(0)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    _load().oracle_encode(_ptr(data), _ptr(offsets), n, coder, _ptr(codes),
                          _ptr(exact), ctypes.addressof(perfect))
    return codes, exact, bool(perfect.value)


def alpha_params(data: np.ndarray, offsets: np.ndarray, max_length: int | None = 8):
    """Byte-range coder parameters: (map uint8[256], w, K, applies).
    max_length: K; None takes the paper's longest K that fits 64 bits,
    floor(64 / w) (Section 3.2: 12 letters in 5 bits, 10 in 6).  The GPU
    library codes K = 8."""
    n = offsets.shape[0] - 1
    rank = np.zeros(256, dtype=np.uint8)
    w, k = ctypes.c_int(0), ctypes.c_int(0)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    rc = _load().oracle_alpha_params_k(_ptr(data), _ptr(offsets), n, int(max_length or 0), _ptr(rank),
                                       ctypes.addressof(w), ctypes.addressof(k))
    return rank, w.value, k.value, rc == 0


def encode_alpha(data: np.ndarray, offsets: np.ndarray, max_length: int | None = 8):
    """Byte-range coder: (codes uint64[n], exact uint8[n], perfect, w, K), or
    None when the byte range needs more than 6 bits (or K * w > 64).
    max_length as in alpha_params."""
    n = offsets.shape[0] - 1
    codes = np.empty(n, dtype=np.uint64)
    exact = np.empty(n, dtype=np.uint8)
    perfect, w, k = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    rc = _load().oracle_encode_alpha_k(_ptr(data), _ptr(offsets), n, int(max_length or 0), _ptr(codes),
                                       _ptr(exact), ctypes.addressof(perfect), ctypes.addressof(w),
                                       ctypes.addressof(k))
    if rc != 0:
        return None
    return codes, exact, bool(perfect.value), w.value, k.value


def stable_argsort(data: np.ndarray, offsets: np.ndarray, index_u64: bool = False,
                   threads: int | None = None) -> np.ndarray:
    """Stable argsort of the strings, unsigned-byte lexicographic order."""
    n = offsets.shape[0] - 1
    perm = np.empty(n, dtype=np.uint64 if index_u64 else np.uint32)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    rc = _load().oracle_stable_argsort(_ptr(data), _ptr(offsets), n, _ptr(perm),
                                       1 if index_u64 else 0, _threads(threads))
    if rc != 0:
        raise MemoryError("oracle_stable_argsort: out of memory")
    return perm


def check_sorted(data: np.ndarray, offsets: np.ndarray, perm: np.ndarray,
                 threads: int | None = None) -> int:
    """-1 if perm is the stable argsort, else the first failing position."""
    n = offsets.shape[0] - 1
    if perm.shape[0] != n:
        return 0
    perm = np.ascontiguousarray(perm)
    if perm.dtype not in (np.uint32, np.uint64):
        raise TypeError("perm must be uint32 or uint64")
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    return int(_load().oracle_check_sorted(_ptr(data), _ptr(offsets), n,
                                           _ptr(perm),
                                           1 if perm.dtype == np.uint64 else 0,
                                           _threads(threads)))


def stable_argsort_batched(data: np.ndarray, offsets: np.ndarray, seg_offsets: np.ndarray,
                           threads: int | None = None) -> np.ndarray:
    """Per-instance stable argsort as local uint32 indices, laid out like the
    strings (instance s at positions seg_offsets[s] .. seg_offsets[s+1]-1)."""
    n = offsets.shape[0] - 1
    perm = np.empty(n, dtype=np.uint32)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    seg = np.ascontiguousarray(seg_offsets, dtype=np.uint64)
    rc = _load().oracle_stable_argsort_batched(_ptr(data), _ptr(offsets), _ptr(seg),
                                               seg.shape[0] - 1, _ptr(perm), _threads(threads))
    if rc != 0:
        raise MemoryError("oracle_stable_argsort_batched: out of memory")
    return perm


def check_sorted_batched(data: np.ndarray, offsets: np.ndarray, seg_offsets: np.ndarray,
                         perm: np.ndarray, threads: int | None = None) -> int:
    """-1 if every instance holds its stable argsort (local indices)."""
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    seg = np.ascontiguousarray(seg_offsets, dtype=np.uint64)
    return int(_load().oracle_check_sorted_batched(_ptr(data), _ptr(offsets), _ptr(seg),
                                                   seg.shape[0] - 1, _ptr(perm), _threads(threads)))


def string_compare(data: np.ndarray, offsets: np.ndarray, i: int, j: int) -> int:
    return int(_load().oracle_string_compare(_ptr(data), _ptr(offsets), i, j))


# ---- numeric coders ---------------------------------------------------------
#
# The paper benchmarks Integer, Long and Double arrays (Section 6.1, Table 4) and names a
# perfect date-time coding (Section 3.2) without giving bit layouts.  Two
# plain definitions serve as the oracle: the order itself, written from each
# type's compareTo semantics (integers by value; doubles as Double.compare:
# NaN equal to NaN and above everything, -0.0 below 0.0), and the code of each
# value written from the two's complement and IEEE 754 layouts.

NUM_U64, NUM_I64, NUM_I32, NUM_F64, NUM_F32, NUM_DATETIME = 0, 1, 2, 3, 4, 5


def numeric_argsort(values: np.ndarray, type: int) -> np.ndarray:
    """Stable argsort in compareTo order, by numeric comparisons only."""
    idx = np.arange(values.size, dtype=np.int64)
    if type in (NUM_F64, NUM_F32):
        with np.errstate(invalid="ignore"):  # signalling NaNs widen to NaNs
            v = values.astype(np.float64)
        nan = np.isnan(v)
        val = np.where(nan, 0.0, v)
        zero_sign = np.where((v == 0.0) & ~np.signbit(v), 1, 0)  # -0.0 before 0.0
        return np.lexsort((idx, zero_sign, val, nan.astype(np.int8))).astype(np.int64)
    if type == NUM_U64:
        return np.argsort(values.astype(np.uint64), kind="stable").astype(np.int64)
    return np.argsort(values.astype(np.int64), kind="stable").astype(np.int64)


def numeric_code(values: np.ndarray, type: int) -> np.ndarray:
    """The order-preserving unsigned key of each value, from its bit layout."""
    if type in (NUM_I64, NUM_DATETIME):
        return values.astype(np.int64).view(np.uint64) ^ np.uint64(1 << 63)
    if type == NUM_I32:
        return (values.astype(np.int32).view(np.uint32) ^ np.uint32(1 << 31)).astype(np.uint64)
    if type == NUM_F64:
        x = values.astype(np.float64).view(np.uint64).copy()
        x[np.isnan(values)] = np.uint64(0x7FF8000000000000)
        neg = (x >> np.uint64(63)) == 1
        return np.where(neg, ~x, x | np.uint64(1 << 63))
    if type == NUM_F32:
        x = values.astype(np.float32).view(np.uint32).copy()
        x[np.isnan(values)] = np.uint32(0x7FC00000)
        neg = (x >> np.uint32(31)) == 1
        return np.where(neg, ~x, x | np.uint32(1 << 31)).astype(np.uint64)
    return values.astype(np.uint64)


# ---- BigInteger ---------------------------------------------------------------

def bigint_values(data: np.ndarray, offsets: np.ndarray):
    """Each value's minimal two's complement big-endian bytes as a Python int."""
    return [int.from_bytes(data[int(offsets[i]):int(offsets[i + 1])].tobytes(), "big", signed=True)
            for i in range(offsets.size - 1)]


def bigint_argsort(data: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Stable argsort by numeric value (Python's sort is stable)."""
    v = bigint_values(data, offsets)
    return np.array(sorted(range(len(v)), key=v.__getitem__), dtype=np.int64)


def bigint_bytes(x: int) -> bytes:
    """The minimal two's complement big-endian bytes of x (toByteArray)."""
    return x.to_bytes(((x if x >= 0 else ~x).bit_length() + 8) // 8, "big", signed=True)


# ---- BigDecimal -----------------------------------------------------------------
#
# The paper benchmarks BigDecimal arrays (Section 6.1, Table 4) without giving
# a coder.  A value here is its decimal text in the form Java's
# BigDecimal(String) accepts: an optional sign, digits with at most one
# decimal point and at least one digit, then optionally an exponent
# [eE][+-]digits.  The order is compareTo's: numeric value with the scale
# ignored (1.0 equals 1.00), and the sort is stable, so equal values keep
# index order.  The oracle is that definition written out: each text's exact
# rational value (Python's Fraction), then Python's stable sort.

import re as _re
from fractions import Fraction as _Fraction

_DECIMAL_TEXT = _re.compile(r"[+-]?(?:[0-9]+\.?[0-9]*|\.[0-9]+)(?:[eE][+-]?[0-9]+)?")


def bigdecimal_value(text: bytes) -> _Fraction:
    """The exact value of one decimal text; ValueError outside the grammar."""
    s = bytes(text).decode("ascii")
    if not _DECIMAL_TEXT.fullmatch(s):
        raise ValueError(f"not a decimal: {s!r}")
    mant, _, exp = s.replace("E", "e").partition("e")
    sign = -1 if mant.startswith("-") else 1
    mant = mant.lstrip("+-")
    whole, _, frac = mant.partition(".")
    digits = int((whole + frac) or "0")
    scale = len(frac) - (int(exp) if exp else 0)
    return sign * _Fraction(digits, 1) / _Fraction(10) ** scale if scale >= 0 else \
        sign * _Fraction(digits * 10 ** (-scale), 1)


def bigdecimal_key(text: bytes):
    """A sort key equal to the text's exact value for comparisons: Python's
    Decimal, which compares finite values exactly and keeps the exponent
    apart from the digits, so exponents near 10^9 cost nothing (the Fraction
    of 1E+999999999 would be a billion-digit integer).  ValueError outside
    the grammar."""
    import decimal
    s = bytes(text).decode("ascii")
    if not _DECIMAL_TEXT.fullmatch(s):
        raise ValueError(f"not a decimal: {s!r}")
    return decimal.Decimal(s)


def bigdecimal_argsort(data: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Stable argsort of decimal texts by numeric value."""
    v = [bigdecimal_key(data[int(offsets[i]):int(offsets[i + 1])].tobytes()) for i in range(offsets.size - 1)]
    return np.array(sorted(range(len(v)), key=v.__getitem__), dtype=np.int64)
