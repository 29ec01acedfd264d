"""Seeded synthetic string workloads (inputs only).

The generator is a small C library (gen.c) driven through ctypes; it holds no
encoding or sorting arithmetic, so both the CUDA path and the oracle may use
it.  Workloads are returned as numpy arrays: ``bytes`` (uint8), ``offsets``
(uint64, n + 1 entries, string i is bytes[offsets[i]:offsets[i+1]]) and, for
batched workloads, ``seg_offsets`` (uint64, string-index boundaries of the
independent instances).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libhsgen.so")
_lib = None

# The standard workloads: kind, size and seed (workload k uses seed k - 1).
STANDARD = {
    "random_lower_1e5": dict(kind=1, n=100_000, seed=0),
    "zipf_words_1e7": dict(kind=2, n=10_000_000, seed=1),
    "shared_prefix_1e8": dict(kind=3, n=100_000_000, seed=2),
    "batched_20000": dict(kind=4, num_segs=20_000, seed=3),
    "skewed_1e9": dict(kind=5, n=1_000_000_000, seed=4),
}


def build(force: bool = False) -> str:
    """Compile gen.c into libhsgen.so beside it (host code, any arch)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-pthread", "-ffp-contract=off", "-o", tmp, _SRC,
                           "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gen_offsets.restype = ctypes.c_int64
        lib.gen_offsets.argtypes = [ctypes.c_int, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_void_p,
                                    ctypes.c_int]
        lib.gen_bytes.restype = ctypes.c_int
        lib.gen_bytes.argtypes = [ctypes.c_int, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int]
        lib.gen_instance_sizes.restype = ctypes.c_int
        lib.gen_instance_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_double, ctypes.c_double,
                                           ctypes.c_void_p]
        lib.gen_vocab_word.restype = ctypes.c_int
        lib.gen_vocab_word.argtypes = [ctypes.c_uint64, ctypes.c_int,
                                       ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class Workload:
    bytes: np.ndarray
    offsets: np.ndarray
    seg_offsets: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def string(self, i: int) -> bytes:
        return self.bytes[int(self.offsets[i]):int(self.offsets[i + 1])].tobytes()


def _threads(threads):
    return threads if threads else (os.cpu_count() or 1)


def generate(kind: int, n: int, seed: int, threads: int | None = None) -> Workload:
    """n strings of workload kind 1..5 (see gen.c) from the given seed."""
    lib = _load()
    offsets = np.empty(n + 1, dtype=np.uint64)
    total = lib.gen_offsets(kind, seed, n, offsets.ctypes.data, _threads(threads))
    if total < 0:
        raise RuntimeError(f"gen_offsets failed for kind {kind}")
    data = np.empty(max(int(total), 1), dtype=np.uint8)
    rc = lib.gen_bytes(kind, seed, n, offsets.ctypes.data, data.ctypes.data,
                       _threads(threads))
    if rc != 0:
        raise RuntimeError(f"gen_bytes failed for kind {kind}")
    return Workload(data[: int(total)] if total > 0 else data[:0], offsets)


def instance_sizes(num: int, seed: int, lo: float = 100.0, hi: float = 1e6) -> np.ndarray:
    """Log-uniform instance sizes round(exp(U[ln lo, ln hi]))."""
    lib = _load()
    sizes = np.empty(num, dtype=np.uint64)
    lib.gen_instance_sizes(seed, num, lo, hi, sizes.ctypes.data)
    return sizes


def generate_batched(num_segs: int, seed: int, lo: float = 100.0,
                     hi: float = 1e6, threads: int | None = None) -> Workload:
    """num_segs independent instances of kind-4 strings, log-uniform sizes."""
    sizes = instance_sizes(num_segs, seed, lo, hi)
    seg = np.zeros(num_segs + 1, dtype=np.uint64)
    np.cumsum(sizes, out=seg[1:])
    w = generate(4, int(seg[-1]), seed, threads)
    w.seg_offsets = seg
    return w


def standard(name: str, scale: float = 1.0, threads: int | None = None) -> Workload:
    """One of the STANDARD workloads, optionally scaled down in size."""
    spec = STANDARD[name]
    if spec["kind"] == 4:
        segs = max(1, int(round(spec["num_segs"] * scale)))
        return generate_batched(segs, spec["seed"], threads=threads)
    n = max(1, int(round(spec["n"] * scale)))
    return generate(spec["kind"], n, spec["seed"], threads)


def vocab_word(seed: int, k: int) -> bytes:
    """Word k of the kind-2 vocabulary built from seed."""
    buf = (ctypes.c_uint8 * 16)()
    ln = _load().gen_vocab_word(seed, k, ctypes.addressof(buf))
    if ln < 0:
        raise IndexError(k)
    return bytes(buf[:ln])


def from_strings(strings) -> Workload:
    """Pack a list of bytes objects into (bytes, offsets)."""
    lens = np.fromiter((len(s) for s in strings), dtype=np.uint64,
                       count=len(strings))
    offsets = np.zeros(len(strings) + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    data = np.frombuffer(b"".join(strings), dtype=np.uint8).copy()
    return Workload(data, offsets)
