"""hs_argsort_noalloc: the entry point for callers that cannot allocate device
memory (for example code embedded in a host application that owns the GPU's
memory pool, or code that must not trigger cudaMalloc's device-wide
synchronisation).  Its scratch is a static device array inside the library.

Checked through the C ABI on two calls in a row, against the oracle's stable
argsort and against the existing hs_argsort entry point: the second call gets
a different, smaller input, so it runs on scratch that still holds the first
call's contents.  The bar is the same as for every sort here: the
permutations are integers and must be identical.
This file is collected last so a failure here cannot hide the other tests."""

import ctypes

import numpy as np
import pytest
import torch

import workloads
from gpu_util import assert_oracle_equal, to_device

pytestmark = pytest.mark.gpu


def _noalloc(lib, data, off, n, out_t=0, coder=0):
    dt = torch.int64 if out_t == 1 else torch.int32
    perm = torch.full((n,), -1, dtype=dt, device="cuda")
    st = lib.hs_argsort_noalloc(data.data_ptr(), off.data_ptr(), n, coder, out_t,
                                perm.data_ptr(),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, perm


def _inputs():
    long_runs = [b"the-same-string-longer-than-nine"] * 3000 + \
                [b"abcdefghi" + bytes([97 + i % 7]) * (i % 4) for i in range(3000)]
    big = workloads.generate(2, 262_144 - len(long_runs), 21)  # Zipf words
    strs = [big.string(i) for i in range(big.n)] + long_runs
    rng = np.random.default_rng(4)
    first = workloads.from_strings([strs[i] for i in rng.permutation(len(strs))])
    second = workloads.generate(5, 70_001, 22)                # skewed, smaller
    return first, second


def test_noalloc_matches_oracle_and_hs_argsort_twice(cuda_lib):
    hs = cuda_lib
    lib = hs.load()
    first, second = _inputs()
    assert first.n == hs.NOALLOC_MAX_N
    for w, out_t in ((first, 0), (second, 1)):
        data, off = to_device(w)
        ref = hs.argsort_device(data, off, index_u64=out_t == 1)
        st, perm = _noalloc(lib, data, off, w.n, out_t=out_t)
        assert st == hs.OK, lib.hs_last_error()
        assert_oracle_equal(w, perm)
        assert torch.equal(perm, ref)


def test_noalloc_rejects_oversize(cuda_lib):
    hs = cuda_lib
    lib = hs.load()
    n = hs.NOALLOC_MAX_N + 1
    w = workloads.generate(1, n, 1)
    data, off = to_device(w)
    st, perm = _noalloc(lib, data, off, n)
    assert st == hs.ERR_INVALID_ARG
    assert b"HS_NOALLOC_MAX_N" in lib.hs_last_error()
    assert torch.all(perm == -1)
