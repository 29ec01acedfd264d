"""GPU parity for the numeric coders: codes and permutations of int, float
and date-time arrays against the oracle, bit-exact."""

import numpy as np
import pytest

import oracle
from gpu_util import perm_numpy
from test_oracle_numeric import _special_f32, _special_f64

pytestmark = pytest.mark.gpu

TYPES = ["f64", "f32", "i64", "i32", "u64", "datetime"]


def _values(name, n, seed):
    """(numpy values, numeric type, int64-or-native array to hand to torch)."""
    rng = np.random.default_rng(seed)
    if name == "f64":
        v = _special_f64(rng, n)
        return v, oracle.NUM_F64, v
    if name == "f32":
        v = _special_f32(rng, n)
        return v, oracle.NUM_F32, v
    if name == "i64":
        v = rng.integers(-(1 << 63), (1 << 63) - 1, size=n, dtype=np.int64) >> rng.integers(0, 64, size=n)
        return v, oracle.NUM_I64, v
    if name == "i32":
        v = (rng.integers(-(1 << 31), (1 << 31) - 1, size=n, dtype=np.int64).astype(np.int32)
             >> rng.integers(0, 32, size=n).astype(np.int32))
        return v, oracle.NUM_I32, v
    if name == "u64":
        v = rng.integers(0, 1 << 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
        return v, oracle.NUM_U64, v.view(np.int64)
    # date-times: ns since the epoch over 1900..2100, many repeated instants
    span = 200 * 365 * 86400 * 10**9
    v = rng.integers(-70 * 365 * 86400 * 10**9, span, size=n, dtype=np.int64)
    v[rng.random(n) < 0.3] = v[0]
    return v, oracle.NUM_DATETIME, v


def _sort(hs, arr, t, **kw):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    return hs.argsort_numeric(x, type=t, **kw), hs.encode_numeric(x, type=t)


@pytest.mark.parametrize("name", TYPES)
@pytest.mark.parametrize("n", [1, 2, 4097, 100_003, 1_000_003])
def test_numeric_argsort_matches_oracle(cuda_lib, name, n):
    v, t, arr = _values(name, n, n + len(name))
    perm, codes = _sort(cuda_lib, arr, t)
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), oracle.numeric_code(v, t))
    assert np.array_equal(perm_numpy(perm).astype(np.int64), oracle.numeric_argsort(v, t))


@pytest.mark.parametrize("name", ["f64", "i32", "datetime"])
def test_numeric_u64_index(cuda_lib, name):
    v, t, arr = _values(name, 300_001, 5)
    perm, _ = _sort(cuda_lib, arr, t, index_u64=True)
    got = perm_numpy(perm)
    assert got.dtype == np.uint64
    assert np.array_equal(got.astype(np.int64), oracle.numeric_argsort(v, t))


def test_numeric_ties_keep_index_order(cuda_lib):
    """A few distinct doubles repeated 300,000 times, -0.0 and 0.0 and NaNs
    of every sign and payload among them: equal values stay in index order,
    -0.0 sorts before 0.0 and every NaN after +infinity."""
    rng = np.random.default_rng(3)
    pool = np.array([0.0, -0.0, 1.5, -1.5, np.inf, np.nan], np.float64)
    v = pool[rng.integers(0, pool.size, size=300_000)]
    bits = v.view(np.uint64)
    nan = np.isnan(v)
    bits[nan] |= rng.integers(0, 1 << 51, size=int(nan.sum()), dtype=np.uint64) | np.uint64(1)
    bits[nan & (rng.random(v.size) < 0.5)] |= np.uint64(1 << 63)
    perm, _ = _sort(cuda_lib, v, oracle.NUM_F64)
    assert np.array_equal(perm_numpy(perm).astype(np.int64), oracle.numeric_argsort(v, oracle.NUM_F64))


@pytest.mark.parametrize("name,passes", [("i32", 4), ("f32", 4), ("i64", 8)])
def test_numeric_pass_count(cuda_lib, name, passes):
    """32-bit values leave the top digits of their codes constant, so only
    four radix passes run."""
    hs = cuda_lib
    v, t, arr = _values(name, 200_000, 9)
    hs.stats_enable(True)
    try:
        perm, _ = _sort(hs, arr, t)
        st = hs.stats_read()
    finally:
        hs.stats_enable(False)
    assert st["onesweep"]["launches"] == passes
    assert np.array_equal(perm_numpy(perm).astype(np.int64), oracle.numeric_argsort(v, t))


def test_numeric_rejects_bad_input(cuda_lib):
    import torch
    hs = cuda_lib
    x = torch.zeros(10, dtype=torch.int16, device="cuda")
    with pytest.raises(ValueError):
        hs.argsort_numeric(x)
    with pytest.raises(ValueError):
        hs.argsort_numeric(torch.zeros(10, dtype=torch.float64, device="cuda"), type=oracle.NUM_F32)
    with pytest.raises(Exception):
        hs.argsort_numeric(torch.zeros(10, dtype=torch.int64, device="cuda"), type=17)
