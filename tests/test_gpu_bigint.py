"""GPU parity for the BigInteger coder: the stable argsort by numeric value
of big integers given as minimal two's complement bytes."""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import perm_numpy, to_device

pytestmark = pytest.mark.gpu


def _values(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        r = rng.random()
        if r < 0.1 and out:
            out.append(out[int(rng.integers(0, len(out)))])  # repeats
            continue
        nbits = int(rng.integers(0, 320))
        x = int.from_bytes(rng.bytes((nbits + 7) // 8 + 1), "big") >> (8 - nbits % 8 if nbits % 8 else 8)
        if r < 0.2:
            x = int(rng.choice([0, -1, 127, 128, -128, -129, 255, 256, -256, -257]))
        out.append(-x if rng.random() < 0.5 else x)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4097, 100_003])
@pytest.mark.parametrize("index_u64", [False, True])
def test_bigint_argsort_matches_oracle(cuda_lib, n, index_u64):
    hs = cuda_lib
    vals = _values(n, n)
    w = workloads.from_strings([oracle.bigint_bytes(x) for x in vals])
    data, off = to_device(w)
    got = perm_numpy(hs.argsort_bigint(data, off, index_u64=index_u64)).astype(np.int64)
    assert np.array_equal(got, oracle.bigint_argsort(w.bytes, w.offsets))


def test_bigint_long_values(cuda_lib):
    """Values of up to 32767 bytes, equal prefixes of many bytes."""
    hs = cuda_lib
    rng = np.random.default_rng(4)
    base = int.from_bytes(rng.bytes(3000), "big")
    vals = [base + int(rng.integers(0, 5)) << 16 for _ in range(3000)] + [-(base << 8), 1 << 262000]
    w = workloads.from_strings([oracle.bigint_bytes(x) for x in vals])
    data, off = to_device(w)
    got = perm_numpy(hs.argsort_bigint(data, off)).astype(np.int64)
    assert np.array_equal(got, oracle.bigint_argsort(w.bytes, w.offsets))


@pytest.mark.parametrize("bad", [b"\x00\x05", b"\xff\xff", b"", b"\x01" * 32768])
def test_bigint_rejects_non_minimal_empty_and_long(cuda_lib, bad):
    hs = cuda_lib
    w = workloads.from_strings([b"\x01", bad, b"\x02"])
    data, off = to_device(w)
    with pytest.raises(Exception):
        hs.argsort_bigint(data, off)
