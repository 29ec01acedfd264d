"""Bounded device-side waits: a wait that runs out reports HS_ERR_TIMEOUT to
the caller, and the GPU keeps serving the next call.

The wait is made to run out the safe way: one tile of every radix pass never
publishes its counts (a flag that nothing sets), and the poll budget is cut
to a few thousand polls, so the tiles after it give up within milliseconds.
The input codes perfectly (lowercase strings of at most 8 letters), so after
the radix passes nothing reads the unwritten positions; the fix-up kernels
would do nothing after a give-up in any case."""

import numpy as np
import pytest

import workloads
from gpu_util import assert_oracle_equal, to_device

pytestmark = pytest.mark.gpu


def _short_words(n, seed):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 9, size=n)
    chars = rng.integers(97, 123, size=int(lens.sum())).astype(np.uint8)
    off = np.zeros(n + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    return workloads.Workload(chars, off)


@pytest.mark.parametrize("withhold", [0, 5])
def test_wait_runs_out_and_next_call_succeeds(cuda_lib, withhold):
    hs = cuda_lib
    w = _short_words(40 * 6144 + 17, 3)     # 41 radix tiles, packed words, perfect codes
    data, off = to_device(w)
    hs.test_bounded_waits(spin_limit=2000, withhold_tile=withhold)
    try:
        with pytest.raises(hs.HuskyError) as e:
            hs.argsort_device(data, off)
        assert e.value.status == hs.ERR_TIMEOUT
        assert "wait" in str(e.value)
    finally:
        hs.test_bounded_waits(0, -1)
    assert_oracle_equal(w, hs.argsort_device(data, off))


def test_wait_hook_rejects_bad_tile(cuda_lib):
    hs = cuda_lib
    with pytest.raises(hs.HuskyError) as e:
        hs.test_bounded_waits(0, -2)
    assert e.value.status == hs.ERR_INVALID_ARG
