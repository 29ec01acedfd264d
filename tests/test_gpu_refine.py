"""GPU parity for the refinement of long runs of equal codes (Section 3.1
Step 3 on strings that share long prefixes): several 7-byte rounds, with the
window keys gathered per member or, when the runs hold most of the strings,
read from one array of every string's window written in string order.
Each case is compared element by element with the oracle's stable argsort."""

import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import assert_oracle_equal, perm_numpy, to_device

pytestmark = pytest.mark.gpu

ALPHA = np.frombuffer(b"0123456789ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz", dtype=np.uint8)


def _prefix_strings(n_shared, n_unique, groups, prefix_len, seed):
    """n_shared strings of `groups` random prefixes of prefix_len chars plus
    0-6 random chars (some end inside the prefix's last window, some are
    the bare prefix), and n_unique random strings of 4-30 chars."""
    rng = np.random.default_rng(seed)
    prefixes = [bytes(rng.choice(ALPHA, size=prefix_len)) for _ in range(groups)]
    out = []
    for _ in range(n_shared):
        p = prefixes[int(rng.integers(0, groups))]
        r = rng.random()
        if r < 0.05:
            out.append(p[: prefix_len - int(rng.integers(1, 5))])  # ends inside the prefix
        elif r < 0.10:
            out.append(p)
        else:
            out.append(p + bytes(rng.choice(ALPHA, size=int(rng.integers(1, 7)))))
    for _ in range(n_unique):
        out.append(bytes(rng.choice(ALPHA, size=int(rng.integers(4, 31)))))
    order = rng.permutation(len(out))
    return [out[i] for i in order]


@pytest.mark.parametrize("index_u64", [False, True])
@pytest.mark.parametrize("prefix_len", [20, 40])
def test_runs_holding_every_string(cuda_lib, index_u64, prefix_len):
    """All strings in a handful of runs that stay constant for several rounds
    (prefixes of 20 and 40 chars against 9 coded ones): the window array
    serves every round."""
    hs = cuda_lib
    w = workloads.from_strings(_prefix_strings(150_000, 0, 5, prefix_len, prefix_len))
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off, index_u64=index_u64))


def test_runs_holding_a_minority(cuda_lib):
    """Runs with a fifth of the strings: each member's window is gathered."""
    hs = cuda_lib
    w = workloads.from_strings(_prefix_strings(40_000, 160_000, 4, 30, 7))
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


def test_runs_near_the_switch(cuda_lib):
    """Runs holding about two fifths of the strings, around the point where
    the window array starts to pay."""
    hs = cuda_lib
    for shared, seed in ((79_000, 3), (81_000, 4)):
        w = workloads.from_strings(_prefix_strings(shared, 200_000 - shared, 6, 33, seed))
        data, off = to_device(w)
        assert_oracle_equal(w, hs.argsort_device(data, off))


def test_batched_instances_of_shared_prefixes(cuda_lib):
    """The same through hs_argsort_batched: runs never cross instances, and
    each member's window comes from its global string index."""
    hs = cuda_lib
    w = workloads.from_strings(_prefix_strings(120_000, 10_000, 4, 36, 11))
    seg = np.array([0, 1, 30_000, 30_001, 90_000, w.n], dtype=np.uint64)
    data, off = to_device(w)
    d_seg = torch.from_numpy(seg.view(np.int64)).cuda()
    got = perm_numpy(hs.argsort_batched(data, off, d_seg)).astype(np.uint32)
    want = oracle.stable_argsort_batched(w.bytes, w.offsets, seg)
    assert np.array_equal(got, want)
