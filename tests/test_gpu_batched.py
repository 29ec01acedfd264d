"""GPU parity for hs_argsort_batched: every instance's local permutation
equals the oracle's stable argsort of that instance, bit for bit."""

import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import to_device

pytestmark = pytest.mark.gpu


def _run(hs, w, seg):
    data, off = to_device(w)
    d_seg = torch.from_numpy(np.ascontiguousarray(seg).view(np.int64)).cuda()
    perm = hs.argsort_batched(data, off, d_seg)
    return perm.cpu().numpy().view(np.uint32)


def _check(w, seg, got):
    want = oracle.stable_argsort_batched(w.bytes, w.offsets, seg)
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{bad.size} positions differ; first at {bad[0]}")


def test_small_instances_with_empty_and_single(cuda_lib):
    hs = cuda_lib
    w = workloads.generate_batched(60, 5, lo=1, hi=5000)
    seg = w.seg_offsets.copy()
    seg[3] = seg[2]          # empty instance
    seg[7] = seg[6] + 1      # single-string instance
    _check(w, seg, _run(hs, w, seg))


def test_single_instance_equals_hs_argsort(cuda_lib):
    hs = cuda_lib
    w = workloads.generate(2, 300_000, 8)
    seg = np.array([0, w.n], dtype=np.uint64)
    got = _run(hs, w, seg)
    data, off = to_device(w)
    ref = hs.argsort_device(data, off).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("kind", [1, 2, 3, 5])
def test_mixed_workloads(cuda_lib, kind):
    """Instances cut from each workload kind, so every fix-up class (warp,
    CTA, refinement) runs inside instances and runs never cross them."""
    hs = cuda_lib
    w = workloads.generate(kind, 600_000, 30 + kind)
    rng = np.random.default_rng(kind)
    cuts = np.sort(rng.choice(np.arange(1, w.n), size=40, replace=False))
    seg = np.concatenate([[0], cuts, [w.n]]).astype(np.uint64)
    _check(w, seg, _run(hs, w, seg))


def test_long_identical_runs_across_boundaries(cuda_lib):
    """Equal long strings straddling instance boundaries: each instance sorts
    its own copies (runs must end at the boundary)."""
    hs = cuda_lib
    strs = [b"the-same-string-longer-than-nine"] * 9000 + [b"abcdefghij" + bytes([97 + i % 3]) for i in range(9000)]
    rng = np.random.default_rng(0)
    w = workloads.from_strings([strs[i] for i in rng.permutation(len(strs))])
    seg = np.array([0, 1, 2500, 2501, 7000, 12000, w.n], dtype=np.uint64)
    _check(w, seg, _run(hs, w, seg))


def test_high_bytes_fall_back_to_byte8(cuda_lib):
    hs = cuda_lib
    rng = np.random.default_rng(2)
    strs = [bytes(rng.integers(0, 256, size=rng.integers(0, 14)).astype(np.uint8)) for _ in range(30_000)]
    w = workloads.from_strings(strs)
    seg = np.array([0, 10_000, 10_001, 30_000], dtype=np.uint64)
    _check(w, seg, _run(hs, w, seg))


def test_bad_seg_offsets_rejected(cuda_lib):
    hs = cuda_lib
    w = workloads.generate(1, 1000, 1)
    for seg in ([0, 600, 400, 1000], [1, 500, 1000], [0, 500, 999]):
        with pytest.raises(hs.HuskyError) as e:
            _run(hs, w, np.array(seg, dtype=np.uint64))
        assert e.value.status == hs.ERR_INVALID_ARG


def test_matches_per_instance_plain_loop(cuda_lib):
    hs = cuda_lib
    w = workloads.generate_batched(12, 9, lo=100, hi=200_000)
    got = _run(hs, w, w.seg_offsets)
    for s in range(12):
        lo, hi = int(w.seg_offsets[s]), int(w.seg_offsets[s + 1])
        sub = workloads.from_strings([w.string(i) for i in range(lo, hi)])
        data, off = to_device(sub)
        ref = hs.argsort_device(data, off).cpu().numpy().view(np.uint32)
        assert np.array_equal(got[lo:hi], ref), s


@pytest.mark.slow
def test_batched_2000_instances(cuda_lib):
    """The batched workload's shape at 2,000 instances (log-uniform 100..1e6,
    about 2.2e8 strings), checked by the per-instance property check."""
    hs = cuda_lib
    w = workloads.standard("batched_20000", scale=0.1)
    got = _run(hs, w, w.seg_offsets)
    assert oracle.check_sorted_batched(w.bytes, w.offsets, w.seg_offsets, got) == -1


@pytest.mark.slow
def test_batched_20000_instances_literal_size(cuda_lib):
    """The batched workload at its literal size: 20,000 instances of
    log-uniform sizes 100..1e6, about 2.17e9 strings in one call (more than
    2^31 positions; each instance's local indices stay below 2^31), checked
    instance by instance by the oracle's property check."""
    hs = cuda_lib
    w = workloads.standard("batched_20000")
    assert w.n > 2**31 and len(w.seg_offsets) == 20_001
    got = _run(hs, w, w.seg_offsets)
    assert oracle.check_sorted_batched(w.bytes, w.offsets, w.seg_offsets, got) == -1


@pytest.mark.parametrize("num_segs", [3, 511, 20_000, 300_000])
def test_instance_id_packed_into_the_key(cuda_lib, num_segs):
    """Lowercase strings (the byte-range coder's 5 bits, a 41-bit key) with the
    instance id packed above the key: 3 .. 300,000 instances (up to 19 bits)
    all fit; duplicates and strings longer than the code stress the fix-up
    across instance boundaries."""
    hs = cuda_lib
    rng = np.random.default_rng(num_segs)
    n = 1_200_000
    cuts = np.sort(rng.choice(np.arange(1, n), size=num_segs - 1, replace=False))
    seg = np.concatenate([[0], cuts, [n]]).astype(np.uint64)
    vocab = [bytes(rng.integers(97, 123, size=rng.integers(3, 16)).astype(np.uint8)) for _ in range(3000)]
    strs = [vocab[i] for i in rng.integers(0, len(vocab), size=n)]
    w = workloads.from_strings(strs)
    _check(w, seg, _run(hs, w, seg))


def test_instance_ids_too_wide_for_the_packed_key(cuda_lib):
    """2**23 + 5 instances need 24 bits: with the 41-bit key of lowercase
    text that passes 64, so the batched sort keeps the instance ids in their
    own array.  Mostly single-string instances, some longer, an empty one."""
    hs = cuda_lib
    rng = np.random.default_rng(11)
    num_segs = (1 << 23) + 5
    sizes = np.ones(num_segs, np.int64)
    np.add.at(sizes, rng.integers(1, num_segs, size=200_000), 1)
    sizes[0] = 0
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    w = workloads.generate(1, int(seg[-1]), 12)     # lowercase, lengths 4..12
    _check(w, seg, _run(hs, w, seg))
