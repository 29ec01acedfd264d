"""GPU checks of the learned path (HS_MODE_LEARNED).

The permutation is integer work and must equal the oracle's bit for bit,
whatever the model does.  The model's pieces are checked against the FP64
oracle: the FP32 gradient within 1e-4 relative error, the FP64-summed
least-squares leaves within 1e-6, the sample indices exactly (both sides
implement SplitMix64), and the bucket function by the monotonicity the
method relies on.  The gain test shows what training buys over the untrained
linear bucketer on skewed keys."""

import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import assert_oracle_equal, assert_stable_sorted, to_device
from oracle import rmi_oracle as R

pytestmark = pytest.mark.gpu

PARAM_ORDER = [("W1", (32,)), ("b1", (32,)), ("W2", (32, 32)), ("b2", (32,)), ("w3", (32,)), ("b3", ())]


def _pack(p):
    return np.concatenate([np.atleast_1d(np.asarray(p[k], dtype=np.float64)).ravel() for k, _ in PARAM_ORDER])


def _unpack(v):
    out, o = {}, 0
    for k, shape in PARAM_ORDER:
        size = int(np.prod(shape)) if shape else 1
        out[k] = v[o:o + size].reshape(shape) if shape else np.float64(v[o])
        o += size
    return out


@pytest.mark.parametrize("kind", [1, 2, 3, 5])
@pytest.mark.parametrize("index_u64", [False, True])
def test_learned_matches_oracle(cuda_lib, kind, index_u64):
    hs = cuda_lib
    w = workloads.generate(kind, 1_000_003, 50 + kind)
    data, off = to_device(w)
    perm = hs.argsort_device(data, off, mode=hs.MODE_LEARNED, index_u64=index_u64)
    assert_oracle_equal(w, perm)


@pytest.mark.parametrize("bits", [9, 21, 23, 24])
@pytest.mark.parametrize("kind", [2, 5])
def test_learned_forced_bucket_bits_match_oracle(cuda_lib, kind, bits):
    """Above about 2.7e8 keys the learned path takes 23 or 24 bucket bits and
    three 9-bit partition passes (the branch of the 1e9 skewed workload).
    Forcing those widths at 1e6 strings checks that branch element by
    element against the oracle, with the u64 permutation the 1e9 workload
    uses; 9 bits (one pass, buckets far above the in-CTA bound) and 21 bits
    (a partial last digit) cover the other widths."""
    hs = cuda_lib
    w = workloads.generate(kind, 1_000_003, 70 + kind)
    data, off = to_device(w)
    hs.learned_force_bucket_bits(bits)
    try:
        perm = hs.argsort_device(data, off, mode=hs.MODE_LEARNED, index_u64=True)
        _, _, info = hs.learned_profile(data, off)
    finally:
        hs.learned_force_bucket_bits(0)
    assert info["bits"] == bits
    assert_oracle_equal(w, perm)


@pytest.mark.parametrize("bits", [1, 5, 12, 18])
@pytest.mark.parametrize("kind", [2, 5])
def test_learned_composite_bucket_widths(cuda_lib, kind, bits):
    """Byte-range keys carry the bucket id above them (one word through the
    partition), and the in-bucket sort works on windows of whole buckets,
    queueing their tie runs itself.  With 1 or 5 bucket bits every bucket is
    longer than a window, so the overflow sort and the tie runs found inside
    it carry the whole result; 12 bits give windows of many buckets, 18 bits
    windows of one or two.  Zipf words (kind 2) tie heavily past the 8 coded
    chars; skewed strings (kind 5) have a hot first letter."""
    hs = cuda_lib
    w = workloads.generate(kind, 300_007, 90 + kind)
    data, off = to_device(w)
    hs.learned_force_bucket_bits(bits)
    try:
        perm = hs.argsort_device(data, off, mode=hs.MODE_LEARNED, index_u64=kind == 5)
    finally:
        hs.learned_force_bucket_bits(0)
    assert_oracle_equal(w, perm)


@pytest.mark.slow
def test_learned_3e8_crosses_to_wide_buckets(cuda_lib):
    """3e8 skewed strings: the first size at which the learned path picks
    more than 18 bucket bits on its own; checked by the property check."""
    hs = cuda_lib
    w = workloads.generate(5, 300_000_000, 4)
    data, off = to_device(w)
    perm = hs.argsort_device(data, off, mode=hs.MODE_LEARNED, index_u64=True)
    del data, off
    assert_stable_sorted(w, perm)


@pytest.mark.slow
def test_learned_full_skewed_1e9(cuda_lib):
    """The learned arm of the 1e9 skewed workload as the bench runs it (u64
    permutation, 24 bucket bits), checked by the property check (a
    permutation, in order, equal strings by index), which fixes the stable
    argsort uniquely."""
    hs = cuda_lib
    w = workloads.standard("skewed_1e9")
    data, off = to_device(w)
    perm = hs.argsort_device(data, off, mode=hs.MODE_LEARNED, index_u64=True)
    del data, off
    assert perm.dtype.itemsize == 8
    assert_stable_sorted(w, perm)


@pytest.mark.parametrize("case", ["equal_long", "few_distinct", "sorted", "byte8_fallback", "just_above_min"])
def test_learned_edge_cases(cuda_lib, case):
    hs = cuda_lib
    n = 200_000
    if case == "equal_long":
        strs = [b"the-same-string-longer-than-nine"] * n
    elif case == "few_distinct":
        strs = [b"word%02dxxxxxxxx" % (i % 37) + bytes([97 + i % 5]) for i in range(n)]
    elif case == "sorted":
        strs = [b"%010d" % i for i in range(n)]
    elif case == "byte8_fallback":
        rng = np.random.default_rng(1)
        strs = [bytes(rng.integers(0, 256, size=rng.integers(0, 12)).astype(np.uint8)) for _ in range(n)]
    else:
        w = workloads.generate(2, 65_536, 3)
        strs = [w.string(i) for i in range(w.n)]
    w = workloads.from_strings(strs)
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off, mode=hs.MODE_LEARNED))


def test_learned_small_n_uses_plain(cuda_lib):
    hs = cuda_lib
    w = workloads.generate(5, 1000, 2)
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off, mode=hs.MODE_LEARNED))


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_fp64_oracle(cuda_lib, seed):
    hs = cuda_lib
    rng = np.random.default_rng(seed)
    p = R.init_params(seed)
    for k in p:
        p[k] = np.asarray(p[k], dtype=np.float64) + rng.normal(0, 0.05, np.shape(p[k]))
    for k in ("W1", "W2", "w3"):
        p[k] = np.abs(p[k])
    T = 1500
    x = np.sort(rng.uniform(0, 1, T)).astype(np.float32)
    t = ((np.arange(T) + 0.5) / T).astype(np.float32)
    p32 = _pack(p).astype(np.float32)
    # the oracle sees exactly the FP32 inputs the kernel sees
    pq = _unpack(p32.astype(np.float64))
    loss_o, g_o = R.loss_and_grad(pq, x.astype(np.float64), t.astype(np.float64))
    loss_g, g_g = hs.rmi_grad(torch.from_numpy(p32).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    gg = _unpack(g_g.cpu().numpy().astype(np.float64))
    assert abs(loss_g - loss_o) <= 1e-4 * abs(loss_o)
    for k, _ in PARAM_ORDER:
        a, b = np.atleast_1d(gg[k]), np.atleast_1d(g_o[k])
        scale = max(np.max(np.abs(b)), 1e-12)
        assert np.max(np.abs(a - b)) <= 1e-4 * scale, k


def test_leaf_fit_matches_fp64_oracle(cuda_lib):
    hs = cuda_lib
    rng = np.random.default_rng(7)
    m = 50_000
    x = np.sort(rng.uniform(0, 1, m) ** 2).astype(np.float32)
    t = ((np.arange(m) + 0.5) / m).astype(np.float32)
    cuts = np.sort(rng.choice(np.arange(1, m), size=255, replace=False))
    starts = np.concatenate([[0], cuts, [m]]).astype(np.uint32)
    starts[10] = starts[9]                              # an empty leaf
    starts[20] = starts[19] + 1                         # a single-point leaf
    starts = np.maximum.accumulate(starts)
    got = hs.rmi_leaf_fit(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(),
                          torch.from_numpy(starts.view(np.int32)).cuda())
    want = R.leaf_fit(x.astype(np.float64), t.astype(np.float64), starts.astype(np.int64))
    for g, w_ in zip(got, want):
        assert np.allclose(g.cpu().numpy().astype(np.float64), w_, rtol=1e-6, atol=1e-7)


def test_sample_indices_match_oracle(cuda_lib):
    hs = cuda_lib
    for n, seed in [(1_000_000, 0x5DEECE66D), (12_345_678, 3)]:
        got = hs.rmi_sample_indices(n, seed).cpu().numpy()
        assert np.array_equal(got, R.sample_indices(n, seed))


@pytest.mark.parametrize("kind", [1, 2, 5])
def test_bucket_function_is_monotone(cuda_lib, kind):
    hs = cuda_lib
    w = workloads.generate(kind, 2_000_000, 60 + kind)
    data, off = to_device(w)
    keys, buckets, info = hs.learned_profile(data, off)
    k = keys.cpu().numpy().view(np.uint64)
    b = buckets.cpu().numpy().view(np.uint32)
    order = np.argsort(k, kind="stable")
    assert np.all(np.diff(b[order].astype(np.int64)) >= 0)
    assert b.max() < (1 << info["bits"])
    assert info["loss1"] <= info["loss0"] * 1.0001   # the gradient steps do not make it worse


def test_training_gain_over_linear_bucketer(cuda_lib):
    """On the skewed workload (first letter Zipf(1.5): ~45% of keys in 1/26
    of code space) the trained model spreads the distinct keys over far more
    buckets than the untrained linear bucketer, which piles thousands of
    distinct keys into single buckets.  Counted on distinct keys, since a
    bucket holding many copies of one key is no fault of the model."""
    hs = cuda_lib
    w = workloads.generate(5, 4_000_000, 4)
    data, off = to_device(w)
    keys, b_trained, info = hs.learned_profile(data, off)
    _, b_linear, _ = hs.learned_profile(data, off, linear=True)
    B = 1 << info["bits"]
    _, first = np.unique(keys.cpu().numpy().view(np.uint64), return_index=True)
    stats = []
    for b in (b_trained, b_linear):
        b = b.cpu().numpy().view(np.uint32)
        count = np.bincount(b, minlength=B)
        distinct = np.bincount(b[first], minlength=B)
        stats.append((count, distinct, np.percentile(distinct[distinct > 0], 99)))
    (ct, dt, p99t), (cl, dl, p99l) = stats
    assert p99t * 10 < p99l
    assert dt.max() < dl.max()
    assert (ct > 4096).sum() <= (cl > 4096).sum()
    assert (ct > 0).sum() > 2 * (cl > 0).sum()        # the model spreads keys over more buckets
