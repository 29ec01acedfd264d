"""Pins for the FP64 learned-bucketer oracle.

Gradients are pinned by central finite differences (independent of the
chain-rule code), the forward pass by a network set up to compute a known
function, the least-squares leaf fit by exact lines and by numpy.polyfit (a
library routine), and the bucket function by the monotonicity it must have.
"""

import numpy as np
import pytest

from oracle import rmi_oracle as R


def _random_params(rng, positive=True):
    p = R.init_params(int(rng.integers(1 << 30)))
    for k in p:
        p[k] = np.asarray(p[k], dtype=np.float64) + rng.normal(0, 0.05, np.shape(p[k]))
    if positive:
        for k in ("W1", "W2", "w3"):
            p[k] = np.abs(p[k])
    p["b3"] = np.float64(p["b3"])
    return p


def _loss(p, x, t):
    y, _ = R.forward(p, x)
    return float(np.mean((y - t) ** 2))


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = _random_params(rng, positive=False)
    x = np.sort(rng.uniform(0, 1, 257))
    t = np.linspace(0, 1, 257)
    _, g = R.loss_and_grad(p, x, t)
    h = 1e-6
    for k in p:
        flat = np.atleast_1d(p[k]).ravel()
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            def shifted(d):
                q = {kk: np.array(vv, dtype=np.float64, copy=True) for kk, vv in p.items()}
                arr = np.atleast_1d(q[k]).reshape(-1)
                arr[i] += d
                q[k] = arr.reshape(np.shape(p[k])) if np.ndim(p[k]) else np.float64(arr[0])
                return _loss(q, x, t)
            fd = (shifted(h) - shifted(-h)) / (2 * h)
            an = np.atleast_1d(g[k]).ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, an)


def test_forward_known_function():
    """W1 = e0, W2 = e0 e0^T, w3 = e0, zero biases: y = h(h(x)) = x on [0, 1]."""
    H = R.HIDDEN
    e0 = np.zeros(H); e0[0] = 1.0
    p = dict(W1=e0.copy(), b1=np.zeros(H), W2=np.outer(e0, e0), b2=np.zeros(H),
             w3=e0.copy(), b3=np.float64(0.25))
    x = np.linspace(0, 1, 11)
    y, _ = R.forward(p, x)
    assert np.allclose(y, x + 0.25, atol=0, rtol=0)


def test_sgd_projects_weights_not_biases():
    H = R.HIDDEN
    p = dict(W1=np.full(H, 0.1), b1=np.zeros(H), W2=np.full((H, H), 0.1),
             b2=np.zeros(H), w3=np.full(H, 0.1), b3=np.float64(0.0))
    g = {k: np.ones_like(np.asarray(v)) for k, v in p.items()}
    q = R.sgd_step(p, g, lr=1.0)
    assert np.all(q["W1"] == 0) and np.all(q["W2"] == 0) and np.all(q["w3"] == 0)
    assert np.all(q["b1"] == -1.0) and np.all(q["b2"] == -1.0) and q["b3"] == -1.0


def test_leaf_fit_exact_lines_and_polyfit():
    rng = np.random.default_rng(5)
    x = np.sort(rng.uniform(0, 1, 600))
    t = np.empty_like(x)
    starts = np.array([0, 200, 200, 450, 600])
    t[0:200] = 0.3 * x[0:200] + 0.1                 # exact line
    t[200:450] = rng.uniform(0, 1, 250)              # noisy
    t[450:600] = -2.0 * x[450:600] + 3.0             # negative slope
    slope, icept, lo, hi = R.leaf_fit(x, t, starts)
    assert slope[0] == pytest.approx(0.3, abs=1e-12)
    assert icept[0] == pytest.approx(0.1, abs=1e-12)
    assert slope[1] == 0.0 and icept[1] == lo[1]     # empty leaf
    k, b = np.polyfit(x[200:450], t[200:450], 1)
    if k >= 0:
        assert slope[2] == pytest.approx(k, rel=1e-9)
        assert icept[2] == pytest.approx(b, rel=1e-9, abs=1e-12)
    assert slope[3] == 0.0 and icept[3] == pytest.approx(t[450:600].mean())
    assert np.allclose(lo, starts[:-1] / 600) and np.allclose(hi, starts[1:] / 600)


def test_position_and_bucket_monotone():
    rng = np.random.default_rng(9)
    p = _random_params(rng, positive=True)
    codes = np.sort(rng.integers(0, 1 << 62, size=20000, dtype=np.uint64))
    cmin, cmax = int(codes[0]), int(codes[-1])
    s = R.feature_shift(cmin, cmax)
    x = R.feature(codes, cmin, s)
    assert np.all(np.diff(x) >= 0) and x.max() < 1.0
    y, _ = R.forward(p, x)
    assert np.all(np.diff(y) >= 0)
    leaves = 64
    l = R.leaf_of(y, leaves)
    starts = np.searchsorted(l, np.arange(leaves + 1))
    t = np.arange(x.size) / x.size
    lp = R.leaf_fit(x, t, starts)
    pos = R.position(p, lp, x, leaves)
    assert np.all(np.diff(pos) >= 0)
    b = R.bucket_of(pos, 1 << 10)
    assert np.all(np.diff(b) >= 0) and b.min() >= 0 and b.max() < 1 << 10


def test_training_reduces_loss():
    rng = np.random.default_rng(1)
    x = np.sort(rng.beta(0.5, 2.0, 4096))
    t = np.arange(x.size) / x.size
    p = R.init_params(0)
    l0, _ = R.loss_and_grad(p, x, t)
    for _ in range(200):
        _, g = R.loss_and_grad(p, x, t)
        p = R.sgd_step(p, g, lr=0.5)
    l1, _ = R.loss_and_grad(p, x, t)
    assert l1 < 0.5 * l0
    for k in ("W1", "W2", "w3"):
        assert np.all(p[k] >= 0)


def test_root_can_be_concave():
    """With ramps (unlike relu) a non-negative-weight root follows a concave
    CDF: the quantile init interpolates the empirical CDF of a skewed sample
    within a small error, far better than the identity."""
    rng = np.random.default_rng(3)
    x = np.sort(rng.beta(0.3, 3.0, 20000))           # mass piled near 0: concave CDF
    t = (np.arange(x.size) + 0.5) / x.size
    p = R.quantile_init(x)
    y, _ = R.forward(p, x)
    assert np.max(np.abs(y - t)) < 0.04
    assert np.max(np.abs(x - t)) > 0.4                # the linear map is far off
    assert np.all(np.diff(y) >= 0)


def test_thresholds_reproduce_the_root_step_function():
    """leaf(X) from the table equals floor(root(X 2^-24) L) at every X probed,
    including each threshold and its predecessor."""
    rng = np.random.default_rng(4)
    x = np.sort(rng.uniform(0, 1, 5000) ** 3)
    p = R.quantile_init(x)
    L = 64
    T = R.thresholds(p, L)
    assert np.all(np.diff(T) >= 0)
    probe = np.unique(np.concatenate([T, np.maximum(T - 1, 0),
                                      rng.integers(0, 1 << 24, 2000)]))
    probe = probe[probe < (1 << 24)]
    y, _ = R.forward(p, probe * 2.0 ** -24)
    assert np.array_equal(R.leaf_by_table(T, probe), R.leaf_of(y, L))


def test_sample_indices_one_per_block():
    idx = R.sample_indices(1_000_050, seed=7)
    assert idx.shape[0] == 10_000
    assert np.all(idx // 100 == np.arange(10_000))
    assert np.all(np.diff(idx) > 0)
    # the finaliser on 0 is 0, so block 0 of seed 0 is sampled at offset 0
    assert R.sample_indices(100, seed=0)[0] == 0
    # published SplitMix64 stream for seed 1234567: 6457827717110365317,
    # 3203168211198807973 (state advanced by 0x9E3779B97F4A7C15 before mixing)
    g = 0x9E3779B97F4A7C15
    M = (1 << 64) - 1
    assert R.mix64((1234567 + g) & M) == 6457827717110365317
    assert R.mix64((1234567 + 2 * g) & M) == 3203168211198807973
    seed = (1234567 + g) & M   # block k = 0 mixes k ^ seed = seed
    assert R.sample_indices(100, seed=seed)[0] == 6457827717110365317 % 100
    ks = np.arange(5, dtype=np.int64)
    idx = R.sample_indices(500, seed=99)
    assert [int(i) for i in idx] == [int(k) * 100 + R.mix64(int(k) ^ 99) % 100 for k in ks]


def test_leaf_relative_positions_monotone_and_finer():
    """Keys that share a 24-bit feature get distinct positions once each leaf
    works on the key's offset from its base; positions stay monotone."""
    rng = np.random.default_rng(11)
    # 40 clusters of 2,000 keys inside 2^30-wide windows, and one far key that
    # makes the range ~2^62 (shift 38): each cluster shares one 24-bit feature
    base = (np.arange(40, dtype=np.uint64) + np.uint64(1)) << np.uint64(55)
    low = rng.integers(0, 1 << 30, size=(40, 2000)).astype(np.uint64)
    keys = np.sort(np.concatenate([(base[:, None] + low).ravel(), [np.uint64((1 << 62) - 1)]]))
    cmin, cmax = int(keys[0]), int(keys[-1])
    shift = R.feature_shift(cmin, cmax)
    X = ((keys - np.uint64(cmin)) >> np.uint64(shift)).astype(np.int64)
    assert np.unique(X).size < 100
    t = (np.arange(keys.size) + 0.5) / keys.size
    p = R.quantile_init(X * 2.0 ** -24)
    L = 256                      # more leaves than clusters, as in use (4096)
    T = R.thresholds(p, L)
    leaf = R.leaf_by_table(T, X)
    kb, sc = R.leaf_bases(T, cmin, shift, L)
    xl = R.leaf_offsets(keys, leaf, kb, sc)
    assert np.all(xl >= 0) and np.all(xl <= 1.0)
    starts = np.searchsorted(leaf, np.arange(L + 1))
    slope, icept, lo, hi_ = R.leaf_fit(xl, t, starts)
    pos = np.clip(slope[leaf] * xl + icept[leaf], lo[leaf], hi_[leaf])
    assert np.all(np.diff(pos) >= 0)
    b = R.bucket_of(pos, 1 << 12)
    assert np.unique(b).size > 20 * np.unique(X).size   # far finer than the feature
