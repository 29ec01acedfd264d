"""Learned-bucketer (RMI) oracle -- TEST INFRASTRUCTURE ONLY.

FP64 numpy restatement of the recursive-model index that steers the learned
sort path.  The paper has no learned model: Huskysort's only requirement on a
bucketing of the codes is the one it states for husky codes themselves
(Section 3.2): whenever x > y the sort key of x must not be below that of y.
A bucket function that is monotone non-decreasing in the code therefore leaves
only equal-bucket elements to be ordered, which is exactly what the learned
path relies on.  The model below is built so that monotonicity holds by
construction, in FP64 here and in FP32 on the device:

  feature    x(code) = ((code - cmin) >> shift) * 2**-24, shift chosen so the
             shifted range fits in 24 bits (exact in FP32 and FP64);
  root       y = w3 . h(W2 h(W1 x + b1) + b2) + b3, 1 -> 32 -> 32 -> 1, with
             the ramp h(z) = min(max(z, 0), 1) and W1, W2, w3 >= 0 (projected
             after every SGD step), so y is non-decreasing in x.  (With relu
             and non-negative weights the root could only be convex; sums of
             ramps can follow any monotone, e.g. concave, CDF.);
  init       first-layer ramp j rises over [q_j, q_{j+1}] between consecutive
             1/32-quantiles of the sample, second layer identity, w3 = 1/32:
             the untrained root already interpolates the empirical CDF;
  training   full-batch gradient descent on mean squared error against the
             empirical CDF targets t_j = j / m of the sorted sample;
  leaves     leaf(x) = clamp(floor(y(x) * L), 0, L - 1), L linear leaves;
             leaf l is fitted by least squares to the sample points routed to
             it, slope clamped >= 0, and its output is clamped into the band
             [c_l, c_{l+1}] where c_l is the fraction of sample points routed
             to leaves below l;
  bucket     bucket(x) = min(B - 1, floor(pos(x) * B)).

  leaf-relative inputs: the 24-bit feature only routes keys to leaves; each
             leaf's line is evaluated on the key's full offset from the
             leaf's base key, kb_l = cmin + (T_l << shift) (T_0 = 0), scaled
             by s_l = 2^-e_l, e_l the bit length of the leaf's key range, so
             keys sharing a 24-bit feature are still told apart.  The offset
             is >= 0 for every key routed to the leaf, and converting it to
             floating point and scaling are monotone, so pos stays monotone.

  leaf table leaf(X) = number of thresholds <= X, thresholds T_l = the least
             integer feature X with floor(root(X 2^-24) L) >= l, l = 1..L-1
             (the exact step function of the monotone root, as a table).

Nothing here is shared with the CUDA library.  The derivative of the ramp is
taken as 1 strictly inside (0, 1) and 0 elsewhere.
"""

import numpy as np

HIDDEN = 32
FEATURE_BITS = 24


def feature_shift(cmin: int, cmax: int) -> int:
    """Right shift that brings (cmax - cmin) below 2**24."""
    span = int(cmax) - int(cmin)
    return max(0, span.bit_length() - FEATURE_BITS)


def feature(codes: np.ndarray, cmin: int, shift: int) -> np.ndarray:
    """x = ((code - cmin) >> shift) * 2**-24 as float64 (exact)."""
    c = codes.astype(np.uint64)
    q = (c - np.uint64(cmin)) >> np.uint64(shift)
    return q.astype(np.float64) * (2.0 ** -FEATURE_BITS)


MAX_SLOPE = float(1 << 20)


def ramp(z):
    return np.minimum(np.maximum(z, 0.0), 1.0)


def ramp_grad(z):
    return ((z > 0.0) & (z < 1.0)).astype(np.float64)


def init_params(seed: int = 0) -> dict:
    """A monotone starting point: ramps spread evenly over [0, 1), identity
    second layer, readout 1/32 -- the root is then y = x."""
    rng = np.random.default_rng(seed)
    W1 = np.full(HIDDEN, float(HIDDEN))
    b1 = -np.arange(HIDDEN, dtype=np.float64)
    W2 = np.eye(HIDDEN) + rng.uniform(0.0, 1e-3, size=(HIDDEN, HIDDEN))
    b2 = np.zeros(HIDDEN)
    w3 = np.full(HIDDEN, 1.0 / HIDDEN)
    b3 = 0.0
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, w3=w3, b3=np.float64(b3))


def quantile_init(x_sorted: np.ndarray) -> dict:
    """Ramp j rises over [q_j, q_{j+1}], q_j = x at rank floor(j m / 32) of
    the sorted sample (q_32 = the last x); slopes capped at 2^20; identity
    second layer; w3 = 1/32.  root(x) is then the piecewise-linear
    interpolation of the empirical CDF through the 33 quantile knots."""
    m = x_sorted.shape[0]
    q = np.array([x_sorted[min(m - 1, (j * m) // HIDDEN)] for j in range(HIDDEN)] +
                 [x_sorted[m - 1]], dtype=np.float64)
    W1 = np.empty(HIDDEN)
    b1 = np.empty(HIDDEN)
    for j in range(HIDDEN):
        width = q[j + 1] - q[j]
        W1[j] = MAX_SLOPE if width * MAX_SLOPE <= 1.0 else 1.0 / width
        b1[j] = -q[j] * W1[j]
    return dict(W1=W1, b1=b1, W2=np.eye(HIDDEN), b2=np.zeros(HIDDEN),
                w3=np.full(HIDDEN, 1.0 / HIDDEN), b3=np.float64(0.0))


def forward(p: dict, x: np.ndarray):
    """Root network output y for every x, plus the activations."""
    z1 = np.outer(x, p["W1"]) + p["b1"]          # (m, 32)
    h1 = ramp(z1)
    z2 = h1 @ p["W2"].T + p["b2"]                # (m, 32)
    h2 = ramp(z2)
    y = h2 @ p["w3"] + p["b3"]                   # (m,)
    return y, (z1, h1, z2, h2)


def loss_and_grad(p: dict, x: np.ndarray, t: np.ndarray):
    """Mean squared error (1/m) sum (y - t)^2 and its exact gradient by the
    chain rule through both ramp layers."""
    m = x.shape[0]
    y, (z1, h1, z2, h2) = forward(p, x)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / m                             # dL/dy
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.float64(dy.sum())
    dz2 = np.outer(dy, p["w3"]) * ramp_grad(z2)  # dL/dz2
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * ramp_grad(z1)        # dL/dz1
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def sgd_step(p: dict, g: dict, lr: float) -> dict:
    """theta <- theta - lr * grad, then clamp the weights (not the biases) to
    be non-negative so the root stays monotone."""
    q = {k: p[k] - lr * g[k] for k in p}
    for k in ("W1", "W2", "w3"):
        q[k] = np.maximum(q[k], 0.0)
    q["b3"] = np.float64(q["b3"])
    return q


def leaf_of(y: np.ndarray, leaves: int) -> np.ndarray:
    """Leaf index clamp(floor(y * L), 0, L - 1)."""
    v = np.floor(y * leaves)
    return np.clip(v, 0, leaves - 1).astype(np.int64)


def leaf_fit(x: np.ndarray, t: np.ndarray, leaf_start: np.ndarray):
    """Least-squares line per leaf over contiguous point ranges.

    leaf_start has L + 1 entries; leaf l owns points leaf_start[l] ..
    leaf_start[l+1] - 1.  Returns (slope, intercept, band_lo, band_hi), each of
    length L.  Normal equations: slope = (S Sxy - Sx Sy) / (S Sxx - Sx^2),
    intercept = (Sy - slope Sx) / S.  A leaf with fewer than two points, no
    spread in x, or a negative fitted slope gets slope 0 and intercept mean(t)
    (or its band start when empty).  Bands: c_l = leaf_start[l] / m.
    """
    L = leaf_start.shape[0] - 1
    m = leaf_start[-1]
    slope = np.zeros(L)
    icept = np.zeros(L)
    lo = leaf_start[:-1].astype(np.float64) / max(m, 1)
    hi = leaf_start[1:].astype(np.float64) / max(m, 1)
    for l in range(L):
        a, b = leaf_start[l], leaf_start[l + 1]
        S = b - a
        if S == 0:
            icept[l] = lo[l]
            continue
        xs, ts = x[a:b], t[a:b]
        Sx, Sy = xs.sum(), ts.sum()
        Sxx, Sxy = (xs * xs).sum(), (xs * ts).sum()
        den = S * Sxx - Sx * Sx
        if S >= 2 and den > 0.0:
            k = (S * Sxy - Sx * Sy) / den
        else:
            k = 0.0
        if k < 0.0:
            k = 0.0
        slope[l] = k
        icept[l] = (Sy - k * Sx) / S
    return slope, icept, lo, hi


def position(p: dict, leaf_params, x: np.ndarray, leaves: int) -> np.ndarray:
    """pos(x) = clamp(a_l x + b_l, c_l, c_{l+1}) with l = leaf(root(x))."""
    slope, icept, lo, hi = leaf_params
    y, _ = forward(p, x)
    l = leaf_of(y, leaves)
    return np.clip(slope[l] * x + icept[l], lo[l], hi[l])


def bucket_of(pos: np.ndarray, buckets: int) -> np.ndarray:
    """bucket = min(B - 1, floor(pos * B)), pos in [0, 1]."""
    b = np.floor(pos * buckets).astype(np.int64)
    return np.clip(b, 0, buckets - 1)


def thresholds(p: dict, leaves: int) -> np.ndarray:
    """T_l (l = 1..L-1) = least integer X in [0, 2^24) with
    floor(root(X 2^-24) L) >= l, else 2^24; by bisection on the monotone root."""
    out = np.empty(leaves - 1, dtype=np.int64)
    top = 1 << FEATURE_BITS
    for l in range(1, leaves):
        lo, hi = 0, top
        while lo < hi:
            mid = (lo + hi) // 2
            y, _ = forward(p, np.array([mid * 2.0 ** -FEATURE_BITS]))
            if leaf_of(y, leaves)[0] >= l:
                hi = mid
            else:
                lo = mid + 1
        out[l - 1] = lo
    return out


def leaf_by_table(thresh: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Number of thresholds <= X (thresholds sorted)."""
    return np.searchsorted(thresh, X, side="right")


def mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014)."""
    M = (1 << 64) - 1
    z &= M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def sample_indices(n: int, seed: int, stride: int = 100) -> np.ndarray:
    """One index per block of `stride` consecutive elements, at offset
    splitmix64(seed ^ k) mod stride within block k (SplitMix64 finaliser:
    Steele, Lea and Flood, OOPSLA 2014)."""
    m = n // stride
    k = np.arange(m, dtype=np.uint64)
    z = k ^ np.uint64(seed)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (k * np.uint64(stride) + z % np.uint64(stride)).astype(np.int64)


def leaf_bases(thresh: np.ndarray, cmin: int, shift: int, leaves: int):
    """(kb_l, s_l) per leaf: base key cmin + (T_l << shift) with T_0 = 0 and
    T_l = thresh[l-1]; s_l = 2^-e_l, e_l = bit length of
    (T_{l+1} - T_l) << shift (T_L = 2^24); s_l = 1 for an empty range."""
    T = np.concatenate([[0], np.asarray(thresh, dtype=np.int64), [1 << FEATURE_BITS]])
    kb = [int(cmin) + (int(T[l]) << shift) for l in range(leaves)]
    sc = []
    for l in range(leaves):
        rng = (int(T[l + 1]) - int(T[l])) << shift
        sc.append(2.0 ** -rng.bit_length() if rng > 0 else 1.0)
    return kb, np.array(sc)


def leaf_offsets(keys: np.ndarray, leaf: np.ndarray, kb, sc) -> np.ndarray:
    """Scaled offset (key - kb_l) * s_l of every key within its leaf."""
    out = np.empty(keys.shape[0])
    for i, (k, l) in enumerate(zip(keys, leaf)):
        out[i] = float(int(k) - kb[int(l)]) * sc[int(l)]
    return out
