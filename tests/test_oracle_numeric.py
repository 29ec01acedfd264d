"""Pins for the oracle's numeric coders.

The codes are pinned by hand-worked values from the IEEE 754 and two's
complement layouts; the order by the compareTo rules it restates (-0.0 below
0.0, NaN equal to NaN and above +infinity); and the two against each other:
sorting by code must give the compareTo order, with equal codes exactly for
values compareTo calls equal."""

import numpy as np
import pytest

import oracle


def test_hand_worked_codes():
    f64 = np.array([1.0, -1.0, 0.0, -0.0, np.inf, -np.inf, np.nan], np.float64)
    assert [hex(int(c)) for c in oracle.numeric_code(f64, oracle.NUM_F64)] == [
        "0xbff0000000000000", "0x400fffffffffffff", "0x8000000000000000", "0x7fffffffffffffff",
        "0xfff0000000000000", "0xfffffffffffff", "0xfff8000000000000"]
    f32 = np.array([1.0, -1.0, -0.0], np.float32)
    assert [hex(int(c)) for c in oracle.numeric_code(f32, oracle.NUM_F32)] == ["0xbf800000", "0x407fffff", "0x7fffffff"]
    i64 = np.array([-1, 0, -(1 << 63), (1 << 63) - 1], np.int64)
    assert [hex(int(c)) for c in oracle.numeric_code(i64, oracle.NUM_I64)] == [
        "0x7fffffffffffffff", "0x8000000000000000", "0x0", "0xffffffffffffffff"]
    i32 = np.array([-1, 0, -(1 << 31)], np.int32)
    assert [hex(int(c)) for c in oracle.numeric_code(i32, oracle.NUM_I32)] == ["0x7fffffff", "0x80000000", "0x0"]


def test_double_order_special_values():
    """Written out by hand in Double.compare order."""
    order = [-np.inf, -1e308, -1.0, -5e-324, -0.0, 0.0, 5e-324, 1.0, 1e308, np.inf, np.nan]
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(order))
    v = np.array(order, np.float64)[perm]
    got = oracle.numeric_argsort(v, oracle.NUM_F64)
    assert list(perm[got]) == list(range(len(order)))


def _special_f64(rng, n):
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 5e-324, -5e-324, 1.0, -1.0], np.float64)
    v = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
    pick = rng.random(n) < 0.2
    v[pick] = specials[rng.integers(0, specials.size, size=int(pick.sum()))]
    nan_payload = rng.random(n) < 0.02  # NaNs with other payloads and signs
    bits = v.view(np.uint64)
    bits[nan_payload] = np.uint64(0x7FF0000000000001) | rng.integers(0, 1 << 50, size=int(nan_payload.sum()), dtype=np.uint64)
    bits[nan_payload & (rng.random(n) < 0.5)] |= np.uint64(1 << 63)
    return v


def _special_f32(rng, n):
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.0, -1.0], np.float32)
    v = (rng.standard_normal(n) * 10.0 ** rng.integers(-37, 37, size=n)).astype(np.float32)
    pick = rng.random(n) < 0.2
    v[pick] = specials[rng.integers(0, specials.size, size=int(pick.sum()))]
    nan_payload = rng.random(n) < 0.02
    bits = v.view(np.uint32)
    bits[nan_payload] = np.uint32(0x7F800001) | rng.integers(0, 1 << 22, size=int(nan_payload.sum()), dtype=np.uint32)
    bits[nan_payload & (rng.random(n) < 0.5)] |= np.uint32(1 << 31)
    return v


@pytest.mark.parametrize("type", ["f64", "f32", "i64", "i32", "u64"])
def test_code_order_is_compare_order(type):
    """Sorting by code (stable) reproduces the compareTo order, and codes
    are equal exactly where compareTo finds equality."""
    rng = np.random.default_rng(7)
    n = 20_000
    if type == "f64":
        v, t = _special_f64(rng, n), oracle.NUM_F64
    elif type == "f32":
        v, t = _special_f32(rng, n), oracle.NUM_F32
    elif type == "i64":
        v, t = rng.integers(-(1 << 63), (1 << 63) - 1, size=n, dtype=np.int64) >> rng.integers(0, 64, size=n), oracle.NUM_I64
    elif type == "i32":
        v, t = rng.integers(-(1 << 31), (1 << 31) - 1, size=n, dtype=np.int64).astype(np.int32) >> rng.integers(0, 32, size=n).astype(np.int32), oracle.NUM_I32
    else:
        v, t = rng.integers(0, 1 << 63, size=n, dtype=np.uint64) >> rng.integers(0, 64, size=n).astype(np.uint64), oracle.NUM_U64
    codes = oracle.numeric_code(v, t)
    want = oracle.numeric_argsort(v, t)
    assert np.array_equal(np.argsort(codes, kind="stable"), want)
    c = codes[want]
    if t in (oracle.NUM_F64, oracle.NUM_F32):
        with np.errstate(invalid="ignore"):
            w = v[want].astype(np.float64)
        same = (w[1:] == w[:-1]) & (np.signbit(w[1:]) == np.signbit(w[:-1])) | (np.isnan(w[1:]) & np.isnan(w[:-1]))
    else:
        w = v[want]
        same = w[1:] == w[:-1]
    assert np.array_equal(c[1:] == c[:-1], same)
    assert np.all(c[1:] >= c[:-1])
