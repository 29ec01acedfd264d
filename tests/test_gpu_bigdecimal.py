"""GPU parity for the BigDecimal coder: the stable argsort by numeric value
(compareTo's order: scale ignored, equal values in index order) of decimal
texts, against the oracle's exact rational values."""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import perm_numpy, to_device

pytestmark = pytest.mark.gpu

SPECIAL = [b"0", b"-0", b"+0.0", b"0E-5", b"1", b"-1", b"1E+999999999", b"-1E+999999999", b"1E-999999999",
           b"-1E-999999999", b"9.99", b"-9.99"]


def _texts(n, seed):
    """Decimal texts of every form: signs, leading and trailing zeros, a point
    anywhere or nowhere, exponents, zeros, the same value at other scales,
    long mantissas sharing their first 40 digits, and repeats."""
    rng = np.random.default_rng(seed)
    digits = list("0123456789")
    out = []
    for _ in range(n):
        r = rng.random()
        if r < 0.08 and out:
            out.append(out[int(rng.integers(0, len(out)))])  # a repeat
            continue
        if r < 0.14 and out:  # the same value at another scale
            t = out[int(rng.integers(0, len(out)))].decode()
            if "e" in t.lower():
                out.append(t.encode())
            elif "." in t:
                out.append((t + "0" * int(rng.integers(1, 4))).encode())
            else:
                out.append((t + ".00").encode())
            continue
        if r < 0.18:
            out.append(SPECIAL[int(rng.integers(0, len(SPECIAL)))])
            continue
        sign = ["", "-", "+"][int(rng.choice(3, p=[0.45, 0.45, 0.10]))]
        if r < 0.28:  # ties past the byte coder's 8 bytes
            whole = "3141592653589793238462643383279502884197" + "".join(
                rng.choice(digits, size=int(rng.integers(0, 30))))
            frac = ""
        else:
            whole = "".join(rng.choice(digits, size=int(rng.integers(0, 14))))
            frac = "".join(rng.choice(digits, size=int(rng.integers(0, 14))))
        if not whole and not frac:
            whole = "0"
        mant = whole + ("." + frac if frac or rng.random() < 0.2 else "")
        exp = ""
        if rng.random() < 0.4:
            exp = ["E", "e"][int(rng.integers(0, 2))] + ["", "+", "-"][int(rng.integers(0, 3))] + \
                str(int(rng.integers(0, 60)))
        out.append((sign + mant + exp).encode())
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 1024, 4097, 100_003])
@pytest.mark.parametrize("index_u64", [False, True])
def test_bigdecimal_argsort_matches_oracle(cuda_lib, n, index_u64):
    hs = cuda_lib
    w = workloads.from_strings(_texts(n, n + 17))
    data, off = to_device(w)
    got = perm_numpy(hs.argsort_bigdecimal(data, off, index_u64=index_u64)).astype(np.int64)
    assert np.array_equal(got, oracle.bigdecimal_argsort(w.bytes, w.offsets))


def test_equal_values_at_other_scales_keep_index_order(cuda_lib):
    hs = cuda_lib
    texts = [b"1.50", b"-2", b"15E-1", b"1.5", b"-2.000", b"0.15E+1", b"0", b"-0.0", b"150E-2", b"-20E-1"]
    w = workloads.from_strings(texts)
    data, off = to_device(w)
    got = perm_numpy(hs.argsort_bigdecimal(data, off)).astype(np.int64)
    assert got.tolist() == [1, 4, 9, 6, 7, 0, 2, 3, 5, 8]
    assert np.array_equal(got, oracle.bigdecimal_argsort(w.bytes, w.offsets))


@pytest.mark.parametrize("bad", [b"", b"-", b".", b"1e", b"1.2.3", b"1e5.5", b" 1", b"1_0", b"abc", b"NaN",
                                 b"1E+1000000000"])
def test_texts_outside_the_grammar_are_rejected(cuda_lib, bad):
    hs = cuda_lib
    w = workloads.from_strings([b"1", bad, b"2"])
    data, off = to_device(w)
    with pytest.raises(Exception) as e:
        hs.argsort_bigdecimal(data, off)
    assert "decimal" in str(e.value)
    ok = workloads.from_strings([b"2", b"1"])  # the context stays usable
    d2, o2 = to_device(ok)
    assert perm_numpy(hs.argsort_bigdecimal(d2, o2)).tolist() == [1, 0]
