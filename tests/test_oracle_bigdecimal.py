"""Pins for the oracle's BigDecimal order (the paper's Section 6.1 and
Table 4 benchmark BigDecimal arrays; compareTo orders by value, scale
ignored).  Hand-worked exact values, a hand-ordered list with groups of
equal values, agreement with Python's decimal module on random texts, and
the texts outside the grammar."""

import decimal
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import read_golden


def _pack(texts):
    off = np.zeros(len(texts) + 1, np.uint64)
    np.cumsum([len(t) for t in texts], out=off[1:])
    data = np.frombuffer(b"".join(texts), dtype=np.uint8).copy() if texts else np.zeros(0, np.uint8)
    return data, off


@pytest.mark.parametrize("row", read_golden("bigdecimal_values.txt"), ids=lambda r: r[0])
def test_hand_worked_values(row):
    text, num, den = row[0].encode(), int(row[1]), int(row[2])
    assert oracle.bigdecimal_value(text) == Fraction(num, den)


def test_hand_ordered_list_with_equal_groups():
    # ascending by value; texts on one line are equal values, in index order
    groups = [
        [b"-1E+3", b"-1000.0"],
        [b"-999.5"],
        [b"-1", b"-1.00", b"-0.1E+1"],
        [b"-0.5", b"-.5"],
        [b"-1E-10"],
        [b"0", b"-0", b"0.000", b"0E+99"],
        [b"1E-10"],
        [b"0.5", b"5E-1"],
        [b"1", b"1.0", b"+1", b"10E-1"],
        [b"1.5"],
        [b"10", b"1E+1", b"1e1"],
        [b"9.99E+999"],
    ]
    order = [t for g in groups for t in g]
    rng = random.Random(5)
    shuffled = order[:]
    rng.shuffle(shuffled)
    data, off = _pack(shuffled)
    got = [shuffled[i] for i in oracle.bigdecimal_argsort(data, off)]
    # the value groups come out in order; inside a group, in input (index) order
    flat = [t for g in groups for t in sorted(g, key=shuffled.index)]
    assert got == flat


def test_agrees_with_the_decimal_module():
    rng = random.Random(7)
    for _ in range(2000):
        sign = rng.choice(["", "-", "+"])
        whole = "".join(rng.choice("0123456789") for _ in range(rng.randint(0, 12)))
        frac = "".join(rng.choice("0123456789") for _ in range(rng.randint(0, 12)))
        if not whole and not frac:
            whole = "0"
        mant = whole + ("." + frac if frac or rng.random() < 0.3 else "")
        exp = f"E{rng.choice(['', '+', '-'])}{rng.randint(0, 400)}" if rng.random() < 0.5 else ""
        text = (sign + mant + exp).encode()
        assert oracle.bigdecimal_value(text) == Fraction(decimal.Decimal(text.decode())), text


def test_sort_key_orders_as_the_exact_values():
    """The sort key (Decimal) orders and equates texts exactly as their
    Fraction values do, on random texts with moderate exponents."""
    rng = random.Random(11)
    texts = []
    for _ in range(600):
        whole = "".join(rng.choice("0123456789") for _ in range(rng.randint(0, 6)))
        frac = "".join(rng.choice("0123456789") for _ in range(rng.randint(0, 6)))
        mant = (whole or "0") + ("." + frac if frac else "")
        exp = f"E{rng.randint(-30, 30)}" if rng.random() < 0.5 else ""
        texts.append((rng.choice(["", "-"]) + mant + exp).encode())
    for a, b in zip(texts, texts[1:] + texts[:1]):
        fa, fb = oracle.bigdecimal_value(a), oracle.bigdecimal_value(b)
        ka, kb = oracle.bigdecimal_key(a), oracle.bigdecimal_key(b)
        assert (fa < fb) == (ka < kb) and (fa == fb) == (ka == kb), (a, b)


def test_extreme_exponents_ordered_by_hand():
    # ascending; texts on one line are equal values
    groups = [
        [b"-1E+999999999", b"-10E+999999998"],
        [b"-9.99E+999999998"],
        [b"-1"],
        [b"-1E-999999999"],
        [b"0", b"0E+999999999"],
        [b"1E-999999999", b"0.1E-999999998"],
        [b"2E-999999999"],
        [b"1"],
        [b"9.99E+999999998"],
        [b"1E+999999999"],
    ]
    order = [t for g in groups for t in g]
    shuffled = order[::-1]
    data, off = _pack(shuffled)
    got = [shuffled[i] for i in oracle.bigdecimal_argsort(data, off)]
    assert got == [t for g in groups for t in sorted(g, key=shuffled.index)]


@pytest.mark.parametrize("text", [b"", b"-", b"+", b".", b"1e", b"1E+", b"1.2.3", b"1e5.5", b" 1", b"1 ",
                                  b"1_000", b"abc", b"0x10", b"inf", b"NaN", b"--1", b"1e--2", b"e5"])
def test_texts_outside_the_grammar(text):
    with pytest.raises(ValueError):
        oracle.bigdecimal_value(text)
    with pytest.raises(ValueError):
        oracle.bigdecimal_key(text)
