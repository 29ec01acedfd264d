"""Pins for the oracle's BigInteger order: hand-ordered values around the
sign and byte-length boundaries, and the minimal encoding of Java's
toByteArray worked by hand."""

import numpy as np

import oracle
import workloads


def test_minimal_bytes_hand_worked():
    assert oracle.bigint_bytes(0) == b"\x00"
    assert oracle.bigint_bytes(-1) == b"\xff"
    assert oracle.bigint_bytes(127) == b"\x7f"
    assert oracle.bigint_bytes(128) == b"\x00\x80"
    assert oracle.bigint_bytes(-128) == b"\x80"
    assert oracle.bigint_bytes(-129) == b"\xff\x7f"
    assert oracle.bigint_bytes(256) == b"\x01\x00"
    assert oracle.bigint_bytes(-(1 << 64)) == b"\xff" + b"\x00" * 8


def test_order_hand_worked():
    order = [-(1 << 64), -129, -128, -1, 0, 127, 128, 256, 1 << 64]
    rng = np.random.default_rng(1)
    perm = rng.permutation(len(order))
    w = workloads.from_strings([oracle.bigint_bytes(order[i]) for i in perm])
    got = oracle.bigint_argsort(w.bytes, w.offsets)
    assert [order[perm[i]] for i in got] == order


def test_ties_keep_index_order():
    vals = [5, -3, 5, 0, -3, 5]
    w = workloads.from_strings([oracle.bigint_bytes(x) for x in vals])
    assert list(oracle.bigint_argsort(w.bytes, w.offsets)) == [1, 4, 3, 0, 2, 5]
