"""Pins for the oracle's stable argsort and its property checker.

The argsort is checked against a worked example (tests/golden/tiny_sort.txt),
against Python's own stable sort (an independent implementation), and through
the characterisation it must satisfy (permutation + sorted + stable), on random
and adversarial inputs.  The checker is checked by planting mistakes.
"""

import numpy as np
import pytest

import oracle
import workloads
from conftest import literal, read_golden


def _python_sort(w):
    return np.array(sorted(range(w.n), key=w.string), dtype=np.int64)


def test_worked_example():
    rows = dict((r[0], r[1]) for r in read_golden("tiny_sort.txt"))
    w = workloads.from_strings(literal(rows["strings"]))
    expected = np.array(literal(rows["perm"]))
    for threads in (1, 3):
        assert np.array_equal(oracle.stable_argsort(w.bytes, w.offsets,
                                                    threads=threads), expected)
    assert oracle.check_sorted(w.bytes, w.offsets,
                               expected.astype(np.uint32)) == -1


def _random_strings(rng, n, alphabet, max_len):
    lens = rng.integers(0, max_len + 1, size=n)
    return [bytes(rng.choice(alphabet, size=L).astype(np.uint8)) for L in lens]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("threads", [1, 2, 5])
def test_matches_python_sorted(seed, threads):
    rng = np.random.default_rng(seed)
    alphabet = np.array([0x00, 0x01, 0x61, 0x62, 0x7F, 0x80, 0xFF])
    w = workloads.from_strings(_random_strings(rng, 3000, alphabet, 6))
    perm = oracle.stable_argsort(w.bytes, w.offsets, threads=threads)
    assert np.array_equal(perm.astype(np.int64), _python_sort(w))


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5])
def test_workloads_match_python_sorted(kind):
    w = workloads.generate(kind, 20000, 7)
    perm = oracle.stable_argsort(w.bytes, w.offsets, index_u64=True, threads=4)
    assert np.array_equal(perm.astype(np.int64), _python_sort(w))
    assert oracle.check_sorted(w.bytes, w.offsets, perm) == -1


@pytest.mark.parametrize("case", ["equal", "empty", "sorted", "reverse",
                                  "prefix16", "nul"])
def test_adversarial(case):
    n = 1000
    if case == "equal":
        strs = [b"same-string-longer-than-nine"] * n
    elif case == "empty":
        strs = [b""] * n
    elif case == "sorted":
        strs = [b"%08d" % i for i in range(n)]
    elif case == "reverse":
        strs = [b"%08d" % (n - i) for i in range(n)]
    elif case == "prefix16":
        strs = [b"P" * 16 + b"%03d" % (i % 97) for i in range(n)]
    else:
        strs = [b"a" + b"\x00" * (i % 5) for i in range(n)]
    w = workloads.from_strings(strs)
    perm = oracle.stable_argsort(w.bytes, w.offsets, threads=3)
    assert np.array_equal(perm.astype(np.int64), _python_sort(w))
    if case in ("equal", "empty", "sorted"):
        assert np.array_equal(perm, np.arange(n))


def test_empty_input():
    w = workloads.from_strings([])
    assert oracle.stable_argsort(w.bytes, w.offsets).shape == (0,)
    assert oracle.check_sorted(w.bytes, w.offsets, np.zeros(0, np.uint32)) == -1


def test_checker_catches_planted_mistakes():
    w = workloads.from_strings([b"b", b"a", b"a", b"c", b"a"])
    good = np.array([1, 2, 4, 0, 3], dtype=np.uint32)
    assert oracle.check_sorted(w.bytes, w.offsets, good) == -1
    swapped = good.copy(); swapped[[2, 3]] = swapped[[3, 2]]      # order
    assert oracle.check_sorted(w.bytes, w.offsets, swapped) >= 0
    unstable = good.copy(); unstable[[0, 1]] = unstable[[1, 0]]  # stability
    assert oracle.check_sorted(w.bytes, w.offsets, unstable) == 1
    dup = good.copy(); dup[2] = 2                                # repeat
    assert oracle.check_sorted(w.bytes, w.offsets, dup) >= 0
    far_dup = np.array([1, 2, 1, 0, 3], dtype=np.uint32)         # non-adjacent repeat
    assert oracle.check_sorted(w.bytes, w.offsets, far_dup) >= 0
    oob = good.copy(); oob[4] = 5                                # range
    assert oracle.check_sorted(w.bytes, w.offsets, oob) == 4
    assert oracle.check_sorted(w.bytes, w.offsets, good[:4]) == 0  # length
    assert oracle.check_sorted(w.bytes, w.offsets, good.astype(np.uint64)) == -1


def test_checker_threads_agree():
    w = workloads.generate(2, 50000, 3)
    perm = oracle.stable_argsort(w.bytes, w.offsets, threads=4)
    for t in (1, 7):
        assert oracle.check_sorted(w.bytes, w.offsets, perm, threads=t) == -1
    bad = perm.copy()
    j = 31337
    while oracle.string_compare(w.bytes, w.offsets, int(bad[j]), int(bad[j + 1])) == 0:
        j += 1
    bad[[j, j + 1]] = bad[[j + 1, j]]
    for t in (1, 7):
        assert oracle.check_sorted(w.bytes, w.offsets, bad, threads=t) == j + 1


def test_batched_oracle_matches_per_instance():
    """The batched oracle equals the single-input oracle run on each instance
    (and Python's sorted), including empty and single-string instances."""
    w = workloads.generate_batched(40, 3, lo=1, hi=3000)
    seg = w.seg_offsets.copy()
    seg[5] = seg[4]   # an empty instance
    got = oracle.stable_argsort_batched(w.bytes, w.offsets, seg, threads=3)
    for s in range(seg.shape[0] - 1):
        lo, hi = int(seg[s]), int(seg[s + 1])
        sub = workloads.from_strings([w.string(i) for i in range(lo, hi)])
        want = np.array(sorted(range(hi - lo), key=sub.string), dtype=np.uint32)
        assert np.array_equal(got[lo:hi], want), s
    assert oracle.check_sorted_batched(w.bytes, w.offsets, seg, got) == -1


def test_batched_checker_catches_planted_mistakes():
    w = workloads.from_strings([b"b", b"a", b"a", b"c", b"z", b"y"])
    seg = np.array([0, 4, 6], dtype=np.uint64)
    good = np.array([1, 2, 0, 3, 1, 0], dtype=np.uint32)
    assert oracle.check_sorted_batched(w.bytes, w.offsets, seg, good) == -1
    unstable = good.copy(); unstable[[0, 1]] = unstable[[1, 0]]
    assert oracle.check_sorted_batched(w.bytes, w.offsets, seg, unstable) == 1
    global_idx = good.copy(); global_idx[4] = 5          # not a local index
    assert oracle.check_sorted_batched(w.bytes, w.offsets, seg, global_idx) == 4
    wrong_order = good.copy(); wrong_order[[4, 5]] = wrong_order[[5, 4]]
    assert oracle.check_sorted_batched(w.bytes, w.offsets, seg, wrong_order) == 5
