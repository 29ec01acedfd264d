"""Pins for the oracle's encoder (Algorithm 4 and Algorithms 2/3).

The encoder is pinned to things other than itself: codes worked by hand
(tests/golden/husky_codes.txt), the order property of Section 3.2 brute-forced
over every short string on small alphabets, the perfectness claim of Section 5
("for ASCII strings, it is nine"), and the exactness reading for NUL bytes.
"""

import itertools

import numpy as np
import pytest

import oracle
import workloads
from conftest import literal, read_golden


def _code(coder, s):
    return oracle.ascii_to_long(s) if coder == "ASCII7" else oracle.byte_to_long(s)


@pytest.mark.parametrize("row", read_golden("husky_codes.txt"),
                         ids=lambda r: f"{r[0]}:{r[1]}")
def test_hand_worked_codes(row):
    coder, text, expected = row[0], literal(row[1]), int(row[2], 16)
    assert _code(coder, text) == expected


def _all_strings(alphabet, max_len, min_len=0):
    out = []
    for L in range(min_len, max_len + 1):
        out.extend(bytes(t) for t in itertools.product(alphabet, repeat=L))
    return out


ALPHABETS_ASCII = [b"abcd", bytes([0x00, 0x01, 0x7E, 0x7F])]
ALPHABETS_BYTE = [b"abcd", bytes([0x00, 0x01, 0x80, 0xFF])]


@pytest.mark.parametrize("coder,alphabet",
                         [("ASCII7", a) for a in ALPHABETS_ASCII] +
                         [("BYTE8", a) for a in ALPHABETS_BYTE])
def test_order_property_pairwise(coder, alphabet):
    """Section 3.2 with p applying only to ties: for every ordered pair,
    code(a) < code(b) implies a < b, and a < b implies code(a) <= code(b);
    a == b implies equal codes.  85 strings, 7,225 pairs per alphabet."""
    strs = _all_strings(alphabet, 3)
    codes = [_code(coder, s) for s in strs]
    for a, ca in zip(strs, codes):
        for b, cb in zip(strs, codes):
            if ca < cb:
                assert a < b, (a, b)
            if a < b:
                assert ca <= cb, (a, b)
            if a == b:
                assert ca == cb


@pytest.mark.parametrize("coder,alphabet,lengths", [
    ("ASCII7", b"ab", (8, 11)),
    ("BYTE8", b"ab", (7, 10)),
    ("ASCII7", bytes([0x00, 0x7F]), (7, 10)),
])
def test_order_property_across_truncation(coder, alphabet, lengths):
    """Strings straddling the 9-char (8-byte) cap: codes are non-decreasing
    along the sorted order, which is equivalent to the pairwise property."""
    strs = sorted(_all_strings(alphabet, lengths[1], lengths[0]))
    codes = np.array([_code(coder, s) for s in strs], dtype=np.uint64)
    assert np.all(codes[1:] >= codes[:-1])


def test_ascii_perfect_up_to_nine():
    """Section 5: nine ASCII chars fit; distinct NUL-free strings of length
    <= 9 never collide (all 1,023 strings over {a, b})."""
    strs = _all_strings(b"ab", 9)
    codes = {oracle.ascii_to_long(s) for s in strs}
    assert len(codes) == len(strs)


def test_byte8_perfect_up_to_eight():
    strs = _all_strings(bytes([0x01, 0xFF]), 8)
    codes = {oracle.byte_to_long(s) for s in strs}
    assert len(codes) == len(strs)


def test_nul_shares_code_and_is_not_exact():
    """'a' and 'a\\0' share a code, so exactness must look at the last byte."""
    w = workloads.from_strings([b"a", b"a\x00", b"", b"abcdefghi",
                                b"abcdefghij", b"\x00"])
    codes, exact, perfect = oracle.encode(w.bytes, w.offsets, oracle.CODER_ASCII7)
    assert codes[0] == codes[1]
    assert list(exact) == [1, 0, 1, 1, 0, 0]
    assert not perfect


def test_perfect_flag_short_strings():
    w = workloads.from_strings([b"abc", b"xyz", b"", b"abcdefghi"])
    _, exact, perfect = oracle.encode(w.bytes, w.offsets, oracle.CODER_ASCII7)
    assert perfect and exact.all()
    _, _, perfect8 = oracle.encode(w.bytes, w.offsets, oracle.CODER_BYTE8)
    assert not perfect8  # 9 chars exceed the 8-byte cap


def test_array_encoder_matches_scalar():
    w = workloads.generate(1, 2000, 11)
    codes, _, _ = oracle.encode(w.bytes, w.offsets, oracle.CODER_ASCII7)
    for i in range(0, 2000, 37):
        assert codes[i] == oracle.ascii_to_long(w.string(i))


# ---- alphabet-rank coder -------------------------------------------------------

@pytest.mark.parametrize("row", read_golden("alpha_codes.txt"))
def test_alpha_hand_worked_codes(row):
    strs = literal(row[0])
    w_, k_ = int(row[1]), int(row[2])
    want = [int(x, 16) for x in row[3].split()]
    wl = workloads.from_strings(strs)
    codes, exact, perfect, w, k = oracle.encode_alpha(wl.bytes, wl.offsets)
    assert (w, k) == (w_, k_)
    got = [int(c) for c in codes][-len(want):]
    assert got == want


@pytest.mark.parametrize("s_count, w_", [(1, 1), (2, 2), (3, 2), (4, 3), (7, 3), (8, 4), (15, 4), (16, 5),
                                        (26, 5), (31, 5), (32, 6), (62, 6), (63, 6)])
def test_alpha_width_and_length_table(s_count, w_):
    """Bit width for byte ranges of s values, worked by hand from
    w = ceil(log2(s + 1)); the length is 8 chars throughout; a range of 64
    needs 7 bits and the coder does not apply.  Only the two ends matter:
    the bytes in between need not occur."""
    wl = workloads.from_strings([bytes([40]), bytes([40 + s_count - 1])])
    m, w, k, applies = oracle.alpha_params(wl.bytes, wl.offsets)
    assert (w, k, applies) == (w_, 8, True)
    assert m[40] == 1 and m[40 + s_count - 1] == s_count and m[39] == 0
    wl = workloads.from_strings([bytes([40]), bytes([40 + 63])])
    assert oracle.alpha_params(wl.bytes, wl.offsets)[3] is False


@pytest.mark.parametrize("alphabet", [b"abcd", b"\x00\x01\x02\x03", b"\x7e\x7f\x80\x81", b"\xfc\xfd\xfe\xff",
                                      b"\x00\x10\x20\x30"])
def test_alpha_order_property_pairwise(alphabet):
    """Section 3.2's rule for the byte-range coder, over every string of
    length 0..3 on a 4-symbol alphabet (NUL, the 0x7F/0x80 boundary and the
    top bytes included, and one with gaps): a < b implies code(a) <= code(b),
    code(a) < code(b) implies a < b, and all these strings (length <= K) get
    distinct codes."""
    strs = [b""] + [bytes(t) for L in (1, 2, 3) for t in itertools.product(alphabet, repeat=L)]
    wl = workloads.from_strings(strs)
    codes, exact, perfect, w, k = oracle.encode_alpha(wl.bytes, wl.offsets)
    assert perfect and all(exact)
    for i, a in enumerate(strs):
        for j, b in enumerate(strs):
            if a < b:
                assert codes[i] < codes[j]
    assert len(set(int(c) for c in codes)) == len(strs)


def test_alpha_truncation_and_nul():
    """Strings agreeing on the first 8 chars share a code and are not exact;
    a NUL byte inside the range has a value of its own, so x and x + NUL
    differ (unlike ASCII7, where they share a code)."""
    strs = [b"abcdefghi", b"abcdefghz", b"abcdefgh", b"a", b"abcdefghijklmnopqrstuvwxyz"]
    wl = workloads.from_strings(strs)
    codes, exact, perfect, w, k = oracle.encode_alpha(wl.bytes, wl.offsets)
    assert (w, k) == (5, 8)
    assert codes[0] == codes[1] == codes[2]
    assert list(exact) == [0, 0, 1, 1, 0] and not perfect
    strs = [b"\x05", b"\x05\x00", b"\x1f\x1f\x1f"]      # range 0x00..0x1f: 32 values, 6 bits
    wl = workloads.from_strings(strs)
    codes, exact, perfect, w, k = oracle.encode_alpha(wl.bytes, wl.offsets)
    assert (w, k) == (6, 8) and perfect
    assert codes[0] < codes[1] < codes[2]
    assert oracle.encode_alpha(*_ws([b"a", b"a\x00"])) is None   # 0x00..0x61 needs 7 bits


# ---- the byte-range coder at the paper's own length (Section 3.2) ------------

@pytest.mark.parametrize("alphabet, w_, k_", [(b"abcdefghijklmnopqrstuvwxyz", 5, 12),
                                             (b"ABCDEFGHIJKLMNOPQRSTUVWXYZ[\\]^_`abcdefghijklmnopqrstuvwxyz", 6, 10)])
def test_alpha_paper_length_is_perfect_for_letters(alphabet, w_, k_):
    """Section 3.2: case-independent letters code in 5 bits and case-dependent
    ones in 6, so 12 and 10 of them fit 64 bits.  At that length every string
    of up to K letters is coded exactly: distinct strings get distinct codes,
    in the strings' order.  Checked on 3,000 random strings of length 0..K
    (all pairs), every string of length <= 2, and strings that differ only in
    their K-th letter; a (K+1)-th letter is truncated away."""
    rng = np.random.default_rng(len(alphabet))
    al = list(alphabet)
    strs = {b"", bytes([al[0]]), bytes([al[-1]])}
    strs |= {bytes([a, b]) for a in al[:6] + al[-3:] for b in al[:4] + al[-2:]}
    for _ in range(3000):
        L = int(rng.integers(0, k_ + 1))
        strs.add(bytes(al[int(x)] for x in rng.integers(0, len(al), size=L)))
    stem = bytes(al[int(x)] for x in rng.integers(0, len(al), size=k_ - 1))
    strs |= {stem + bytes([c]) for c in (al[0], al[1], al[-1])}
    strs = sorted(strs)
    wl = workloads.from_strings(strs)
    codes, exact, perfect, w, k = oracle.encode_alpha(wl.bytes, wl.offsets, max_length=None)
    assert (w, k) == (w_, k_)
    assert perfect and all(exact)
    c = [int(x) for x in codes]
    assert all(a < b for a, b in zip(c, c[1:]))      # sorted strings, strictly increasing codes
    assert max(c) < (1 << (k_ * w_))
    long_ = workloads.from_strings([stem + bytes([al[3]]) + bytes([al[5]]), stem + bytes([al[3]])])
    lc, le, lp, _, _ = oracle.encode_alpha(long_.bytes, long_.offsets, max_length=None)
    assert lc[0] == lc[1] and list(le) == [0, 1] and not lp


def test_alpha_length_parameter():
    """K is a parameter: the same letters at K = 8 (the GPU library's length)
    and at the paper's K = 12 give codes that agree on the first 8 letters:
    the K = 12 code shifted right by 4 letters (20 bits) is the K = 8 code for
    strings of up to 8 letters; K * w above 64 bits does not apply."""
    strs = [b"", b"a", b"abc", b"zzzzzzzz", b"hello", b"abcdefgh"]
    wl = workloads.from_strings(strs + [b"z"])
    c8, _, _, w8, k8 = oracle.encode_alpha(wl.bytes, wl.offsets)
    c12, _, _, w12, k12 = oracle.encode_alpha(wl.bytes, wl.offsets, max_length=None)
    assert (w8, k8, w12, k12) == (5, 8, 5, 12)
    for a, b in zip(c8, c12):
        assert int(b) >> 20 == int(a)
    assert oracle.encode_alpha(wl.bytes, wl.offsets, max_length=13) is None   # 65 bits


def _ws(strs):
    wl = workloads.from_strings(strs)
    return wl.bytes, wl.offsets


# ---- the Unicode coder (Section 4.3 unicodeToLong) -------------------------

def test_unicode_hand_worked_codes():
    """Worked by hand: units packed 16 bits each, most significant first,
    zero-padded to four, then shifted right by one."""
    assert oracle.unicode_to_long([]) == 0
    assert oracle.unicode_to_long([0x0041, 0x4E2D]) == 0x0020A71680000000
    assert oracle.unicode_to_long([0xFFFF] * 4) == 0x7FFFFFFFFFFFFFFF
    assert oracle.unicode_to_long([1, 2, 3, 4, 5]) == 0x0000800100018002  # 0x0001000200030004 >>> 1


UNITS = [0x0000, 0x0041, 0x00E9, 0x7FFF, 0x8000, 0xD800, 0xFFFF]


def test_unicode_order_property_pairwise():
    """a < b in code-unit order implies code(a) <= code(b), and code(a) <
    code(b) implies a < b, over every string of 0..3 units from a set with
    surrogate and high units; the >>> 1 only merges neighbours."""
    strs = [list(t) for L in range(4) for t in itertools.product(UNITS, repeat=L)]
    codes = [oracle.unicode_to_long(s) for s in strs]
    for (a, ca), (b, cb) in itertools.product(zip(strs, codes), repeat=2):
        if a < b:
            assert ca <= cb
        if ca < cb:
            assert a < b


def test_unicode_shift_merges_only_the_last_bit():
    """The shift loses the low bit of the fourth unit and nothing else."""
    assert oracle.unicode_to_long([7, 7, 7, 0x100]) == oracle.unicode_to_long([7, 7, 7, 0x101])
    assert oracle.unicode_to_long([7, 7, 7, 0x100]) < oracle.unicode_to_long([7, 7, 7, 0x102])
    assert oracle.unicode_to_long([7, 7, 6, 0xFFFF]) < oracle.unicode_to_long([7, 7, 7, 0])


def test_unicode_coder_is_the_byte_coder_on_big_endian_bytes():
    """On the UTF-16BE bytes of a string the byte coder (8 bits x 8) packs the
    same four units; the Unicode code is that code shifted right by one."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        u = [int(x) for x in rng.integers(0, 65536, size=int(rng.integers(0, 7)))]
        be = b"".join(x.to_bytes(2, "big") for x in u)
        assert oracle.byte_to_long(be) >> 1 == oracle.unicode_to_long(u)
        assert oracle.byte_to_long(be) == oracle.units_to_long(u, 4, 16, 0xFFFF)
