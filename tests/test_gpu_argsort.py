"""GPU parity: the CUDA path through the C ABI against the oracle.

Integer work, so the bar is bit-exact: codes equal the oracle's Algorithm 4
codes, permutations equal the oracle's stable argsort element by element (or,
at sizes the oracle cannot re-sort quickly, satisfy the property check that
characterises the stable argsort uniquely)."""

import numpy as np
import pytest

import oracle
import workloads
from conftest import literal, read_golden
from gpu_util import assert_oracle_equal, assert_stable_sorted, perm_numpy, to_device

pytestmark = pytest.mark.gpu


# ---- Step 1 ------------------------------------------------------------------

@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("coder", [1, 2])
def test_encode_matches_oracle(cuda_lib, kind, coder):
    hs = cuda_lib
    w = workloads.generate(kind, 300_001, 11 + kind)
    data, off = to_device(w)
    codes, exact, used = hs.encode(data, off, coder=coder)
    want, want_exact, perfect = oracle.encode(w.bytes, w.offsets, coder)
    assert used == coder
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), want)
    assert exact == perfect


def test_encode_edge_strings(cuda_lib):
    hs = cuda_lib
    strs = [b"", b"a", b"a\x00", b"\x00", b"abcdefghi", b"abcdefghij", b"\x7f" * 9,
            b"z" * 40, b"ab"]
    w = workloads.from_strings(strs)
    data, off = to_device(w)
    for coder in (1, 2):
        codes, exact, _ = hs.encode(data, off, coder=coder)
        want, _, perfect = oracle.encode(w.bytes, w.offsets, coder)
        assert np.array_equal(codes.cpu().numpy().view(np.uint64), want)
        assert exact == perfect


@pytest.mark.parametrize("coder", [1, 2])
def test_encode_staged_and_unstaged_tiles(cuda_lib, coder):
    """Tiles of 1024 strings whose bytes fit the shared stage build each code
    from two aligned shared words; tiles of long strings read each string
    from global memory.  Alternate the two kinds tile by tile, with lengths
    0..12 around the 8- and 9-char limits, NUL bytes, high bytes (BYTE8) and
    a ragged last tile; codes, the all-exact flag and the argsort must equal
    the oracle's."""
    hs = cuda_lib
    rng = np.random.default_rng(5 + coder)
    top = 256 if coder == 2 else 128
    strs = []
    for t in range(12):
        for _ in range(1024):
            n_bytes = int(rng.integers(20, 70)) if t % 3 == 1 else int(rng.integers(0, 13))
            b = rng.integers(0, top, size=n_bytes).astype(np.uint8)
            if rng.random() < 0.3:
                b = (97 + b % 26).astype(np.uint8)
            strs.append(bytes(b))
    strs += [b"x" * 9, b"y" * 8 + b"\x00", b""]
    w = workloads.from_strings(strs)
    data, off = to_device(w)
    codes, exact, used = hs.encode(data, off, coder=coder)
    want, _, perfect = oracle.encode(w.bytes, w.offsets, coder)
    assert used == coder
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), want)
    assert exact == perfect
    assert_oracle_equal(w, hs.argsort_device(data, off, coder=coder))


def test_encode_golden(cuda_lib):
    hs = cuda_lib
    rows = read_golden("husky_codes.txt")
    for coder_name, coder in (("ASCII7", 1), ("BYTE8", 2)):
        sel = [r for r in rows if r[0] == coder_name and (coder == 2 or
               all(b < 0x80 for b in literal(r[1])))]
        w = workloads.from_strings([literal(r[1]) for r in sel])
        data, off = to_device(w)
        codes, _, _ = hs.encode(data, off, coder=coder)
        got = codes.cpu().numpy().view(np.uint64)
        assert [int(x) for x in got] == [int(r[2], 16) for r in sel]


def test_ascii7_domain_error_and_auto(cuda_lib):
    """ASCII7 rejects high bytes; AUTO takes the byte-range coder when the
    strings span few byte values (high bytes or not) and falls back to BYTE8
    when a high byte comes with a wide range."""
    hs = cuda_lib
    w = workloads.from_strings([b"abc", b"\xc3\xa9t\xc3\xa9", b"ab\x80", b"zz"])   # 0x61..0xc3: 7 bits
    data, off = to_device(w)
    with pytest.raises(hs.HuskyError) as e:
        hs.encode(data, off, coder=hs.CODER_ASCII7)
    assert e.value.status == hs.ERR_CODER_DOMAIN
    codes, _, used = hs.encode(data, off, coder=hs.CODER_AUTO)
    assert used == hs.CODER_BYTE8
    want, _, _ = oracle.encode(w.bytes, w.offsets, oracle.CODER_BYTE8)
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), want)
    assert_oracle_equal(w, hs.argsort_device(data, off))
    # high bytes in a narrow range 0x80..0x9e (31 values, 5 bits): the range coder
    rng = np.random.default_rng(3)
    strs = [b"\x80", b"\x9e"] + [bytes(rng.integers(0x80, 0x9f, size=rng.integers(0, 14)).astype(np.uint8))
                                for _ in range(5000)]
    w = workloads.from_strings(strs)
    data, off = to_device(w)
    codes, _, used = hs.encode(data, off, coder=hs.CODER_AUTO)
    assert used == hs.CODER_ALPHA
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), oracle.encode_alpha(w.bytes, w.offsets)[0])
    assert_oracle_equal(w, hs.argsort_device(data, off))
    # 200 byte values: the range needs 8 bits
    strs = [bytes([b]) * 3 for b in range(56, 256)] + \
           [bytes(rng.integers(56, 256, size=rng.integers(0, 14)).astype(np.uint8)) for _ in range(5000)]
    w = workloads.from_strings(strs)
    data, off = to_device(w)
    with pytest.raises(hs.HuskyError) as e:
        hs.encode(data, off, coder=hs.CODER_ALPHA)
    assert e.value.status == hs.ERR_CODER_DOMAIN
    codes, _, used = hs.encode(data, off, coder=hs.CODER_AUTO)
    assert used == hs.CODER_BYTE8
    want, _, _ = oracle.encode(w.bytes, w.offsets, oracle.CODER_BYTE8)
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), want)
    assert_oracle_equal(w, hs.argsort_device(data, off))


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5])
def test_alpha_encode_matches_oracle(cuda_lib, kind):
    """The byte-range coder against the oracle's: same codes and all-exact
    flag on the lowercase workloads (w = 5, K = 8); kind 3 spans '0'..'z'
    (75 values) and is refused."""
    hs = cuda_lib
    w = workloads.generate(kind, 300_001, 31 + kind)
    data, off = to_device(w)
    if kind == 3:
        with pytest.raises(hs.HuskyError) as e:
            hs.encode(data, off, coder=hs.CODER_ALPHA)
        assert e.value.status == hs.ERR_CODER_DOMAIN
        assert oracle.encode_alpha(w.bytes, w.offsets) is None
        return
    codes, exact, used = hs.encode(data, off, coder=hs.CODER_ALPHA)
    want, _, perfect, ww, kk = oracle.encode_alpha(w.bytes, w.offsets)
    assert used == hs.CODER_ALPHA and (ww, kk) == (5, 8)
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), want)
    assert exact == perfect


def test_alpha_edge_alphabets(cuda_lib):
    """Narrow byte ranges (w = 1, 2, 4, 6), NUL bytes, empty strings, and the
    argsort through them."""
    hs = cuda_lib
    cases = [[b"a" * k for k in range(0, 40)],
             [b"ab"[i % 2: i % 2 + 1] * (i % 23) for i in range(3000)],
             [bytes([48 + (i * 7) % 10]) * (1 + i % 19) + b"\x00" * (i % 3) for i in range(5000)],
             [b"", b"\x00", b"\x00\x00", b"\x00\x01", b"\x01"] * 100]
    for strs in cases:
        w = workloads.from_strings(strs)
        data, off = to_device(w)
        codes, exact, used = hs.encode(data, off, coder=hs.CODER_ALPHA)
        want, _, perfect, _, _ = oracle.encode_alpha(w.bytes, w.offsets)
        assert np.array_equal(codes.cpu().numpy().view(np.uint64), want)
        assert exact == perfect
        assert_oracle_equal(w, hs.argsort_device(data, off))


def test_decreasing_offsets_rejected(cuda_lib):
    hs = cuda_lib
    import torch
    data = torch.zeros(64, dtype=torch.uint8, device="cuda")
    off = torch.tensor([0, 5, 3, 9], dtype=torch.int64, device="cuda")
    with pytest.raises(hs.HuskyError) as e:
        hs.argsort_device(data, off)
    assert e.value.status == hs.ERR_INVALID_ARG


def test_workspace_too_small(cuda_lib):
    hs = cuda_lib
    import ctypes
    import torch
    w = workloads.generate(1, 1000, 0)
    data, off = to_device(w)
    perm = torch.empty(1000, dtype=torch.int32, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st = hs.load().hs_argsort(data.data_ptr(), off.data_ptr(), 1000, 0, 0, 0,
                              perm.data_ptr(), ws.data_ptr(), 1024,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == hs.ERR_WORKSPACE


# ---- Steps 1-3 ----------------------------------------------------------------

def test_worked_example(cuda_lib):
    hs = cuda_lib
    rows = dict((r[0], r[1]) for r in read_golden("tiny_sort.txt"))
    w = workloads.from_strings(literal(rows["strings"]))
    data, off = to_device(w)
    perm = hs.argsort_device(data, off)
    assert list(perm_numpy(perm)) == literal(rows["perm"])


@pytest.mark.parametrize("n", [1, 2, 3, 31, 4095, 4096, 4097, 8193, 100_003])
@pytest.mark.parametrize("kind", [1, 2, 5])
def test_sizes_and_ragged_tails(cuda_lib, kind, n):
    hs = cuda_lib
    w = workloads.generate(kind, n, 100 + n)
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("index_u64", [False, True])
def test_workloads_scaled(cuda_lib, kind, index_u64):
    hs = cuda_lib
    w = workloads.generate(kind, 1_000_003, 7 * kind)
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off, index_u64=index_u64))


@pytest.mark.parametrize("run", [2, 31, 32, 33, 2047, 2048, 2049, 5000, 70_000])
@pytest.mark.parametrize("shape", ["identical", "suffix", "deep"])
def test_run_size_classes(cuda_lib, run, shape):
    """Runs of equal husky codes at every size-class boundary: identical long
    strings, distinct suffixes after a shared 9-char prefix, and ties that
    need several 7-byte refinement windows."""
    hs = cuda_lib
    rng = np.random.default_rng(run)
    strs = []
    for i in range(run):
        if shape == "identical":
            s = b"abcdefghijklmnop"
        elif shape == "suffix":
            s = b"abcdefghi" + bytes(rng.integers(97, 100, size=rng.integers(0, 6)).astype(np.uint8))
        else:
            s = b"x" * 30 + bytes(rng.integers(97, 99, size=rng.integers(0, 12)).astype(np.uint8))
        strs.append(s)
    strs += [b"short", b"abcdefgh", b"abcdefghi", b"zzzz"] * 3
    order = rng.permutation(len(strs))
    w = workloads.from_strings([strs[i] for i in order])
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


@pytest.mark.parametrize("case", ["equal_long", "equal_short", "empty", "sorted",
                                  "reverse", "nul", "binary", "long_strings"])
def test_adversarial(cuda_lib, case):
    hs = cuda_lib
    n = 20_000
    rng = np.random.default_rng(3)
    if case == "equal_long":
        strs = [b"the-same-string-longer-than-nine"] * n
    elif case == "equal_short":
        strs = [b"same"] * n
    elif case == "empty":
        strs = [b""] * n
    elif case == "sorted":
        strs = [b"%012d" % i for i in range(n)]
    elif case == "reverse":
        strs = [b"%012d" % (n - i) for i in range(n)]
    elif case == "nul":
        strs = [b"a" + b"\x00" * (i % 13) + (b"b" if i % 3 == 0 else b"") for i in range(n)]
    elif case == "binary":
        strs = [bytes(rng.integers(0, 256, size=rng.integers(0, 20)).astype(np.uint8)) for _ in range(n)]
    else:
        strs = [b"q" * int(rng.integers(0, 3000)) + bytes([97 + i % 3]) for i in range(2000)]
    w = workloads.from_strings(strs)
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


def test_empty_input(cuda_lib):
    hs = cuda_lib
    w = workloads.from_strings([])
    data, off = to_device(w)
    assert hs.argsort_device(data, off).numel() == 0


def test_host_inputs_roundtrip(cuda_lib):
    hs = cuda_lib
    import torch
    w = workloads.generate(2, 200_000, 5)
    data = torch.from_numpy(w.bytes).pin_memory()
    off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
    perm = hs.argsort(data, off)
    assert not perm.is_cuda
    assert_oracle_equal(w, perm)


@pytest.mark.parametrize("index_u64", [False, True])
def test_host_inputs_into_a_reused_pinned_output(cuda_lib, index_u64):
    """The host entry point writes into a caller's pinned tensor, call after
    call; a tensor of the wrong type or size, or not pinned, is refused."""
    hs = cuda_lib
    import torch
    dt = torch.int64 if index_u64 else torch.int32
    out = None
    for seed in (5, 6):
        w = workloads.generate(2, 100_000, seed)
        data = torch.from_numpy(w.bytes).pin_memory()
        off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
        if out is None:
            out = torch.full((w.n,), -1, dtype=dt).pin_memory()
        got = hs.argsort(data, off, index_u64=index_u64, out=out)
        assert got.data_ptr() == out.data_ptr()
        assert_oracle_equal(w, out)
    for bad in (torch.empty(w.n, dtype=dt), torch.empty(w.n + 1, dtype=dt).pin_memory(),
                torch.empty(w.n, dtype=torch.int32 if index_u64 else torch.int64).pin_memory()):
        with pytest.raises(ValueError):
            hs.argsort(data, off, index_u64=index_u64, out=bad)


@pytest.mark.parametrize("n_copies", [40, 3000, 70_001])
@pytest.mark.parametrize("odd", ["none", "smaller", "greater", "longer", "shorter"])
def test_runs_of_copies_with_one_odd_member(cuda_lib, n_copies, odd):
    """Runs of copies of one long string are final after the code sort (the
    copies stay in index order); a single member that differs after byte 9,
    placed away from every sampled position, must still be found and
    sorted.  Sizes cover the warp (<= 32), CTA (<= 2048) and large classes."""
    hs = cuda_lib
    base = b"abcdefghijklmnopqrstu"
    strs = [base] * n_copies
    j = (n_copies * 7) // 13 + 1
    if odd == "smaller":
        strs[j] = base[:15] + b"a" + base[16:]
    elif odd == "greater":
        strs[j] = base[:15] + b"z" + base[16:]
    elif odd == "longer":
        strs[j] = base + b"!"
    elif odd == "shorter":
        strs[j] = base[:-1]
    rng = np.random.default_rng(n_copies)
    strs += [bytes(rng.integers(97, 123, size=12).astype(np.uint8)) for _ in range(500)]
    order = rng.permutation(len(strs))
    w = workloads.from_strings([strs[i] for i in order])
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


@pytest.mark.parametrize("n_copies", [40, 3000, 70_001])
@pytest.mark.parametrize("case", ["none", "tail_byte", "len15_last", "len16_last", "shorter", "exact8"])
def test_runs_of_copies_of_short_long_strings(cuda_lib, n_copies, case):
    """Packed words, runs of copies of 12-16 byte strings (the code covers
    8): the fix-up's filters must find one odd member that differs at byte
    11, at the last byte of a 15- or 16-byte string, by its length, or is
    the 8-byte prefix itself (exactly coded, same code).  Sizes cover the
    CTA-sized (copies filter) and large classes."""
    hs = cuda_lib
    base = {"len15_last": b"abcdefghijklmno", "len16_last": b"abcdefghijklmnop"}.get(case, b"abcdefghijkl")
    strs = [base] * n_copies
    j = (n_copies * 5) // 11 + 1
    if case == "tail_byte":
        strs[j] = base[:11] + b"a" + base[12:]
    elif case == "len15_last":
        strs[j] = base[:14] + b"a"
    elif case == "len16_last":
        strs[j] = base[:15] + b"a"
    elif case == "shorter":
        strs[j] = base[:-1]
    elif case == "exact8":
        strs[j] = base[:8]
    rng = np.random.default_rng(n_copies)
    strs += [bytes(rng.integers(97, 123, size=int(rng.integers(3, 14))).astype(np.uint8)) for _ in range(500)]
    order = rng.permutation(len(strs))
    w = workloads.from_strings([strs[i] for i in order])
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


@pytest.mark.parametrize("case", ["pinned_u32", "pageable_u64", "learned", "byte8", "offset0"])
def test_host_entry_point_chunks(cuda_lib, case):
    """hs_argsort_host: inputs and output in host memory, copied in chunks of
    whole tiles (1e6 strings = four chunks) with each chunk encoded as it
    arrives; the permutation must equal the oracle's in every mode."""
    hs = cuda_lib
    import torch
    kind = 5 if case in ("learned", "pageable_u64") else 2
    w = workloads.generate(kind, 1_000_003, 70 + len(case))
    if case == "byte8":   # a high byte late in the input: ASCII7 finds it, AUTO re-encodes
        b = w.bytes.copy()
        b[int(w.offsets[900_000])] = 0xE9
        w = workloads.Workload(b, w.offsets)
    if case == "offset0":  # string 0 starts past the buffer's first byte
        b = np.concatenate([np.full(37, 0x41, np.uint8), w.bytes])
        w = workloads.Workload(b, w.offsets + np.uint64(37))
    data = torch.from_numpy(w.bytes)
    off = torch.from_numpy(w.offsets.view(np.int64))
    if case != "pageable_u64":
        data, off = data.pin_memory(), off.pin_memory()
    mode = hs.MODE_LEARNED if case == "learned" else hs.MODE_PLAIN
    perm = hs.argsort(data, off, mode=mode, index_u64=case in ("pageable_u64", "learned"))
    assert not perm.is_cuda
    assert_oracle_equal(w, perm)


def _letters(n, lo, hi, seed, maxlen=12):
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, maxlen + 1, size=n).astype(np.uint64)
    offsets = np.zeros(n + 1, np.uint64)
    np.cumsum(lens, out=offsets[1:])
    return workloads.Workload(rng.integers(lo, hi + 1, size=int(offsets[-1])).astype(np.uint8), offsets)


def test_host_entry_point_range_widened_by_a_later_chunk(cuda_lib):
    """Host inputs under the byte-range coder: the chunks are encoded with
    the first chunk's range.  Letters 'c'..'x' with one 'a' in the last
    chunk keep the width (5 bits) but shift every code, so that sort is
    encoded once more with the whole range; with the 'a' in the first
    chunk it is not."""
    hs = cuda_lib
    import torch
    encodes = {}
    for where in ("none", "first", "last"):
        w = _letters(3_000_000, 99, 120, 51)
        if where != "none":
            w.bytes[int(w.offsets[5 if where == "first" else w.n - 7])] = 97
        data = torch.from_numpy(w.bytes).pin_memory()
        off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
        hs.stats_enable(True)
        try:
            perm = hs.argsort(data, off)
            encodes[where] = hs.stats_read()["encode"]["launches"]
        finally:
            hs.stats_enable(False)
        assert_oracle_equal(w, perm)
    assert encodes["first"] == encodes["none"] and encodes["last"] == encodes["none"] + 1, encodes


def test_host_entry_point_rejects_bad_input(cuda_lib):
    hs = cuda_lib
    import ctypes
    import torch
    lib = hs.load()
    n = 600_000      # three chunks of 262,144
    w = workloads.generate(1, n, 3)
    off = w.offsets.copy()
    off[262_144] = off[262_144 * 2] + 1     # a chunk boundary moves backwards
    data = torch.from_numpy(w.bytes).pin_memory()
    bad = torch.from_numpy(off.view(np.int64)).pin_memory()
    perm = torch.empty(n, dtype=torch.int32).pin_memory()
    nbytes = hs.host_workspace_size(n, int(off[-1]))
    ws = hs.workspace(nbytes, "cuda")
    st = lib.hs_argsort_host(data.data_ptr(), bad.data_ptr(), n, 0, 0, 0, perm.data_ptr(),
                             ws.data_ptr(), nbytes, None)
    assert st == hs.ERR_INVALID_ARG
    d_off = torch.from_numpy(w.offsets.view(np.int64)).cuda()
    st = lib.hs_argsort_host(data.data_ptr(), d_off.data_ptr(), n, 0, 0, 0, perm.data_ptr(),
                             ws.data_ptr(), nbytes, None)
    assert st == hs.ERR_INVALID_ARG and b"host" in lib.hs_last_error()
    st = lib.hs_argsort_host(data.data_ptr(), bad.data_ptr(), n, 0, 0, 0, perm.data_ptr(),
                             ws.data_ptr(), 1024, None)
    assert st in (hs.ERR_INVALID_ARG, hs.ERR_WORKSPACE)


def test_repeated_calls_reuse_workspace(cuda_lib):
    hs = cuda_lib
    for seed in range(3):
        w = workloads.generate(5, 50_000 + seed, seed)
        data, off = to_device(w)
        assert_oracle_equal(w, hs.argsort_device(data, off))


# ---- full-size workloads (the bench's launch configuration) -------------------

@pytest.mark.slow
def test_full_zipf_words_1e7(cuda_lib):
    hs = cuda_lib
    w = workloads.standard("zipf_words_1e7")
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


@pytest.mark.slow
def test_full_shared_prefix_1e8(cuda_lib):
    hs = cuda_lib
    w = workloads.standard("shared_prefix_1e8")
    data, off = to_device(w)
    perm = hs.argsort_device(data, off)
    del data, off
    assert_stable_sorted(w, perm)


@pytest.mark.slow
def test_full_skewed_1e9(cuda_lib):
    """1e9 skewed words (10 GB of bytes) with the u64 permutation, as the
    bench runs them; checked by the property check (a permutation, in
    order, equal strings by index), which fixes the stable argsort."""
    hs = cuda_lib
    w = workloads.standard("skewed_1e9")
    data, off = to_device(w)
    perm = hs.argsort_device(data, off, index_u64=True)
    del data, off
    assert perm.dtype.itemsize == 8
    assert_stable_sorted(w, perm)


@pytest.mark.slow
def test_random_lower_1e5(cuda_lib):
    hs = cuda_lib
    w = workloads.standard("random_lower_1e5")
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off))


def test_shutdown_then_sort_again(cuda_lib):
    """hs_shutdown after host-path calls and timed calls releases the cached
    streams and events; the next calls recreate them and stay exact."""
    hs = cuda_lib
    import torch
    w = workloads.generate(2, 300_000, 9)
    data = torch.from_numpy(w.bytes).pin_memory()
    off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
    hs.stats_enable(True)
    assert_oracle_equal(w, hs.argsort(data, off))
    hs.stats_enable(False)
    hs.shutdown()
    hs.shutdown()
    assert_oracle_equal(w, hs.argsort(data, off))
    d_data, d_off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(d_data, d_off))


# ---- packed (code, index) words ---------------------------------------------

def _onesweep_bytes_per_key(hs, w, **kw):
    """Sorts w and returns the onesweep passes' algorithmic bytes per key and
    launch: 16 or less when the codes and indices travel as one word (the
    fix-up's refinement sorts count there too: keep large mixed runs out)."""
    data, off = to_device(w)
    hs.stats_enable(True)
    try:
        perm = hs.argsort_device(data, off, **kw)
        st = hs.stats_read().get("onesweep")
    finally:
        hs.stats_enable(False)
    assert_oracle_equal(w, perm)
    n = w.offsets.size - 1
    return None if st is None else st["algo_bytes"] / (st["launches"] * n)


@pytest.mark.parametrize("n", [5_000, 300_000])
def test_packed_runs_mixing_exact_and_longer(cuda_lib, n):
    """With the index packed below the code the not-exact bit is not in the
    key, so one run of equal codes can hold 8-char strings and the longer
    strings they begin; the 8-char ones must come first, each group in index
    order.  Shorter strings (the code's last char is padding) and copies of
    long strings are mixed in."""
    hs = cuda_lib
    rng = np.random.default_rng(n)
    # runs of a few hundred: CTA-sized, so no refinement sort adds to the figure
    stems = [bytes(rng.integers(97, 123, size=8).astype(np.uint8)) for _ in range(max(40, n // 750))]
    strs = []
    for _ in range(n):
        s = stems[int(rng.integers(0, len(stems)))]
        r = int(rng.integers(0, 4))
        if r == 1:
            s = s + bytes(rng.integers(97, 100, size=int(rng.integers(1, 4))).astype(np.uint8))
        elif r == 2:
            s = s[: int(rng.integers(0, 8))]
        strs.append(s)
    w = workloads.from_strings(strs)
    assert _onesweep_bytes_per_key(hs, w) <= 16.0


@pytest.mark.parametrize("n,packed", [(65_536, True), (65_537, False)])
@pytest.mark.parametrize("index_u64", [False, True])
def test_packed_index_width_boundary(cuda_lib, n, packed, index_u64):
    """Asked for, a 58-value byte range codes at w = 6 (48-bit codes): 2^16 strings
    still pack their 16-bit index below the code, one more does not and
    sorts (key, index) pairs with the not-exact bit in the key."""
    hs = cuda_lib
    rng = np.random.default_rng(n)
    lens = rng.integers(0, 14, size=n)
    strs = [bytes(rng.integers(65, 123, size=int(m)).astype(np.uint8)) for m in lens]
    strs[0] = b"A" * 3
    strs[1] = b"z" * 12 + b"A"
    w = workloads.from_strings(strs)
    per_key = _onesweep_bytes_per_key(hs, w, index_u64=index_u64, coder=hs.CODER_ALPHA)
    assert (per_key <= 16.0) == packed


@pytest.mark.parametrize("case", ["perfect", "perfect_u64", "same_long", "same_short", "two"])
def test_packed_degenerate(cuda_lib, case):
    """Packed words when every string is exact (the last pass writes the
    permutation), when all codes are equal (no pass runs), and at n = 2."""
    hs = cuda_lib
    rng = np.random.default_rng(11)
    if case.startswith("perfect"):
        strs = [bytes(rng.integers(97, 123, size=int(rng.integers(0, 9))).astype(np.uint8)) for _ in range(50_000)]
    elif case == "same_long":
        strs = [b"abcdefghijk"] * 9_000 + [b"abcdefghij"] * 5
    elif case == "same_short":
        strs = [b"abcd"] * 9_000
    else:
        strs = [b"bbbbbbbbb", b"bbbbbbbb"]
    order = rng.permutation(len(strs))
    w = workloads.from_strings([strs[i] for i in order])
    data, off = to_device(w)
    assert_oracle_equal(w, hs.argsort_device(data, off, index_u64=case == "perfect_u64"))


# ---- UTF-16 strings (the paper's Unicode coder) ------------------------------

def _utf16_units(rng, n):
    """Code units from ASCII, Latin-1, CJK, surrogate and private-use ranges,
    0..10 units long, with repeated strings and shared prefixes."""
    ranges = [(0x20, 0x7F), (0xC0, 0x100), (0x4E00, 0xA000), (0xD800, 0xE000), (0xE000, 0x10000)]
    out = []
    for _ in range(n):
        r = int(rng.integers(0, 10))
        if r == 0 and out:
            out.append(list(out[int(rng.integers(0, len(out)))]))
            continue
        u = []
        for _k in range(int(rng.integers(0, 11))):
            lo, hi = ranges[int(rng.integers(0, len(ranges)))]
            u.append(int(rng.integers(lo, hi)))
        if r == 1 and out:
            u = out[int(rng.integers(0, len(out)))][:4] + u
        out.append(u)
    return out


@pytest.mark.parametrize("n", [3_000, 200_000])
def test_utf16_big_endian_code_unit_order(cuda_lib, n):
    """UTF-16 strings passed as big-endian bytes: the byte coder's code is the
    paper's Unicode code (4 x 16-bit units) before its >>> 1, which unsigned
    keys do not need, and the permutation is the stable sort in code-unit
    order (a Java String's order), checked against Python's sort of the unit
    tuples as well as the oracle."""
    hs = cuda_lib
    rng = np.random.default_rng(n)
    units = _utf16_units(rng, n)
    w = workloads.from_strings([b"".join(x.to_bytes(2, "big") for x in u) for u in units])
    data, off = to_device(w)
    codes, _, coder = hs.encode(data, off, coder=hs.CODER_BYTE8)
    assert coder == hs.CODER_BYTE8
    got = codes.cpu().numpy().view(np.uint64)
    for i in range(0, n, max(1, n // 3000)):
        assert int(got[i]) >> 1 == oracle.unicode_to_long(units[i])
    p = hs.argsort_device(data, off)
    assert list(perm_numpy(p)) == sorted(range(n), key=lambda i: units[i])
    assert_oracle_equal(w, p)


# ---- already-sorted inputs ----------------------------------------------------

def _strings(w):
    return [w.bytes[int(w.offsets[i]):int(w.offsets[i + 1])].tobytes() for i in range(w.offsets.size - 1)]


def _sorted_strings(kind, n, seed):
    w0 = workloads.generate(kind, n, seed)
    s = _strings(w0)
    return [s[i] for i in oracle.stable_argsort(w0.bytes, w0.offsets)]


def _launches(st, kind):
    return st.get(kind, {}).get("launches", 0)


def _sort_with_stats(hs, fn):
    hs.stats_enable(True)
    try:
        perm = fn()
        st = hs.stats_read()
    finally:
        hs.stats_enable(False)
    return perm, st


@pytest.mark.parametrize("kind", [1, 2, 3, 5])
@pytest.mark.parametrize("index_u64", [False, True])
def test_sorted_input_short_circuits(cuda_lib, kind, index_u64):
    """An input already in order (its ties in index order) is recognised
    during the encode: no radix pass runs and the permutation is the
    identity.  Sorted shared-prefix strings have equal codes throughout and
    go through the pair comparison."""
    hs = cuda_lib
    w = workloads.from_strings(_sorted_strings(kind, 200_003, 40 + kind))
    data, off = to_device(w)
    perm, st = _sort_with_stats(hs, lambda: hs.argsort_device(data, off, index_u64=index_u64))
    assert _launches(st, "onesweep") == 0 and _launches(st, "identity") == 1
    assert np.array_equal(perm_numpy(perm), np.arange(w.offsets.size - 1, dtype=perm_numpy(perm).dtype))
    assert_oracle_equal(w, perm)


@pytest.mark.parametrize("where", ["inside", "tile_boundary", "second_tile_boundary", "last", "equal_code"])
def test_one_inversion_in_sorted_input(cuda_lib, where):
    """A sorted input with one adjacent pair swapped is sorted in full, wherever
    the pair falls: inside an encoder tile, across a tile boundary, at the
    end, or as two strings with equal codes that only the full comparison
    tells apart."""
    hs = cuda_lib
    strs = _sorted_strings(2, 300_000, 77)
    if where == "equal_code":
        strs = sorted(set(strs) | {b"abcdefghij", b"abcdefghik", b"abcdefgh"})
        i = strs.index(b"abcdefghij")
    else:
        i = {"inside": 5_000, "tile_boundary": 1_023, "second_tile_boundary": 2_047,
             "last": len(strs) - 2}[where]
        while strs[i] == strs[i + 1]:
            i -= 1
    strs[i], strs[i + 1] = strs[i + 1], strs[i]
    w = workloads.from_strings(strs)
    data, off = to_device(w)
    perm, st = _sort_with_stats(hs, lambda: hs.argsort_device(data, off))
    assert _launches(st, "onesweep") > 0
    assert_oracle_equal(w, perm)


@pytest.mark.parametrize("swap", [None, 262_143, 600_000])
def test_sorted_input_through_host_entry_point(cuda_lib, swap):
    """Host inputs arrive in chunks of 262,144 strings, each encoded as it
    lands; the test of a chunk's first string against the previous chunk's
    last must see an inversion placed exactly there."""
    hs = cuda_lib
    import torch
    strs = _sorted_strings(1, 1_000_003, 91)  # random lowercase: neighbours differ
    if swap is not None:
        assert strs[swap] != strs[swap + 1]
        strs[swap], strs[swap + 1] = strs[swap + 1], strs[swap]
    w = workloads.from_strings(strs)
    data = torch.from_numpy(w.bytes).pin_memory()
    off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
    perm, st = _sort_with_stats(hs, lambda: hs.argsort(data, off))
    assert (_launches(st, "onesweep") == 0) == (swap is None)
    assert_oracle_equal(w, perm)


# ---- host entry point: the permutation leaves while the fix-up runs ----------

def _host_case(case, n=400_000):
    rng = np.random.default_rng(hash(case) % 1000)
    if case == "rewrites":      # packed words, a few runs of different strings after 8 equal chars
        strs = [bytes(rng.integers(97, 123, size=int(rng.integers(4, 12))).astype(np.uint8)) for _ in range(n)]
        for k in range(0, n, 997):
            strs[k] = b"qqqqqqqq" + bytes(rng.integers(97, 100, size=int(rng.integers(1, 5))).astype(np.uint8))
    elif case == "refinement":  # one huge run of equal codes that is not copies: refinement rounds
        strs = [b"abcdefgh" + bytes(rng.integers(97, 100, size=int(rng.integers(0, 24))).astype(np.uint8))
                for _ in range(n)]
    else:                       # runs of copies only: nothing is rewritten
        words = [bytes(rng.integers(97, 123, size=int(rng.integers(9, 14))).astype(np.uint8)) for _ in range(300)]
        strs = [words[int(i)] for i in rng.integers(0, len(words), size=n)]
    return workloads.from_strings(strs)


@pytest.mark.parametrize("case", ["rewrites", "refinement", "copies"])
@pytest.mark.parametrize("index_u64", [False, True])
@pytest.mark.parametrize("coder", ["auto", "ascii7", "byte8"])
def test_host_entry_point_copy_during_fixup(cuda_lib, case, index_u64, coder):
    """The permutation is copied out as soon as it is written (by tie
    detection for packed words and BYTE8, by the last radix pass for ASCII7
    keys); what the fix-up rewrites afterwards (a range, or everything after
    refinement rounds) is copied again."""
    hs = cuda_lib
    import torch
    w = _host_case(case)
    data = torch.from_numpy(w.bytes).pin_memory()
    off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
    c = {"auto": hs.CODER_AUTO, "ascii7": hs.CODER_ASCII7, "byte8": hs.CODER_BYTE8}[coder]
    assert_oracle_equal(w, hs.argsort(data, off, coder=c, index_u64=index_u64))


def test_host_entry_point_pageable_output(cuda_lib):
    """The C entry point with pageable (numpy) inputs and output: the early
    copy then blocks the host, after the fix-up has been launched."""
    import ctypes
    import torch
    hs = cuda_lib
    w = _host_case("rewrites", 300_000)
    n = w.offsets.size - 1
    out = np.zeros(n, np.uint32)
    need = ctypes.c_size_t(0)
    lib = hs.load()
    assert lib.hs_host_workspace_size(n, int(w.offsets[-1]), hs.MODE_PLAIN, hs.U32, ctypes.byref(need)) == 0
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    st = lib.hs_argsort_host(w.bytes.ctypes.data, w.offsets.ctypes.data, n, hs.MODE_PLAIN, hs.CODER_AUTO, hs.U32,
                             out.ctypes.data, ws.data_ptr(), ws.numel(), None)
    assert st == 0, hs.load().hs_last_error()
    assert_oracle_equal(w, torch.from_numpy(out.view(np.int32)))


# ---- tile-shape tuner ------------------------------------------------------------

@pytest.mark.parametrize("kind,layout", [(2, 0), (5, 1)])
def test_tile_shape_tuner(cuda_lib, kind, layout):
    """The first sort of a size class times two passes in each shape and
    keeps one; the sort that tunes and the sorts after it are exact, and a
    tuner switched off leaves new classes on the default shape."""
    hs = cuda_lib
    hs.autotune(2)
    try:
        # zipf words pack their codes with the index; ASCII7 keys on skewed words travel as pairs
        w = workloads.generate(kind, 1_500_000, 17 + kind)
        data, off = to_device(w)
        coder = hs.CODER_AUTO if layout == 0 else hs.CODER_ASCII7
        n = w.offsets.size - 1
        assert hs.autotune_choice(layout, n) == 0
        assert_oracle_equal(w, hs.argsort_device(data, off, coder=coder))
        chosen = hs.autotune_choice(layout, n)
        assert chosen in (8, 12)
        assert_oracle_equal(w, hs.argsort_device(data, off, coder=coder))
        assert hs.autotune_choice(layout, n) == chosen
        hs.autotune(2)
        hs.autotune(0)
        assert_oracle_equal(w, hs.argsort_device(data, off, coder=coder))
        assert hs.autotune_choice(layout, n) == 0
    finally:
        hs.autotune(2)


@pytest.mark.parametrize("n,packed", [(1 << 24, True), ((1 << 24) + 1, False)])
def test_packed_index_width_boundary_lowercase(cuda_lib, n, packed):
    """Lowercase text codes in 40 bits: 2^24 strings fill the word with their
    24-bit index, one more takes the (key, payload) pairs.  Checked by the
    order property at this size, and the pass layout by its bytes."""
    hs = cuda_lib
    w = workloads.generate(1, n, 5)
    data, off = to_device(w)
    hs.stats_enable(True)
    try:
        perm = hs.argsort_device(data, off)
        st = hs.stats_read()["onesweep"]
    finally:
        hs.stats_enable(False)
    per_key = st["algo_bytes"] / (st["launches"] * n)
    assert (per_key <= 16.0) == packed
    assert_stable_sorted(w, perm)


@pytest.mark.parametrize("host", [False, True])
def test_mode_auto(cuda_lib, host):
    """HS_MODE_AUTO sorts exactly, on device and host inputs (it resolves to
    the plain path)."""
    hs = cuda_lib
    import torch
    w = workloads.generate(5, 200_000, 21)
    if host:
        data = torch.from_numpy(w.bytes).pin_memory()
        off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
        assert_oracle_equal(w, hs.argsort(data, off, mode=hs.MODE_AUTO))
    else:
        data, off = to_device(w)
        assert_oracle_equal(w, hs.argsort_device(data, off, mode=hs.MODE_AUTO))
