"""The C-ABI library loads and exports every symbol its headers declare, and
host-side argument validation works without a GPU (no compute calls)."""

import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"HS_API\s+[\w\s\*]+?\b(hs_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2012_00866_gb300 as hs
    return hs.load()


def test_headers_declare_the_boundary():
    names = _declared_functions()
    for required in ("hs_encode", "hs_argsort", "hs_argsort_batched",
                     "hs_workspace_size", "hs_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_names_match_headers():
    import paper_2012_00866_gb300 as hs
    assert set(hs.EXPORTS) >= set(_declared_functions())


def test_workspace_size_host_only():
    import paper_2012_00866_gb300 as hs
    sizes = [hs.workspace_size(n) for n in (0, 1, 1000, 10**6, 10**7)]
    assert all(b >= a for a, b in zip(sizes, sizes[1:]))
    assert sizes[-1] >= 10**7 * 24   # two key and two payload buffers at least
    with pytest.raises(hs.HuskyError) as e:
        hs.workspace_size(10, mode=7)
    assert e.value.status == hs.ERR_INVALID_ARG


def test_noalloc_limit_fits_its_scratch():
    """hs_argsort_noalloc carves the hs_argsort layout out of its 16 MiB
    static array: at HS_NOALLOC_MAX_N strings that layout must still fit."""
    import paper_2012_00866_gb300 as hs
    assert hs.workspace_size(hs.NOALLOC_MAX_N) <= 16 << 20
    assert hs.workspace_size(hs.NOALLOC_MAX_N + 1) >= hs.workspace_size(hs.NOALLOC_MAX_N)


def test_mode_auto_uses_the_plain_workspace():
    import paper_2012_00866_gb300 as hs
    for n in (1000, 10**6):
        assert hs.workspace_size(n, mode=hs.MODE_AUTO) == hs.workspace_size(n, mode=hs.MODE_PLAIN)


def test_argument_validation_without_gpu(lib):
    import paper_2012_00866_gb300 as hs
    vp = ctypes.c_void_p
    # n = 0 is a no-op and touches nothing
    assert lib.hs_argsort(None, None, 0, 0, 0, 0, None, None, 0, None) == hs.OK
    # bad enums, n too large, NULL pointers: rejected before any CUDA call
    assert lib.hs_argsort(vp(16), vp(16), 5, 9, 0, 0, vp(16), vp(256), 1 << 20, None) == hs.ERR_INVALID_ARG
    assert lib.hs_argsort(vp(16), vp(16), 5, 0, 9, 0, vp(16), vp(256), 1 << 20, None) == hs.ERR_INVALID_ARG
    assert lib.hs_argsort(vp(16), vp(16), 5, 0, 0, 9, vp(16), vp(256), 1 << 20, None) == hs.ERR_INVALID_ARG
    assert lib.hs_argsort(vp(16), vp(16), hs.MAX_N + 1, 0, 0, 0, vp(16), vp(256), 1 << 20, None) == hs.ERR_INVALID_ARG
    assert lib.hs_argsort(None, vp(16), 5, 0, 0, 0, vp(16), vp(256), 1 << 20, None) == hs.ERR_INVALID_ARG
    assert b"null" in lib.hs_last_error()
    # workspace too small is reported before any device work
    assert lib.hs_argsort(vp(16), vp(16), 5, 0, 0, 0, vp(16), vp(256), 16, None) == hs.ERR_WORKSPACE
    assert lib.hs_last_error() != b""


def test_batched_rejects_an_oversize_instance_without_gpu(lib):
    """Local indices are 31-bit.  With more strings than num_segs instances
    of 2^31 - 1 can hold, some instance is too large: rejected on the host,
    before the workspace check or any device work."""
    import paper_2012_00866_gb300 as hs
    vp = ctypes.c_void_p
    n = 1 << 32                       # 2 instances hold at most 2^32 - 2 strings
    st = lib.hs_argsort_batched(vp(16), vp(16), vp(16), 2, n, 0, vp(16), None, 0, None)
    assert st == hs.ERR_INVALID_ARG
    assert b"2^31" in lib.hs_last_error()
    st = lib.hs_argsort_batched(vp(16), vp(16), vp(16), 1, 1 << 31, 0, vp(16), None, 0, None)
    assert st == hs.ERR_INVALID_ARG
    # at the limit the host check passes and the missing workspace is reported
    st = lib.hs_argsort_batched(vp(16), vp(16), vp(16), 1, (1 << 31) - 1, 0, vp(16), None, 0, None)
    assert st == hs.ERR_WORKSPACE


def test_no_cpu_fallback_without_gpu():
    """The product path must fail loudly (not fall back) without a GPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2012_00866_gb300 as hs
    data = torch.zeros(4, dtype=torch.uint8)
    off = torch.zeros(3, dtype=torch.int64)
    with pytest.raises(Exception):
        hs.argsort(data, off)


def test_shutdown_without_gpu(lib):
    """hs_shutdown releases nothing it never made and may be called twice."""
    import paper_2012_00866_gb300 as hs
    assert lib.hs_shutdown() == hs.OK
    assert lib.hs_shutdown() == hs.OK
