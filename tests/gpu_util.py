"""Helpers shared by the GPU tests: moving workloads to the device and
checking permutations against the oracle."""

import numpy as np
import torch

import oracle


def to_device(w, device="cuda"):
    data = torch.from_numpy(w.bytes if w.bytes.size else np.zeros(1, np.uint8)).to(device)
    off = torch.from_numpy(w.offsets.view(np.int64)).to(device)
    return data, off


def perm_numpy(t):
    a = t.cpu().numpy()
    return a.view(np.uint32) if a.dtype == np.int32 else a.view(np.uint64)


def assert_oracle_equal(w, perm, threads=None):
    """Element-by-element equality with the oracle's stable argsort."""
    got = perm_numpy(perm)
    want = oracle.stable_argsort(w.bytes, w.offsets, index_u64=got.dtype == np.uint64,
                                 threads=threads)
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{bad.size} of {got.size} positions differ; first at "
                             f"{bad[0]}: got {got[bad[0]]} want {want[bad[0]]}")


def assert_stable_sorted(w, perm, threads=None):
    """Property check: permutation, sorted, stable (unique characterisation)."""
    got = perm_numpy(perm)
    bad = oracle.check_sorted(w.bytes, w.offsets, got, threads=threads)
    assert bad == -1, f"sortedness/stability violated at position {bad}"
