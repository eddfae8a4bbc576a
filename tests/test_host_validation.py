"""Host-side argument checks of the C ABI that run before any CUDA call (CPU only).

build_odf_noalloc validates its arguments on the host before it selects a device, so every
invalid call below returns MPSA_EINVAL without touching a GPU (the pointers are never
dereferenced).  mpsa_grid_size is plain host arithmetic and is compared with the oracle's
grid definition (App. E).
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from oracle import synthesis as sy

W12 = wl.ODF_WIDTHS_12


@pytest.fixture(scope="module")
def lib():
    import os
    from paper_2105_13611_gb300 import binding
    from paper_2105_13611_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return binding.load_library(b.LIB)


def call_noalloc(lib, N, bounds, widths, mean_kind=0, n_rows=1):
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    w = np.ascontiguousarray(widths, dtype=np.float64)
    dummy = C.c_void_p(16)   # never dereferenced: the checks fail first
    return lib.build_odf_noalloc(0, dummy, n_rows, N, len(b) - 1, b.ctypes.data_as(C.POINTER(C.c_int64)), len(w),
                                 w.ctypes.data_as(C.POINTER(C.c_double)), mean_kind, dummy, None)


def test_noalloc_rejects_invalid_arguments(lib):
    N = 1000
    good_b = [0, 400, 1000]
    cases = [
        (N, good_b, W12, 0, 0),                     # n_rows = 0
        (N, good_b, [], 0, 1),                      # no steps
        (N, good_b, np.full(33, 1 / 33), 0, 1),     # more than 32 steps
        (N, good_b, W12 * 0.9, 0, 1),               # widths do not sum to 1
        (N, good_b, np.r_[W12[:-1], -W12[-1]], 0, 1),   # negative width
        (N, good_b, W12, 2, 1),                     # unknown mean kind
        (N, [0, 400, 400, 1000], W12, 0, 1),        # empty interval
        (N, [0, 600, 400], W12, 0, 1),              # decreasing bounds
        (N, [0, 400, 1001], W12, 0, 1),             # beyond N
        (N, [-1, 400, 1000], W12, 0, 1),            # negative start
        (1 << 23, [0, 1 << 21], W12, 0, 1),         # interval of 2^21 points
        (N, np.arange(65538), W12, 0, 1),           # more than 65,536 intervals
        (N, good_b, W12, 0, 65536),                 # more rows than one launch's grid holds
    ]
    for N_, b, w, mk, rows in cases:
        assert call_noalloc(lib, N_, b, w, mk, rows) == -1, (N_, len(b), len(w), mk, rows)


def test_grid_size_matches_the_oracle(lib):
    from paper_2105_13611_gb300 import binding
    for lam0, lam1, R in [(300.0, 400.0, 2e6), (9.0, 10000.0, 2e6), (300.0, 300.0001, 5e5), (500.0, 1500.0, 1000.0)]:
        g = binding.LGrid(lam0, lam1, R)
        assert lib.mpsa_grid_size(C.byref(g)) == sy.grid_size(lam0, lam1, R)


def test_binding_checks_odf_buffers_before_the_call(lib):
    # dtype, shape and device of the ODF buffers are checked in the binding before any C call
    # (a float32 or undersized output would otherwise be written past its end)
    import torch
    from paper_2105_13611_gb300 import binding
    b, w = np.array([0, 400, 1000]), W12
    k32 = torch.zeros((2, 1000), dtype=torch.float32)
    good = torch.zeros((2, 2, 12), dtype=torch.float64)
    bad = [
        (torch.zeros((2, 1000), dtype=torch.float64), good, "float32"),      # kappa not float32
        (k32, torch.zeros((2, 2, 12), dtype=torch.float32), "float64"),     # output not float64
        (k32, torch.zeros((2, 2, 11), dtype=torch.float64), "shape"),       # output too small
        (k32, torch.zeros((1, 2, 12), dtype=torch.float64), "shape"),       # rows differ
        (k32, good, "cuda:0"),                                              # host tensors
    ]
    for kappa, out, msg in bad:
        with pytest.raises(ValueError, match=msg):
            binding.build_odf_noalloc(0, kappa, b, w, out)
