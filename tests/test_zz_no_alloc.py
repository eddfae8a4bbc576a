"""build_odf_noalloc: the allocation-free variant of build_odf (through the C ABI).

Some callers cannot allocate device memory at all (their device memory belongs to
another framework's caching allocator, or they run a latency-critical loop where a
cudaMalloc or a synchronising cudaFree is not allowed).  build_odf_noalloc stages its
small inputs in a fixed library-owned array instead of allocated scratch; its results
must equal those of build_odf, also on consecutive calls that reuse that array with
different shapes.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as wl

from gpu_util import ODF_RTOL

pytestmark = pytest.mark.gpu


def test_noalloc_matches_build_odf_on_two_calls():
    import torch
    from paper_2105_13611_gb300 import binding

    ctx = binding.Context(0)
    rng = np.random.default_rng(11)
    cases = [
        (rng.lognormal(0, 4, (3, 50_001)), wl.equal_intervals(50_001, 7), wl.ODF_WIDTHS_12),
        (np.r_[np.zeros(900), rng.lognormal(-3, 2, 4100)][None, :], np.array([0, 5, 1000, 5000]), np.array([0.5, 0.3, 0.2])),
    ]
    for kappa_np, bounds, widths in cases:
        k = torch.from_numpy(np.ascontiguousarray(kappa_np, dtype=np.float32)).cuda()
        shape = (k.shape[0], len(bounds) - 1, len(widths))
        ref = torch.empty(shape, dtype=torch.float64, device="cuda")
        got = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
        ctx.build_odf(k, bounds, widths, ref)
        binding.build_odf_noalloc(0, k, bounds, widths, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.allclose(g, r, rtol=ODF_RTOL, atol=0), np.max(np.abs(g - r) / np.maximum(np.abs(r), 1e-300))


def test_noalloc_rejects_too_many_intervals():
    import torch
    from paper_2105_13611_gb300 import binding

    k = torch.zeros((1, 70_000), dtype=torch.float32, device="cuda")
    out = torch.empty((1, 65_537, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.MpsaError) as e:
        binding.build_odf_noalloc(0, k, np.arange(65_538, dtype=np.int64), [1.0], out)
    assert "65536" in str(e.value)
