"""GPU parity of build_odf against the FP64 oracle ODF (through the C ABI)."""
import numpy as np
import pytest

import workloads as wl
from oracle import odf as od
from oracle import synthesis as sy

from gpu_util import ODF_RTOL, gpu_context, gpu_synth

pytestmark = pytest.mark.gpu
W12 = wl.ODF_WIDTHS_12


def gpu_odf(kappa_np, bounds, widths, mean="arith"):
    import torch
    from paper_2105_13611_gb300 import binding
    ctx = binding.Context(0)
    k = torch.from_numpy(np.ascontiguousarray(kappa_np, dtype=np.float32)).cuda()
    if k.ndim == 1:
        k = k[None, :]
    out = torch.empty((k.shape[0], len(bounds) - 1, len(widths)), dtype=torch.float64, device="cuda")
    ctx.build_odf(k, bounds, widths, out, mean_kind=binding.MEAN_GEOM if mean == "geom" else binding.MEAN_ARITH)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(kappa, bounds, widths, rtol=ODF_RTOL, mean="arith"):
    kappa = np.asarray(kappa, dtype=np.float32)
    g = gpu_odf(kappa, bounds, widths, mean)
    rows = kappa[None, :] if kappa.ndim == 1 else kappa
    for r in range(rows.shape[0]):
        o = od.odf(rows[r].astype(np.float64), bounds, widths, mean=mean)
        scale = np.maximum(np.abs(o), 1e-300)
        rel = np.abs(g[r] - o) / scale
        ok = (rel <= rtol) | ((o == 0) & (g[r] == 0))
        assert ok.all(), (r, np.argwhere(~ok)[:5], g[r][~ok][:5], o[~ok][:5])
    return g


def test_random_lognormal_intervals():
    rng = np.random.default_rng(1)
    x = rng.lognormal(0, 5, (3, 100_003))
    g = check(x, wl.equal_intervals(100_003, 7), W12)
    assert np.all(np.diff(g, axis=2) >= 0)


def adversarial_cases(n=5000):
    rng = np.random.default_rng(2)
    return [np.zeros(n), np.full(n, 3.5), np.r_[np.zeros(n - 1), 1e30], np.repeat([1.0, 2.0, 3.0], [2000, 1, 2999]),
             np.r_[np.zeros(n // 2), np.ones(n - n // 2)], rng.integers(0, 3, n).astype(float),
             np.r_[1e-40 * np.ones(100), rng.lognormal(0, 1, n - 100)],          # denormals
             rng.lognormal(-80, 10, n),                                          # very small and wide
             1.0 + 1e-2 * rng.random(n),                                         # narrow: 1 % spread
             1.0 + 1e-6 * rng.random(n),                                         # a few ulps apart
             np.r_[np.zeros(3000), 1.0 + 1e-3 * rng.random(n - 3000)]]           # zeros + narrow


def test_adversarial():
    for x in adversarial_cases():
        check(x, [0, len(x)], W12)


def test_narrow_large_intervals():
    # smooth, narrow opacity over long intervals (the far-wing dominated rows of the table)
    rng = np.random.default_rng(5)
    n = 120_000
    x = 1e3 * (1.0 + 0.05 * np.sin(np.linspace(0, 40, n)) + 1e-4 * rng.random(n))
    check(x, wl.equal_intervals(n, 3), W12)


def test_small_and_ragged_intervals():
    rng = np.random.default_rng(3)
    x = rng.lognormal(0, 2, 1000)
    for b in ([0, 1], [0, 5, 11, 12, 13, 40, 1000], [3, 997]):
        check(x, b, W12)
    check(x, [0, 1000], [0.5, 0.5])
    check(x, [0, 1000], [1.0])
    check(x, [0, 1000], np.full(32, 1 / 32))


def test_synthesised_opacity_odf():
    # ODF of the GPU's own opacity against the oracle ODF of the same FP32 array (<= 1e-5),
    # and end to end against the oracle opacity (order statistics inherit the opacity bound 1e-4)
    w = wl.config_tiny(n_lines=400, lam=(300.0, 303.1), seed=8)
    ctx, L = gpu_context(w)
    kg, kcg, _ = gpu_synth(ctx, w, np.arange(4))
    b = wl.equal_intervals(kg.shape[1], 5)
    g = check(kg, b, W12)
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    for s in range(4):
        pl = sy.prepare(L, se, ss, el, w.T[s], w.P[s], w.grid)
        k, slack, W = sy.kappa_dense(pl)
        o = od.odf(k, b, W12)
        rel = np.abs(g[s] - o) / (o + pl.kappa_c)
        assert rel.max() <= 1e-4 + (slack.max() / pl.kappa_c if slack.max() > 0 else 0)


# ---- geometric means (exp of the sub-bin integral of ln kappa; a sub-bin reaching into zeros is 0)

def test_geometric_random_lognormal_intervals():
    rng = np.random.default_rng(11)
    x = rng.lognormal(0, 5, (2, 100_003))
    g = check(x, wl.equal_intervals(100_003, 7), W12, mean="geom")
    assert np.all(np.diff(g, axis=2) >= 0)


def test_geometric_adversarial():
    for x in adversarial_cases():
        check(x, [0, len(x)], W12, mean="geom")


def test_geometric_small_ragged_and_zero_boundaries():
    rng = np.random.default_rng(12)
    x = rng.lognormal(0, 2, 1000)
    x[rng.random(1000) < 0.3] = 0.0
    for b in ([0, 1], [0, 5, 11, 12, 13, 40, 1000], [3, 997]):
        check(x, b, W12, mean="geom")
    check(x, [0, 1000], np.full(32, 1 / 32), mean="geom")
    check(x, [0, 1000], [1.0], mean="geom")


def test_geometric_below_arithmetic():
    # AM-GM on every sub-bin of a positive array
    rng = np.random.default_rng(13)
    x = rng.lognormal(-3, 3, 50_000)
    b = wl.equal_intervals(50_000, 4)
    ga = gpu_odf(x, b, W12, "arith")
    gg = check(x, b, W12, mean="geom")
    assert np.all(gg <= ga * (1 + 1e-12))


# ---- long intervals and many ragged ones

def test_long_intervals():
    # 60 000 values per interval, two rows, both kinds of mean
    rng = np.random.default_rng(21)
    x = rng.lognormal(0, 4, (2, 180_000))
    check(x, wl.equal_intervals(180_000, 3), W12)
    check(x, wl.equal_intervals(180_000, 3), W12, mean="geom")


def test_many_ragged_intervals():
    # far more (row, interval) CTAs than SMs, ragged lengths and unaligned starts
    rng = np.random.default_rng(23)
    n = 200_001
    x = rng.lognormal(0, 3, (2, n))
    cuts = np.sort(rng.choice(np.arange(1, n), 1199, replace=False))
    b = np.r_[0, cuts, n]
    check(x, b, W12)
    check(x, b, W12, mean="geom")


def test_gather_and_multiselect_paths():
    # means with at most 12 steps take the count-then-gather kernel, which leaves an
    # interval to the exact multi-select when it is longer than 65,536 points or when its target
    # bins hold more than 8,192 values; mixed in one call, every interval must match the oracle
    rng = np.random.default_rng(29)
    parts = [rng.lognormal(0, 4, 65_536),                  # longest gathered interval
             rng.lognormal(0, 4, 65_537),                  # one point longer: multi-select
             np.full(20_000, 3.25),                        # one bin, 20,000 candidates: multi-select
             np.full(8_192, 7.5),                          # one bin, exactly the candidate capacity
             np.full(8_193, 9.5),                          # one value over it: multi-select
             1.0 + 1e-3 * rng.random(30_000),              # a few bins, most values are candidates
             rng.lognormal(-20, 8, 4097)]
    x = np.concatenate(parts)
    b = np.r_[0, np.cumsum([len(p) for p in parts])]
    check(x, b, W12)
    check(x, b, W12, mean="geom")
    # zeros in a gathered interval: all below the first boundary (a gap of zeros), and a
    # boundary among them (the zeros are candidates of a boundary bin)
    for nz in (3000, 5000):
        z = np.r_[np.zeros(nz), rng.lognormal(0, 2, 30_000 - nz)]
        check(z, [0, len(z)], W12, mean="geom")
        check(z, [0, len(z)], W12)
    # 13 steps: every interval through the multi-select
    w13 = np.r_[np.full(9, 0.1), 0.04, 0.03, 0.02, 0.01]
    check(x, b, w13)
    # one step and two steps (no boundary, one boundary)
    check(x, b, [1.0])
    check(x, b, [0.5, 0.5])
