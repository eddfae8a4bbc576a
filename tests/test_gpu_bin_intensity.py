"""GPU parity of odf_intensity (bin intensities from an ODF table) against the FP64 oracle."""
import numpy as np
import pytest

import workloads as wl
from oracle import bin_intensity as bi
from oracle import spectrum as spc

from gpu_util import gpu_context

pytestmark = pytest.mark.gpu
MUS = [1.0, 0.8, 0.6, 0.4, 0.2]
W12 = wl.ODF_WIDTHS_12
RTOL = 1e-4
# the output is FP32: intensities far below FP32's normal range (far-UV bins of cool rays)
# are compared absolutely
ATOL = 1e-34


def close(g, o):
    err = np.abs(g - o) - RTOL * np.abs(o)
    return err.max() <= ATOL, float((np.abs(g - o) / np.maximum(np.abs(o), 1e-300))[np.abs(o) > 1e-30].max(initial=0))


def run_gpu(lt, lp, odf, kc, lam, widths, m, T, P, mus, status=False):
    import torch
    from paper_2105_13611_gb300 import binding
    ctx = binding.Context(0)
    nT, nP = len(lt), len(lp)
    K, ns = odf.shape[-2], odf.shape[-1]
    d_odf = torch.from_numpy(np.ascontiguousarray(odf.reshape(nT * nP, K, ns), dtype=np.float64)).cuda()
    d_kc = torch.from_numpy(np.ascontiguousarray(np.reshape(kc, -1), dtype=np.float32)).cuda()
    m, T, P = (torch.from_numpy(np.ascontiguousarray(np.atleast_2d(a), dtype=np.float64)).cuda() for a in (m, T, P))
    out = torch.empty((m.shape[0], len(mus), K), dtype=torch.float32, device="cuda")
    st = torch.empty(m.shape[0], dtype=torch.int32, device="cuda") if status else None
    ctx.odf_intensity(lt, lp, d_odf, d_kc, lam, widths, m, T, P, mus, out, st)
    torch.cuda.synchronize()
    return (out.cpu().numpy(), st.cpu().numpy()) if status else out.cpu().numpy()


def oracle(lt, lp, odf, kc, lam, widths, m, T, P, mus):
    nT, nP = len(lt), len(lp)
    tab = odf.reshape(nT, nP, odf.shape[-2], odf.shape[-1])
    return bi.bin_intensity(tab, np.reshape(kc, (nT, nP)).astype(np.float64), lt, lp, lam, widths, m, T, P, mus)


def test_parity_random_table_and_rays():
    lt, lp, odf, kc, lam = wl.odf_table_synthetic(7, 5, 9, 12, seed=31)
    m, T, P = wl.ray_atmospheres(6, 40, seed=32)
    # stretch two rays beyond the grid in T and P (the coordinates clamp to the edges)
    T[4] *= 0.4
    P[5] *= 1e4
    g = run_gpu(lt, lp, odf, kc, lam, W12, m, T, P, MUS)
    for r in range(m.shape[0]):
        o = oracle(lt, lp, odf, kc, lam, W12, m[r], T[r], P[r], MUS)
        ok, rel = close(g[r], o)
        assert ok, (r, rel)


@pytest.mark.parametrize("n_mu,ns", [(1, 1), (3, 3), (16, 32), (5, 12)])
def test_parity_shapes(n_mu, ns):
    lt, lp, odf, kc, lam = wl.odf_table_synthetic(4, 3, 70, ns, seed=33 + ns)
    w = np.full(ns, 1.0 / ns)
    mus = np.linspace(1.0, 0.1, n_mu)
    m, T, P = wl.ray_atmospheres(3, 17, seed=34)
    g = run_gpu(lt, lp, odf, kc, lam, w, m, T, P, mus)
    for r in range(3):
        o = oracle(lt, lp, odf, kc, lam, w, m[r], T[r], P[r], mus)
        ok, rel = close(g[r], o)
        assert ok, (r, rel)


def test_isothermal_is_planck():
    lt, lp, odf, kc, lam = wl.odf_table_synthetic(5, 4, 33, 12, seed=35)
    D = 50
    m = 10 ** np.linspace(-5, 2, D)
    T = np.full(D, 6400.0)
    P = 10 ** np.linspace(-1, 6, D)
    g = run_gpu(lt, lp, odf, kc, lam, W12, m, T, P, MUS)[0]
    B = spc.planck_lambda(lam * 1e-7, 6400.0)
    assert np.allclose(g, B[None, :], rtol=2e-5, atol=ATOL)


def test_ray_status_marks_bad_rays():
    lt, lp, odf, kc, lam = wl.odf_table_synthetic(4, 3, 20, 12, seed=36)
    m, T, P = wl.ray_atmospheres(4, 12, seed=37)
    m[1, 5] = m[1, 4]          # column mass not increasing
    T[2, 3] = -10.0            # negative temperature
    g, st = run_gpu(lt, lp, odf, kc, lam, W12, m, T, P, MUS, status=True)
    assert list(st) == [0, 1, 1, 0]
    assert np.isnan(g[1]).all() and np.isnan(g[2]).all()
    for r in (0, 3):
        o = oracle(lt, lp, odf, kc, lam, W12, m[r], T[r], P[r], MUS)
        ok, rel = close(g[r], o)
        assert ok, (r, rel)


def test_table_from_build_odf():
    # the table of the library's own synthesis and build_odf on a 3 x 3 T-P grid
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=300, lam=(300.0, 301.0), seed=38)
    nT, nP = 3, 3
    Tg = np.exp(np.linspace(np.log(3500.0), np.log(20000.0), nT))
    Pg = 10 ** np.linspace(1.0, 6.0, nP)
    TT, PP = np.meshgrid(Tg, Pg, indexing="ij")
    w.T, w.P = TT.reshape(-1), PP.reshape(-1)
    ctx, _ = gpu_context(w)
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    kap = torch.empty((nT * nP, N), dtype=torch.float32, device="cuda")
    kc = torch.empty(nT * nP, dtype=torch.float32, device="cuda")
    ctx.synth_opacity(w.grid, np.arange(nT * nP), kap, kc)
    K = 6
    b = wl.equal_intervals(N, K)
    odf = torch.empty((nT * nP, K, 12), dtype=torch.float64, device="cuda")
    ctx.build_odf(kap, b, W12, odf)
    torch.cuda.synchronize()
    lam_edges = w.grid.lam0_nm * np.exp(b * np.log1p(1.0 / w.grid.R))
    lam = 0.5 * (lam_edges[:-1] + lam_edges[1:])
    lt, lp = np.log10(Tg), np.log10(Pg)
    m, T, P = wl.ray_atmospheres(3, 30, seed=39)
    g = run_gpu(lt, lp, odf.cpu().numpy(), kc.cpu().numpy(), lam, W12, m, T, P, MUS)
    for r in range(3):
        o = oracle(lt, lp, odf.cpu().numpy(), kc.cpu().numpy(), lam, W12, m[r], T[r], P[r], MUS)
        ok, rel = close(g[r], o)
        assert ok, (r, rel)


def test_full_size_sampled_rays():
    # the benchmark's configuration (57 x 25 table, 328 bins x 12 sub-bins, 80 depths, 5 mu)
    # on 256 rays; two rays checked against the oracle
    lt, lp, odf, kc, lam = wl.odf_table_synthetic(57, 25, 328, 12, seed=40)
    m, T, P = wl.ray_atmospheres(256, 80, seed=41)
    g = run_gpu(lt, lp, odf, kc, lam, W12, m, T, P, MUS)
    assert np.isfinite(g).all()
    for r in (0, 201):
        o = oracle(lt, lp, odf, kc, lam, W12, m[r], T[r], P[r], MUS)
        ok, rel = close(g[r], o)
        assert ok, (r, rel)
