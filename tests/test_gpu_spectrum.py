"""GPU parity of synth_spectrum against the FP64 oracle formal solution (through the C ABI)."""
import numpy as np
import pytest

import workloads as wl
from oracle import spectrum as spc
from oracle import synthesis as sy

from gpu_util import gpu_context

pytestmark = pytest.mark.gpu
MUS = [1.0, 0.8, 0.6, 0.4, 0.2]


def run_gpu(ctx, m, T, P, win, comp=0):
    import torch
    from paper_2105_13611_gb300 import binding
    N = binding.grid_size(win.lam0_nm, win.lam1_nm, win.R)
    out = torch.empty((len(MUS), N), dtype=torch.float32, device="cuda")
    ctx.synth_spectrum(m, T, P, win, MUS, out, comp=comp)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("Teff,logg,D", [(5772.0, 4.44, 12), (9000.0, 3.0, 9), (4000.0, 1.5, 7)])
def test_spectrum_parity(Teff, logg, D):
    w = wl.config_tiny(n_lines=50, lam=(300.0, 300.5), R=5e5, seed=21)
    ctx, L = gpu_context(w)
    m, T, P = spc.grey_atmosphere(D, Teff, logg)
    win = wl.Grid(300.1, 300.3, 5e5)     # lines outside the window reach in with their wings
    g = run_gpu(ctx, m, T, P, win)
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    o = spc.spectrum(L, se, ss, el, m, T, P, win, MUS)
    rel = np.abs(g - o) / o
    assert rel.max() < 1e-4, rel.max()


def test_isothermal_spectrum_is_planck():
    w = wl.config_tiny(n_lines=30, lam=(300.0, 300.5), R=5e5, seed=22)
    ctx, L = gpu_context(w)
    D = 10
    m = 10 ** np.linspace(-4, 3, D)
    T = np.full(D, 6500.0)
    P = 1e4 * m
    win = wl.Grid(300.0, 300.5, 5e5)
    g = run_gpu(ctx, m, T, P, win)
    N = sy.grid_size(win.lam0_nm, win.lam1_nm, win.R)
    B = spc.planck_lambda(sy.grid_lambda_nm(win.lam0_nm, win.R, np.arange(N)) * 1e-7, 6500.0)
    assert np.allclose(g, B[None, :], rtol=2e-5)


@pytest.mark.parametrize("Teff,logg,D,win,lines_lam,n_lines", [
    (5772.0, 4.44, 80, (300.0, 305.0), (298.0, 307.0), 2500),     # 5 nm, 8.3k points
    (3500.0, 1.0, 120, (500.0, 510.0), (497.0, 513.0), 2000),     # cool giant, 120 depths
    (12000.0, 5.0, 40, (400.0, 900.0), (390.0, 910.0), 3000),     # a 500 nm window (4e5 points)
])
def test_spectrum_parity_realistic(Teff, logg, D, win, lines_lam, n_lines):
    # the spectrum workload's shapes: 40-120 depths of a grey atmosphere, windows of 5-500 nm at
    # R = 5e5 over a list of 2000-3000 lines that extends beyond the window (wings reach in);
    # the oracle evaluates sampled wavelengths (random points and the cores of strong lines)
    w = wl.config_tiny(n_lines=n_lines, lam=lines_lam, R=5e5, seed=23)
    ctx, L = gpu_context(w)
    m, T, P = spc.grey_atmosphere(D, Teff, logg)
    g = wl.Grid(win[0], win[1], 5e5)
    I = run_gpu(ctx, m, T, P, g)
    N = I.shape[1]
    rng = np.random.default_rng(3)
    lnq = np.log1p(1 / g.R)
    inside = np.nonzero((L.lam_nm > win[0]) & (L.lam_nm < win[1]))[0]
    top = inside[np.argsort(L.log_gf[inside])[-15:]]
    centres = np.round(np.log(L.lam_nm[top] / g.lam0_nm) / lnq).astype(np.int64)
    js = np.unique(np.clip(np.r_[rng.integers(0, N, 45), centres, centres + 3], 0, N - 1))
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    o, dI = spc.spectrum_at(L, se, ss, el, m, T, P, g, MUS, js)
    err = np.abs(I[:, js].astype(np.float64) - o)
    assert np.all(err <= 1e-4 * o + dI * 1.001), (err / o).max()
