"""GPU parity of the closed-form continuum (synth_continuum; paper Sect. 2.1 sources electron
scattering, H I bound-free and free-free, Rayleigh on H I) and of spectra that use it, against
the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import continuum as co
from oracle import physics as ph
from oracle import spectrum as spc
from oracle import synthesis as sy

from gpu_util import gpu_context

pytestmark = pytest.mark.gpu
MUS = [1.0, 0.8, 0.6, 0.4, 0.2]


@pytest.mark.parametrize("eos", [False, True])
def test_continuum_rows(eos):
    # 9-10000 nm at R = 4000 (every H I edge of levels 1..8 inside), rows from 2000 K to 2e5 K
    import torch
    from paper_2105_13611_gb300 import binding
    T, P = wl.tp_grid_dfsynthe()
    rows = np.array([0, 12, 24, 300, 612, 900, 1100, 1424], dtype=np.int32)
    ctx = binding.Context(0)
    el = wl.eos_table(15) if eos else wl.elements(15)
    (ctx.set_atmosphere_grid_eos if eos else ctx.set_atmosphere_grid)(el, T, P)
    g = wl.Grid(9.0, 10000.0, 4000.0)
    N = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
    out = torch.empty((len(rows), N), dtype=torch.float32, device="cuda")
    ctx.synth_continuum(g, rows, out)
    torch.cuda.synchronize()
    kg = out.cpu().numpy().astype(np.float64)
    lam = sy.grid_lambda_nm(g.lam0_nm, g.R, np.arange(N))
    edge = ph.H_PLANCK * ph.C_LIGHT / (co.CHI_H_EV * ph.EV) * 1e7 * np.arange(1, co.N_LEVELS + 1) ** 2
    # the two grid points beside each edge may fall on either side in FP32 and FP64
    near = np.zeros(N, dtype=bool)
    for e in edge:
        j = np.searchsorted(lam, e)
        near[max(j - 1, 0):j + 1] = True
    for i, r in enumerate(rows):
        pop = ph.populations_eos(T[r], P[r], el) if eos else ph.populations(T[r], P[r], el)
        U_HI = float(ph.partition_functions(el, T[r])[0, 0]) if eos else float(el.U1[0])
        ko = co.kappa_c(lam, pop, U_HI=U_HI)
        rel = np.abs(kg[i] - ko) / ko
        assert np.all(rel[~near] < 2e-5), (r, rel[~near].max(), lam[~near][np.argmax(rel[~near])])
        assert np.all(np.isfinite(kg[i])) and np.all(kg[i] > 0)


def test_continuum_sources_and_errors():
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny()
    ctx, _ = gpu_context(w)
    g = wl.Grid(80.0, 3000.0, 2000.0)
    N = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
    parts = []
    for src in (binding.CONT_ELEC, binding.CONT_HBF, binding.CONT_HFF, binding.CONT_HRAY):
        o = torch.empty((2, N), dtype=torch.float32, device="cuda")
        ctx.synth_continuum(g, [0, 3], o, sources=src)
        parts.append(o.double())
    tot = torch.empty((2, N), dtype=torch.float32, device="cuda")
    ctx.synth_continuum(g, [0, 3], tot)
    assert torch.allclose(tot.double(), sum(parts), rtol=1e-6, atol=0)
    with pytest.raises(binding.MpsaError):
        ctx.synth_continuum(g, [0], tot[:1], sources=16)
    with pytest.raises(binding.MpsaError):
        ctx.synth_continuum(g, [7], tot[:1])


def test_spectrum_with_closed_form_continuum():
    # a grey atmosphere with the closed-form continuum in the radiative transfer (the cut keeps the
    # flat continuum), sampled wavelengths across the Balmer edge, against the oracle
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=400, lam=(355.0, 375.0), R=5e5, seed=61)
    ctx, L = gpu_context(w)
    m, T, P = spc.grey_atmosphere(50, 9000.0, 4.0)
    win = wl.Grid(360.0, 370.0, 5e5)
    N = binding.grid_size(win.lam0_nm, win.lam1_nm, win.R)
    out = torch.empty((len(MUS), N), dtype=torch.float32, device="cuda")
    ctx.synth_spectrum(m, T, P, win, MUS, out, opts=binding.make_opts(continuum=binding.CONT_ALL))
    torch.cuda.synchronize()
    I = out.cpu().numpy().astype(np.float64)
    lam = sy.grid_lambda_nm(win.lam0_nm, win.R, np.arange(N))
    balmer = ph.H_PLANCK * ph.C_LIGHT / (co.CHI_H_EV * ph.EV) * 1e7 * 4
    jb = int(np.searchsorted(lam, balmer))
    rng = np.random.default_rng(2)
    js = np.unique(np.r_[rng.integers(0, N, 40), jb - 30, jb - 3, jb + 2, jb + 30])
    js = js[(js < jb - 1) | (js > jb)]
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    o, dI = spc.spectrum_at(L, se, ss, el, m, T, P, win, MUS, js, continuum=("elec", "bf", "ff", "ray"))
    err = np.abs(I[:, js] - o)
    assert np.all(err <= 1e-4 * o + dI * 1.001), (err / o).max()
    # the flat-continuum spectrum differs (the continuum matters)
    flat = torch.empty_like(out)
    ctx.synth_spectrum(m, T, P, win, MUS, flat)
    torch.cuda.synchronize()
    assert not np.allclose(flat.cpu().numpy(), I, rtol=1e-3)
