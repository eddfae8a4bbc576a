"""GPU parity of the multi-stage equation of state (paper App. A: Saha-Boltzmann ratios between
stages I..V, temperature-dependent partition functions, particle and charge conservation)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import workloads as wl
from oracle import physics as ph
from oracle import synthesis as sy

from gpu_util import opacity_violations, rel_report

pytestmark = pytest.mark.gpu


def check_row(row, pop, n_el, rtol=1e-10):
    assert abs(row[2] / pop.n_e - 1) < rtol
    assert abs(row[4] / pop.rho - 1) < 1e-12
    if pop.n_HI > 1e-250:
        assert abs(row[3] / pop.n_HI - 1) < rtol
    nu = row[5:5 + 5 * n_el].reshape(n_el, 5)
    big = pop.NU > 1e-250
    assert np.all(np.abs(nu[big] / pop.NU[big] - 1) < rtol), np.max(np.abs(nu[big] / pop.NU[big] - 1))
    assert np.all(nu[~big] <= 1e-240)


def test_eos_populations_whole_table():
    # every row of the 57 x 25 T-P grid with two compositions, stages up to V
    from paper_2105_13611_gb300 import binding
    tab = wl.eos_table(15)
    T, P = wl.tp_grid_dfsynthe()
    ab = wl.abundance_scales(2, tab.n, seed=41)
    ctx = binding.Context(0)
    ctx.set_atmosphere_grid_eos(tab, T, P, abund_scale=ab)
    rows = ctx.get_populations(0, 2 * len(T))
    assert rows.shape == (2 * len(T), 5 + 5 * tab.n)
    for r in range(0, 2 * len(T), 3):
        comp, p = divmod(r, len(T))
        pop = ph.populations_eos(T[p], P[p], tab, ab[comp])
        assert rows[r, 0] == T[p] and rows[r, 1] == P[p]
        check_row(rows[r], pop, tab.n)


def test_two_stage_table_matches_the_single_ionisation_oracle():
    # set_atmosphere_grid is the two-stage, constant-U case of the same solver
    from paper_2105_13611_gb300 import binding
    el = wl.elements(15)
    T, P = wl.tp_grid_dfsynthe()
    ctx = binding.Context(0)
    ctx.set_atmosphere_grid(el, T, P)
    rows = ctx.get_populations(0, len(T))
    for r in range(0, len(T), 7):
        pop = ph.populations(T[r], P[r], el)
        assert abs(rows[r, 2] / pop.n_e - 1) < 1e-10
        nu = rows[r, 5:].reshape(el.n, 5)
        assert np.allclose(nu[:, :2], pop.NU, rtol=1e-10, atol=1e-290) and np.all(nu[:, 2:] == 0)


@pytest.mark.parametrize("n_lines,lam,seed", [(300, (300.0, 302.0), 51), (60, (9.0, 10000.0), 52)])
def test_eos_opacity_parity(n_lines, lam, seed):
    # lines of stages I-III on the multi-stage populations: opacity against the oracle (dense)
    from paper_2105_13611_gb300 import binding
    R = 2e6 if lam[1] < 1000 else 4000.0
    w = wl.config_tiny(n_lines=n_lines, lam=lam, R=R, seed=seed)
    w.T = np.array([3000.0, 8000.0, 20000.0, 60000.0])
    w.P = np.array([1e5, 1e2, 1e6, 1e4])
    tab = wl.eos_table(w.n_metals)
    se, ss = wl.species_table_eos(w.n_metals, 3)
    L = wl.linelist(n_lines, len(se), lam[0], lam[1], seed)
    ctx = binding.Context(0)
    ctx.load_linelist(L, se, ss)
    ctx.set_atmosphere_grid_eos(tab, w.T, w.P)
    import torch
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    kap = torch.empty((4, N), dtype=torch.float32, device="cuda")
    kc = torch.empty(4, dtype=torch.float32, device="cuda")
    ctx.synth_opacity(w.grid, np.arange(4), kap, kc)
    torch.cuda.synchronize()
    kg, kcg = kap.cpu().numpy(), kc.cpu().numpy()
    for s in range(4):
        pl = sy.prepare(L, se, ss, tab, w.T[s], w.P[s], w.grid, w.cut, w.kc_factor)
        k, slack, _ = sy.kappa_dense(pl)
        assert abs(kcg[s] / pl.kappa_c - 1) < 2e-5
        bad, err, bound = opacity_violations(kg[s], k, pl.kappa_c, slack)
        assert len(bad) == 0, (s, bad[:5], rel_report(kg[s], k, pl.kappa_c))


def test_stage_beyond_the_table_is_rejected():
    # a species in stage III needs an element table with three stages or more
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=20, lam=(300.0, 300.2), seed=53)
    se, ss = wl.species_table_eos(w.n_metals, 3)
    L = wl.linelist(20, len(se), 300.0, 300.2, 53)
    ctx = binding.Context(0)
    ctx.load_linelist(L, se, ss)
    ctx.set_atmosphere_grid(wl.elements(w.n_metals), w.T, w.P)
    import torch
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    kap = torch.empty((1, N), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.MpsaError) as e:
        ctx.synth_opacity(w.grid, [0], kap)
    assert e.value.code == binding.MPSA_EINVAL and "stage" in str(e.value)
