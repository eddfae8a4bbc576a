"""Batched form: one persistent, graph-captured launch over rows of several grids gives the
results of the per-call entry points (within the opacity / ODF tolerances), on every replay."""
import numpy as np
import pytest

import workloads as wl
from oracle import synthesis as sy

from gpu_util import ODF_RTOL, gpu_context, opacity_violations

pytestmark = pytest.mark.gpu


def test_batch_matches_per_call_and_replays():
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=300, lam=(300.0, 303.0), R=2e6, seed=41)
    ab = wl.abundance_scales(2, wl.elements(w.n_metals).n, seed=3)
    ctx, L = gpu_context(w, abund=ab)
    nP = len(w.T)
    grids = [wl.Grid(300.0, 303.0, 2e6), wl.Grid(301.0, 301.7, 5e5)]
    sels = [[0, 5, 2, 7], [6, 1, 3]]
    means = [binding.MEAN_ARITH, binding.MEAN_GEOM]
    groups, ref = [], []
    for g, sel, mk in zip(grids, sels, means):
        N = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
        kap = torch.full((len(sel), N), -1.0, dtype=torch.float32, device="cuda")
        kc = torch.empty(len(sel), dtype=torch.float32, device="cuda")
        b = wl.equal_intervals(N, 3)
        odf = torch.empty((len(sel), 3, 12), dtype=torch.float64, device="cuda")
        groups.append(dict(grid=g, sel=sel, kappa=kap, kappa_c=kc, bounds=b, widths=wl.ODF_WIDTHS_12, odf=odf,
                           mean_kind=mk))
        # per-call reference
        k2 = torch.empty_like(kap)
        kc2 = torch.empty_like(kc)
        ctx.synth_opacity(g, sel, k2, kc2)
        o2 = torch.empty_like(odf)
        ctx.build_odf(k2, b, wl.ODF_WIDTHS_12, o2, mean_kind=mk)
        ref.append((k2, kc2, o2))
    batch = binding.Batch(ctx, groups, autotune=True)
    info = batch.info()
    assert info["n_rows"] == 7 and info["n_units"] > 0 and len(info["tune_ms_per_mpoint"]) == 4
    for rep in range(2):
        for g in groups:
            g["kappa"].fill_(-1.0)
        batch.run()
        torch.cuda.synchronize()
        for g, (k2, kc2, o2) in zip(groups, ref):
            kb, kr = g["kappa"].cpu().numpy(), k2.cpu().numpy()
            assert np.all(kb >= 0)
            assert np.allclose(kb, kr, rtol=1e-5, atol=0)
            assert np.allclose(g["kappa_c"].cpu().numpy(), kc2.cpu().numpy(), rtol=0, atol=0)
            assert np.allclose(g["odf"].cpu().numpy(), o2.cpu().numpy(), rtol=1e-5, atol=0)
    # and against the oracle for one row of each grid
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    for g, sel, grp in zip(grids, sels, groups):
        cp = sel[0]
        comp, p = divmod(cp, nP)
        pl = sy.prepare(L, se, ss, el, w.T[p], w.P[p], g, abund_scale=ab[comp])
        k, slack, _ = sy.kappa_dense(pl)
        bad, _, _ = opacity_violations(grp["kappa"][0].cpu().numpy(), k, pl.kappa_c, slack)
        assert len(bad) == 0
    batch.close()
