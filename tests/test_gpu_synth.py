"""GPU parity of synth_opacity against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import workloads as wl
from oracle import synthesis as sy

from gpu_util import gpu_context, gpu_synth, opacity_violations, rel_report

pytestmark = pytest.mark.gpu


def oracle_dense(w, L, T, P, abund=None):
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    pl = sy.prepare(L, se, ss, el, T, P, w.grid, w.cut, w.kc_factor, abund_scale=abund)
    k, slack, W = sy.kappa_dense(pl)
    return pl, k, slack, W


@pytest.mark.parametrize("n_lines,lam,seed", [(40, (300.0, 300.6), 7), (400, (300.0, 303.1), 8), (3, (500.0, 500.2), 9)])
def test_dense_parity_small(n_lines, lam, seed):
    # several 2048-point tiles with a ragged tail, all four (T, P) points at once
    w = wl.config_tiny(n_lines=n_lines, lam=lam, seed=seed)
    ctx, L = gpu_context(w)
    sel = np.arange(len(w.T))
    kg, kcg, evg = gpu_synth(ctx, w, sel)
    for s in sel:
        pl, k, slack, W = oracle_dense(w, L, w.T[s], w.P[s])
        assert abs(kcg[s] / pl.kappa_c - 1) < 1e-5
        bad, err, bound = opacity_violations(kg[s], k, pl.kappa_c, slack)
        assert len(bad) == 0, (s, bad[:10], err[bad[:10]], bound[bad[:10]], rel_report(kg[s], k, pl.kappa_c))
        # evaluations: outer windows include at most 4 padding points per line
        assert W <= evg[s] <= W + 8 * n_lines + 16


def test_precision_naive_runs_and_agrees():
    w = wl.config_tiny(n_lines=200, lam=(300.0, 301.0), seed=12)
    ctx, L = gpu_context(w)
    kc_, _, _ = gpu_synth(ctx, w, [1], precision=0)
    kn_, _, _ = gpu_synth(ctx, w, [1], precision=1)
    pl, k, slack, W = oracle_dense(w, L, w.T[1], w.P[1])
    bad, _, _ = opacity_violations(kn_[0], k, pl.kappa_c, slack)
    assert len(bad) == 0
    assert np.array_equal(kc_[0] > 0, kn_[0] > 0)


def test_compositions_and_row_selection():
    # abundance scales per element; rows selected out of order from a 2-composition table
    w = wl.config_tiny(n_lines=120, lam=(300.0, 300.8), seed=13)
    ab = wl.abundance_scales(2, wl.elements(w.n_metals).n, seed=5)
    ctx, L = gpu_context(w, abund=ab)
    nP = len(w.T)
    sel = [1 * nP + 2, 0 * nP + 0, 1 * nP + 3]
    kg, kcg, _ = gpu_synth(ctx, w, sel)
    for r, cp in enumerate(sel):
        comp, p = divmod(cp, nP)
        pl, k, slack, W = oracle_dense(w, L, w.T[p], w.P[p], abund=ab[comp])
        assert abs(kcg[r] / pl.kappa_c - 1) < 1e-5
        bad, _, _ = opacity_violations(kg[r], k, pl.kappa_c, slack)
        assert len(bad) == 0, (r, bad[:5])


def test_extreme_damping_and_pressures():
    # high pressure (Lorentzian, a >> 1) and low pressure (a << 1e-6) rows
    w = wl.config_tiny(n_lines=60, lam=(400.0, 400.5), seed=14)
    w.T = np.array([2000.0, 3000.0, 50000.0, 200000.0])
    w.P = np.array([1e8, 1e-4, 1e8, 1e-4])
    ctx, L = gpu_context(w)
    kg, kcg, _ = gpu_synth(ctx, w, np.arange(4))
    for s in range(4):
        pl, k, slack, W = oracle_dense(w, L, w.T[s], w.P[s])
        assert abs(kcg[s] / pl.kappa_c - 1) < 2e-5
        bad, err, bound = opacity_violations(kg[s], k, pl.kappa_c, slack)
        assert len(bad) == 0, (s, bad[:5], rel_report(kg[s], k, pl.kappa_c))


def test_microturbulence():
    # a micro-turbulent speed of 2 km/s widens every Doppler width (context-wide setting)
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=150, lam=(300.0, 301.0), seed=22)
    L = w.lines()
    se, ss = wl.species_table(w.n_metals)
    el = wl.elements(w.n_metals)
    ctx = binding.Context(0)
    ctx.load_linelist(L, se, ss)
    ctx.set_atmosphere_grid(el, w.T, w.P, vturb=2e5)
    kg, kcg, _ = gpu_synth(ctx, w, np.arange(4))
    for s in range(4):
        pl = sy.prepare(L, se, ss, el, w.T[s], w.P[s], w.grid, w.cut, w.kc_factor, vturb=2e5)
        k, slack, W = sy.kappa_dense(pl)
        assert abs(kcg[s] / pl.kappa_c - 1) < 1e-5
        bad, err, bound = opacity_violations(kg[s], k, pl.kappa_c, slack)
        assert len(bad) == 0, (s, bad[:5], rel_report(kg[s], k, pl.kappa_c))


def test_wide_grid_far_wing_forms():
    # 9-10000 nm at R = 4000 (28k points, 14 tiles) with strongly damped rows: far wings span
    # factors of tens in wavelength, so |v| passes 1e6 on many tiles as well as staying below
    # it (the two lists of the paired-reciprocal far form) and passes 1e9 on some (the y form)
    w = wl.config_tiny(n_lines=80, lam=(9.0, 10000.0), R=4000.0, seed=21)
    w.T = np.array([3000.0, 6000.0, 12000.0, 40000.0])
    w.P = np.array([1e8, 1e7, 1e8, 1e6])
    ctx, L = gpu_context(w)
    kg, kcg, _ = gpu_synth(ctx, w, np.arange(4))
    for s in range(4):
        pl, k, slack, W = oracle_dense(w, L, w.T[s], w.P[s])
        assert abs(kcg[s] / pl.kappa_c - 1) < 2e-5
        bad, err, bound = opacity_violations(kg[s], k, pl.kappa_c, slack)
        assert len(bad) == 0, (s, bad[:5], rel_report(kg[s], k, pl.kappa_c))


@pytest.mark.parametrize("lam", [(500.0, 501.0), (500.0, 505.0)])
def test_narrow_grid_far_lines_cover_the_last_tile(lam):
    # a window shorter than one 2048-point tile (1 nm at R = 5e5), and one of two tiles whose
    # second is partial, inside a list spread over 450-560 nm: most lines are far from the
    # tile, and at these pressures their wings reach the window.  A far line whose windows
    # reach the grid's last point takes the unmasked forms on the last tile (the points past
    # the grid's end are evaluated and not stored); dense parity against the oracle
    w = wl.config_tiny(n_lines=3000, lam=lam, R=5e5, seed=31)
    w.T = np.array([5000.0, 8000.0, 15000.0, 30000.0])
    w.P = np.array([1e6, 1e7, 1e8, 1e5])
    se, ss = wl.species_table(w.n_metals)
    L = wl.linelist(3000, len(se), 450.0, 560.0, 31)
    ctx, _ = gpu_context(w, lines=L)
    kg, kcg, evg = gpu_synth(ctx, w, np.arange(4))
    lnq = np.log1p(1 / w.grid.R)
    centre = np.log(L.lam_nm / w.grid.lam0_nm) / lnq
    far = (centre < -2048) | (centre > kg.shape[1] + 2048)
    assert far.mean() > 0.9
    for s in range(4):
        pl, k, slack, W = oracle_dense(w, L, w.T[s], w.P[s])
        assert abs(kcg[s] / pl.kappa_c - 1) < 2e-5
        bad, err, bound = opacity_violations(kg[s], k, pl.kappa_c, slack)
        assert len(bad) == 0, (s, bad[:5], rel_report(kg[s], k, pl.kappa_c))
        assert W <= evg[s] <= W + 8 * len(L) + 16
        lo, hi = sy.windows(pl)
        # far lines reach the window on every row (the case this test is about)
        assert np.count_nonzero(far & (hi >= lo)) > 50, s


def test_full_size_sampled():
    # the 20,000-line, 575,365-point, 4-point workload in the launch configuration of the benchmark;
    # the oracle evaluates sampled grid points one by one (random points and the cores of strong lines)
    w = wl.config_small()
    ctx, L = gpu_context(w)
    kg, kcg, evg = gpu_synth(ctx, w, np.arange(4))
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    rng = np.random.default_rng(0)
    for s in range(4):
        pl = sy.prepare(L, se, ss, el, w.T[s], w.P[s], w.grid, w.cut, w.kc_factor)
        assert abs(kcg[s] / pl.kappa_c - 1) < 1e-5
        strong = np.argsort(pl.kappa0)[-40:]
        lnq = np.log1p(1 / w.grid.R)
        centres = np.round(np.log(L.lam_nm[strong] / w.grid.lam0_nm) / lnq).astype(np.int64)
        js = np.unique(np.clip(np.r_[rng.integers(0, pl.N, 150), centres, centres + 3, centres - 17], 0, pl.N - 1))
        ko, so = sy.kappa_at(pl, js)
        bad, err, bound = opacity_violations(kg[s][js], ko, pl.kappa_c, so)
        assert len(bad) == 0, (s, js[bad[:5]], rel_report(kg[s][js], ko, pl.kappa_c))
        assert np.all(np.isfinite(kg[s])) and np.all(kg[s] >= 0)
        lo, hi = sy.windows(pl)
        W = int(np.sum(np.maximum(hi - lo + 1, 0)))
        assert W <= evg[s] <= W + 8 * len(L)


def test_precision_variants_against_oracle():
    # the four library precisions on the same rows (compensated FP32, plain FP32 sums, all FP64,
    # compensated FP32 from an FP32-rounded population table): all within the opacity tolerance;
    # the all-FP64 variant within 1e-7 (outside the edge slack, the FP32 output rounding)
    w = wl.config_tiny(n_lines=400, lam=(300.0, 303.1), seed=8)
    ctx, L = gpu_context(w)
    sel = np.arange(4)
    res = {p: gpu_synth(ctx, w, sel, precision=p)[0] for p in (0, 1, 2, 3)}
    for s in sel:
        pl, k, slack, W = oracle_dense(w, L, w.T[s], w.P[s])
        for p in (0, 1, 2, 3):
            bad, _, _ = opacity_violations(res[p][s], k, pl.kappa_c, slack)
            assert len(bad) == 0, (p, s)
        m = slack == 0
        rel64 = np.abs(res[2][s][m].astype(np.float64) - k[m]) / (k[m] + pl.kappa_c)
        assert rel64.max() < 1e-7        # FP32 output rounding bounds it


def _table_row_oracle(job):
    # one bench row at sampled grid points, in a spawned process (own copy of the line list)
    r, T, P, js = job
    w = wl.config_table()
    L = w.lines()
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    pl = sy.prepare(L, se, ss, el, T, P, w.grid, w.cut, w.kc_factor)
    ko, so = sy.kappa_at(pl, js)
    return r, pl.kappa_c, ko, so


def test_table_workload_sampled():
    # the benchmark's own workload and launch: 5e6 lines over 9-10000 nm at R = 2e6 (14.0 M
    # points), the 8 (T, P) rows of one bench step in one synth_opacity call, then build_odf
    # over the 328 intervals.  The oracle evaluates 60 sampled points of every row one by one
    # (random points and points at and beside the cores of the strongest lines of the row, in
    # spawned processes) and the ODF of sampled intervals on the same FP32 opacity.
    import multiprocessing as mp

    import torch
    from oracle import odf as od
    from paper_2105_13611_gb300 import binding
    w = wl.config_table()
    ctx, L = gpu_context(w)
    rows = [277, 879, 232, 964, 1354, 1044, 1321, 297]
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    kap = torch.empty((len(rows), N), dtype=torch.float32, device="cuda")
    kc = torch.empty(len(rows), dtype=torch.float32, device="cuda")
    ctx.synth_opacity(w.grid, rows, kap, kc)
    b = wl.equal_intervals(N, w.n_intervals)
    odf = torch.empty((len(rows), w.n_intervals, 12), dtype=torch.float64, device="cuda")
    ctx.build_odf(kap, b, w.widths, odf)
    torch.cuda.synchronize()
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    rng = np.random.default_rng(5)
    lnq = np.log1p(1 / w.grid.R)
    # the strongest lines of the list by gf e^{-E/kT} at each row's temperature
    strength = L.log_gf.astype(np.float64)
    jobs, samples = [], {}
    for i, r in enumerate(rows):
        top = np.argsort(strength - L.E_eV / (8.617333262e-5 * w.T[r]) / np.log(10))[-6:]
        centres = np.round(np.log(L.lam_nm[top] / w.grid.lam0_nm) / lnq).astype(np.int64)
        js = np.unique(np.clip(np.r_[rng.integers(0, N, 42), centres, centres + 4, centres - 9], 0, N - 1))
        samples[r] = (i, js, kap[i, torch.from_numpy(js).cuda()].cpu().numpy())
        jobs.append((r, float(w.T[r]), float(w.P[r]), js))
    with mp.get_context("spawn").Pool(min(len(rows), 8)) as pool:
        res = pool.map(_table_row_oracle, jobs)
    for r, kc_o, ko, so in res:
        i, js, kg = samples[r]
        assert len(js) >= 50
        assert abs(float(kc[i]) / kc_o - 1) < 1e-5, r
        bad, err, bound = opacity_violations(kg, ko, kc_o, so)
        assert len(bad) == 0, (r, js[bad[:5]], rel_report(kg, ko, kc_o))
        og = odf[i].cpu().numpy()
        for k in rng.choice(w.n_intervals, 4, replace=False):
            x = kap[i, int(b[k]):int(b[k + 1])].cpu().numpy().astype(np.float64)
            o = od.odf(x, [0, len(x)], w.widths)[0]
            assert np.all(np.abs(og[k] - o) <= 1e-5 * np.abs(o) + 1e-300), (r, k)


def test_no_line_passes_the_cut():
    # a cut far above every line's centre opacity: no window, zero opacity and zero evaluations
    # on every row (the degenerate case of the cut rule); the continuum stays defined
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=50, lam=(300.0, 300.3), seed=71)
    ctx, L = gpu_context(w)
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    kap = torch.full((4, N), -1.0, dtype=torch.float32, device="cuda")
    kc = torch.empty(4, dtype=torch.float32, device="cuda")
    ev = torch.empty(4, dtype=torch.int64, device="cuda")
    ctx.synth_opacity(w.grid, np.arange(4), kap, kc, ev, opts=binding.make_opts(cut=1e12))
    torch.cuda.synchronize()
    assert float(kap.abs().max()) == 0.0 and int(ev.sum()) == 0
    for s in range(4):
        pl = sy.prepare(L, *wl.species_table(w.n_metals), wl.elements(w.n_metals), w.T[s], w.P[s], w.grid,
                        1e12, w.kc_factor)
        assert abs(float(kc[s]) / pl.kappa_c - 1) < 1e-5
        lo, hi = sy.windows(pl)
        assert np.all(hi < lo)


def test_single_point_and_single_line():
    # a one-point grid and a one-line list
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=1, lam=(400.0, 400.0001), seed=72)
    ctx, L = gpu_context(w)
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    kap = torch.empty((4, N), dtype=torch.float32, device="cuda")
    kc = torch.empty(4, dtype=torch.float32, device="cuda")
    ctx.synth_opacity(w.grid, np.arange(4), kap, kc)
    cont = torch.empty((4, N), dtype=torch.float32, device="cuda")
    ctx.synth_continuum(w.grid, np.arange(4), cont)
    torch.cuda.synchronize()
    kg = kap.cpu().numpy()
    for s in range(4):
        pl, k, slack, W = oracle_dense(w, L, w.T[s], w.P[s])
        bad, _, _ = opacity_violations(kg[s], k, pl.kappa_c, slack)
        assert len(bad) == 0
    assert np.all(np.isfinite(cont.cpu().numpy())) and float(cont.min()) > 0


def test_unsorted_list_is_sorted_by_the_library():
    # load_linelist takes a list in any order and sorts a copy by wavelength (stably): the
    # opacity of a shuffled list equals that of the sorted one bit for bit, and the oracle's
    w = wl.config_tiny(n_lines=400, lam=(300.0, 303.1), seed=8)
    ctx, L = gpu_context(w)
    sel = np.arange(len(w.T))
    kg, kcg, evg = gpu_synth(ctx, w, sel)
    perm = np.random.default_rng(73).permutation(len(L))
    ctx2, _ = gpu_context(w, lines=L.subset(perm))
    kg2, kcg2, evg2 = gpu_synth(ctx2, w, sel)
    assert np.array_equal(kg, kg2) and np.array_equal(kcg, kcg2) and np.array_equal(evg, evg2)
    for s in sel:
        pl, k, slack, W = oracle_dense(w, L, w.T[s], w.P[s])
        bad, _, _ = opacity_violations(kg2[s], k, pl.kappa_c, slack)
        assert len(bad) == 0
