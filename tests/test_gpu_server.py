"""Continuous-batching server: every request's result is the same alone and in the mix
(within the opacity / ODF tolerances), and equals the direct entry points."""
import numpy as np
import pytest

import workloads as wl
from oracle import odf as od
from oracle import spectrum as spc
from oracle import synthesis as sy

from gpu_util import ODF_RTOL, gpu_context

pytestmark = pytest.mark.gpu
MUS = [1.0, 0.8, 0.6, 0.4, 0.2]


def make_requests(w):
    reqs = []
    for Teff, logg, D, win in [(5772.0, 4.44, 12, (300.1, 300.3)), (9000.0, 3.0, 9, (300.0, 300.25)),
                               (4200.0, 2.0, 20, (300.2, 300.45))]:
        m, T, P = spc.grey_atmosphere(D, Teff, logg)
        reqs.append(("spec", (m, T, P, wl.Grid(win[0], win[1], 5e5))))
    from paper_2105_13611_gb300 import binding
    g1, g2 = wl.Grid(300.0, 300.5, 5e5), wl.Grid(300.1, 300.4, 5e5)
    n1, n2 = binding.grid_size(g1.lam0_nm, g1.lam1_nm, g1.R), binding.grid_size(g2.lam0_nm, g2.lam1_nm, g2.R)
    reqs.append(("odf", ([0, 1, 2, 3], g1, [0, 100, 500, n1], wl.ODF_WIDTHS_12)))
    reqs.append(("odf", ([3, 1], g2, [0, n2], [0.5, 0.3, 0.2])))
    reqs.append(("odf", ([2, 0], g2, [0, 40, n2], wl.ODF_WIDTHS_12, binding.MEAN_GEOM)))
    return reqs


def run(server, reqs, together):
    tickets, out = [], []
    for kind, a in reqs:
        t = server.submit_spectrum(*a[:3], a[3], MUS) if kind == "spec" else server.submit_odf(*a)
        if not together:
            out.append(server.wait(t)[0])
        else:
            tickets.append(t)
    for t in tickets:
        out.append(server.wait(t)[0])
    return out


def test_alone_equals_in_the_mix_and_direct():
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=80, lam=(299.9, 300.6), R=5e5, seed=31)
    ctx, L = gpu_context(w)
    reqs = make_requests(w)
    # direct entry points
    direct = []
    for kind, a in reqs:
        if kind == "spec":
            N = binding.grid_size(a[3].lam0_nm, a[3].lam1_nm, a[3].R)
            o = torch.empty((len(MUS), N), dtype=torch.float32, device="cuda")
            ctx.synth_spectrum(a[0], a[1], a[2], a[3], MUS, o)
            direct.append(o.cpu().numpy())
        else:
            sel, g, b, wd = a[:4]
            mk = a[4] if len(a) > 4 else binding.MEAN_ARITH
            N = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
            k = torch.empty((len(sel), N), dtype=torch.float32, device="cuda")
            ctx.synth_opacity(g, sel, k)
            o = torch.empty((len(sel), len(b) - 1, len(wd)), dtype=torch.float64, device="cuda")
            ctx.build_odf(k, b, wd, o, mean_kind=mk)
            direct.append(o.cpu().numpy())
    torch.cuda.synchronize()
    srv = binding.Server(ctx, hbm_budget_bytes=8 << 30, max_inflight=1, rows_per_chunk=4)
    alone = run(srv, reqs, together=False)
    srv.close()
    srv = binding.Server(ctx, hbm_budget_bytes=8 << 30, max_inflight=4, rows_per_chunk=4)
    mixed = run(srv, reqs, together=True)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for (kind, _), d, a1, m1 in zip(reqs, direct, alone, mixed):
        a1 = a1[0] if isinstance(a1, tuple) else a1
        m1 = m1[0] if isinstance(m1, tuple) else m1
        tol = 1e-4 if kind == "spec" else ODF_RTOL
        assert np.allclose(a1, m1, rtol=tol, atol=0)
        assert np.allclose(a1, d, rtol=tol, atol=0)


def test_budget_admission_and_errors():
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=40, lam=(300.0, 300.3), R=5e5, seed=32)
    ctx, L = gpu_context(w)
    # a budget below one request's estimate is rejected at submission
    srv = binding.Server(ctx, hbm_budget_bytes=1 << 10, max_inflight=2)
    m, T, P = spc.grey_atmosphere(8, 6000.0, 4.0)
    with pytest.raises(binding.MpsaError) as e:
        srv.submit_spectrum(m, T, P, wl.Grid(300.0, 300.1, 5e5), MUS)
    assert e.value.code == binding.MPSA_ENOMEM
    srv.close()
    # a budget that fits one request at a time still completes all of them (admission waits)
    srv = binding.Server(ctx, hbm_budget_bytes=64 << 20, max_inflight=4)
    ts = [srv.submit_spectrum(m, T, P, wl.Grid(300.0, 300.1, 5e5), MUS) for _ in range(5)]
    res = [srv.wait(t)[0] for t in ts]
    assert all(np.array_equal(r, res[0]) for r in res)
    assert srv.stats()["bytes_peak"] <= 64 << 20
    srv.close()


def test_served_results_match_the_oracle():
    # every request served in the mix against the FP64 oracle: spectra within 1e-4 (plus the
    # edge-slack bound), arithmetic ODFs end to end (oracle opacity -> oracle ODF; order
    # statistics inherit the opacity bound 1e-4 (o + kappa_c) + slack), geometric ODFs against
    # the oracle's geometric ODF of the same rows' GPU opacity (<= 1e-5) and the served
    # continuum against the oracle's
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_tiny(n_lines=80, lam=(299.9, 300.6), R=5e5, seed=31)
    ctx, L = gpu_context(w)
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    reqs = make_requests(w)
    srv = binding.Server(ctx, hbm_budget_bytes=8 << 30, max_inflight=4, rows_per_chunk=4)
    tickets = [srv.submit_spectrum(*a[:3], a[3], MUS) if kind == "spec" else srv.submit_odf(*a) for kind, a in reqs]
    served = [srv.wait(t)[0] for t in tickets]
    srv.close()
    for (kind, a), res in zip(reqs, served):
        if kind == "spec":
            m, T, P, win = a
            N = res.shape[1]
            js = np.arange(N)
            o, dI = spc.spectrum_at(L, se, ss, el, m, T, P, win, MUS, js)
            assert np.all(np.abs(res.astype(np.float64) - o) <= 1e-4 * o + dI * 1.001)
            continue
        odf_g, kc_g = res
        sel, g, b, wd = a[:4]
        geom = len(a) > 4 and a[4] == binding.MEAN_GEOM
        if geom:
            N = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
            k = torch.empty((len(sel), N), dtype=torch.float32, device="cuda")
            ctx.synth_opacity(g, sel, k)
            torch.cuda.synchronize()
            kn = k.cpu().numpy().astype(np.float64)
        for r, p in enumerate(sel):
            pl = sy.prepare(L, se, ss, el, w.T[p], w.P[p], g, w.cut, w.kc_factor)
            assert abs(float(kc_g[r]) / pl.kappa_c - 1) < 1e-5
            if geom:
                o = od.odf(kn[r], b, wd, mean="geom")
                assert np.all(np.abs(odf_g[r] - o) <= ODF_RTOL * np.abs(o) + 1e-300)
            else:
                k_o, slack, _ = sy.kappa_dense(pl)
                o = od.odf(k_o, b, wd)
                assert np.all(np.abs(odf_g[r] - o) <= 1e-4 * (o + pl.kappa_c) + slack.max() * 1.001)
