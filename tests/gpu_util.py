"""Helpers shared by the GPU parity tests: set up the CUDA context from a workload
and evaluate the oracle on the same seeded inputs."""
import numpy as np

import workloads as wl

OPACITY_RTOL = 1e-4      # |k_gpu - k_orc| <= 1e-4 (k_orc + kappa_c) + slack (opacity tolerance)
ODF_RTOL = 1e-5          # ODF steps from an identical FP32 opacity array


def gpu_context(w, lines=None, abund=None):
    from paper_2105_13611_gb300 import binding
    ctx = binding.Context(0)
    L = lines if lines is not None else w.lines()
    se, ss = wl.species_table(w.n_metals)
    ctx.load_linelist(L, se, ss)
    ctx.set_atmosphere_grid(wl.elements(w.n_metals), w.T, w.P, abund_scale=abund)
    return ctx, L


def gpu_synth(ctx, w, sel, precision=0):
    import torch
    from paper_2105_13611_gb300 import binding
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    kap = torch.empty((len(sel), N), dtype=torch.float32, device="cuda")
    kc = torch.empty(len(sel), dtype=torch.float32, device="cuda")
    ev = torch.empty(len(sel), dtype=torch.int64, device="cuda")
    ctx.synth_opacity(w.grid, sel, kap, kc, ev, opts=binding.make_opts(w.cut, w.kc_factor, precision))
    torch.cuda.synchronize()
    return kap.cpu().numpy(), kc.cpu().numpy(), ev.cpu().numpy()


def opacity_violations(k_gpu, k_orc, kc, slack, rtol=OPACITY_RTOL):
    """Indices where the GPU opacity breaks the tolerance |dk| <= rtol (k + kc) + slack."""
    k_gpu = np.asarray(k_gpu, dtype=np.float64)
    err = np.abs(k_gpu - k_orc)
    bound = rtol * (k_orc + kc) + slack * (1 + 1e-3)
    return np.nonzero(err > bound)[0], err, bound


def rel_report(k_gpu, k_orc, kc):
    k_gpu = np.asarray(k_gpu, dtype=np.float64)
    rel = np.abs(k_gpu - k_orc) / (k_orc + kc)
    m = k_orc >= kc
    plain = np.abs(k_gpu[m] - k_orc[m]) / k_orc[m] if m.any() else np.zeros(1)
    return dict(max_rel_floor=float(rel.max()), p99_rel_floor=float(np.quantile(rel, 0.99)),
                max_rel_above_kc=float(plain.max()), n_above_kc=int(m.sum()))
