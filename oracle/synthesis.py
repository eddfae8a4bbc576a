"""Line-by-line opacity synthesis in FP64 (oracle; test infrastructure only).

Steps, in the order of App. E of the paper:
  1. populations at the (T, P) point (physics.populations);
  2. per-line terms of Eq. (l_nu_line) (physics.line_terms);
  3. pre-selection / cut: a line contributes at grid point j iff its absorption
     coefficient ell_i(lambda_j) >= t_p (Sect. 4.3, App. E).  Following the flat
     continuum of the synthetic workload, kappa_c = kc_factor * median_i kappa0_i
     with kappa0_i = S_i H(0, a_i) (lower middle order statistic for an even
     count) and t_p = cut * kappa_c;
  4. summation of ell_i(lambda_j) over all lines onto the log-lambda grid
     lambda_j = lambda_0 (1 + 1/R)^j (App. E), in FP64.

v_ij = (c/lambda_j - nu0_i)/dnuD_i is the exact frequency offset of Eq. (l_nu_line).
Since H is even and decreasing in |v| and v_ij is monotone in j, each line's
contributing set is one contiguous index window, found by bisection.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import physics
from .voigt import H

C = physics.C_LIGHT


def grid_size(lam0_nm: float, lam1_nm: float, R: float) -> int:
    """N = floor(ln(lam1/lam0) / ln(1 + 1/R)) + 1 points of lambda_j = lam0 (1+1/R)^j."""
    return int(math.floor(math.log(lam1_nm / lam0_nm) / math.log1p(1.0 / R))) + 1


def grid_lambda_nm(lam0_nm: float, R: float, j) -> np.ndarray:
    return lam0_nm * np.exp(np.asarray(j, dtype=np.float64) * math.log1p(1.0 / R))


@dataclass
class PointLines:
    """All per-line quantities of one (T, P) point needed for synthesis."""
    pop: physics.Populations
    terms: physics.LineTerms
    kappa0: np.ndarray
    kappa_c: float
    t: float
    lam0_nm: float
    R: float
    N: int


def lower_median(x: np.ndarray) -> float:
    s = np.sort(np.asarray(x, dtype=np.float64))
    return float(s[(len(s) - 1) // 2])


def prepare(lines, species_el, species_stage, el, T, P, grid, cut=1e-3, kc_factor=1e-2,
            abund_scale=None, vturb=0.0) -> PointLines:
    # an element table with stages beyond II (n_stages) takes the multi-stage equation of state
    pop = physics.populations_eos(T, P, el, abund_scale) if hasattr(el, "n_stages") else \
        physics.populations(T, P, el, abund_scale)
    terms = physics.line_terms(lines, species_el, species_stage, el, pop, vturb)
    kappa0 = terms.S * H(0.0, terms.a)
    kc = kc_factor * lower_median(kappa0)
    N = grid_size(grid.lam0_nm, grid.lam1_nm, grid.R)
    return PointLines(pop, terms, kappa0, kc, cut * kc, grid.lam0_nm, grid.R, N)


def ell(pl: PointLines, i, j):
    """ell_i(lambda_j) of Eq. (l_nu_line) for line indices i and grid indices j (broadcast)."""
    lam_cm = grid_lambda_nm(pl.lam0_nm, pl.R, j) * 1e-7
    v = (C / lam_cm - pl.terms.nu0[i]) / pl.terms.dnuD[i]
    return pl.terms.S[i] * H(v, pl.terms.a[i])


def windows(pl: PointLines, level: float = 1.0):
    """Per line, the index window [lo, hi] where ell >= level * t (lo > hi when empty)."""
    L = len(pl.kappa0)
    i = np.arange(L)
    thr = level * pl.t
    lnq = math.log1p(1.0 / pl.R)
    lam0 = C / pl.terms.nu0 * 1e7
    x0 = np.log(lam0 / pl.lam0_nm) / lnq
    jf = np.clip(np.floor(x0), 0, pl.N - 1).astype(np.int64)
    jc = np.clip(jf + 1, 0, pl.N - 1)
    # the grid point of largest ell is one of the two neighbours of the centre
    ef, ec = ell(pl, i, jf), ell(pl, i, jc)
    jm = np.where(ec > ef, jc, jf)
    ok = np.maximum(ef, ec) >= thr
    # upper edge: largest j >= jm with ell >= thr
    lo_u = jm.copy(); hi_u = np.full(L, pl.N, dtype=np.int64)
    while True:
        act = ok & (hi_u - lo_u > 1)
        if not act.any():
            break
        mid = (lo_u + hi_u) // 2
        good = np.zeros(L, dtype=bool)
        good[act] = ell(pl, i[act], mid[act]) >= thr
        lo_u = np.where(act & good, mid, lo_u)
        hi_u = np.where(act & ~good, mid, hi_u)
    # lower edge: smallest j <= jm with ell >= thr
    hi_l = jm.copy(); lo_l = np.full(L, -1, dtype=np.int64)
    while True:
        act = ok & (hi_l - lo_l > 1)
        if not act.any():
            break
        mid = (lo_l + hi_l) // 2
        good = np.zeros(L, dtype=bool)
        good[act] = ell(pl, i[act], mid[act]) >= thr
        hi_l = np.where(act & good, mid, hi_l)
        lo_l = np.where(act & ~good, mid, lo_l)
    lo = np.where(ok, hi_l, 1)
    hi = np.where(ok, lo_u, 0)
    return lo, hi


def kappa_dense(pl: PointLines, slack_band: float = 3e-5):
    """Dense opacity on the whole grid plus the edge slack.

    Returns (kappa[N], slack[N], W) where W = sum of window lengths (the exact
    number of (line, grid point) contributions) and slack_j = sum of ell_i(j) over
    lines whose |ell_i(j)/t - 1| <= slack_band (contributions whose inclusion a
    correct lower-precision evaluation may decide either way).
    """
    kappa = np.zeros(pl.N)
    slack = np.zeros(pl.N)
    lo, hi = windows(pl)
    lo2, hi2 = windows(pl, 1.0 - slack_band)
    W = int(np.sum(np.maximum(hi - lo + 1, 0)))
    for i in np.nonzero(hi2 >= lo2)[0]:
        j = np.arange(lo2[i], hi2[i] + 1)
        e = ell(pl, i, j)
        inc = e >= pl.t
        kappa[j[inc]] += e[inc]
        near = np.abs(e / pl.t - 1.0) <= slack_band
        slack[j[near]] += e[near]
    return kappa, slack, W


def kappa_at(pl: PointLines, js, slack_band: float = 3e-5):
    """Opacity and edge slack at selected grid indices only."""
    js = np.asarray(js, dtype=np.int64)
    lo2, hi2 = windows(pl, 1.0 - slack_band)
    kap = np.zeros(len(js)); sl = np.zeros(len(js))
    live = np.nonzero(hi2 >= lo2)[0]
    for n, j in enumerate(js):
        ii = live[(lo2[live] <= j) & (hi2[live] >= j)]
        if len(ii) == 0:
            continue
        e = ell(pl, ii, j)
        kap[n] = np.sum(e[e >= pl.t])
        sl[n] = np.sum(e[np.abs(e / pl.t - 1.0) <= slack_band])
    return kap, sl


def h_upper_bound(v, a):
    """An upper bound of H(v, a): splitting the convolution integral of H at |t| = |v|/2 gives
    H <= 4a / (sqrt(pi) v^2) + exp(-v^2 / 4) (and H <= H(0, a) <= 1 always)."""
    v = np.abs(np.asarray(v, dtype=np.float64))
    with np.errstate(divide="ignore"):
        b = 4.0 * a / (math.sqrt(math.pi) * v * v) + np.exp(-v * v / 4.0)
    return np.minimum(b, 1.0)


def kappa_at_chunked(lines, species_el, species_stage, el, T, P, grid, js, cut=1e-3, kc_factor=1e-2,
                     abund_scale=None, vturb=0.0, slack_band=3e-5, chunk=2_000_000):
    """kappa_at for line lists too large to prepare at once, in chunks of `chunk` lines: the same
    steps (populations; the line terms; kappa_c = kc_factor times the lower median of kappa0 over
    every line of the list, t = cut kappa_c; at each grid index of js the sum of ell over the
    lines with ell >= t there, and the edge slack).  A line takes part only if S times the upper
    bound of H at its smallest |v| over the sampled points reaches t (1 - slack_band), which no
    line that contributes or lies in the slack band can fail.  Returns (kappa, slack, kappa_c)."""
    js = np.asarray(js, dtype=np.int64)
    pop = physics.populations_eos(T, P, el, abund_scale) if hasattr(el, "n_stages") else \
        physics.populations(T, P, el, abund_scale)
    L = len(lines)
    lnk0 = np.empty(L)
    for i in range(0, L, chunk):
        sub = lines.subset(slice(i, min(i + chunk, L)))
        t_ = physics.line_terms(sub, species_el, species_stage, el, pop, vturb)
        lnk0[i:i + len(sub)] = np.log(t_.S * H(0.0, t_.a))
    kc = kc_factor * float(np.exp(np.partition(lnk0, (L - 1) // 2)[(L - 1) // 2]))
    del lnk0
    t = cut * kc
    thr = (1.0 - slack_band) * t
    lam_cm = grid_lambda_nm(grid.lam0_nm, grid.R, js) * 1e-7
    nu = C / lam_cm
    nu_lo, nu_hi = float(nu.min()), float(nu.max())
    kap = np.zeros(len(js))
    sl = np.zeros(len(js))
    for i in range(0, L, chunk):
        sub = lines.subset(slice(i, min(i + chunk, L)))
        tt = physics.line_terms(sub, species_el, species_stage, el, pop, vturb)
        # smallest |nu - nu0| over the sampled points is at least the distance to [nu_lo, nu_hi]
        dmin = np.maximum(np.maximum(nu_lo - tt.nu0, tt.nu0 - nu_hi), 0.0)
        keep = np.nonzero(tt.S * h_upper_bound(dmin / tt.dnuD, tt.a) >= thr)[0]
        for n, j in enumerate(js):
            v = (nu[n] - tt.nu0[keep]) / tt.dnuD[keep]
            e = tt.S[keep] * H(v, tt.a[keep])
            kap[n] += float(np.sum(e[e >= t]))
            sl[n] += float(np.sum(e[np.abs(e / t - 1.0) <= slack_band]))
    return kap, sl, kc
