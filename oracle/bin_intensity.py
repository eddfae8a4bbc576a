"""Bin intensities from a tabulated ODF (module III via ODF tables), FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sect. 2.3 (the ODF approach, I_ODF = sum over sub-bins of I_s times the sub-bin width)
and App. E (the bin intensity at the bin centre lambda_c):

    I_bin,i(mu) = sum_s w_s,i I_lambda_c(kappa_tot,s,i; mu),

where I_lambda_c is the emergent intensity of the formal solution (oracle.spectrum) of the
atmosphere with, at every depth, kappa_tot,s,i = kappa_c + kappa_s,i: the continuum plus the
mean line opacity of sub-bin s of bin i.  The table holds kappa_s,i on a T-P grid for one
composition; for an atmosphere point it is interpolated linearly on that grid (Sect. 2.3).

Readings (the paper does not fix them):
  * the interpolation is bilinear in (log10 T, log10 P), the coordinates in which the
    table grid is spaced, applied to the opacities themselves; outside the grid the
    coordinates are clamped to its edges;
  * the continuum opacity is tabulated with the ODF (one value per T-P point, as the
    synthesis returns it) and interpolated the same way;
  * S = B_lambda(T) at the bin centre (LTE, no scattering), the same formal solution as the
    spectrum path.
"""
from __future__ import annotations

import numpy as np

from . import spectrum


def cell_weights(axis, x):
    """Index i and fraction f of x on a strictly increasing axis, clamped to the axis ends:
    x = (1 - f) axis[i] + f axis[i + 1] with 0 <= i <= len(axis) - 2 and 0 <= f <= 1
    (an axis of one value gives i = 0, f = 0)."""
    axis = np.asarray(axis, dtype=np.float64)
    n = len(axis)
    if n == 1:
        return 0, 0.0
    if x <= axis[0]:
        return 0, 0.0
    if x >= axis[-1]:
        return n - 2, 1.0
    i = int(np.searchsorted(axis, x, side="right")) - 1
    i = min(max(i, 0), n - 2)
    return i, (x - axis[i]) / (axis[i + 1] - axis[i])


def interpolate(table, log10_T, log10_P, T, P):
    """Bilinear interpolation of table[nT][nP][...] at (log10 T, log10 P)."""
    table = np.asarray(table, dtype=np.float64)
    iT, fT = cell_weights(log10_T, np.log10(T))
    iP, fP = cell_weights(log10_P, np.log10(P))
    jT = min(iT + 1, table.shape[0] - 1)
    jP = min(iP + 1, table.shape[1] - 1)
    return ((1 - fT) * (1 - fP) * table[iT, iP] + (1 - fT) * fP * table[iT, jP] +
            fT * (1 - fP) * table[jT, iP] + fT * fP * table[jT, jP])


def bin_intensity(odf, kappa_c, log10_T, log10_P, lam_c_nm, widths, m, T, P, mus):
    """I[n_mu][K] of one atmosphere (column mass m, T, P per depth, top to bottom).

    odf[nT][nP][K][n_steps]: sub-bin mean line opacities on the T-P grid;
    kappa_c[nT][nP]: continuum opacity on the same grid; lam_c_nm[K]: bin centres;
    widths[n_steps]: sub-bin widths (fractions of the bin, summing to 1)."""
    odf = np.asarray(odf, dtype=np.float64)
    kappa_c = np.asarray(kappa_c, dtype=np.float64)
    D = len(m)
    K, ns = odf.shape[2], odf.shape[3]
    kap_s = np.empty((D, K, ns))
    kap_c = np.empty(D)
    for d in range(D):
        kap_s[d] = interpolate(odf, log10_T, log10_P, T[d], P[d])
        kap_c[d] = interpolate(kappa_c, log10_T, log10_P, T[d], P[d])
    out = np.zeros((len(mus), K))
    for k in range(K):
        S = spectrum.planck_lambda(lam_c_nm[k] * 1e-7, np.asarray(T, dtype=np.float64))
        for s in range(ns):
            tau = spectrum.optical_depth(kap_c + kap_s[:, k, s], m)
            for q, mu in enumerate(mus):
                out[q, k] += widths[s] * spectrum.formal_solution(tau, S, mu)
    return out
