"""Opacity distribution function (ODF) step means in FP64 (oracle; test infrastructure only).

Sect. 2.3 and App. E of the paper: the high-resolution opacity of each
wavelength interval (bin) is sorted in ascending order, the sorted profile is
split into sub-bins whose widths are given fractions of the bin, and each
sub-bin is replaced by its mean.  Readings:
  * every grid point of an interval carries equal weight (on a log-lambda grid
    the points are equally spaced in ln lambda);
  * sub-bin boundaries fall at cumulative width fractions c_s = w_1 + ... + w_s,
    accumulated left to right in FP64, with c_n forced to 1; a boundary that falls
    inside a point's rank cell splits that point fractionally: with the sorted
    values x_(0) <= ... <= x_(n-1) and x(u) = x_(floor(u n)),
    m_s = (1/w_s) * integral_{c_{s-1}}^{c_s} x(u) du;
  * "arithmetic" is the plain mean above; "geometric" is exp of the same
    integral of ln x (the DFSYNTHE default, Sect. 2.3).
"""
from __future__ import annotations

import math

import numpy as np


def cumulative_widths(widths) -> np.ndarray:
    w = [float(x) for x in widths]
    c = [0.0]
    acc = 0.0
    for x in w:
        acc = acc + x
        c.append(acc)
    c[-1] = 1.0
    return np.array(c)


def step_means_sorted(xs: np.ndarray, widths) -> np.ndarray:
    """Step means of one interval whose values are already sorted ascending."""
    n = len(xs)
    c = cumulative_widths(widths)
    w = np.asarray(widths, dtype=np.float64)
    pref = np.concatenate([[0.0], np.cumsum(xs.astype(np.float64))])

    def F(u):  # integral_0^{u} x(t) dt in rank units (t in [0, n])
        k = int(math.floor(u))
        if k >= n:
            return pref[n]
        return pref[k] + (u - k) * float(xs[k])

    out = np.empty(len(w))
    for s in range(len(w)):
        out[s] = (F(c[s + 1] * n) - F(c[s] * n)) / (w[s] * n)
    return out


def geom_step_means_sorted(xs: np.ndarray, widths) -> np.ndarray:
    """Geometric step means exp((1/w_s) integral ln x(u) du) of sorted non-negative values.

    A step whose rank range overlaps the zero values (with positive length) has geometric
    mean 0 (the geometric mean of a set containing 0); otherwise the integral runs over
    positive values only.
    """
    n = len(xs)
    z = int(np.count_nonzero(xs == 0))
    c = cumulative_widths(widths)
    w = np.asarray(widths, dtype=np.float64)
    lx = np.log(xs[z:].astype(np.float64))
    pref = np.concatenate([[0.0], np.cumsum(lx)])

    def F(u):  # integral of ln x over ranks [z, u) for u >= z
        k = int(math.floor(u))
        if k >= n:
            return pref[n - z]
        return pref[k - z] + (u - k) * float(lx[k - z])

    out = np.empty(len(w))
    for s in range(len(w)):
        a, b = c[s] * n, c[s + 1] * n
        out[s] = 0.0 if a < z else math.exp((F(b) - F(a)) / (w[s] * n))
    return out


def odf(kappa: np.ndarray, bounds, widths, mean: str = "arith") -> np.ndarray:
    """ODF table of one opacity array: [K][n_steps] FP64.

    kappa: [N] opacity (any float dtype; compared and summed in FP64).
    bounds: [K+1] integer interval bounds (interval k = [b_k, b_{k+1})).
    """
    b = np.asarray(bounds, dtype=np.int64)
    K = len(b) - 1
    out = np.empty((K, len(widths)))
    for k in range(K):
        xs = np.sort(np.asarray(kappa[b[k]:b[k + 1]], dtype=np.float64))
        if mean == "geom":
            out[k] = geom_step_means_sorted(xs, widths)
        else:
            out[k] = step_means_sorted(xs, widths)
    return out
