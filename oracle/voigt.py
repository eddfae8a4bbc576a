"""Voigt function H(v, a) in FP64 (oracle; test infrastructure only).

H(v, a) = (a/pi) * integral exp(-t^2) / ((v - t)^2 + a^2) dt = Re w(v + i a),
the profile of Eq. (l_nu_line) with v = dnu/dnuD and a = gamma/(4 pi dnuD).
The Faddeeva function w(z) is taken from scipy.special.wofz (a library
primitive).  The GPU path uses a different, FP32 method.
"""
from __future__ import annotations

import numpy as np
from scipy.special import wofz


def H(v, a):
    v = np.asarray(v, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    return wofz(np.abs(v) + 1j * a).real


def H_upper_bound_v(a, r):
    """A v beyond which H(v, a) < r is guaranteed.

    Splitting the convolution integral at |t| = v/2 gives
    H(v, a) <= 4a/(sqrt(pi) v^2) + exp(-v^2/4); each term is <= r/2 when
    v >= max(sqrt(8a/(sqrt(pi) r)), 2 sqrt(ln(2/r))).
    """
    a = np.asarray(a, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    return np.maximum(np.sqrt(8.0 * a / (np.sqrt(np.pi) * r)), 2.0 * np.sqrt(np.log(np.maximum(2.0 / r, 1.0)))) + 1.0
