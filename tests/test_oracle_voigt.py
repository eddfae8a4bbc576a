"""Pins of the oracle's Voigt function against closed forms and quadrature (not gpu)."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle.voigt import H, H_upper_bound_v

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))


def test_core_equals_erfcx():
    # H(0, a) = erfcx(a) = exp(a^2) erfc(a); computed with Python's math library (independent of scipy)
    for a in [1e-8, 1e-3, 0.1, 0.5, 1.0, 2.0, 5.0, 20.0]:
        ref = math.exp(a * a) * math.erfc(a)
        assert abs(H(0.0, a) / ref - 1) < 1e-10
    g = GOLD["erfcx_1"]
    assert abs(H(0.0, 1.0) / g["value"] - 1) < g["rtol"]


def test_gaussian_limit():
    v = np.linspace(0, 6, 61)
    # the Lorentzian part a/(sqrt(pi) v^2) must stay far below exp(-v^2): take a = 1e-30
    assert np.allclose(H(v, 1e-30), np.exp(-v * v), rtol=1e-10, atol=0)


def test_lorentzian_asymptote():
    # w(z) ~ (i / (sqrt(pi) z)) (1 + 1/(2 z^2) + 3/(4 z^4) + 15/(8 z^6)) for |z| -> inf, Im z > 0
    for v in [30.0, 100.0, 1e3, 1e5]:
        for a in [1e-6, 1e-2, 1.0, 10.0]:
            z = complex(v, a)
            w = 1j / (math.sqrt(math.pi) * z) * (1 + 1 / (2 * z ** 2) + 3 / (4 * z ** 4) + 15 / (8 * z ** 6))
            assert abs(H(v, a) / w.real - 1) < 1e-9


def test_normalisation():
    # integral of H over v equals sqrt(pi); tails beyond |v| = V add 2a/(sqrt(pi) V) to leading order
    for a in [1e-3, 0.1, 1.0, 3.0]:
        V = 400.0
        val, _ = integrate.quad(lambda v: H(v, a), 0, V, points=[0, 1, 2, 4, 8], limit=500, epsabs=0, epsrel=1e-11)
        tail = a / (math.sqrt(math.pi) * V) * (1 + 1 / (2 * V * V))
        assert abs(2 * (val + tail) / math.sqrt(math.pi) - 1) < 1e-7


def test_even_and_monotone():
    v = np.linspace(0, 50, 2001)
    for a in [1e-10, 1e-3, 0.3, 2.0, 30.0]:
        h = H(v, a)
        assert np.array_equal(h, H(-v, a))
        assert np.all(np.diff(h) <= 0)


def test_defining_integral():
    # H(v, a) = (1/pi) * integral_{-pi/2}^{pi/2} exp(-(v + a tan th)^2) dth  (t = v + a tan th in the convolution)
    for v, a in [(0.3, 0.05), (1.7, 0.5), (3.0, 1e-2), (4.0, 2.0), (10.0, 0.3), (2.0, 10.0)]:
        th0 = math.atan(-v / a)
        f = lambda th: math.exp(-(v + a * math.tan(th)) ** 2)
        val, _ = integrate.quad(f, -math.pi / 2, math.pi / 2, points=[th0], limit=400, epsabs=0, epsrel=1e-12)
        assert abs(H(v, a) / (val / math.pi) - 1) < 1e-9


def test_upper_bound():
    rng = np.random.default_rng(0)
    a = 10 ** rng.uniform(-12, 3, 2000)
    r = 10 ** rng.uniform(-20, -0.5, 2000) * H(0.0, a)
    vb = H_upper_bound_v(a, r)
    assert np.all(H(vb, a) < r)
