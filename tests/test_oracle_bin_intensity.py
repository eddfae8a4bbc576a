"""Pins of the oracle's bin intensities from a tabulated ODF (not gpu)."""
import math

import numpy as np
from scipy import integrate

from oracle import bin_intensity as bi
from oracle import spectrum as spc
from oracle.physics import C_LIGHT, H_PLANCK, K_BOLTZ

MUS = [1.0, 0.8, 0.6, 0.4, 0.2]
W12 = np.r_[np.full(9, 0.1), 0.05, 0.04, 0.01]


def axes(rng, nT=7, nP=5):
    lt = np.sort(rng.uniform(3.3, 5.3, nT))
    lp = np.sort(rng.uniform(-4.0, 8.0, nP))
    return lt, lp


def test_interpolation_reproduces_bilinear_functions():
    # a + b x + c y + d x y (x = log10 T, y = log10 P) is reproduced exactly inside the grid,
    # at the nodes, and at the clamped coordinates outside it
    rng = np.random.default_rng(1)
    lt, lp = axes(rng)
    a, b, c, d = 2.0, -0.7, 0.3, 0.11
    f = lambda x, y: a + b * x + c * y + d * x * y
    tab = f(lt[:, None], lp[None, :])
    for _ in range(200):
        x, y = rng.uniform(lt[0], lt[-1]), rng.uniform(lp[0], lp[-1])
        assert abs(bi.interpolate(tab, lt, lp, 10 ** x, 10 ** y) - f(x, y)) < 1e-12 * (1 + abs(f(x, y)))
    for i in range(len(lt)):
        for j in range(len(lp)):
            assert abs(bi.interpolate(tab, lt, lp, 10 ** lt[i], 10 ** lp[j]) - tab[i, j]) < 1e-12 * (1 + abs(tab[i, j]))
    x, y = lt[-1] + 0.5, lp[0] - 2.0
    assert abs(bi.interpolate(tab, lt, lp, 10 ** x, 10 ** y) - f(lt[-1], lp[0])) < 1e-12
    # vector-valued cells interpolate componentwise
    tab2 = np.stack([tab, 3 * tab], axis=-1)
    v = bi.interpolate(tab2, lt, lp, 10 ** 4.1, 10 ** 1.3)
    assert abs(v[1] - 3 * v[0]) < 1e-12 * abs(v[1])


def test_isothermal_atmosphere_gives_planck():
    # constant T: S is constant with depth and every sub-bin intensity equals B(lambda_c, T)
    rng = np.random.default_rng(2)
    lt, lp = axes(rng)
    K = 4
    odf = np.sort(10 ** rng.uniform(-3, 3, (len(lt), len(lp), K, 12)), axis=-1)
    kc = 10 ** rng.uniform(-2, 0, (len(lt), len(lp)))
    lam = np.array([150.0, 300.0, 551.0, 2200.0])
    D = 30
    m = 10 ** np.linspace(-5, 2, D)
    T = np.full(D, 7300.0)
    P = 10 ** np.linspace(-1, 6, D)
    I = bi.bin_intensity(odf, kc, lt, lp, lam, W12, m, T, P, MUS)
    B = spc.planck_lambda(lam * 1e-7, 7300.0)
    assert np.allclose(I, B[None, :], rtol=1e-12, atol=0)


def test_eddington_barbier_per_subbin():
    # a table constant over T-P and S = alpha + beta m (T chosen so that B(lambda_c, T) is
    # linear in m): sub-bin s sees tau = (kappa_c + kappa_s) m, so I_s = alpha + beta mu /
    # (kappa_c + kappa_s) and I_bin = alpha + beta mu sum_s w_s / (kappa_c + kappa_s)
    rng = np.random.default_rng(3)
    lt, lp = axes(rng, 3, 3)
    ks = np.sort(10 ** rng.uniform(-2, 2, 12))
    kc0 = 0.37
    odf = np.broadcast_to(ks, (3, 3, 1, 12)).copy()
    kc = np.full((3, 3), kc0)
    lam_nm = 420.0
    lam = lam_nm * 1e-7
    c1 = 2 * H_PLANCK * C_LIGHT ** 2 / lam ** 5
    c2 = H_PLANCK * C_LIGHT / (lam * K_BOLTZ)
    alpha = spc.planck_lambda(lam, 5000.0)
    beta = 0.8 * alpha
    m = np.r_[1e-14, 10 ** np.linspace(-6, 3, 80)]
    S = alpha + beta * m
    T = c2 / np.log1p(c1 / S)
    P = 10 ** np.linspace(0, 5, len(m))
    I = bi.bin_intensity(odf, kc, lt, lp, [lam_nm], W12, m, T, P, MUS)
    for q, mu in enumerate(MUS):
        expect = alpha + beta * mu * np.sum(W12 / (kc0 + ks))
        assert abs(I[q, 0] / expect - 1) < 1e-9


def quad_intensity(tau, S, mu):
    # I = integral_0^inf S~(tau) exp(-tau/mu) dtau/mu, S~ = S_0 above the first point,
    # piecewise linear between the points and continued linearly below the last one
    f = lambda t, a, b: (a + b * t) * math.exp(-t / mu) / mu
    tot = integrate.quad(f, 0.0, tau[0], args=(S[0], 0.0), epsabs=0, epsrel=1e-13)[0]
    for d in range(len(tau) - 1):
        b = (S[d + 1] - S[d]) / (tau[d + 1] - tau[d])
        tot += integrate.quad(f, tau[d], tau[d + 1], args=(S[d] - b * tau[d], b), epsabs=0, epsrel=1e-13)[0]
    b = (S[-1] - S[-2]) / (tau[-1] - tau[-2])
    tot += integrate.quad(f, tau[-1], np.inf, args=(S[-1] - b * tau[-1], b), epsabs=0, epsrel=1e-13)[0]
    return tot


def test_against_quadrature():
    # a random table, continuum and non-grey-like atmosphere: the bin intensity equals the
    # width-weighted sum of the integrals of S e^{-tau/mu} over the interpolated opacities
    rng = np.random.default_rng(4)
    lt, lp = axes(rng, 5, 4)
    K = 2
    odf = np.sort(10 ** rng.uniform(-2, 2, (len(lt), len(lp), K, 3)), axis=-1)
    kc = 10 ** rng.uniform(-2, -1, (len(lt), len(lp)))
    w = np.array([0.5, 0.3, 0.2])
    lam = np.array([380.0, 910.0])
    D = 12
    m = 10 ** np.linspace(-3, 2, D)
    T = 10 ** np.linspace(3.55, 4.2, D)
    P = 10 ** np.linspace(1.0, 6.0, D)
    I = bi.bin_intensity(odf, kc, lt, lp, lam, w, m, T, P, MUS)
    for k in range(K):
        S = spc.planck_lambda(lam[k] * 1e-7, T)
        for q, mu in enumerate(MUS):
            tot = 0.0
            for s in range(3):
                kap = np.array([bi.interpolate(odf[:, :, k, s], lt, lp, T[d], P[d]) +
                                bi.interpolate(kc, lt, lp, T[d], P[d]) for d in range(D)])
                tau = spc.optical_depth(kap, m)
                tot += w[s] * quad_intensity(tau, S, mu)
            assert abs(I[q, k] / tot - 1) < 1e-9, (k, mu, I[q, k], tot)
