"""Pins of the oracle's closed-form continuum (not gpu): textbook constants, edges and scaling laws."""
import json
import math
import os

import numpy as np

import workloads as wl
from oracle import continuum as co
from oracle import physics as ph

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))


def pop_at(T, P):
    return ph.populations(T, P, wl.elements(5))


def test_constants_against_textbook_values():
    for key, val in [("kramers_bound_free_cgs", co.kramers_bf_constant()),
                     ("kramers_free_free_cgs", co.kramers_ff_constant()),
                     ("thomson_cross_section_cm2", co.SIGMA_T)]:
        g = GOLD[key]
        assert abs(val / g["value"] - 1) < g["rtol"], (key, val)


def test_electron_scattering_alone():
    pop = pop_at(9000.0, 1e4)
    lam = np.array([50.0, 300.0, 2000.0])
    k = co.kappa_c(lam, pop, sources=("elec",))
    assert np.allclose(k, pop.n_e * 6.6524587321e-25 / pop.rho, rtol=1e-14)


def test_lyman_and_balmer_edges():
    # bound-free of level n switches on at lambda = lambda_L n^2: just shortward of the Lyman and
    # Balmer edges the H I bound-free opacity jumps up
    pop = pop_at(6000.0, 1e4)
    edge = ph.H_PLANCK * ph.C_LIGHT / (co.CHI_H_EV * ph.EV) * 1e7
    g = GOLD["lyman_edge_nm"]
    assert abs(edge / g["value"] - 1) < g["rtol"]
    for n in (1, 2):
        e = edge * n * n
        lo, hi = co.kappa_c([e * (1 - 1e-6)], pop, sources=("bf",))[0], co.kappa_c([e * (1 + 1e-6)], pop, sources=("bf",))[0]
        assert lo > 2 * hi, (n, lo, hi)
    # no level at all longward of the last level's edge
    far = edge * (co.N_LEVELS ** 2) * 1.01
    assert co.kappa_c([far], pop, sources=("bf",))[0] == 0.0


def test_nu_cubed_scaling_and_stimulated_emission():
    # between the Lyman and Balmer edges only n = 1 contributes: alpha / (1 - e^{-h nu/kT}) scales as nu^-3;
    # free-free scales as nu^-3 times the same factor
    pop = pop_at(12000.0, 1e3)
    h, k, c = ph.H_PLANCK, ph.K_BOLTZ, ph.C_LIGHT
    for src in (("bf",), ("ff",)):
        lam = np.array([100.0, 200.0]) if src == ("bf",) else np.array([400.0, 800.0])
        a = co.kappa_c(lam, pop, sources=src)
        nu = c / (lam * 1e-7)
        stim = -np.expm1(-h * nu / (k * pop.T))
        r = (a / stim) * nu ** 3
        assert abs(r[1] / r[0] - 1) < 1e-12, src
    # at h nu / kT = ln 2 the stimulated-emission factor is 1/2
    lam_half = h * c / (k * pop.T * math.log(2.0)) * 1e7
    a = co.kappa_c([lam_half], pop, sources=("ff",))[0]
    nu = c / (lam_half * 1e-7)
    full = co.kramers_ff_constant() * pop.n_e * pop.n_stage[0, 1] / (math.sqrt(pop.T) * nu ** 3) / pop.rho
    assert abs(a / full - 0.5) < 1e-12


def test_rayleigh_series():
    # sigma_R lambda^4 tends to 5.799e-13 cm^2 A^4 at long wavelengths; the series is held at 1300 A below
    for L in (1e6, 3e6):
        s = co.rayleigh_hi(L * 1e-8)
        assert abs(s * L ** 4 / 5.799e-13 - 1) < 3e-6 * (1e6 / L) ** 2
    assert co.rayleigh_hi(1000e-8) == co.rayleigh_hi(1300e-8)
    pop = pop_at(5000.0, 1e5)
    k = co.kappa_c([500.0], pop, sources=("ray",))[0]
    assert abs(k / (pop.n_HI * co.rayleigh_hi(500e-7) / pop.rho) - 1) < 1e-14


def test_sources_add():
    pop = pop_at(7000.0, 1e4)
    lam = np.exp(np.linspace(math.log(30.0), math.log(5000.0), 50))
    tot = co.kappa_c(lam, pop)
    parts = sum(co.kappa_c(lam, pop, sources=(s,)) for s in ("elec", "bf", "ff", "ray"))
    assert np.allclose(tot, parts, rtol=1e-14)
