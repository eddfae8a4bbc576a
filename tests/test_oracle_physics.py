"""Pins of oracle populations and line terms (not gpu)."""
import json
import math
import os

import numpy as np
from scipy import integrate

import workloads as wl
from oracle import physics as ph
from oracle.voigt import H

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))


def hydrogen_only():
    return wl.Elements(["H"], np.array([1.008]), np.array([13.598]), np.array([2.0]), np.array([1.0]), np.array([12.0]))


def test_pure_hydrogen_closed_form():
    # x = n_e/n_nuc; P = (1 + x) n_nuc kT and x^2/(1-x) = Phi/n_nuc give x = sqrt(Phi kT/(P + Phi kT))
    el = hydrogen_only()
    k = 1.380649e-16
    for T in [3000.0, 6000.0, 9000.0, 15000.0, 50000.0]:
        for P in [1e-2, 1e2, 1e4, 1e7]:
            phi = 2 * 1.0 / 2.0 * (2 * math.pi * 9.1093837015e-28 * k * T / 6.62607015e-27 ** 2) ** 1.5 \
                * math.exp(-13.598 * 1.602176634e-12 / (k * T))
            x = math.sqrt(phi * k * T / (P + phi * k * T))
            pop = ph.populations(T, P, el)
            assert abs(pop.n_e / pop.n_nuc / x - 1) < 1e-11, (T, P)


def test_conservation():
    el = wl.elements(15)
    rng = np.random.default_rng(1)
    for T, P in zip(np.exp(rng.uniform(math.log(2000), math.log(2e5), 20)), 10 ** rng.uniform(-4, 8, 20)):
        pop = ph.populations(T, P, el, abund_scale=np.exp(rng.uniform(-4, 2, el.n)))
        assert abs(pop.n_stage[:, 1].sum() / pop.n_e - 1) < 1e-12          # charge
        assert abs((pop.n_nuc + pop.n_e) * ph.K_BOLTZ * T / P - 1) < 1e-12  # particles
        assert np.all(pop.n_stage >= 0)


def one_line(lam_nm, loggf, E, sp, lgR=-8.0, lgS=-8.0, lgW=-8.0):
    f32 = lambda x: np.array([x], dtype=np.float32)
    return wl.LineList(np.array([lam_nm]), f32(loggf), f32(E), np.array([sp], dtype=np.int32), f32(lgR), f32(lgS), f32(lgW))


def test_integrated_cross_section():
    # integral over nu of ell equals (pi e^2/(m_e c)) g f (N/U)/rho e^{-E/kT}(1-e^{-h nu/kT}); with E = 0 and
    # h nu/kT = 36 the last two factors are 1, so rho * int ell dnu / (g f N/U) must equal 0.02654 cm^2 Hz
    el = wl.elements(5); se, ss = wl.species_table(5)
    pop = ph.populations(4000.0, 1e4, el)
    L = one_line(100.0, 0.0, 0.0, 0)
    t = ph.line_terms(L, se, ss, el, pop)
    S, a, dnu = t.S[0], t.a[0], t.dnuD[0]
    val, _ = integrate.quad(lambda v: H(v, a), 0, np.inf, limit=400, epsabs=0, epsrel=1e-10)
    integral = 2 * val * S * dnu            # int ell dnu = S dnuD int H dv
    sigma = integral * pop.rho / pop.NU[se[0], ss[0]]
    g = GOLD["classical_oscillator_cross_section_cm2_Hz"]
    assert abs(sigma / g["value"] - 1) < g["rtol"]


def test_boltzmann_factor():
    el = wl.elements(5); se, ss = wl.species_table(5)
    pop = ph.populations(6000.0, 1e4, el)
    t1 = ph.line_terms(one_line(350.0, -2.0, 1.0, 2), se, ss, el, pop)
    t2 = ph.line_terms(one_line(350.0, -2.0, 3.5, 2), se, ss, el, pop)
    kB = GOLD["boltzmann_eV_per_K"]["value"]
    assert abs(t2.S[0] / t1.S[0] / math.exp(-2.5 / (kB * 6000.0)) - 1) < 1e-6


def test_doppler_width_hydrogen():
    # a line of a hydrogen-mass species: dnuD/nu0 = sqrt(2kT/m_H)/c
    el = wl.Elements(["H", "He", "X"], np.array([1.008, 4.0026, 1.008]), np.array([13.598, 24.587, 13.598]),
                     np.array([2.0, 1.0, 2.0]), np.array([1.0, 2.0, 1.0]), np.array([12.0, 10.93, 6.0]))
    se, ss = np.array([2, 2], dtype=np.int32), np.array([0, 1], dtype=np.int32)
    pop = ph.populations(1e4, 1e4, el)
    t = ph.line_terms(one_line(500.0, 0.0, 0.0, 0), se, ss, el, pop)
    vth = t.dnuD[0] / t.nu0[0] * 2.99792458e10 / 1e5
    g = GOLD["hydrogen_thermal_speed_1e4K_km_s"]
    assert abs(vth / g["value"] - 1) < g["rtol"]
    # thermal width scales as sqrt(T)
    pop4 = ph.populations(4e4, 1e4, el)
    t4 = ph.line_terms(one_line(500.0, 0.0, 0.0, 0), se, ss, el, pop4)
    assert abs(t4.dnuD[0] / t.dnuD[0] - 2.0) < 1e-12


def test_microturbulence():
    # App. E: the Doppler width takes the micro-turbulent speed in quadrature with the thermal
    # one (for hydrogen mass at 1e4 K, 12.85 km/s and 5 km/s give 13.79 km/s), and the
    # integrated cross-section, S dnuD int H dv, does not depend on it
    el = wl.Elements(["H", "He", "X"], np.array([1.008, 4.0026, 1.008]), np.array([13.598, 24.587, 13.598]),
                     np.array([2.0, 1.0, 2.0]), np.array([1.0, 2.0, 1.0]), np.array([12.0, 10.93, 6.0]))
    se, ss = np.array([2, 2], dtype=np.int32), np.array([0, 1], dtype=np.int32)
    pop = ph.populations(1e4, 1e4, el)
    L = one_line(500.0, 0.0, 0.0, 0)
    g = GOLD["hydrogen_thermal_speed_1e4K_km_s"]
    t0 = ph.line_terms(L, se, ss, el, pop, vturb=0.0)
    t5 = ph.line_terms(L, se, ss, el, pop, vturb=5e5)
    v5 = t5.dnuD[0] / t5.nu0[0] * 2.99792458e10 / 1e5
    assert abs(v5 / math.hypot(g["value"], 5.0) - 1) < g["rtol"]
    ints = []
    for t in (t0, t5):
        val, _ = integrate.quad(lambda v: H(v, t.a[0]), 0, np.inf, limit=400, epsabs=0, epsrel=1e-10)
        ints.append(2 * val * t.S[0] * t.dnuD[0])
    assert abs(ints[1] / ints[0] - 1) < 1e-8


def test_lorentz_width():
    # for a >> 1 the profile is Lorentzian with FWHM in frequency gamma/(2 pi): ell(dnu = gamma/(4 pi)) = ell(0)/2
    el = wl.elements(5); se, ss = wl.species_table(5)
    pop = ph.populations(6000.0, 1e8, el)
    L = one_line(350.0, -2.0, 1.0, 0, lgR=15.0, lgS=-30.0, lgW=-30.0)
    t = ph.line_terms(L, se, ss, el, pop)
    a = t.a[0]
    assert a > 100
    v_half = t.gamma[0] / (4 * math.pi) / t.dnuD[0]
    assert abs(H(v_half, a) / H(0.0, a) - 0.5) < 2 / a ** 2


def test_density_pure_hydrogen():
    # rho = n_nuc * m_H with the textbook hydrogen-atom mass 1.6735575e-24 g (the table carries the rounded weight 1.008 amu: 1.6e-4)
    pop = ph.populations(8000.0, 1e4, hydrogen_only())
    assert abs(pop.rho / (pop.n_nuc * 1.6735575e-24) - 1) < 3e-4
    # stage I of hydrogen has U = 2: N/U = n_HI / 2
    assert abs(pop.NU[0, 0] / (pop.n_HI / 2.0) - 1) < 1e-15


def test_stimulated_emission_and_lambda_scaling():
    # at h nu/kT = ln 2 the stimulated-emission factor is 1/2; S also scales as 1/dnuD, i.e. as lambda
    el = wl.elements(5); se, ss = wl.species_table(5)
    T = 6000.0
    pop = ph.populations(T, 1e4, el)
    lam_half = 6.62607015e-27 * 2.99792458e10 / (1.380649e-16 * T * math.log(2.0)) * 1e7  # nm
    lam_one = 50.0  # h nu/kT = 48
    s_half = ph.line_terms(one_line(lam_half, -1.0, 2.0, 4), se, ss, el, pop).S[0]
    s_one = ph.line_terms(one_line(lam_one, -1.0, 2.0, 4), se, ss, el, pop).S[0]
    assert abs(s_half / s_one / (0.5 * lam_half / lam_one) - 1) < 1e-12


def test_pressure_broadening_perturbers():
    # Stark width scales with n_e and van der Waals width with n_HI: FWHM = 10^lg * n / (2 pi)
    el = wl.elements(5); se, ss = wl.species_table(5)
    pop = ph.populations(9000.0, 1e8, el)
    tS = ph.line_terms(one_line(350.0, -2.0, 1.0, 0, lgR=-30.0, lgS=-2.0, lgW=-30.0), se, ss, el, pop)
    tW = ph.line_terms(one_line(350.0, -2.0, 1.0, 0, lgR=-30.0, lgS=-30.0, lgW=-2.0), se, ss, el, pop)
    assert abs(tS.gamma[0] / (1e-2 * pop.n_e) - 1) < 1e-6
    assert abs(tW.gamma[0] / (1e-2 * pop.n_HI) - 1) < 1e-6
    assert abs(tS.a[0] * 4 * math.pi * tS.dnuD[0] / tS.gamma[0] - 1) < 1e-14


# ---- multi-stage equation of state (App. A): Newton-Raphson on the neutral and electron densities

def two_stage_table(el):
    # the reduced element table as a two-stage table with constant partition functions
    n = el.n
    chi = np.zeros((n, 4)); chi[:, 0] = el.chi_eV
    lnU = np.zeros((n, 5, 3)); lnU[:, 0, 0] = np.log(el.U1); lnU[:, 1, 0] = np.log(el.U2)
    return wl.EosTable(el.symbol, el.mass_amu, el.log_eps, np.full(n, 2, dtype=np.int32), chi, lnU)


def test_eos_two_stages_equal_the_single_ionisation_balance():
    # stages I-II with fixed U: the Newton solution equals the bisection of the single-ionisation
    # charge balance (itself pinned by the pure-hydrogen closed form above)
    el = wl.elements(15)
    tab = two_stage_table(el)
    rng = np.random.default_rng(3)
    for T, P in zip(np.exp(rng.uniform(math.log(2000), math.log(2e5), 25)), 10 ** rng.uniform(-4, 8, 25)):
        ab = np.exp(rng.uniform(-4, 2, el.n))
        a, b = ph.populations(T, P, el, ab), ph.populations_eos(T, P, tab, ab)
        assert abs(b.n_e / a.n_e - 1) < 1e-11, (T, P)
        assert np.allclose(b.NU[:, :2], a.NU, rtol=1e-10, atol=0)
        assert abs(b.rho / a.rho - 1) < 1e-12 and abs(b.n_HI / a.n_HI - 1) < 1e-10


def test_eos_pure_hydrogen_closed_form():
    el = hydrogen_only()
    tab = two_stage_table(el)
    k = 1.380649e-16
    for T in [3000.0, 9000.0, 50000.0]:
        for P in [1e-2, 1e4, 1e7]:
            phi = (2 * math.pi * 9.1093837015e-28 * k * T / 6.62607015e-27 ** 2) ** 1.5 \
                * math.exp(-13.598 * 1.602176634e-12 / (k * T))
            x = math.sqrt(phi * k * T / (P + phi * k * T))
            pop = ph.populations_eos(T, P, tab)
            assert abs(pop.n_e / pop.n_nuc / x - 1) < 1e-11, (T, P)


def test_eos_pure_hydrogen_temperature_dependent_partition_function():
    # pure hydrogen whose neutral stage has the table's partition function ln U_I = c0 + c1 x + c2 x^2,
    # x = ln(T / 5040 K), and U_II = 1: the ionised fraction is the pure-hydrogen closed form with
    # Phi = 2 (U_II / U_I(T)) (2 pi m_e k T / h^2)^{3/2} e^{-chi/kT}, and N/U of stage I is n_HI / U_I(T)
    c0, c1, c2 = 0.7, 0.3, 0.05
    lnU = np.zeros((1, 5, 3))
    lnU[0, 0] = [c0, c1, c2]
    tab = wl.EosTable(["H"], np.array([1.008]), np.array([12.0]), np.array([2], dtype=np.int32),
                      np.array([[13.598, 0.0, 0.0, 0.0]]), lnU)
    k, eV = 1.380649e-16, 1.602176634e-12
    for T in [3000.0, 5040.0, 9000.0, 20000.0, 50000.0]:
        x = math.log(T / 5040.0)
        U1 = math.exp(c0 + c1 * x + c2 * x * x)
        for P in [1e-2, 1e4, 1e7]:
            phi = 2 * 1.0 / U1 * (2 * math.pi * 9.1093837015e-28 * k * T / 6.62607015e-27 ** 2) ** 1.5 \
                * math.exp(-13.598 * eV / (k * T))
            xi = math.sqrt(phi * k * T / (P + phi * k * T))
            pop = ph.populations_eos(T, P, tab)
            assert abs(pop.n_e / pop.n_nuc / xi - 1) < 1e-11, (T, P)
            assert abs(pop.NU[0, 0] / (pop.n_HI / U1) - 1) < 1e-12, (T, P)


def test_eos_helium_three_stages_cubic():
    # pure helium with stages I-III and fixed U: with y = n_e / n_tot, a = Phi_0 / n_tot and
    # b = Phi_1 / n_tot, charge and particle conservation give y^3 + 2a y^2 + (3ab - a) y - 2ab = 0,
    # whose single positive root (one sign change) comes from numpy.roots
    tab = wl.EosTable(["He"], np.array([4.0026]), np.array([12.0]), np.array([3], dtype=np.int32),
                      np.array([[24.587, 54.418, 0.0, 0.0]]), np.zeros((1, 5, 3)))
    tab.lnU[0, :3, 0] = np.log([1.0, 2.0, 1.0])
    k, eV = 1.380649e-16, 1.602176634e-12
    for T in [8000.0, 20000.0, 40000.0, 100000.0]:
        for P in [1e-2, 1e2, 1e6]:
            s = (2 * math.pi * 9.1093837015e-28 * k * T / 6.62607015e-27 ** 2) ** 1.5
            n_tot = P / (k * T)
            a = 2 * 2.0 / 1.0 * s * math.exp(-24.587 * eV / (k * T)) / n_tot
            b = 2 * 1.0 / 2.0 * s * math.exp(-54.418 * eV / (k * T)) / n_tot
            r = np.roots([1.0, 2 * a, 3 * a * b - a, -2 * a * b])
            y = float(max(z.real for z in r if abs(z.imag) < 1e-12 * abs(z) and z.real > 0))
            pop = ph.populations_eos(T, P, tab)
            assert abs(pop.n_e / n_tot / y - 1) < 1e-8, (T, P, pop.n_e / n_tot, y)


def test_eos_saha_ratios_and_conservation():
    # temperature-dependent partition functions, stages up to V: every adjacent pair of stages
    # satisfies the Saha-Boltzmann ratio, and charge, particles and each element's nuclei are conserved
    tab = wl.eos_table(15)
    rng = np.random.default_rng(7)
    k, eV = ph.K_BOLTZ, ph.EV
    for T, P in zip(np.exp(rng.uniform(math.log(2000), math.log(2e5), 30)), 10 ** rng.uniform(-4, 8, 30)):
        ab = np.exp(rng.uniform(-3, 1, tab.n))
        pop = ph.populations_eos(T, P, tab, ab)
        U = ph.partition_functions(tab, T)
        s = (2 * math.pi * ph.M_ELECTRON * k * T / ph.H_PLANCK ** 2) ** 1.5
        for e in range(tab.n):
            for j in range(tab.n_stages[e] - 1):
                lo, hi = pop.n_stage[e, j], pop.n_stage[e, j + 1]
                if lo > 1e-280 and hi > 1e-280:
                    phi = 2 * U[e, j + 1] / U[e, j] * s * math.exp(-tab.chi_eV[e, j] * eV / (k * T))
                    assert abs(hi * pop.n_e / lo / phi - 1) < 1e-10, (T, P, e, j)
        q = (pop.n_stage * np.arange(5)[None, :]).sum()
        assert abs(q / pop.n_e - 1) < 1e-12
        assert abs((pop.n_nuc + pop.n_e) * k * T / P - 1) < 1e-12
        eps = 10.0 ** (tab.log_eps - 12.0) * ab
        assert np.allclose(pop.n_stage.sum(axis=1), eps / eps.sum() * pop.n_nuc, rtol=1e-12, atol=0)
        assert np.all(pop.n_stage >= 0) and np.all(pop.n_stage[np.arange(5)[None, :] >= tab.n_stages[:, None]] == 0)


def test_eos_partition_function_at_reference_temperature():
    # x = ln(T / 5040 K) vanishes at 5040 K: U_j = exp(c0) there; U grows with T where c1, c2 >= 0
    tab = wl.eos_table(15)
    U = ph.partition_functions(tab, 5040.0)
    for e in range(tab.n):
        assert np.allclose(U[e, :tab.n_stages[e]], np.exp(tab.lnU[e, :tab.n_stages[e], 0]), rtol=1e-15)
    assert np.all(ph.partition_functions(tab, 20000.0) >= U)
