"""The oracle's pins catch plausible mistakes (not gpu).

Each case plants one mistake in the oracle, on the CPU, for the duration of the test: a dropped
term, a wrong sign, factor or index, a transposed order. It does so by replacing one oracle
function or constant. At least one of the pins chosen for that mistake must then fail. The
pins are the tests of `test_oracle_*.py`, called unchanged.
"""
import dataclasses
import math

import numpy as np
import pytest

import test_oracle_bin_intensity as t_bi
import test_oracle_continuum as t_co
import test_oracle_odf as t_odf
import test_oracle_physics as t_ph
import test_oracle_spectrum as t_sp
import test_oracle_synthesis as t_sy
import test_oracle_voigt as t_v
from oracle import bin_intensity as bi
from oracle import continuum as co
from oracle import odf as od
from oracle import physics as ph
from oracle import spectrum as spc
from oracle import synthesis as sy
from oracle import voigt

# the oracle's own functions, taken before any case replaces them
_H = voigt.H
_line_terms = ph.line_terms
_cum_widths = od.cumulative_widths
_step_means = od.step_means_sorted
_planck = spc.planck_lambda
_formal = spc.formal_solution
_windows = sy.windows
_grid_size = sy.grid_size
_rayleigh = co.rayleigh_hi
_cell_weights = bi.cell_weights


def _bound_without_8(a, r):
    # the window bound with its Lorentz term sqrt(8a / (sqrt(pi) r)) read as sqrt(a / (sqrt(pi) r))
    a = np.asarray(a, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    return np.maximum(np.sqrt(a / (math.sqrt(math.pi) * r)), 2.0 * np.sqrt(np.maximum(np.log(2.0 / r), 0.0)))


def _terms(change):
    """line_terms with `change(terms, lines, pop)` applied to its result."""
    def f(lines, species_el, species_stage, el, pop, vturb=0.0):
        return change(_line_terms(lines, species_el, species_stage, el, pop, vturb), lines, pop)
    return f


def _saha_no_three_halves(T, chi_eV, U1, U2):
    # the (2 pi m_e k T / h^2) factor without its 3/2 power
    return (2.0 * U2 / U1) * (2.0 * math.pi * ph.M_ELECTRON * ph.K_BOLTZ * T / ph.H_PLANCK ** 2) \
        * np.exp(-chi_eV / (ph.K_EV * T))


def _formal_constant_source_layers(tau, S, mu):
    # the formal solution with the source taken constant in each layer (linear term dropped)
    tau = np.asarray(tau, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    D = len(tau)
    I = S[D - 1] + mu * (S[D - 1] - S[D - 2]) / (tau[D - 1] - tau[D - 2])
    for d in range(D - 2, -1, -1):
        ex = math.exp(-(tau[d + 1] - tau[d]) / mu)
        I = I * ex + S[d] * (1.0 - ex)
    ex = math.exp(-tau[0] / mu)
    return I * ex + S[0] * (1.0 - ex)


def _formal_mu_ignored(tau, S, mu):
    # the formal solution along the vertical (mu dropped from every optical path)
    return _formal(tau, S, 1.0)


def _optical_depth_left_sum(kappa, m):
    # optical depth by the left Riemann sum instead of the trapezoid rule
    kappa = np.asarray(kappa, dtype=np.float64)
    tau = np.empty_like(kappa)
    tau[0] = kappa[0] * m[0]
    for d in range(1, len(m)):
        tau[d] = tau[d - 1] + kappa[d - 1] * (m[d] - m[d - 1])
    return tau


def _upper_median(x):
    s = np.sort(np.asarray(x, dtype=np.float64))
    return float(s[len(s) // 2])


def _windows_one_short(pl, level=1.0):
    # every non-empty window loses its last point
    lo, hi = _windows(pl, level)
    return lo, np.where(hi >= lo, hi - 1, hi)


def _partition_functions_mutant(dx_sign=1.0, with_c2=True):
    # U[e, j](T) = exp(c0 + c1 x + c2 x^2) with x's sign or the x^2 term as given
    def f(eos, T):
        x = dx_sign * math.log(T / 5040.0)
        c = np.asarray(eos.lnU, dtype=np.float64)
        U = np.exp(c[:, :, 0] + c[:, :, 1] * x + (c[:, :, 2] * x * x if with_c2 else 0.0))
        j = np.arange(c.shape[1])[None, :]
        return np.where(j < np.asarray(eos.n_stages)[:, None], U, 0.0)
    return f


def _swapped_fraction(axis, x):
    i, f = _cell_weights(axis, x)
    return i, 1.0 - f


def _set(module, name, value):
    return lambda mp: mp.setattr(module, name, value)


# name -> (plant the mistake, the pins that must catch it)
CASES = {
    # Voigt function
    "voigt: Lorentz wing dropped (Gaussian only)": (
        _set(t_v, "H", lambda v, a: np.exp(-np.square(np.asarray(v, dtype=np.float64))) + 0.0 * np.asarray(a)),
        [t_v.test_core_equals_erfcx, t_v.test_lorentzian_asymptote]),
    "voigt: damping parameter doubled": (
        _set(t_v, "H", lambda v, a: _H(v, 2.0 * np.asarray(a, dtype=np.float64))),
        [t_v.test_core_equals_erfcx, t_v.test_lorentzian_asymptote]),
    "voigt: centre shifted by 0.01 Doppler width": (
        _set(t_v, "H", lambda v, a: _H(np.asarray(v, dtype=np.float64) - 0.01, a)),
        [t_v.test_even_and_monotone]),
    "voigt: window bound without the factor 8 of its Lorentz term": (
        _set(t_v, "H_upper_bound_v", _bound_without_8),
        [t_v.test_upper_bound]),
    # line terms and populations
    "line strength: stimulated-emission factor dropped": (
        _set(ph, "line_terms", _terms(lambda t, L, pop: dataclasses.replace(
            t, S=t.S / -np.expm1(-ph.H_PLANCK * t.nu0 / (ph.K_BOLTZ * pop.T))))),
        [t_ph.test_stimulated_emission_and_lambda_scaling]),
    "line strength: Boltzmann factor with the wrong sign": (
        _set(ph, "line_terms", _terms(lambda t, L, pop: dataclasses.replace(
            t, S=t.S * np.exp(2.0 * np.asarray(L.E_eV, dtype=np.float64) / (ph.K_EV * pop.T))))),
        [t_ph.test_boltzmann_factor]),
    "Doppler width: kT in place of 2kT": (
        _set(ph, "line_terms", _terms(lambda t, L, pop: dataclasses.replace(
            t, dnuD=t.dnuD / math.sqrt(2.0), u=t.u / math.sqrt(2.0), a=t.a * math.sqrt(2.0),
            S=t.S * math.sqrt(2.0)))),
        [t_ph.test_doppler_width_hydrogen]),
    "damping parameter: 2 pi in place of 4 pi": (
        _set(ph, "line_terms", _terms(lambda t, L, pop: dataclasses.replace(t, a=2.0 * t.a))),
        [t_ph.test_pressure_broadening_perturbers]),
    "Saha equation: 3/2 power dropped": (
        _set(ph, "saha_phi", _saha_no_three_halves),
        [t_ph.test_pure_hydrogen_closed_form]),
    "partition functions: x^2 term dropped": (
        _set(ph, "partition_functions", _partition_functions_mutant(with_c2=False)),
        [t_ph.test_eos_pure_hydrogen_temperature_dependent_partition_function]),
    "partition functions: x = ln(5040 K / T)": (
        _set(ph, "partition_functions", _partition_functions_mutant(dx_sign=-1.0)),
        [t_ph.test_eos_pure_hydrogen_temperature_dependent_partition_function,
         t_ph.test_eos_partition_function_at_reference_temperature]),
    # ODF step means
    "ODF: widths taken in reverse order": (
        _set(od, "cumulative_widths", lambda widths: _cum_widths(list(widths)[::-1])),
        [t_odf.test_brute_force_rational]),
    "ODF: values sorted in descending order": (
        _set(od, "step_means_sorted", lambda xs, widths: _step_means(xs[::-1], widths)),
        [t_odf.test_brute_force_rational, t_odf.test_monotone_and_mean]),
    "ODF: arithmetic means where geometric ones are asked for": (
        _set(od, "geom_step_means_sorted", lambda xs, widths: _step_means(xs, widths)),
        [t_odf.test_geometric_brute_force_and_zeros]),
    # spectrum
    "formal solution: linear source term dropped": (
        _set(spc, "formal_solution", _formal_constant_source_layers),
        [t_sp.test_linear_source_eddington_barbier]),
    "formal solution: mu dropped from the optical paths": (
        _set(spc, "formal_solution", _formal_mu_ignored),
        [t_sp.test_linear_source_eddington_barbier]),
    "optical depth: left sum for the trapezoid": (
        _set(spc, "optical_depth", _optical_depth_left_sum),
        [t_sp.test_optical_depth_trapezoid]),
    "Planck function: temperature off by 1 %": (
        _set(spc, "planck_lambda", lambda lam, T: _planck(lam, 1.01 * T)),
        [t_sp.test_planck_stefan_boltzmann]),
    # synthesis
    "kappa_c: upper median for the lower": (
        _set(sy, "lower_median", _upper_median),
        [t_sy.test_lower_median]),
    "cut windows: last point of each window lost": (
        _set(sy, "windows", _windows_one_short),
        [t_sy.test_window_edges_and_sampling]),
    "grid: one point too many": (
        _set(sy, "grid_size", lambda lam0, lam1, R: _grid_size(lam0, lam1, R) + 1),
        [t_sy.test_grid_size_pins, t_sy.test_grid_size_brute_force]),
    # continuum
    "Rayleigh scattering: lambda^-2 in place of lambda^-4": (
        _set(co, "rayleigh_hi", lambda lam: _rayleigh(lam) * np.maximum(
            np.asarray(lam, dtype=np.float64) * 1e8, co.RAYLEIGH_MIN_ANGSTROM) ** 2),
        [t_co.test_rayleigh_series]),
    "electron scattering: Thomson cross-section doubled": (
        _set(co, "SIGMA_T", 2.0 * co.SIGMA_T),
        [t_co.test_constants_against_textbook_values]),
    # bin intensities
    "T-P interpolation: weights of the two cell corners swapped": (
        _set(bi, "cell_weights", _swapped_fraction),
        [t_bi.test_interpolation_reproduces_bilinear_functions]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    plant, pins = CASES[name]
    plant(monkeypatch)
    caught = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake: {name}"


def test_pins_pass_without_a_planted_mistake():
    # the same pins, on the oracle as it stands
    for _, pins in CASES.values():
        for pin in pins:
            pin()
