"""Continuous opacity from the closed-form sources in FP64 (oracle; test infrastructure only).

Sect. 2.1 of the paper lists the continuum of MPS-ATLAS: bound-free and free-free absorption
of H I, H-, He and metals, electron scattering and Rayleigh scattering on H I, He I and H2
(App. G groups them as 'H1', 'Hray', 'Elec', ...).  The sources that have closed forms are
written out here; the others need tabulated cross-sections and are not part of this oracle.
Per unit volume, at frequency nu = c / lambda:
  * electron scattering: n_e sigma_T;
  * hydrogen bound-free from the levels n = 1 .. N_LEVELS of H I (Kramers' cross-section,
    Gaunt factor 1): sigma_n(nu) = K_bf / (n^5 nu^3) for nu >= nu_n = chi_H / (h n^2), with
    K_bf = 64 pi^4 m_e e^10 / (3 sqrt(3) c h^6), and level populations from the Boltzmann
    distribution inside H I, N_n = n_HI (2 n^2 / U_HI) exp(-chi_H (1 - 1/n^2) / kT);
  * hydrogen free-free (Kramers, Gaunt factor 1): K_ff n_e n_HII / (sqrt(T) nu^3), with
    K_ff = (4 e^6 / (3 m_e h c)) sqrt(2 pi / (3 k m_e));
  * both absorption terms times the stimulated-emission factor 1 - exp(-h nu / kT);
  * Rayleigh scattering on H I: n_HI sigma_R with the series in the wavelength
    sigma_R = 5.799e-13 / L^4 + 1.422e-6 / L^6 + 2.784 / L^8 cm^2 (L in Angstrom; the series
    of Dalgarno (1962) used by Kurucz (1970)), evaluated at L = max(lambda, 1300 Angstrom)
    because the series diverges towards Lyman alpha.
kappa_c = (sum of the above) / rho, in cm^2 g^-1.
"""
from __future__ import annotations

import math

import numpy as np

from . import physics

N_LEVELS = 8
CHI_H_EV = 13.598
SIGMA_T = 6.6524587321e-25      # cm^2 (CODATA 2018)
RAYLEIGH_MIN_ANGSTROM = 1300.0


def kramers_bf_constant():
    """K_bf = 64 pi^4 m_e e^10 / (3 sqrt(3) c h^6) [cm^2 Hz^3]."""
    return 64.0 * math.pi ** 4 * physics.M_ELECTRON * physics.E_CHARGE ** 10 / (
        3.0 * math.sqrt(3.0) * physics.C_LIGHT * physics.H_PLANCK ** 6)


def kramers_ff_constant():
    """K_ff = (4 e^6 / (3 m_e h c)) sqrt(2 pi / (3 k m_e)) [cgs: cm^5 K^1/2 Hz^3]."""
    e, m, h, c, k = physics.E_CHARGE, physics.M_ELECTRON, physics.H_PLANCK, physics.C_LIGHT, physics.K_BOLTZ
    return 4.0 * e ** 6 / (3.0 * m * h * c) * math.sqrt(2.0 * math.pi / (3.0 * k * m))


def rayleigh_hi(lam_cm):
    """sigma_R of H I [cm^2] at the wavelengths lam_cm."""
    L = np.maximum(np.asarray(lam_cm, dtype=np.float64) * 1e8, RAYLEIGH_MIN_ANGSTROM)
    L2 = L * L
    return (5.799e-13 + (1.422e-6 + 2.784 / L2) / L2) / (L2 * L2)


def kappa_c(lam_nm, pop: physics.Populations, U_HI: float = 2.0, sources=("elec", "bf", "ff", "ray")):
    """Continuous opacity [cm^2 g^-1] at wavelengths lam_nm of one (T, P) point.

    pop: the populations (n_e, n_HI, rho and the H II density pop.n_stage[0, 1]); U_HI is the
    H I partition function used for the level populations."""
    lam_cm = np.asarray(lam_nm, dtype=np.float64) * 1e-7
    nu = physics.C_LIGHT / lam_cm
    T = pop.T
    kT = physics.K_BOLTZ * T
    stim = -np.expm1(-physics.H_PLANCK * nu / kT)
    alpha = np.zeros_like(nu)
    if "elec" in sources:
        alpha = alpha + pop.n_e * SIGMA_T
    if "bf" in sources:
        Kbf = kramers_bf_constant()
        chi = CHI_H_EV * physics.EV
        for n in range(1, N_LEVELS + 1):
            Nn = pop.n_HI * 2.0 * n * n / U_HI * math.exp(-chi * (1.0 - 1.0 / (n * n)) / kT)
            nu_n = chi / (physics.H_PLANCK * n * n)
            alpha = alpha + np.where(nu >= nu_n, Nn * Kbf / (n ** 5 * nu ** 3), 0.0) * stim
    if "ff" in sources:
        n_hii = float(pop.n_stage[0, 1])
        alpha = alpha + kramers_ff_constant() * pop.n_e * n_hii / (math.sqrt(T) * nu ** 3) * stim
    if "ray" in sources:
        alpha = alpha + pop.n_HI * rayleigh_hi(lam_cm)
    return alpha / pop.rho
