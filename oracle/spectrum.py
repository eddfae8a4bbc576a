"""Emergent intensity by an LTE formal solution in FP64 (oracle; test infrastructure only).

Eq. (Ilambda) of the paper: I_lambda(mu) = integral_0^inf S_lambda exp(-tau_lambda/mu) dtau_lambda/mu,
with S_lambda = B_lambda(T) in LTE without scattering (Sect. 2).  The paper's
module III uses Feautrier / iterative solvers with scattering (App. D); the
synthetic spectrum workload reduces this to the plain integral, evaluated layer
by layer with S linear in tau inside each layer:

  tau_0 = kappa_0 m_0,  tau_{d+1} = tau_d + (kappa_d + kappa_{d+1}) (m_{d+1} - m_d)/2,
  bottom: I_{D-1} = S_{D-1} + mu dS/dtau (diffusion approximation),
  layer d: I_d = I_{d+1} e^{-D} + S_d (1 - e^{-D}) + (S_{d+1} - S_d) (1 - e^{-D}(1 + D))/D,
           D = (tau_{d+1} - tau_d)/mu,
  top: I = I_0 e^{-tau_0/mu} + S_0 (1 - e^{-tau_0/mu}) (isothermal above the first point).

The grey model atmosphere: tau log-spaced, T = Teff (3/4 (tau + 2/3))^{1/4},
m = tau / kappa_bar, P = g m.
"""
from __future__ import annotations

import math

import numpy as np

from . import physics, synthesis


def planck_lambda(lam_cm, T):
    """B_lambda(T) = 2 h c^2 / lambda^5 / (exp(h c/(lambda k T)) - 1) [erg s^-1 cm^-2 sr^-1 cm^-1]."""
    h, c, k = physics.H_PLANCK, physics.C_LIGHT, physics.K_BOLTZ
    lam_cm = np.asarray(lam_cm, dtype=np.float64)
    return 2.0 * h * c * c / lam_cm ** 5 / np.expm1(h * c / (lam_cm * k * T))


def grey_atmosphere(D: int, Teff: float, logg: float, log_tau_top=-6.8, log_tau_bot=2.0, kappa_bar=0.1):
    """The grey model atmosphere of the spectrum workload (an input, from workloads)."""
    import workloads
    return workloads.grey_atmosphere(D, Teff, logg, log_tau_top, log_tau_bot, kappa_bar)


def optical_depth(kappa, m):
    """tau[d] along depth for kappa[d] (per unit mass) on column mass m[d] (trapezoid)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    tau = np.empty_like(kappa)
    tau[0] = kappa[0] * m[0]
    for d in range(1, len(m)):
        tau[d] = tau[d - 1] + 0.5 * (kappa[d - 1] + kappa[d]) * (m[d] - m[d - 1])
    return tau


def formal_solution(tau, S, mu):
    """Emergent I(mu) for source function S on optical depths tau (top to bottom)."""
    tau = np.asarray(tau, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    D = len(tau)
    dS = (S[D - 1] - S[D - 2]) / (tau[D - 1] - tau[D - 2])
    I = S[D - 1] + mu * dS
    for d in range(D - 2, -1, -1):
        x = (tau[d + 1] - tau[d]) / mu
        ex = math.exp(-x)
        I = I * ex + S[d] * (1.0 - ex) + (S[d + 1] - S[d]) * ((1.0 - ex * (1.0 + x)) / x if x > 0 else 0.0)
    ex = math.exp(-tau[0] / mu)
    return I * ex + S[0] * (1.0 - ex)


def spectrum(lines, species_el, species_stage, el, m, T, P, win_grid, mus, cut=1e-3, kc_factor=1e-2,
             abund_scale=None, vturb=0.0, continuum=None):
    """I[n_mu][N_win] of one atmosphere over a window grid (FP64, dense).  continuum: None for the
    flat continuum of the cut rule, or a tuple of continuum.kappa_c sources added per wavelength
    instead (the cut keeps the flat continuum)."""
    D = len(m)
    N = synthesis.grid_size(win_grid.lam0_nm, win_grid.lam1_nm, win_grid.R)
    kap = np.empty((D, N))
    S = np.empty((D, N))
    lam_cm = synthesis.grid_lambda_nm(win_grid.lam0_nm, win_grid.R, np.arange(N)) * 1e-7
    for d in range(D):
        pl = synthesis.prepare(lines, species_el, species_stage, el, T[d], P[d], win_grid, cut, kc_factor,
                               abund_scale, vturb)
        k, _, _ = synthesis.kappa_dense(pl)
        kap[d] = k + (pl.kappa_c if continuum is None else _continuum(lam_cm, pl.pop, el, T[d], continuum))
        S[d] = planck_lambda(lam_cm, T[d])
    out = np.empty((len(mus), N))
    for j in range(N):
        tau = optical_depth(kap[:, j], m)
        for q, mu in enumerate(mus):
            out[q, j] = formal_solution(tau, S[:, j], mu)
    return out


def _continuum(lam_cm, pop, el, T, sources):
    # closed-form continuum at the grid wavelengths; U_HI of the element table at T
    from . import continuum, physics as ph
    U_HI = float(ph.partition_functions(el, T)[0, 0]) if hasattr(el, "n_stages") else float(el.U1[0])
    return continuum.kappa_c(np.asarray(lam_cm) * 1e7, pop, U_HI=U_HI, sources=sources)


def spectrum_at(lines, species_el, species_stage, el, m, T, P, win_grid, mus, js, cut=1e-3, kc_factor=1e-2,
                abund_scale=None, vturb=0.0, slack_band=3e-5, continuum=None):
    """I[n_mu][len(js)] of one atmosphere at the window grid indices js only (same steps as
    `spectrum`; the opacity of each depth comes from synthesis.kappa_at), together with a bound
    on how far I can move when contributions inside the edge-slack band of the cut are taken
    or dropped: dI[n_mu][len(js)] = max over the two one-sided perturbations kappa +- slack of
    |I(kappa +- slack) - I(kappa)|."""
    js = np.asarray(js, dtype=np.int64)
    D = len(m)
    kap = np.empty((D, len(js)))
    sl = np.empty((D, len(js)))
    S = np.empty((D, len(js)))
    lam_cm = synthesis.grid_lambda_nm(win_grid.lam0_nm, win_grid.R, js) * 1e-7
    for d in range(D):
        pl = synthesis.prepare(lines, species_el, species_stage, el, T[d], P[d], win_grid, cut, kc_factor,
                               abund_scale, vturb)
        k, s = synthesis.kappa_at(pl, js, slack_band)
        kap[d] = k + (pl.kappa_c if continuum is None else _continuum(lam_cm, pl.pop, el, T[d], continuum))
        sl[d] = s
        S[d] = planck_lambda(lam_cm, T[d])
    out = np.empty((len(mus), len(js)))
    dI = np.zeros((len(mus), len(js)))
    for n in range(len(js)):
        tau = optical_depth(kap[:, n], m)
        tau_hi = optical_depth(kap[:, n] + sl[:, n], m)
        tau_lo = optical_depth(np.maximum(kap[:, n] - sl[:, n], 0.0), m)
        for q, mu in enumerate(mus):
            out[q, n] = formal_solution(tau, S[:, n], mu)
            if np.any(sl[:, n] > 0):
                dI[q, n] = max(abs(formal_solution(tau_hi, S[:, n], mu) - out[q, n]),
                               abs(formal_solution(tau_lo, S[:, n], mu) - out[q, n]))
    return out, dI
