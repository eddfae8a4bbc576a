"""Populations and line terms in FP64 (oracle; test infrastructure only).

Follows Sect. 2.1 of the paper: LTE populations from the Saha-Boltzmann
equations with the electron density found iteratively from particle and charge
conservation (App. A), and the line absorption coefficient of Eq. (l_nu_line)
with the Doppler width of App. E.

Readings where the paper is silent:
  * single ionisation only (stages I, II) with fixed partition functions;
  * the gas is H, He and the metals of the element table (no molecules);
  * total damping gamma = 10^lgR + 10^lgS * n_e + 10^lgW * n_HI (per-perturber
    Stark and van der Waals widths, no temperature scaling).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# CODATA 2018, cgs
C_LIGHT = 2.99792458e10          # cm s^-1
H_PLANCK = 6.62607015e-27        # erg s
K_BOLTZ = 1.380649e-16           # erg K^-1
M_ELECTRON = 9.1093837015e-28    # g
E_CHARGE = 4.803204712570263e-10  # statC
AMU = 1.66053906660e-24          # g
EV = 1.602176634e-12             # erg
K_EV = K_BOLTZ / EV              # eV K^-1 (8.617333262e-5)


@dataclass
class Populations:
    """State of the gas at one (T, P) point (App. A)."""
    T: float
    P: float
    n_e: float          # electron density [cm^-3]
    n_nuc: float        # nuclei (atoms + ions) density [cm^-3]
    n_HI: float         # neutral hydrogen density [cm^-3]
    rho: float          # mass density [g cm^-3]
    n_stage: np.ndarray  # [n_el, 2] number densities of stages I and II
    NU: np.ndarray       # [n_el, 2] N_k / U_k


def saha_phi(T, chi_eV, U1, U2):
    """Phi(T) = n_II n_e / n_I = (2 U_II / U_I) (2 pi m_e k T / h^2)^{3/2} exp(-chi / kT)."""
    return (2.0 * U2 / U1) * (2.0 * math.pi * M_ELECTRON * K_BOLTZ * T / H_PLANCK ** 2) ** 1.5 \
        * np.exp(-chi_eV / (K_EV * T))


def populations(T: float, P: float, el, abund_scale=None) -> Populations:
    """Electron density by charge balance, then stage populations (App. A, reduced).

    Particle conservation: P = (n_nuc + n_e) k T.  Each element with number fraction
    f_el ionises once: n_II = f n_nuc Phi/(n_e + Phi).  Charge conservation
    n_e = sum_el n_II gives g(n_e) = n_e - sum f (P/kT - n_e) Phi/(n_e + Phi), strictly
    increasing on (0, P/kT), negative at 0 and positive at P/kT, so the root is
    unique; it is bracketed by bisection in ln n_e to full double precision (the
    paper's Newton iteration stops at 1e-4, App. A).
    """
    eps = 10.0 ** (el.log_eps - 12.0)
    if abund_scale is not None:
        eps = eps * np.asarray(abund_scale, dtype=np.float64)
    frac = eps / eps.sum()
    phi = saha_phi(T, el.chi_eV, el.U1, el.U2)
    n_tot = P / (K_BOLTZ * T)

    def g(ne):
        nn = n_tot - ne
        return ne - np.sum(frac * nn * phi / (ne + phi))

    lo, hi = math.log(1e-300), math.log(n_tot)
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if g(math.exp(mid)) > 0.0:
            hi = mid
        else:
            lo = mid
        if hi - lo < 1e-15:
            break
    n_e = math.exp(0.5 * (lo + hi))
    n_nuc = n_tot - n_e
    # n_II/n_I = Phi/n_e: n_I = f n_nuc n_e/(n_e + Phi) avoids the cancellation of f n_nuc - n_II
    # when stage I is almost fully ionised
    n2 = frac * n_nuc * phi / (n_e + phi)
    n1 = frac * n_nuc * n_e / (n_e + phi)
    rho = n_nuc * float(np.sum(frac * el.mass_amu * AMU))
    stage = np.stack([n1, n2], axis=1)
    NU = np.stack([n1 / el.U1, n2 / el.U2], axis=1)
    return Populations(T, P, n_e, n_nuc, float(n1[0]), rho, stage, NU)


def partition_functions(eos, T):
    """U[e, j](T) = exp(c0 + c1 x + c2 x^2), x = ln(T / 5040 K), for the stages of each element
    (zero beyond an element's last stage)."""
    x = math.log(T / 5040.0)
    c = np.asarray(eos.lnU, dtype=np.float64)
    U = np.exp(c[:, :, 0] + c[:, :, 1] * x + c[:, :, 2] * x * x)
    j = np.arange(c.shape[1])[None, :]
    return np.where(j < np.asarray(eos.n_stages)[:, None], U, 0.0)


def populations_eos(T: float, P: float, eos, abund_scale=None, tol: float = 1e-13, max_iter: int = 500) -> Populations:
    """Multi-stage LTE equation of state (App. A, following the scheme the paper describes).

    Every element e has stages j = 0 .. J_e - 1 linked by the Saha-Boltzmann equation
    n_{e,j+1} n_e / n_{e,j} = Phi_{e,j}(T) = (2 U_{j+1}/U_j) (2 pi m_e k T/h^2)^{3/2} e^{-chi_j/kT}
    with temperature-dependent partition functions U_j(T).  Written in the unknowns of App. A,
    the neutral densities n_{e,0} and the electron density n_e, the equations are
      f_e   = sum_j n_{e,j} - a_e n_nuc = 0           (nuclei of each element, a_e its fraction)
      f_ele = sum_e sum_j j n_{e,j} - n_e = 0         (charge conservation)
    with n_{e,j} = n_{e,0} prod_{i<j} Phi_{e,i}/n_e and n_nuc = P/kT - n_e (particle
    conservation, no molecules).  They are solved by Newton-Raphson: the Jacobian
    M = d f / d n is factorised by triangular (LU) decomposition, M dn = -f, and the step is
    applied until every relative change |dn_i / n_i| is below `tol`.  (The paper stops at
    1e-4; the oracle iterates to double precision.)  Steps are shortened so that no density
    drops below a tenth of its value in one iteration.
    """
    from scipy.linalg import lu_factor, lu_solve
    eps = 10.0 ** (np.asarray(eos.log_eps, dtype=np.float64) - 12.0)
    if abund_scale is not None:
        eps = eps * np.asarray(abund_scale, dtype=np.float64)
    frac = eps / eps.sum()
    ne_ = len(frac)
    ns = np.asarray(eos.n_stages)
    J = np.asarray(eos.lnU).shape[1]          # stage columns of the tables (I .. V)
    U = partition_functions(eos, T)
    kT = K_BOLTZ * T
    saha = (2.0 * math.pi * M_ELECTRON * kT / H_PLANCK ** 2) ** 1.5
    phi = np.zeros((ne_, max(J - 1, 1)))
    for e in range(ne_):
        for j in range(ns[e] - 1):
            phi[e, j] = 2.0 * U[e, j + 1] / U[e, j] * saha * math.exp(-eos.chi_eV[e, j] / (K_EV * T))
    n_tot = P / kT
    charge = np.arange(J, dtype=np.float64)

    def stage_factors(n_e):
        # r[e, j] = prod_{i<j} Phi_{e,i} / n_e (r[e, 0] = 1; zero beyond the last stage)
        r = np.zeros((ne_, J))
        r[:, 0] = 1.0
        for j in range(1, J):
            r[:, j] = np.where(j < ns, r[:, j - 1] * phi[:, j - 1] / n_e, 0.0)
        return r

    # start: electrons from hydrogen alone (closed form of the pure-H Saha balance), neutrals
    # from the stage factors at that n_e
    x = math.sqrt(phi[0, 0] * kT / (P + phi[0, 0] * kT)) if phi[0, 0] > 0 else 1e-10
    n_e = max(x * n_tot / (1.0 + x), 1e-30 * n_tot)
    r = stage_factors(n_e)
    n0 = frac * (n_tot - n_e) / r.sum(axis=1)
    for _ in range(max_iter):
        r = stage_factors(n_e)
        s0 = r.sum(axis=1)                      # sum_j r_j
        s1 = r @ charge                         # sum_j j r_j
        s2 = r @ (charge * charge)              # sum_j j^2 r_j
        n_nuc = n_tot - n_e
        f = np.empty(ne_ + 1)
        f[:ne_] = n0 * s0 - frac * n_nuc
        f[ne_] = np.dot(n0, s1) - n_e
        M = np.zeros((ne_ + 1, ne_ + 1))
        M[np.arange(ne_), np.arange(ne_)] = s0                 # d f_e / d n_{e,0}
        M[:ne_, ne_] = -n0 * s1 / n_e + frac                    # d f_e / d n_e (d r_j / d n_e = -j r_j / n_e)
        M[ne_, :ne_] = s1                                       # d f_ele / d n_{e,0}
        M[ne_, ne_] = -np.dot(n0, s2) / n_e - 1.0               # d f_ele / d n_e
        dn = lu_solve(lu_factor(M), -f)
        cur = np.r_[n0, n_e]
        lam = 1.0
        neg = dn < -0.9 * cur
        if np.any(neg):
            lam = float(np.min(-0.9 * cur[neg] / dn[neg]))
        new = cur + lam * dn
        rel = np.abs(lam * dn) / np.maximum(np.abs(cur), 1e-300)
        n0, n_e = new[:ne_], float(new[ne_])
        if rel.max() < tol:
            break
    r = stage_factors(n_e)
    n_nuc = n_tot - n_e
    stage = n0[:, None] * r
    NU = np.where(U > 0, stage / np.where(U > 0, U, 1.0), 0.0)
    rho = n_nuc * float(np.sum(frac * np.asarray(eos.mass_amu) * AMU))
    return Populations(T, P, n_e, n_nuc, float(stage[0, 0]), rho, stage, NU)


@dataclass
class LineTerms:
    """Per-line quantities of Eq. (l_nu_line) at one (T, P) point."""
    nu0: np.ndarray      # line-centre frequency [Hz]
    dnuD: np.ndarray     # Doppler width [Hz]  (App. E)
    u: np.ndarray        # sqrt(2kT/m + vturb^2) [cm/s]
    gamma: np.ndarray    # total damping [s^-1]
    a: np.ndarray        # damping parameter gamma / (4 pi dnuD)
    S: np.ndarray        # strength: ell = S * H(v, a)  [cm^2 g^-1]


def line_terms(lines, species_el, species_stage, el, pop: Populations, vturb=0.0) -> LineTerms:
    """Eq. (l_nu_line): ell_nu = (sqrt(pi) e^2/(m_e c)) g f /(rho dnuD) (N_k/U_k) e^{-E/kT}
    (1 - e^{-h nu0/kT}) H(dnu/dnuD, gamma/(4 pi dnuD)), with dnuD = (nu0/c) sqrt(2kT/m + vturb^2)."""
    T = pop.T
    lam_cm = np.asarray(lines.lam_nm, dtype=np.float64) * 1e-7
    nu0 = C_LIGHT / lam_cm
    sp = np.asarray(lines.species)
    e_idx = species_el[sp]
    stage = species_stage[sp]
    m = el.mass_amu[e_idx] * AMU
    u = np.sqrt(2.0 * K_BOLTZ * T / m + vturb ** 2)
    dnuD = nu0 * u / C_LIGHT
    gamma = (10.0 ** np.asarray(lines.log_gR, dtype=np.float64)
             + 10.0 ** np.asarray(lines.log_gS, dtype=np.float64) * pop.n_e
             + 10.0 ** np.asarray(lines.log_gW, dtype=np.float64) * pop.n_HI)
    a = gamma / (4.0 * math.pi * dnuD)
    gf = 10.0 ** np.asarray(lines.log_gf, dtype=np.float64)
    NU = pop.NU[e_idx, stage]
    E = np.asarray(lines.E_eV, dtype=np.float64)
    boltz = np.exp(-E / (K_EV * T))
    stim = -np.expm1(-H_PLANCK * nu0 / (K_BOLTZ * T))
    S = (math.sqrt(math.pi) * E_CHARGE ** 2 / (M_ELECTRON * C_LIGHT)) * gf * NU / (pop.rho * dnuD) * boltz * stim
    return LineTerms(nu0, dnuD, u, gamma, a, S)
