"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *draws* inputs: it holds tables of element data, seeded random
line lists, (T, P) grids, interval bounds, sub-bin widths and request streams.
It contains none of the method's arithmetic (no populations, no profiles, no
opacities, no sorting or step means); both the FP64 oracle and the CUDA path
receive these arrays as plain inputs.

Shapes and distributions follow the workloads of the method (MPS-ATLAS,
Witzke et al. 2021): line lists of Kurucz/VALD size (Sect. 2.3 quotes >1e8
lines), the DFSYNTHE 57 x 25 T-P grid (Sect. 4.2), a log-lambda grid
lambda_n = lambda_0 (1 + 1/R)^(n-1) (App. E), equal log-lambda bins and the
12-sub-bin width set (Sect. 2.3, App. E).  Real line lists, bin grids and
model atmospheres are not available, so seeded synthetic stand-ins are used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Element table (input data, not arithmetic).  Columns: symbol, atomic mass
# [amu], first ionisation energy [eV], fixed partition functions U_I, U_II,
# solar-like abundance log eps (H = 12).  Partition functions are held fixed
# (temperature independent); this is a convention of the synthetic workload.
# H and He are always present (elements 0 and 1) and carry no lines.
# ---------------------------------------------------------------------------
ELEMENTS = [
    ("H", 1.008, 13.598, 2.0, 1.0, 12.00),
    ("He", 4.0026, 24.587, 1.0, 2.0, 10.93),
    ("Fe", 55.845, 7.902, 25.0, 40.0, 7.50),
    ("Ca", 40.078, 6.113, 1.1, 2.1, 6.34),
    ("Mg", 24.305, 7.646, 1.0, 2.0, 7.60),
    ("Si", 28.085, 8.152, 9.3, 5.6, 7.51),
    ("Ti", 47.867, 6.828, 27.0, 50.0, 4.95),
    ("Na", 22.990, 5.139, 2.0, 1.0, 6.24),
    ("Al", 26.982, 5.986, 5.8, 1.0, 6.45),
    ("Cr", 51.996, 6.767, 9.5, 7.2, 5.64),
    ("Ni", 58.693, 7.640, 29.0, 9.5, 6.22),
    ("Mn", 54.938, 7.434, 6.4, 7.5, 5.43),
    ("Co", 58.933, 7.881, 31.0, 25.0, 4.99),
    ("V", 50.942, 6.746, 38.0, 31.0, 3.93),
    ("Sc", 44.956, 6.561, 10.0, 20.0, 3.15),
    ("Sr", 87.62, 5.695, 1.0, 2.0, 2.87),
    ("Ba", 137.327, 5.212, 1.3, 3.0, 2.18),
]

# Ionisation energies [eV] beyond the first (II -> III, III -> IV, IV -> V), approximate
# standard values used as the synthetic stand-in for the multi-stage equation of state:
# H has stages I-II, He I-III, every metal I-V (App. E of the paper: N_j/U_j up to j = 5).
IONISATION_HIGHER = {
    "H": (), "He": (54.418,), "Fe": (16.199, 30.651, 54.91), "Ca": (11.872, 50.913, 67.27),
    "Mg": (15.035, 80.144, 109.27), "Si": (16.346, 33.493, 45.142), "Ti": (13.576, 27.492, 43.268),
    "Na": (47.286, 71.62, 98.94), "Al": (18.829, 28.448, 119.99), "Cr": (16.486, 30.96, 49.16),
    "Ni": (18.169, 35.19, 54.9), "Mn": (15.64, 33.668, 51.2), "Co": (17.084, 33.5, 51.3),
    "V": (14.634, 29.311, 46.709), "Sc": (12.8, 24.757, 73.49), "Sr": (11.03, 42.89, 57.0),
    "Ba": (10.004, 35.84, 47.0),
}
MAX_STAGES = 5

# The 12-step sub-bin widths of the DFSYNTHE ODF: nine of 0.1, then 0.05,
# 0.04, 0.01 (Sect. 2.3 / App. E; the configuration of Castelli 2005).
ODF_WIDTHS_12 = np.array([0.1] * 9 + [0.05, 0.04, 0.01], dtype=np.float64)


@dataclass
class Elements:
    """Element data as arrays; metals are elements 2..n_el-1."""
    symbol: list
    mass_amu: np.ndarray
    chi_eV: np.ndarray
    U1: np.ndarray
    U2: np.ndarray
    log_eps: np.ndarray

    @property
    def n(self) -> int:
        return len(self.symbol)


def elements(n_metals: int) -> Elements:
    """H, He and the first ``n_metals`` metals of the table."""
    if not 1 <= n_metals <= len(ELEMENTS) - 2:
        raise ValueError("n_metals out of range")
    rows = ELEMENTS[: 2 + n_metals]
    col = lambda i: np.array([r[i] for r in rows], dtype=np.float64)
    return Elements([r[0] for r in rows], col(1), col(2), col(3), col(4), col(5))


@dataclass
class EosTable:
    """Element data of the multi-stage equation of state (App. A, E of the paper).

    Element e has stages 0 .. n_stages[e]-1 (I, II, ...); chi_eV[e, j] is the ionisation
    energy from stage j to j + 1; the partition function of stage j is given by
    ln U_j(T) = lnU[e, j, 0] + lnU[e, j, 1] x + lnU[e, j, 2] x^2 with x = ln(T / 5040 K).
    Unused entries (stages at or beyond n_stages) are zero."""
    symbol: list
    mass_amu: np.ndarray     # [n]
    log_eps: np.ndarray      # [n]
    n_stages: np.ndarray     # int32 [n], 1..5
    chi_eV: np.ndarray       # [n, 4]
    lnU: np.ndarray          # [n, 5, 3]

    @property
    def n(self) -> int:
        return len(self.symbol)


def eos_table(n_metals: int, seed: int = 1010) -> EosTable:
    """H, He and the first ``n_metals`` metals with all their stages up to V (H: I-II, He: I-III).

    The first ionisation energies and the constant terms of stages I and II are those of the
    element table (partition functions U1, U2 at 5040 K); the constant terms of the higher
    stages are ground-state weights drawn from {1, ..., 30} and the temperature terms of every
    stage are drawn as c1 ~ U(0, 0.4), c2 ~ U(0, 0.1) (a seeded synthetic stand-in for fits to
    tabulated partition functions); H II and He III (bare nuclei) and H I keep constant U."""
    rng = np.random.default_rng(seed)
    rows = ELEMENTS[: 2 + n_metals]
    n = len(rows)
    ns = np.array([2 if r[0] == "H" else (3 if r[0] == "He" else MAX_STAGES) for r in rows], dtype=np.int32)
    chi = np.zeros((n, MAX_STAGES - 1))
    lnU = np.zeros((n, MAX_STAGES, 3))
    for e, r in enumerate(rows):
        chi[e, 0] = r[2]
        chi[e, 1:ns[e] - 1] = IONISATION_HIGHER[r[0]][: ns[e] - 2]
        g0 = np.r_[r[3], r[4], rng.integers(1, 31, MAX_STAGES - 2)].astype(np.float64)
        c1 = rng.uniform(0.0, 0.4, MAX_STAGES)
        c2 = rng.uniform(0.0, 0.1, MAX_STAGES)
        for j in range(ns[e]):
            const = (r[0] == "H") or (r[0] == "He" and j == 2)
            lnU[e, j] = [math.log(g0[j]), 0.0 if const else c1[j], 0.0 if const else c2[j]]
    col = lambda i: np.array([r[i] for r in rows], dtype=np.float64)
    return EosTable([r[0] for r in rows], col(1), col(5), ns, chi, lnU)


def species_table_eos(n_metals: int, n_stages: int = 3):
    """Line-bearing species of the metals in stages I .. n_stages: species s maps to element
    2 + s // n_stages and stage s % n_stages."""
    el = np.repeat(np.arange(2, 2 + n_metals, dtype=np.int32), n_stages)
    stage = np.tile(np.arange(n_stages, dtype=np.int32), n_metals)
    return el, stage


def species_table(n_metals: int):
    """Line-bearing species: (element index, ion stage) for every metal, stages I and II.

    Species s maps to element 2 + s // 2 and stage s % 2 (0 = neutral, 1 = singly ionised).
    """
    el = np.repeat(np.arange(2, 2 + n_metals, dtype=np.int32), 2)
    stage = np.tile(np.array([0, 1], dtype=np.int32), n_metals)
    return el, stage


@dataclass
class LineList:
    """Structure-of-arrays line list, sorted by wavelength."""
    lam_nm: np.ndarray      # float64 [L], ascending
    log_gf: np.ndarray      # float32 [L]
    E_eV: np.ndarray        # float32 [L], lower-level excitation energy
    species: np.ndarray     # int32 [L], index into species_table
    log_gR: np.ndarray      # float32 [L], log10 radiative damping [s^-1]
    log_gS: np.ndarray      # float32 [L], log10 Stark width per electron [s^-1 cm^3]
    log_gW: np.ndarray      # float32 [L], log10 van der Waals width per H I atom [s^-1 cm^3]

    def __len__(self):
        return len(self.lam_nm)

    def subset(self, idx) -> "LineList":
        return LineList(*(getattr(self, f)[idx] for f in
                          ("lam_nm", "log_gf", "E_eV", "species", "log_gR", "log_gS", "log_gW")))


def linelist(n_lines: int, n_species: int, lam_lo_nm: float, lam_hi_nm: float, seed: int) -> LineList:
    """Seeded synthetic line list.

    lambda log-uniform in [lam_lo, lam_hi]; log gf ~ N(-3, 1.5); E ~ U(0, 10) eV;
    species uniform over ``n_species`` (element, ion) pairs; log damping constants
    (radiative, Stark, van der Waals) each ~ N(-8, 0.5).  Float fields are rounded
    to float32 once here so that every consumer sees identical values.
    """
    rng = np.random.default_rng(seed)
    lam = np.exp(rng.uniform(math.log(lam_lo_nm), math.log(lam_hi_nm), n_lines))
    order = np.argsort(lam, kind="stable")
    lam = lam[order]
    gf = rng.normal(-3.0, 1.5, n_lines).astype(np.float32)
    E = rng.uniform(0.0, 10.0, n_lines).astype(np.float32)
    sp = rng.integers(0, n_species, n_lines).astype(np.int32)
    damp = rng.normal(-8.0, 0.5, (3, n_lines)).astype(np.float32)
    return LineList(lam, gf, E, sp, damp[0], damp[1], damp[2])


@dataclass
class Grid:
    """Log-lambda grid lambda_j = lam0 * (1 + 1/R)^j, j = 0..N-1 (App. E)."""
    lam0_nm: float
    lam1_nm: float
    R: float


def tp_grid_dfsynthe(nT: int = 57, nP: int = 25, Tlo=2000.0, Thi=200000.0, logPlo=-4.0, logPhi=8.0):
    """T log-spaced in [Tlo, Thi], log P evenly spaced (cgs); returns (T[nT*nP], P[nT*nP]) T-major."""
    T = np.exp(np.linspace(math.log(Tlo), math.log(Thi), nT))
    P = 10.0 ** np.linspace(logPlo, logPhi, nP)
    TT, PP = np.meshgrid(T, P, indexing="ij")
    return TT.reshape(-1).copy(), PP.reshape(-1).copy()


def equal_intervals(n_points: int, K: int) -> np.ndarray:
    """Bounds b_0..b_K of K intervals of (nearly) equal point count on a log grid.

    On a log-lambda grid equal point counts are equal log-lambda widths.
    b_k = floor(k * n_points / K), computed in integer arithmetic.
    """
    k = np.arange(K + 1, dtype=np.int64)
    return (k * n_points) // K


def abundance_scales(n_comp: int, n_elements: int, seed: int) -> np.ndarray:
    """Per-element abundance scale factors ~ logU(0.01, 10) for the metals; H, He fixed at 1."""
    rng = np.random.default_rng(seed)
    s = np.ones((n_comp, n_elements))
    s[:, 2:] = np.exp(rng.uniform(math.log(0.01), math.log(10.0), (n_comp, n_elements - 2)))
    return s


def grey_atmosphere(D: int, Teff: float, logg: float, log_tau_top=-6.8, log_tau_bot=2.0, kappa_bar=0.1):
    """Model-atmosphere input of the spectrum workload: D depths with tau log-spaced from
    10^log_tau_top to 10^log_tau_bot, the grey Eddington law T = Teff (3/4 (tau + 2/3))^(1/4),
    column mass m = tau / kappa_bar and hydrostatic pressure P = g m.  Returns (m, T, P)."""
    tau = 10.0 ** np.linspace(log_tau_top, log_tau_bot, D)
    T = Teff * (0.75 * (tau + 2.0 / 3.0)) ** 0.25
    m = tau / kappa_bar
    P = 10.0 ** logg * m
    return m, T, P


def odf_table_synthetic(nT: int, nP: int, K: int, n_steps: int, seed: int, lam_lo_nm=9.0, lam_hi_nm=10000.0):
    """Seeded synthetic ODF table on the DFSYNTHE-style T-P grid (tp_grid_dfsynthe with nT x nP
    points): returns (log10_T [nT], log10_P [nP], odf [nT*nP][K][n_steps] (per grid point and
    bin a median 10^U(-2, 2) times 10^N(0, 1) spreads, sorted ascending over the sub-bins),
    kappa_c [nT*nP] float32 = 10^U(-3, 0), lam_c_nm [K] (centres of K log-equal bins))."""
    rng = np.random.default_rng(seed)
    T, P = tp_grid_dfsynthe(nT, nP)
    lt = np.log10(T.reshape(nT, nP)[:, 0]).copy()
    lp = np.log10(P.reshape(nT, nP)[0, :]).copy()
    base = 10.0 ** rng.uniform(-2.0, 2.0, (nT * nP, K, 1))
    odf = np.sort(base * 10.0 ** rng.normal(0.0, 1.0, (nT * nP, K, n_steps)), axis=-1)
    kc = (10.0 ** rng.uniform(-3.0, 0.0, nT * nP)).astype(np.float32)
    edges = np.exp(np.linspace(math.log(lam_lo_nm), math.log(lam_hi_nm), K + 1))
    return lt, lp, odf, kc, 0.5 * (edges[:-1] + edges[1:])


def ray_atmospheres(n_rays: int, D: int, seed: int):
    """n_rays grey atmospheres of D depths (Teff ~ U(3500, 12000) K, log g ~ U(1, 5), the
    spectrum workload's model), as float64 arrays [n_rays][D] of m, T, P."""
    rng = np.random.default_rng(seed)
    m = np.empty((n_rays, D))
    T = np.empty((n_rays, D))
    P = np.empty((n_rays, D))
    for r in range(n_rays):
        m[r], T[r], P[r] = grey_atmosphere(D, rng.uniform(3500.0, 12000.0), rng.uniform(1.0, 5.0))
    return m, T, P


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n_lines: int
    n_metals: int
    grid: Grid
    T: np.ndarray
    P: np.ndarray
    n_intervals: int
    widths: np.ndarray = field(default_factory=lambda: ODF_WIDTHS_12.copy())
    seed: int = 0
    cut: float = 1e-3         # profile cut relative to the flat continuum
    kc_factor: float = 1e-2   # flat continuum = kc_factor * median line-centre opacity

    @property
    def n_species(self):
        return 2 * self.n_metals

    def lines(self) -> LineList:
        return linelist(self.n_lines, self.n_species, self.grid.lam0_nm, self.grid.lam1_nm, self.seed)


def config_small() -> Workload:
    """Plain method: 20,000 lines, 10 species, 300-400 nm at R = 2e6, 4 (T, P) points at log P = 4,
    10 equal log-lambda intervals x 12 steps."""
    T = np.array([4000.0, 6000.0, 9000.0, 15000.0])
    P = np.full(4, 1e4)
    return Workload("lines20k_300-400nm_R2e6_4pts", 20000, 5, Grid(300.0, 400.0, 2e6), T, P, 10, seed=1000)


def config_table() -> Workload:
    """Full ODF table: 5e6 lines, 30 species, 9-10000 nm at R = 2e6, 57 T x 25 P, 328 intervals."""
    T, P = tp_grid_dfsynthe()
    return Workload("lines5M_9-10000nm_R2e6_57x25", 5_000_000, 15, Grid(9.0, 10000.0, 2e6), T, P, 328, seed=1001)


def config_tiny(n_lines=40, lam=(300.0, 300.6), R=2e6, seed=7, n_metals=5) -> Workload:
    """Small case for parity tests: a few lines on a few thousand grid points."""
    T = np.array([4000.0, 6000.0, 9000.0, 15000.0])
    P = np.full(4, 1e4)
    return Workload(f"tiny{n_lines}", n_lines, n_metals, Grid(lam[0], lam[1], R), T, P, 3, seed=seed)
