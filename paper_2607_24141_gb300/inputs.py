"""Seeded synthetic atmospheres, line lists and pixel grids.

This module only *generates inputs*; it holds none of the synthesis
arithmetic (no line opacity, transfer or instrument maths).  Both the FP64
CPU oracle (``oracle/``) and the CUDA library read the arrays it returns, so
the two implementations see bit-identical inputs.

The recipes stand in for the paper's Kurucz atmospheres, line catalogs and
APOGEE pixel grids, none of which are available.  They take only the paper's
shapes: a logarithmic grid at R_grid = 300,000 (Sec. 2.1, Eqs. 1-2), a
72-layer plane-parallel atmosphere, Voigt lines described by
(lambda, log gf, E_low, gamma_rad, gamma_4, gamma_6, species) (Eqs. 4-5),
1500-1700 nm APOGEE-like windows with an 8,575-pixel log-uniform detector
grid (Sec. 7, Eq. for f_p), and the Sun/Arcturus-like labels of Sec. 6.

Atmosphere recipe (every config):
  x_j = -6.875 + 0.125 j (j = 0..71), tau_j = 10**x_j
  T_j**4 = 0.75 Teff**4 (tau_j + 2/3)                       (grey Eddington)
  m_j = m_ref tau_j**0.7,  m_ref = 3 * 10**(-0.4 (log g - 4.44))  g cm^-2
  P_gas = g m;  P_e = 1e-4 g m_ref tau (Teff/5777)**4
  n_e = P_e/kT, n_pert = (P_gas - P_e)/kT, rho = 1.3 m_u P_gas/kT
  kappa_c(d, i) = kappa0(d) (lambda_i / 500 nm)**-1, kappa0 = tau**0.3/(0.7 m_ref)
  species: log10 f_s ~ N(mu, 1); per-layer jitter 10**N(0, 0.1);
           pop_{s,d} = f_s 10**[M/H] n_tot(d) / U_s, U_s = 10**U[0, 1.5]
           f_s is the absorbing lower level's share of all particles (abundance,
           ionisation and excitation folded together).  mu sets the line strength
           against the continuum; it is chosen per workload so that the normalised
           spectrum has a realistic line-depth distribution (median f ~ 0.9-0.95,
           strongest lines saturated, 5th percentile ~ 0.4-0.5) rather than a
           saturated line forest: mu = -9.5 (solar optical, 500 nm, config 0),
           -12.5 (300-1000 nm, 3e6 lines, config 2), -14 (APOGEE-like H band,
           2e5-3e5 lines at 4-5x the line density, configs 1, 3, 4); -6 for the
           hand-sized test problems.
  masses U[12, 60] amu; band (molecule-like) species U[26, 28] amu
  microturbulence xi = 1 km/s
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# CODATA 2018, cgs.  Only used to build the input atmosphere (pressures to
# number densities); the synthesis constants live separately in each
# implementation.
_K_B = 1.380649e-16
_M_U = 1.66053906660e-24

N_DEPTH = 72
R_GRID = 300_000.0


@dataclasses.dataclass
class Atmosphere:
    """One star's depth structure, FP64, depth index 0 = top of the atmosphere."""
    teff: float
    logg: float
    m: np.ndarray          # [n_depth] column mass, g cm^-2 (increasing)
    T: np.ndarray          # [n_depth] K
    rho: np.ndarray        # [n_depth] g cm^-3
    n_e: np.ndarray        # [n_depth] cm^-3
    n_pert: np.ndarray     # [n_depth] cm^-3
    pop: np.ndarray        # [n_species, n_depth] n_s/U_s, cm^-3
    mass_amu: np.ndarray   # [n_species]
    xi_cms: float
    kappa0: np.ndarray     # [n_depth] continuum at 500 nm, cm^2 g^-1

    @property
    def n_depth(self) -> int:
        return int(self.m.shape[0])

    @property
    def n_species(self) -> int:
        return int(self.pop.shape[0])


@dataclasses.dataclass
class Grid:
    """Logarithmic synthesis grid lambda_i = lambda0 (1 + 1/R)^i (Eq. 1)."""
    lambda0_nm: float
    R_grid: float
    n_lambda: int


@dataclasses.dataclass
class LineList:
    """Structure-of-arrays line list in caller order (unsorted)."""
    lambda_nm: np.ndarray      # float64 [n_lines]
    log_gf: np.ndarray         # float32
    E_low_eV: np.ndarray       # float32
    log_gamma_rad: np.ndarray  # float32, log10 s^-1
    log_gamma4: np.ndarray     # float32, log10 cm^3 s^-1
    log_gamma6: np.ndarray     # float32, log10 cm^3 s^-1
    species: np.ndarray        # int32
    half_window: int           # W, grid points

    @property
    def n_lines(self) -> int:
        return int(self.lambda_nm.shape[0])

    def subset(self, idx: np.ndarray) -> "LineList":
        return LineList(self.lambda_nm[idx].copy(), self.log_gf[idx].copy(),
                        self.E_low_eV[idx].copy(), self.log_gamma_rad[idx].copy(),
                        self.log_gamma4[idx].copy(), self.log_gamma6[idx].copy(),
                        self.species[idx].copy(), self.half_window)


@dataclasses.dataclass
class Instrument:
    """Doppler shift, Gaussian broadening and Gaussian LSF onto detector pixels."""
    v_r_kms: float
    v_b_kms: float
    R_lsf: float
    pix_lambda_nm: np.ndarray  # float64 [n_pix]


@dataclasses.dataclass
class Problem:
    """One synthesis problem: atmosphere + grid + lines (+ instrument)."""
    name: str
    atmos: Atmosphere
    grid: Grid
    lines: LineList
    kappa_c: np.ndarray                 # float64 [n_depth, n_lambda]
    instrument: Optional[Instrument] = None
    elem_of_species: Optional[np.ndarray] = None   # int32 [n_species]
    n_elem: int = 0
    sigma_c: Optional[np.ndarray] = None   # float64 [n_depth, n_lambda] continuum scattering, or None

    @property
    def n_evals(self) -> int:
        """(line, lambda, depth) Voigt evaluations inside the clipped windows."""
        return int(window_points(self.grid, self.lines).sum()) * self.atmos.n_depth


def n_lambda_for(lmin_nm: float, lmax_nm: float, R: float = R_GRID) -> int:
    """Number of grid points spanning [lmin, lmax] (Eq. 2, exact form)."""
    return int(math.floor(math.log(lmax_nm / lmin_nm) / math.log1p(1.0 / R))) + 1


def center_index(grid: Grid, lambda_nm: np.ndarray) -> np.ndarray:
    """Integer centre placement i_l = floor(x_l + 1/2), x_l = ln(lambda_l/lambda_0)/ln r.

    This is the generator's own copy of the placement rule, used only to count
    work (``window_points``) and to pick sampled columns in tests.
    """
    x = np.log(lambda_nm / grid.lambda0_nm) / math.log1p(1.0 / grid.R_grid)
    return np.floor(x + 0.5).astype(np.int64)


def window_points(grid: Grid, lines: LineList) -> np.ndarray:
    """Grid points inside each line's window |i - i_l| <= W, clipped to the grid."""
    il = center_index(grid, lines.lambda_nm)
    lo = np.maximum(il - lines.half_window, 0)
    hi = np.minimum(il + lines.half_window, grid.n_lambda - 1)
    return np.maximum(hi - lo + 1, 0)


def grid_lambda_nm(grid: Grid) -> np.ndarray:
    return grid.lambda0_nm * np.exp(np.arange(grid.n_lambda) * math.log1p(1.0 / grid.R_grid))


# ----------------------------------------------------------------------------
# atmosphere
# ----------------------------------------------------------------------------

# mean log10 population share mu of the absorbing levels per workload (module docstring)
MU_OPTICAL = -9.5
MU_BROAD = -12.5
MU_HBAND = -14.0


def make_atmosphere(teff: float, logg: float, n_species: int, seed: int,
                    metallicity: float = 0.0, band_species=(), xi_kms: float = 1.0,
                    n_depth: int = N_DEPTH, log_abund_mean: float = -6.0) -> Atmosphere:
    rng = np.random.default_rng(seed)
    j = np.arange(n_depth)
    x = -6.875 + 0.125 * j if n_depth == 72 else np.linspace(-6.875, 2.0, n_depth)
    tau = 10.0 ** x
    T = (0.75 * teff ** 4 * (tau + 2.0 / 3.0)) ** 0.25
    g = 10.0 ** logg
    m_ref = 3.0 * 10.0 ** (-0.4 * (logg - 4.44))
    m = m_ref * tau ** 0.7
    P_gas = g * m
    P_e = 1e-4 * g * m_ref * tau * (teff / 5777.0) ** 4
    kT = _K_B * T
    n_e = P_e / kT
    n_pert = (P_gas - P_e) / kT
    n_tot = P_gas / kT
    rho = 1.3 * _M_U * P_gas / kT
    kappa0 = tau ** 0.3 / (0.7 * m_ref)

    log_f = rng.normal(log_abund_mean, 1.0, n_species)
    jitter = rng.normal(0.0, 0.1, (n_species, n_depth))
    U = 10.0 ** rng.uniform(0.0, 1.5, n_species)
    mass = rng.uniform(12.0, 60.0, n_species)
    for s in band_species:
        mass[s] = rng.uniform(26.0, 28.0)
    pop = (10.0 ** (log_f[:, None] + jitter + metallicity)) * n_tot[None, :] / U[:, None]
    return Atmosphere(teff=teff, logg=logg, m=m, T=T, rho=rho, n_e=n_e, n_pert=n_pert,
                      pop=pop, mass_amu=mass, xi_cms=xi_kms * 1e5, kappa0=kappa0)


def make_kappa_c(atmos: Atmosphere, grid: Grid) -> np.ndarray:
    lam = grid_lambda_nm(grid)
    return np.ascontiguousarray(atmos.kappa0[:, None] * (lam[None, :] / 500.0) ** -1.0)


# ----------------------------------------------------------------------------
# line lists
# ----------------------------------------------------------------------------

def _atomic_lines(rng, n, lam_lo, lam_hi, species_choices, centres="loguniform"):
    if centres == "loguniform":
        lam = np.exp(rng.uniform(math.log(lam_lo), math.log(lam_hi), n))
    elif centres == "inv_uniform":   # pdf ~ lambda^-2
        lam = 1.0 / rng.uniform(1.0 / lam_hi, 1.0 / lam_lo, n)
    else:
        raise ValueError(centres)
    log_gf = np.clip(rng.normal(-2.0, 1.5, n), -6.0, 1.0)
    E = rng.uniform(0.0, 10.0, n)
    sp = rng.choice(np.asarray(species_choices), n)
    g_rad = rng.normal(8.0, 0.5, n)
    g4 = rng.normal(-5.5, 0.5, n)
    g6 = rng.normal(-7.5, 0.5, n)
    return lam, log_gf, E, sp, g_rad, g4, g6


def _band_lines(rng, n_bands, per_band, spacing_nm, lam_lo, lam_hi, band_species):
    starts = rng.uniform(lam_lo, lam_hi - per_band * spacing_nm, n_bands)
    lam = (starts[:, None] + spacing_nm * np.arange(per_band)[None, :]).ravel()
    n = lam.size
    log_gf = rng.normal(-3.0, 1.0, n)
    E = rng.uniform(0.0, 3.0, n)
    sp = np.repeat(rng.choice(np.asarray(band_species), n_bands), per_band)
    g_rad = rng.normal(8.0, 0.5, n)
    g4 = rng.normal(-5.5, 0.5, n)
    g6 = rng.normal(-7.5, 0.5, n)
    return lam, log_gf, E, sp, g_rad, g4, g6


def _pack(parts, W) -> LineList:
    cols = [np.concatenate([p[k] for p in parts]) for k in range(7)]
    lam, log_gf, E, sp, g_rad, g4, g6 = cols
    return LineList(lambda_nm=lam.astype(np.float64), log_gf=log_gf.astype(np.float32),
                    E_low_eV=E.astype(np.float32), log_gamma_rad=g_rad.astype(np.float32),
                    log_gamma4=g4.astype(np.float32), log_gamma6=g6.astype(np.float32),
                    species=sp.astype(np.int32), half_window=int(W))


def apogee_pixels(n_pix: int = 8575) -> np.ndarray:
    """APOGEE-like detector grid: log10(lambda/A) = 4.179 + 6e-6 p."""
    return 10.0 ** (4.179 + 6e-6 * np.arange(n_pix)) / 10.0


# ----------------------------------------------------------------------------
# the five workloads (and scaled-down variants for element-wise parity)
# ----------------------------------------------------------------------------

def config0(seed: int = 0, n_lambda: int = 4000, n_lines: int = 2000, W: int = 1000) -> Problem:
    """Tiny forward: solar atmosphere, 4,000 points from 500 nm, 2,000 lines, W = 1,000."""
    n_species = 12
    atmos = make_atmosphere(5777.0, 4.44, n_species, seed, log_abund_mean=MU_OPTICAL)
    grid = Grid(500.0, R_GRID, n_lambda)
    lam_hi = float(grid_lambda_nm(grid)[-1])
    rng = np.random.default_rng(seed + 1000)
    lines = _pack([_atomic_lines(rng, n_lines, 500.0, lam_hi, np.arange(n_species))], W)
    return Problem("config0", atmos, grid, lines, make_kappa_c(atmos, grid))


def config1(seed: int = 1, lam_lo: float = 1500.0, lam_hi: float = 1700.0,
            n_bands: int = 133, per_band: int = 500, n_atomic: int = 133_500, W: int = 1500,
            n_pix: Optional[int] = 8575, name: str = "config1") -> Problem:
    """APOGEE-like window: Teff 4500, log g 2, 1500-1700 nm, 2e5 lines over 40 species
    (one third in 133 molecule-like bands of 500 lines at 0.02 nm spacing), W = 1,500,
    instrument v_r = 12.3 km/s, Gaussian LSF R = 22,500, 8,575 pixels."""
    n_species = 40
    band_sp = (36, 37, 38, 39)
    atmos = make_atmosphere(4500.0, 2.0, n_species, seed, band_species=band_sp, log_abund_mean=MU_HBAND)
    grid = Grid(lam_lo, R_GRID, n_lambda_for(lam_lo, lam_hi))
    rng = np.random.default_rng(seed + 1000)
    parts = [_atomic_lines(rng, n_atomic, lam_lo, lam_hi, np.arange(36))]
    if n_bands:
        parts.append(_band_lines(rng, n_bands, per_band, 0.02, lam_lo, lam_hi, band_sp))
    lines = _pack(parts, W)
    inst = None
    if n_pix:
        pix = apogee_pixels(8575)
        if lam_lo != 1500.0 or lam_hi != 1700.0:   # scaled variant: pixels 100 grid points inside
            margin = (1.0 + 1.0 / R_GRID) ** 100
            pix = pix[(pix > lam_lo * margin) & (pix < lam_hi / margin)][:n_pix]
        inst = Instrument(12.3, 0.0, 22_500.0, pix)
    elem = (np.arange(n_species) % 20).astype(np.int32)
    return Problem(name, atmos, grid, lines, make_kappa_c(atmos, grid), inst, elem, 20)


def config2(seed: int = 2, lam_lo: float = 300.0, lam_hi: float = 1000.0,
            n_lines: int = 3_000_000, W: int = 2000, R: float = R_GRID) -> Problem:
    """Broad optical: solar atmosphere, 300-1000 nm, 3e6 lines over 80 species with
    centre density proportional to lambda^-2, W = 2,000, full-resolution output
    (R_grid = 3e5 unless R is given)."""
    n_species = 80
    atmos = make_atmosphere(5777.0, 4.44, n_species, seed, log_abund_mean=MU_BROAD)
    grid = Grid(lam_lo, R, n_lambda_for(lam_lo, lam_hi, R))
    rng = np.random.default_rng(seed + 1000)
    lines = _pack([_atomic_lines(rng, n_lines, lam_lo, lam_hi, np.arange(n_species),
                                 centres="inv_uniform")], W)
    return Problem("config2", atmos, grid, lines, make_kappa_c(atmos, grid))


def config2_sweep_point(R: float = R_GRID, lam_hi: float = 1000.0, seed: int = 2, lam_lo: float = 300.0,
                        n_lines_full: int = 3_000_000) -> Problem:
    """One point of the scaling sweeps of Sec. 3.2 on the config-2 recipe: grid sampling
    R (the line windows keep their width in wavelength, W = 2,000 R / 3e5 grid points)
    and span lam_lo..lam_hi (the line density of the 300-1000 nm list, proportional to
    lambda^-2, so the list holds n_lines_full (1/lam_lo - 1/lam_hi) / (1/300 - 1/1000)
    lines)."""
    frac = (1.0 / lam_lo - 1.0 / lam_hi) / (1.0 / 300.0 - 1.0 / 1000.0)
    W = max(1, int(round(2000.0 * R / R_GRID)))
    return config2(seed=seed, lam_lo=lam_lo, lam_hi=lam_hi, n_lines=max(1, int(round(n_lines_full * frac))), W=W,
                   R=R)


def config3(seed: int = 3, lam_lo: float = 1500.0, lam_hi: float = 1700.0,
            n_bands: int = 80, per_band: int = 500, n_atomic: int = 80_000, W: int = 1500,
            n_pix: Optional[int] = 8575):
    """Differentiable calibration: config-1 grid and instrument with 1.2e5 lines.
    Returns (problem, truth) where truth holds the seeded Delta log gf ~ N(0, 0.1),
    Delta log gamma6 ~ N(0, 0.2) and the noise draw (seed 7, sigma = 1/200)."""
    prob = config1(seed=seed, lam_lo=lam_lo, lam_hi=lam_hi, n_bands=n_bands, per_band=per_band,
                   n_atomic=n_atomic, W=W, n_pix=n_pix, name="config3")
    rng = np.random.default_rng(7)
    nl = prob.lines.n_lines
    truth = {
        "dlog_gf": rng.normal(0.0, 0.1, nl).astype(np.float32),
        "dlog_gamma6": rng.normal(0.0, 0.2, nl).astype(np.float32),
        "noise": rng.normal(0.0, 1.0 / 200.0, prob.instrument.pix_lambda_nm.size
                            if prob.instrument is not None else prob.grid.n_lambda),
        "weight": 200.0 ** 2,
    }
    return prob, truth


def wavelength_slice(prob: Problem, lam_lo_nm: float, n_points: int) -> Problem:
    """The same problem restricted to n_points grid points starting at the first grid
    point >= lam_lo_nm: the grid keeps its step (lambda_0 moves to that point), the
    lines are those whose windows reach the slice, kappa_c is cut to the slice, and
    there is no instrument.  Pure data selection, used to time slow references on a
    bounded part of a workload."""
    g = prob.grid
    lnr = math.log1p(1.0 / g.R_grid)
    i0 = int(math.ceil(math.log(lam_lo_nm / g.lambda0_nm) / lnr - 1e-9))
    i0 = max(0, min(i0, g.n_lambda - 1))
    n = max(1, min(n_points, g.n_lambda - i0))
    grid = Grid(g.lambda0_nm * math.exp(i0 * lnr), g.R_grid, n)
    il = center_index(g, prob.lines.lambda_nm)
    W = prob.lines.half_window
    keep = np.nonzero((il + W >= i0) & (il - W <= i0 + n - 1))[0]
    sig = None if prob.sigma_c is None else np.ascontiguousarray(prob.sigma_c[:, i0:i0 + n])
    return Problem(prob.name + "-slice", prob.atmos, grid, prob.lines.subset(keep),
                   np.ascontiguousarray(prob.kappa_c[:, i0:i0 + n]), None, prob.elem_of_species, prob.n_elem, sig)


def with_scattering_batch(batch: "Batch", r0: float = 1.0, lam_ref_nm: float = 400.0) -> "Batch":
    """with_scattering applied to every star of a batch (each star's own kappa_c and layers)."""
    sig = [with_scattering(batch.star(k), r0, lam_ref_nm).sigma_c for k in range(batch.n_stars)]
    return dataclasses.replace(batch, name=batch.name + "+scat", sigma_c=sig)


def with_scattering(prob: Problem, r0: float = 1.0, lam_ref_nm: float = 400.0) -> Problem:
    """The same problem with a continuum scattering coefficient (Eq. 6 with sigma_c > 0):
    sigma_c = kappa_c r0 (lambda / lam_ref)^-4 / (1 + tau_d), tau_d = 10^(-6.875 + 0.125 d)
    the recipe's reference optical depth of layer d (linspace of the same range for other
    layer counts): Rayleigh-like in wavelength, strongest in the upper layers, negligible
    where the continuum thermalises."""
    nd = prob.atmos.n_depth
    x = -6.875 + 0.125 * np.arange(nd) if nd == 72 else np.linspace(-6.875, 2.0, nd)
    lam = grid_lambda_nm(prob.grid)
    ratio = r0 * (lam[None, :] / lam_ref_nm) ** -4.0 / (1.0 + 10.0 ** x[:, None])
    return dataclasses.replace(prob, name=prob.name + "+scat", sigma_c=np.ascontiguousarray(prob.kappa_c * ratio))


def small_config1(n_lambda_span_nm: float = 2.0, lines_scale: float = 0.01, seed: int = 11,
                  W: int = 1500, with_instrument: bool = True) -> Problem:
    """Scaled-down config 1 for element-wise parity: same recipe, a ~2 nm slice."""
    lam_lo = 1600.0
    lam_hi = lam_lo + n_lambda_span_nm
    frac = n_lambda_span_nm / 200.0
    n_atomic = max(8, int(round(133_500 * frac)))
    n_bands = max(1, int(round(133 * frac))) if n_lambda_span_nm > 10.5 else 0
    return config1(seed=seed, lam_lo=lam_lo, lam_hi=lam_hi, n_bands=n_bands, per_band=500,
                   n_atomic=n_atomic, W=W, n_pix=8575 if with_instrument else None,
                   name="config1-small")


def config4_stars(seed: int = 4, n_stars: int = 64):
    """Per-star labels for the batched workload: Teff ~ U[3500, 7000], log g ~ U[1, 5],
    [M/H] ~ U[-2, 0.5], plus line-count draws N_k = round(exp U[ln 2e4, ln 3e5])."""
    rng = np.random.default_rng(seed)
    teff = rng.uniform(3500.0, 7000.0, n_stars)
    logg = rng.uniform(1.0, 5.0, n_stars)
    mh = rng.uniform(-2.0, 0.5, n_stars)
    nk = np.round(np.exp(rng.uniform(math.log(2e4), math.log(3e5), n_stars))).astype(np.int64)
    return teff, logg, mh, nk


@dataclasses.dataclass
class Batch:
    """Many stars on one grid with one master line list; star k uses the master
    lines ``subsets[k]`` (indices, any order).  Corrections are per master line."""
    name: str
    atmos: list                 # [S] Atmosphere (shared n_depth and species set)
    grid: Grid
    lines: LineList             # master list, caller order
    kappa_c: list               # [S] float64 [n_depth, n_lambda]
    subsets: list               # [S] int32 index arrays into the master list
    instrument: Optional[Instrument] = None
    elem_of_species: Optional[np.ndarray] = None
    n_elem: int = 0
    sigma_c: Optional[list] = None  # [S] float64 [n_depth, n_lambda] continuum scattering, or None

    @property
    def n_stars(self) -> int:
        return len(self.atmos)

    def star(self, k: int) -> Problem:
        """Star k as a single-star problem (its own line subset, caller order kept)."""
        return Problem("%s[%d]" % (self.name, k), self.atmos[k], self.grid, self.lines.subset(self.subsets[k]),
                       self.kappa_c[k], self.instrument, self.elem_of_species, self.n_elem,
                       None if self.sigma_c is None else self.sigma_c[k])

    @property
    def n_evals(self) -> int:
        wp = window_points(self.grid, self.lines)
        return int(sum(int(wp[s].sum()) for s in self.subsets)) * self.atmos[0].n_depth


def _tau1_layer(atmos: Atmosphere) -> int:
    """Layer whose recipe optical depth is closest to tau = 1 (log tau = 0)."""
    nd = atmos.n_depth
    x = -6.875 + 0.125 * np.arange(nd) if nd == 72 else np.linspace(-6.875, 2.0, nd)
    return int(np.argmin(np.abs(x)))


def strength_proxy(atmos: Atmosphere, lines: LineList) -> np.ndarray:
    """Line-strength proxy log gf + log10(pop_s/rho at tau = 1) - 5040 E_low / T(tau = 1),
    a simplified keep test (lines selected by strength, Sec. 2.2)."""
    j = _tau1_layer(atmos)
    pr = np.log10(np.maximum(atmos.pop[:, j], 1e-300) / atmos.rho[j])
    return lines.log_gf.astype(np.float64) + pr[lines.species] - 5040.0 * lines.E_low_eV.astype(np.float64) / atmos.T[j]


def _batch_atmospheres(teff, logg, mh, n_species, band_species, chem_seed, grid):
    """One atmosphere per star from the shared recipe: the same species set (abundance
    pattern, partition functions, masses: one chemistry seed) scaled by [M/H]."""
    atm = [make_atmosphere(float(t), float(g), n_species, chem_seed, metallicity=float(z),
                           band_species=band_species, log_abund_mean=MU_HBAND) for t, g, z in zip(teff, logg, mh)]
    return atm, [make_kappa_c(a, grid) for a in atm]


def config4(seed: int = 4, n_stars: int = 64, n_atomic: int = 200_000, n_bands: int = 200,
            per_band: int = 500, lam_lo: float = 1500.0, lam_hi: float = 1700.0, W: int = 1500,
            n_pix: Optional[int] = 8575, nk_scale: float = 1.0) -> Batch:
    """Batched many-star workload: 64 stars with seeded (Teff, log g, [M/H]) on the
    config-1 grid and instrument; a master list of 3e5 lines (config-1 recipe: 2e5
    atomic + 200 bands of 500); star k keeps its top-N_k lines by the strength proxy,
    N_k = round(exp U[ln 2e4, ln 3e5]) (times nk_scale, for scaled-down variants)."""
    base = config1(seed=seed, lam_lo=lam_lo, lam_hi=lam_hi, n_bands=n_bands, per_band=per_band,
                   n_atomic=n_atomic, W=W, n_pix=n_pix, name="config4")
    teff, logg, mh, nk = config4_stars(seed, n_stars)
    atm, kc = _batch_atmospheres(teff, logg, mh, base.atmos.n_species, (36, 37, 38, 39), seed + 500, base.grid)
    nl = base.lines.n_lines
    subsets = []
    for a, n in zip(atm, nk):
        n = int(min(nl, max(1, round(n * nk_scale))))
        order = np.argsort(-strength_proxy(a, base.lines), kind="stable")
        subsets.append(np.sort(order[:n]).astype(np.int32))
    return Batch("config4", atm, base.grid, base.lines, kc, subsets, base.instrument, base.elem_of_species,
                 base.n_elem)


def config4_joint(seed: int = 4, n_common: int = 100_000, **kw):
    """Joint two-star calibration step: solar-like (5777, 4.44, 0.0) and giant-like
    (4286, 1.66, -0.52) stars on the config-4 master list, both using the n_common
    lines with the highest mean strength proxy, shared corrections.  Returns
    (batch, truth) with truth corrections Delta log gf ~ N(0, 0.1), Delta log gamma6
    ~ N(0, 0.2) on the master list and per-star pixel noise (seed 7, sigma 1/200)."""
    full = config4(seed=seed, n_stars=1, **kw)
    teff, logg, mh = np.array([5777.0, 4286.0]), np.array([4.44, 1.66]), np.array([0.0, -0.52])
    atm, kc = _batch_atmospheres(teff, logg, mh, full.atmos[0].n_species, (36, 37, 38, 39), seed + 500, full.grid)
    score = 0.5 * (strength_proxy(atm[0], full.lines) + strength_proxy(atm[1], full.lines))
    n = int(min(n_common, full.lines.n_lines))
    common = np.sort(np.argsort(-score, kind="stable")[:n]).astype(np.int32)
    b = Batch("config4-joint", atm, full.grid, full.lines, kc, [common, common.copy()], full.instrument,
              full.elem_of_species, full.n_elem)
    rng = np.random.default_rng(7)
    nl = full.lines.n_lines
    n_out = full.instrument.pix_lambda_nm.size if full.instrument is not None else full.grid.n_lambda
    truth = {"dlog_gf": rng.normal(0.0, 0.1, nl).astype(np.float32),
             "dlog_gamma6": rng.normal(0.0, 0.2, nl).astype(np.float32),
             "noise": rng.normal(0.0, 1.0 / 200.0, (2, n_out)),
             "weight": 200.0 ** 2}
    return b, truth


HC_EV_CM = 1.239841984e-4     # h c in eV cm: 1 cm^-1 of level energy in eV (CODATA 2018)


def config4_joint_grouped(seed: int = 4, n_complexes: int = 25_281, n_records: int = 42_886, **kw):
    """Four-parameter grouped calibration workload (Sec. 6: 42,886 catalog records in
    25,281 correction groups over 1500-1700 nm): the solar-like and giant-like stars of
    config4_joint on a list of component complexes.  The n_complexes strongest lines of
    the config-4 master list (mean strength proxy of the two stars) each get k - 1
    companions (k - 1 drawn so that the list holds n_records lines) of the same species,
    within +-0.02 nm and +-1 cm^-1 of the parent, the parent's gf split evenly over the k
    components and its damping constants copied (hyperfine- or isotope-like structure).
    Returns (batch, truth): both stars use every record; truth holds "complex_of_line"
    [n_records], per-complex corrections "x" [4][n_complexes] (Delta log gf ~ N(0, 0.1),
    Delta log gamma_rad, gamma_4 ~ N(0, 0.3), Delta log gamma_6 ~ N(0, 0.2)), the per-line
    "strength" (mean strength proxy, FP32) for the grouping pass, per-star pixel noise
    (sigma 1/200) and the weight 200^2."""
    full = config4(seed=seed, n_stars=1, **kw)
    teff, logg, mh = np.array([5777.0, 4286.0]), np.array([4.44, 1.66]), np.array([0.0, -0.52])
    atm, kc = _batch_atmospheres(teff, logg, mh, full.atmos[0].n_species, (36, 37, 38, 39), seed + 500, full.grid)
    score = 0.5 * (strength_proxy(atm[0], full.lines) + strength_proxy(atm[1], full.lines))
    parents = np.sort(np.argsort(-score, kind="stable")[:n_complexes])
    rng = np.random.default_rng(seed + 900)
    extra = np.bincount(rng.integers(0, parents.size, max(n_records - parents.size, 0)), minlength=parents.size)
    k = 1 + extra
    cid = np.repeat(np.arange(parents.size), k)
    src = parents[cid]
    first = np.concatenate([[True], cid[1:] != cid[:-1]])
    L = full.lines.subset(src)
    n = src.size
    dl = rng.uniform(-0.02, 0.02, n)
    dE = rng.uniform(-1.0, 1.0, n) * HC_EV_CM
    L.lambda_nm = np.where(first, L.lambda_nm, L.lambda_nm + dl)
    L.E_low_eV = np.where(first, L.E_low_eV, np.maximum(L.E_low_eV.astype(np.float64) + dE, 0.0)).astype(np.float32)
    L.log_gf = (L.log_gf.astype(np.float64) - np.log10(k[cid])).astype(np.float32)
    strength = (0.5 * (strength_proxy(atm[0], L) + strength_proxy(atm[1], L))).astype(np.float32)
    allk = np.arange(n, dtype=np.int32)
    b = Batch("config4-joint-grouped", atm, full.grid, L, kc, [allk, allk.copy()], full.instrument,
              full.elem_of_species, full.n_elem)
    n_out = full.instrument.pix_lambda_nm.size if full.instrument is not None else full.grid.n_lambda
    x = np.stack([rng.normal(0.0, 0.1, parents.size), rng.normal(0.0, 0.3, parents.size),
                  rng.normal(0.0, 0.3, parents.size), rng.normal(0.0, 0.2, parents.size)]).astype(np.float32)
    truth = {"complex_of_line": cid.astype(np.int32), "x": x, "strength": strength,
             "noise": rng.normal(0.0, 1.0 / 200.0, (2, n_out)), "weight": 200.0 ** 2}
    return b, truth


def small_batch(n_stars: int = 3, span_nm: float = 2.0, seed: int = 21, W: int = 1500,
                with_instrument: bool = True) -> Batch:
    """Scaled-down config 4 for element-wise parity: a ~2 nm slice of the config-1
    recipe, stars with uneven line subsets (one empty-ish, one full, one random)."""
    lam_lo = 1600.0
    lam_hi = lam_lo + span_nm
    frac = span_nm / 200.0
    base = config1(seed=seed, lam_lo=lam_lo, lam_hi=lam_hi, n_bands=0, per_band=500,
                   n_atomic=max(8, int(round(200_000 * frac))), W=W,
                   n_pix=8575 if with_instrument else None, name="batch-small")
    teff, logg, mh, _ = config4_stars(seed, n_stars)
    atm, kc = _batch_atmospheres(teff, logg, mh, base.atmos.n_species, (36, 37, 38, 39), seed + 500, base.grid)
    nl = base.lines.n_lines
    rng = np.random.default_rng(seed + 9)
    subsets = []
    for k in range(n_stars):
        if k % 3 == 0:
            idx = np.arange(nl)
        elif k % 3 == 1:
            idx = np.sort(rng.choice(nl, max(1, nl // 7), replace=False))
        else:
            idx = np.sort(rng.choice(nl, nl // 2, replace=False))
        subsets.append(idx.astype(np.int32))
    return Batch("batch-small", atm, base.grid, base.lines, kc, subsets, base.instrument, base.elem_of_species,
                 base.n_elem)
