"""Tiny hand-sized problems for the oracle pins and the element-wise GPU parity."""
import numpy as np

from paper_2607_24141_gb300 import inputs as I


def tiny_problem(n_lambda=64, n_depth=3, n_lines=8, W=20, seed=5, lam0=600.0, n_species=3,
                 instrument=False, E_max=3.0):
    atmos = I.make_atmosphere(5000.0, 4.0, n_species, seed, n_depth=n_depth)
    grid = I.Grid(lam0, I.R_GRID, n_lambda)
    lam = I.grid_lambda_nm(grid)
    rng = np.random.default_rng(seed + 17)
    # centres spread over (and slightly beyond) the grid so some windows are clipped
    lo, hi = lam[0] * (1 - 10 / I.R_GRID), lam[-1] * (1 + 10 / I.R_GRID)
    lines = I.LineList(
        lambda_nm=np.exp(rng.uniform(np.log(lo), np.log(hi), n_lines)),
        log_gf=rng.normal(-1.0, 1.0, n_lines).astype(np.float32),
        E_low_eV=rng.uniform(0.0, E_max, n_lines).astype(np.float32),
        log_gamma_rad=rng.normal(8.0, 0.5, n_lines).astype(np.float32),
        log_gamma4=rng.normal(-5.5, 0.5, n_lines).astype(np.float32),
        log_gamma6=rng.normal(-7.5, 0.5, n_lines).astype(np.float32),
        species=rng.integers(0, n_species, n_lines).astype(np.int32),
        half_window=W)
    inst = None
    if instrument:
        sig = 1.0 / (2 * np.sqrt(2 * np.log(2)) * 22500.0) / np.log1p(1 / I.R_GRID)
        i_lo, i_hi = int(6 * sig), n_lambda - 1 - int(6 * sig)
        pix = lam[i_lo] * np.exp(np.arange(0, (i_hi - i_lo) * np.log1p(1 / I.R_GRID),
                                           1.0 / 22500.0 / 3.0))
        inst = I.Instrument(12.3, 0.0, 22500.0, pix[pix < lam[i_hi]])
    elem = (np.arange(n_species) % 2).astype(np.int32)
    return I.Problem("tiny", atmos, grid, lines, I.make_kappa_c(atmos, grid), inst, elem, 2)
