"""Vectorised numpy statement of the centre-test ratio (a third implementation, beside
the oracle's and the device's, used to count kept pairs in the tests): per (line, depth),
the peak of the line's term at its centre grid point bounded with H <= 1, over the
continuum there."""
import numpy as np

H_ = 6.62607015e-27
K_ = 1.380649e-16
C_ = 2.99792458e10
E_ = 4.80320471e-10
ME = 9.1093837015e-28
EV = 1.602176634e-12
AMU = 1.66053906660e-24


def centre_ratios(prob, corrections=None):
    at, ll, g = prob.atmos, prob.lines, prob.grid
    corr = corrections or {}
    lnr = np.log1p(1.0 / g.R_grid)
    il = np.floor(np.log(ll.lambda_nm / g.lambda0_nm) / lnr + 0.5).astype(np.int64)
    ic = np.clip(il, 0, g.n_lambda - 1)
    nu_c = C_ / (g.lambda0_nm * 1e-7 * np.exp(ic * lnr))
    nu_l = C_ / (ll.lambda_nm * 1e-7)
    sp = ll.species
    T = at.T[None, :]
    dnu = nu_l[:, None] * np.sqrt(2 * K_ * T / (at.mass_amu[sp][:, None] * AMU) + at.xi_cms ** 2) / C_
    gf = 10.0 ** (ll.log_gf.astype(np.float64) + np.asarray(corr.get("dlog_gf", 0.0), np.float64))
    dab = 0.0
    if corr.get("dabund") is not None:
        dab = np.asarray(corr["dabund"], np.float64)[prob.elem_of_species[sp]][:, None]
    pop = at.pop[sp, :] * 10.0 ** dab
    A = (np.pi * E_ ** 2 / (ME * C_)) * gf[:, None] * pop / at.rho[None, :] \
        * np.exp(-ll.E_low_eV.astype(np.float64)[:, None] * EV / (K_ * T)) / (np.sqrt(np.pi) * dnu)
    stim = 1.0 - np.exp(-H_ * nu_c[:, None] / (K_ * T))
    return stim * A / prob.kappa_c[:, ic].T
