"""Pins of the oracle's line opacity (Sec. 2.1, Eqs. 1, 4, 5)."""
import numpy as np
import pytest
from scipy.special import wofz

from paper_2607_24141_gb300 import inputs as I
from tiny import tiny_problem

# CODATA 2018 cgs, typed independently of the oracle source
H_ = 6.62607015e-27
K_ = 1.380649e-16
C_ = 2.99792458e10
E_ = 4.80320471e-10
ME = 9.1093837015e-28
EV = 1.602176634e-12
AMU = 1.66053906660e-24


def centre_ratios(prob):
    """Per (line, depth): the peak of the line's term at its centre grid point, bounded with
    H <= 1, over the continuum there: stim(ic, d) A_ld / kappa_c(ic, d), ic = i_l clipped."""
    at, ll, g = prob.atmos, prob.lines, prob.grid
    r = 1.0 + 1.0 / g.R_grid
    out = np.zeros((ll.n_lines, at.n_depth))
    for l in range(ll.n_lines):
        il = int(np.floor(np.log(ll.lambda_nm[l] / g.lambda0_nm) / np.log(r) + 0.5))
        ic = min(max(il, 0), g.n_lambda - 1)
        nu_c = C_ / (g.lambda0_nm * 1e-7 * r ** ic)
        nu_l = C_ / (ll.lambda_nm[l] * 1e-7)
        sp = ll.species[l]
        for d in range(at.n_depth):
            T = at.T[d]
            dnu = nu_l * np.sqrt(2 * K_ * T / (at.mass_amu[sp] * AMU) + at.xi_cms ** 2) / C_
            A = (np.pi * E_ ** 2 / (ME * C_)) * 10.0 ** float(ll.log_gf[l]) * at.pop[sp, d] / at.rho[d] \
                * np.exp(-float(ll.E_low_eV[l]) * EV / (K_ * T)) / (np.sqrt(np.pi) * dnu)
            out[l, d] = (1.0 - np.exp(-H_ * nu_c / (K_ * T))) * A / prob.kappa_c[d, ic]
    return out


def brute_kappa(prob, eta=0.0):
    """Triple loop over (lambda, depth, line), written in frequency variables; with eta > 0
    only the (line, depth) pairs whose centre ratio reaches eta."""
    at, ll, g = prob.atmos, prob.lines, prob.grid
    r = 1.0 + 1.0 / g.R_grid
    out = np.zeros((at.n_depth, g.n_lambda))
    keep = centre_ratios(prob) >= eta if eta > 0 else np.ones((ll.n_lines, at.n_depth), bool)
    il = [int(np.floor(np.log(ll.lambda_nm[l] / g.lambda0_nm) / np.log(r) + 0.5)) for l in range(ll.n_lines)]
    for i in range(g.n_lambda):
        lam_i = g.lambda0_nm * 1e-7 * r ** i
        nu = C_ / lam_i
        for d in range(at.n_depth):
            T = at.T[d]
            s = 0.0
            for l in range(ll.n_lines):
                if abs(i - il[l]) > ll.half_window or not keep[l, d]:
                    continue
                sp = ll.species[l]
                nu_l = C_ / (ll.lambda_nm[l] * 1e-7)
                dv = np.sqrt(2 * K_ * T / (at.mass_amu[sp] * AMU) + at.xi_cms ** 2)
                dnu = nu_l * dv / C_
                gam = 10.0 ** float(ll.log_gamma_rad[l]) + 10.0 ** float(ll.log_gamma4[l]) * at.n_e[d] \
                    + 10.0 ** float(ll.log_gamma6[l]) * at.n_pert[d]
                a = gam / (4 * np.pi * dnu)
                v = (nu - nu_l) / dnu
                phi = wofz(v + 1j * a).real / (np.sqrt(np.pi) * dnu)
                s += (np.pi * E_ ** 2 / (ME * C_)) * 10.0 ** float(ll.log_gf[l]) * at.pop[sp, d] / at.rho[d] \
                    * np.exp(-float(ll.E_low_eV[l]) * EV / (K_ * T)) * phi
            out[d, i] = s * (1.0 - np.exp(-H_ * nu / (K_ * T)))
    return out


def test_kappa_matches_brute_force(oracle):
    prob = tiny_problem()
    ref = brute_kappa(prob)
    got = oracle.kappa_line(prob)
    m = ref > 0
    assert np.all((got > 0) == m)
    # both sides form the frequency offset in FP64 (the brute force from lambda_0 r**i, whose
    # rounding grows with i): each carries the ~1e-10 conditioning of a Gaussian core
    # (test_kappa_against_extended_precision_brute_force)
    assert np.max(np.abs(got[m] / ref[m] - 1)) < 2e-9


def test_kappa_column_subset_equals_full(oracle):
    prob = tiny_problem(n_lambda=80, n_lines=10, seed=9)
    full = oracle.kappa_line(prob)
    cols = np.array([0, 7, 33, 79])
    sub = oracle.kappa_line(prob, cols)
    assert np.array_equal(sub, full[:, cols])


def test_window_rule_and_dropped_lines(oracle):
    prob = tiny_problem(n_lambda=50, n_lines=1, W=5, seed=1)
    lam = I.grid_lambda_nm(prob.grid)
    # integer centre placement i_l = floor(x_l + 1/2), window |i - i_l| <= W
    for x, (lo, hi) in [(10.6, (6, 16)), (10.4, (5, 15)), (2.2, (0, 7))]:
        prob.lines.lambda_nm[:] = prob.grid.lambda0_nm * np.exp(x * np.log1p(1 / prob.grid.R_grid))
        nz = np.nonzero(oracle.kappa_line(prob)[0] > 0)[0]
        assert nz.min() == lo and nz.max() == hi
    # a line whose window misses the grid contributes nothing
    prob.lines.lambda_nm[:] = lam[-1] * np.exp(7 * np.log1p(1 / prob.grid.R_grid))
    assert np.all(oracle.kappa_line(prob) == 0)


def test_integrated_line_strength(oracle):
    """Int kappa dnu over an isolated weak line = (pi e^2/m c) gf n/(rho U) e^{-E/kT}
    times the fraction of the normalised profile inside the window (Eq. 4, Int phi dnu = 1)."""
    W = 3000
    prob = tiny_problem(n_lambda=2 * W + 1, n_depth=2, n_lines=1, W=W, seed=2)
    lam = I.grid_lambda_nm(prob.grid)
    prob.lines.lambda_nm[:] = lam[W]
    at, ll = prob.atmos, prob.lines
    k = oracle.kappa_line(prob)
    lnr = np.log1p(1 / prob.grid.R_grid)
    nu = C_ / (lam * 1e-7)
    sp = ll.species[0]
    for d in range(at.n_depth):
        T = at.T[d]
        stim = 1.0 - np.exp(-H_ * nu / (K_ * T))
        integral = np.sum(k[d] / stim * nu * lnr)       # Int dnu = Int nu dln(nu)
        S = (np.pi * E_ ** 2 / (ME * C_)) * 10.0 ** float(ll.log_gf[0]) * at.pop[sp, d] / at.rho[d] \
            * np.exp(-float(ll.E_low_eV[0]) * EV / (K_ * T))
        nu_l = nu[W]
        dv = np.sqrt(2 * K_ * T / (at.mass_amu[sp] * AMU) + at.xi_cms ** 2)
        dnu = nu_l * dv / C_
        gam = 10.0 ** float(ll.log_gamma_rad[0]) + 10.0 ** float(ll.log_gamma4[0]) * at.n_e[d] \
            + 10.0 ** float(ll.log_gamma6[0]) * at.n_pert[d]
        a = gam / (4 * np.pi * dnu)
        v_hi = (nu[0] - nu_l) / dnu                  # window edges in Doppler units
        v_lo = (nu_l - nu[-1]) / dnu
        tail = a / np.pi * (1 / v_hi + 1 / v_lo)     # Lorentz wings outside the window
        assert abs(integral / (S * (1 - tail)) - 1) < 1e-6


def test_abundance_and_gf_corrections_scale(oracle):
    prob = tiny_problem(seed=4)
    base = oracle.kappa_line(prob)
    nl = prob.lines.n_lines
    # Delta log gf = c for every line scales kappa by 10^c; Delta [X/H] = c likewise (Eq. 10)
    k1 = oracle.kappa_line(prob, corrections={"dlog_gf": np.full(nl, 0.3)})
    assert np.allclose(k1, base * 10 ** 0.3, rtol=1e-13, atol=0)
    k2 = oracle.kappa_line(prob, corrections={"dabund": np.full(prob.n_elem, -0.2)})
    assert np.allclose(k2, base * 10 ** -0.2, rtol=1e-13, atol=0)


def test_centre_test_matches_brute_force(oracle):
    """Continuum-referenced centre test: eta strictly between two pair ratios, so that no
    pair sits on the threshold; about half of the (line, depth) pairs are rejected."""
    prob = tiny_problem(seed=4)
    ratios = np.unique(centre_ratios(prob))
    k = ratios.size // 2
    eta = float(np.sqrt(ratios[k - 1] * ratios[k]))
    ref = brute_kappa(prob, eta)
    got = oracle.kappa_line(prob, corrections={"centre_eta": eta})
    full = oracle.kappa_line(prob)
    assert np.all((got > 0) == (ref > 0))
    m = ref > 0
    # both sides form the frequency offset in FP64 (the brute force from lambda_0 r**i, whose
    # rounding grows with i): each carries the ~1e-10 conditioning of a Gaussian core
    # (test_kappa_against_extended_precision_brute_force)
    assert np.max(np.abs(got[m] / ref[m] - 1)) < 2e-9
    assert np.any(got < full * (1 - 1e-6))          # the cut removed something


def test_centre_test_limits(oracle):
    prob = tiny_problem(seed=5)
    full = oracle.forward(prob)
    off = oracle.forward(prob, {"centre_eta": 0.0})
    assert np.array_equal(off["kline"], full["kline"]) and np.array_equal(off["f"], full["f"])
    none = oracle.forward(prob, {"centre_eta": 1e300})
    assert np.all(none["kline"] == 0.0)
    assert np.array_equal(none["F"], none["Fc"])


@pytest.mark.parametrize("shift,W", [(0, 20), (150, 400)])
def test_kappa_against_extended_precision_brute_force(oracle, shift, W):
    """The line sum against the same triple loop in 30-digit arithmetic (mpmath: grid
    wavelengths lambda_0 (1 + 1/R)^i exact, frequency offsets, Doppler widths, the
    Faddeeva function w(z) = exp(-z^2) erfc(-iz)), cell by cell within the FP64
    conditioning of the oracle's own arithmetic: 4e-14 relative for the Voigt function
    and the products of Eqs. 4-5, plus each term's sensitivity to its frequency offset
    v = (lambda_l/lambda_i - 1) c/dv_D times three roundings of lambda_l/lambda_i - 1
    (|dH/dv| = 2 |v H - a L|).  lambda_l/lambda_i - 1 carries an absolute rounding of
    ~4e-16, i.e. a relative one of 4e-16 / |u|: in a Gaussian core at |v| ~ 3 the bound
    reaches ~1e-10, and 75 Doppler widths out in a damping wing (the second case, every
    line moved 150 grid points off the grid, W = 400) still ~2e-12; a uniform 1e-13 is
    below what FP64 offsets allow.  The oracle sits at 0.6-0.7 of the bound."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    prob = tiny_problem(seed=12, W=W)
    prob.lines.lambda_nm[:] *= (1.0 + 1.0 / prob.grid.R_grid) ** shift
    at, ll, g = prob.atmos, prob.lines, prob.grid
    got = oracle.kappa_line(prob)
    r = 1 + 1 / mp.mpf(g.R_grid)
    lnr = np.log1p(1.0 / g.R_grid)
    il = [int(np.floor(np.log(ll.lambda_nm[l] / g.lambda0_nm) / lnr + 0.5)) for l in range(ll.n_lines)]
    C, K, E, MEc, EV_, AMU_ = (mp.mpf(x) for x in (C_, K_, E_, ME * C_, EV, AMU))
    H_ = mp.mpf(6.62607015e-27)
    pref = mp.pi * E ** 2 / MEc
    n_tight = n_cells = 0
    worst = used = 0.0
    for i in range(g.n_lambda):
        lam_i = mp.mpf(g.lambda0_nm) * mp.mpf("1e-7") * r ** i
        nu = C / lam_i
        for d in range(at.n_depth):
            T = mp.mpf(at.T[d])
            s, bound_v = mp.mpf(0), mp.mpf(0)
            for l in range(ll.n_lines):
                if abs(i - il[l]) > ll.half_window:
                    continue
                sp = int(ll.species[l])
                lam_l = mp.mpf(ll.lambda_nm[l]) * mp.mpf("1e-7")
                nu_l = C / lam_l
                dv = mp.sqrt(2 * K * T / (mp.mpf(at.mass_amu[sp]) * AMU_) + mp.mpf(at.xi_cms) ** 2)
                dnu = nu_l * dv / C
                gam = (mp.mpf(10) ** mp.mpf(float(ll.log_gamma_rad[l])) + mp.mpf(10) ** mp.mpf(float(ll.log_gamma4[l]))
                       * mp.mpf(at.n_e[d]) + mp.mpf(10) ** mp.mpf(float(ll.log_gamma6[l])) * mp.mpf(at.n_pert[d]))
                a = gam / (4 * mp.pi * dnu)
                v = (nu - nu_l) / dnu
                z = mp.mpc(v, a)
                w = mp.exp(-z * z) * mp.erfc(-1j * z)
                A = (pref * mp.mpf(10) ** mp.mpf(float(ll.log_gf[l])) * mp.mpf(at.pop[sp, d]) / mp.mpf(at.rho[d])
                     * mp.exp(-mp.mpf(float(ll.E_low_eV[l])) * EV_ / (K * T)) / (mp.sqrt(mp.pi) * dnu))
                s += A * mp.re(w)
                dHdv = abs(2 * (v * mp.re(w) - a * mp.im(w)))
                bound_v += A * dHdv * (3 * mp.mpf(2) ** -53) * C / dv
            if s == 0:
                assert got[d, i] == 0.0
                continue
            stim = 1 - mp.exp(-H_ * nu / (K * T))
            ref = float(s * stim)
            bound = 4e-14 * abs(ref) + float(bound_v * stim)
            n_cells += 1
            n_tight += bound < 1e-13 * abs(ref)
            assert abs(got[d, i] - ref) <= bound, (i, d, got[d, i], ref, bound / abs(ref))
            worst = max(worst, abs(got[d, i] / ref - 1))
            used = max(used, abs(got[d, i] - ref) / bound)
    print("cells %d, of which %d with a bound below 1e-13 relative; largest relative error %.2g, "
          "largest fraction of its bound %.2g" % (n_cells, n_tight, worst, used))
    assert n_cells > 100
