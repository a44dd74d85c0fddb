"""Pins of the oracle's instrument stage (Sec. 7: shift S(v_r), broadening B(v_b),
LSF + sampling K, applied to F and F_c before the ratio, Eq. 9)."""
import numpy as np

from paper_2607_24141_gb300 import inputs as I
from tiny import tiny_problem

C_KMS = 2.99792458e5


def setup(n_lambda=600, v_r=12.3, v_b=0.0, R=22500.0):
    prob = tiny_problem(n_lambda=n_lambda, n_lines=0)
    lam = I.grid_lambda_nm(prob.grid)
    pix = np.geomspace(lam[100], lam[-100], 120)
    return prob, I.Instrument(v_r, v_b, R, pix)


def test_constant_spectrum_stays_constant(oracle):
    prob, inst = setup()
    taps = oracle.instrument_taps(prob, inst)
    out = oracle.apply_taps(*taps, np.full(prob.grid.n_lambda, 3.25))
    assert np.max(np.abs(out / 3.25 - 1)) < 1e-14


def test_kernel_moments_and_shift_sign(oracle):
    """Each row is a Gaussian in ln(lambda) centred on the rest wavelength
    lambda_p/(1 + v_r/c) with sigma^2 = sigma_LSF^2 + (v_b/c)^2, sigma_LSF = 1/(2.3548 R)."""
    for v_r, v_b in [(12.3, 0.0), (-40.0, 3.0)]:
        prob, inst = setup(v_r=v_r, v_b=v_b)
        tap0, ntap, w = oracle.instrument_taps(prob, inst)
        lam = I.grid_lambda_nm(prob.grid)
        sig = np.sqrt((1 / (2 * np.sqrt(2 * np.log(2)) * inst.R_lsf)) ** 2 + (v_b / C_KMS) ** 2)
        for p in range(0, inst.pix_lambda_nm.size, 7):
            idx = tap0[p] + np.arange(ntap[p])
            wk = w[p, :ntap[p]]
            lnl = np.log(lam[idx])
            mean = np.sum(wk * lnl)
            var = np.sum(wk * (lnl - mean) ** 2)
            # redshift (v_r > 0) means a pixel sees bluer rest-frame light
            assert abs(mean - np.log(inst.pix_lambda_nm[p] / (1 + v_r / C_KMS))) < 1e-9
            # 5-sigma truncation removes a relative 1.5e-5 of the variance
            assert abs(var / sig ** 2 - 1) < 5e-5


def test_integer_grid_shift_equals_index_shift(oracle):
    prob, inst0 = setup(v_r=0.0)
    k = 7
    v = C_KMS * ((1 + 1 / prob.grid.R_grid) ** k - 1)
    inst = I.Instrument(v, 0.0, inst0.R_lsf, inst0.pix_lambda_nm)
    rng = np.random.default_rng(0)
    F = rng.uniform(1, 2, prob.grid.n_lambda)
    a = oracle.apply_taps(*oracle.instrument_taps(prob, inst), F)
    Fs = np.roll(F, k)             # Fs[j] = F[j - k]: the spectrum moved redward by k steps
    b = oracle.apply_taps(*oracle.instrument_taps(prob, inst0), Fs)
    assert np.max(np.abs(a - b)) < 1e-11


def test_adjoint_identity(oracle):
    prob, inst = setup()
    taps = oracle.instrument_taps(prob, inst)
    rng = np.random.default_rng(1)
    x = rng.normal(size=prob.grid.n_lambda)
    y = rng.normal(size=inst.pix_lambda_nm.size)
    lhs = np.dot(oracle.apply_taps(*taps, x), y)
    rhs = np.dot(x, oracle.apply_taps_T(*taps, y, prob.grid.n_lambda))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_edge_rows_renormalise(oracle):
    prob = tiny_problem(n_lambda=300, n_lines=0)
    lam = I.grid_lambda_nm(prob.grid)
    inst = I.Instrument(0.0, 0.0, 22500.0, np.array([lam[1], lam[150], lam[-2]]))
    tap0, ntap, w = oracle.instrument_taps(prob, inst)
    assert tap0[0] == 0 and tap0[2] + ntap[2] - 1 == prob.grid.n_lambda - 1
    assert np.allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    assert ntap[0] < ntap[1] and ntap[2] < ntap[1]
