"""Pins of the oracle's formal solution (Sec. 2.1, Eqs. 6-8) and Planck source."""
import numpy as np
from scipy.special import expn

from paper_2607_24141_gb300 import inputs as I
from tiny import tiny_problem


def taus(n=30, top=1e-7, bottom=80.0):
    return np.geomspace(top, bottom, n)


def test_constant_source(oracle):
    for tmax in (0.3, 5.0, 80.0):
        t = taus(bottom=tmax)
        S = np.full(t.size, 2.5)
        F = oracle.flux_tau(t, S)
        assert abs(F / (np.pi * 2.5 * (1 - 2 * expn(3, tmax))) - 1) < 1e-13


def test_linear_source_eddington_barbier(oracle):
    a, b = 1.7, 0.9
    t = taus(40, 1e-6, 60.0)
    F = oracle.flux_tau(t, a + b * t)
    assert abs(F / (np.pi * (a + 2 * b / 3)) - 1) < 1e-12
    # finite depth: 2 pi [a (1/2 - E3) + b (1/3 - E4 - tau E3)]
    t = taus(40, 1e-6, 2.0)
    F = oracle.flux_tau(t, a + b * t)
    ref = 2 * np.pi * (a * (0.5 - expn(3, 2.0)) + b * (1 / 3 - expn(4, 2.0) - 2.0 * expn(3, 2.0)))
    assert abs(F / ref - 1) < 1e-12


def test_interval_integrals_against_quadrature(oracle):
    """Piecewise-linear S: compare with 64-point Gauss-Legendre per interval of S E_2."""
    rng = np.random.default_rng(0)
    t = np.sort(rng.uniform(0.01, 6.0, 12))
    S = rng.uniform(0.5, 3.0, 12)
    x, w = np.polynomial.legendre.leggauss(64)
    edges = np.concatenate([[0.0], t])
    s0 = (S[1] - S[0]) / (t[1] - t[0])
    Sn = np.concatenate([[S[0] - s0 * t[0]], S])
    total = 0.0
    for k in range(len(edges) - 1):
        a_, b_ = edges[k], edges[k + 1]
        tt = 0.5 * (b_ - a_) * x + 0.5 * (b_ + a_)
        Sl = Sn[k] + (Sn[k + 1] - Sn[k]) * (tt - a_) / (b_ - a_)
        total += 0.5 * (b_ - a_) * np.sum(w * Sl * expn(2, tt))
    assert abs(oracle.flux_tau(t, S) / (2 * np.pi * total) - 1) < 1e-10


def test_flux_dtau_matches_difference_quotient(oracle):
    rng = np.random.default_rng(1)
    t = np.cumsum(rng.uniform(0.02, 0.6, 15))
    S = rng.uniform(0.5, 3.0, 15)
    g = oracle.flux_dtau(t, S)
    for j in range(15):
        h = 1e-6 * t[j]
        tp, tm = t.copy(), t.copy()
        tp[j] += h
        tm[j] -= h
        fd = (oracle.flux_tau(tp, S) - oracle.flux_tau(tm, S)) / (2 * h)
        assert abs(fd - g[j]) < 1e-6 * np.max(np.abs(g))


def test_planck_stefan_boltzmann_and_wien(oracle):
    sigma = 5.670374419e-5           # erg cm^-2 s^-1 K^-4
    b_wien = 0.2897771955            # cm K
    for T in (3500.0, 5777.0, 9000.0):
        lam = np.geomspace(50.0, 2e6, 200001)          # nm
        B = np.array([oracle.planck_nm(l, T) for l in lam[::50]])
        # per-nm radiance integrated over nm = sigma T^4 / pi
        lg = np.log(lam[::50])
        integral = np.trapezoid(B * lam[::50], lg)
        assert abs(integral / (sigma * T ** 4 / np.pi) - 1) < 1e-6
        grid = np.linspace(0.8, 1.2, 4001) * b_wien / T * 1e7
        peak = grid[np.argmax([oracle.planck_nm(l, T) for l in grid])]
        assert abs(peak / (b_wien / T * 1e7) - 1) < 1e-4


def test_zero_lines_gives_continuum_exactly(oracle):
    prob = tiny_problem(n_lines=0)
    out = oracle.forward(prob)
    assert np.array_equal(out["F"], out["Fc"])
    assert np.all(out["f"] == 1.0)


def test_trapezoid_optical_depth_closed_form(oracle):
    """chi = alpha + beta m: trapezoid exact, tau_0 = chi_0 m_0 above the first layer."""
    prob = tiny_problem(n_lambda=3, n_depth=12, n_lines=0)
    m = prob.atmos.m
    alpha, beta = 0.4, 0.02
    chi = alpha + beta * m
    prob.kappa_c = np.ascontiguousarray(np.repeat(chi[:, None], 3, axis=1))
    F, Fc = oracle.flux(prob, np.arange(3), np.zeros((12, 3)))
    tau = chi[0] * m[0] + alpha * (m - m[0]) + beta * (m * m - m[0] ** 2) / 2
    lam = I.grid_lambda_nm(prob.grid)
    for i in range(3):
        S = np.array([oracle.planck_nm(lam[i], T) for T in prob.atmos.T])
        assert abs(F[i] / oracle.flux_tau(tau, S) - 1) < 1e-13
