"""Pins of the oracle's exponential integrals E_n (flux closed form, Eqs. 7-8)."""
import numpy as np
from scipy.special import expn


def test_expn_matches_scipy(oracle):
    x = np.concatenate([np.logspace(-12, 0, 200), np.linspace(1.0, 3.0, 100), np.linspace(3, 700, 300)])
    for n in (1, 2, 3, 4, 5):
        got = oracle.expn(n, x)
        ref = expn(n, x)
        m = ref > 1e-300
        assert np.max(np.abs(got[m] / ref[m] - 1)) < 2e-14, n


def test_expn_at_zero(oracle):
    for n in (2, 3, 4, 5):
        assert oracle.expn(n, np.array([0.0]))[0] == 1.0 / (n - 1)


def test_expn_recurrence(oracle):
    # n E_{n+1}(x) = e^{-x} - x E_n(x)
    x = np.concatenate([np.logspace(-6, 0, 50), np.linspace(1, 30, 60)])
    for n in (1, 2, 3):
        lhs = n * oracle.expn(n + 1, x)
        rhs = np.exp(-x) - x * oracle.expn(n, x)
        assert np.max(np.abs(lhs - rhs) / np.abs(lhs)) < 1e-12


def test_expn_derivative(oracle):
    # d E_n / dx = -E_{n-1}
    x = np.linspace(0.05, 20, 200)
    h = 1e-6 * x
    for n in (2, 3, 4):
        fd = (oracle.expn(n, x + h) - oracle.expn(n, x - h)) / (2 * h)
        assert np.max(np.abs(fd + oracle.expn(n - 1, x)) / oracle.expn(n - 1, x)) < 1e-7
