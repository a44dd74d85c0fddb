"""Pins of the oracle's Voigt function H(a,v) = Re w(v + ia) (Eq. 4's profile,
phi = H/(sqrt(pi) dnu_D), with a and v of Eq. 5) against values fixed by
mathematics and by an independent library (scipy's Faddeeva function)."""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import erfcx, wofz


def lattice():
    a = np.logspace(-5, 1.3, 40)
    v = np.concatenate([np.linspace(0, 12, 241), np.linspace(12, 40, 57), np.logspace(np.log10(40), np.log10(2500), 40)])
    A, V = np.meshgrid(a, v, indexing="ij")
    return A.ravel(), V.ravel()


def test_voigt_matches_faddeeva_lattice(oracle):
    a, v = lattice()
    H, L, dH = oracle.voigt(a, v)
    w = wofz(v + 1j * a)
    core = v * v + a * a < 49
    # both regions (Fourier quadrature inside |z| = 7, continued fraction outside)
    assert np.max(np.abs(H[core] / w.real[core] - 1)) < 1e-12
    assert np.max(np.abs(H[~core] / w.real[~core] - 1)) < 1e-12
    assert np.max(np.abs(L - w.imag) / np.abs(w.imag).clip(1e-300)) < 1e-10


def test_voigt_matches_high_precision_faddeeva():
    """Against w(z) = exp(-z^2) erfc(-iz) in 40-digit arithmetic (mpmath), on the
    lattice points nearest the |z| = 7 seam and the smallest damping, where a small
    H is the sum of an O(1) Gaussian and an O(a) damping term."""
    mpmath = pytest.importorskip("mpmath")
    from oracle import oracle as o
    o.build()
    a = np.array([1e-5, 1e-4, 1e-3, 1e-2, 0.1, 1.0, 3.0])
    v = np.array([0.0, 0.5, 2.0, 4.0, 5.5, 6.5, 6.9, 6.999, 7.001, 7.5, 12.0, 60.0])
    A, V = (x.ravel() for x in np.meshgrid(a, v, indexing="ij"))
    H, L, dH = o.voigt(A, V)
    mpmath.mp.dps = 40
    ref_w = [mpmath.exp(-z * z) * mpmath.erfc(-1j * z) for z in (mpmath.mpc(x, y) for x, y in zip(V, A))]
    ref_H = np.array([float(mpmath.re(w)) for w in ref_w])
    ref_L = np.array([float(mpmath.im(w)) for w in ref_w])
    # dH/da = Re(i w'(z)) with w' = -2 z w + 2i/sqrt(pi)
    ref_dH = np.array([float(mpmath.re(1j * (-2 * mpmath.mpc(x, y) * w + 2j / mpmath.sqrt(mpmath.pi))))
                       for x, y, w in zip(V, A, ref_w)])
    assert np.max(np.abs(H / ref_H - 1)) < 1e-13
    nz = np.abs(ref_L) > 0
    assert np.max(np.abs(L[nz] / ref_L[nz] - 1)) < 1e-12
    assert np.max(np.abs(dH - ref_dH) / np.abs(ref_dH)) < 1e-11


def test_voigt_negative_v_symmetry(oracle):
    a, v = lattice()
    Hp, Lp, dp = oracle.voigt(a, v)
    Hm, Lm, dm = oracle.voigt(a, -v)
    assert np.array_equal(Hp, Hm)
    assert np.array_equal(dp, dm)
    assert np.array_equal(Lp, -Lm)


def test_voigt_line_centre_is_erfcx(oracle):
    a = np.logspace(-5, 1.5, 200)
    H, _, _ = oracle.voigt(a, np.zeros_like(a))
    assert np.max(np.abs(H / erfcx(a) - 1)) < 1e-10


def test_voigt_gaussian_limit(oracle):
    # a -> 0: H = exp(-v^2) - (2a/sqrt(pi)) (1 - 2 v D(v)) + O(a^2), D Dawson's integral
    from scipy.special import dawsn
    v = np.linspace(0, 4, 81)
    a = 1e-6
    H, _, _ = oracle.voigt(np.full_like(v, a), v)
    first = np.exp(-v * v) - 2 * a / np.sqrt(np.pi) * (1 - 2 * v * dawsn(v))
    assert np.max(np.abs(H - first)) < 5e-12


def test_voigt_lorentz_wing(oracle):
    # large v: H -> a/(sqrt(pi) v^2) (1 + (3 - 2a^2)/(2 v^2) + ...)
    a = np.array([1e-4, 1e-2, 0.3, 2.0])
    for v in [300.0, 1000.0, 2500.0]:
        H, _, _ = oracle.voigt(a, np.full_like(a, v))
        lead = a / (np.sqrt(np.pi) * v * v) * (1 + (3 - 2 * a * a) / (2 * v * v))
        assert np.max(np.abs(H / lead - 1)) < 1e-9


@pytest.mark.parametrize("a", [1e-3, 0.05, 1.0])
def test_voigt_normalisation(oracle, a):
    # Int H dv = sqrt(pi): numerical core plus the analytic Lorentz tail beyond V
    V = 400.0
    f = lambda v: float(oracle.voigt(np.array([a]), np.array([v]))[0][0])  # noqa: E731
    core = 2 * integrate.quad(f, 0, V, limit=400, points=[1, 3, 6, 10, 30], epsabs=1e-14, epsrel=1e-12)[0]
    tail = 2 * (a / np.sqrt(np.pi)) * (1 / V + (3 - 2 * a * a) / (6 * V ** 3))
    assert abs((core + tail) / np.sqrt(np.pi) - 1) < 2e-9


def test_voigt_dHda_matches_difference_quotient(oracle):
    rng = np.random.default_rng(3)
    a = 10 ** rng.uniform(-3, 1, 400)
    v = np.concatenate([rng.uniform(0, 10, 200), 10 ** rng.uniform(1, 3.3, 200)])
    _, _, dH = oracle.voigt(a, v)
    h = 1e-6 * a
    Hp, _, _ = oracle.voigt(a + h, v)
    Hm, _, _ = oracle.voigt(a - h, v)
    fd = (Hp - Hm) / (2 * h)
    w = wofz(v + 1j * a)
    ref = 2 * (v * w.imag + a * w.real) - 2 / np.sqrt(np.pi)  # from w' = -2 z w + 2i/sqrt(pi)
    assert np.max(np.abs(dH - ref) / np.abs(ref)) < 1e-6
    assert np.max(np.abs(dH - fd) / np.abs(ref)) < 1e-4
