"""CPU checks of the far-wing forms the line kernels evaluate in FP32.

The far-wing kernels (cells with |z|^2 = v^2 + a^2 >= 400) use a five-term polynomial in
t = 1/|z|^2 for H(a, v) and a six-term one for dH/da (Eqs. 4-5: the Voigt profile and the
damping derivative of the line gradients).  Lines far from the whole wavelength tile take
reduced forms in p = 1/v^2 instead, two terms at |v| >= 100 and three at |v| >= 30, both for
a^2 <= 1.5.  These tests pin the stated truncation bounds in FP64: the polynomials against the
Faddeeva function (scipy.special.wofz), and the reduced forms against the polynomials, over
dense (a, v) lattices of the regions where the kernels use them.  They restate the series, so
a dropped term or a wrong coefficient in either form fails here.  They do not call the CUDA
path.
"""
import numpy as np
import pytest

SQPI = np.sqrt(np.pi)


def far_poly(a2, t):
    """sqrt(pi)/a x the five-term H series and sqrt(pi) x the six-term dH/da series in t."""
    h = t * (1 + 1.5 * t + (3.75 - 2 * a2) * t**2 - 15 * a2 * t**3 + 12 * a2**2 * t**4)
    d = t * (1 + (1.5 - 2 * a2) * t + (3.75 - 12 * a2) * t**2 + a2 * (12 * a2 - 67.5) * t**3
             + 180 * a2**2 * t**4 - 120 * a2**3 * t**5)
    return h, d


def reduced(a2, p, three):
    """The reduced forms in p = 1/v^2 (t = p - a^2 p^2 + a^4 p^3 - ... substituted)."""
    h = p + (1.5 - a2) * p**2
    d = p + (1.5 - 3 * a2) * p**2
    if three:
        h = h + (3.75 - 5 * a2 + a2**2) * p**3
        d = d + (3.75 - 15 * a2 + 5 * a2**2) * p**3
    return h, d


def test_far_polynomials_match_faddeeva():
    wofz = pytest.importorskip("scipy.special").wofz
    a = np.concatenate([np.geomspace(1e-6, 1.2247, 160), np.linspace(0.01, 19.9, 160)])[:, None]
    v = np.geomspace(1.0, 3000.0, 2500)[None, :]
    z2 = v**2 + a**2
    far = np.broadcast_to(z2 >= 400.0, z2.shape)
    t = 1.0 / z2
    h, d = far_poly(a**2, t)
    w = wofz(v + 1j * a)
    H = w.real
    dHda = (1j * (-2.0 * (v + 1j * a) * w + 2j / SQPI)).real   # d/da Re w(v + ia) = Re(i w')
    rel_h = np.abs(a * h / SQPI / H - 1.0)[far]
    # dH/da changes sign near v ~ a: measure it against its far-wing scale t/sqrt(pi)
    err_d = (np.abs(d / SQPI - dHda) / (t / SQPI))[far]
    assert rel_h.max() < 3e-7
    assert err_d.max() < 3e-7


@pytest.mark.parametrize("vmin, three, bound_h, bound_d", [
    (100.0, False, 4e-8, 8e-8),     # two-term reduced form
    (30.0, True, 2.7e-8, 4.7e-8),   # three-term reduced form
])
def test_reduced_forms_against_the_polynomials(vmin, three, bound_h, bound_d):
    a2 = np.linspace(0.0, 1.5, 601)[:, None]
    v = np.geomspace(vmin, 1e4, 4000)[None, :]
    p = 1.0 / v**2
    h, d = far_poly(a2, 1.0 / (v**2 + a2))
    hr, dr = reduced(a2, p, three)
    assert np.abs(hr / h - 1.0).max() < bound_h
    assert np.abs(dr / d - 1.0).max() < bound_d


def test_reduced_forms_need_their_regions():
    """Just outside their regions the reduced forms miss the bounds (so the distance
    thresholds of the kernels, |v| >= 100 and |v| >= 30, are not slack)."""
    a2 = np.linspace(0.0, 1.5, 61)[:, None]
    for vmin, three, bound in ((60.0, False, 4e-8), (20.0, True, 2.7e-8)):
        v = np.geomspace(vmin, 2 * vmin, 200)[None, :]
        h, _ = far_poly(a2, 1.0 / (v**2 + a2))
        hr, _ = reduced(a2, 1.0 / v**2, three)
        assert np.abs(hr / h - 1.0).max() > bound


def test_factored_backward_sum_equals_the_cell_sum():
    """The backward's per-depth sums over a thread's points factor: sum_i G_i (b1 s_i + b2 s_i^2
    + b3 s_i^3) = b1 X1 + b2 X2 + b3 X3 with Xk = sum_i G_i s_i^k."""
    rng = np.random.default_rng(5)
    G = rng.normal(size=(6, 4))
    s = rng.uniform(1e-6, 1e-2, size=4)
    b = rng.normal(size=(6, 3))
    cell = sum(G[:, i] * (b[:, 0] * s[i] + b[:, 1] * s[i]**2 + b[:, 2] * s[i]**3) for i in range(4))
    X = np.stack([G @ s, G @ s**2, G @ s**3], axis=1)
    assert np.allclose(cell, (b * X).sum(axis=1), rtol=1e-13, atol=0)


def _laplace_mid(x, a, nc):
    """The mid-wing Laplace series of the FP32 kernels in FP64, nc corrections:
    H sqrt(pi) = a sum_n c_n t^(n+1) U_2n and dH/da sqrt(pi) = sum_n c_n (2n+1) t^(n+1) T_2n+2
    (t = 1/|z|^2, Chebyshev recurrences in w = 2 - 4 a^2 t, c_n+1 = c_n (2n+1)/2)."""
    t = 1.0 / (x * x + a * a)
    w = 2.0 - 4.0 * a * a * t
    u0, um, g0, gm = 1.0, -1.0, 0.5 * w, 1.0
    tp, c, sh, sd = t, 1.0, 0.0, 0.0
    for n in range(nc + 1):
        sh += c * tp * u0
        sd += c * (2 * n + 1) * tp * g0
        u0, um = w * u0 - um, u0
        g0, gm = w * g0 - gm, g0
        c *= (2 * n + 1) * 0.5
        tp *= t
    return a * sh / np.sqrt(np.pi), sd / np.sqrt(np.pi)


@pytest.mark.parametrize("zmin,zmax,h_bound,d_bound", [(6, 8, 2.6e-7, 6e-5), (8, 12, 4.1e-9, 6.4e-7),
                                                       (12, 20, 1e-9, 1e-8)])
def test_mid_series_truncation(zmin, zmax, h_bound, d_bound):
    """The six-correction Laplace series of the near-core kernels' mid wing (6 <= |z| <
    20) against scipy's Faddeeva function: H within 2.6e-7 relative and dH/da within
    6e-5 relative to itself (largest where it crosses zero) at |z| = 6, far less further
    out; five corrections would miss the bound at |z| = 6."""
    from scipy.special import wofz
    a = np.concatenate([np.logspace(-4, 0, 25), np.linspace(1.0, zmin - 0.1, 30)])

    def worst(nc):
        eh = ed = 0.0
        for r in np.linspace(zmin, zmax, 40):
            for aa in a[a < r]:
                x = np.sqrt(r * r - aa * aa)
                H, dH = _laplace_mid(x, aa, nc)
                w = wofz(x + 1j * aa)
                dref = 2 * (x * w.imag + aa * w.real) - 2 / np.sqrt(np.pi)
                eh = max(eh, abs(H / w.real - 1))
                ed = max(ed, abs(dH - dref) / abs(dref))
        return eh, ed

    eh, ed = worst(6)
    assert eh < h_bound and ed < d_bound, (eh, ed)
    if zmin == 6:
        eh5, ed5 = worst(5)
        assert eh5 > h_bound or ed5 > d_bound
