"""Pins of the oracle's scattering source function (Eq. 6, S = eps B + (1 - eps) J, with
J the mean intensity of the same slab): the Lambda operator against closed forms of
J for constant and linear sources, against adaptive quadrature of the E_1 kernel, the
solved source against the exact sqrt(eps) law of a scattering-dominated isothermal
atmosphere, and sigma_c = 0 against the LTE flux."""
import numpy as np
import pytest

from tiny import tiny_problem

special = pytest.importorskip("scipy.special")
integrate = pytest.importorskip("scipy.integrate")


def _tau_grid(nd, lo=-6.0, hi=2.0, seed=0):
    rng = np.random.default_rng(seed)
    x = np.sort(np.concatenate([[lo, hi], rng.uniform(lo, hi, nd - 2)]))
    return 10.0 ** x


def test_lambda_of_constant_source(oracle):
    """S = 1 on [0, T]: J(tau) = 1 - E2(tau)/2 - E2(T - tau)/2 (the linear extrapolation to
    tau = 0 and the interpolation both represent a constant exactly)."""
    tau = _tau_grid(40)
    T = tau[-1]
    Lam = oracle.lambda_matrix(tau)
    J = Lam @ np.ones(tau.size)
    ref = 1.0 - 0.5 * special.expn(2, tau) - 0.5 * special.expn(2, T - tau)
    np.testing.assert_allclose(J, ref, rtol=1e-12, atol=1e-14)


def test_lambda_of_linear_source(oracle):
    """S = t on [0, T]: J(tau) = tau + E3(tau)/2 - T E2(T - tau)/2 - E3(T - tau)/2."""
    tau = _tau_grid(35, seed=1)
    T = tau[-1]
    J = oracle.lambda_matrix(tau) @ tau
    ref = tau + 0.5 * special.expn(3, tau) - 0.5 * T * special.expn(2, T - tau) - 0.5 * special.expn(3, T - tau)
    np.testing.assert_allclose(J, ref, rtol=1e-11, atol=1e-13)


def test_lambda_against_quadrature(oracle):
    """An arbitrary piecewise-linear source: J = 1/2 Int S(t) E_1(|t - tau_j|) dt by
    adaptive quadrature of each interval (the logarithmic singularity sits at an
    interval end), with the first segment extrapolated to t = 0."""
    tau = _tau_grid(12, lo=-3.0, hi=1.0, seed=2)
    S = np.random.default_rng(3).uniform(0.5, 2.0, tau.size)
    J = oracle.lambda_matrix(tau) @ S
    s0 = (S[1] - S[0]) / (tau[1] - tau[0])
    knots = np.concatenate([[0.0], tau])
    vals = np.concatenate([[S[0] - s0 * tau[0]], S])
    for j in range(tau.size):
        tot = 0.0
        for k in range(knots.size - 1):
            a, b, Sa, Sb = knots[k], knots[k + 1], vals[k], vals[k + 1]

            def f(t):
                return (Sa + (Sb - Sa) * (t - a) / (b - a)) * special.exp1(abs(t - tau[j]))
            tot += integrate.quad(f, a, b, limit=200, epsabs=1e-15, epsrel=1e-13)[0]
        assert abs(J[j] - 0.5 * tot) <= 1e-10 * abs(0.5 * tot), (j, J[j], 0.5 * tot)


def _isothermal(oracle, eps, n):
    tau = np.concatenate([[1e-8], np.geomspace(1e-6, 1e6, n)])
    return tau, oracle.scatter_source(tau, np.full(tau.size, eps), np.ones(tau.size))


@pytest.mark.parametrize("eps", [0.5, 0.1, 1e-2])
def test_sqrt_eps_law(oracle, eps):
    """Isothermal (B = 1), constant eps, effectively semi-infinite: the exact solution
    has S(0) = sqrt(eps) B, and S -> B deep inside (thermalisation depth ~ 1/sqrt(eps)).
    The piecewise-linear source converges to it at second order in the grid step (the
    small surface value carries the discretisation error of J relative to the deep B,
    so small eps needs finer grids)."""
    tau, S = _isothermal(oracle, eps, 800)
    assert abs(S[0] / np.sqrt(eps) - 1) < 2.5e-3, S[0]
    mid = np.argmin(np.abs(tau - 100.0 / np.sqrt(eps)))
    assert abs(S[mid] - 1) < 1e-3
    e1 = abs(_isothermal(oracle, eps, 400)[1][0] / np.sqrt(eps) - 1)
    e2 = abs(S[0] / np.sqrt(eps) - 1)
    assert e2 < e1 / 3.0 or e2 < 1e-5, (e1, e2)
    # the fixed point of the iteration S <- eps B + (1 - eps) Lambda S
    Lam = oracle.lambda_matrix(tau)
    np.testing.assert_allclose(S, eps + (1 - eps) * (Lam @ S), rtol=1e-10, atol=1e-12)


def test_no_scattering_is_lte(oracle):
    """sigma_c = 0 everywhere gives eps = 1, S = B and the LTE flux bit for bit."""
    prob = tiny_problem(n_lambda=150, n_depth=12, n_lines=10, W=60, seed=4)
    import dataclasses
    ref = oracle.forward(prob)
    got = oracle.forward(dataclasses.replace(prob, sigma_c=np.zeros_like(prob.kappa_c)))
    assert np.array_equal(got["F"], ref["F"]) and np.array_equal(got["Fc"], ref["Fc"])


def test_scattering_lowers_the_surface_source(oracle):
    """With sigma_c > 0 in the upper layers, the emergent continuum drops below the LTE
    one where the scattering albedo is large (blue), and the line-to-continuum ratio
    stays in (0, 1]."""
    from paper_2607_24141_gb300 import inputs as I
    prob = tiny_problem(n_lambda=150, n_depth=30, n_lines=10, W=60, seed=4, lam0=350.0)
    sc = I.with_scattering(prob, r0=3.0)
    lte, scat = oracle.forward(prob), oracle.forward(sc)
    assert np.all(scat["Fc"] < lte["Fc"])
    assert np.all(scat["f"] > 0) and np.all(scat["f"] <= 1 + 1e-12)


def _cd(fun, x, j, h):
    """Richardson-extrapolated central difference of fun along coordinate j."""
    def d(hh):
        xp, xm = x.copy(), x.copy()
        xp[j] += hh
        xm[j] -= hh
        return (fun(xp) - fun(xm)) / (2 * hh)
    return (4 * d(h) - d(2 * h)) / 3


@pytest.mark.parametrize("grid,rtol", [("smooth", 1e-8), ("log", 2e-5)])
def test_lambda_dtau_against_differences(oracle, grid, rtol):
    """dJ_j/dtau_m at fixed layer values against differences of Lambda(tau) S (every
    layer moved in turn, including the bottom one and tau_j itself).  On a grid of
    well-separated layers the differences are accurate to 1e-8; on a logarithmic grid
    with steps down to 6e-4 the cancellation inside the segment weights (eps/D per
    weight) limits a difference quotient to ~1e-5 of the row, still far below any
    missing or mis-signed term."""
    if grid == "smooth":
        tau = np.array([0.2, 0.5, 0.9, 1.4, 2.0, 2.7, 3.5, 4.4, 5.4])
    else:
        tau = _tau_grid(9, lo=-3.0, hi=1.0, seed=5)
    S = np.random.default_rng(6).uniform(0.5, 2.0, tau.size)
    dJ = oracle.lambda_dtau(tau, S)
    for m in range(tau.size):
        h = 2e-3 * min(tau[m] - (tau[m - 1] if m else 0.0), (tau[m + 1] - tau[m]) if m + 1 < tau.size else tau[m])
        for j in range(tau.size):
            fd = _cd(lambda t: (oracle.lambda_matrix(t) @ S)[j], tau, m, h)
            tol = rtol * max(abs(fd), 1e-3 * np.max(np.abs(dJ[j])))
            assert abs(dJ[j, m] - fd) <= tol, (j, m, dJ[j, m], fd)


def test_scatter_adjoint_against_differences(oracle):
    """dF/dtau and dF/deps of the emergent flux of the solved source against differences
    of the flux itself."""
    rng = np.random.default_rng(8)
    tau = _tau_grid(12, lo=-4.0, hi=1.5, seed=9)
    eps = rng.uniform(0.05, 1.0, tau.size)
    B = np.linspace(1.0, 3.0, tau.size)
    gt, ge = oracle.scatter_adjoint(tau, eps, B, 1.0)
    for m in range(tau.size):
        h = 2e-3 * min(tau[m] - (tau[m - 1] if m else 0.0), (tau[m + 1] - tau[m]) if m + 1 < tau.size else tau[m])
        fd = _cd(lambda t: oracle.scatter_flux(t, eps, B), tau, m, h)
        tol = 2e-5 * max(abs(fd), 1e-3 * np.max(np.abs(gt)))      # as for Lambda on a log grid
        assert abs(gt[m] - fd) <= tol, ("tau", m, gt[m], fd)
    for j in range(tau.size):
        fd = _cd(lambda e: oracle.scatter_flux(tau, e, B), eps, j, 1e-5)
        assert abs(ge[j] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(ge))), ("eps", j, ge[j], fd)


def test_gradients_with_scattering_against_differences(oracle):
    """The whole reverse pass with sigma_c > 0 (line corrections -> kappa_line -> tau and
    eps -> solved source -> flux -> chi^2) against central differences of the forward."""
    from paper_2607_24141_gb300 import inputs as I
    prob = I.with_scattering(tiny_problem(n_lambda=160, n_depth=10, n_lines=7, W=60, seed=21, lam0=380.0,
                                          E_max=1.0), r0=3.0)
    prob.lines.log_gf[:] -= 4.0
    rng = np.random.default_rng(2)
    corr = {"dlog_gf": rng.normal(0, 0.1, 7), "dlog_gamma6": rng.normal(0, 0.2, 7)}
    f0 = oracle.forward(prob, corr)["f"]
    y = f0 + rng.normal(0, 0.01, f0.size)
    w = np.full(f0.size, 200.0 ** 2)
    L, ggf, gg6, _, _ = oracle.gradient(prob, y, w, corr)
    for key, g in (("dlog_gf", ggf), ("dlog_gamma6", gg6)):
        for j in range(7):
            def L_at(v):
                c = {k: vv.copy() for k, vv in corr.items()}
                c[key] = v
                return oracle.chi2(y, w, oracle.forward(prob, c)["f"])[0]
            # steps 5e-4 and 1e-3: the chi^2 of the solved scattering source carries FP64
            # rounding noise near 1e-13 of its value, which swamps a quotient at 1e-4
            fd = _cd(L_at, corr[key], j, 5e-4)
            assert abs(g[j] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(g))), (key, j, g[j], fd)
