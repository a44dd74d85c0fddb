"""Pins of the oracle's hand-written reverse pass (Sec. 6): every gradient
against central finite differences of the oracle's own forward."""
import numpy as np
import pytest

from tiny import tiny_problem


@pytest.mark.parametrize("instrument", [False, True])
def test_gradient_matches_central_differences(oracle, instrument):
    """g = (df/d delta)^T dL/df with df/d delta from central differences of the
    oracle's forward (h = 1e-4); dL/df is the pinned chi-square seed."""
    prob = tiny_problem(n_lambda=160, n_depth=10, n_lines=7, W=60, seed=21, instrument=instrument, E_max=1.0)
    prob.lines.log_gf[:] -= 4.0      # saturated cores and unsaturated wings (f from ~0.4 to ~0.95)
    rng = np.random.default_rng(2)
    corr = {"dlog_gf": rng.normal(0, 0.1, 7), "dlog_gamma6": rng.normal(0, 0.2, 7),
            "dabund": rng.normal(0, 0.1, prob.n_elem), "dlog_gamma_rad": rng.normal(0, 0.2, 7),
            "dlog_gamma4": rng.normal(0, 0.2, 7)}
    n_out = prob.instrument.pix_lambda_nm.size if instrument else prob.grid.n_lambda
    f0 = oracle.forward(prob, corr)["f"]
    y = f0 + rng.normal(0, 0.01, n_out)
    w = np.full(n_out, 200.0 ** 2)
    L, ggf, gg6, gab, fwd = oracle.gradient(prob, y, w, corr)
    _, dLdf = oracle.chi2(y, w, f0)
    h = 1e-4
    for key, g in [("dlog_gf", ggf), ("dlog_gamma6", gg6), ("dabund", gab),
                   ("dlog_gamma_rad", fwd["g_gamma_rad"]), ("dlog_gamma4", fwd["g_gamma4"])]:
        for j in range(len(corr[key])):
            cp = {k: v.copy() for k, v in corr.items()}
            cm = {k: v.copy() for k, v in corr.items()}
            cp[key][j] += h
            cm[key][j] -= h
            dfd = (oracle.forward(prob, cp)["f"] - oracle.forward(prob, cm)["f"]) / (2 * h)
            fd = float(np.dot(dLdf, dfd))
            scale = max(abs(fd), 1e-3 * np.max(np.abs(g)))
            # rounding of f (a few ulp) enters the difference quotient as ~ |dL/df| eps / h
            noise = 10 * np.sqrt(n_out) * np.max(np.abs(dLdf)) * 1.2e-16 / h
            assert abs(g[j] - fd) <= 1e-6 * scale + noise, (key, j, g[j], fd)


def test_chi2_seed(oracle):
    rng = np.random.default_rng(0)
    y, f = rng.normal(size=50), rng.normal(size=50)
    w = rng.uniform(1, 2, 50)
    L, dL = oracle.chi2(y, w, f)
    assert np.isclose(L, np.sum(w * (y - f) ** 2), rtol=1e-14)
    for j in range(0, 50, 9):
        e = np.zeros(50)
        e[j] = 1e-6
        fd = (oracle.chi2(y, w, f + e)[0] - oracle.chi2(y, w, f - e)[0]) / 2e-6
        assert abs(fd - dL[j]) < 1e-6 * abs(dL[j]) + 1e-9


def test_damping_families_split_the_damping_gradient(oracle):
    """The three damping gradients are the parts of one derivative: scaling every
    family of a line by the same 10^delta scales its damping parameter a by 10^delta,
    so their sum is the central difference of L along that joint direction; a family
    whose coefficient is negligible has a negligible gradient."""
    prob = tiny_problem(n_lambda=120, n_depth=8, n_lines=5, W=50, seed=5, instrument=False, E_max=1.0)
    prob.lines.log_gf[:] -= 4.0
    prob.lines.log_gamma4[1] = -60.0          # a negligible Stark coefficient
    rng = np.random.default_rng(9)
    f0 = oracle.forward(prob)["f"]
    y = f0 + rng.normal(0, 0.01, f0.size)
    w = np.full(f0.size, 1e4)
    r = oracle.gradient4(prob, y, w)
    assert abs(r["gamma4"][1]) <= 1e-40 * np.max(np.abs(r["gamma6"]))
    assert np.all(r["gamma_rad"] != 0.0) and np.all(r["gamma6"] != 0.0)
    h = 1e-4
    for j in range(5):
        def L_at(t):
            c = {k: np.zeros(5) for k in ("dlog_gamma_rad", "dlog_gamma4", "dlog_gamma6")}
            for k in c:
                c[k][j] = t
            return oracle.chi2(y, w, oracle.forward(prob, c)["f"])[0]
        # Richardson-extrapolated central difference (the h^2 term cancels)
        d1 = (L_at(h) - L_at(-h)) / (2 * h)
        d2 = (L_at(2 * h) - L_at(-2 * h)) / (4 * h)
        fd = (4 * d1 - d2) / 3
        tot = r["gamma_rad"][j] + r["gamma4"][j] + r["gamma6"][j]
        assert abs(tot - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(r["gamma6"]))) + 1e-9, (j, tot, fd)
