"""Continuum scattering in the formal solution (Eq. 6) on the device against the FP64
oracle: F, F_c and f in both precision forms for blue and infrared problems, sigma_c = 0
against the LTE kernel, and the API's state rules."""
import dataclasses

import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from gpu_util import rel_metric, run_forward, run_gradient
from tiny import tiny_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_lambda,n_depth,lam0,r0", [(300, 30, 350.0, 3.0), (500, 72, 320.0, 2.0),
                                                      (200, 128, 400.0, 5.0), (150, 2, 330.0, 1.0)])
def test_scattering_parity(oracle, n_lambda, n_depth, lam0, r0):
    prob = tiny_problem(n_lambda=n_lambda, n_depth=n_depth, n_lines=30, W=150, seed=n_depth, lam0=lam0)
    prob.lines.log_gf[:] -= 3.0
    sc = I.with_scattering(prob, r0=r0)
    ref = oracle.forward(sc)
    lte = oracle.forward(prob)
    for prec, ftol, ntol in ((pz.PZ_MIXED, 1e-5, 1e-4), (pz.PZ_FP64, 1e-9, 1e-6)):   # f is FP32
        got = run_forward(sc, prec)
        eF = np.max(np.abs(got["F"] / ref["F"] - 1))
        eFc = np.max(np.abs(got["Fc"] / ref["Fc"] - 1))
        ef = np.max(np.abs(got["f"] - ref["f"]))
        print("scatter nd=%d prec=%d: F %.3g Fc %.3g f %.3g (scattering moves Fc by %.3g)"
              % (n_depth, prec, eF, eFc, ef, np.max(np.abs(ref["Fc"] / lte["Fc"] - 1))))
        assert eFc < (1e-9 if prec == pz.PZ_MIXED else 1e-10), eFc     # no line opacity in F_c
        assert eF < ftol and ef < ntol, (eF, ef)
        got["synth"].close()


def test_scattering_with_instrument(oracle):
    prob = I.with_scattering(I.small_config1(n_lambda_span_nm=2.0, seed=5), r0=50.0)
    ref = oracle.forward(prob)
    got = run_forward(prob, pz.PZ_MIXED, want_kline=False)
    assert np.max(np.abs(got["f"] - ref["f"])) < 1e-4
    got["synth"].close()


def test_zero_scattering_is_the_lte_kernel():
    prob = tiny_problem(n_lambda=400, n_depth=40, n_lines=30, W=150, seed=6, lam0=380.0)
    prob.lines.log_gf[:] -= 3.0
    for prec in (pz.PZ_MIXED, pz.PZ_FP64):
        a = run_forward(prob, prec, want_kline=False)
        b = run_forward(dataclasses.replace(prob, sigma_c=np.zeros_like(prob.kappa_c)), prec, want_kline=False)
        # F: the two contexts' line opacities differ only by the order of the near-core
        # shared-memory atomics (FP32 in the mixed form); F_c has no line opacity
        assert np.max(np.abs(b["F"] / a["F"] - 1)) < (1e-7 if prec == pz.PZ_MIXED else 1e-14)
        assert np.max(np.abs(b["Fc"] / a["Fc"] - 1)) < 1e-14
        a["synth"].close()
        b["synth"].close()


def test_scattering_state_rules():
    import torch
    prob = tiny_problem(n_lambda=200, n_depth=20, n_lines=10, W=60, seed=3, lam0=360.0)
    s = pz.Synthesizer(prob)
    bad = prob.kappa_c.copy()
    bad[3, 7] = -1.0
    with pytest.raises(pz.PzError) as e:
        pz.pz_set_scattering(s.ctx, bad)
    assert e.value.status == pz.PZ_EINVAL
    f_lte = s.forward().cpu().numpy()
    pz.pz_set_scattering(s.ctx, I.with_scattering(prob, r0=3.0).sigma_c)
    with pytest.raises(pz.PzError) as e:          # the flux must be recomputed
        pz.pz_instrument(s.ctx, 0.0, 0.0, 0.0, None)
    assert e.value.status == pz.PZ_ESTATE
    f_sc = s.forward()
    assert np.max(np.abs(f_sc.cpu().numpy() - f_lte)) > 1e-6
    pz.pz_set_scattering(s.ctx, None)
    # the LTE spectrum again (up to the order of the near-core shared-memory atomics)
    np.testing.assert_allclose(s.forward().cpu().numpy(), f_lte, rtol=0, atol=1e-6)
    s.close()


def test_scattering_batch_matches_the_oracle_per_star(oracle):
    b = I.with_scattering_batch(I.small_batch(n_stars=2, span_nm=1.0, seed=23, with_instrument=False), r0=200.0)
    s = pz.Synthesizer(b, pz.PZ_FP64)
    f = s.forward().cpu().numpy().astype(np.float64)
    for k in range(b.n_stars):
        ref = oracle.forward(b.star(k))
        assert np.max(np.abs(f[k] - ref["f"])) < 1e-6
    s.close()


@pytest.mark.parametrize("n_depth,instrument", [(30, False), (72, True)])
def test_scattering_gradients(oracle, n_depth, instrument):
    """The reverse pass through the scattering source (adjoint of the linear system, the
    dependence of J on the optical depths, eps = 1 - sigma/chi) against the oracle's."""
    prob = I.with_scattering(tiny_problem(n_lambda=600, n_depth=n_depth, n_lines=40, W=200, seed=n_depth + 3,
                                          lam0=360.0, instrument=instrument), r0=3.0)
    prob.lines.log_gf[:] -= 3.0
    rng = np.random.default_rng(11)
    nl = prob.lines.n_lines
    corr = {"dlog_gf": rng.normal(0, 0.1, nl), "dlog_gamma6": rng.normal(0, 0.2, nl),
            "dabund": rng.normal(0, 0.1, prob.n_elem)}
    corr = {k: v.astype(np.float32).astype(np.float64) for k, v in corr.items()}
    f0 = oracle.forward(prob, corr)
    n_out = f0["f"].size
    y = (f0["f"] + rng.normal(0, 1 / 200, n_out)).astype(np.float32).astype(np.float64)
    w = 200.0 ** 2
    L, ggf, gg6, gab, _ = oracle.gradient(prob, y, np.full(n_out, w), corr, fwd=f0)
    c32 = {k: v.astype(np.float32) for k, v in corr.items()}
    for prec, tol in ((pz.PZ_MIXED, 1e-3), (pz.PZ_FP64, 1e-5)):
        got = run_gradient(prob, y.astype(np.float32), np.float32(w), prec, c32)
        errs = (rel_metric(got["g_gf"], ggf).max(), rel_metric(got["g_g6"], gg6).max(),
                rel_metric(got["g_ab"][:prob.n_elem], gab).max())
        print("scattering gradients nd=%d prec=%d:" % (n_depth, prec), errs)
        assert max(errs) < tol, (prec, errs)


@pytest.mark.parametrize("r0", [1e4, 1e8])
def test_scattering_dominated_solve_converges_or_reports(oracle, r0):
    """eps near 0 in the upper layers (sigma_c up to r0 kappa_c): the FP64-refined solve
    either converges, and then F and f match the oracle's at the parity bars, or it
    reports PZ_ENUMERIC through pz_sync_status; an unconverged result is never returned
    silently, and the flux is finite either way."""
    prob = tiny_problem(n_lambda=160, n_depth=40, n_lines=20, W=60, seed=41, lam0=340.0)
    prob.lines.log_gf[:] -= 3.0
    sc = I.with_scattering(prob, r0=r0)
    ref = oracle.forward(sc)
    # the system I - diag(1 - eps) Lambda has a condition number ~ 1/eps_min: two FP64
    # solves (the oracle's pivoted elimination, the device's refinement) agree to about
    # 1e-15 / eps_min
    eps_min = float(np.min(sc.kappa_c / (sc.kappa_c + sc.sigma_c)))
    for prec, ftol in ((pz.PZ_MIXED, 1e-5), (pz.PZ_FP64, max(1e-9, 1e-15 / eps_min))):
        got = run_forward(sc, prec, want_kline=False)
        s = got["synth"]
        try:
            pz.pz_sync_status(s.ctx)
            converged = True
        except pz.PzError as e:
            assert e.status == pz.PZ_ENUMERIC, e
            converged = False
        eF = float(np.max(np.abs(got["F"] / ref["F"] - 1)))
        print("r0 %.0e prec %d: converged %s, F rel err %.3g" % (r0, prec, converged, eF))
        assert np.all(np.isfinite(got["F"])) and np.all(np.isfinite(got["Fc"]))
        if converged:
            assert eF < ftol, eF
        s.close()
