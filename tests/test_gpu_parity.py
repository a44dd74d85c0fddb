"""Element-wise parity of the CUDA path with the FP64 oracle (forward)."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from gpu_util import kappa_rel, run_forward
from tiny import tiny_problem

pytestmark = pytest.mark.gpu

F_TOL = 1e-4          # |Delta f_norm| bound for the mixed path
KAPPA_TOL = 3e-5      # relative kappa_line bound (where kappa_line > 1e-6 kappa_c)


@pytest.fixture(scope="module")
def cfg0(oracle):
    prob = I.config0()
    return prob, oracle.forward(prob)


def test_config0_mixed(cfg0):
    prob, ref = cfg0
    got = run_forward(prob, pz.PZ_MIXED)
    assert kappa_rel(got["kline"], ref["kline"], prob.kappa_c) < KAPPA_TOL
    assert np.max(np.abs(got["F"] / ref["F"] - 1)) < 1e-5
    assert np.max(np.abs(got["Fc"] / ref["Fc"] - 1)) < 1e-12
    df = np.abs(got["f"] - ref["f"])
    assert df.max() < F_TOL
    print("config0 mixed: max|df| %.3g p99 %.3g rms %.3g" % (df.max(), np.percentile(df, 99), np.sqrt(np.mean(df ** 2))))


def test_config0_fp64_form(cfg0):
    prob, ref = cfg0
    got = run_forward(prob, pz.PZ_FP64)
    assert kappa_rel(got["kline"], ref["kline"], prob.kappa_c) < 1e-6   # kline is returned as FP32
    assert np.max(np.abs(got["F"] / ref["F"] - 1)) < 1e-9
    assert np.max(np.abs(got["f"] - ref["f"])) < 1e-6


@pytest.mark.parametrize("tiling", [(4, 8, 4, 32, 1), (2, 8, 4, 32, 2), (4, 6, 4, 16, 4), (2, 12, 3, 8, 1), (4, 12, 2, 64, 1),
                                    (4, 6, 1, 32, 1), (4, 6, 2, 16, 6), (2, 6, 4, 16, 6), (2, 8, 2, 32, 5),
                                    (4, 6, 4, 32, 5), (4, 8, 3, 32, 3)])
def test_tilings_agree(oracle, tiling):
    prob = tiny_problem(n_lambda=1037, n_depth=17, n_lines=300, W=400, seed=3)
    prob.lines.log_gf[:] -= 3.0
    ref = oracle.forward(prob)
    got = run_forward(prob, pz.PZ_MIXED, tiling=tiling)
    assert kappa_rel(got["kline"], ref["kline"], prob.kappa_c) < KAPPA_TOL
    assert np.max(np.abs(got["f"] - ref["f"])) < F_TOL


def test_small_config1_with_instrument(oracle):
    prob = I.small_config1(n_lambda_span_nm=3.0)
    ref = oracle.forward(prob)
    got = run_forward(prob, pz.PZ_MIXED)
    assert kappa_rel(got["kline"], ref["kline"], prob.kappa_c) < KAPPA_TOL
    df = np.abs(got["f"] - ref["f"])
    assert df.max() < F_TOL
    got64 = run_forward(prob, pz.PZ_FP64)
    assert np.max(np.abs(got64["f"] - ref["f"])) < 1e-6


def test_corrections_forward(oracle):
    prob = tiny_problem(n_lambda=700, n_depth=12, n_lines=40, W=300, seed=8)
    prob.lines.log_gf[:] -= 4.0
    rng = np.random.default_rng(4)
    corr = {"dlog_gf": rng.normal(0, 0.3, 40), "dlog_gamma6": rng.normal(0, 0.5, 40),
            "dabund": rng.normal(0, 0.2, prob.n_elem)}
    corr = {k: v.astype(np.float32).astype(np.float64) for k, v in corr.items()}
    ref = oracle.forward(prob, corr)
    c32 = {k: v.astype(np.float32) for k, v in corr.items()}
    got = run_forward(prob, pz.PZ_MIXED, corrections=c32)
    assert kappa_rel(got["kline"], ref["kline"], prob.kappa_c) < KAPPA_TOL
    assert np.max(np.abs(got["f"] - ref["f"])) < F_TOL


# ---- edge cases --------------------------------------------------------------

def test_zero_lines_is_continuum_exactly():
    prob = tiny_problem(n_lambda=333, n_lines=0, n_depth=9)
    for prec in (pz.PZ_MIXED, pz.PZ_FP64):
        got = run_forward(prob, prec)
        assert np.all(got["kline"] == 0)
        assert np.array_equal(got["F"], got["Fc"])
        assert np.all(got["f"] == 1.0)


@pytest.mark.parametrize("n_lambda,n_depth,W", [(1, 2, 0), (3, 2, 5), (129, 3, 0), (257, 80, 40), (1000, 72, 1)])
def test_degenerate_shapes(oracle, n_lambda, n_depth, W):
    prob = tiny_problem(n_lambda=n_lambda, n_depth=n_depth, n_lines=25, W=W, seed=n_lambda)
    prob.lines.log_gf[:] -= 3.0
    ref = oracle.forward(prob)
    for prec, ktol, ftol in ((pz.PZ_MIXED, KAPPA_TOL, F_TOL), (pz.PZ_FP64, 1e-6, 1e-6)):
        got = run_forward(prob, prec)
        assert kappa_rel(got["kline"], ref["kline"], prob.kappa_c) < ktol
        assert np.max(np.abs(got["f"] - ref["f"])) < ftol


def test_lines_outside_grid_are_dropped(oracle):
    prob = tiny_problem(n_lambda=200, n_lines=10, W=10, seed=2)
    lam = I.grid_lambda_nm(prob.grid)
    r = 1 + 1 / prob.grid.R_grid
    prob.lines.lambda_nm[:5] = lam[0] * r ** -40.0      # window misses the grid
    prob.lines.lambda_nm[5:] = lam[-1] * r ** 30.0
    got = run_forward(prob, pz.PZ_MIXED)
    assert np.all(got["kline"] == 0)
    assert got["synth"].n_evals == 0


# ---- full-size configurations, sampled (launch configuration of the benchmark) ----

def sampled_columns(n_lambda, T=128, k=12, seed=0):
    rng = np.random.default_rng(seed)
    fixed = [0, T - 1, T, n_lambda // 2, n_lambda - 2, n_lambda - 1]
    return np.unique(np.concatenate([fixed, rng.integers(0, n_lambda, k)]))


def test_config1_full_sampled(oracle):
    prob = I.config1()
    got = run_forward(prob, pz.PZ_MIXED)
    cols = sampled_columns(prob.grid.n_lambda)
    kref = oracle.kappa_line(prob, cols)
    assert kappa_rel(got["kline"][:, cols], kref, prob.kappa_c[:, cols]) < KAPPA_TOL
    F, Fc = oracle.flux(prob, cols, kref)
    assert np.max(np.abs(got["F"][cols] / F - 1)) < 1e-5
    # sampled pixels: the oracle computes every tap column of the pixel
    taps = oracle.instrument_taps(prob, prob.instrument)
    for p in (0, 4321, prob.instrument.pix_lambda_nm.size - 1):
        c = taps[0][p] + np.arange(taps[1][p])
        kc = oracle.kappa_line(prob, c)
        Fp, Fcp = oracle.flux(prob, c, kc)
        w = taps[2][p, :taps[1][p]]
        f_ref = np.dot(w, Fp) / np.dot(w, Fcp)
        assert abs(got["f"][p] - f_ref) < F_TOL


def test_config2_full_sampled(oracle):
    prob = I.config2()
    got = run_forward(prob, pz.PZ_MIXED)
    cols = sampled_columns(prob.grid.n_lambda, k=8, seed=2)
    kref = oracle.kappa_line(prob, cols)
    assert kappa_rel(got["kline"][:, cols], kref, prob.kappa_c[:, cols]) < KAPPA_TOL
    F, Fc = oracle.flux(prob, cols, kref)
    assert np.max(np.abs(got["f"][cols] - F / Fc)) < F_TOL
