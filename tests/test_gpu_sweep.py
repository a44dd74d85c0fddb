"""Parity at the other grid samplings and spans of the scaling sweeps (Sec. 3.2): the
config-2 recipe at R_grid = 1e4, 3e4 and 1e5 (line windows of fixed width in wavelength,
W = 2,000 R / 3e5), element by element on a slice and on sampled columns of the whole
300-1000 nm grid, in both precision forms."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from gpu_util import kappa_rel, run_forward

pytestmark = pytest.mark.gpu
KAPPA_TOL = 3e-5
F_TOL = 1e-4


@pytest.mark.parametrize("R", [1e4, 3e4, 1e5])
def test_sweep_sampling_slice_parity(oracle, R):
    prob = I.config2_sweep_point(R=R, n_lines_full=100_000)
    sl = I.wavelength_slice(prob, 600.0, 700)
    ref = oracle.forward(sl)
    for prec, ktol, ftol in ((pz.PZ_MIXED, KAPPA_TOL, F_TOL), (pz.PZ_FP64, 1e-6, 1e-6)):
        got = run_forward(sl, prec)
        assert kappa_rel(got["kline"], ref["kline"], sl.kappa_c) < ktol, (R, prec)
        assert np.max(np.abs(got["f"] - ref["f"])) < ftol, (R, prec)
        got["synth"].close()


@pytest.mark.parametrize("R", [1e4, 3e4])
def test_sweep_sampling_full_grid_sampled(oracle, R):
    prob = I.config2_sweep_point(R=R, n_lines_full=300_000)
    got = run_forward(prob, pz.PZ_MIXED)
    rng = np.random.default_rng(int(R))
    n = prob.grid.n_lambda
    cols = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.integers(0, n, 16)]))
    kref = oracle.kappa_line(prob, cols)
    assert kappa_rel(got["kline"][:, cols], kref, prob.kappa_c[:, cols]) < KAPPA_TOL
    got["synth"].close()


def test_sweep_span_point():
    """The shortest span of the sweep (300-400 nm): the line list is the 300-1000 nm
    density restricted to the span, and the forward runs end to end."""
    p = I.config2_sweep_point(lam_hi=400.0, n_lines_full=60_000)
    full = I.config2_sweep_point(n_lines_full=60_000)
    frac = (1 / 300 - 1 / 400) / (1 / 300 - 1 / 1000)
    assert p.lines.n_lines == round(60_000 * frac)
    assert p.grid.n_lambda == I.n_lambda_for(300.0, 400.0) and full.grid.n_lambda == I.n_lambda_for(300.0, 1000.0)
    got = run_forward(p, pz.PZ_MIXED, want_kline=False)
    assert np.all(np.isfinite(got["f"])) and got["f"].max() <= 1.0 + 1e-6
    got["synth"].close()
