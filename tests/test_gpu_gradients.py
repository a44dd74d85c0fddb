"""Parity of the hand-written CUDA reverse pass with the oracle's adjoint."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from gpu_util import rel_metric, run_gradient
from tiny import tiny_problem

pytestmark = pytest.mark.gpu
G_TOL = 1e-3


def _check(prob, oracle, corr, instrument_noise=1.0 / 200):
    # the device reads FP32 corrections: give the oracle the same rounded values
    corr = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in corr.items()}
    rng = np.random.default_rng(7)
    n_out = prob.instrument.pix_lambda_nm.size if prob.instrument is not None else prob.grid.n_lambda
    f0 = oracle.forward(prob, corr)
    # the device objective reads FP32 targets: give the oracle the same rounded values
    y = (f0["f"] + rng.normal(0, instrument_noise, n_out)).astype(np.float32).astype(np.float64)
    w = 200.0 ** 2
    L, ggf, gg6, gab, _ = oracle.gradient(prob, y, np.full(n_out, w), corr, fwd=f0)
    c32 = {k: v.astype(np.float32) for k, v in corr.items()}
    out = {}
    for prec in (pz.PZ_MIXED, pz.PZ_FP64):
        got = run_gradient(prob, y.astype(np.float32), np.float32(w), prec, c32)
        tol = G_TOL if prec == pz.PZ_MIXED else 1e-5
        e1 = rel_metric(got["g_gf"], ggf).max()
        e2 = rel_metric(got["g_g6"], gg6).max()
        e3 = rel_metric(got["g_ab"][:prob.n_elem], gab).max()
        assert e1 < tol and e2 < tol and e3 < tol, (prec, e1, e2, e3)
        out[prec] = (e1, e2, e3)
    return out


@pytest.mark.parametrize("tiling", [(4, 6, 4, 32, 5), (4, 8, 4, 32, 3), (4, 8, 3, 32, 2), (4, 12, 2, 64, 1),
                                    (2, 8, 4, 16, 5), (2, 6, 4, 16, 6), (4, 6, 1, 128, 3)])
def test_tilings_agree_on_gradients(oracle, tiling):
    """The reverse pass of each line-kernel tiling (lambda points per thread, layers per
    warp, warps per CTA, lines per chunk, CTAs per SM) against the oracle's adjoint, on a
    layer count that leaves the last slab of every tiling partly or wholly past the bottom
    layer.  A slab, line or point that a tiling drops or counts twice is an O(1) error."""
    prob = tiny_problem(n_lambda=1037, n_depth=17, n_lines=300, W=400, seed=3)
    n = prob.grid.n_lambda
    f0 = oracle.forward(prob)
    rng = np.random.default_rng(17)
    y = (f0["f"] + rng.normal(0, 1e-3, n)).astype(np.float32).astype(np.float64)
    w = 1e4
    _, ggf, gg6, _, _ = oracle.gradient(prob, y, np.full(n, w), fwd=f0)
    got = run_gradient(prob, y.astype(np.float32), np.float32(w), pz.PZ_MIXED, tiling=tiling)
    e1 = rel_metric(got["g_gf"], ggf).max()
    e2 = rel_metric(got["g_g6"], gg6).max()
    assert e1 < G_TOL and e2 < G_TOL, (tiling, e1, e2)


def test_small_calibration_gradients(oracle):
    prob = I.small_config1(n_lambda_span_nm=3.0, seed=13)
    nl = prob.lines.n_lines
    rng = np.random.default_rng(5)
    corr = {"dlog_gf": np.zeros(nl), "dlog_gamma6": np.zeros(nl), "dabund": np.zeros(prob.n_elem)}
    print(_check(prob, oracle, corr))
    corr = {"dlog_gf": rng.normal(0, 0.1, nl), "dlog_gamma6": rng.normal(0, 0.2, nl),
            "dabund": rng.normal(0, 0.1, prob.n_elem)}
    print(_check(prob, oracle, corr))


def test_identity_instrument_gradients(oracle):
    prob = tiny_problem(n_lambda=900, n_depth=20, n_lines=60, W=350, seed=31)
    prob.lines.log_gf[:] -= 4.0
    rng = np.random.default_rng(6)
    corr = {"dlog_gf": rng.normal(0, 0.1, 60), "dlog_gamma6": rng.normal(0, 0.2, 60),
            "dabund": rng.normal(0, 0.1, prob.n_elem)}
    print(_check(prob, oracle, corr))


def test_autograd_function_matches_direct_call(oracle):
    import torch
    prob = tiny_problem(n_lambda=500, n_depth=12, n_lines=30, W=200, seed=9, instrument=True)
    prob.lines.log_gf[:] -= 4.0
    s = pz.Synthesizer(prob)
    Fn = pz.SynthesisFunction
    nl = prob.lines.n_lines
    dgf = torch.zeros(nl, dtype=torch.float32, device="cuda", requires_grad=True)
    dg6 = torch.zeros(nl, dtype=torch.float32, device="cuda", requires_grad=True)
    dab = torch.zeros(prob.n_elem, dtype=torch.float32, device="cuda", requires_grad=True)
    f = Fn.apply(s, dgf, dg6, dab)
    y = torch.ones_like(f)
    L = ((y - f) ** 2).sum() * 4e4
    L.backward()
    ref = oracle.gradient(prob, np.ones(f.numel()), np.full(f.numel(), 4e4),
                          {"dlog_gf": np.zeros(nl), "dlog_gamma6": np.zeros(nl), "dabund": np.zeros(prob.n_elem)})
    assert rel_metric(dgf.grad.cpu().numpy().astype(np.float64), ref[1]).max() < G_TOL
    assert rel_metric(dg6.grad.cpu().numpy().astype(np.float64), ref[2]).max() < G_TOL
    assert rel_metric(dab.grad.cpu().numpy().astype(np.float64), ref[3]).max() < G_TOL


def test_config3_full_size_gradients_match_the_fp64_form():
    """The calibration workload at full size (37,550 points, 1.2e5 lines, 8,575 pixels):
    mixed-path gradients for every line and element against the plain FP64 GPU form
    (which the small cases pin to the oracle's adjoint), metric c17, at the seeded
    S/N-200 target and at zero corrections."""
    import torch
    prob, truth = I.config3()
    n_out = prob.instrument.pix_lambda_nm.size
    s = pz.Synthesizer(prob, pz.PZ_MIXED)
    s.set_corrections(truth["dlog_gf"], truth["dlog_gamma6"], None)
    f_true = s.forward().cpu().numpy().astype(np.float64)
    s.close()
    y = (f_true + truth["noise"]).astype(np.float32)
    w = np.float32(truth["weight"])
    zero = {"dlog_gf": np.zeros(prob.lines.n_lines, np.float32),
            "dlog_gamma6": np.zeros(prob.lines.n_lines, np.float32),
            "dabund": np.zeros(prob.n_elem, np.float32)}
    mixed = run_gradient(prob, y, w, pz.PZ_MIXED, zero)
    ref = run_gradient(prob, y, w, pz.PZ_FP64, zero)
    assert abs(mixed["loss"] / ref["loss"] - 1) < 1e-4
    e1 = rel_metric(mixed["g_gf"], ref["g_gf"]).max()
    e2 = rel_metric(mixed["g_g6"], ref["g_g6"]).max()
    e3 = rel_metric(mixed["g_ab"][:prob.n_elem], ref["g_ab"][:prob.n_elem]).max()
    print("config3 full size: loss %.6g, max rel err gf %.3g g6 %.3g abund %.3g" % (ref["loss"], e1, e2, e3))
    assert e1 < G_TOL and e2 < G_TOL and e3 < G_TOL
    torch.cuda.synchronize()
