"""Continuum-referenced centre test on the device against the FP64 oracle with the same
selection fraction: kept-pair counts, line opacity, flux and gradients of both forms,
and its limits (off = unchanged, everything rejected = continuum)."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from centre_util import centre_ratios
from gpu_util import kappa_rel, rel_metric

pytestmark = pytest.mark.gpu

ETA = 1e-3            # the paper's selection fraction


def _run(prob, prec, eta, corr=None, y=None, w=None):
    import torch
    s = pz.Synthesizer(prob, prec)
    if corr:
        s.set_corrections(corr.get("dlog_gf"), corr.get("dlog_gamma6"), corr.get("dabund"))
    kept = pz.pz_set_centre_test(s.ctx, eta)
    nd, nl = prob.atmos.n_depth, prob.grid.n_lambda
    kl = torch.empty((nd, nl), dtype=torch.float32, device=s.device)
    f = s.forward(kl)
    out = {"kept": kept, "kline": kl.cpu().numpy().astype(np.float64), "f": f.cpu().numpy().astype(np.float64)}
    if y is not None:
        dev = s.device
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        wt = torch.tensor(np.broadcast_to(w, y.shape), dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        dLdf = torch.empty(y.size, dtype=torch.float32, device=dev)
        s.loss(yt, wt, loss, dLdf)
        n = prob.lines.n_lines
        g1 = torch.empty(n, dtype=torch.float32, device=dev)
        g2 = torch.empty(n, dtype=torch.float32, device=dev)
        s.backward(dLdf, g1, g2, None)
        out.update(g_gf=g1.cpu().numpy().astype(np.float64), g_g6=g2.cpu().numpy().astype(np.float64))
    torch.cuda.synchronize()
    s.close()
    return out


def _expected_kept(prob, eta, corr=None):
    r = centre_ratios(prob, corr)
    near = np.abs(r / eta - 1) < 1e-9          # pairs on the threshold (none expected)
    return int((r >= eta).sum()), int(near.sum())


def test_centre_test_parity_and_gradients(oracle):
    prob = I.small_config1(n_lambda_span_nm=3.0, seed=13)
    nl = prob.lines.n_lines
    rng = np.random.default_rng(8)
    corr = {"dlog_gf": rng.normal(0, 0.1, nl).astype(np.float32),
            "dlog_gamma6": rng.normal(0, 0.2, nl).astype(np.float32)}
    c64 = {k: v.astype(np.float64) for k, v in corr.items()}
    ref = oracle.forward(prob, dict(c64, centre_eta=ETA))
    full = oracle.forward(prob, c64)
    n_out = prob.instrument.pix_lambda_nm.size
    y = (ref["f"] + rng.normal(0, 1 / 200, n_out)).astype(np.float32).astype(np.float64)
    w = np.full(n_out, 200.0 ** 2)
    _, ggf, gg6, _, _ = oracle.gradient(prob, y, w, dict(c64, centre_eta=ETA), fwd=ref)
    kept, ambiguous = _expected_kept(prob, ETA, c64)
    assert ambiguous == 0
    # the plain FP64 form still exchanges f, y and dL/df as FP32 through the C ABI; with
    # the sums cancelling over fewer pairs its gradients carry ~2e-5 of that rounding
    for prec, ktol, ftol, gtol in ((pz.PZ_MIXED, 3e-5, 1e-4, 1e-3), (pz.PZ_FP64, 1e-6, 1e-6, 1e-4)):
        got = _run(prob, prec, ETA, corr, y.astype(np.float32), np.float32(w[0]))
        assert got["kept"] == kept
        assert kappa_rel(got["kline"], ref["kline"], prob.kappa_c) < ktol
        assert np.max(np.abs(got["f"] - ref["f"])) < ftol
        assert rel_metric(got["g_gf"], ggf).max() < gtol
        assert rel_metric(got["g_g6"], gg6).max() < gtol
    # the cut changes the spectrum (report of the test's effect at this size)
    print("centre test eta=%g: kept %d of %d pairs, max |f_cut - f_full| %.3g"
          % (ETA, kept, nl * prob.atmos.n_depth, np.max(np.abs(ref["f"] - full["f"]))))


def test_centre_test_limits():
    prob = I.small_config1(n_lambda_span_nm=2.0, seed=3, with_instrument=False)
    base = _run(prob, pz.PZ_MIXED, 0.0)
    assert 0 < base["kept"] <= prob.lines.n_lines * prob.atmos.n_depth
    import torch
    s = pz.Synthesizer(prob, pz.PZ_MIXED)
    kl = torch.empty((prob.atmos.n_depth, prob.grid.n_lambda), dtype=torch.float32, device=s.device)
    s.forward(kl)
    # eta = 0 is the plain path (equal up to the order of the near-core shared-memory atomics)
    assert kappa_rel(kl.cpu().numpy().astype(np.float64), base["kline"], prob.kappa_c) < 1e-6
    s.close()
    none = _run(prob, pz.PZ_MIXED, 1e300)
    assert none["kept"] == 0
    assert np.all(none["kline"] == 0.0) and np.all(none["f"] == 1.0)
    with pytest.raises(pz.PzError) as e:
        _run(prob, pz.PZ_MIXED, -1.0)
    assert e.value.status == pz.PZ_EINVAL


def test_centre_test_config1_full_sampled(oracle):
    prob = I.config1()
    got = _run(prob, pz.PZ_MIXED, ETA)
    kept, ambiguous = _expected_kept(prob, ETA)
    assert abs(got["kept"] - kept) <= ambiguous
    rng = np.random.default_rng(4)
    cols = np.unique(np.concatenate([[0, 127, 128, prob.grid.n_lambda - 1], rng.integers(0, prob.grid.n_lambda, 10)]))
    kref = oracle.kappa_line(prob, cols, {"centre_eta": ETA})
    assert kappa_rel(got["kline"][:, cols], kref, prob.kappa_c[:, cols]) < 3e-5
