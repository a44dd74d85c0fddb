"""Full-size parity against the FP64 oracle's stored results (tests/golden, written by
the scripts there, which call only the oracle):

* the calibration workload (37,550 points, 1.2e5 lines, 8,575 pixels): normalised flux
  on every pixel, chi^2, and the gradients of every line and element at zero
  corrections; the stored oracle adjoint is itself checked against central differences
  of the oracle's loss on 200 seeded lines;
* the 64-star batch in the benchmark's launch configuration: every pixel and every line
  gradient of the two stars with the fewest lines (chi^2 weights of one star at a time),
  and 12 pixels of the star with the most lines and of star 17.

Bars: |df| <= 1e-4, gradients within 1e-3 (error metric |g - ref| / max(|ref|, 1e-3
max|ref|)); the plain FP64 GPU form of the calibration workload within 1e-6 / 1e-5."""
import os

import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from gpu_util import rel_metric

HERE = os.path.dirname(os.path.abspath(__file__))
F_TOL, G_TOL = 1e-4, 1e-3


def _golden(name):
    path = os.path.join(HERE, "golden", name + "_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("stored oracle results %s not present" % path)
    return dict(np.load(path))


def test_config3_oracle_adjoint_matches_central_differences():
    """The stored oracle adjoint of the full-size calibration workload against central
    differences (h = 1e-4) of the oracle's own loss on 200 seeded lines, 1e-6."""
    gd = _golden("config3")
    for key, gmax in (("gf", gd["g_gf_max"]), ("g6", gd["g_g6_max"])):
        adj, fd = gd["adj_g_" + key], gd["fd_g_" + key]
        err = np.abs(adj - fd) / np.maximum(np.abs(fd), 1e-3 * gmax)
        assert err.max() < 1e-6, (key, err.max())
    assert gd["fd_lines"].size == 200


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [pz.PZ_MIXED, pz.PZ_FP64])
def test_config3_full_size_against_the_oracle(prec):
    import torch
    gd = _golden("config3")
    prob, _ = I.config3()
    nl, n_elem = prob.lines.n_lines, prob.n_elem
    s = pz.Synthesizer(prob, prec)
    dev = s.device
    z = torch.zeros(nl, dtype=torch.float32, device=dev)
    s.set_corrections(z, z, torch.zeros(n_elem, dtype=torch.float32, device=dev))
    f = s.forward()
    y = torch.tensor(gd["y"], dtype=torch.float32, device=dev)
    w = torch.full_like(y, 200.0 ** 2)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    dLdf = torch.empty_like(y)
    s.loss(y, w, loss, dLdf)
    g = [torch.empty(nl, dtype=torch.float32, device=dev) for _ in range(2)]
    gab = torch.empty(n_elem, dtype=torch.float32, device=dev)
    s.backward(dLdf, g[0], g[1], gab)
    torch.cuda.synchronize()
    df = np.abs(f.cpu().numpy().astype(np.float64) - gd["f"])
    e = [rel_metric(g[0].cpu().numpy().astype(np.float64), gd["g_gf"].astype(np.float64)).max(),
         rel_metric(g[1].cpu().numpy().astype(np.float64), gd["g_g6"].astype(np.float64)).max(),
         rel_metric(gab.cpu().numpy().astype(np.float64), gd["g_ab"]).max()]
    lr = abs(loss.item() / float(gd["loss"]) - 1)
    print("config3 %s vs oracle: |df| max %.3g p99 %.3g rms %.3g; loss %.3g; grad gf %.3g g6 %.3g abund %.3g"
          % ("mixed" if prec == pz.PZ_MIXED else "fp64", df.max(), np.quantile(df, 0.99), np.sqrt(np.mean(df ** 2)),
             lr, *e))
    ftol, gtol, ltol = (F_TOL, G_TOL, 1e-4) if prec == pz.PZ_MIXED else (1e-6, 1e-5, 1e-6)
    assert df.max() < ftol and max(e) < gtol and lr < ltol
    s.close()


@pytest.mark.gpu
def test_config4_stars_against_the_oracle():
    import torch
    gd = _golden("config4")
    b = I.config4()
    assert [len(x) for x in b.subsets] == list(gd["n_lines_per_star"])
    s = pz.Synthesizer(b)
    dev = s.device
    nl, n_elem = b.lines.n_lines, b.n_elem
    z = torch.zeros(nl, dtype=torch.float32, device=dev)
    zab = torch.zeros(n_elem, dtype=torch.float32, device=dev)
    s.set_corrections(z, z, zab)
    f = s.forward().cpu().numpy().astype(np.float64)
    for k in gd["full_stars"]:
        df = np.abs(f[k] - gd["star%d_f" % k])
        print("config4 star %d: |df| max %.3g rms %.3g" % (k, df.max(), np.sqrt(np.mean(df ** 2))))
        assert df.max() < F_TOL
    pix = gd["sampled_pixels"]
    for k in gd["sampled_stars"]:
        df = np.abs(f[k][pix] - gd["star%d_f_sampled" % k])
        print("config4 star %d sampled: |df| max %.3g" % (k, df.max()))
        assert df.max() < F_TOL
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = [torch.empty(nl, dtype=torch.float32, device=dev) for _ in range(2)]
    gab = torch.empty(n_elem, dtype=torch.float32, device=dev)
    n_out = s.n_out
    for k in gd["full_stars"]:
        y = torch.zeros((b.n_stars, n_out), dtype=torch.float32, device=dev)
        w = torch.zeros_like(y)
        y[k] = torch.tensor(gd["star%d_y" % k], device=dev)
        w[k] = 200.0 ** 2
        s.calib_step(y, w, 0.0, 0.0, 0.0, loss, g[0], g[1], gab)
        torch.cuda.synchronize()
        sub = b.subsets[k]
        e = [rel_metric(g[0].cpu().numpy()[sub].astype(np.float64), gd["star%d_g_gf" % k].astype(np.float64)).max(),
             rel_metric(g[1].cpu().numpy()[sub].astype(np.float64), gd["star%d_g_g6" % k].astype(np.float64)).max(),
             rel_metric(gab.cpu().numpy().astype(np.float64), gd["star%d_g_ab" % k]).max()]
        other = np.setdiff1d(np.arange(nl), sub)
        assert np.all(g[0].cpu().numpy()[other] == 0.0)
        lr = abs(loss.item() / float(gd["star%d_loss" % k]) - 1)
        print("config4 star %d gradients: gf %.3g g6 %.3g abund %.3g, loss %.3g" % (k, *e, lr))
        assert max(e) < G_TOL and lr < 1e-4
    s.close()
