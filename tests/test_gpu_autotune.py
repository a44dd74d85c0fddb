"""The line-kernel autotuner: it keeps a supported tiling, invalidates the forward
state, and the spectrum and gradients computed afterwards still match the oracle."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from gpu_util import kappa_rel, rel_metric
from tiny import tiny_problem

pytestmark = pytest.mark.gpu

SUPPORTED = {(4, 6, 1), (4, 6, 2), (4, 6, 3), (4, 6, 4), (4, 6, 5), (4, 6, 6), (4, 8, 1), (4, 8, 2), (4, 8, 3),
             (4, 12, 1), (4, 12, 2), (2, 6, 4), (2, 6, 6), (2, 8, 2), (2, 8, 3), (2, 8, 4), (2, 8, 5), (2, 12, 1),
             (2, 12, 2), (2, 12, 3)}


def test_autotune_keeps_results(oracle):
    import torch
    prob = tiny_problem(n_lambda=1037, n_depth=17, n_lines=300, W=400, seed=5)
    ref = oracle.forward(prob)
    rng = np.random.default_rng(2)
    n = prob.grid.n_lambda
    # the device objective reads FP32 targets: the oracle gets the same rounded values
    y = (ref["f"] + rng.normal(0, 1e-3, n)).astype(np.float32).astype(np.float64)
    w = np.full(n, 1e4)
    _, ggf, gg6, _, _ = oracle.gradient(prob, y, w, fwd=ref)

    s = pz.Synthesizer(prob, pz.PZ_MIXED)
    dev = s.device
    s.forward()
    yt = torch.tensor(y, dtype=torch.float32, device=dev)
    wt = torch.tensor(w, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    dLdf = torch.empty(n, dtype=torch.float32, device=dev)
    s.loss(yt, wt, loss, dLdf)
    nl = prob.lines.n_lines
    g_gf = torch.empty(nl, dtype=torch.float32, device=dev)
    g_g6 = torch.empty(nl, dtype=torch.float32, device=dev)
    s.backward(dLdf, g_gf, g_g6, None)

    res = pz.pz_autotune(s.ctx, with_backward=True, reps=1)
    J, DS, GW, LC, MINB = res["tiling"]
    assert (J, DS, MINB) in SUPPORTED and 1 <= GW <= 4 and 16 <= LC <= 256
    assert res["candidates"] >= 20
    assert res["fwd_ms"] > 0 and res["bwd_ms"] > 0

    # the forward state is invalidated by the tuning passes
    with pytest.raises(pz.PzError) as e:
        pz.pz_flux(s.ctx)
    assert e.value.status == pz.PZ_ESTATE

    kl = torch.empty((prob.atmos.n_depth, n), dtype=torch.float32, device=dev)
    f = s.forward(kl)
    s.loss(yt, wt, loss, dLdf)
    s.backward(dLdf, g_gf, g_g6, None)
    torch.cuda.synchronize()
    assert kappa_rel(kl.cpu().numpy().astype(np.float64), ref["kline"], prob.kappa_c) < 3e-5
    assert np.max(np.abs(f.cpu().numpy() - ref["f"])) < 1e-4
    assert np.max(rel_metric(g_gf.cpu().numpy().astype(np.float64), ggf)) < 1e-3
    assert np.max(rel_metric(g_g6.cpu().numpy().astype(np.float64), gg6)) < 1e-3


def test_autotune_forward_only_and_errors():
    prob = tiny_problem(n_lambda=600, n_depth=9, n_lines=80, W=120, seed=6)
    s = pz.Synthesizer(prob, pz.PZ_MIXED)
    res = pz.pz_autotune(s.ctx, with_backward=False, reps=1)
    assert res["bwd_ms"] == 0.0 and res["fwd_ms"] > 0
    with pytest.raises(pz.PzError) as e:
        pz.pz_autotune(s.ctx, reps=0)
    assert e.value.status == pz.PZ_EINVAL
    s64 = pz.Synthesizer(prob, pz.PZ_FP64)
    with pytest.raises(pz.PzError) as e:
        pz.pz_autotune(s64.ctx)
    assert e.value.status == pz.PZ_EINVAL
