"""Four-parameter grouped calibration on the device (Sec. 6, Eq. 10 with linked groups)
against the FP64 oracle: the four per-line gradients of pz_backward4 in both forms, and
the captured group evaluation (objective and group gradients) of pz_group_eval."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I
from gpu_util import rel_metric

pytestmark = pytest.mark.gpu
KEYS = ("dlog_gf", "dlog_gamma_rad", "dlog_gamma4", "dlog_gamma6")


def _rounded(d):
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in d.items()}


def _target(oracle, prob, corr, seed):
    rng = np.random.default_rng(seed)
    f0 = oracle.forward(prob, corr)
    n_out = f0["f"].size
    y = (f0["f"] + rng.normal(0, 1 / 200, n_out)).astype(np.float32).astype(np.float64)
    return y, np.full(n_out, 200.0 ** 2), f0


def test_backward4_parity(oracle):
    import torch
    prob = I.small_config1(n_lambda_span_nm=3.0, seed=13)
    nl = prob.lines.n_lines
    rng = np.random.default_rng(5)
    corr = _rounded({"dlog_gf": rng.normal(0, 0.1, nl), "dlog_gamma_rad": rng.normal(0, 0.3, nl),
                     "dlog_gamma4": rng.normal(0, 0.3, nl), "dlog_gamma6": rng.normal(0, 0.2, nl)})
    y, w, f0 = _target(oracle, prob, corr, 7)
    ref = oracle.gradient4(prob, y, w, corr, fwd=f0)
    for prec, tol in ((pz.PZ_MIXED, 1e-3), (pz.PZ_FP64, 1e-5)):
        s = pz.Synthesizer(prob, prec)
        s.set_corrections(corr["dlog_gf"].astype(np.float32), corr["dlog_gamma6"].astype(np.float32), None)
        pz.pz_set_damping_corrections(s.ctx, corr["dlog_gamma_rad"].astype(np.float32),
                                      corr["dlog_gamma4"].astype(np.float32))
        f = s.forward()
        dev = s.device
        assert np.max(np.abs(f.cpu().numpy() - f0["f"])) < (1e-4 if prec == pz.PZ_MIXED else 1e-6)
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        wt = torch.tensor(w, dtype=torch.float32, device=dev)
        dLdf = torch.empty(y.size, dtype=torch.float32, device=dev)
        s.loss(yt, wt, None, dLdf)
        g = [torch.empty(nl, dtype=torch.float32, device=dev) for _ in range(4)]
        pz.pz_backward4(s.ctx, dLdf, g[0], g[1], g[2], g[3])
        got = [x.cpu().numpy().astype(np.float64) for x in g]
        errs = [rel_metric(got[0], ref["gf"]).max(), rel_metric(got[1], ref["gamma_rad"]).max(),
                rel_metric(got[2], ref["gamma4"]).max(), rel_metric(got[3], ref["gamma6"]).max()]
        print("backward4", prec, errs)
        assert max(errs) < tol, (prec, errs)
        # the first pass is pz_backward's: same gf and van der Waals gradients
        h = [torch.empty(nl, dtype=torch.float32, device=dev) for _ in range(2)]
        s.backward(dLdf, h[0], h[1], None)
        for a, b in ((h[0], got[0]), (h[1], got[3])):
            assert rel_metric(a.cpu().numpy().astype(np.float64), b).max() < 1e-6
        s.close()


def _grouping(nl, seed):
    rng = np.random.default_rng(seed)
    G = max(nl // 3, 1)
    q = rng.integers(0, G, nl).astype(np.int32)
    q[rng.uniform(size=nl) < 0.05] = -1                  # some lines take no correction
    q[:G] = np.arange(G)                                  # every group has a member
    rng.shuffle(q)
    used = np.unique(q[q >= 0])
    remap = -np.ones(G, np.int32)
    remap[used] = np.arange(used.size)
    return np.where(q >= 0, remap[np.maximum(q, 0)], -1).astype(np.int32), int(used.size)


@pytest.mark.parametrize("prec", [pz.PZ_MIXED, pz.PZ_FP64])
def test_group_eval_parity(oracle, prec):
    import torch
    prob = I.small_config1(n_lambda_span_nm=2.0, seed=17)
    nl = prob.lines.n_lines
    q, G = _grouping(nl, 3)
    rng = np.random.default_rng(11)
    x = rng.normal(0, [[0.1], [0.3], [0.3], [0.2]], (4, G)).astype(np.float32)
    e = oracle.expand_groups(x.astype(np.float64), q)
    corr = {k: e[j] for j, k in enumerate(KEYS)}
    y, w, f0 = _target(oracle, prob, corr, 8)
    ref = oracle.gradient4(prob, y, w, corr, fwd=f0)
    g_ref = oracle.group_sum(np.stack([ref["gf"], ref["gamma_rad"], ref["gamma4"], ref["gamma6"]]), q, G)
    s = pz.Synthesizer(prob, prec)
    s.forward()                                            # configures the instrument once
    pz.pz_set_line_groups(s.ctx, q, G)
    dev = s.device
    yt = torch.tensor(y, dtype=torch.float32, device=dev)
    wt = torch.tensor(w, dtype=torch.float32, device=dev)
    xt = torch.tensor(x, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.empty((4, G), dtype=torch.float32, device=dev)
    pz.pz_group_eval(s.ctx, yt, wt, xt, loss, g)
    L1, g1 = loss.item(), g.cpu().numpy().astype(np.float64)
    tol = 1e-3 if prec == pz.PZ_MIXED else 1e-5
    assert abs(L1 / ref["L"] - 1) < (1e-3 if prec == pz.PZ_MIXED else 1e-5)
    errs = [rel_metric(g1[j], g_ref[j]).max() for j in range(4)]
    print("group eval", prec, errs, "groups", G, "of", nl, "lines")
    assert max(errs) < tol, errs
    # the corrections left in the context are the expanded x
    gf, g6, _ = s.get_corrections()
    np.testing.assert_array_equal(gf, np.where(q >= 0, x[0][np.maximum(q, 0)], 0).astype(np.float32))
    np.testing.assert_array_equal(g6, np.where(q >= 0, x[3][np.maximum(q, 0)], 0).astype(np.float32))
    # a replay of the captured graph on new x
    xt.mul_(0.5)
    pz.pz_group_eval(s.ctx, yt, wt, xt, loss, g)
    e2 = oracle.expand_groups(0.5 * x.astype(np.float64), q)
    ref2 = oracle.gradient4(prob, y, w, {k: e2[j] for j, k in enumerate(KEYS)})
    assert abs(loss.item() / ref2["L"] - 1) < (1e-3 if prec == pz.PZ_MIXED else 1e-5)
    s.close()


def test_group_eval_state_errors():
    import torch
    prob = I.small_config1(n_lambda_span_nm=1.0, seed=2)
    s = pz.Synthesizer(prob)
    s.forward()
    dev = s.device
    y = torch.ones(s.n_out, dtype=torch.float32, device=dev)
    x = torch.zeros((4, 1), dtype=torch.float32, device=dev)
    with pytest.raises(pz.PzError) as e:
        pz.pz_group_eval(s.ctx, y, None, x)
    assert e.value.status == pz.PZ_ESTATE
    with pytest.raises(pz.PzError) as e:
        pz.pz_set_line_groups(s.ctx, np.full(prob.lines.n_lines, 5, np.int32), 3)
    assert e.value.status == pz.PZ_EINVAL
    s.close()


def test_group_eval_batch_parity(oracle):
    """Two stars with uneven line subsets sharing the grouped corrections: the objective
    is the sum over the stars and each group gradient sums its members over the stars."""
    import torch
    b = I.small_batch(n_stars=2, span_nm=1.5, seed=41)
    nl = b.lines.n_lines
    q, G = _grouping(nl, 5)
    rng = np.random.default_rng(13)
    x = rng.normal(0, [[0.1], [0.3], [0.3], [0.2]], (4, G)).astype(np.float32)
    e = oracle.expand_groups(x.astype(np.float64), q)
    L_ref, g_line = 0.0, np.zeros((4, nl))
    ys = []
    for k in range(b.n_stars):
        pk = b.star(k)
        sub = b.subsets[k]
        corr = {key: e[j][sub] for j, key in enumerate(KEYS)}
        y, w, f0 = _target(oracle, pk, corr, 20 + k)
        ys.append(y)
        r = oracle.gradient4(pk, y, w, corr, fwd=f0)
        L_ref += r["L"]
        for j, key in enumerate(("gf", "gamma_rad", "gamma4", "gamma6")):
            np.add.at(g_line[j], sub, r[key])
    g_ref = oracle.group_sum(g_line, q, G)
    s = pz.Synthesizer(b, pz.PZ_MIXED)
    s.forward()
    pz.pz_set_line_groups(s.ctx, q, G)
    dev = s.device
    yt = torch.tensor(np.stack(ys), dtype=torch.float32, device=dev)
    wt = torch.full_like(yt, 200.0 ** 2)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.empty((4, G), dtype=torch.float32, device=dev)
    pz.pz_group_eval(s.ctx, yt, wt, torch.tensor(x, device=dev), loss, g)
    assert abs(loss.item() / L_ref - 1) < 1e-3
    g1 = g.cpu().numpy().astype(np.float64)
    errs = [rel_metric(g1[j], g_ref[j]).max() for j in range(4)]
    print("group eval batch", errs)
    assert max(errs) < 1e-3, errs
    r_rad, r_4 = s.get_damping_corrections()
    np.testing.assert_array_equal(r_rad, np.where(q >= 0, x[1][np.maximum(q, 0)], 0).astype(np.float32))
    np.testing.assert_array_equal(r_4, np.where(q >= 0, x[2][np.maximum(q, 0)], 0).astype(np.float32))
    s.close()


def test_autograd_function4_matches_the_oracle(oracle):
    import torch
    prob = I.small_config1(n_lambda_span_nm=1.5, seed=19)
    nl = prob.lines.n_lines
    rng = np.random.default_rng(3)
    c = {k: rng.normal(0, 0.2, nl).astype(np.float32) for k in KEYS}
    c64 = {k: v.astype(np.float64) for k, v in c.items()}
    y, w, f0 = _target(oracle, prob, c64, 9)
    ref = oracle.gradient4(prob, y, w, c64, fwd=f0)
    s = pz.Synthesizer(prob)
    dev = s.device
    t = {k: torch.tensor(v, device=dev, requires_grad=True) for k, v in c.items()}
    f = pz.SynthesisFunction4.apply(s, t["dlog_gf"], t["dlog_gamma_rad"], t["dlog_gamma4"], t["dlog_gamma6"], None)
    yt = torch.tensor(y, dtype=torch.float32, device=dev)
    L = (((yt - f) ** 2) * float(w[0])).double().sum()
    L.backward()
    assert abs(L.item() / ref["L"] - 1) < 1e-3
    for key, rk in zip(KEYS, ("gf", "gamma_rad", "gamma4", "gamma6")):
        err = rel_metric(t[key].grad.cpu().numpy().astype(np.float64), ref[rk]).max()
        assert err < 1e-3, (key, err)
    s.close()
