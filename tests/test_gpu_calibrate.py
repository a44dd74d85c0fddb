"""Multi-update L-BFGS line-list calibration (Sec. 6) on a small two-star batch with
seeded true corrections and S/N-200 noise: the chi-square falls toward the noise floor,
and the reported final objective is the objective at the returned corrections."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import calibrate
from paper_2607_24141_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_lbfgs_calibration_recovers_the_fit():
    import torch
    b = I.small_batch(n_stars=2, span_nm=3.0, seed=31)
    nl = b.lines.n_lines
    rng = np.random.default_rng(12)
    truth_gf = rng.normal(0, 0.1, nl).astype(np.float32)
    truth_g6 = rng.normal(0, 0.2, nl).astype(np.float32)
    s = pz.Synthesizer(b, pz.PZ_MIXED)
    s.set_corrections(truth_gf, truth_g6, None)
    f_true = s.forward()
    sn = 1000.0                                      # S/N high enough that the corrections dominate chi^2
    noise = torch.tensor(rng.normal(0, 1 / sn, tuple(f_true.shape)), dtype=torch.float32, device=f_true.device)
    y = (f_true + noise).contiguous()
    w = torch.full_like(y, sn ** 2)
    loss = torch.zeros(1, dtype=torch.float64, device=y.device)
    s.calib_step(y, w, 0.0, 0.0, 0.0, loss, None, None, None)      # captures the step once
    chi2_truth = float(loss.item())
    s.set_corrections(np.zeros(nl, np.float32), np.zeros(nl, np.float32), None)
    s.forward()
    res = calibrate.lbfgs(s, y, w, n_updates=15)
    n_data = y.numel()
    print("L-BFGS: chi2 %.4g -> %.4g (%.4g at the true corrections) over %d updates, %d evaluations, %.3f s "
          "(n_data %d)" % (res["loss_start"], res["loss_final"], chi2_truth, res["updates"], res["evals"],
                           res["seconds"], n_data))
    assert res["updates"] == 15
    assert res["loss_start"] > 5.0 * chi2_truth
    assert res["loss_final"] < 0.2 * res["loss_start"]
    assert res["loss_final"] < 1.1 * chi2_truth         # at or below the fit of the true corrections
    # the reported objective is the objective at the returned corrections
    s.set_corrections(res["dlog_gf"], res["dlog_gamma6"], None)
    f = s.forward()
    chi2 = float(((y - f) ** 2 * w).double().sum())
    assert abs(chi2 / res["loss_final"] - 1) < 1e-4
    s.close()


def test_grouped_lbfgs_calibration():
    """Four corrections per linked group (Eq. 10 with q(l)): L-BFGS over pz_group_eval
    fits a two-star slice with true group corrections to below the chi-square of the
    truth."""
    import torch
    b = I.small_batch(n_stars=2, span_nm=3.0, seed=33)
    nl = b.lines.n_lines
    rng = np.random.default_rng(14)
    G = nl // 2
    q = rng.integers(0, G, nl).astype(np.int32)
    q[:G] = np.arange(G)
    rng.shuffle(q)
    x_true = np.stack([rng.normal(0, 0.1, G), rng.normal(0, 0.3, G), rng.normal(0, 0.3, G),
                       rng.normal(0, 0.2, G)]).astype(np.float32)
    s = pz.Synthesizer(b, pz.PZ_MIXED)
    xl = x_true[:, q]
    s.set_corrections(xl[0], xl[3], None)
    pz.pz_set_damping_corrections(s.ctx, xl[1], xl[2])
    f_true = s.forward()
    sn = 1000.0
    y = (f_true + torch.tensor(rng.normal(0, 1 / sn, tuple(f_true.shape)), dtype=torch.float32,
                               device=f_true.device)).contiguous()
    w = torch.full_like(y, sn ** 2)
    pz.pz_set_line_groups(s.ctx, q, G)
    loss = torch.zeros(1, dtype=torch.float64, device=y.device)
    pz.pz_group_eval(s.ctx, y, w, torch.tensor(x_true, device=y.device), loss, None)
    chi2_truth = float(loss.item())
    res = calibrate.lbfgs_groups(s, y, w, q, G, n_updates=15)
    print("grouped L-BFGS: chi2 %.4g -> %.4g (%.4g at the truth), %d updates, %d evaluations, %.3f s, %d groups"
          % (res["loss_start"], res["loss_final"], chi2_truth, res["updates"], res["evals"], res["seconds"], G))
    assert res["updates"] == 15
    assert res["loss_start"] > 3.0 * chi2_truth
    assert res["loss_final"] < 0.25 * res["loss_start"]
    assert res["loss_final"] < 1.1 * chi2_truth
    # the context holds the expanded fit
    gf, g6, _ = s.get_corrections()
    xf = res["groups"].cpu().numpy()
    np.testing.assert_array_equal(gf, xf[0][q])
    np.testing.assert_array_equal(g6, xf[3][q])
    s.close()


@pytest.mark.timeout(300)
def test_joint_fit_through_one_nccl_rank_matches_the_plain_fit():
    """The device path of the joint calibration over ranks: with one NCCL rank the all-reduce
    of loss and gradient and the broadcast of the starting point are identities, so the fit
    through process_group= must equal the plain fit bit for bit.  The plain FP64 form is
    used because it is bit-reproducible from run to run (the mixed form's near-core atomics
    are not)."""
    import os
    import socket

    import torch
    import torch.distributed as dist
    if not dist.is_nccl_available():
        pytest.skip("torch.distributed has no NCCL backend")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    saved = {k: os.environ.get(k) for k in ("MASTER_ADDR", "MASTER_PORT")}
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dev = torch.device("cuda", torch.cuda.current_device())
    b = I.small_batch(n_stars=2, span_nm=3.0, seed=31)
    nl = b.lines.n_lines
    rng = np.random.default_rng(12)
    s = pz.Synthesizer(b, pz.PZ_FP64)
    s.set_corrections(rng.normal(0, 0.1, nl).astype(np.float32), rng.normal(0, 0.2, nl).astype(np.float32), None)
    f_true = s.forward()
    y = (f_true + torch.tensor(rng.normal(0, 1e-3, tuple(f_true.shape)), dtype=torch.float32, device=dev)).contiguous()
    w = torch.full_like(y, 1e6)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=dev)
    try:
        out = []
        for pg in (None, dist.group.WORLD):
            s.set_corrections(np.zeros(nl, np.float32), np.zeros(nl, np.float32), None)
            s.forward()
            out.append(calibrate.lbfgs(s, y, w, n_updates=10, process_group=pg))
    finally:
        dist.destroy_process_group()
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    plain, joint = out
    assert np.array_equal(plain["dlog_gf"].cpu().numpy(), joint["dlog_gf"].cpu().numpy())
    assert np.array_equal(plain["dlog_gamma6"].cpu().numpy(), joint["dlog_gamma6"].cpu().numpy())
    assert plain["loss_start"] == joint["loss_start"] and plain["loss_final"] == joint["loss_final"]
    assert plain["evals"] == joint["evals"]
    assert joint["loss_final"] < 0.2 * joint["loss_start"]
