"""Host logic of the L-BFGS calibration driver on a linear least-squares stand-in for the
synthesizer (CPU): the driver reports the objective at zero and at the returned
corrections, and on a quadratic it reaches the exact least-squares minimum."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_24141_gb300 import calibrate


class LinearSynth:
    """f = 1 + J c with c = (dlog_gf, dlog_gamma6); the same calls as a Synthesizer."""

    def __init__(self, n_lines, n_data, seed=0):
        g = torch.Generator().manual_seed(seed)
        self.n_lines = n_lines
        self.J = torch.randn(n_data, 2 * n_lines, generator=g, dtype=torch.float64) * 0.1
        self.c = torch.zeros(2 * n_lines, dtype=torch.float64)
        self.steps = 0

    def set_corrections(self, dlog_gf, dlog_gamma6, dabund, stream=None):
        self.c = torch.cat([torch.as_tensor(dlog_gf).double(), torch.as_tensor(dlog_gamma6).double()])

    def f(self):
        return 1.0 + self.J @ self.c

    def calib_step(self, y, w, lr_gf, lr_g6, lr_ab, loss, g_gf, g_g6, g_ab, stream=None):
        assert lr_gf == lr_g6 == lr_ab == 0.0
        r = y.double() - self.f()
        loss[0] = (w.double() * r * r).sum()
        g = -2.0 * self.J.T @ (w.double() * r)
        g_gf.copy_(g[:self.n_lines])
        g_g6.copy_(g[self.n_lines:])
        self.steps += 1


def _problem(seed=0):
    s = LinearSynth(40, 300, seed)
    g = torch.Generator().manual_seed(seed + 1)
    truth = torch.randn(80, generator=g, dtype=torch.float64) * 0.1
    s.c = truth
    y = (s.f() + torch.randn(300, generator=g, dtype=torch.float64) / 200).float()
    w = torch.full_like(y, 200.0 ** 2)
    s.c = torch.zeros(80, dtype=torch.float64)
    return s, y, w


def test_driver_reports_start_and_final_objectives():
    s, y, w = _problem()
    w64 = w.double()
    L0 = float((w64 * (y.double() - 1.0) ** 2).sum())
    res = calibrate.lbfgs(s, y, w, n_updates=10)
    assert res["loss_start"] == pytest.approx(L0, rel=1e-6)
    assert res["updates"] == 10
    assert res["evals"] >= 10 and s.steps == res["evals"] + 2
    s.set_corrections(res["dlog_gf"], res["dlog_gamma6"], None)
    r = y.double() - s.f()
    assert res["loss_final"] == pytest.approx(float((w64 * r * r).sum()), rel=1e-6)
    assert res["loss_final"] < 1e-2 * res["loss_start"]


def test_driver_reaches_the_least_squares_minimum():
    s, y, w = _problem(3)
    sw = np.sqrt(w.double().numpy())
    A = s.J.numpy() * sw[:, None]
    b = (y.double().numpy() - 1.0) * sw
    c_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    L_min = float(((A @ c_ls - b) ** 2).sum())
    res = calibrate.lbfgs(s, y, w, n_updates=60)
    # FP32 corrections (as the device path holds them) bound how close it can get
    assert res["loss_final"] <= L_min * (1 + 1e-3)
    est = np.concatenate([res["dlog_gf"].numpy(), res["dlog_gamma6"].numpy()])
    assert np.max(np.abs(est - c_ls)) < 1e-2


def test_driver_without_gamma6():
    s, y, w = _problem(5)
    res = calibrate.lbfgs(s, y, w, n_updates=20, fit_gamma6=False)
    assert np.all(res["dlog_gamma6"].numpy() == 0.0)
    sw = np.sqrt(w.double().numpy())
    A = s.J.numpy()[:, :40] * sw[:, None]
    b = (y.double().numpy() - 1.0) * sw
    L_min = float(((A @ np.linalg.lstsq(A, b, rcond=None)[0] - b) ** 2).sum())
    assert res["loss_final"] <= L_min * (1 + 1e-3)
