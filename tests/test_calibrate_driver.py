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


class LinearSynthWithState(LinearSynth):
    """LinearSynth with the read-back calls save_state needs and a line list."""

    def __init__(self, n_lines, n_data, seed=0):
        super().__init__(n_lines, n_data, seed)
        from paper_2607_24141_gb300 import inputs as I
        rng = np.random.default_rng(seed)
        self.prob = type("P", (), {})()
        self.prob.lines = I.LineList(
            lambda_nm=np.sort(rng.uniform(1500, 1700, n_lines)), log_gf=rng.normal(-2, 1, n_lines).astype(np.float32),
            E_low_eV=rng.uniform(0, 5, n_lines).astype(np.float32),
            log_gamma_rad=np.full(n_lines, 8.0, np.float32), log_gamma4=np.full(n_lines, -5.5, np.float32),
            log_gamma6=np.full(n_lines, -7.5, np.float32), species=rng.integers(0, 4, n_lines).astype(np.int32),
            half_window=1500)
        self.damp = (np.zeros(n_lines, np.float32), np.zeros(n_lines, np.float32))
        self.ab = np.zeros(3, np.float32)

    def get_corrections(self):
        c = self.c.numpy().astype(np.float32)
        return c[:self.n_lines].copy(), c[self.n_lines:].copy(), self.ab.copy()

    def get_damping_corrections(self):
        return self.damp[0].copy(), self.damp[1].copy()

    def set_corrections(self, dlog_gf, dlog_gamma6, dabund, stream=None):
        super().set_corrections(dlog_gf, dlog_gamma6, dabund, stream)
        if dabund is not None:
            self.ab = np.asarray(dabund, np.float32).copy()

    def set_damping_corrections(self, rad, g4, stream=None):
        self.damp = (np.asarray(rad, np.float32).copy(), np.asarray(g4, np.float32).copy())


def _state_problem(seed):
    s = LinearSynthWithState(40, 300, seed)
    g = torch.Generator().manual_seed(seed + 1)
    s.c = torch.randn(80, generator=g, dtype=torch.float64) * 0.1
    y = (s.f() + torch.randn(300, generator=g, dtype=torch.float64) / 200).float()
    s.c = torch.zeros(80, dtype=torch.float64)
    return s, y, torch.full_like(y, 200.0 ** 2)


def test_saved_fit_resumes_where_it_stopped(tmp_path):
    """Six updates, save, load into a fresh context, six more: the same corrections as
    twelve updates in one run (the L-BFGS history and step travel with the state)."""
    s, y, w = _state_problem(7)
    straight = calibrate.lbfgs(s, y, w, n_updates=12)
    s, y, w = _state_problem(7)
    first = calibrate.lbfgs(s, y, w, n_updates=6)
    path = str(tmp_path / "fit.pt")
    calibrate.save_state(path, s, first, meta={"note": "six updates"})
    s2, y2, w2 = _state_problem(7)
    state = calibrate.load_state(path, s2)
    assert state["meta"]["note"] == "six updates"
    np.testing.assert_array_equal(s2.c.numpy(), s.c.numpy())       # corrections restored
    second = calibrate.lbfgs(s2, y2, w2, n_updates=6, resume=state)
    np.testing.assert_allclose(second["dlog_gf"].numpy(), straight["dlog_gf"].numpy(), rtol=1e-5, atol=1e-7)
    assert second["loss_final"] == pytest.approx(straight["loss_final"], rel=1e-6)


def test_state_is_bound_to_its_line_list(tmp_path):
    s, y, w = _state_problem(2)
    res = calibrate.lbfgs(s, y, w, n_updates=3)
    path = str(tmp_path / "fit.pt")
    calibrate.save_state(path, s, res)
    other, _, _ = _state_problem(3)                 # another catalog
    with pytest.raises(ValueError):
        calibrate.load_state(path, other)
    same = LinearSynthWithState(40, 300, 2)
    calibrate.load_state(path, same)
    edited = LinearSynthWithState(40, 300, 2)
    edited.prob.lines.log_gf[5] += 0.01             # one edited record changes the digest
    with pytest.raises(ValueError):
        calibrate.load_state(path, edited)
