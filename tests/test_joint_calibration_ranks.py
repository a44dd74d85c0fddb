"""Joint calibration over ranks (Sec. 6, the shared corrections of several stars), on two
gloo ranks on the CPU: the stars of one fit are split between the ranks, each rank
evaluates its own stars at the shared corrections, and the driver sums the loss and the
gradient over the ranks with one all-reduce per evaluation.  Both ranks must return the
same corrections, the least-squares minimum of the whole fit, and report the whole fit's
objective.  The synthesizer is a linear least-squares stand-in with the Synthesizer's calls."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

N_LINES, N_ROWS = 40, 300


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fit(seed=11):
    """Rows of the whole fit (the pixels of all its stars): f = 1 + J c, c = (dlog_gf, dlog_gamma6)."""
    g = torch.Generator().manual_seed(seed)
    J = torch.randn(N_ROWS, 2 * N_LINES, generator=g, dtype=torch.float64) * 0.1
    truth = torch.randn(2 * N_LINES, generator=g, dtype=torch.float64) * 0.1
    y = (1.0 + J @ truth + torch.randn(N_ROWS, generator=g, dtype=torch.float64) / 200).float()
    return J, y, torch.full_like(y, 200.0 ** 2)


class RowsSynth:
    """The stars of one rank: the rows of J it owns, with the calls lbfgs makes."""

    def __init__(self, J):
        self.J = J
        self.n_lines = N_LINES
        self.c = torch.zeros(2 * N_LINES, dtype=torch.float64)

    def set_corrections(self, dlog_gf, dlog_gamma6, dabund, stream=None):
        self.c = torch.cat([torch.as_tensor(dlog_gf).double(), torch.as_tensor(dlog_gamma6).double()])

    def calib_step(self, y, w, lr_gf, lr_g6, lr_ab, loss, g_gf, g_g6, g_ab, stream=None):
        r = y.double() - (1.0 + self.J @ self.c)
        loss[0] = (w.double() * r * r).sum()
        g = -2.0 * self.J.T @ (w.double() * r)
        g_gf.copy_(g[:N_LINES])
        g_g6.copy_(g[N_LINES:])


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from paper_2607_24141_gb300 import calibrate
        J, y, w = _fit()
        rows = slice(rank * N_ROWS // ws, (rank + 1) * N_ROWS // ws)     # this rank's stars
        res = calibrate.lbfgs(RowsSynth(J[rows]), y[rows], w[rows], n_updates=60, process_group=dist.group.WORLD)
        q.put((rank, res["dlog_gf"].numpy(), res["dlog_gamma6"].numpy(), res["loss_start"], res["loss_final"],
               res["evals"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_joint_fit_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    from paper_2607_24141_gb300 import calibrate
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=150) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (_, gf0, g60, ls0, lf0, ev0), (_, gf1, g61, ls1, lf1, ev1) = out
    # the ranks saw the same sums, so they took the same steps
    assert np.array_equal(gf0, gf1) and np.array_equal(g60, g61)
    assert ev0 == ev1 and ls0 == ls1 and lf0 == lf1

    J, y, w = _fit()
    sw = np.sqrt(w.double().numpy())
    A = J.numpy() * sw[:, None]
    b = (y.double().numpy() - 1.0) * sw
    c_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    L_min = float(((A @ c_ls - b) ** 2).sum())
    assert ls0 == pytest.approx(float((b ** 2).sum()), rel=1e-6)          # the whole fit at zero corrections
    assert lf0 <= L_min * (1 + 1e-3)
    assert np.max(np.abs(np.concatenate([gf0, g60]) - c_ls)) < 1e-2
    # the same fit in one process over all the rows
    one = calibrate.lbfgs(RowsSynth(J), y, w, n_updates=60)
    assert one["loss_final"] == pytest.approx(lf0, rel=1e-3)
