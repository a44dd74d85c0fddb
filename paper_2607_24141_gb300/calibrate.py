"""Multi-update line-list calibration (Sec. 6): L-BFGS over shared line corrections of
one or more stars.

Every function and gradient evaluation is one captured graph launch: either
``pz_calib_step`` with zero learning rates (per-line Delta log gf and Delta log gamma_6),
or ``pz_group_eval`` (the four corrections of Eq. 10 -- gf and the radiative, Stark and
van der Waals damping -- shared by the members of each linked group).  Each runs the
corrections, line opacity, transfer, instrument, chi-square over all stars and the
hand-written reverse pass on the device.  The optimiser that proposes the next
corrections is PyTorch's L-BFGS (two-loop recursion with a strong-Wolfe line search) on
device tensors; it does no synthesis arithmetic.  The paper drives its shared
Sun-Arcturus fit the same way (40 L-BFGS updates).
"""
from __future__ import annotations

import time


def _minimise(set_and_eval, n_params, dev, n_updates, history):
    """L-BFGS on a float64 device vector of n_params; set_and_eval(x) -> (loss, grad)."""
    import torch

    x = torch.zeros(n_params, dtype=torch.float64, device=dev, requires_grad=True)
    evals = [0]
    t_eval = [0.0]

    def objective():
        t = time.perf_counter()
        loss, grad = set_and_eval(x.detach())
        evals[0] += 1
        x.grad = grad.to(torch.float64)
        out = float(loss)                       # a copy: the buffer is rewritten by the next evaluation
        t_eval[0] += time.perf_counter() - t
        return out

    opt = torch.optim.LBFGS([x], lr=1.0, max_iter=n_updates, max_eval=4 * n_updates, history_size=history,
                            line_search_fn="strong_wolfe", tolerance_grad=0.0, tolerance_change=0.0)
    sync = torch.cuda.synchronize if x.is_cuda else (lambda: None)
    objective()                                 # untimed: captures the step's graph for these buffers
    evals[0] = 0
    t_eval[0] = 0.0
    sync()
    t0 = time.perf_counter()
    loss0 = opt.step(objective)                 # runs the n_updates iterations; returns the first loss
    sync()
    seconds = time.perf_counter() - t0
    n_evals = evals[0]
    eval_seconds = t_eval[0]
    updates = int(opt.state[x]["n_iter"])
    final = objective()                         # the objective at the accepted corrections
    return x.detach(), {"loss_start": loss0, "loss_final": final, "evals": n_evals, "updates": updates,
                        "seconds": seconds, "eval_seconds": eval_seconds}


def lbfgs(synth, y, w=None, n_updates=40, history=10, fit_gamma6=True, stream=None):
    """Minimise L = sum_stars sum_p w (y - f)^2 over the shared per-line corrections
    Delta log gf (and Delta log gamma_6).

    synth: a Synthesizer (one or many stars) on which pz_instrument has run once;
    y, w: device FP32 [S][n_out] target and weights (w may be None: unit weights).
    Returns {"dlog_gf", "dlog_gamma6": device FP32 [n_lines], "loss_start",
    "loss_final": the objective at zero and at the final corrections, "evals":
    objective evaluations of the loop, "updates": L-BFGS iterations, "seconds": wall
    time of the loop, after one untimed evaluation that captures the step,
    "eval_seconds": the part of it spent from each evaluation's launch to its loss
    readback}.
    """
    import torch

    dev = y.device
    nl = synth.n_lines
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g_gf = torch.empty(nl, dtype=torch.float32, device=dev)
    g_g6 = torch.empty(nl, dtype=torch.float32, device=dev)
    c_gf = torch.zeros(nl, dtype=torch.float32, device=dev)
    c_g6 = torch.zeros(nl, dtype=torch.float32, device=dev)

    def set_and_eval(x):
        c_gf.copy_(x[:nl])
        if fit_gamma6:
            c_g6.copy_(x[nl:])
        synth.set_corrections(c_gf, c_g6, None, stream)
        synth.calib_step(y, w, 0.0, 0.0, 0.0, loss, g_gf, g_g6, None, stream)
        return loss[0], (torch.cat([g_gf, g_g6]) if fit_gamma6 else g_gf)

    x, res = _minimise(set_and_eval, 2 * nl if fit_gamma6 else nl, dev, n_updates, history)
    res["dlog_gf"] = x[:nl].float().clone()
    res["dlog_gamma6"] = x[nl:].float().clone() if fit_gamma6 else torch.zeros_like(res["dlog_gf"])
    return res


def lbfgs_groups(synth, y, w, group_of_line, n_groups, n_updates=40, history=10, stream=None):
    """Minimise the chi-square over the four corrections of Eq. 10 per linked group
    (Delta log gf, Delta log gamma_rad, Delta log gamma_4, Delta log gamma_6), each
    shared by the group's members (Sec. 6).  group_of_line: host int32 [n_lines] in
    [0, n_groups) or -1.  Each evaluation is one captured pz_group_eval.
    Returns the fields of lbfgs() with "x": device FP32 [4][n_groups] instead of the
    per-line corrections."""
    import torch

    from . import pz_group_eval, pz_set_line_groups
    dev = y.device
    G = int(n_groups)
    pz_set_line_groups(synth.ctx, group_of_line, G)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.empty((4, G), dtype=torch.float32, device=dev)
    x32 = torch.zeros((4, G), dtype=torch.float32, device=dev)

    def set_and_eval(x):
        x32.copy_(x.view(4, G))
        pz_group_eval(synth.ctx, y, w, x32, loss, g, stream)
        return loss[0], g.view(-1)

    x, res = _minimise(set_and_eval, 4 * G, dev, n_updates, history)
    res["x"] = x.view(4, G).float().clone()
    return res
