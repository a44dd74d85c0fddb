"""Multi-update line-list calibration (Sec. 6): L-BFGS over the shared per-line
corrections Delta log gf and Delta log gamma_6 of one or more stars.

Every function and gradient evaluation is one captured ``pz_calib_step`` with zero
learning rates: corrections applied on the device, line opacity, transfer,
instrument, chi-square over all stars and the hand-written reverse pass, replayed as
one CUDA-graph launch.  The optimiser that proposes the next corrections is PyTorch's
L-BFGS (two-loop recursion with a strong-Wolfe line search) on device tensors; it does
no synthesis arithmetic.  The paper drives its shared Sun-Arcturus fit the same way
(40 L-BFGS updates).
"""
from __future__ import annotations

import time


def lbfgs(synth, y, w=None, n_updates=40, history=10, fit_gamma6=True, stream=None):
    """Minimise L = sum_stars sum_p w (y - f)^2 over the shared corrections.

    synth: a Synthesizer (one or many stars) on which pz_instrument has run once;
    y, w: device FP32 [S][n_out] target and weights (w may be None: unit weights).
    Returns {"dlog_gf", "dlog_gamma6": device FP32 [n_lines], "loss_start",
    "loss_final": the objective at zero and at the final corrections, "evals":
    objective evaluations of the loop, "updates": L-BFGS iterations, "seconds": wall
    time of the loop, after one untimed evaluation that captures the step}.
    """
    import torch

    dev = y.device
    nl = synth.n_lines
    x = torch.zeros(2 * nl if fit_gamma6 else nl, dtype=torch.float64, device=dev, requires_grad=True)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    g_gf = torch.empty(nl, dtype=torch.float32, device=dev)
    g_g6 = torch.empty(nl, dtype=torch.float32, device=dev)
    c_gf = torch.zeros(nl, dtype=torch.float32, device=dev)
    c_g6 = torch.zeros(nl, dtype=torch.float32, device=dev)
    evals = [0]

    def objective():
        with torch.no_grad():
            c_gf.copy_(x[:nl])
            if fit_gamma6:
                c_g6.copy_(x[nl:])
        synth.set_corrections(c_gf, c_g6, None, stream)
        synth.calib_step(y, w, 0.0, 0.0, 0.0, loss, g_gf, g_g6, None, stream)
        evals[0] += 1
        grad = torch.cat([g_gf, g_g6]) if fit_gamma6 else g_gf
        x.grad = grad.to(torch.float64)
        return float(loss[0])                   # a copy: the buffer is rewritten by the next evaluation

    opt = torch.optim.LBFGS([x], lr=1.0, max_iter=n_updates, max_eval=4 * n_updates, history_size=history,
                            line_search_fn="strong_wolfe", tolerance_grad=0.0, tolerance_change=0.0)
    sync = torch.cuda.synchronize if y.is_cuda else (lambda: None)
    objective()                                 # untimed: captures the step's graph for these buffers
    evals[0] = 0
    sync()
    t0 = time.perf_counter()
    loss0 = opt.step(objective)                 # runs the n_updates iterations; returns the first loss
    sync()
    seconds = time.perf_counter() - t0
    n_evals = evals[0]
    updates = int(opt.state[x]["n_iter"])
    final = objective()                         # the objective at the accepted corrections
    with torch.no_grad():
        out_gf = x[:nl].float().clone()
        out_g6 = x[nl:].float().clone() if fit_gamma6 else torch.zeros_like(out_gf)
    return {"dlog_gf": out_gf, "dlog_gamma6": out_g6, "loss_start": loss0, "loss_final": final,
            "evals": n_evals, "updates": updates, "seconds": seconds}
