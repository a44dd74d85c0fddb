"""Multi-update line-list calibration (Sec. 6): L-BFGS over shared line corrections of
one or more stars.

A joint fit may spread its stars over ranks (one process per GPU, each rank a Synthesizer of
its own stars on the same line list): every rank evaluates its stars at the same corrections,
and one all-reduce per evaluation sums the loss and the shared gradient over the ranks, so
that every rank takes the same L-BFGS steps.  That sum is the only exchange of the path.

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

import hashlib
import time

import numpy as np


def _sum_over_ranks(process_group):
    """The exchange of a joint fit over ranks: the loss and the gradient of this rank's
    stars, packed in one FP64 vector, summed over the group by one all-reduce.  Every rank
    receives the same sums, so the line searches of all ranks take the same decisions and
    issue the same sequence of collectives."""
    import torch
    import torch.distributed as dist

    def reduce(loss, grad):
        buf = torch.cat([torch.as_tensor(loss, dtype=torch.float64, device=grad.device).reshape(1),
                         grad.to(torch.float64)])
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=process_group)
        return buf[0], buf[1:]
    return reduce


def _minimise(set_and_eval, n_params, dev, n_updates, history, resume=None, process_group=None):
    """L-BFGS on a float64 device vector of n_params; set_and_eval(x) -> (loss, grad).
    resume: {"x", "optimizer"} of an earlier run (see save_state) to continue from.
    process_group: sum each evaluation over the ranks of this torch.distributed group
    (None: this process alone); the starting point is taken from the group's first rank."""
    import torch

    x = torch.zeros(n_params, dtype=torch.float64, device=dev, requires_grad=True)
    if resume is not None:
        with torch.no_grad():
            x.copy_(torch.as_tensor(resume["x"], dtype=torch.float64, device=dev))
    reduce = None
    if process_group is not None:
        import torch.distributed as dist
        reduce = _sum_over_ranks(process_group)
        with torch.no_grad():
            dist.broadcast(x.detach(), src=dist.get_global_rank(process_group, 0), group=process_group)
    evals = [0]
    t_eval = [0.0]

    def objective():
        t = time.perf_counter()
        loss, grad = set_and_eval(x.detach())
        if reduce is not None:
            loss, grad = reduce(loss, grad)
        evals[0] += 1
        x.grad = grad.to(torch.float64)
        out = float(loss)                       # a copy: the buffer is rewritten by the next evaluation
        t_eval[0] += time.perf_counter() - t
        return out

    opt = torch.optim.LBFGS([x], lr=1.0, max_iter=n_updates, max_eval=4 * n_updates, history_size=history,
                            line_search_fn="strong_wolfe", tolerance_grad=0.0, tolerance_change=0.0)
    if resume is not None and resume.get("optimizer") is not None:
        opt.load_state_dict(resume["optimizer"])
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
                        "seconds": seconds, "eval_seconds": eval_seconds, "x": x.detach().clone(),
                        "optimizer": opt.state_dict()}


def lbfgs(synth, y, w=None, n_updates=40, history=10, fit_gamma6=True, stream=None, resume=None,
          process_group=None):
    """Minimise L = sum_stars sum_p w (y - f)^2 over the shared per-line corrections
    Delta log gf (and Delta log gamma_6).

    synth: a Synthesizer (one or many stars) on which pz_instrument has run once;
    y, w: device FP32 [S][n_out] target and weights (w may be None: unit weights).
    Returns {"dlog_gf", "dlog_gamma6": device FP32 [n_lines], "loss_start",
    "loss_final": the objective at zero and at the final corrections, "evals":
    objective evaluations of the loop, "updates": L-BFGS iterations, "seconds": wall
    time of the loop, after one untimed evaluation that captures the step,
    "eval_seconds": the part of it spent from each evaluation's launch to its loss
    readback, "x" and "optimizer": the final parameter vector and the L-BFGS state, which
    save_state stores and resume= takes back to continue the fit}.
    process_group: a torch.distributed group over whose ranks the stars of a joint fit
    are spread (each rank's synth holds its own stars and the same line list); the loss
    and the gradients then cover the stars of every rank, "loss_start" and "loss_final"
    included, and every rank returns the same corrections.  None: synth's stars alone.
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

    x, res = _minimise(set_and_eval, 2 * nl if fit_gamma6 else nl, dev, n_updates, history, resume, process_group)
    res["dlog_gf"] = x[:nl].float().clone()
    res["dlog_gamma6"] = x[nl:].float().clone() if fit_gamma6 else torch.zeros_like(res["dlog_gf"])
    return res


def lbfgs_groups(synth, y, w, group_of_line, n_groups, n_updates=40, history=10, stream=None, resume=None,
                 process_group=None):
    """Minimise the chi-square over the four corrections of Eq. 10 per linked group
    (Delta log gf, Delta log gamma_rad, Delta log gamma_4, Delta log gamma_6), each
    shared by the group's members (Sec. 6).  group_of_line: host int32 [n_lines] in
    [0, n_groups) or -1.  Each evaluation is one captured pz_group_eval.
    Returns the fields of lbfgs() with "x": device FP32 [4][n_groups] instead of the
    per-line corrections.  process_group: as for lbfgs (the groups must be the same on
    every rank)."""
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

    x, res = _minimise(set_and_eval, 4 * G, dev, n_updates, history, resume, process_group)
    res["groups"] = x.view(4, G).float().clone()
    return res


# ---------------------------------------------------------------------------
# saving and restoring a calibration (corrections bound to their line list)
# ---------------------------------------------------------------------------

def catalog_digest(lines) -> str:
    """SHA-256 of the line list a set of corrections applies to (centres, log gf,
    E_low, the three damping constants and species, in caller order): corrections are
    an overlay on one catalog and must not be applied to another."""
    h = hashlib.sha256()
    for a, dt in ((lines.lambda_nm, np.float64), (lines.log_gf, np.float32), (lines.E_low_eV, np.float32),
                  (lines.log_gamma_rad, np.float32), (lines.log_gamma4, np.float32),
                  (lines.log_gamma6, np.float32), (lines.species, np.int32)):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    h.update(str(int(lines.half_window)).encode())
    return h.hexdigest()


def save_state(path, synth, result=None, meta=None):
    """Write the context's current corrections (Delta log gf, Delta log gamma_6, the
    radiative and Stark corrections and the abundance offsets), the digest of its line
    list and, if given, the optimiser state of an lbfgs / lbfgs_groups result
    ("x", "optimizer") to path (torch.save format)."""
    import torch
    gf, g6, ab = synth.get_corrections()
    rad, g4 = synth.get_damping_corrections()
    state = {"digest": catalog_digest(synth.prob.lines), "n_lines": int(synth.n_lines),
             "dlog_gf": gf, "dlog_gamma6": g6, "dlog_gamma_rad": rad, "dlog_gamma4": g4, "dabund": ab,
             "meta": dict(meta or {})}
    if result is not None:
        state["x"] = result["x"].detach().cpu()
        state["optimizer"] = _to_cpu(result["optimizer"])
    torch.save(state, path)


def load_state(path, synth, device=None):
    """Read a file written by save_state, check that it belongs to this context's line
    list (ValueError otherwise), apply its corrections to the context and return the
    state; its "x" / "optimizer" (if present) continue a fit through resume=."""
    import torch
    state = torch.load(path, map_location="cpu", weights_only=False)
    if state.get("digest") != catalog_digest(synth.prob.lines) or state.get("n_lines") != synth.n_lines:
        raise ValueError("load_state: %s holds corrections for another line list" % path)
    synth.set_corrections(state["dlog_gf"], state["dlog_gamma6"], state["dabund"])
    synth.set_damping_corrections(state["dlog_gamma_rad"], state["dlog_gamma4"])
    if "optimizer" in state and device is not None:
        state["optimizer"] = _to_device(state["optimizer"], device)
    return state


def _to_cpu(obj):
    import torch
    if isinstance(obj, torch.Tensor):
        return obj.detach().cpu()
    if isinstance(obj, dict):
        return {k: _to_cpu(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return type(obj)(_to_cpu(v) for v in obj)
    return obj


def _to_device(obj, device):
    import torch
    if isinstance(obj, torch.Tensor):
        return obj.to(device)
    if isinstance(obj, dict):
        return {k: _to_device(v, device) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return type(obj)(_to_device(v, device) for v in obj)
    return obj
