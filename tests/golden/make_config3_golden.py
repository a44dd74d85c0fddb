#!/usr/bin/env python
"""Writes tests/golden/config3_oracle.npz: the FP64 oracle's forward and adjoint of
the differentiable-calibration workload at full size, and central differences of
the oracle's loss for 200 seeded random lines.

Workload: the APOGEE-like grid (1500-1700 nm at R_grid = 3e5, 37,550 points),
1.2e5 lines, 72 layers, Doppler shift 12.3 km/s, Gaussian LSF R = 22,500 onto
8,575 pixels.  The target is the oracle's normalised flux at the seeded true
corrections (Delta log gf ~ N(0, 0.1), Delta log gamma6 ~ N(0, 0.2)) plus the
seeded S/N-200 noise, rounded to FP32 (the form a device objective reads).  The
loss is chi^2 with w = 200^2 (Sec. 6); gradients are taken at zero corrections
with respect to every line's Delta log gf and Delta log gamma6 (Eq. 10) and the
20 abundances.

The central differences (h = 1e-4) re-evaluate only what a line's correction
changes: that line's own term of the window sum (Eqs. 4-5), by the oracle on a
one-line problem over the window, added to the full forward's kappa_line; the
flux at those columns (Eqs. 7-8); the instrument and the loss.  They check the
oracle's hand-written adjoint at full size.

Only oracle/ computes anything here; the inputs come from the seeded generators.
Run once (about an hour on 8 cores):  python tests/golden/make_config3_golden.py
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2607_24141_gb300 import inputs as I  # noqa: E402

H_FD = 1e-4
N_FD_LINES = 200


def log(msg):
    print("[%s] %s" % (time.strftime("%H:%M:%S"), msg), flush=True)


def loss_difference(y, w, f_plus, f_minus):
    """L(f+) - L(f-) for L = sum w (y - f)^2, in the cancellation-free form
    sum w (f- - f+) (2y - f+ - f-)."""
    return float(np.sum(w * (f_minus - f_plus) * (2.0 * y - f_plus - f_minus)))


def central_differences(prob, fwd, y, w, lines, h=H_FD):
    """(d L / d Delta log gf, d L / d Delta log gamma6) of the oracle's loss by central
    differences for each line in ``lines`` (caller indices)."""
    W = prob.lines.half_window
    n = prob.grid.n_lambda
    il = I.center_index(prob.grid, prob.lines.lambda_nm)
    tap0, ntap, wt = fwd["taps"]
    gc = fwd["gc"]
    out = np.zeros((2, len(lines)))
    for k, l in enumerate(lines):
        lo, hi = max(0, int(il[l]) - W - 2), min(n - 1, int(il[l]) + W + 2)
        if hi < lo:
            continue
        cols = np.arange(lo, hi + 1)
        one = I.Problem(prob.name + "-line", prob.atmos, prob.grid, prob.lines.subset(np.array([l])),
                        prob.kappa_c, None, prob.elem_of_species, prob.n_elem)
        base_k = fwd["kline"][:, cols]
        k0 = oracle.kappa_line(one, cols)
        for j, key in enumerate(("dlog_gf", "dlog_gamma6")):
            f_pm = []
            for s in (+h, -h):
                ks = oracle.kappa_line(one, cols, corrections={key: np.array([s])})
                F_cols, _ = oracle.flux(prob, cols, base_k + (ks - k0))
                F = fwd["F"].copy()
                F[cols] = F_cols
                f_pm.append(oracle.apply_taps(tap0, ntap, wt, F) / gc)
            out[j, k] = loss_difference(y, w, f_pm[0], f_pm[1]) / (2.0 * h)
    return out


def make(prob, truth, seed_lines=200):
    nl = prob.lines.n_lines
    n_out = prob.instrument.pix_lambda_nm.size
    t0 = time.time()
    log("forward at the true corrections (%d lines, %d points, %.3g evaluations)"
        % (nl, prob.grid.n_lambda, prob.n_evals))
    true_corr = {"dlog_gf": truth["dlog_gf"].astype(np.float64),
                 "dlog_gamma6": truth["dlog_gamma6"].astype(np.float64)}
    f_true = oracle.forward(prob, true_corr)["f"]
    y = (f_true + truth["noise"]).astype(np.float32)
    w = np.full(n_out, float(truth["weight"]))
    log("forward at zero corrections")
    zero = {"dlog_gf": np.zeros(nl), "dlog_gamma6": np.zeros(nl), "dabund": np.zeros(prob.n_elem)}
    fwd = oracle.forward(prob, zero)
    log("adjoint")
    L, g_gf, g_g6, g_ab, fwd = oracle.gradient(prob, y.astype(np.float64), w, zero, fwd=fwd)
    rng = np.random.default_rng(seed_lines)
    lines = np.sort(rng.choice(nl, size=min(N_FD_LINES, nl), replace=False))
    log("central differences on %d lines" % lines.size)
    fd = central_differences(prob, fwd, y.astype(np.float64), w, lines)
    log("done in %.0f s" % (time.time() - t0))
    return {"y": y, "f": fwd["f"], "loss": np.float64(L), "g_gf": g_gf.astype(np.float32),
            "g_g6": g_g6.astype(np.float32), "g_ab": g_ab, "g_gf_max": np.max(np.abs(g_gf)),
            "g_g6_max": np.max(np.abs(g_g6)), "fd_lines": lines.astype(np.int64),
            "fd_g_gf": fd[0], "fd_g_g6": fd[1], "adj_g_gf": g_gf[lines], "adj_g_g6": g_g6[lines],
            "fd_h": np.float64(H_FD), "n_evals": np.int64(prob.n_evals)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "config3_oracle.npz"))
    ap.add_argument("--span-nm", type=float, default=None,
                    help="a slice of the recipe instead of the full 1500-1700 nm (for a quick dry run)")
    args = ap.parse_args()
    oracle.build()
    if args.span_nm:
        prob, truth = I.config3(lam_lo=1600.0, lam_hi=1600.0 + args.span_nm, n_atomic=int(80_000 * args.span_nm / 200),
                                n_bands=int(80 * args.span_nm / 200) if args.span_nm > 12 else 0)
    else:
        prob, truth = I.config3()
    res = make(prob, truth)
    np.savez_compressed(args.out, **res)
    log("wrote %s" % args.out)


if __name__ == "__main__":
    main()
