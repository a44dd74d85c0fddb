#!/usr/bin/env python
"""Writes tests/golden/config4_oracle.npz: FP64 oracle results for stars of the
batched many-star workload (64 stars on the APOGEE-like grid and instrument, star k
keeping its strongest N_k lines of a 3e5-line master list; stars are independent,
Sec. 9).

* The two stars with the fewest lines, in full: the target y (the oracle's
  normalised flux at seeded true corrections Delta log gf ~ N(0, 0.1), Delta log
  gamma6 ~ N(0, 0.2) on the master list, plus S/N-200 noise, rounded to FP32), the
  normalised flux f at zero corrections on all 8,575 pixels, chi^2 with w = 200^2,
  and the gradients for every line of the star (caller order of its subset) and
  the 20 abundances (Sec. 6, Eq. 10).
* The star with the most lines and star 17: f at zero corrections on 12 seeded
  pixels, each from the oracle's line sum on that pixel's instrument taps.

Only oracle/ computes anything here; the inputs come from the seeded generators.
Run once (about half an hour on 8 cores):  python tests/golden/make_config4_golden.py
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

N_SAMPLED_PIXELS = 12


def log(msg):
    print("[%s] %s" % (time.strftime("%H:%M:%S"), msg), flush=True)


def truth_and_noise(b):
    """Seeded true corrections on the master list and per-star pixel noise."""
    rng = np.random.default_rng(7)
    nl = b.lines.n_lines
    n_out = b.instrument.pix_lambda_nm.size
    return (rng.normal(0.0, 0.1, nl).astype(np.float32), rng.normal(0.0, 0.2, nl).astype(np.float32),
            rng.normal(0.0, 1.0 / 200.0, (b.n_stars, n_out)))


def full_star(b, k, tg, t6, noise):
    p = b.star(k)
    idx = b.subsets[k]
    nl = p.lines.n_lines
    n_out = b.instrument.pix_lambda_nm.size
    log("star %d in full: %d lines, %.3g evaluations per pass" % (k, nl, p.n_evals))
    f_true = oracle.forward(p, {"dlog_gf": tg[idx].astype(np.float64),
                                "dlog_gamma6": t6[idx].astype(np.float64)})["f"]
    y = (f_true + noise[k]).astype(np.float32)
    zero = {"dlog_gf": np.zeros(nl), "dlog_gamma6": np.zeros(nl), "dabund": np.zeros(p.n_elem)}
    fwd = oracle.forward(p, zero)
    L, g_gf, g_g6, g_ab, fwd = oracle.gradient(p, y.astype(np.float64), np.full(n_out, 200.0 ** 2), zero,
                                               fwd=fwd)
    return {"y": y, "f": fwd["f"], "loss": np.float64(L), "g_gf": g_gf.astype(np.float32),
            "g_g6": g_g6.astype(np.float32), "g_ab": g_ab, "n_lines": np.int64(nl)}


def sampled_pixels(b, k, pixels, taps):
    p = b.star(k)
    tap0, ntap, wt = taps
    log("star %d sampled: %d lines, %d pixels" % (k, p.lines.n_lines, len(pixels)))
    out = np.empty(len(pixels))
    for j, q in enumerate(pixels):
        cols = tap0[q] + np.arange(ntap[q])
        kl = oracle.kappa_line(p, cols)
        F, Fc = oracle.flux(p, cols, kl)
        wq = wt[q, :ntap[q]]
        out[j] = np.dot(wq, F) / np.dot(wq, Fc)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "config4_oracle.npz"))
    args = ap.parse_args()
    oracle.build()
    t0 = time.time()
    b = I.config4()
    sizes = np.array([len(s) for s in b.subsets])
    full = [int(k) for k in np.argsort(sizes, kind="stable")[:2]]
    sampled = sorted({int(np.argmax(sizes)), 17} - set(full))
    tg, t6, noise = truth_and_noise(b)
    res = {"full_stars": np.array(full, np.int64), "sampled_stars": np.array(sampled, np.int64),
           "n_lines_per_star": sizes.astype(np.int64)}
    for k in full:
        for key, v in full_star(b, k, tg, t6, noise).items():
            res["star%d_%s" % (k, key)] = v
    taps = oracle.instrument_taps(b.star(sampled[0]), b.instrument)
    rng = np.random.default_rng(11)
    n_out = b.instrument.pix_lambda_nm.size
    pixels = np.sort(np.concatenate([[0, n_out - 1], rng.choice(np.arange(1, n_out - 1), N_SAMPLED_PIXELS - 2,
                                                               replace=False)])).astype(np.int64)
    res["sampled_pixels"] = pixels
    for k in sampled:
        res["star%d_f_sampled" % k] = sampled_pixels(b, k, pixels, taps)
    np.savez_compressed(args.out, **res)
    log("wrote %s in %.0f s" % (args.out, time.time() - t0))


if __name__ == "__main__":
    main()
