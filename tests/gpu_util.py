"""Helpers for the GPU tests: run the C-ABI path on a Problem, compare with the oracle."""
import numpy as np

import paper_2607_24141_gb300 as pz


def run_forward(prob, precision=pz.PZ_MIXED, corrections=None, tiling=None, want_kline=True):
    import torch
    s = pz.Synthesizer(prob, precision)
    if tiling:
        pz.pz_set_tiling(s.ctx, *tiling)
    if corrections:
        s.set_corrections(corrections.get("dlog_gf"), corrections.get("dlog_gamma6"), corrections.get("dabund"))
    nd, nl = prob.atmos.n_depth, prob.grid.n_lambda
    dev = s.device
    kl = torch.empty((nd, nl), dtype=torch.float32, device=dev) if want_kline else None
    F = torch.empty(nl, dtype=torch.float64, device=dev)
    Fc = torch.empty(nl, dtype=torch.float64, device=dev)
    f = s.forward(kl, F, Fc)
    torch.cuda.synchronize()
    out = {"F": F.cpu().numpy(), "Fc": Fc.cpu().numpy(), "f": f.cpu().numpy().astype(np.float64), "synth": s}
    if want_kline:
        out["kline"] = kl.cpu().numpy().astype(np.float64)
    return out


def run_gradient(prob, y, w, precision=pz.PZ_MIXED, corrections=None, tiling=None):
    import torch
    r = run_forward(prob, precision, corrections, tiling, want_kline=False)
    s = r["synth"]
    dev = s.device
    yt = torch.tensor(y, dtype=torch.float32, device=dev)
    wt = torch.tensor(np.broadcast_to(w, y.shape), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    dLdf = torch.empty(y.size, dtype=torch.float32, device=dev)
    s.loss(yt, wt, loss, dLdf)
    nl = prob.lines.n_lines
    g_gf = torch.empty(nl, dtype=torch.float32, device=dev)
    g_g6 = torch.empty(nl, dtype=torch.float32, device=dev)
    g_ab = torch.empty(max(prob.n_elem, 1), dtype=torch.float32, device=dev)
    s.backward(dLdf, g_gf, g_g6, g_ab if corrections and corrections.get("dabund") is not None else None)
    torch.cuda.synchronize()
    r.update(loss=float(loss.item()), dLdf=dLdf.cpu().numpy(), g_gf=g_gf.cpu().numpy().astype(np.float64),
             g_g6=g_g6.cpu().numpy().astype(np.float64), g_ab=g_ab.cpu().numpy().astype(np.float64))
    return r


def rel_metric(g, ref):
    """|g - ref| / max(|ref|, 1e-3 max|ref|) elementwise (gradient error metric)."""
    floor = 1e-3 * np.max(np.abs(ref)) if ref.size else 0.0
    return np.abs(g - ref) / np.maximum(np.abs(ref), floor)


def kappa_rel(got, ref, kc):
    """Relative kappa error where kappa_line > 1e-6 kappa_c."""
    m = ref > 1e-6 * kc
    if not np.any(m):
        return 0.0
    return float(np.max(np.abs(got[m] / ref[m] - 1)))
