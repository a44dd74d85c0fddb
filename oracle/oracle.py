"""ctypes wrapper of the FP64 CPU oracle (``pz_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The wrapper only marshals numpy arrays; every arithmetic step of the oracle is
in the C file, except plain numpy steps that are themselves definitions:
applying the instrument's banded weights (a weighted sum over taps), the
species-to-element sum of per-line gradients, the linked correction groups of
Sec. 6 (a group's correction copied to its members, member gradients summed per
group) and the greedy grouping pass that forms them (a plain loop over seeds).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pz_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


class _Problem(C.Structure):
    _fields_ = [
        ("n_depth", C.c_int32), ("n_species", C.c_int32),
        ("m", _dp), ("T", _dp), ("rho", _dp), ("n_e", _dp), ("n_pert", _dp), ("pop", _dp),
        ("mass_amu", _dp), ("xi_cms", C.c_double), ("kappa_c", _dp),
        ("lambda0_nm", C.c_double), ("R_grid", C.c_double), ("n_lambda", C.c_int64),
        ("n_lines", C.c_int64), ("lambda_nm", _dp),
        ("log_gf", _fp), ("E_low_eV", _fp), ("log_gamma_rad", _fp), ("log_gamma4", _fp),
        ("log_gamma6", _fp), ("species", _ip), ("half_window", C.c_int32),
        ("dlog_gf", _dp), ("dlog_gamma6", _dp), ("dabund", _dp), ("elem_of_species", _ip),
        ("centre_eta", C.c_double),
        ("dlog_gamma_rad", _dp), ("dlog_gamma4", _dp),
        ("sigma_c", _dp),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over columns)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.pzo_voigt_vec.argtypes = [C.c_int64, _dp, _dp, _dp, _dp, _dp]
        L.pzo_expn_vec.argtypes = [C.c_int, C.c_int64, _dp, _dp]
        L.pzo_expn.argtypes = [C.c_int, C.c_double]
        L.pzo_expn.restype = C.c_double
        L.pzo_kappa_line.argtypes = [C.POINTER(_Problem), C.c_int64, _lp, _dp]
        L.pzo_flux.argtypes = [C.POINTER(_Problem), C.c_int64, _lp, _dp, _dp, _dp]
        L.pzo_instrument_taps.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, C.c_double,
                                          C.c_int64, _dp, _lp, _ip, _dp, C.c_int32]
        L.pzo_instrument_taps.restype = C.c_int
        L.pzo_rt_adjoint.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp]
        L.pzo_line_grad.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp, _dp, _dp]
        L.pzo_chi2.argtypes = [C.c_int64, _dp, _dp, _dp, _dp]
        L.pzo_chi2.restype = C.c_double
        L.pzo_flux_tau.argtypes = [C.c_int, _dp, _dp]
        L.pzo_flux_tau.restype = C.c_double
        L.pzo_flux_dtau.argtypes = [C.c_int, _dp, _dp, _dp]
        L.pzo_lambda_matrix.argtypes = [C.c_int, _dp, _dp]
        L.pzo_scatter_source.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
        L.pzo_scatter_adjoint.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, _dp, _dp]
        L.pzo_scatter_flux.argtypes = [C.c_int, _dp, _dp, _dp]
        L.pzo_scatter_flux.restype = C.c_double
        L.pzo_lambda_dtau.argtypes = [C.c_int, _dp, _dp, _dp]
        L.pzo_planck_nm.argtypes = [C.c_double, C.c_double]
        L.pzo_planck_nm.restype = C.c_double
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t):
    return a.ctypes.data_as(t)


class _Keep:
    """Holds the numpy arrays a _Problem points into."""

    def __init__(self, prob, corrections=None):
        at, ll = prob.atmos, prob.lines
        self.arrs = {
            "m": _d(at.m), "T": _d(at.T), "rho": _d(at.rho), "n_e": _d(at.n_e),
            "n_pert": _d(at.n_pert), "pop": _d(at.pop), "mass": _d(at.mass_amu),
            "kc": _d(prob.kappa_c), "lam": _d(ll.lambda_nm),
            "gf": np.ascontiguousarray(ll.log_gf, np.float32),
            "E": np.ascontiguousarray(ll.E_low_eV, np.float32),
            "grad": np.ascontiguousarray(ll.log_gamma_rad, np.float32),
            "g4": np.ascontiguousarray(ll.log_gamma4, np.float32),
            "g6": np.ascontiguousarray(ll.log_gamma6, np.float32),
            "sp": np.ascontiguousarray(ll.species, np.int32),
        }
        P = _Problem()
        P.n_depth = at.n_depth
        P.n_species = at.n_species
        A = self.arrs
        P.m, P.T, P.rho = _ptr(A["m"], _dp), _ptr(A["T"], _dp), _ptr(A["rho"], _dp)
        P.n_e, P.n_pert, P.pop = _ptr(A["n_e"], _dp), _ptr(A["n_pert"], _dp), _ptr(A["pop"], _dp)
        P.mass_amu = _ptr(A["mass"], _dp)
        P.xi_cms = at.xi_cms
        P.kappa_c = _ptr(A["kc"], _dp)
        P.lambda0_nm = prob.grid.lambda0_nm
        P.R_grid = prob.grid.R_grid
        P.n_lambda = prob.grid.n_lambda
        P.n_lines = ll.n_lines
        P.lambda_nm = _ptr(A["lam"], _dp)
        P.log_gf, P.E_low_eV = _ptr(A["gf"], _fp), _ptr(A["E"], _fp)
        P.log_gamma_rad, P.log_gamma4, P.log_gamma6 = _ptr(A["grad"], _fp), _ptr(A["g4"], _fp), _ptr(A["g6"], _fp)
        P.species = _ptr(A["sp"], _ip)
        P.half_window = ll.half_window
        if getattr(prob, "sigma_c", None) is not None:
            A["sig"] = _d(prob.sigma_c)
            P.sigma_c = _ptr(A["sig"], _dp)
        if corrections:
            if corrections.get("dlog_gf") is not None:
                A["dgf"] = _d(corrections["dlog_gf"])
                P.dlog_gf = _ptr(A["dgf"], _dp)
            if corrections.get("dlog_gamma6") is not None:
                A["dg6"] = _d(corrections["dlog_gamma6"])
                P.dlog_gamma6 = _ptr(A["dg6"], _dp)
            for key, field in (("dlog_gamma_rad", "dlog_gamma_rad"), ("dlog_gamma4", "dlog_gamma4")):
                if corrections.get(key) is not None:
                    A[key] = _d(corrections[key])
                    setattr(P, field, _ptr(A[key], _dp))
            if corrections.get("dabund") is not None:
                A["dab"] = _d(corrections["dabund"])
                A["eos"] = np.ascontiguousarray(prob.elem_of_species, np.int32)
                P.dabund = _ptr(A["dab"], _dp)
                P.elem_of_species = _ptr(A["eos"], _ip)
            # continuum-referenced centre test (0 = off)
            P.centre_eta = float(corrections.get("centre_eta") or 0.0)
        self.P = P


# ---------------------------------------------------------------------------
# elementary functions
# ---------------------------------------------------------------------------

def voigt(a, v):
    """H(a,v), L(a,v) = Im w, dH/da, elementwise."""
    a, v = np.broadcast_arrays(np.asarray(a, np.float64), np.asarray(v, np.float64))
    a, v = _d(a.ravel()), _d(v.ravel())
    H, L, dH = np.empty_like(a), np.empty_like(a), np.empty_like(a)
    lib().pzo_voigt_vec(a.size, _ptr(a, _dp), _ptr(v, _dp), _ptr(H, _dp), _ptr(L, _dp), _ptr(dH, _dp))
    return H, L, dH


def expn(n, x):
    x = _d(np.atleast_1d(x))
    out = np.empty_like(x)
    lib().pzo_expn_vec(int(n), x.size, _ptr(x, _dp), _ptr(out, _dp))
    return out


def flux_tau(tau, S):
    tau, S = _d(tau), _d(S)
    return lib().pzo_flux_tau(tau.size, _ptr(tau, _dp), _ptr(S, _dp))


def flux_dtau(tau, S):
    tau, S = _d(tau), _d(S)
    out = np.empty_like(tau)
    lib().pzo_flux_dtau(tau.size, _ptr(tau, _dp), _ptr(S, _dp), _ptr(out, _dp))
    return out


def lambda_matrix(tau):
    """Lambda [nd][nd] of the piecewise-linear source on the layers tau: J = Lambda S."""
    tau = _d(tau)
    out = np.empty((tau.size, tau.size))
    lib().pzo_lambda_matrix(tau.size, _ptr(tau, _dp), _ptr(out, _dp))
    return out


def scatter_source(tau, eps, B):
    """S solving S = eps B + (1 - eps) Lambda S on the layers tau."""
    tau, eps, B = _d(tau), _d(eps), _d(B)
    out = np.empty_like(tau)
    lib().pzo_scatter_source(tau.size, _ptr(tau, _dp), _ptr(eps, _dp), _ptr(B, _dp), _ptr(out, _dp))
    return out


def scatter_flux(tau, eps, B):
    """Emergent flux of the solved scattering source on explicit layers."""
    tau, eps, B = _d(tau), _d(eps), _d(B)
    return lib().pzo_scatter_flux(tau.size, _ptr(tau, _dp), _ptr(eps, _dp), _ptr(B, _dp))


def scatter_adjoint(tau, eps, B, Fbar=1.0):
    """(dL/dtau, dL/deps) of the scattering flux for dL/dF = Fbar."""
    tau, eps, B = _d(tau), _d(eps), _d(B)
    gt, ge = np.empty_like(tau), np.empty_like(tau)
    lib().pzo_scatter_adjoint(tau.size, _ptr(tau, _dp), _ptr(eps, _dp), _ptr(B, _dp), float(Fbar), _ptr(gt, _dp),
                              _ptr(ge, _dp))
    return gt, ge


def lambda_dtau(tau, S):
    """dJ_j/dtau_m at fixed layer values S."""
    tau, S = _d(tau), _d(S)
    out = np.empty((tau.size, tau.size))
    lib().pzo_lambda_dtau(tau.size, _ptr(tau, _dp), _ptr(S, _dp), _ptr(out, _dp))
    return out


def planck_nm(lambda_nm, T):
    return lib().pzo_planck_nm(float(lambda_nm), float(T))


# ---------------------------------------------------------------------------
# synthesis stages
# ---------------------------------------------------------------------------

def kappa_line(prob, cols=None, corrections=None):
    """kappa_line[d, c] for grid columns ``cols`` (default: all)."""
    if cols is None:
        cols = np.arange(prob.grid.n_lambda)
    cols = np.ascontiguousarray(cols, np.int64)
    k = _Keep(prob, corrections)
    out = np.empty((prob.atmos.n_depth, cols.size))
    lib().pzo_kappa_line(C.byref(k.P), cols.size, _ptr(cols, _lp), _ptr(out, _dp))
    return out


def flux(prob, cols, kline):
    cols = np.ascontiguousarray(cols, np.int64)
    kline = _d(kline)
    k = _Keep(prob)
    F, Fc = np.empty(cols.size), np.empty(cols.size)
    lib().pzo_flux(C.byref(k.P), cols.size, _ptr(cols, _lp), _ptr(kline, _dp), _ptr(F, _dp), _ptr(Fc, _dp))
    return F, Fc


def instrument_taps(prob, inst, max_taps=4096):
    pix = _d(inst.pix_lambda_nm)
    n = pix.size
    tap0 = np.empty(n, np.int64)
    ntap = np.empty(n, np.int32)
    w = np.zeros((n, max_taps))
    k = _Keep(prob)
    rc = lib().pzo_instrument_taps(C.byref(k.P), inst.v_r_kms, inst.v_b_kms, inst.R_lsf, n,
                                   _ptr(pix, _dp), _ptr(tap0, _lp), _ptr(ntap, _ip), _ptr(w, _dp), max_taps)
    if rc != 0:
        raise ValueError("oracle instrument_taps failed: %d" % rc)
    width = int(ntap.max())
    return tap0, ntap, np.ascontiguousarray(w[:, :width])


def apply_taps(tap0, ntap, w, F):
    """(K F)_p = sum_k w_pk F[tap0_p + k]."""
    out = np.zeros(tap0.size)
    for k in range(w.shape[1]):
        m = k < ntap
        out[m] += w[m, k] * F[tap0[m] + k]
    return out


def apply_taps_T(tap0, ntap, w, g, n_lambda):
    """(K^T g)_i."""
    out = np.zeros(n_lambda)
    for k in range(w.shape[1]):
        m = k < ntap
        np.add.at(out, tap0[m] + k, w[m, k] * g[m])
    return out


def forward(prob, corrections=None):
    """Full forward on every column: kappa_line, F, F_c, f (instrument applied if present)."""
    cols = np.arange(prob.grid.n_lambda)
    kl = kappa_line(prob, cols, corrections)
    F, Fc = flux(prob, cols, kl)
    out = {"kline": kl, "F": F, "Fc": Fc}
    if prob.instrument is not None:
        taps = instrument_taps(prob, prob.instrument)
        g, gc = apply_taps(*taps, F), apply_taps(*taps, Fc)
        out.update(g=g, gc=gc, f=g / gc, taps=taps)
    else:
        out["f"] = F / Fc
    return out


def chi2(y, w, f):
    y, w, f = _d(y), _d(np.broadcast_to(w, np.shape(y))), _d(f)
    dL = np.empty_like(f)
    L = lib().pzo_chi2(f.size, _ptr(y, _dp), _ptr(w, _dp), _ptr(f, _dp), _ptr(dL, _dp))
    return L, dL


def gradient(prob, y, w, corrections=None, fwd=None):
    """Loss and hand-written adjoint: returns (L, g_gf, g_g6, g_abund, fwd)."""
    if fwd is None:
        fwd = forward(prob, corrections)
    L, dLdf = chi2(y, w, fwd["f"])
    if prob.instrument is not None:
        tap0, ntap, wt = fwd["taps"]
        dLdF = apply_taps_T(tap0, ntap, wt, dLdf / fwd["gc"], prob.grid.n_lambda)
    else:
        dLdF = dLdf / fwd["Fc"]
    k = _Keep(prob, corrections)
    kl = _d(fwd["kline"])
    G = np.empty_like(kl)
    lib().pzo_rt_adjoint(C.byref(k.P), _ptr(kl, _dp), _ptr(_d(dLdF), _dp), _ptr(G, _dp))
    ggf = np.empty(prob.lines.n_lines)
    gg6 = np.empty(prob.lines.n_lines)
    grad = np.empty(prob.lines.n_lines)
    gg4 = np.empty(prob.lines.n_lines)
    lib().pzo_line_grad(C.byref(k.P), _ptr(G, _dp), _ptr(ggf, _dp), _ptr(gg6, _dp), _ptr(grad, _dp), _ptr(gg4, _dp))
    gab = None
    if prob.elem_of_species is not None:
        gab = np.zeros(prob.n_elem)
        np.add.at(gab, prob.elem_of_species[prob.lines.species], ggf)
    fwd["g_gamma_rad"], fwd["g_gamma4"] = grad, gg4
    return L, ggf, gg6, gab, fwd


def gradient4(prob, y, w, corrections=None, fwd=None):
    """The four per-line gradients of Eq. 10 (gf and the three damping families):
    {"L", "gf", "gamma_rad", "gamma4", "gamma6", "abund", "fwd"}."""
    L, ggf, gg6, gab, fwd = gradient(prob, y, w, corrections, fwd)
    return {"L": L, "gf": ggf, "gamma_rad": fwd["g_gamma_rad"], "gamma4": fwd["g_gamma4"], "gamma6": gg6,
            "abund": gab, "fwd": fwd}


# ---------------------------------------------------------------------------
# linked correction groups (Sec. 6, Eq. 10 with q(l))
# ---------------------------------------------------------------------------

def expand_groups(x_group, group_of_line):
    """Per-line corrections delta_{q(l)}: x_group [..., n_groups] -> [..., n_lines];
    lines with q(l) = -1 take no correction."""
    x_group = np.asarray(x_group, np.float64)
    q = np.asarray(group_of_line, np.int64)
    out = np.zeros(x_group.shape[:-1] + (q.size,))
    m = q >= 0
    out[..., m] = x_group[..., q[m]]
    return out


def group_sum(g_line, group_of_line, n_groups):
    """dL/ddelta_q = sum over the members l of q of dL/ddelta_l (chain rule through the copy)."""
    g_line = np.asarray(g_line, np.float64)
    q = np.asarray(group_of_line, np.int64)
    out = np.zeros(g_line.shape[:-1] + (int(n_groups),))
    m = q >= 0
    for k in np.nonzero(m)[0]:
        out[..., q[k]] += g_line[..., k]
    return out


def build_line_groups(lambda_nm, E_low_eV, species, strength, dE_eV, dlam_nm):
    """Greedy strength-ordered grouping (Sec. 6): take the lines from the strongest down
    (equal strengths by index); a line not yet grouped opens a new group and takes every
    line not yet grouped of the same species (ion stage included) whose lower-level energy
    is within dE_eV of its own and whose wavelength is within dlam_nm of its own.  Groups
    are numbered in the order they open.  Returns (group_of_line int32, n_groups)."""
    lam = np.asarray(lambda_nm, np.float64)
    E = np.asarray(E_low_eV, np.float32).astype(np.float64)
    sp = np.asarray(species, np.int64)
    st = np.asarray(strength, np.float32)
    n = lam.size
    order = sorted(range(n), key=lambda k: (-float(st[k]), k))
    q = np.full(n, -1, np.int32)
    G = 0
    for s in order:
        if q[s] >= 0:
            continue
        q[s] = G
        free = (q < 0) & (sp == sp[s]) & (np.abs(E - E[s]) <= dE_eV) & (np.abs(lam - lam[s]) <= dlam_nm)
        q[free] = G
        G += 1
    return q, G
