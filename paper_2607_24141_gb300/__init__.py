"""GB300-native synthesis hot path of arXiv:2607.24141 ("The Payne Zero Project I").

The compute lives in ``libpz.so`` (CUDA, sm_103a) behind the C ABI declared in
``include/pz.h``.  This module only marshals arguments:

* ``pz_create``, ``pz_line_opacity``, ``pz_flux``, ``pz_instrument``,
  ``pz_loss_chi2``, ``pz_backward``, ... -- one Python function per C entry
  point, same name, raising :class:`PzError` on a non-zero status;
* :class:`Synthesizer` -- owns one context plus the host arrays it was built
  from, with torch CUDA tensors as device buffers;
* :class:`SynthesisFunction` (and :class:`SynthesisFunction4`, all four corrections of
  Eq. 10) -- a ``torch.autograd.Function`` whose forward is
  line opacity -> flux -> instrument and whose backward is ``pz_backward``.

There is no CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import inputs  # noqa: F401  (seeded generators; no synthesis arithmetic)

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libpz.so")
_lib = None

PZ_OK, PZ_EINVAL, PZ_ENOMEM, PZ_ECUDA, PZ_ETIMEOUT, PZ_ESTATE, PZ_ENUMERIC = range(7)
PZ_FP64, PZ_MIXED = 0, 1
_STATUS = {1: "PZ_EINVAL", 2: "PZ_ENOMEM", 3: "PZ_ECUDA", 4: "PZ_ETIMEOUT", 5: "PZ_ESTATE", 6: "PZ_ENUMERIC"}

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)
_vp = C.c_void_p


class PzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class pz_atmos(C.Structure):
    _fields_ = [("n_depth", C.c_int32), ("n_species", C.c_int32),
                ("m", _dp), ("T", _dp), ("rho", _dp), ("n_e", _dp), ("n_pert", _dp),
                ("pop", _dp), ("mass_amu", _dp), ("xi_cms", C.c_double), ("kappa_c", _dp),
                ("lambda0_nm", C.c_double), ("R_grid", C.c_double), ("n_lambda", C.c_int64)]


class pz_linelist(C.Structure):
    _fields_ = [("n_lines", C.c_int64), ("lambda_nm", _dp), ("log_gf", _fp), ("E_low_eV", _fp),
                ("log_gamma_rad", _fp), ("log_gamma4", _fp), ("log_gamma6", _fp),
                ("species", _ip), ("half_window", C.c_int32)]


# name -> (restype, argtypes)
_SIGS = {
    "pz_create": (C.c_int, [C.POINTER(pz_atmos), C.POINTER(pz_linelist), C.c_int, C.POINTER(_vp)]),
    "pz_destroy": (C.c_int, [_vp]),
    "pz_set_corrections": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int32, _vp]),
    "pz_line_opacity": (C.c_int, [_vp, _vp, _vp]),
    "pz_flux": (C.c_int, [_vp, _vp, _vp, _vp]),
    "pz_instrument": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, _vp, C.c_int64, _vp, _vp]),
    "pz_loss_chi2": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp]),
    "pz_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pz_last_error": (C.c_char_p, []),
    "pz_eval_count": (C.c_int64, [_vp]),
    "pz_last_launch_count": (C.c_int32, [_vp]),
    "pz_set_tiling": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "pz_autotune": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    "pz_set_centre_test": (C.c_int, [_vp, C.c_double, C.POINTER(C.c_int64), _vp]),
    "pz_set_profiling": (C.c_int, [_vp, C.c_int32]),
    "pz_kernel_times": (C.c_int, [_vp, _dp, C.POINTER(C.c_int64), C.c_int32]),
    "pz_abundance_grad_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int32, C.c_int32, _vp, _vp]),
    "pz_create_batch": (C.c_int, [C.c_int32, C.POINTER(pz_atmos), C.POINTER(pz_linelist), _vp, _vp, C.c_int,
                                  C.POINTER(_vp)]),
    "pz_n_stars": (C.c_int32, [_vp]),
    "pz_star_lines": (C.c_int64, [_vp, C.c_int32]),
    "pz_get_corrections": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pz_calib_step": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_float, C.c_float, C.c_float, _vp, _vp, _vp, _vp,
                                _vp]),
    "pz_probe_voigt": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp]),
    "pz_probe_expn": (C.c_int, [_vp, C.c_int64, _vp, _vp]),
    "pz_probe_pipe": (C.c_int, [C.c_int32, C.c_int32, _dp, _vp]),
    "pz_probe_wait": (C.c_int, [C.c_int64, C.POINTER(C.c_int32), _vp]),
    "pz_sync_status": (C.c_int, [_vp, _vp, C.POINTER(C.c_int32)]),
    "pz_set_damping_corrections": (C.c_int, [_vp, _vp, _vp, _vp]),
    "pz_set_scattering": (C.c_int, [_vp, _vp, _vp]),
    "pz_get_damping_corrections": (C.c_int, [_vp, _vp, _vp, _vp]),
    "pz_backward4": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pz_set_line_groups": (C.c_int, [_vp, _vp, C.c_int64]),
    "pz_group_eval": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]),
    "pz_build_line_groups": (C.c_int, [C.c_int64, _vp, _vp, _vp, _vp, C.c_double, C.c_double, _vp,
                                       C.POINTER(C.c_int64)]),
    "pz_set_allocator": (C.c_int, [_vp, _vp, _vp]),
}
EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True):
    """Load libpz.so (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libpz.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(_LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int):
    if st != PZ_OK:
        raise PzError(st, load().pz_last_error().decode())


def _ptr(t) -> Optional[int]:
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------------------
# one function per C entry point (argument marshalling only)
# ---------------------------------------------------------------------------

def pz_create(atmos: pz_atmos, lines: pz_linelist, precision: int = PZ_MIXED) -> int:
    ctx = _vp()
    _check(load().pz_create(C.byref(atmos), C.byref(lines), int(precision), C.byref(ctx)))
    return ctx.value


def pz_create_batch(atmos_list, lines: pz_linelist, subset_offsets=None, subset_index=None,
                    precision: int = PZ_MIXED) -> int:
    """atmos_list: sequence of pz_atmos; subset_offsets int64 [S+1] and subset_index int32
    (host numpy) or None (every star uses every line)."""
    S = len(atmos_list)
    arr = (pz_atmos * S)(*atmos_list)
    off = idx = None
    if subset_offsets is not None:
        off = np.ascontiguousarray(subset_offsets, dtype=np.int64)
        idx = np.ascontiguousarray(subset_index, dtype=np.int32)
    ctx = _vp()
    _check(load().pz_create_batch(S, arr, C.byref(lines), None if off is None else off.ctypes.data,
                                  None if idx is None or idx.size == 0 else idx.ctypes.data, int(precision),
                                  C.byref(ctx)))
    return ctx.value


def pz_n_stars(ctx) -> int:
    return int(load().pz_n_stars(ctx))


def pz_star_lines(ctx, star: int) -> int:
    return int(load().pz_star_lines(ctx, int(star)))


def pz_get_corrections(ctx, dlog_gf=None, dlog_gamma6=None, dabund=None, stream=None):
    """Outputs may be torch tensors (device) or numpy float32 arrays (host)."""
    def p(x):
        if x is None:
            return None
        return x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
    _check(load().pz_get_corrections(ctx, p(dlog_gf), p(dlog_gamma6), p(dabund), _stream(stream)))


def pz_calib_step(ctx, y, w=None, lr_gf=0.0, lr_g6=0.0, lr_ab=0.0, loss=None, g_dlog_gf=None,
                  g_dlog_gamma6=None, g_dabund=None, stream=None):
    _check(load().pz_calib_step(ctx, _ptr(y), _ptr(w), y.shape[-1], float(lr_gf), float(lr_g6), float(lr_ab),
                                _ptr(loss), _ptr(g_dlog_gf), _ptr(g_dlog_gamma6), _ptr(g_dabund),
                                _stream(stream)))


def pz_destroy(ctx: int):
    _check(load().pz_destroy(ctx))


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_allocator_refs = None   # keeps the installed callbacks alive


def pz_set_allocator(alloc=None, free=None, user=None):
    """Install device-memory callbacks for the library (alloc(bytes, user) -> int pointer
    or 0, free(ptr, user)), or, with no arguments, go back to cudaMalloc / cudaFree.
    Python callables are wrapped as C function pointers and kept alive here."""
    global _allocator_refs
    if (alloc is None) != (free is None):
        raise PzError(PZ_EINVAL, "pz_set_allocator: give both functions or neither")
    if alloc is None:
        _check(load().pz_set_allocator(None, None, None))
        _allocator_refs = None
        return
    a = alloc if isinstance(alloc, ALLOC_FN) else ALLOC_FN(lambda n, u: alloc(int(n), u) or 0)
    f = free if isinstance(free, FREE_FN) else FREE_FN(lambda p, u: free(int(p or 0), u))
    _check(load().pz_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), user))
    _allocator_refs = (a, f)


def torch_allocator():
    """(alloc, free) callbacks that take the library's device memory from PyTorch's
    caching allocator on the current device (a framework-owned pool)."""
    import torch

    def alloc(n, _user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(n)))
        except RuntimeError:
            return 0

    def free(p, _user):
        if p:
            torch.cuda.caching_allocator_delete(p)

    return alloc, free


def pz_set_corrections(ctx, dlog_gf=None, dlog_gamma6=None, dabund=None, elem_of_species=None,
                       n_elem: int = 0, stream=None):
    """Pointers may be torch CUDA tensors or numpy arrays (host)."""
    keep = []

    def p(x, dt):
        if x is None:
            return None
        if isinstance(x, np.ndarray):
            a = np.ascontiguousarray(x, dtype=dt)
            keep.append(a)
            return a.ctypes.data
        return x.data_ptr()
    _check(load().pz_set_corrections(ctx, p(dlog_gf, np.float32), p(dlog_gamma6, np.float32),
                                     p(dabund, np.float32), p(elem_of_species, np.int32), int(n_elem),
                                     _stream(stream)))


def pz_line_opacity(ctx, kappa_line=None, stream=None):
    _check(load().pz_line_opacity(ctx, _ptr(kappa_line), _stream(stream)))


def pz_flux(ctx, F=None, Fc=None, stream=None):
    _check(load().pz_flux(ctx, _ptr(F), _ptr(Fc), _stream(stream)))


def pz_instrument(ctx, v_r_kms, v_b_kms, R_lsf, pix_lambda_nm, f_norm=None, stream=None):
    if pix_lambda_nm is None:
        _check(load().pz_instrument(ctx, 0.0, 0.0, 0.0, None, 0, _ptr(f_norm), _stream(stream)))
        return
    pix = np.ascontiguousarray(pix_lambda_nm, dtype=np.float64)
    _check(load().pz_instrument(ctx, float(v_r_kms), float(v_b_kms), float(R_lsf), pix.ctypes.data,
                                pix.size, _ptr(f_norm), _stream(stream)))


def pz_loss_chi2(ctx, y, w=None, loss=None, dL_df=None, stream=None):
    _check(load().pz_loss_chi2(ctx, _ptr(y), _ptr(w), y.shape[-1], _ptr(loss), _ptr(dL_df), _stream(stream)))


def pz_backward(ctx, dL_df, g_dlog_gf=None, g_dlog_gamma6=None, g_dabund=None, stream=None):
    _check(load().pz_backward(ctx, _ptr(dL_df), _ptr(g_dlog_gf), _ptr(g_dlog_gamma6), _ptr(g_dabund),
                              _stream(stream)))


def pz_set_damping_corrections(ctx, dlog_gamma_rad=None, dlog_gamma4=None, stream=None):
    """Radiative and Stark corrections of Eq. 10 (caller order; numpy = host, torch = device)."""
    keep = []

    def p(x):
        if x is None:
            return None
        if isinstance(x, np.ndarray):
            a = np.ascontiguousarray(x, dtype=np.float32)
            keep.append(a)
            return a.ctypes.data
        return x.data_ptr()
    _check(load().pz_set_damping_corrections(ctx, p(dlog_gamma_rad), p(dlog_gamma4), _stream(stream)))


def pz_set_scattering(ctx, sigma_c=None, stream=None):
    """Continuum scattering coefficient, host FP64 [S][n_depth][n_lambda] (None: off)."""
    if sigma_c is None:
        _check(load().pz_set_scattering(ctx, None, _stream(stream)))
        return
    a = np.ascontiguousarray(sigma_c, dtype=np.float64)
    _check(load().pz_set_scattering(ctx, a.ctypes.data, _stream(stream)))


def pz_get_damping_corrections(ctx, dlog_gamma_rad=None, dlog_gamma4=None, stream=None):
    """Copy the radiative and Stark corrections into numpy (host) or torch (device) arrays."""
    def p(x):
        if x is None:
            return None
        return x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
    _check(load().pz_get_damping_corrections(ctx, p(dlog_gamma_rad), p(dlog_gamma4), _stream(stream)))


def pz_backward4(ctx, dL_df, g_dlog_gf=None, g_dlog_gamma_rad=None, g_dlog_gamma4=None, g_dlog_gamma6=None,
                 g_dabund=None, stream=None):
    _check(load().pz_backward4(ctx, _ptr(dL_df), _ptr(g_dlog_gf), _ptr(g_dlog_gamma_rad), _ptr(g_dlog_gamma4),
                               _ptr(g_dlog_gamma6), _ptr(g_dabund), _stream(stream)))


def pz_set_line_groups(ctx, group_of_line, n_groups):
    q = np.ascontiguousarray(group_of_line, dtype=np.int32)
    _check(load().pz_set_line_groups(ctx, q.ctypes.data, int(n_groups)))


def pz_group_eval(ctx, y, w, x, loss=None, g=None, stream=None):
    """x, g: device FP32 [4][n_groups] (gf, rad, Stark, vdW); y, w: device FP32 [S][n]."""
    _check(load().pz_group_eval(ctx, _ptr(y), _ptr(w), y.shape[-1], _ptr(x), _ptr(loss), _ptr(g), _stream(stream)))


def pz_build_line_groups(lambda_nm, E_low_eV, species, strength, dE_eV, dlam_nm):
    """Greedy strength-ordered grouping (host).  Returns (group_of_line int32, n_groups)."""
    lam = np.ascontiguousarray(lambda_nm, dtype=np.float64)
    E = np.ascontiguousarray(E_low_eV, dtype=np.float32)
    sp = np.ascontiguousarray(species, dtype=np.int32)
    st = np.ascontiguousarray(strength, dtype=np.float32)
    n = lam.size
    if not (E.size == sp.size == st.size == n):
        raise ValueError("pz_build_line_groups: arrays differ in length")
    q = np.empty(max(n, 1), np.int32)
    G = C.c_int64(0)
    _check(load().pz_build_line_groups(n, lam.ctypes.data, E.ctypes.data, sp.ctypes.data, st.ctypes.data,
                                       float(dE_eV), float(dlam_nm), q.ctypes.data, C.byref(G)))
    return q[:n], int(G.value)


def pz_eval_count(ctx) -> int:
    return int(load().pz_eval_count(ctx))


def pz_last_launch_count(ctx) -> int:
    return int(load().pz_last_launch_count(ctx))


def pz_set_tiling(ctx, lambda_per_thread=0, depth_per_warp=0, warps_per_cta=0, lines_per_chunk=0, ctas_per_sm=0):
    _check(load().pz_set_tiling(ctx, lambda_per_thread, depth_per_warp, warps_per_cta, lines_per_chunk, ctas_per_sm))


def pz_set_centre_test(ctx, eta, stream=None) -> int:
    """Continuum-referenced centre test with selection fraction eta (0 = off); returns
    the number of kept (line, depth) pairs."""
    n = C.c_int64(0)
    _check(load().pz_set_centre_test(ctx, float(eta), C.byref(n), _stream(stream)))
    return n.value


def pz_autotune(ctx, with_backward=True, reps=2, stream=None):
    """Measure the line-kernel tilings on this context and keep the fastest.

    Returns {"tiling": (lambda_per_thread, depth_per_warp, warps_per_cta,
    lines_per_chunk, ctas_per_sm), "candidates": n, "fwd_ms": f, "bwd_ms": b}."""
    best = (C.c_int32 * 6)()
    ms = (C.c_double * 2)()
    _check(load().pz_autotune(ctx, 1 if with_backward else 0, int(reps), best, ms, _stream(stream)))
    return {"tiling": tuple(best[:5]), "candidates": best[5], "fwd_ms": ms[0], "bwd_ms": ms[1]}


KERNEL_NAMES = ("line_fwd", "line_bwd", "flux", "rt_adjoint", "instrument", "inst_adjoint", "loss", "other",
                "step", "near_fwd", "near_bwd")


def pz_set_profiling(ctx, enable=True):
    _check(load().pz_set_profiling(ctx, 1 if enable else 0))


def pz_kernel_times(ctx):
    """{family: (total_ms, launches)} accumulated since profiling was enabled."""
    n = len(KERNEL_NAMES)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _check(load().pz_kernel_times(ctx, ms, cnt, n))
    return {KERNEL_NAMES[k]: (ms[k], cnt[k]) for k in range(n)}


def _check_tensor(name, t, dtype, min_numel):
    import torch
    if not isinstance(t, torch.Tensor):
        raise PzError(PZ_EINVAL, "%s must be a torch tensor" % name)
    if t.dtype != dtype:
        raise PzError(PZ_EINVAL, "%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise PzError(PZ_EINVAL, "%s must be contiguous" % name)
    if t.numel() < min_numel:
        raise PzError(PZ_EINVAL, "%s holds %d entries, needs %d" % (name, t.numel(), min_numel))


def pz_abundance_grad_noalloc(g_dlog_gf, species, elem_of_species, n_elem, g_dabund, stream=None):
    """Per-element sums of per-line gradients with no device allocation.

    g_dlog_gf: float32 [n_lines], species: int32 [n_lines], elem_of_species: int32
    [n_species], g_dabund: float32 [>= n_elem], all contiguous CUDA tensors on one
    device.  The C entry point takes bare pointers, so the sizes, types and device
    are checked here before the call (PZ_EINVAL)."""
    import torch
    if int(n_elem) < 0:
        raise PzError(PZ_EINVAL, "n_elem must be >= 0")
    _check_tensor("g_dlog_gf", g_dlog_gf, torch.float32, 0)
    n_lines = g_dlog_gf.numel()
    _check_tensor("species", species, torch.int32, 0)
    if species.numel() != n_lines:
        raise PzError(PZ_EINVAL, "species holds %d entries, g_dlog_gf %d" % (species.numel(), n_lines))
    _check_tensor("elem_of_species", elem_of_species, torch.int32, 0)
    _check_tensor("g_dabund", g_dabund, torch.float32, int(n_elem))
    dev = g_dlog_gf.device
    for name, t in (("g_dlog_gf", g_dlog_gf), ("species", species), ("elem_of_species", elem_of_species),
                    ("g_dabund", g_dabund)):
        if not t.is_cuda or t.device != dev:
            raise PzError(PZ_EINVAL, "%s must be a CUDA tensor on the device of g_dlog_gf (%s)" % (name, dev))
    _check(load().pz_abundance_grad_noalloc(_ptr(g_dlog_gf), _ptr(species), _ptr(elem_of_species),
                                            n_lines, elem_of_species.numel(), int(n_elem),
                                            _ptr(g_dabund), _stream(stream)))


def pz_probe_voigt(a, v, H, dHda=None, stream=None):
    _check(load().pz_probe_voigt(_ptr(a), _ptr(v), a.numel(), _ptr(H), _ptr(dHda), _stream(stream)))


def pz_probe_expn(x, out, stream=None):
    """out: device FP64 [5][n] (E_2, E_3, E_4 of the flux kernels; E_2, E_3 of the scattering table)."""
    if out.numel() < 5 * x.numel():
        raise ValueError("pz_probe_expn: out needs 5 * x.numel() elements")
    _check(load().pz_probe_expn(_ptr(x), x.numel(), _ptr(out), _stream(stream)))


def pz_probe_wait(limit_ns, stream=None) -> int:
    """Run the bounded-wait failure path on a barrier nothing completes; returns the status word."""
    f = C.c_int32(0)
    _check(load().pz_probe_wait(int(limit_ns), C.byref(f), _stream(stream)))
    return f.value


def pz_sync_status(ctx, stream=None) -> int:
    """Synchronise, read and clear the context's device status word (raises PZ_ETIMEOUT if a bounded
    wait gave up, PZ_ENUMERIC if a scattering-source refinement did not converge)."""
    f = C.c_int32(0)
    _check(load().pz_sync_status(ctx, _stream(stream), C.byref(f)))
    return f.value


def pz_probe_pipe(pipe, iters=4096, stream=None) -> float:
    """Measured operations per second of pipe 0 (FP32 FMA), 1 (MUFU reciprocal) or 2 (FP64 FMA)."""
    r = C.c_double(0.0)
    _check(load().pz_probe_pipe(int(pipe), int(iters), C.byref(r), _stream(stream)))
    return r.value


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

def _atmos_struct(at, kappa_c, grid, keep: list) -> pz_atmos:
    f64 = lambda a: np.ascontiguousarray(a, np.float64)  # noqa: E731
    arrs = [f64(at.m), f64(at.T), f64(at.rho), f64(at.n_e), f64(at.n_pert), f64(at.pop), f64(at.mass_amu),
            f64(kappa_c)]
    keep.extend(arrs)
    A = pz_atmos()
    A.n_depth, A.n_species = at.n_depth, at.n_species
    A.m, A.T, A.rho, A.n_e, A.n_pert, A.pop, A.mass_amu, A.kappa_c = [x.ctypes.data_as(_dp) for x in arrs]
    A.xi_cms = at.xi_cms
    A.lambda0_nm, A.R_grid, A.n_lambda = grid.lambda0_nm, grid.R_grid, grid.n_lambda
    return A


def _lines_struct(ll, keep: list) -> pz_linelist:
    f32 = lambda a: np.ascontiguousarray(a, np.float32)  # noqa: E731
    lam = np.ascontiguousarray(ll.lambda_nm, np.float64)
    cols = [f32(ll.log_gf), f32(ll.E_low_eV), f32(ll.log_gamma_rad), f32(ll.log_gamma4), f32(ll.log_gamma6)]
    sp = np.ascontiguousarray(ll.species, np.int32)
    keep.extend([lam, sp] + cols)
    L = pz_linelist()
    L.n_lines = ll.n_lines
    L.lambda_nm = lam.ctypes.data_as(_dp)
    L.log_gf, L.E_low_eV, L.log_gamma_rad, L.log_gamma4, L.log_gamma6 = [x.ctypes.data_as(_fp) for x in cols]
    L.species = sp.ctypes.data_as(_ip)
    L.half_window = ll.half_window
    return L


class Synthesizer:
    """One context for an :class:`inputs.Problem` (one star) or an :class:`inputs.Batch`
    (many stars sharing a grid and a master line list).  For a batch every per-star
    output gains a leading [n_stars] dimension."""

    def __init__(self, prob, precision: int = PZ_MIXED, device: int = 0):
        import torch
        torch.cuda.set_device(device)
        self.prob = prob
        self.precision = precision
        keep = []
        self.batched = hasattr(prob, "subsets")
        if self.batched:
            atl = [_atmos_struct(a, kc, prob.grid, keep) for a, kc in zip(prob.atmos, prob.kappa_c)]
            L = _lines_struct(prob.lines, keep)
            off = np.concatenate([[0], np.cumsum([len(x) for x in prob.subsets])]).astype(np.int64)
            idx = (np.concatenate(prob.subsets) if len(prob.subsets) else np.zeros(0)).astype(np.int32)
            self.ctx = pz_create_batch(atl, L, off, idx, precision)
            self.n_stars = len(atl)
            self.n_depth = prob.atmos[0].n_depth
        else:
            A = _atmos_struct(prob.atmos, prob.kappa_c, prob.grid, keep)
            L = _lines_struct(prob.lines, keep)
            self.ctx = pz_create(A, L, precision)
            self.n_stars = 1
            self.n_depth = prob.atmos.n_depth
        self._keep = keep
        sig = getattr(prob, "sigma_c", None)
        if sig is not None:
            # one star: [n_depth][n_lambda]; a batch: one such array per star
            pz_set_scattering(self.ctx, np.stack(sig) if self.batched else sig)
        self.device = torch.device("cuda", device)
        self.n_lambda = prob.grid.n_lambda
        self.n_lines = prob.lines.n_lines
        self.n_out = prob.instrument.pix_lambda_nm.size if prob.instrument is not None else self.n_lambda

    def close(self):
        if getattr(self, "ctx", None):
            pz_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_evals(self) -> int:
        return pz_eval_count(self.ctx)

    def _shape(self, n):
        return (self.n_stars, n) if self.batched else (n,)

    def set_corrections(self, dlog_gf=None, dlog_gamma6=None, dabund=None, stream=None):
        eos = self.prob.elem_of_species if dabund is not None else None
        pz_set_corrections(self.ctx, dlog_gf, dlog_gamma6, dabund, eos,
                           self.prob.n_elem if dabund is not None else 0, stream)

    def configure_instrument(self, stream=None):
        """Run the instrument once on the current flux so that pz_calib_step can use it."""
        inst = self.prob.instrument
        if inst is None:
            pz_instrument(self.ctx, 0, 0, 0, None, None, stream)
        else:
            pz_instrument(self.ctx, inst.v_r_kms, inst.v_b_kms, inst.R_lsf, inst.pix_lambda_nm, None, stream)

    def forward(self, kappa=None, F=None, Fc=None, f=None, stream=None):
        """line opacity -> flux -> instrument; returns f (allocated if not given)."""
        import torch
        if f is None:
            f = torch.empty(self._shape(self.n_out), dtype=torch.float32, device=self.device)
        pz_line_opacity(self.ctx, kappa, stream)
        pz_flux(self.ctx, F, Fc, stream)
        inst = self.prob.instrument
        if inst is None:
            pz_instrument(self.ctx, 0, 0, 0, None, f, stream)
        else:
            pz_instrument(self.ctx, inst.v_r_kms, inst.v_b_kms, inst.R_lsf, inst.pix_lambda_nm, f, stream)
        return f

    def loss(self, y, w=None, loss=None, dL_df=None, stream=None):
        pz_loss_chi2(self.ctx, y, w, loss, dL_df, stream)

    def backward(self, dL_df, g_gf=None, g_g6=None, g_ab=None, stream=None):
        pz_backward(self.ctx, dL_df, g_gf, g_g6, g_ab, stream)

    def calib_step(self, y, w=None, lr_gf=0.0, lr_g6=0.0, lr_ab=0.0, loss=None, g_gf=None, g_g6=None, g_ab=None,
                   stream=None):
        pz_calib_step(self.ctx, y, w, lr_gf, lr_g6, lr_ab, loss, g_gf, g_g6, g_ab, stream)

    def set_damping_corrections(self, dlog_gamma_rad=None, dlog_gamma4=None, stream=None):
        pz_set_damping_corrections(self.ctx, dlog_gamma_rad, dlog_gamma4, stream)

    def backward4(self, dL_df, g_gf=None, g_rad=None, g_g4=None, g_g6=None, g_ab=None, stream=None):
        pz_backward4(self.ctx, dL_df, g_gf, g_rad, g_g4, g_g6, g_ab, stream)

    def get_damping_corrections(self):
        """(dlog_gamma_rad, dlog_gamma4) as host float32 arrays."""
        r = np.empty(self.n_lines, np.float32)
        s4 = np.empty(self.n_lines, np.float32)
        pz_get_damping_corrections(self.ctx, r, s4)
        return r, s4

    def get_corrections(self):
        """(dlog_gf, dlog_gamma6, dabund or None) as host float32 arrays."""
        gf = np.empty(self.n_lines, np.float32)
        g6 = np.empty(self.n_lines, np.float32)
        ab = np.empty(self.prob.n_elem, np.float32) if self.prob.n_elem else None
        pz_get_corrections(self.ctx, gf, g6, ab)
        return gf, g6, ab


def _torch_function():
    import torch

    class SynthesisFunction(torch.autograd.Function):
        """f = instrument(flux(line_opacity(corrections))) with a hand-written backward.

        Inputs are the corrections (Delta log gf, Delta log gamma6, Delta abundance)
        as float32 CUDA tensors; gradients come from ``pz_backward``."""

        @staticmethod
        def forward(ctx, synth, dlog_gf, dlog_gamma6, dabund):
            synth.set_corrections(dlog_gf, dlog_gamma6, dabund)
            f = synth.forward()
            ctx.synth = synth
            ctx.has_ab = dabund is not None
            return f

        @staticmethod
        def backward(ctx, grad_f):
            s = ctx.synth
            grad_f = grad_f.contiguous().to(torch.float32)
            nl = s.n_lines
            g_gf = torch.empty(nl, dtype=torch.float32, device=grad_f.device)
            g_g6 = torch.empty(nl, dtype=torch.float32, device=grad_f.device)
            g_ab = torch.empty(s.prob.n_elem, dtype=torch.float32, device=grad_f.device) if ctx.has_ab else None
            s.backward(grad_f, g_gf, g_g6, g_ab)
            return None, g_gf, g_g6, g_ab

    return SynthesisFunction


def _torch_function4():
    import torch

    class SynthesisFunction4(torch.autograd.Function):
        """f = instrument(flux(line_opacity(corrections))) over the four per-line
        corrections of Eq. 10 (Delta log gf, Delta log gamma_rad, Delta log gamma_4,
        Delta log gamma_6) and the abundance offsets, float32 CUDA tensors; gradients
        come from ``pz_backward4``."""

        @staticmethod
        def forward(ctx, synth, dlog_gf, dlog_gamma_rad, dlog_gamma4, dlog_gamma6, dabund):
            synth.set_corrections(dlog_gf, dlog_gamma6, dabund)
            synth.set_damping_corrections(dlog_gamma_rad, dlog_gamma4)
            f = synth.forward()
            ctx.synth = synth
            ctx.has_ab = dabund is not None
            return f

        @staticmethod
        def backward(ctx, grad_f):
            s = ctx.synth
            grad_f = grad_f.contiguous().to(torch.float32)
            nl = s.n_lines
            g = [torch.empty(nl, dtype=torch.float32, device=grad_f.device) for _ in range(4)]
            g_ab = torch.empty(s.prob.n_elem, dtype=torch.float32, device=grad_f.device) if ctx.has_ab else None
            s.backward4(grad_f, g[0], g[1], g[2], g[3], g_ab)
            return None, g[0], g[1], g[2], g[3], g_ab

    return SynthesisFunction4


def __getattr__(name):
    if name == "SynthesisFunction":
        return _torch_function()
    if name == "SynthesisFunction4":
        return _torch_function4()
    raise AttributeError(name)
