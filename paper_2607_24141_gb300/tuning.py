"""Persistent cache of measured line-kernel tilings.

``pz_autotune`` times the compiled tilings of the line kernels on a context's own
workload (several seconds on a full spectrum).  The best tiling depends on the GPU,
on the library build and on the shape of the workload, not on its exact numbers, so
it is stored in a JSON file keyed by

* the GPU (device name and SM count),
* a hash of the library's sources (a rebuilt library with changed kernels re-tunes),
* the shape class of the context: stars, precision, layers, and the grid size, the
  window half-width and the line density (lines per grid point and star), each rounded
  on a log2 scale,
* and whether the tiling was timed on the forward alone (suffix "|fwd"): the backward
  kernels' best tiling can differ, so a forward-only entry never serves a fwd+bwd context,

and applied with ``pz_set_tiling`` when the same key comes back.  Host-side
bookkeeping only: nothing of the synthesis runs here.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
import tempfile

from . import pz_autotune, pz_set_tiling

_PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(_PKG, "tuning_cache.json")


def library_hash() -> str:
    """Hash of the CUDA sources and the public header the library is built from."""
    h = hashlib.sha256()
    csrc = os.path.join(_PKG, "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    with open(os.path.join(os.path.dirname(_PKG), "include", "pz.h"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def _log2_bucket(x: float) -> int:
    return int(round(math.log2(x))) if x > 0 else -99


def shape_class_of(prob, precision: int) -> str:
    """Shape key of a problem (single star, or a batch with .subsets) at a precision."""
    n_lambda = prob.grid.n_lambda
    batched = hasattr(prob, "subsets")
    if batched:
        lines = sum(len(x) for x in prob.subsets) / max(len(prob.subsets), 1)
        nd = prob.atmos[0].n_depth
        n_stars = len(prob.subsets)
    else:
        lines = prob.lines.n_lines
        nd = prob.atmos.n_depth
        n_stars = 1
    return "S%d-p%d-nd%d-nl%d-W%d-lpp%d" % (n_stars, precision, nd, _log2_bucket(n_lambda),
                                            _log2_bucket(prob.lines.half_window),
                                            _log2_bucket(2.0 * lines / max(n_lambda, 1)))


def shape_class(synth) -> str:
    """Shape key of a Synthesizer's workload (see the module docstring)."""
    return shape_class_of(synth.prob, synth.precision)


def cache_key(gpu: str, lib_hash: str, shape: str, with_backward: bool = True) -> str:
    """Key of a cache entry: GPU, library build, shape class, and "|fwd" for a tiling
    timed on the forward alone."""
    return "%s|%s|%s%s" % (gpu, lib_hash, shape, "" if with_backward else "|fwd")


def lookup(prob, precision: int, device=None, path: str = DEFAULT_CACHE, with_backward: bool = True):
    """The cached tiling (5 ints) for this GPU, library build and problem shape, or None."""
    key = cache_key(gpu_key(device), library_hash(), shape_class_of(prob, precision), with_backward)
    entry = _load(path).get(key)
    if entry and len(entry.get("tiling", ())) == 5:
        return tuple(entry["tiling"])
    return None


def gpu_key(device=None) -> str:
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device() if device is None else device)
    return "%s/%dsm" % (props.name, props.multi_processor_count)


def _load(path):
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _store(path, data):
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".tmp")
    with os.fdopen(fd, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune_cached(synth, path: str = DEFAULT_CACHE, with_backward: bool = True, reps: int = 2, stream=None,
                    write: bool = True):
    """Apply the cached tiling for this GPU, library build and workload shape, or tune
    (pz_autotune) and store the result.  Returns pz_autotune's dict plus "cached"
    (True when nothing was timed) and "key"."""
    key = cache_key(gpu_key(synth.device.index), library_hash(), shape_class(synth), with_backward)
    data = _load(path)
    entry = data.get(key)
    if entry and len(entry.get("tiling", ())) == 5:
        pz_set_tiling(synth.ctx, *entry["tiling"])
        return {"tiling": tuple(entry["tiling"]), "candidates": 0, "fwd_ms": entry.get("fwd_ms"),
                "bwd_ms": entry.get("bwd_ms"), "cached": True, "key": key}
    res = pz_autotune(synth.ctx, with_backward=with_backward, reps=reps, stream=stream)
    res["cached"] = False
    res["key"] = key
    if write:
        data = _load(path)
        data[key] = {"tiling": list(res["tiling"]), "fwd_ms": res["fwd_ms"], "bwd_ms": res["bwd_ms"]}
        _store(path, data)
    return res
