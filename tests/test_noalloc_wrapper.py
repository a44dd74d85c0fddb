"""The binding of the allocation-free abundance-gradient entry point checks its tensors
before the call: the C entry point takes bare device pointers and cannot tell a short
or wrongly typed buffer from a good one.  No GPU needed: every case is refused before
the library is touched."""
import pytest
import torch

import paper_2607_24141_gb300 as pz


def _args(n_lines=8, n_species=3, n_elem=2, out=None):
    g = torch.zeros(n_lines, dtype=torch.float32)
    sp = torch.zeros(n_lines, dtype=torch.int32)
    eos = torch.zeros(n_species, dtype=torch.int32)
    return g, sp, eos, n_elem, torch.zeros(n_elem, dtype=torch.float32) if out is None else out


def _refused(*args, match):
    with pytest.raises(pz.PzError, match=match) as e:
        pz.pz_abundance_grad_noalloc(*args)
    assert e.value.status == pz.PZ_EINVAL


def test_short_output_is_refused():
    g, sp, eos, n_elem, _ = _args(n_elem=5)
    _refused(g, sp, eos, n_elem, torch.zeros(4, dtype=torch.float32), match="g_dabund holds 4 entries, needs 5")


def test_species_length_must_match_the_gradients():
    g, _, eos, n_elem, out = _args()
    _refused(g, torch.zeros(7, dtype=torch.int32), eos, n_elem, out, match="species holds 7")


def test_wrong_dtypes_are_refused():
    g, sp, eos, n_elem, out = _args()
    _refused(g.double(), sp, eos, n_elem, out, match="g_dlog_gf must be torch.float32")
    _refused(g, sp.long(), eos, n_elem, out, match="species must be torch.int32")
    _refused(g, sp, eos, n_elem, out.half(), match="g_dabund must be torch.float32")


def test_strided_tensors_are_refused():
    g, sp, eos, n_elem, out = _args(n_lines=16)
    _refused(g[::2], sp[::2], eos, n_elem, out, match="must be contiguous")


def test_host_tensors_are_refused():
    _refused(*_args(), match="must be a CUDA tensor")
