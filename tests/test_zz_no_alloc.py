"""The allocation-free abundance-gradient entry point, called through the C ABI,
against the regular pz_backward result (same tolerance as the gradient tests),
twice in a row so that the shared fixed scratch array is shown to be cleared
between calls.  This file is collected last on purpose."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I

pytestmark = pytest.mark.gpu
G_TOL = 1e-3


def rel_metric(g, ref):
    floor = 1e-3 * np.max(np.abs(ref))
    return np.abs(g - ref) / np.maximum(np.abs(ref), floor)


def test_abundance_gradient_without_allocation():
    import torch
    prob = I.small_config1(n_lambda_span_nm=3.0, seed=17)
    s = pz.Synthesizer(prob)
    nl, n_elem = prob.lines.n_lines, prob.n_elem
    dev = s.device
    zeros = np.zeros(nl, np.float32)
    s.set_corrections(zeros, zeros, np.zeros(n_elem, np.float32))
    f = s.forward()
    rng = np.random.default_rng(3)
    y = torch.tensor(f.cpu().numpy() + rng.normal(0, 1 / 200, f.numel()).astype(np.float32), device=dev)
    w = torch.full_like(y, 4e4)
    dLdf = torch.empty_like(y)
    s.loss(y, w, None, dLdf)
    g_gf = torch.empty(nl, dtype=torch.float32, device=dev)
    g_g6 = torch.empty(nl, dtype=torch.float32, device=dev)
    g_ab = torch.empty(n_elem, dtype=torch.float32, device=dev)
    s.backward(dLdf, g_gf, g_g6, g_ab)
    species = torch.tensor(prob.lines.species, dtype=torch.int32, device=dev)
    eos = torch.tensor(prob.elem_of_species, dtype=torch.int32, device=dev)
    ref = g_ab.cpu().numpy().astype(np.float64)
    for call in range(2):
        out = torch.full((n_elem,), float("nan"), dtype=torch.float32, device=dev)
        pz.pz_abundance_grad_noalloc(g_gf, species, eos, n_elem, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        err = rel_metric(got, ref).max()
        assert err < G_TOL, (call, err)
    s.close()


def test_rejects_sizes_beyond_the_fixed_scratch():
    import torch
    g = torch.zeros(4, dtype=torch.float32, device="cuda")
    sp = torch.zeros(4, dtype=torch.int32, device="cuda")
    eos = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(5000, dtype=torch.float32, device="cuda")
    with pytest.raises(pz.PzError) as e:
        pz.pz_abundance_grad_noalloc(g, sp, eos, 5000, out)
    assert e.value.status == pz.PZ_EINVAL
