"""Error behaviour of the C ABI (validation launches nothing)."""
import numpy as np
import pytest

import paper_2607_24141_gb300 as pz
from tiny import tiny_problem

pytestmark = pytest.mark.gpu


def test_invalid_inputs_rejected():
    prob = tiny_problem()
    prob.atmos.m[2] = prob.atmos.m[1]           # not strictly increasing
    with pytest.raises(pz.PzError) as e:
        pz.Synthesizer(prob)
    assert e.value.status == pz.PZ_EINVAL
    prob = tiny_problem()
    prob.lines.species[0] = 99
    with pytest.raises(pz.PzError):
        pz.Synthesizer(prob)
    prob = tiny_problem()
    prob.kappa_c[0, 0] = np.nan
    with pytest.raises(pz.PzError):
        pz.Synthesizer(prob)


def test_call_order_enforced():
    import torch
    s = pz.Synthesizer(tiny_problem())
    with pytest.raises(pz.PzError) as e:
        pz.pz_flux(s.ctx)
    assert e.value.status == pz.PZ_ESTATE
    with pytest.raises(pz.PzError) as e:
        pz.pz_backward(s.ctx, torch.zeros(64, device="cuda"))
    assert e.value.status == pz.PZ_ESTATE
    s.forward()
    y = torch.zeros(10, device="cuda")
    with pytest.raises(pz.PzError) as e:
        s.loss(y)
    assert e.value.status == pz.PZ_EINVAL


def test_instrument_rejects_pixels_off_grid():
    prob = tiny_problem(n_lambda=300)
    s = pz.Synthesizer(prob)
    pz.pz_line_opacity(s.ctx)
    pz.pz_flux(s.ctx)
    with pytest.raises(pz.PzError):
        pz.pz_instrument(s.ctx, 0.0, 0.0, 22500.0, np.array([100.0, 101.0]))
    with pytest.raises(pz.PzError):
        pz.pz_instrument(s.ctx, 0.0, 0.0, -1.0, np.array([600.01]))


def test_launch_count_and_eval_count():
    prob = tiny_problem(n_lambda=400, n_lines=12, W=30)
    s = pz.Synthesizer(prob)
    pz.pz_line_opacity(s.ctx)
    assert pz.pz_last_launch_count(s.ctx) == 3      # near-core, far-wing line records, far-wing kernels
    assert s.n_evals == prob.n_evals


def test_bounded_wait_reports_instead_of_hanging():
    # a barrier phase that nothing completes: the wait gives up after 2 ms and sets bit 0
    assert pz.pz_probe_wait(2_000_000) == 1
    # a context whose staged chunks all arrive reports a clean status
    s = pz.Synthesizer(tiny_problem())
    s.forward()
    assert pz.pz_sync_status(s.ctx) == 0
    with pytest.raises(pz.PzError) as e:
        pz.pz_probe_wait(0)
    assert e.value.status == pz.PZ_EINVAL
