"""Caller-supplied device allocator (pz_set_allocator): the library's device memory
comes from the caller's callbacks, an allocation failure surfaces as PZ_ENOMEM with
everything taken so far handed back, and the allocator cannot change under live
contexts."""
import pytest

import paper_2607_24141_gb300 as pz
from paper_2607_24141_gb300 import inputs as I


def test_allocator_arguments_are_validated():
    """Host-side rules, no device involved: both callbacks or neither."""
    with pytest.raises(pz.PzError) as e:
        pz.pz_set_allocator(lambda n, u: 0, None)
    assert e.value.status == pz.PZ_EINVAL
    calls = []
    pz.pz_set_allocator(lambda n, u: calls.append(n) or 0, lambda p, u: None)
    pz.pz_set_allocator()            # back to cudaMalloc / cudaFree
    assert calls == []               # installing or removing allocates nothing


@pytest.mark.gpu
def test_allocation_failure_is_reported_and_nothing_leaks():
    import gc

    import torch
    gc.collect()                     # contexts other tests left to the garbage collector
    prob = I.small_config1(n_lambda_span_nm=1.0, seed=3)
    alloc, free = pz.torch_allocator()
    live = {}

    def make(limit):
        def a(n, u):
            if limit is not None and len(live) >= limit:
                return 0
            p = alloc(n, u)
            if p:
                live[p] = n
            return p

        def f(p, u):
            live.pop(p)
            free(p, u)
        return a, f

    # the full context through PyTorch's pool: same result as cudaMalloc memory
    pz.pz_set_allocator(*make(None))
    try:
        s = pz.Synthesizer(prob)
        assert live, "the context took no memory from the caller's allocator"
        f1 = s.forward().cpu()
        s.close()
        assert not live, "buffers not handed back on destroy"
    finally:
        pz.pz_set_allocator()
    s = pz.Synthesizer(prob)
    f0 = s.forward().cpu()
    # the allocator cannot change while a context exists
    with pytest.raises(pz.PzError) as e:
        pz.pz_set_allocator(*make(None))
    assert e.value.status == pz.PZ_ESTATE
    s.close()
    assert torch.equal(f0, f1)
    # failure after a few allocations: PZ_ENOMEM from pz_create, nothing left behind
    for limit in (0, 3, 12):
        pz.pz_set_allocator(*make(limit))
        try:
            with pytest.raises(pz.PzError) as e:
                pz.Synthesizer(prob)
            assert e.value.status == pz.PZ_ENOMEM
            assert not live, (limit, len(live))
        finally:
            pz.pz_set_allocator()
