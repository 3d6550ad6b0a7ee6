"""The no-allocation backward entry point (eec_eval_stamp_bwd_noalloc).

It serves callers that cannot allocate device memory (their GPU memory is reserved by their own
allocator, or a cudaMalloc's synchronisation is unacceptable in their loop). It must give the
same gradients as the allocating eec_eval_stamp_bwd, through the C ABI, on consecutive calls that
share the library's fixed scratch array, and refuse contexts larger than that array. This file
is collected last so that a run stopping at the first failure has run every other test first.
"""
import os

import numpy as np
import pytest

import netgen

pytestmark = pytest.mark.gpu
TOL = 1e-8   # the gradient tolerance of the GPU parity tests


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def _grads(eec, circ, fn, x, gA, gb):
    import torch
    gx = torch.full((circ.n,), float("nan"), dtype=torch.float64, device="cuda")
    gW = torch.full((circ.n_dev,), float("nan"), dtype=torch.float64, device="cuda")
    gL = torch.full((circ.n_dev,), float("nan"), dtype=torch.float64, device="cuda")
    fn(circ.ctx, x, gA, gb, gx, gW, gL)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (gx, gW, gL)]


def _close(got, ref):
    floor = 1e-6 * max(np.abs(ref).max(), 1e-300)
    return (np.abs(got - ref) / np.maximum(np.abs(ref), floor)).max() <= TOL


def test_noalloc_backward_matches_allocating_backward_on_consecutive_calls(eec):
    import torch
    cards = netgen.default_cards()
    nets = [netgen.sram(64, 64), netgen.random_logic(5000, seed=3)]
    circs = [eec.Circuit(net, cards) for net in nets]
    for call in range(2):
        for net, circ in zip(nets, circs):
            rng = netgen.Rng(100 + call, 7)
            x = torch.as_tensor(netgen.random_x(net, seed=call), device="cuda")
            gA = torch.as_tensor(rng.normal(circ.nnz), device="cuda")
            gb = torch.as_tensor(rng.normal(circ.n), device="cuda")
            ref = _grads(eec, circ, eec.eec_eval_stamp_bwd, x, gA, gb)
            got = _grads(eec, circ, eec.eec_eval_stamp_bwd_noalloc, x, gA, gb)
            for g, r in zip(got, ref):
                assert np.all(np.isfinite(g))
                assert _close(g, r)


def test_noalloc_backward_on_a_fresh_context_allocates_nothing(eec):
    # A fresh context: the no-allocation entry point runs first, so the allocating backward has
    # never created its own scratch. Device memory is the same before and after a further call.
    import torch
    cards = netgen.default_cards()
    net = netgen.random_logic(4000, seed=5)
    circ = eec.Circuit(net, cards)
    rng = netgen.Rng(300, 7)
    x = torch.as_tensor(netgen.random_x(net, seed=9), device="cuda")
    gA = torch.as_tensor(rng.normal(circ.nnz), device="cuda")
    gb = torch.as_tensor(rng.normal(circ.n), device="cuda")
    outs = [torch.empty(k, dtype=torch.float64, device="cuda") for k in (circ.n, circ.n_dev, circ.n_dev)]
    eec.eec_eval_stamp_bwd_noalloc(circ.ctx, x, gA, gb, *outs)
    torch.cuda.synchronize()
    first = [t.cpu().numpy() for t in outs]
    free0, _ = torch.cuda.mem_get_info()
    eec.eec_eval_stamp_bwd_noalloc(circ.ctx, x, gA, gb, *outs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    second = [t.cpu().numpy() for t in outs]
    ref = _grads(eec, circ, eec.eec_eval_stamp_bwd, x, gA, gb)
    for a, b, r in zip(first, second, ref):
        assert np.array_equal(a, b)
        assert np.all(np.isfinite(a)) and _close(a, r)


def test_noalloc_backward_rejects_contexts_beyond_the_fixed_scratch(eec):
    import torch
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "eec.h")).read()
    limit = int(re.search(r"#define\s+EEC_NOALLOC_MAX_DEV\s+(\d+)", hdr).group(1))
    assert limit == eec.EEC_NOALLOC_MAX_DEV
    net = netgen.random_logic(200_000)
    assert net.n_dev > limit
    circ = eec.Circuit(net, netgen.default_cards(), color=False)
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    gA = torch.zeros(circ.nnz, dtype=torch.float64, device="cuda")
    gb = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    with pytest.raises(eec.EECError) as e:
        _grads(eec, circ, eec.eec_eval_stamp_bwd_noalloc, x, gA, gb)
    assert e.value.code == eec.EEC_EINVAL and "EEC_NOALLOC_MAX_DEV" in str(e.value)
