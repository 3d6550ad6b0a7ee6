"""Row-block partitions of one netlist, the multi-GPU design for a netlist larger than one GPU:
each rank owns a block of free nodes (rows), evaluates every device touching an owned row after
a halo exchange of the other voltages those devices see, and stamps only its owned rows. Here
the ranks are emulated one after another (no kernels wait on one another): the owned rows of
every part must equal the monolithic rows exactly, and together the parts cover every row.

CPU: the oracle (which sums each entry in element order: the parts keep that order for their
owned rows). GPU: the library's deterministic segmented reduction (original-device order)."""
import numpy as np
import pytest

import netgen
import oracle

CARDS = netgen.default_cards()
NETS = [(lambda: netgen.sram(6, 8), 3), (lambda: netgen.random_logic(600, seed=3), 4),
        (lambda: netgen.inverter_chain(40), 2), (lambda: netgen.ota5t(), 2)]


def _rows_equal(rp, col, A, b, prp, pcol, pA, pb, rows):
    for u in rows:
        a0, a1 = rp[u], rp[u + 1]
        p0, p1 = prp[u], prp[u + 1]
        assert np.array_equal(col[a0:a1], pcol[p0:p1]), u
        assert np.array_equal(A[a0:a1], pA[p0:p1]), u
        assert b[u] == pb[u], u


@pytest.mark.parametrize("make,k", NETS, ids=lambda v: getattr(v, "__name__", str(v)))
def test_oracle_partitions_reassemble_the_monolithic_system(make, k):
    net = make()
    x = netgen.random_x(net, seed=4, lo=-0.1, hi=1.1)
    o = oracle.Oracle(net, CARDS)
    ref = o.eval_stamp(x)
    rp, col, unk = o.pattern()
    covered = np.zeros(o.n, bool)
    parts = netgen.partition_rows(net, k)
    assert sum(p.n_dev for p, _ in parts) >= net.n_dev   # cut devices are evaluated twice
    for sub, owned in parts:
        op = oracle.Oracle(sub, CARDS)
        r = op.eval_stamp(x)
        prp, pcol, punk = op.pattern()
        assert np.array_equal(punk, unk)                  # the unknowns keep their numbering
        rows = unk[owned]
        _rows_equal(rp, col, ref["A"], ref["b"], prp, pcol, r["A"], r["b"], rows)
        assert not covered[rows].any()
        covered[rows] = True
    assert covered.all()


@pytest.mark.gpu
@pytest.mark.parametrize("make,k", NETS, ids=lambda v: getattr(v, "__name__", str(v)))
def test_gpu_partitions_reassemble_the_monolithic_system(make, k):
    import torch
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as eec
    net = make()
    x = netgen.random_x(net, seed=4, lo=-0.1, hi=1.1)
    xt = torch.as_tensor(x, device="cuda")
    whole = eec.Circuit(net, CARDS, color=False, variant=eec.EEC_VARIANT_SEGREDUCE)
    A, b, _ = whole.eval_stamp(xt)
    A, b = A.cpu().numpy(), b.cpu().numpy()
    rp, col, unk = whole.pattern()
    covered = np.zeros(whole.n, bool)
    for sub, owned in netgen.partition_rows(net, k):
        part = eec.Circuit(sub, CARDS, color=False, variant=eec.EEC_VARIANT_SEGREDUCE)
        pA, pb, _ = part.eval_stamp(xt)
        prp, pcol, punk = part.pattern()
        assert np.array_equal(punk, unk)
        rows = unk[owned]
        _rows_equal(rp, col, A, b, prp, pcol, pA.cpu().numpy(), pb.cpu().numpy(), rows)
        covered[rows] = True
        assert part.status() == 0
    assert covered.all()
