"""GPU parity under modified nodal analysis of the rails (rail_mode 1): the rails are unknowns and
every held node adds its source current. The CUDA path (every schedule, the backward, the host-
buffer entry point and the DC Newton loop) against the oracle in the same mode, with the
tolerances of the eliminated form (per entry 1e-12 of max(|oracle|, sum of |contributions|))."""
import numpy as np
import pytest

import netgen
import oracle
from helpers import rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-12
CARDS = netgen.default_cards()
MNA = 1


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def rails(net):
    return [i for i in range(1, net.n_nodes) if net.node_fixed[i]]


def mna_x(net, n, seed):
    """Node voltages ~ U[0, 1] on every non-ground node, source currents ~ 1e-4 N(0, 1)."""
    x = np.empty(n)
    x[: net.n_nodes - 1] = netgen.Rng(seed, 8).uniform(net.n_nodes - 1)
    x[net.n_nodes - 1:] = 1e-4 * netgen.Rng(seed, 9).normal(n - net.n_nodes + 1)
    return x


NETS = [netgen.ota5t, lambda: netgen.sram(8, 8), lambda: netgen.ripple_adder(4, seed=2),
        lambda: netgen.inverter_chain(48, vin=0.3), lambda: netgen.random_logic(600, seed=4)]


@pytest.mark.parametrize("make", NETS)
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_eval_stamp_matches_oracle_under_mna(eec, make, variant):
    net = make()
    o = oracle.Oracle(net, CARDS, rail_mode=MNA)
    circ = eec.Circuit(net, CARDS, variant=variant, rail_mode=eec.EEC_RAIL_MNA_BRANCH)
    assert circ.n == o.n == net.n_nodes - 1 + len(rails(net))
    x = mna_x(net, circ.n, seed=3)
    A, b, q = circ.eval_stamp(dev(x))
    assert circ.status() == 0
    r = o.eval_stamp(x, want_q=True, want_scale=True)
    eA = rel_err(A.cpu().numpy(), r["A"], r["A_scale"])
    eb = rel_err(b.cpu().numpy(), r["b"], r["b_scale"])
    assert eA.max() <= TOL, (eA.max(), int(eA.argmax()))
    assert eb.max() <= TOL, (eb.max(), int(eb.argmax()))
    qg = q.cpu().numpy().reshape(4, -1)
    scale = np.maximum(np.abs(r["q"]).max(axis=0, keepdims=True), 1e-300)
    assert (np.abs(qg - r["q"]) / scale).max() <= 1e-13


def test_colours_and_host_buffers_under_mna(eec):
    import torch
    net = netgen.ripple_adder(8, seed=1)
    o = oracle.Oracle(net, CARDS, rail_mode=MNA)
    ocol, oC = o.color_greedy(rule=0)
    assert oC == int(np.count_nonzero(net.dev_type < 0))    # one colour per PMOS (VDD clique)
    circ = eec.Circuit(net, CARDS, variant=eec.EEC_VARIANT_ATOMIC,
                       rail_mode=eec.EEC_RAIL_MNA_BRANCH)
    assert circ.n_colors == oC and np.array_equal(circ.colors, ocol)
    x = mna_x(net, circ.n, seed=8)
    hA = torch.empty(circ.nnz, dtype=torch.float64).pin_memory()
    hb = torch.empty(circ.n, dtype=torch.float64).pin_memory()
    hx = torch.as_tensor(x).pin_memory()
    eec.eec_eval_stamp_host(circ.ctx, hx, hA, hb, None)
    torch.cuda.synchronize()
    r = o.eval_stamp(x, want_scale=True)
    assert rel_err(hA.numpy(), r["A"], r["A_scale"]).max() <= TOL
    assert rel_err(hb.numpy(), r["b"], r["b_scale"]).max() <= TOL


@pytest.mark.parametrize("make", [lambda: netgen.sram(8, 8), netgen.ota5t])
def test_backward_matches_oracle_under_mna(eec, make):
    net = make()
    o = oracle.Oracle(net, CARDS, rail_mode=MNA)
    circ = eec.Circuit(net, CARDS, rail_mode=eec.EEC_RAIL_MNA_BRANCH)
    x = mna_x(net, circ.n, seed=4)
    rng = netgen.Rng(12, 3)
    gA, gb = rng.normal(circ.nnz), rng.normal(circ.n)
    got = circ.bwd(dev(x), dev(gA), dev(gb))
    ref = o.eval_stamp_grad(x, gA, gb)
    for g, r in zip(got, ref):
        g = g.cpu().numpy()
        floor = 1e-6 * max(np.abs(r).max(), 1e-300)
        assert (np.abs(g - r) / np.maximum(np.abs(r), floor)).max() <= 1e-8
    # source currents enter A and b only through the constant linear part
    assert np.all(got[0].cpu().numpy()[net.n_nodes - 1:] == 0.0)


@pytest.mark.parametrize("make", [netgen.ota5t, lambda: netgen.ring_oscillator(11),
                                  lambda: netgen.ripple_adder(4)])
def test_gpu_newton_under_mna_reaches_the_oracle_operating_point(eec, make):
    import torch
    net = make()
    o = oracle.Oracle(net, CARDS, rail_mode=MNA)
    R = rails(net)
    x0 = np.zeros(o.n)
    x0[np.array(R) - 1] = net.node_vfix[R]          # start with the rails at their sources
    ref, _ = o.dc_solve(x0=x0)
    circ = eec.Circuit(net, CARDS, variant=eec.EEC_VARIANT_ATOMIC,
                       rail_mode=eec.EEC_RAIL_MNA_BRANCH)
    x = dev(x0)
    A, b, _ = circ.new_outputs(want_q=False)
    it = eec.eec_newton_dc(circ.ctx, x, A, b)
    assert 1 <= it <= 200
    assert circ.status() == 0
    xh = x.cpu().numpy()
    nv = net.n_nodes - 1
    np.testing.assert_allclose(xh[:nv], ref[:nv], rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(xh[nv:], ref[nv:], rtol=1e-6, atol=1e-15)
    np.testing.assert_allclose(xh[np.array(R) - 1], net.node_vfix[R], rtol=1e-14, atol=1e-15)
    # the node voltages are the eliminated form's operating point
    oe = oracle.Oracle(net, CARDS)
    xe, _ = oe.dc_solve()
    _, _, ue = oe.pattern()
    free = np.nonzero(ue >= 0)[0]
    np.testing.assert_allclose(xh[free - 1], xe[ue[free]], rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("variant", [0, 2, 4, 5])
@pytest.mark.parametrize("make", [netgen.ota5t, lambda: netgen.sram(8, 8)])
def test_transient_stamp_under_mna(eec, variant, make):
    import torch
    net = make()
    o = oracle.Oracle(net, CARDS, rail_mode=MNA)
    circ = eec.Circuit(net, CARDS, variant=variant, rail_mode=eec.EEC_RAIL_MNA_BRANCH)
    x = mna_x(net, circ.n, seed=5)
    qprev = o.eval_stamp(mna_x(net, circ.n, seed=6), want_q=True)["q"]
    iprev = 1e-5 * np.random.default_rng(4).normal(size=(4, net.n_dev))
    A, b, q = circ.new_outputs(want_q=True)
    i = torch.empty_like(q)
    eec.eec_eval_stamp_tran(circ.ctx, dev(x), dev(qprev.reshape(-1)), dev(iprev.reshape(-1)),
                            2e11, 1.0, A, b, q, i)
    assert circ.status() == 0
    r = o.eval_stamp_tran(x, qprev, iprev, 2e11, 1.0, want_scale=True)
    assert rel_err(A.cpu().numpy(), r["A"], r["A_scale"]).max() <= TOL
    assert rel_err(b.cpu().numpy(), r["b"], r["b_scale"]).max() <= TOL
