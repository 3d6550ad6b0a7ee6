"""Pins of the oracle's error scales (CPU only).

Every GPU parity check divides |gpu - oracle| by max(|oracle|, S_e), where S_e is the sum of the
sizes of the contributions to the entry, accumulated by the oracle in shadow arrays. A scale that
is too large would silently loosen every parity check, so the scales are pinned here:
  * S_e bounds the entry it belongs to (|sum| <= sum of |terms|), for the DC and the transient
    stamp, at ordinary and at wide bias;
  * on a one-device circuit every S_e equals a sum written out by hand from the device's own
    currents, conductances, charges and capacitances and the linear elements on that entry;
  * at zero integration coefficients the transient scales are the DC scales, bit for bit.
In the transient stamp a device adds three stamps to A[t][u]: its conductance G_tu, its
intrinsic charge capacitance alpha C^int_tu and its overlap capacitance alpha C^ov_tu; each is
one contribution, so the intrinsic/overlap cancellation of the gate row (C_gd, C_gs near zero in
saturation) is judged against the size of the two capacitances, not against their small sum.
"""
import numpy as np
import pytest

import netgen
import oracle
from helpers import tiny_net

CARDS = netgen.default_cards()
EPS = np.finfo(float).eps


def _bounded(val, scale):
    # |sum of terms| <= sum of |terms|; the two sums round differently, by a few ulp of the scale
    assert np.all(np.abs(val) <= scale * (1 + 64 * EPS) + 1e-300)


@pytest.mark.parametrize("make", [lambda: netgen.inverter_chain(16), netgen.ota5t,
                                  lambda: netgen.sram(4, 5), lambda: netgen.random_logic(300, seed=3),
                                  lambda: netgen.ripple_adder(2)], ids=["chain", "ota", "sram", "logic", "adder"])
@pytest.mark.parametrize("lo,hi", [(0.0, 1.0), (-3.0, 4.0)])
def test_scales_bound_their_entries(make, lo, hi):
    net = make()
    o = oracle.Oracle(net, CARDS)
    x = netgen.random_x(net, seed=2, lo=lo, hi=hi)
    r = o.eval_stamp(x, want_scale=True)
    _bounded(r["A"], r["A_scale"])
    _bounded(r["b"], r["b_scale"])
    qprev = o.eval_stamp(netgen.random_x(net, seed=3), want_q=True)["q"]
    iprev = np.random.default_rng(4).normal(size=(4, net.n_dev)) * 1e-5
    for alpha, beta in ((1e9, 0.0), (2e11, 1.0)):
        t = o.eval_stamp_tran(x, qprev, iprev, alpha, beta, want_scale=True)
        _bounded(t["A"], t["A_scale"])
        _bounded(t["b"], t["b_scale"])


def _one_device():
    # node 0 ground, node 1 a 1 V rail; the NMOS's d, g, s, b on free nodes 2..5, each with a
    # resistor (d to the rail, the others to ground)
    G = [1e-3, 1e-4, 2e-4, 3e-4]
    net = tiny_net("one", [1, 1, 0, 0, 0, 0], [0, 1.0, 0, 0, 0, 0], [(2, 3, 4, 5)], [1],
                   W=[3e-6], L=[0.4e-6], res=[(1, 2), (3, 0), (4, 0), (5, 0)], resG=G)
    return net, np.array(G)


def _pos(o):
    rp, col, _ = o.pattern()
    pos = {}
    for i in range(o.n):
        for p in range(rp[i], rp[i + 1]):
            pos[(i, int(col[p]))] = p
    return pos


def test_one_device_dc_scales_are_the_hand_sums():
    net, Gres = _one_device()
    o = oracle.Oracle(net, CARDS)
    x = np.array([0.9, 0.7, 0.1, 0.05])        # unknowns are nodes 2..5 = d, g, s, b
    r = o.eval_stamp(x, want_scale=True)
    I, Gd, _ = oracle.device_eval(CARDS[0], 1, 3e-6, 0.4e-6, x)
    pos = _pos(o)
    As = np.zeros(o.nnz)
    bs = np.zeros(o.n)
    for t in range(4):
        As[pos[(t, t)]] += net.gshunt + Gres[t]
    bs[0] += Gres[0] * 1.0                      # the drain resistor's rail current into b
    for t in (0, 2, 3):                          # DC: rows d, s, b (no gate current)
        for u in range(4):
            As[pos[(t, u)]] += abs(Gd[t, u])
        bs[t] += abs(I[t]) + sum(abs(Gd[t, u]) * abs(x[u]) for u in range(4))
    np.testing.assert_allclose(r["A_scale"], As, rtol=4 * EPS, atol=0)
    np.testing.assert_allclose(r["b_scale"], bs, rtol=4 * EPS, atol=0)


def test_one_device_transient_scales_are_the_hand_sums():
    net, Gres = _one_device()
    o = oracle.Oracle(net, CARDS)
    x = np.array([0.9, 0.7, 0.1, 0.05])
    W = 3e-6
    qprev = np.array([[1e-16], [-3e-16], [2e-16], [5e-17]])
    iprev = np.array([[1e-6], [-2e-6], [4e-7], [3e-7]])
    alpha, beta = 2e11, 1.0
    r = o.eval_stamp_tran(x, qprev, iprev, alpha, beta, want_scale=True)
    I, Gd, _ = oracle.device_eval(CARDS[0], 1, W, 0.4e-6, x)
    Q, C = oracle.device_charge(CARDS[0], 1, W, 0.4e-6, x)
    # overlap capacitances from the overlap charges CGSO W (Vg - Vs) into g (minus into s) and
    # CGDO W (Vg - Vd) into g (minus into d)
    f = netgen.CARD_FIELDS
    cs, cd = CARDS[0][f.index("CGSO")] * W, CARDS[0][f.index("CGDO")] * W
    Cov = np.zeros((4, 4))
    Cov[1, 1], Cov[1, 0], Cov[1, 2] = cs + cd, -cd, -cs
    Cov[0, 0], Cov[0, 1] = cd, -cd
    Cov[2, 2], Cov[2, 1] = cs, -cs
    pos = _pos(o)
    As = np.zeros(o.nnz)
    bs = np.zeros(o.n)
    for t in range(4):
        As[pos[(t, t)]] += net.gshunt + Gres[t]
    bs[0] += Gres[0] * 1.0
    for t in range(4):                          # all four rows, gate row included
        size = np.abs(Gd[t]) + alpha * np.abs(C[t] - Cov[t]) + alpha * np.abs(Cov[t])
        for u in range(4):
            As[pos[(t, u)]] += size[u]
        bs[t] += (abs(I[t]) + alpha * (abs(Q[t]) + abs(qprev[t, 0])) + beta * abs(iprev[t, 0])
                  + float(size @ np.abs(x)))
    np.testing.assert_allclose(r["A_scale"], As, rtol=8 * EPS, atol=0)
    np.testing.assert_allclose(r["b_scale"], bs, rtol=8 * EPS, atol=0)
    # the gate-drain entry: its intrinsic and overlap parts are counted apart
    gd = pos[(1, 0)]
    assert r["A_scale"][gd] >= alpha * abs(Cov[1, 0])


@pytest.mark.parametrize("make", [lambda: netgen.sram(3, 3), netgen.ota5t])
def test_transient_scales_at_zero_coefficients_are_the_dc_scales(make):
    net = make()
    o = oracle.Oracle(net, CARDS)
    x = netgen.random_x(net, seed=6)
    dc = o.eval_stamp(x, want_scale=True)
    tr = o.eval_stamp_tran(x, np.zeros((4, net.n_dev)), None, 0.0, 0.0, want_scale=True)
    assert np.array_equal(tr["A_scale"], dc["A_scale"])
    assert np.array_equal(tr["b_scale"], dc["b_scale"])
