"""Circuit-level pins of the oracle (CPU only): closed-form DC solutions, the KCL identity of the
stamp, the MNA pattern, the Newton loop, and the gradient/adjoint against finite differences."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.special import lambertw

import netgen
import oracle
from helpers import tiny_net

KB, QE = 1.380649e-23, 1.602176634e-19
VT = KB * 300.15 / QE
CARDS = netgen.default_cards()


def csr(o, A):
    rp, col, _ = o.pattern()
    return sp.csr_matrix((A, col, rp), shape=(o.n, o.n))


def test_resistor_divider_closed_form():
    G1, G2, vdd, gs = 1e-3, 3e-3, 1.0, 1e-12
    net = tiny_net("div", [1, 1, 0], [0, vdd, 0], np.zeros((0, 4)), [], res=[(1, 2), (2, 0)],
                   resG=[G1, G2], gshunt=gs)
    o = oracle.Oracle(net, CARDS)
    x, it = o.dc_solve()
    assert o.n == 1
    np.testing.assert_allclose(x[0], G1 * vdd / (G1 + G2 + gs), rtol=1e-14)


def test_current_source_closed_form():
    G, I = 2e-3, 1.5e-4
    net = tiny_net("isrc", [1, 0], [0, 0], np.zeros((0, 4)), [], res=[(1, 0)], resG=[G],
                   isrc=[(0, 1)], ival=[I], gshunt=0.0)
    o = oracle.Oracle(net, CARDS)
    x, _ = o.dc_solve()
    np.testing.assert_allclose(x[0], I / G, rtol=1e-14)


@pytest.mark.parametrize("vsrc,R", [(1.0, 1e3), (0.8, 1e4), (3.0, 100.0)])
def test_diode_resistor_lambert_w(vsrc, R):
    # NMOS with d = g = s = ground and body on node B: no channel current (vds = 0), the two
    # body junctions form one diode of saturation current 2 JS W HDIF from B to ground.
    W = 3e-6
    card = netgen.card(GMIN=0.0)
    cards = np.stack([card, card])
    net = tiny_net("diode", [1, 1, 0], [0, vsrc, 0], [(0, 0, 0, 2)], [1], W=[W], L=[1e-6],
                   res=[(1, 2)], resG=[1 / R], gshunt=0.0)
    o = oracle.Oracle(net, cards)
    x, _ = o.dc_solve(x0=np.array([0.0]))
    Is = 2 * 1e-4 * W * 2e-7
    arg = (Is * R / VT) * math.exp((vsrc + Is * R) / VT)
    Iexact = (VT / R) * lambertw(arg).real - Is
    np.testing.assert_allclose(x[0], vsrc - Iexact * R, rtol=1e-10)


def _kcl_cases():
    yield netgen.inverter_chain(16)
    yield netgen.ring_oscillator(11)
    yield netgen.ota5t()
    yield netgen.sram(4, 5)
    yield netgen.random_logic(300, seed=7)
    yield netgen.concat(netgen.batch_circuits(6, seed=11))


@pytest.mark.parametrize("net", list(_kcl_cases()), ids=lambda n: n.name)
def test_stamp_satisfies_kcl_identity(net):
    # A x_k - b = F(x_k): the linearised system reproduces the full KCL residual at x_k.
    o = oracle.Oracle(net, CARDS)
    for s in range(3):
        x = netgen.random_x(net, seed=100 + s, lo=-0.1, hi=1.1)
        r = o.eval_stamp(x, want_scale=True)
        A = csr(o, r["A"])
        F = o.kcl_residual(x)
        lhs = A @ x - r["b"]
        scale = abs(csr(o, r["A_scale"])) @ np.abs(x) + r["b_scale"]
        assert np.all(np.abs(lhs - F) <= 1e-13 * scale + 1e-30)


@pytest.mark.parametrize("net", list(_kcl_cases()), ids=lambda n: n.name)
def test_pattern_is_symmetric_with_full_diagonal(net):
    o = oracle.Oracle(net, CARDS)
    rp, col, unk = o.pattern()
    S = sp.csr_matrix((np.ones_like(col, dtype=float), col, rp), shape=(o.n, o.n))
    assert (S != S.T).nnz == 0
    assert np.all(S.diagonal() == 1)
    for i in range(o.n):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    free = np.nonzero(net.node_fixed == 0)[0]
    assert np.array_equal(unk[free], np.arange(len(free)))
    assert np.all(unk[net.node_fixed == 1] == -1)


def test_inverter_chain_pattern_count():
    # 64 free outputs; stage 0 (input fixed) touches only out_0, every later stage couples
    # out_i with out_{i-1}: 64 diagonal + 2 * 63 off-diagonal entries.
    o = oracle.Oracle(netgen.inverter_chain(64), CARDS)
    assert o.n == 64 and o.nnz == 64 + 2 * 63


def test_newton_inverter_chain_logic_levels():
    net = netgen.inverter_chain(64, vin=0.0)
    o = oracle.Oracle(net, CARDS)
    x, it, hist = o.dc_solve(history=True)
    assert it < 200
    assert np.all(x[0::2] > 0.99) and np.all(x[1::2] < 0.01)
    assert np.abs(o.kcl_residual(x)).max() <= 1e-12
    assert np.array_equal(hist[-1], x)
    # Each iterate of the history reproduces the next Newton step.
    r = o.eval_stamp(hist[3])
    y = sp.linalg.spsolve(csr(o, r["A"]).tocsc(), r["b"])
    d = y - hist[3]
    m = np.abs(d).max()
    if m > 0.2:
        d *= 0.2 / m
    np.testing.assert_allclose(hist[4], hist[3] + d, rtol=1e-9, atol=1e-12)


def _stamp_functional(o, x, gA, gb):
    r = o.eval_stamp(x)
    return float(gA @ r["A"] + gb @ r["b"])


@pytest.mark.parametrize("net", [netgen.inverter_chain(6, vin=0.3), netgen.ota5t(),
                                 netgen.sram(2, 2), netgen.random_logic(40, seed=3)],
                         ids=lambda n: n.name)
def test_eval_stamp_gradient_matches_central_differences(net):
    o = oracle.Oracle(net, CARDS)
    rng = netgen.Rng(5, 9)
    x = netgen.random_x(net, seed=21, lo=0.05, hi=0.95)
    gA = rng.normal(o.nnz)
    gb = rng.normal(o.n)
    gx, gW, gL = o.eval_stamp_grad(x, gA, gb)
    h = 1e-6
    for i in range(min(o.n, 8)):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (_stamp_functional(o, xp, gA, gb) - _stamp_functional(o, xm, gA, gb)) / (2 * h)
        np.testing.assert_allclose(gx[i], fd, rtol=2e-5, atol=1e-9 * max(1.0, abs(gx).max()))
    W0, L0 = net.W.copy(), net.L.copy()
    for k in range(min(net.n_dev, 6)):
        for arr, g in ((W0, gW), (L0, gL)):
            hp = 1e-6 * arr[k]
            a1, a2 = arr.copy(), arr.copy()
            a1[k] += hp
            a2[k] -= hp
            if arr is W0:
                o.set_sizes(a1, L0); fp = _stamp_functional(o, x, gA, gb)
                o.set_sizes(a2, L0); fm = _stamp_functional(o, x, gA, gb)
            else:
                o.set_sizes(W0, a1); fp = _stamp_functional(o, x, gA, gb)
                o.set_sizes(W0, a2); fm = _stamp_functional(o, x, gA, gb)
            o.set_sizes(W0, L0)
            fd = (fp - fm) / (2 * hp)
            np.testing.assert_allclose(g[k], fd, rtol=2e-5, atol=1e-9 * abs(g).max())


def test_adjoint_sensitivity_matches_finite_difference_of_dc_solves():
    # dV_out/dtheta = -lambda^T dF/dtheta with A^T lambda = e_out, and the stamp gradient with
    # gA_ij = lambda_i x_j, gb = -lambda equals lambda^T dF/dtheta.
    net = netgen.inverter_chain(4, vin=0.45)
    o = oracle.Oracle(net, CARDS)
    x, _ = o.dc_solve()
    out = 0                       # first stage output sits mid-rail (about 0.66 V): sensitive
    assert 0.3 < x[out] < 0.9
    lam = o.adjoint(x, out)
    rp, col, _ = o.pattern()
    rows = np.repeat(np.arange(o.n), np.diff(rp))
    gA = lam[rows] * x[col]
    gb = -lam
    _, gW, gL = o.eval_stamp_grad(x, gA, gb)
    W0, L0 = net.W.copy(), net.L.copy()
    gmax = max(np.abs(gW).max() * W0.max(), np.abs(gL).max() * L0.max())
    for k in range(net.n_dev):
        for which in ("W", "L"):
            base = W0 if which == "W" else L0
            h = 1e-6 * base[k]
            vals = []
            for sgn in (1, -1):
                a = base.copy()
                a[k] += sgn * h
                o.set_sizes(a, L0) if which == "W" else o.set_sizes(W0, a)
                xs, _ = o.dc_solve(x0=x)
                vals.append(xs[out])
            o.set_sizes(W0, L0)
            fd = (vals[0] - vals[1]) / (2 * h)
            g = -(gW if which == "W" else gL)[k]
            # compare relative sensitivities theta * dV/dtheta (volts)
            np.testing.assert_allclose(g * base[k], fd * base[k], rtol=1e-5, atol=1e-7 * gmax)
