"""Pins of the oracle's transient companion stamp (CPU only).

The transient loop (Sec. II, Fig. 1) re-forms A x = b at every Newton iteration of every time
step; the device charges enter through a one-step integration rule. Checked here: the charge
Jacobian against central differences and charge conservation; the KCL identity A x - b =
F(x) + i_cap(x); reduction to the DC stamp at alpha = beta = 0; and a closed-form RC transient
(a gate held in deep subthreshold is a linear overlap capacitor) for backward Euler and the
trapezoidal rule.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import netgen
import oracle
from helpers import tiny_net

CARDS = netgen.default_cards()


def test_charge_jacobian_matches_central_differences_and_conserves_charge():
    rng = np.random.default_rng(7)
    h = 1e-6
    for p, card in ((1, CARDS[0]), (-1, CARDS[1])):
        for _ in range(30):
            V = rng.uniform(-0.1, 1.1, 4)
            if abs(V[0] - V[2]) < 1e-3:
                continue
            Q, C = oracle.device_charge(card, p, 2e-6, 0.5e-6, V)
            Cfd = np.zeros((4, 4))
            for u in range(4):
                Vp, Vm = V.copy(), V.copy()
                Vp[u] += h
                Vm[u] -= h
                Cfd[:, u] = (oracle.device_charge(card, p, 2e-6, 0.5e-6, Vp)[0]
                             - oracle.device_charge(card, p, 2e-6, 0.5e-6, Vm)[0]) / (2 * h)
            scale = np.abs(C).max()
            np.testing.assert_allclose(C, Cfd, rtol=1e-5, atol=1e-6 * scale)
            np.testing.assert_allclose(C.sum(axis=0), 0.0, atol=1e-14 * scale)


@pytest.mark.parametrize("net", [netgen.inverter_chain(12), netgen.ota5t(), netgen.sram(3, 4),
                                 netgen.random_logic(200, seed=2)], ids=lambda n: n.name)
def test_transient_stamp_satisfies_kcl_with_capacitive_currents(net):
    o = oracle.Oracle(net, CARDS)
    rng = np.random.default_rng(3)
    for alpha, beta in ((1e9, 0.0), (2e10, 1.0)):
        x = netgen.random_x(net, seed=4, lo=-0.1, hi=1.1)
        qprev = o.eval_stamp(netgen.random_x(net, seed=5), want_q=True)["q"]
        iprev = rng.normal(size=(4, net.n_dev)) * 1e-5
        r = o.eval_stamp_tran(x, qprev, iprev, alpha, beta, want_scale=True)
        rp, col, _ = o.pattern()
        A = sp.csr_matrix((r["A"], col, rp), shape=(o.n, o.n))
        As = sp.csr_matrix((r["A_scale"], col, rp), shape=(o.n, o.n))
        F = o.kcl_residual(x)
        unk = o.pattern()[2]
        for t in range(4):
            nodes = net.dev_nodes[:, t]
            m = unk[nodes] >= 0
            np.add.at(F, unk[nodes[m]], r["i"][t, m])
        np.testing.assert_allclose(r["i"], alpha * (r["q"] - qprev) - beta * iprev, rtol=1e-15,
                                   atol=1e-30)
        scale = abs(As) @ np.abs(x) + r["b_scale"]
        assert np.all(np.abs(A @ x - r["b"] - F) <= 1e-13 * scale + 1e-30)


def test_zero_integration_coefficients_reduce_to_the_dc_stamp():
    net = netgen.sram(4, 4)
    o = oracle.Oracle(net, CARDS)
    x = netgen.random_x(net, seed=1)
    dc = o.eval_stamp(x, want_q=True)
    tr = o.eval_stamp_tran(x, np.zeros((4, net.n_dev)), None, 0.0, 0.0)
    assert np.array_equal(tr["A"], dc["A"]) and np.array_equal(tr["b"], dc["b"])
    assert np.array_equal(tr["q"], dc["q"]) and not np.any(tr["i"])


@pytest.mark.parametrize("method", [0, 1])
def test_rc_step_response_follows_the_discrete_integrator(method):
    # Source V -> R -> gate of an NMOS (d = s = b = ground) whose threshold is far above the
    # gate swing: Qinv ~ e^-100 Cox W L, the depletion charge is constant (vbs = 0) and the gate
    # charge is the linear overlap charge (CGSO + CGDO) W Vg. No junction or leak currents.
    W, L, R, Vs = 4e-6, 1e-6, 5e3, 1.0
    card = netgen.card(VTH0=5.0, JS=0.0, GMIN=0.0)
    net = tiny_net("rc", [1, 1, 0], [0, Vs, 0], [(0, 2, 0, 0)], [1], W=[W], L=[L],
                   res=[(1, 2)], resG=[1 / R], gshunt=0.0)
    o = oracle.Oracle(net, np.stack([card, card]))
    C = (card[netgen.CARD_FIELDS.index("CGSO")] + card[netgen.CARD_FIELDS.index("CGDO")]) * W
    tau = R * C
    h = tau / 7.0
    n = 40
    traj = o.tran_solve(np.zeros(1), h, n, method=method)
    v = np.zeros(n + 1)
    i_cap = 0.0
    for k in range(n):   # the textbook one-step rules for C dv/dt = (Vs - v)/R
        if method == 0:
            v[k + 1] = (C / h * v[k] + Vs / R) / (C / h + 1 / R)
        else:
            v[k + 1] = (2 * C / h * v[k] + i_cap + Vs / R) / (2 * C / h + 1 / R)
            i_cap = 2 * C / h * (v[k + 1] - v[k]) - i_cap
    np.testing.assert_allclose(traj[:, 0], v, rtol=1e-9, atol=1e-12)
    if method == 0:
        rho = 1 / (1 + h / tau)
        np.testing.assert_allclose(v, Vs * (1 - rho ** np.arange(n + 1)), rtol=1e-12, atol=1e-15)
