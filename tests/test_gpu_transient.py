"""GPU parity of the transient companion stamp (eec_eval_stamp_tran) against the oracle, and a
transient loop whose every Newton iteration is stamped on the GPU against the oracle's own
transient solver. A and b: 1e-12 per entry relative to max(|oracle|, S_e), where S_e is the sum
of the sizes of the contributions to the entry: per device its conductance |G_tu|, its intrinsic
charge capacitance alpha |C^int_tu| and its overlap capacitance alpha |C^ov_tu| (three stamps),
and for b also |I_t|, the sizes of the capacitive-current terms and each stamp's size times
|x_u|; the linear elements as in the DC stamp."""
import numpy as np
import pytest

import netgen
import oracle
from helpers import rel_err, tiny_net

pytestmark = pytest.mark.gpu
TOL = 1e-12
CARDS = netgen.default_cards()


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64).reshape(-1), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def tran_gpu(eec, circ, x, qprev, iprev, alpha, beta):
    import torch
    A, b, q = circ.new_outputs(want_q=True)
    i = torch.empty_like(q)
    eec.eec_eval_stamp_tran(circ.ctx, dev(x), dev(qprev), None if iprev is None else dev(iprev),
                            alpha, beta, A, b, q, i)
    assert circ.status() == 0
    return host(A), host(b), host(q).reshape(4, -1), host(i).reshape(4, -1)


def check(eec, circ, o, x, qprev, iprev, alpha, beta):
    A, b, q, i = tran_gpu(eec, circ, x, qprev, iprev, alpha, beta)
    r = o.eval_stamp_tran(x, qprev, iprev, alpha, beta, want_scale=True)
    assert rel_err(A, r["A"], r["A_scale"]).max() <= TOL
    assert rel_err(b, r["b"], r["b_scale"]).max() <= TOL
    qs = np.maximum(np.abs(r["q"]).max(axis=0, keepdims=True), 1e-300)
    assert (np.abs(q - r["q"]) / qs).max() <= 1e-13
    iscale = alpha * (np.abs(r["q"]) + np.abs(qprev)) + (0 if iprev is None else beta * np.abs(iprev))
    assert (np.abs(i - r["i"]) / np.maximum(iscale, 1e-300)).max() <= 1e-13


@pytest.mark.parametrize("variant", [0, 2, 4, 5])
@pytest.mark.parametrize("make", [lambda: netgen.inverter_chain(64), netgen.ota5t,
                                  lambda: netgen.sram(32, 32), lambda: netgen.random_logic(4000, seed=9)])
def test_transient_stamp_matches_oracle(eec, variant, make):
    net = make()
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, color=True, variant=variant)
    rng = np.random.default_rng(11)
    for alpha, beta in ((1e9, 0.0), (2e11, 1.0), (0.0, 0.0)):
        x = netgen.random_x(net, seed=3, lo=-0.1, hi=1.1)
        qprev = o.eval_stamp(netgen.random_x(net, seed=4), want_q=True)["q"]
        iprev = rng.normal(size=(4, net.n_dev)) * 1e-5 if beta else None
        check(eec, circ, o, x, qprev, iprev, alpha, beta)


def test_transient_stamp_full_size_sram(eec):
    net = netgen.config(2)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, color=True)
    x = netgen.random_x(net)
    qprev = o.eval_stamp(netgen.random_x(net, seed=77), want_q=True)["q"]
    iprev = np.random.default_rng(2).normal(size=(4, net.n_dev)) * 1e-5
    for variant in (0, 2, 4, 5):
        eec.eec_set_variant(circ.ctx, variant)
        check(eec, circ, o, x, qprev, iprev, 4e10, 1.0)


def _gpu_transient(eec, net, cards, h, n, method, variant):
    """Transient by the oracle's rules (Newton with 0.2 V per-node step limits, same
    tolerances), every A, b from the GPU; the small dense solve runs in torch on the GPU."""
    import torch
    circ = eec.Circuit(net, cards, color=True, variant=variant)
    rp, col, _ = circ.pattern()
    rows = torch.as_tensor(np.repeat(np.arange(circ.n), np.diff(rp)), device="cuda")
    cols = torch.as_tensor(col.astype(np.int64), device="cuda")
    alpha, beta = (1.0 / h, 0.0) if method == 0 else (2.0 / h, 1.0)
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    A, b, q = circ.new_outputs(want_q=True)
    ic = torch.empty_like(q)
    qprev = torch.zeros_like(q)
    iprev = torch.zeros_like(q)
    eec.eec_eval_stamp_tran(circ.ctx, x, qprev, iprev, 0.0, 0.0, A, b, qprev, ic)
    traj = [host(x).copy()]
    for _ in range(n):
        for _it in range(200):
            eec.eec_eval_stamp_tran(circ.ctx, x, qprev, iprev, alpha, beta, A, b, q, ic)
            M = torch.zeros(circ.n, circ.n, dtype=torch.float64, device="cuda")
            M.index_put_((rows, cols), A, accumulate=True)
            y = torch.linalg.solve(M, b)
            dx = torch.clamp(y - x, -0.2, 0.2)       # per-node step limit, as the oracle
            x = x + dx
            if float(dx.abs().max()) <= 1e-12 + 1e-9 * float(x.abs().max()):
                break
        eec.eec_eval_stamp_tran(circ.ctx, x, qprev, iprev, alpha, beta, A, b, q, ic)
        qprev, q = q.clone(), qprev
        iprev = ic.clone()
        traj.append(host(x).copy())
    assert circ.status() == 0
    return np.array(traj)


@pytest.mark.parametrize("method", [0, 1])
def test_gpu_stamped_transient_rc_matches_oracle(eec, method):
    W, L, R, Vs = 4e-6, 1e-6, 5e3, 1.0
    card = netgen.card(VTH0=5.0, JS=0.0, GMIN=0.0)
    cards = np.stack([card, card])
    net = tiny_net("rc", [1, 1, 0], [0, Vs, 0], [(0, 2, 0, 0)], [1], W=[W], L=[L], res=[(1, 2)],
                   resG=[1 / R], gshunt=0.0)
    C = 4e-10 * W
    h = R * C / 7
    ref = oracle.Oracle(net, cards).tran_solve(np.zeros(1), h, 30, method=method)
    got = _gpu_transient(eec, net, cards, h, 30, method, variant=2)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("variant", [0, 2, 4, 5])
def test_gpu_stamped_transient_inverter_chain_matches_oracle(eec, variant):
    net = netgen.inverter_chain(6, vin=1.0)   # input stepped from 0 V to 1 V at t = 0
    o = oracle.Oracle(net, CARDS)
    h = 2e-12
    ref = o.tran_solve(np.zeros(net.n_free), h, 25, method=1)
    got = _gpu_transient(eec, net, CARDS, h, 25, 1, variant)
    # both loops stop at |dx| <= 1e-12 + 1e-9 |x|: the states agree far inside that
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10)
    assert np.abs(ref[-1] - ref[0]).max() > 0.5          # the chain really switches


@pytest.mark.parametrize("solver,variant", [(0, 2), (2, 2), (2, 5)])
@pytest.mark.parametrize("method", [0, 1])
def test_library_transient_matches_oracle(eec, method, solver, variant):
    # the library's own transient run (eec_transient: the GPU Newton loop on the companion
    # stamp, every step solved on the GPU) against the oracle's transient solver (dense LU,
    # the same per-node step limit and |dx| test): a 6-stage chain switching its input at t = 0
    import torch
    net = netgen.inverter_chain(6, vin=1.0)
    h, n = 2e-12, 25
    ref = oracle.Oracle(net, CARDS).tran_solve(np.zeros(net.n_free), h, n, method=method)
    circ = eec.Circuit(net, CARDS, variant=variant)   # 5: the pipelined colour schedule
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    traj = torch.empty((n + 1) * circ.n, dtype=torch.float64, device="cuda")
    its = eec.eec_transient(circ.ctx, x, h, n, method=method, traj=traj, solver=solver)
    assert its >= n and circ.status() == 0
    got = host(traj).reshape(n + 1, circ.n)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10)
    np.testing.assert_array_equal(host(x), got[-1])
    assert np.abs(ref[-1] - ref[0]).max() > 0.5          # the chain really switches


@pytest.mark.parametrize("method", [0, 1])
def test_library_transient_rc_and_single_step(eec, method):
    # an RC charge through a resistor into a gate capacitance: the library's run against the
    # oracle (whose BE/TR recurrences are pinned to the exact ones on the CPU); then one step by
    # eec_newton_tran from the run's last state and history equals one more step of the run
    import torch
    W, L, R, Vs = 4e-6, 1e-6, 5e3, 1.0
    card = netgen.card(VTH0=5.0, JS=0.0, GMIN=0.0)
    cards = np.stack([card, card])
    net = tiny_net("rc", [1, 1, 0], [0, Vs, 0], [(0, 2, 0, 0)], [1], W=[W], L=[L], res=[(1, 2)],
                   resG=[1 / R], gshunt=0.0)
    h = R * 4e-10 * W / 7
    ref = oracle.Oracle(net, cards).tran_solve(np.zeros(1), h, 31, method=method)
    circ = eec.Circuit(net, cards, color=True, variant=2)
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    traj = torch.empty(32 * circ.n, dtype=torch.float64, device="cuda")
    eec.eec_transient(circ.ctx, x, h, 31, method=method, traj=traj)
    np.testing.assert_allclose(host(traj).reshape(32, circ.n), ref, rtol=1e-10, atol=1e-13)
    # the step API: 30 steps by the run, then step 31 by eec_newton_tran (backward Euler: the
    # history is the charges at step 30 alone)
    if method == 0:
        x2 = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
        eec.eec_transient(circ.ctx, x2, h, 30, method=0)
        A, b, q = circ.new_outputs(want_q=True)
        q30 = torch.zeros_like(q)
        eec.eec_eval_stamp_tran(circ.ctx, x2, q30, None, 0.0, 0.0, A, b, q30, None)
        it = eec.eec_newton_tran(circ.ctx, x2, q30, None, 1.0 / h, 0.0, A, b, q)
        assert it >= 1
        np.testing.assert_allclose(host(x2), ref[31], rtol=1e-10, atol=1e-13)
