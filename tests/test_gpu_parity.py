"""GPU parity: the CUDA path through the C ABI against the oracle, element by element.

Tolerance for A and b: per entry |gpu - oracle| / max(|oracle|, S_e) <= 1e-12,
where S_e is the sum of |contribution| into that entry (the oracle accumulates it), so rows whose
terms cancel are judged against the size of their terms. Charges: per device relative to the
largest terminal charge of that device. Colourings: bit-exact. Gradients: 1e-8 relative to
max(|oracle|, 1e-6 * max|oracle|).
"""
import numpy as np
import pytest

import netgen
import oracle
from helpers import rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-12
CARDS = netgen.default_cards()
ALL_VARIANTS = [0, 1, 2, 3, 4, 5]
DETERMINISTIC = [0, 1, 3, 4, 5]   # every schedule but the atomic one


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def check_against_oracle(eec, circ, o, x, variant, want_q=True, ref=None):
    eec.eec_set_variant(circ.ctx, variant)
    A, b, q = circ.eval_stamp(dev(x), want_q=want_q)
    assert circ.status() == 0
    r = ref if ref is not None else o.eval_stamp(x, want_q=want_q, want_scale=True)
    eA = rel_err(host(A), r["A"], r["A_scale"])
    eb = rel_err(host(b), r["b"], r["b_scale"])
    assert eA.max() <= TOL, (variant, eA.max(), int(eA.argmax()))
    assert eb.max() <= TOL, (variant, eb.max(), int(eb.argmax()))
    if want_q and r["q"].size:
        qg = host(q).reshape(4, -1)
        scale = np.maximum(np.abs(r["q"]).max(axis=0, keepdims=True), 1e-300)
        assert (np.abs(qg - r["q"]) / scale).max() <= 1e-13
    return host(A), host(b), r


def test_fp64_probe_reports_a_positive_rate(eec):
    f = eec.eec_fp64_peak(256, 4)
    assert 1e11 < f < 1e14


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_config1_inverter_chain_newton_iterates(eec, variant):
    # Sec. I: A, b are re-formed at every Newton iterate; check them along the oracle's DC solve.
    net = netgen.config(1)
    o = oracle.Oracle(net, CARDS)
    _, it, hist = o.dc_solve(history=True)
    circ = eec.Circuit(net, CARDS, color=True)
    assert circ.n_colors == 4
    for k in list(range(0, len(hist), 17)) + [len(hist) - 1]:
        check_against_oracle(eec, circ, o, hist[k], variant)
    x2 = oracle.Oracle(netgen.inverter_chain(64, vin=0.5), CARDS).dc_solve()[0]
    circ2 = eec.Circuit(netgen.inverter_chain(64, vin=0.5), CARDS)
    check_against_oracle(eec, circ2, oracle.Oracle(netgen.inverter_chain(64, vin=0.5), CARDS),
                         x2, variant)


def _edge_nets():
    from helpers import tiny_net
    # no devices at all (resistor network only)
    yield tiny_net("nodev", [1, 1, 0, 0], [0, 1.0, 0, 0], np.zeros((0, 4)), [],
                   res=[(1, 2), (2, 3), (3, 0)], resG=[1e-3, 2e-3, 5e-4])
    # every terminal on a source-held node: nothing to stamp from the device
    yield tiny_net("allfixed", [1, 1, 1, 0], [0, 1.0, 0.4, 0], [(1, 2, 0, 0)], [1], res=[(3, 0)],
                   resG=[1e-3])
    # shorted (d = s), diode-connected (d = g), body on a free node, PMOS mirror pair
    yield tiny_net("odd", [1, 1, 0, 0, 0], [0, 1.0, 0, 0, 0],
                   [(2, 3, 2, 0), (3, 3, 0, 0), (2, 1, 4, 4), (4, 2, 1, 1), (3, 4, 2, 3)],
                   [1, 1, 1, -1, -1], res=[(1, 2), (3, 0)], resG=[1e-3, 1e-4],
                   isrc=[(0, 4)], ival=[1e-5])
    # ragged sizes around the 128-thread block
    for n in (63, 64, 65):
        yield netgen.inverter_chain(n, seed=n)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_edge_cases(eec, variant):
    for net in _edge_nets():
        o = oracle.Oracle(net, CARDS)
        circ = eec.Circuit(net, CARDS, color=True)
        for s in range(2):
            x = netgen.random_x(net, seed=s, lo=-0.2, hi=1.2)
            check_against_oracle(eec, circ, o, x, variant)


def _fan_net(k):
    # k transistors with their drains on one free node (2), each gate on a free node of its own,
    # sources and bodies on the rails: entry (2, 2) and row 2 of b receive k contributions, the
    # gate rows none (their diagonals keep only gshunt)
    from helpers import tiny_net
    fixed = [1, 1] + [0] * (1 + k)
    vfix = [0.0, 1.0] + [0.0] * (1 + k)
    types = [1 if i % 3 else -1 for i in range(k)]
    devs = [(2, 3 + i, 0 if t > 0 else 1, 0 if t > 0 else 1) for i, t in enumerate(types)]
    W = [1e-6 * (1 + (i % 7)) for i in range(k)]
    return tiny_net(f"fan{k}", fixed, vfix, devs, types, W=W, res=[(1, 2)], resG=[1e-4])


@pytest.mark.parametrize("k", [1, 30, 31, 32, 33, 100, 1500])
def test_fan_in_around_the_heavy_entry_bound(eec, k):
    # The segmented reduction's gather sums an entry with fewer than 32 contributions in a group
    # of 32 entries sorted by their count (up to 32 items per lane: the linear part and 31
    # contributions), and one with 32 or more in a warp of its own; 1,500 spreads the pattern
    # over several windows of 1,024 entries.
    net = _fan_net(k)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, color=True)
    for s in range(2):
        x = netgen.random_x(net, seed=70 + s, lo=-0.2, hi=1.2)
        ref = o.eval_stamp(x, want_q=True, want_scale=True)
        outs = {v: check_against_oracle(eec, circ, o, x, v, ref=ref) for v in (2, 3)}
        again = circ.eval_stamp(dev(x))
        assert np.array_equal(host(again[0]), outs[3][0]) and np.array_equal(host(again[1]), outs[3][1])


@pytest.mark.parametrize("variant", [0, 2, 3, 5])
@pytest.mark.parametrize("make", [lambda: netgen.sram(16, 16), netgen.ota5t,
                                  lambda: netgen.random_logic(500, seed=2)])
def test_wide_bias(eec, variant, make):
    # node voltages far outside the rails: forward-biased junctions past the exponent limit
    # (v / Vt > 40, the linear continuation), reverse-mode channels, deep subthreshold and strong
    # inversion in one launch
    net = make()
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, color=True)
    for s in range(3):
        x = netgen.random_x(net, seed=40 + s, lo=-3.0, hi=4.0)
        check_against_oracle(eec, circ, o, x, variant)


@pytest.fixture(scope="module")
def sram_full():
    net = netgen.config(2)
    o = oracle.Oracle(net, CARDS)
    x = netgen.random_x(net)
    ref = o.eval_stamp(x, want_q=True, want_scale=True)
    return net, o, x, ref


def test_config2_sram_all_variants_full_size(eec, sram_full):
    net, o, x, ref = sram_full
    circ = eec.Circuit(net, CARDS, color=True)
    ocol, oC = o.color_greedy()
    assert circ.n_colors == oC >= 512
    assert np.array_equal(circ.colors, ocol)
    outs = {}
    for v in ALL_VARIANTS:
        outs[v] = check_against_oracle(eec, circ, o, x, v, ref=ref)
    # the colour schedules add every entry's contributions in the same colour order; each kernel
    # is compiled on its own, so a multiply-add fused in one may be rounded twice in another:
    # they agree to rounding, not necessarily bitwise
    for v in (1, 4, 5):
        for k in (0, 1):
            scale = ref["A_scale"] if k == 0 else ref["b_scale"]
            assert (np.abs(outs[v][k] - outs[0][k]) / np.maximum(scale, 1e-300)).max() <= 1e-14
    # every schedule except the atomic one is deterministic: two runs agree bitwise
    for v in DETERMINISTIC:
        again = check_against_oracle(eec, circ, o, x, v, ref=ref)
        assert np.array_equal(again[0], outs[v][0]) and np.array_equal(again[1], outs[v][1]), v


def test_config3_random_logic_full_size_and_gpu_colouring(eec):
    net = netgen.config(3)
    o = oracle.Oracle(net, CARDS)
    x = netgen.random_x(net)
    ref = o.eval_stamp(x, want_q=True, want_scale=True)
    ocol, oC = o.color_greedy()
    circ = eec.Circuit(net, CARDS, color=True, algo=eec.EEC_COLOR_JP_INDEX)
    assert circ.n_colors == oC and np.array_equal(circ.colors, ocol)
    for v in (0, 2, 3, 5):
        check_against_oracle(eec, circ, o, x, v, ref=ref)


def test_million_fet_random_logic_full_size(eec):
    # the ~1.0M-FET netlist of the throughput bar (277,778 gates of the config-3 generator):
    # the schedules the bench times there, entry by entry against the oracle
    net = netgen.random_logic(277_778)
    assert net.n_dev > 990_000
    o = oracle.Oracle(net, CARDS)
    x = netgen.random_x(net)
    ref = o.eval_stamp(x, want_q=True, want_scale=True)
    circ = eec.Circuit(net, CARDS, color=True)
    outs = {}
    for v in ALL_VARIANTS:
        outs[v] = check_against_oracle(eec, circ, o, x, v, ref=ref)
    for v in DETERMINISTIC:   # deterministic schedules repeat bitwise
        again = check_against_oracle(eec, circ, o, x, v, ref=ref, want_q=False)
        assert np.array_equal(again[0], outs[v][0]) and np.array_equal(again[1], outs[v][1]), v


def test_config4_batch_full_size(eec):
    nets = netgen.batch_circuits(4096)
    merged = netgen.concat(nets)
    o = oracle.Oracle(merged, CARDS)
    x = netgen.random_x(merged)
    ref = o.eval_stamp(x, want_q=True, want_scale=True)
    circ = eec.Circuit(None, CARDS, color=True, batch=nets)
    assert circ.n_dev == merged.n_dev
    ocol, oC = o.color_greedy()
    assert circ.n_colors == oC and np.array_equal(circ.colors, ocol)
    for v in ALL_VARIANTS:
        check_against_oracle(eec, circ, o, x, v, ref=ref)
    ro, no, do = eec.eec_get_batch_offsets(circ.ctx, len(nets))
    assert ro[-1] == circ.n and no[-1] == circ.nnz


def _valid_coloring(net, col):
    # the devices on every free node carry distinct colours
    nodes = net.dev_nodes
    ok_node = (net.node_fixed == 0)
    pairs = []
    for t in range(4):
        m = ok_node[nodes[:, t]]
        pairs.append(np.stack([nodes[m, t], np.nonzero(m)[0]], 1))
    p = np.concatenate(pairs)
    p = np.unique(p, axis=0)                      # (node, device) once
    key = p[:, 0].astype(np.int64) * (col.max() + 2) + col[p[:, 1]]
    return len(np.unique(key)) == len(key)


@pytest.mark.parametrize("make", [lambda: netgen.inverter_chain(64), lambda: netgen.ring_oscillator(11),
                                  netgen.ota5t, lambda: netgen.sram(32, 32),
                                  lambda: netgen.random_logic(20000, seed=4)])
def test_jones_plassmann_colouring(eec, make):
    net = make()
    o = oracle.Oracle(net, CARDS)
    for order in (None, np.random.default_rng(3).permutation(net.n_dev).astype(np.int32)):
        ocol, oC = o.color_greedy(order=order)
        circ = eec.Circuit(net, CARDS, algo=eec.EEC_COLOR_JP_INDEX, order=order)
        assert circ.n_colors == oC and np.array_equal(circ.colors, ocol)
    circ = eec.Circuit(net, CARDS, algo=eec.EEC_COLOR_JP_RANDOM)
    assert _valid_coloring(net, circ.colors)
    x = netgen.random_x(net)
    check_against_oracle(eec, circ, o, x, 0)


def _grad_close(g, ref, tol=1e-8):
    floor = 1e-6 * np.abs(ref).max()
    err = np.abs(g - ref) / np.maximum(np.abs(ref), floor)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("make", [lambda: netgen.sram(16, 16), lambda: netgen.inverter_chain(64, vin=0.3),
                                  lambda: netgen.random_logic(2000, seed=8), netgen.ota5t])
def test_backward_matches_oracle_nested_duals(eec, make):
    net = make()
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS)
    rng = netgen.Rng(11, 3)
    x = netgen.random_x(net, seed=5)
    gA = rng.normal(circ.nnz)
    gb = rng.normal(circ.n)
    gx, gW, gL = circ.bwd(dev(x), dev(gA), dev(gb))
    ox, oW, oL = o.eval_stamp_grad(x, gA, gb)
    _grad_close(host(gx), ox)
    _grad_close(host(gW), oW)
    _grad_close(host(gL), oL)


@pytest.mark.parametrize("make", [lambda: netgen.sram(8, 8), netgen.ota5t])
def test_backward_at_wide_bias(eec, make):
    # the backward through the exponent-limited junction branch and reverse-mode channels
    net = make()
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS)
    rng = netgen.Rng(21, 3)
    x = netgen.random_x(net, seed=44, lo=-3.0, hi=4.0)
    gA = rng.normal(circ.nnz)
    gb = rng.normal(circ.n)
    gx, gW, gL = circ.bwd(dev(x), dev(gA), dev(gb))
    ox, oW, oL = o.eval_stamp_grad(x, gA, gb)
    _grad_close(host(gx), ox)
    _grad_close(host(gW), oW)
    _grad_close(host(gL), oL)


def test_config5_backward_full_size_vs_oracle_and_fd(eec, sram_full):
    net, o, x, _ = sram_full
    circ = eec.Circuit(net, CARDS)
    rng = netgen.Rng(netgen.DEFAULT_SEED, 12)
    gA = rng.normal(circ.nnz)
    gb = rng.normal(circ.n)
    gx, gW, gL = circ.bwd(dev(x), dev(gA), dev(gb))
    assert circ.status() == 0
    ox, oW, oL = o.eval_stamp_grad(x, gA, gb)
    _grad_close(host(gx), ox)
    _grad_close(host(gW), oW)
    _grad_close(host(gL), oL)
    # central differences (h = 1e-6 relative) of s = <gA, A> + <gb, b> through the GPU forward.
    # A and b are differenced first (exactly zero away from the perturbed device), then weighted:
    # differencing two full million-term sums would add their reduction rounding, which is as
    # large as the tolerance once divided by 2h.
    gAt, gbt = dev(gA), dev(gb)

    def ab_of(xv, W=None, L=None):
        if W is not None:
            import paper_2604_03079_gb300 as m
            m.eec_update_params(circ.ctx, dev(W), dev(L))
        A, b, _ = circ.eval_stamp(dev(xv), want_q=False)
        return A.clone(), b.clone()

    def central(p, m, h):
        return float(((p[0] - m[0]) * gAt).sum() + ((p[1] - m[1]) * gbt).sum()) / (2 * h)

    sel = np.random.default_rng(0).choice(circ.n, 6, replace=False)
    for i in sel:
        h = 1e-6 * max(abs(x[i]), 1e-3)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = central(ab_of(xp), ab_of(xm), h)
        assert abs(fd - ox[i]) <= 1e-5 * max(abs(ox[i]), 1e-3 * np.abs(ox).max())
    W0, L0 = net.W.copy(), net.L.copy()
    for k in np.random.default_rng(1).choice(net.n_dev, 6, replace=False):
        for which, base, ref in (("W", W0, oW), ("L", L0, oL)):
            h = 1e-6 * base[k]
            vals = []
            for sg in (1, -1):
                a = base.copy()
                a[k] += sg * h
                vals.append(ab_of(x, a, L0) if which == "W" else ab_of(x, W0, a))
            fd = central(vals[0], vals[1], h)
            assert abs(fd - ref[k]) <= 1e-5 * max(abs(ref[k]), 1e-3 * np.abs(ref).max()), (which, k)
    ab_of(x, W0, L0)   # restore the sizes


def test_adjoint_dc_sensitivity_of_inverter_chain(eec):
    # Sizing-loop use: dV_out/dtheta = -gtheta with gA_ij = lambda_i x_j, gb = -lambda,
    # A^T lambda = e_out at the oracle's DC solution; compared with the oracle's nested duals for
    # every W/L of the 64-stage chain, and with finite differences of full DC solves.
    net = netgen.inverter_chain(64, vin=0.45)
    o = oracle.Oracle(net, CARDS)
    xs, _ = o.dc_solve()
    circ = eec.Circuit(net, CARDS)
    rp, col, _ = circ.pattern()
    rows = np.repeat(np.arange(circ.n), np.diff(rp))
    for out in (0, circ.n - 1):
        lam = o.adjoint(xs, out)
        gA = lam[rows] * xs[col]
        _, gW, gL = circ.bwd(dev(xs), dev(gA), dev(-lam))
        _, oW, oL = o.eval_stamp_grad(xs, gA, -lam)
        _grad_close(host(gW), oW)
        _grad_close(host(gL), oL)
    sens = -host(gW)   # last output above: tiny; redo for the mid-rail first stage
    lam = o.adjoint(xs, 0)
    _, gW, gL = circ.bwd(dev(xs), dev(lam[rows] * xs[col]), dev(-lam))
    for k in (0, 1):
        h = 1e-6 * net.W[k]
        v = []
        for sg in (1, -1):
            W = net.W.copy()
            W[k] += sg * h
            o.set_sizes(W, net.L)
            v.append(o.dc_solve(x0=xs)[0][0])
        o.set_sizes(net.W, net.L)
        fd = (v[0] - v[1]) / (2 * h)
        assert abs(-host(gW)[k] - fd) <= 1e-5 * abs(fd)
    assert np.all(np.isfinite(sens))


def test_autograd_function_matches_backward(eec):
    import torch
    net = netgen.sram(8, 8)
    circ = eec.Circuit(net, CARDS)
    x = dev(netgen.random_x(net)).requires_grad_(True)
    W = dev(net.W).requires_grad_(True)
    L = dev(net.L).requires_grad_(True)
    A, b = eec.eval_stamp_autograd(circ, x, W, L)
    rng = netgen.Rng(2, 2)
    gA, gb = dev(rng.normal(circ.nnz)), dev(rng.normal(circ.n))
    ((A * gA).sum() + (b * gb).sum()).backward()
    gx, gW, gL = circ.bwd(x.detach(), gA, gb)
    assert torch.allclose(x.grad, gx, rtol=0, atol=0)
    assert torch.allclose(W.grad, gW, rtol=0, atol=0)
    assert torch.allclose(L.grad, gL, rtol=0, atol=0)


def test_update_params_matches_oracle_with_new_sizes(eec):
    net = netgen.random_logic(3000, seed=2)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS)
    W2 = net.W * (0.7 + 0.6 * netgen.Rng(4, 4).uniform(net.n_dev))
    L2 = net.L * (0.7 + 0.6 * netgen.Rng(5, 5).uniform(net.n_dev))
    eec.eec_update_params(circ.ctx, dev(W2), dev(L2))
    o.set_sizes(W2, L2)
    x = netgen.random_x(net)
    for v in ALL_VARIANTS:
        check_against_oracle(eec, circ, o, x, v)
    # a rebuild keeps the updated sizes
    eec.eec_color(circ.ctx, n_dev=net.n_dev)
    eec.eec_build_scatter(circ.ctx)
    check_against_oracle(eec, circ, o, x, 0)


def test_graph_capture_and_autotune(eec):
    import torch
    net = netgen.sram(64, 64)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS)
    x = netgen.random_x(net)
    xt = dev(x)
    A, b, q = circ.new_outputs()
    ms = eec.eec_autotune(circ.ctx, xt, A, b, q, reps=3)
    assert all(m > 0 for m in ms)
    assert eec.eec_get_variant(circ.ctx) == int(np.argmin(ms))
    for v in ALL_VARIANTS:
        eec.eec_set_variant(circ.ctx, v)
        eec.eec_graph_capture(circ.ctx, xt, A, b, q)
        A.zero_()
        b.zero_()
        eec.eec_graph_launch(circ.ctx)
        torch.cuda.synchronize()
        r = o.eval_stamp(x, want_scale=True)
        assert rel_err(host(A), r["A"], r["A_scale"]).max() <= TOL
        assert rel_err(host(b), r["b"], r["b_scale"]).max() <= TOL


def test_batch_capture_graph_replays_every_schedule(eec):
    # after eec_batch_capture_graph, eec_eval_stamp replays a cached graph for every schedule,
    # re-captured when the buffers or the schedule change
    import torch
    nets = netgen.batch_circuits(64, seed=6)
    merged = netgen.concat(nets)
    o = oracle.Oracle(merged, CARDS)
    ctx = eec.eec_batch_create(nets, gshunt=merged.gshunt)
    try:
        eec.eec_set_model_cards(ctx, CARDS)
        eec.eec_color(ctx, n_dev=merged.n_dev)
        n, nnz = eec.eec_build_scatter(ctx)
        eec.eec_batch_capture_graph(ctx, torch.cuda.current_stream())
        for seed in (1, 2):
            x = netgen.random_x(merged, seed=seed)
            r = o.eval_stamp(x, want_scale=True)
            xt = dev(x)
            A = torch.empty(nnz, dtype=torch.float64, device="cuda")
            b = torch.empty(n, dtype=torch.float64, device="cuda")
            for v in ALL_VARIANTS:
                eec.eec_set_variant(ctx, v)
                for _ in range(2):                  # capture, then replay
                    A.fill_(7.0)
                    b.fill_(7.0)
                    eec.eec_eval_stamp(ctx, xt, A, b, None)
                    assert eec.eec_status(ctx) == 0
                    assert rel_err(host(A), r["A"], r["A_scale"]).max() <= TOL, v
                    assert rel_err(host(b), r["b"], r["b_scale"]).max() <= TOL, v
    finally:
        eec.eec_destroy(ctx)


def test_grid_barrier_timeout_is_reported_and_the_context_recovers(eec):
    # One block never arrives: the other blocks give up after their bounded wait (about 1 s),
    # record EEC_ETIMEOUT in the status word and return; nothing hangs or faults.
    import time
    net = netgen.inverter_chain(64)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, color=True)
    x = netgen.random_x(net)
    A, b, _ = circ.new_outputs(want_q=False)
    t0 = time.time()
    eec.eec_test_barrier_timeout(circ.ctx, dev(x), A, b)
    assert circ.status() == eec.EEC_ETIMEOUT
    assert time.time() - t0 < 30
    assert circ.status() == 0                     # cleared by the read
    check_against_oracle(eec, circ, o, x, 1)      # the persistent schedule still works


def test_pipelined_wait_timeout_is_reported_and_the_context_recovers(eec):
    # The first work item never reports its stamps done: the next colour's waits give up after
    # their bounded wait (about 1 s), record EEC_ETIMEOUT and abort the launch; the following
    # launches (the timeout left unread) stamp everything again.
    import time
    import torch
    net = netgen.inverter_chain(64)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, color=True, variant=eec.EEC_VARIANT_COLOR_PIPELINED)
    x = netgen.random_x(net)
    A, b, _ = circ.new_outputs(want_q=False)
    t0 = time.time()
    eec.eec_test_barrier_timeout(circ.ctx, dev(x), A, b)
    torch.cuda.synchronize()
    assert time.time() - t0 < 30
    ref = o.eval_stamp(x, want_scale=True)
    for _ in range(2):
        A, b, _ = circ.eval_stamp(dev(x), want_q=False)
        torch.cuda.synchronize()
        assert rel_err(host(A), ref["A"], ref["A_scale"]).max() <= TOL
        assert rel_err(host(b), ref["b"], ref["b_scale"]).max() <= TOL
    assert circ.status() == eec.EEC_ETIMEOUT
    assert circ.status() == 0
    check_against_oracle(eec, circ, o, x, eec.EEC_VARIANT_COLOR_PIPELINED)


@pytest.mark.parametrize("variant", [1, 4])
def test_timeout_left_unread_does_not_abort_later_launches(eec, variant):
    # A timeout stays recorded in the status word until the host reads it; the next persistent
    # launches (the grid-barrier evaluation, and the grid-barrier colour stamp of the buffered
    # schedule) must still pass every barrier and stamp everything.
    import torch
    net = netgen.inverter_chain(64)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, color=True, color_stamp=2)
    x = netgen.random_x(net)
    A, b, _ = circ.new_outputs(want_q=False)
    eec.eec_test_barrier_timeout(circ.ctx, dev(x), A, b)
    ref = o.eval_stamp(x, want_scale=True)
    eec.eec_set_variant(circ.ctx, variant)
    for _ in range(2):
        A, b, _ = circ.eval_stamp(dev(x), want_q=False)
        torch.cuda.synchronize()
        assert rel_err(host(A), ref["A"], ref["A_scale"]).max() <= TOL
        assert rel_err(host(b), ref["b"], ref["b_scale"]).max() <= TOL
    assert circ.status() == eec.EEC_ETIMEOUT      # the one timeout, reported once
    assert circ.status() == 0


@pytest.mark.parametrize("variant,chunks", [(2, 0), (2, 1), (2, 5), (3, 3), (0, 4)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_entry_point(eec, pinned, variant, chunks):
    # chunks > 1 under the order-free schedules (2 atomic, 3 segmented reduction): charges leave
    # span by span on a second stream; colour schedules (0) ignore the chunk count
    import torch
    net = netgen.sram(24, 20)
    o = oracle.Oracle(net, CARDS)
    circ = eec.Circuit(net, CARDS, variant=variant, host_chunks=chunks)
    mk = (lambda n: torch.empty(n, dtype=torch.float64).pin_memory()) if pinned else \
         (lambda n: torch.empty(n, dtype=torch.float64))
    xh, Ah, bh, qh = mk(circ.n), mk(circ.nnz), mk(circ.n), mk(4 * circ.n_dev)
    side = torch.cuda.Stream()
    for seed in range(3):
        x = netgen.random_x(net, seed=seed)
        xh.copy_(torch.as_tensor(x))
        for t in (Ah, bh, qh):
            t.fill_(float("nan"))
        with torch.cuda.stream(side):       # stream ordering: outputs valid after this sync
            eec.eec_eval_stamp_host(circ.ctx, xh, Ah, bh, qh if seed < 2 else None, side)
        side.synchronize()
        assert circ.status() == 0
        r = o.eval_stamp(x, want_q=True, want_scale=True)
        assert rel_err(Ah.numpy(), r["A"], r["A_scale"]).max() <= TOL
        assert rel_err(bh.numpy(), r["b"], r["b_scale"]).max() <= TOL
        if seed < 2:
            qs = np.maximum(np.abs(r["q"]).max(axis=0, keepdims=True), 1e-300)
            assert (np.abs(qh.numpy().reshape(4, -1) - r["q"]) / qs).max() <= 1e-13
        else:
            assert np.isnan(qh.numpy()).all()   # q not requested: left alone


@pytest.mark.parametrize("make", [lambda: netgen.sram(24, 20), lambda: netgen.random_logic(3000, seed=4),
                                  lambda: netgen.ripple_adder(8)])
def test_color_buffered_stamp_implementations_agree_bitwise(eec, make):
    # per-colour launches, one grid with a grid barrier, one cluster with the cluster barrier:
    # the same additions in the same colour order, so the same bits; and the oracle's values
    net = make()
    o = oracle.Oracle(net, CARDS)
    x = netgen.random_x(net, seed=5)
    ref = o.eval_stamp(x, want_q=True, want_scale=True)
    outs = []
    for mode in (1, 2, 3):
        circ = eec.Circuit(net, CARDS, variant=eec.EEC_VARIANT_COLOR_BUFFERED, color_stamp=mode)
        assert circ.n_colors >= 3
        outs.append(check_against_oracle(eec, circ, o, x, eec.EEC_VARIANT_COLOR_BUFFERED, ref=ref))
    for k in (0, 1):
        assert np.array_equal(outs[1][k], outs[0][k]) and np.array_equal(outs[2][k], outs[0][k])
    # the pipelined schedule adds in the same colour order (its own kernel: equal to rounding)
    circ = eec.Circuit(net, CARDS, variant=eec.EEC_VARIANT_COLOR_PIPELINED)
    pipe = check_against_oracle(eec, circ, o, x, eec.EEC_VARIANT_COLOR_PIPELINED, ref=ref)
    for k, sc in ((0, "A_scale"), (1, "b_scale")):
        assert (np.abs(pipe[k] - outs[0][k]) / np.maximum(ref[sc], 1e-300)).max() <= 1e-14


def test_debug_checks_flag_non_finite_inputs(eec):
    net = netgen.inverter_chain(8)
    circ = eec.Circuit(net, CARDS, debug_checks=True)
    x = netgen.random_x(net)
    x[3] = np.nan
    circ.eval_stamp(dev(x))
    assert circ.status() == eec.EEC_ENUMERIC
    x[3] = 0.5
    circ.eval_stamp(dev(x))
    assert circ.status() == 0
