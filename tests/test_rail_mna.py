"""Modified nodal analysis of the rails (rail_mode 1, CPU only).

Pins of the oracle's MNA form against what does not come from its stamp:
  * the resistor divider's source current in closed form;
  * a lone NMOS between two held nodes: the source currents are minus the terminal currents of
    the device model itself (no stamp involved);
  * on a larger circuit, every source current equals minus the current the elements draw from
    its rail, summed from single-device evaluations; the node voltages equal the eliminated
    form's DC solution; the free-node rows of A x - b equal the eliminated form's KCL residual;
  * colouring: with the rails as unknowns, the free-node rule is the literal any-node rule of
    Sec. II, and the 64-bit adder needs one colour per PMOS (Table II, 896).
Then the library's host side under the same mode: pattern, unknown map and colouring identical
to the oracle's, and the option's validation.
"""
import numpy as np
import pytest

import netgen
import oracle
from helpers import tiny_net

CARDS = netgen.default_cards()


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def rails(net):
    return [i for i in range(1, net.n_nodes) if net.node_fixed[i]]


def test_divider_source_current_closed_form():
    G1, G2, vdd = 1e-3, 3e-3, 1.2
    net = tiny_net("div", [1, 1, 0], [0, vdd, 0], np.zeros((0, 4)), [], res=[(1, 2), (2, 0)],
                   resG=[G1, G2], gshunt=0.0)
    o = oracle.Oracle(net, CARDS, rail_mode=1)
    assert o.n == 3                          # v1, v2, then the current of the VDD source
    _, _, unk = o.pattern()
    assert list(unk) == [-1, 0, 1]
    x, _ = o.dc_solve()
    v2 = vdd * G1 / (G1 + G2)
    np.testing.assert_allclose(x[0], vdd, rtol=1e-14)
    np.testing.assert_allclose(x[1], v2, rtol=1e-13)
    # KCL at the rail: G1 (v1 - v2) + j = 0 (j leaves the node into the source)
    np.testing.assert_allclose(x[2], -G1 * (vdd - v2), rtol=1e-13)


def test_lone_nmos_source_currents_are_the_model_terminal_currents():
    vdd, vg, W, L = 1.0, 0.8, 2e-6, 0.5e-6
    net = tiny_net("nmos", [1, 1, 1], [0, vdd, vg], [(1, 2, 0, 0)], [1], W=[W], L=[L],
                   gshunt=0.0)
    o = oracle.Oracle(net, CARDS, rail_mode=1)
    assert o.n == 4
    x, _ = o.dc_solve()
    I, _, _ = oracle.device_eval(CARDS[0], 1, W, L, np.array([vdd, vg, 0.0, 0.0]))
    assert I[0] > 1e-6                       # the device conducts from VDD to ground
    np.testing.assert_allclose(x[:2], [vdd, vg], rtol=1e-14)
    np.testing.assert_allclose(x[2], -I[0], rtol=1e-12)
    np.testing.assert_allclose(x[3], -I[1], atol=1e-18)


def _node_currents(net, xnode):
    """Current leaving every node into the elements at node voltages xnode, summed from
    single-device model evaluations, resistors, current sources and gshunt."""
    F = np.zeros(net.n_nodes)
    for k in range(net.n_dev):
        nodes = net.dev_nodes[k]
        card = CARDS[int(net.model_id[k])]
        I, _, _ = oracle.device_eval(card, int(net.dev_type[k]), net.W[k], net.L[k], xnode[nodes])
        np.add.at(F, nodes, I)
    for (i, j), G in zip(net.res_nodes, net.res_G):
        F[i] += G * (xnode[i] - xnode[j])
        F[j] -= G * (xnode[i] - xnode[j])
    for (a, b), I in zip(net.isrc_nodes, net.isrc_val):
        F[a] += I
        F[b] -= I
    F[1:] += net.gshunt * xnode[1:]
    return F


@pytest.mark.parametrize("make", [lambda: netgen.ota5t(),
                                  lambda: netgen.inverter_chain(16, vin=0.45)],
                         ids=["ota5t", "chain16"])
def test_mna_solution_against_eliminated_form_and_device_currents(make):
    net = make()
    oe = oracle.Oracle(net, CARDS)
    om = oracle.Oracle(net, CARDS, rail_mode=1)
    R = rails(net)
    assert om.n == net.n_nodes - 1 + len(R)
    xe, _ = oe.dc_solve(max_iter=400)
    _, _, unk_e = oe.pattern()
    _, _, unk_m = om.pattern()
    assert list(unk_m) == [-1] + list(range(net.n_nodes - 1))
    x0 = np.zeros(om.n)
    x0[unk_m[R]] = net.node_vfix[R]          # start on the rails
    xm, _ = om.dc_solve(x0=x0, max_iter=400)
    xnode = np.where(net.node_fixed == 1, net.node_vfix, 0.0)
    free = np.nonzero(unk_e >= 0)[0]
    xnode[free] = xe[unk_e[free]]
    np.testing.assert_allclose(xm[unk_m[1:]], xnode[1:], rtol=0, atol=1e-9)
    F = _node_currents(net, xnode)
    j = xm[net.n_nodes - 1:]
    scale = max(np.abs(F[R]).max(), 1e-12)
    assert np.abs(j + F[R]).max() <= 1e-6 * scale + 1e-15


@pytest.mark.parametrize("make", [lambda: netgen.ota5t(), lambda: netgen.sram(4, 4),
                                  lambda: netgen.ripple_adder(2, seed=3)],
                         ids=["ota5t", "sram4x4", "adder2"])
def test_free_rows_of_the_mna_residual_equal_the_eliminated_residual(make):
    net = make()
    oe = oracle.Oracle(net, CARDS)
    om = oracle.Oracle(net, CARDS, rail_mode=1)
    _, _, unk_e = oe.pattern()
    R = rails(net)
    xe = netgen.random_x(net, seed=11)
    xm = np.zeros(om.n)
    xnode = np.where(net.node_fixed == 1, net.node_vfix, 0.0)
    free = np.nonzero(unk_e >= 0)[0]
    xnode[free] = xe[unk_e[free]]
    xm[: net.n_nodes - 1] = xnode[1:]
    xm[net.n_nodes - 1:] = netgen.Rng(5, 2).normal(len(R)) * 1e-4
    Fe = oe.kcl_residual(xe)
    sm = om.eval_stamp(xm, want_scale=True)
    rp, col, _ = om.pattern()
    import scipy.sparse as sp
    A = sp.csr_matrix((sm["A"], col, rp), shape=(om.n, om.n))
    Fm = A @ xm - sm["b"]
    rows = unk_e[free]
    tol = 1e-12 * (np.abs(Fe) + sm["b_scale"][free - 1] + 1e-12)
    assert (np.abs(Fm[free - 1] - Fe[rows]) <= tol).all()
    # rail rows: the elements' current plus the source current; source rows: v - vfix
    Fn = _node_currents(net, xnode)
    jr = xm[net.n_nodes - 1:]
    rr = np.array(R) - 1
    assert (np.abs(Fm[rr] - (Fn[R] + jr)) <= 1e-12 * (sm["b_scale"][rr] + np.abs(jr))).all()
    np.testing.assert_allclose(Fm[net.n_nodes - 1:], 0.0, atol=1e-15)


def test_rails_as_unknowns_make_the_free_node_rule_the_literal_rule():
    for net in (netgen.ota5t(), netgen.sram(4, 4), netgen.inverter_chain(12)):
        a = oracle.Oracle(net, CARDS, rail_mode=1).color_greedy(rule=0)
        b = oracle.Oracle(net, CARDS).color_greedy(rule=1)
        assert a[1] == b[1] and np.array_equal(a[0], b[0])


def test_table2_adder_colours_under_mna():
    # Table II: 896 colours for the 64-bit adder's 1792 transistors (one per PMOS: VDD clique)
    net = netgen.ripple_adder(64)
    _, C = oracle.Oracle(net, CARDS, rail_mode=1).color_greedy(rule=0)
    assert C == 896 == int(np.count_nonzero(net.dev_type < 0))


def _lib_ctx(eec, net, rule=0):
    ctx = eec.eec_create(conflict_rule=rule, rail_mode=eec.EEC_RAIL_MNA_BRANCH)
    eec.eec_upload_netlist(ctx, net.node_fixed, net.node_vfix, net.dev_nodes, net.dev_type,
                           net.W, net.L, net.model_id, net.res_nodes, net.res_G, net.isrc_nodes,
                           net.isrc_val, net.gshunt)
    eec.eec_set_model_cards(ctx, CARDS)
    return ctx


@pytest.mark.parametrize("make", [lambda: netgen.ota5t(), lambda: netgen.sram(6, 8),
                                  lambda: netgen.ripple_adder(4, seed=2),
                                  lambda: netgen.inverter_chain(40)],
                         ids=["ota5t", "sram6x8", "adder4", "chain40"])
@pytest.mark.parametrize("rule", [0, 2])
def test_library_host_side_equals_oracle_under_mna(eec, make, rule):
    net = make()
    o = oracle.Oracle(net, CARDS, rail_mode=1)
    ctx = _lib_ctx(eec, net, rule)
    try:
        col, C = eec.eec_color(ctx, n_dev=net.n_dev)
        ocol, oC = o.color_greedy(rule=rule)
        assert C == oC and np.array_equal(col, ocol)
        try:
            n, nnz = eec.eec_build_scatter(ctx)
        except eec.EECError as e:          # no GPU here: the host part is still built
            assert e.code == eec.EEC_ECUDA
        rp, colx, unk = eec.eec_get_pattern(ctx, net.n_nodes)
        orp, ocolx, ounk = o.pattern()
        assert np.array_equal(rp, orp) and np.array_equal(colx, ocolx)
        assert np.array_equal(unk, ounk)
        assert len(rp) - 1 == net.n_nodes - 1 + len(rails(net))
    finally:
        eec.eec_destroy(ctx)


def test_rail_mode_validation(eec):
    with pytest.raises(eec.EECError):
        eec.eec_create(rail_mode=2)
    with pytest.raises(eec.EECError):
        eec.eec_create(rail_mode=-1)
    assert eec.eec_default_options().rail_mode == eec.EEC_RAIL_ELIMINATE
    ctx = eec.eec_create(rail_mode=eec.EEC_RAIL_MNA_BRANCH)
    try:
        with pytest.raises(eec.EECError) as e:
            eec.eec_upload_batch(ctx, netgen.batch_circuits(3, seed=1))
        assert e.value.code == eec.EEC_EINVAL
    finally:
        eec.eec_destroy(ctx)
