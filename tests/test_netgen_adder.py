"""The ripple-carry adder generator and the series-resistor transform behind the Table II
colour study (CPU only): functional correctness of the adder through the oracle's DC solve, and
the colour counts the paper prints for the 64-bit adder (tests/golden/adder64_table2.txt)."""
import os

import numpy as np
import pytest

import netgen
import oracle

CARDS = netgen.default_cards()
GOLD = os.path.join(os.path.dirname(__file__), "golden", "adder64_table2.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split(":")
            out[k.strip()] = int(v)
    return out


@pytest.mark.parametrize("n_bits,seed", [(1, 5), (4, 5), (6, 17)])
def test_adder_adds(n_bits, seed):
    net = netgen.ripple_adder(n_bits, seed=seed)
    o = oracle.Oracle(net, CARDS)
    x, _ = o.dc_solve(max_iter=600)
    _, _, unk = o.pattern()
    ins = [i for i in range(2, net.n_nodes) if net.node_fixed[i]]
    bit = lambda v: int(v > 0.5)
    a = sum(bit(net.node_vfix[ins[2 * k]]) << k for k in range(n_bits))
    b = sum(bit(net.node_vfix[ins[2 * k + 1]]) << k for k in range(n_bits))
    cin = bit(net.node_vfix[ins[2 * n_bits]])
    got = sum(bit(x[unk[s]]) << k for k, s in enumerate(net.meta["sums"]))
    got += bit(x[unk[net.meta["cout"]]]) << n_bits
    assert got == a + b + cin


def test_table2_colour_counts():
    g = _golden()
    base = netgen.ripple_adder(64)
    assert base.n_dev == g["transistors"]
    assert oracle.Oracle(base, CARDS).color_greedy(rule=1)[1] == g["base_colors_literal_rule"]
    r14 = netgen.insert_series_resistors(base, per_group=14)
    assert len(r14.res_G) == g["r14_resistors"] and r14.n_dev == g["transistors"]
    rall = netgen.insert_series_resistors(base)
    assert oracle.Oracle(rall, CARDS).color_greedy(rule=0)[1] == g["r89_colors"]


def test_series_resistors_only_split_nets():
    # the transform keeps every device and (with small links) the circuit's DC solution:
    # 10-ohm links carry at most ~1e-4 A, so split nodes sit within ~1e-3 V of their net
    base = netgen.ripple_adder(3, seed=2)
    r = netgen.insert_series_resistors(base, per_group=9, r_ohm=10.0)
    assert r.n_dev == base.n_dev and len(r.res_G) == 27
    xb, _ = oracle.Oracle(base, CARDS).dc_solve(max_iter=600)
    xr, _ = oracle.Oracle(r, CARDS).dc_solve(max_iter=600)
    n_old = int(np.count_nonzero(base.node_fixed == 0))
    np.testing.assert_allclose(xr[:n_old], xb, atol=2e-3)
    # every new node hangs off exactly one original net through one resistor
    new = r.res_nodes[:, 0]
    assert np.all(new >= base.n_nodes) and len(np.unique(new)) == 27
