"""Pins of the oracle's conflict graph and greedy colouring (Sec. I, Sec. II): hand-derived
colourings of small circuits (tests/golden), brute-force validity and chromatic numbers on tiny
graphs, clique lower bounds, and the greedy definition re-checked vertex by vertex."""
import os

import numpy as np
import pytest

import netgen
import oracle
from helpers import chromatic_number, conflict_adjacency, tiny_net

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CARDS = netgen.default_cards()


def read_golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.split()
    return out


def test_ota5t_matches_hand_derived_coloring():
    g = read_golden("ota5t_coloring.txt")
    net = netgen.ota5t()
    adj = conflict_adjacency(net)
    edges = sorted((a, b) for a in range(5) for b in adj[a] if a < b)
    assert edges == sorted(tuple(int(v) for v in e.split("-")) for e in g["edges"])
    col, C = oracle.Oracle(net, CARDS).color_greedy()
    assert col.tolist() == [int(v) for v in g["colors"]]
    assert C == int(g["n_colors"][0]) == chromatic_number(adj)


def test_inverter_chain_and_ring_match_hand_derived_coloring():
    g = read_golden("inverter_chain_coloring.txt")
    col, C = oracle.Oracle(netgen.inverter_chain(6), CARDS).color_greedy()
    assert col.tolist() == [int(v) for v in g["chain6"]] and C == int(g["chain_n_colors"][0])
    col, C = oracle.Oracle(netgen.ring_oscillator(11), CARDS).color_greedy()
    assert col.tolist() == [int(v) for v in g["ring11"]] and C == int(g["ring_n_colors"][0])
    col, C = oracle.Oracle(netgen.inverter_chain(64), CARDS).color_greedy()
    assert C == 4


def _check_greedy(net, rule, order, col):
    adj = conflict_adjacency(net, rule)
    pos = np.empty(net.n_dev, int)
    pos[order] = np.arange(net.n_dev)
    for v in range(net.n_dev):
        for w in adj[v]:
            assert col[v] != col[w]
        earlier = {col[w] for w in adj[v] if pos[w] < pos[v]}
        m = 0
        while m in earlier:
            m += 1
        assert col[v] == m
    return adj


def _random_tiny(seed, n_dev=9, n_nodes=8, p_fixed=0.3):
    rng = np.random.default_rng(seed)
    fixed = (rng.random(n_nodes) < p_fixed).astype(int)
    fixed[0] = 1
    devs = rng.integers(0, n_nodes, size=(n_dev, 4))
    types = rng.choice([1, -1], n_dev)
    return tiny_net(f"rand{seed}", fixed, np.zeros(n_nodes), devs, types)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("rule", [0, 1, 2])
def test_random_tiny_graphs_valid_greedy_and_bounded_by_brute_force(seed, rule):
    net = _random_tiny(seed)
    o = oracle.Oracle(net, CARDS)
    order = np.random.default_rng(seed + 100).permutation(net.n_dev).astype(np.int32)
    for ordr in (None, order):
        col, C = o.color_greedy(rule=rule, order=ordr)
        adj = _check_greedy(net, rule, np.arange(net.n_dev) if ordr is None else ordr, col)
        chi = chromatic_number(adj)
        maxdeg = max((len(a) for a in adj), default=0)
        assert chi <= C <= maxdeg + 1
        assert C == (col.max() + 1 if net.n_dev else 0)


def test_greedy_is_optimal_on_cliques_paths_and_bfs_trees():
    # clique: k devices sharing one free node
    k = 7
    net = tiny_net("clique", [1, 0] + [1] * k, np.zeros(k + 2), [(1, 2 + i, 0, 0) for i in range(k)],
                   [1] * k)
    col, C = oracle.Oracle(net, CARDS).color_greedy()
    assert C == k and sorted(col.tolist()) == list(range(k))
    # path: device i joins free node i and i+1 -> 2 colours in natural order
    n = 8
    net = tiny_net("path", [1] + [0] * (n + 1), np.zeros(n + 2),
                   [(1 + i, 0, 2 + i, 0) for i in range(n)], [1] * n)
    assert oracle.Oracle(net, CARDS).color_greedy()[1] == 2
    # tree in BFS order: a free hub node per device level -> star of stars, bipartite
    devs = [(1, 0, 2, 0), (1, 0, 3, 0), (2, 0, 4, 0), (2, 0, 5, 0), (3, 0, 6, 0)]
    net = tiny_net("tree", [1] + [0] * 6, np.zeros(7), devs, [1] * 5)
    adj = conflict_adjacency(net)
    col, C = oracle.Oracle(net, CARDS).color_greedy()
    assert C == chromatic_number(adj)


def test_sram_clique_bounds_and_rules():
    net = netgen.sram(4, 6)
    o = oracle.Oracle(net, CARDS)
    c0 = o.color_greedy(rule=0)[1]
    c2 = o.color_greedy(rule=2)[1]
    c1 = o.color_greedy(rule=1)[1]
    # word line: 2 * cols access gates (rule 0); bit line: rows access drains (rule 2);
    # rule 1 adds the VDD rail: all 2 * rows * cols PMOS share it.
    assert c0 >= 2 * 6
    assert c2 >= 4 and c2 < c0
    assert c1 >= 2 * 4 * 6
    for rule in (0, 1, 2):
        col, _ = o.color_greedy(rule=rule)
        _check_greedy(net, rule, np.arange(net.n_dev), col)


def test_bad_order_is_rejected():
    o = oracle.Oracle(netgen.ota5t(), CARDS)
    with pytest.raises(ValueError):
        o.color_greedy(order=np.array([0, 1, 1, 2, 3], np.int32))
