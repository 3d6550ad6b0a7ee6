"""Seeded input generators (CPU): the counter-based SplitMix64 stream against the published
first outputs of SplitMix64 from state 0, determinism of every workload, and the sizes of the
workloads that the measurements quote."""
import numpy as np
import pytest

import netgen


def test_splitmix64_published_outputs_from_state_zero():
    # SplitMix64 (Steele, Lea, Flood 2014) started from state 0 begins 0xE220A8397B1DCDAF,
    # 0x6E789E6AA1B965F4, 0x06C45D188009454F
    r = netgen.Rng(0, 0).raw(3)
    assert [int(v) for v in r] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniforms_are_53_bit_and_streams_differ():
    u = netgen.Rng(7, 1).uniform(4096)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))
    assert not np.array_equal(netgen.Rng(7, 1).uniform(16), netgen.Rng(7, 2).uniform(16))
    # bulk draws and one-at-a-time draws walk the same stream
    a, b = netgen.Rng(3, 0), netgen.Rng(3, 0)
    one = [a.uniform1() for _ in range(5)]
    assert np.array_equal(np.array(one), b.uniform(5))


@pytest.mark.parametrize("k,n_dev,n_free", [(1, 128, 64), (2, 393_216, 131_840),
                                            (3, 719_548, 359_774), (5, 393_216, 131_840)])
def test_workload_sizes_and_determinism(k, n_dev, n_free):
    a, b = netgen.config(k), netgen.config(k)
    assert a.n_dev == n_dev and a.n_free == n_free
    for f in ("dev_nodes", "dev_type", "W", "L", "node_fixed", "node_vfix", "res_nodes", "res_G"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    c = netgen.config(k, seed=netgen.DEFAULT_SEED + 1)
    assert not np.array_equal(a.W, c.W)


def test_batch_of_4096_circuits():
    nets = netgen.batch_circuits(4096)
    merged = netgen.concat(nets)
    assert len(nets) == 4096 and merged.n_dev == 1_204_234
    assert merged.n_dev == sum(m.n_dev for m in nets)
    assert merged.n_free == sum(m.n_free for m in nets)


def test_sram_structure():
    # every word line drives the gates of the 2 access transistors of each cell in its row;
    # every bit line carries the access transistors of its column (at 256 x 256: 512 gates per
    # word line, 256 access transistors per bit line)
    rows, cols = 16, 24
    net = netgen.sram(rows, cols)
    assert net.n_dev == 6 * rows * cols
    wl = np.arange(4, 4 + rows)
    bl = np.arange(4 + rows, 4 + rows + 2 * cols)
    gates = np.bincount(net.dev_nodes[:, 1], minlength=net.n_nodes)
    assert np.all(gates[wl] == 2 * cols)
    ds = np.bincount(net.dev_nodes[:, 0], minlength=net.n_nodes) + \
        np.bincount(net.dev_nodes[:, 2], minlength=net.n_nodes)
    assert np.all(ds[bl] == rows)
    assert np.count_nonzero(net.dev_type < 0) == 2 * rows * cols


def test_random_logic_mix_fanout_and_order():
    n = 20_000
    net = netgen.random_logic(n, seed=11)
    gc = net.meta["gate_counts"]
    assert gc["inv"] + gc["nand2"] + gc["nor2"] == n
    for k, share in (("inv", 0.2), ("nand2", 0.4), ("nor2", 0.4)):   # drawn 1:2:2
        sd = (n * share * (1 - share)) ** 0.5
        assert abs(gc[k] - n * share) <= 5 * sd, (k, gc[k])
    assert net.n_dev == 2 * gc["inv"] + 4 * (gc["nand2"] + gc["nor2"])
    # each gate input is two device gates (the N and P of one input); a driver feeds at most 8
    free = net.node_fixed == 0
    gate_uses = np.bincount(net.dev_nodes[:, 1], minlength=net.n_nodes)
    assert np.all(gate_uses[free] % 2 == 0) and gate_uses[free].max() // 2 <= 8
    # a DAG: a gate's inputs come from primary inputs or from gates created before it
    d, g, s = net.dev_nodes[:, 0], net.dev_nodes[:, 1], net.dev_nodes[:, 2]
    out = np.maximum(d, s)
    assert np.all(~free[g] | (g < out))
