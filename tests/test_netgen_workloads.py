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
