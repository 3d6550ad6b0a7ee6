"""The segmented-reduction schedule's gather plan, checked on the CPU through the C ABI's host
check (no GPU). The plan is the layout of the buffer that the evaluation writes and the gather
reads.

* Every entry's items (its linear part, then its contributions) lie inside the buffer, and no
  two entries share an item.
* Light entries (fewer than 32 contributions) sit in their own window of 1,024 entries. Within a
  window they are sorted by their count, ties in entry order, 32 to a group. A group spans
  32 x (1 + its largest count) items.
* Heavy entries follow all windows, one contiguous run each, in entry order.
* The gather's reads, emulated from the plan as the kernel makes them, give every light entry
  the sum of its linear part and its contributions in that order, bit for bit. Heavy entries get
  a fixed lane-strided order.
"""
import numpy as np
import pytest

import netgen
import oracle

CARDS = netgen.default_cards()


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def _netlist_counts(net):
    """Contributions per A/b entry of a netlist, from the oracle's pattern: every device adds one
    to entry (row, column) for its free rows d, s, b and free columns, and one to b's row."""
    o = oracle.Oracle(net, CARDS)
    rp, col, unk = o.pattern()
    n, nnz = len(rp) - 1, len(col)
    a = unk[net.dev_nodes]
    key = np.repeat(np.arange(n), np.diff(rp)).astype(np.int64) * (n + 1) + col
    cnt = np.zeros(nnz + n, np.int64)
    for r in (0, 2, 3):
        m = a[:, r] >= 0
        np.add.at(cnt, nnz + a[m, r], 1)
        for u in range(4):
            mm = m & (a[:, u] >= 0)
            np.add.at(cnt, np.searchsorted(key, a[mm, r].astype(np.int64) * (n + 1) + a[mm, u]), 1)
    return cnt


def _emulate(eec, cnt, seed):
    """Fill the buffer as the evaluation does, run the gather's reads, and return (sums,
    expected light sums in serial order, the plan)."""
    plan = eec.eec_gather_plan_host(cnt)
    W, H = eec.EEC_GATHER_WINDOW, eec.EEC_GATHER_HEAVY
    rng = np.random.default_rng(seed)
    E = len(cnt)
    buf = np.zeros(plan["n_items"])
    owner = np.full(plan["n_items"], -1, np.int64)
    serial = np.zeros(E)
    for e in range(E):
        items = plan["item_of"][e] + plan["step_of"][e] * np.arange(1 + cnt[e])
        assert items.min() >= 0 and items.max() < plan["n_items"], e
        assert (owner[items] == -1).all(), e   # no item shared with another entry
        owner[items] = e
        vals = rng.normal(size=1 + cnt[e]) * np.exp(rng.normal(size=1 + cnt[e]))
        buf[items] = vals
        s = vals[0]
        for v in vals[1:]:
            s += v
        serial[e] = s
        assert plan["step_of"][e] == (32 if cnt[e] < H else 1)
    out = np.full(E, np.nan)
    for w in range(plan["woff"].shape[0]):
        for g in range(32):
            o0, o1 = plan["woff"][w, g], plan["woff"][w, g + 1]
            assert (o1 - o0) % 32 == 0 and o1 >= o0
            nr = (o1 - o0) // 32
            if nr == 0:
                continue
            rows = buf[o0:o1].reshape(nr, 32)
            s = rows[0].copy()
            for k in range(1, nr):
                s = s + rows[k]
            for lane in range(32):
                loc = plan["loc"][w, 32 * g + lane]
                if loc != 0xFFFF:
                    e = w * W + int(loc)
                    assert np.isnan(out[e]), e
                    out[e] = s[lane]
    for e, first, items in plan["heavy"]:
        part = np.array([sum(buf[first + lane:first + items:32], 0.0) for lane in range(32)])
        for off in (16, 8, 4, 2, 1):
            part = part + part[np.arange(32) ^ off]
        assert np.isnan(out[e]), e
        out[e] = part[0]
    return out, serial, plan


def _check(eec, cnt, seed=0):
    cnt = np.asarray(cnt, np.int64)
    W, H = eec.EEC_GATHER_WINDOW, eec.EEC_GATHER_HEAVY
    out, serial, plan = _emulate(eec, cnt, seed)
    light = cnt < H
    assert np.array_equal(out[light], serial[light])            # bit for bit, serial order
    np.testing.assert_allclose(out[~light], serial[~light], rtol=1e-12, atol=1e-12)
    # structure: per window, the light entries sorted by count (ties in entry order), 32 a group,
    # a group as long as its longest run; heavy entries in entry order after the windows
    E = len(cnt)
    for w in range(plan["woff"].shape[0]):
        ents = np.arange(w * W, min(E, (w + 1) * W))
        lt = ents[cnt[ents] < H]
        order = lt[np.lexsort((lt, cnt[lt]))]
        slots = plan["loc"][w].astype(np.int64)
        assert np.array_equal(slots[:len(order)] + w * W, order)
        assert (slots[len(order):] == 0xFFFF).all()
        for g in range((len(order) + 31) // 32):
            grp = order[32 * g:32 * g + 32]
            assert plan["woff"][w, g + 1] - plan["woff"][w, g] == 32 * (1 + cnt[grp].max())
    assert np.array_equal(plan["heavy"][:, 0], np.nonzero(~light)[0])
    if len(plan["heavy"]):
        assert plan["heavy"][0, 1] == (plan["woff"][-1, 32] if E else 0)
        assert np.array_equal(plan["heavy"][:, 2], 1 + cnt[~light])
    return plan


@pytest.mark.parametrize("E", [1, 31, 32, 33, 1023, 1024, 1025, 3000])
def test_window_and_group_boundaries(eec, E):
    rng = np.random.default_rng(E)
    _check(eec, rng.choice([0, 0, 1, 1, 2, 3, 5, 8], size=E), seed=E)


def test_heavy_entries_between_light_ones(eec):
    rng = np.random.default_rng(7)
    cnt = rng.choice([0, 1, 2, 3, 30, 31, 32, 33, 100, 2500], size=5000,
                     p=[.3, .3, .15, .1, .04, .04, .03, .02, .015, .005])
    plan = _check(eec, cnt, seed=7)
    assert len(plan["heavy"]) == np.count_nonzero(cnt >= 32) > 0


@pytest.mark.parametrize("make", [lambda: netgen.random_logic(3000, seed=5),
                                  lambda: netgen.sram(24, 16), netgen.ota5t])
def test_netlist_counts(eec, make):
    _check(eec, _netlist_counts(make()), seed=1)


def test_random_logic_pads_little(eec):
    # counts sorted within a window keep each group's entries of nearly equal length: on random
    # logic the zeros past the entries' ends are about 2 % of the buffer
    cnt = _netlist_counts(netgen.random_logic(3000, seed=5))
    plan = eec.eec_gather_plan_host(cnt)
    assert plan["n_items"] <= 1.03 * (len(cnt) + int(cnt.sum()))


def test_empty_and_invalid(eec):
    plan = eec.eec_gather_plan_host(np.zeros(0, np.int32))
    assert plan["n_items"] == 0 and plan["woff"].shape == (0, 33)
    with pytest.raises(eec.EECError) as e:
        eec.eec_gather_plan_host(np.array([1, -1, 2], np.int32))
    assert e.value.code == eec.EEC_EINVAL
