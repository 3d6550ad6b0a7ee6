"""C-ABI library checks that need no GPU: it builds, loads and exports every entry point declared
in include/eec.h; constants agree across header, binding and generators; host-side argument
validation; the library's host greedy colouring is bit-exact with the oracle's; the library's
host-built MNA pattern equals the oracle's (device upload is allowed to fail without a GPU)."""
import os
import re

import numpy as np
import pytest

import netgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eec.h")


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^EEC_API\s+[\w\s\*]+?\b(eec_\w+)\s*\(", text, flags=re.M)))


def header_defines():
    text = open(HEADER).read()
    return {k: int(v) for k, v in re.findall(r"#define\s+(EEC_\w+)\s+\(?(-?\d+)\)?", text)}


def test_library_exports_every_declared_entry_point(eec):
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(eec.lib, n), n
    assert sorted(eec.EXPORTED) == names
    out = os.popen(f"nm -D --defined-only {eec.LIB_PATH}").read().split()
    exported = sorted(s for s in out if s.startswith("eec_"))
    assert exported == names
    assert not [s for s in out if s.startswith("_ZN3eec")]   # internals stay hidden


def test_constants_agree(eec):
    d = header_defines()
    for k, v in d.items():
        if hasattr(eec, k):
            assert getattr(eec, k) == v, k
    assert d["EEC_CARD_LEN"] == netgen.CARD_LEN == oracle._load().ora_card_len()
    # the no-allocation backward's limit is written twice (header and binding): named here so
    # that a renamed or dropped copy fails instead of being skipped by the loop above
    assert d["EEC_NOALLOC_MAX_DEV"] == eec.EEC_NOALLOC_MAX_DEV


def _ctx_with(eec, net, rule=0, cards=None):
    ctx = eec.eec_create(conflict_rule=rule)
    eec.eec_upload_netlist(ctx, net.node_fixed, net.node_vfix, net.dev_nodes, net.dev_type,
                           net.W, net.L, net.model_id, net.res_nodes, net.res_G, net.isrc_nodes,
                           net.isrc_val, net.gshunt)
    eec.eec_set_model_cards(ctx, netgen.default_cards() if cards is None else cards)
    return ctx


def test_validation_errors(eec):
    net = netgen.ota5t()
    ctx = eec.eec_create()
    try:
        bad = net.dev_nodes.copy()
        bad[2, 1] = net.n_nodes
        with pytest.raises(eec.EECError) as e:
            eec.eec_upload_netlist(ctx, net.node_fixed, net.node_vfix, bad, net.dev_type, net.W,
                                   net.L, net.model_id)
        assert e.value.code == eec.EEC_EINVAL and "out of range" in str(e.value)
        with pytest.raises(eec.EECError):
            eec.eec_upload_netlist(ctx, net.node_fixed, net.node_vfix, net.dev_nodes,
                                   np.full(5, 2), net.W, net.L, net.model_id)
        with pytest.raises(eec.EECError):
            eec.eec_upload_netlist(ctx, net.node_fixed, net.node_vfix, net.dev_nodes,
                                   net.dev_type, -net.W, net.L, net.model_id)
        with pytest.raises(eec.EECError) as e:
            eec.eec_build_scatter(ctx)
        assert e.value.code == eec.EEC_ESTATE
        with pytest.raises(eec.EECError) as e:
            eec.eec_color(ctx, n_dev=5)
        assert e.value.code == eec.EEC_ESTATE
        eec.eec_upload_netlist(ctx, net.node_fixed, net.node_vfix, net.dev_nodes, net.dev_type,
                               net.W, net.L, net.model_id)
        with pytest.raises(eec.EECError):
            eec.eec_color(ctx, order=np.array([0, 1, 1, 2, 3]))
        bad_card = netgen.default_cards().copy()
        bad_card[0, netgen.CARD_FIELDS.index("TOX")] = 0.0
        with pytest.raises(eec.EECError):
            eec.eec_set_model_cards(ctx, bad_card)
        eec.eec_set_model_cards(ctx, netgen.default_cards()[:1])
        with pytest.raises(eec.EECError) as e:
            eec.eec_build_scatter(ctx)   # PMOS devices use card 1
        assert e.value.code == eec.EEC_EINVAL
        with pytest.raises(eec.EECError):
            eec.eec_set_variant(ctx, 7)
        for bad_order in (-1, 2):
            with pytest.raises(eec.EECError):
                eec.eec_set_eval_order(ctx, bad_order)
        eec.eec_set_eval_order(ctx, 0)
        eec.eec_set_eval_order(ctx, 1)
    finally:
        eec.eec_destroy(ctx)
    for bad in ({"host_chunks": -1}, {"host_chunks": 65}, {"block": 48}, {"conflict_rule": 3},
                {"color_stamp": 4}, {"color_stamp": -1}):
        with pytest.raises(eec.EECError):
            eec.eec_create(**bad)
    eec.eec_destroy(eec.eec_create(host_chunks=64))
    assert eec.eec_default_options().host_chunks == 0


def _color_cases():
    yield netgen.inverter_chain(40)
    yield netgen.ring_oscillator(11)
    yield netgen.ota5t()
    yield netgen.sram(8, 8)
    yield netgen.random_logic(3000, seed=5)
    yield netgen.concat(netgen.batch_circuits(20, seed=3))


@pytest.mark.parametrize("net", list(_color_cases()), ids=lambda n: n.name)
@pytest.mark.parametrize("rule", [0, 1, 2])
def test_host_greedy_bit_exact_with_oracle(eec, net, rule):
    if rule == 1 and net.n_dev > 2000:
        pytest.skip("rail cliques make the oracle's literal-rule colouring quadratic")
    o = oracle.Oracle(net, netgen.default_cards())
    ctx = _ctx_with(eec, net, rule)
    try:
        for order in (None, np.random.default_rng(1).permutation(net.n_dev).astype(np.int32)):
            col, C = eec.eec_color(ctx, order=order, n_dev=net.n_dev)
            ocol, oC = o.color_greedy(rule=rule, order=order)
            assert C == oC
            assert np.array_equal(col, ocol)
    finally:
        eec.eec_destroy(ctx)


@pytest.mark.parametrize("net", list(_color_cases()), ids=lambda n: n.name)
def test_host_pattern_equals_oracle_pattern(eec, net):
    o = oracle.Oracle(net, netgen.default_cards())
    ctx = _ctx_with(eec, net)
    try:
        eec.eec_color(ctx, n_dev=net.n_dev)
        try:
            eec.eec_build_scatter(ctx)
        except eec.EECError as e:          # no GPU here: the host part is still built
            assert e.code == eec.EEC_ECUDA
        rp, col, unk = eec.eec_get_pattern(ctx, net.n_nodes)
        orp, ocol, ounk = o.pattern()
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(unk, ounk)
        off = eec.eec_get_color_offsets(ctx)
        cols, C = o.color_greedy()
        assert np.array_equal(np.diff(off), np.bincount(cols, minlength=C))
    finally:
        eec.eec_destroy(ctx)


@pytest.mark.parametrize("rule", [0, 1, 2])
def test_coloring_verifier(eec, rule):
    # every rule gives a race-free DC schedule; only rules 0 and 1 also cover gate rows
    net = netgen.sram(6, 8)
    ctx = _ctx_with(eec, net, rule)
    try:
        eec.eec_color(ctx, n_dev=net.n_dev)
        try:
            eec.eec_build_scatter(ctx)
        except eec.EECError as e:
            assert e.code == eec.EEC_ECUDA
        eec.eec_verify_coloring(ctx, with_gate_rows=False)
        if rule == 2:
            with pytest.raises(eec.EECError) as e:
                eec.eec_verify_coloring(ctx, with_gate_rows=True)
            assert "share colour" in str(e.value)
        else:
            eec.eec_verify_coloring(ctx, with_gate_rows=True)
    finally:
        eec.eec_destroy(ctx)


def test_coloring_verifier_sees_conflicts_across_interleaved_colours(eec):
    # A (colour 0), B (colour 1), C (colour 0) all write row X once gate rows count: A and C
    # conflict there although B, of another colour, lies between them in device order.
    # Under the write-rows rule A conflicts with B (node Y) and C with neither.
    from helpers import tiny_net
    net = tiny_net("interleave", [1, 1, 0, 0, 0, 0], [0, 1.0, 0, 0, 0, 0],
                   [(3, 2, 0, 0), (2, 4, 3, 0), (5, 2, 0, 0)], [1, 1, 1])
    ctx = _ctx_with(eec, net, rule=2)
    try:
        col, C = eec.eec_color(ctx, n_dev=3)
        assert list(col) == [0, 1, 0]
        try:
            eec.eec_build_scatter(ctx)
        except eec.EECError as e:
            assert e.code == eec.EEC_ECUDA
        eec.eec_verify_coloring(ctx, with_gate_rows=False)
        with pytest.raises(eec.EECError) as e:
            eec.eec_verify_coloring(ctx, with_gate_rows=True)
        assert "share colour 0" in str(e.value)
    finally:
        eec.eec_destroy(ctx)


def test_batch_offsets_host(eec):
    nets = netgen.batch_circuits(12, seed=9)
    merged = netgen.concat(nets)
    ctx = eec.eec_create()
    try:
        eec.eec_upload_batch(ctx, nets)
        eec.eec_set_model_cards(ctx, netgen.default_cards())
        eec.eec_color(ctx, n_dev=merged.n_dev)
        try:
            eec.eec_build_scatter(ctx)
        except eec.EECError as e:
            assert e.code == eec.EEC_ECUDA
        rp, col, unk = eec.eec_get_pattern(ctx, merged.n_nodes)
        orp, ocol, _ = oracle.Oracle(merged, netgen.default_cards()).pattern()
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
        ro, no, do = eec.eec_get_batch_offsets(ctx, len(nets))
        assert np.array_equal(np.diff(ro), [m.n_free for m in nets])
        assert np.array_equal(np.diff(do), [m.n_dev for m in nets])
        assert no[-1] == len(col)
        # block diagonal: every column of circuit k's rows lies in circuit k's unknowns
        for k in range(len(nets)):
            r0, r1 = ro[k], ro[k + 1]
            c = col[rp[r0]:rp[r1]]
            assert c.min() >= r0 and c.max() < r1
            assert no[k] == rp[r0]
    finally:
        eec.eec_destroy(ctx)


def test_batch_create_equals_create_and_upload(eec):
    nets = netgen.batch_circuits(9, seed=4)
    merged = netgen.concat(nets)
    pats = []
    for make in (lambda: eec.eec_batch_create(nets, gshunt=1e-12),
                 lambda: _upload_batch(eec, nets)):
        ctx = make()
        try:
            eec.eec_set_model_cards(ctx, netgen.default_cards())
            eec.eec_color(ctx, n_dev=merged.n_dev)
            try:
                eec.eec_build_scatter(ctx)
            except eec.EECError as e:
                assert e.code == eec.EEC_ECUDA
            pats.append(eec.eec_get_pattern(ctx, merged.n_nodes))
        finally:
            eec.eec_destroy(ctx)
    for a, b in zip(*pats):
        assert np.array_equal(a, b)
    with pytest.raises(eec.EECError):
        eec.eec_batch_create([], gshunt=1e-12)
    with pytest.raises(eec.EECError):     # batched contexts take the eliminated rails only
        eec.eec_batch_create(nets, rail_mode=eec.EEC_RAIL_MNA_BRANCH)


def _upload_batch(eec, nets):
    ctx = eec.eec_create()
    eec.eec_upload_batch(ctx, nets)
    return ctx


def test_autograd_function_is_exposed(eec):
    import torch
    assert issubclass(eec.EvalStamp, torch.autograd.Function)
    assert eec.EvalStamp is eec.EvalStamp   # built once


def test_header_is_plain_c_and_a_c_program_links(eec, tmp_path):
    # the boundary is a C ABI: a C99 program sees only include/eec.h and _libeec.so
    import subprocess
    src = os.path.join(ROOT, "tests", "c_abi", "host_calls.c")
    exe = str(tmp_path / "host_calls")
    libdir = os.path.dirname(eec.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), src, "-o", exe, "-L", libdir,
                    "-l:_libeec.so", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stderr)


def test_binding_refuses_buffers_of_the_wrong_length(eec):
    # the C ABI takes bare pointers, so the binding checks every buffer's length against the
    # context before the call (a short buffer would be overrun on the device)
    import torch
    net = netgen.ota5t()
    ctx = _ctx_with(eec, net)
    try:
        eec.eec_color(ctx, n_dev=net.n_dev)
        try:
            eec.eec_build_scatter(ctx)
        except eec.EECError as e:
            assert e.code == eec.EEC_ECUDA
        nd, n, nnz, _ = eec.eec_get_sizes(ctx)
        z = lambda k: torch.zeros(k, dtype=torch.float64)
        with pytest.raises(ValueError, match="A has"):
            eec.eec_eval_stamp(ctx, z(n), z(nnz + 1), z(n))
        with pytest.raises(ValueError, match="q has"):
            eec.eec_eval_stamp(ctx, z(n), z(nnz), z(n), z(4 * nd - 1))
        with pytest.raises(TypeError):          # right lengths: refused only for not being on the GPU
            eec.eec_eval_stamp(ctx, z(n), z(nnz), z(n), z(4 * nd))
        with pytest.raises(ValueError, match="x has"):
            eec.eec_eval_stamp_host(ctx, np.zeros(n + 2), np.zeros(nnz), np.zeros(n))
        with pytest.raises(ValueError, match="gW has"):
            eec.eec_eval_stamp_bwd(ctx, z(n), z(nnz), z(n), z(n), z(nd + 1), z(nd))
        with pytest.raises(ValueError, match="q_prev has"):
            eec.eec_eval_stamp_tran(ctx, z(n), z(nd), None, 1e9, 0.0, z(nnz), z(n), z(4 * nd))
        with pytest.raises(ValueError, match="b has"):
            eec.eec_newton_dc(ctx, z(n), z(nnz), z(n - 1))
        with pytest.raises(ValueError, match="L has"):
            eec.eec_update_params(ctx, z(nd), z(nd + 3))
    finally:
        eec.eec_destroy(ctx)
