"""The sparse LU of eec_newton_dc (solver EEC_SOLVER_LU), checked on the CPU through the C ABI's
host check (no GPU): the multiple-minimum-degree order, the host factorisation with threshold partial
pivoting, and the GPU kernels' refactorisation and triangular solves executed on the host in the
GPU's order. Matrices are the oracle's MNA matrices of several netlist families.

* Backward stability: max|A x - b| / (max|A| max|x| + max|b|) at a few units of rounding, for
  matrices as conditioned as random node voltages make them (up to 1e19: the solutions of two
  correct solvers may then differ entirely, their backward errors may not).
* Accuracy where the problem allows it: with a 1e-3 S shunt on every node (the first stage of
  gshunt stepping) the matrices are well conditioned, and x agrees with a dense LU solve.
* Structure: the factor holds at least A's entries; a matrix with an empty row is singular.
"""
import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp

import netgen
import oracle

CARDS = netgen.default_cards()


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def _system(net, seed=2, shift=0.0, zero_x=False):
    o = oracle.Oracle(net, CARDS)
    rp, col, _ = o.pattern()
    x = np.zeros(o.n) if zero_x else netgen.random_x(net, seed=seed)
    r = o.eval_stamp(x)
    A = r["A"].copy()
    if shift:
        for i in range(o.n):
            A[rp[i] + int(np.nonzero(col[rp[i]:rp[i + 1]] == i)[0][0])] += shift
    return rp, col, A, r["b"]


NETS = [lambda: netgen.inverter_chain(64), netgen.ota5t, lambda: netgen.sram(12, 10),
        lambda: netgen.random_logic(600, seed=3), lambda: netgen.ripple_adder(16),
        lambda: netgen.insert_series_resistors(netgen.ripple_adder(4))]


@pytest.mark.parametrize("make", NETS)
def test_backward_stable_at_random_bias(eec, make):
    rp, col, A, b = _system(make())
    x, nnz_lu, bad = eec.eec_lu_check_host(rp, col, A, b)
    M = sp.csr_matrix((A, col, rp), shape=(len(rp) - 1,) * 2)
    be = np.abs(M @ x - b).max() / (np.abs(A).max() * np.abs(x).max() + np.abs(b).max())
    assert be <= 64 * np.finfo(float).eps, be
    assert nnz_lu >= len(col) and bad == -1


@pytest.mark.parametrize("make", NETS[:5])   # not the 1 mOhm resistors: 1000 S beside 1e-3 S
def test_solution_matches_dense_lu_when_well_conditioned(eec, make):
    rp, col, A, b = _system(make(), shift=1e-3)
    x, _, _ = eec.eec_lu_check_host(rp, col, A, b)
    M = sp.csr_matrix((A, col, rp), shape=(len(rp) - 1,) * 2).toarray()
    xr = la.solve(M, b)
    assert np.abs(x - xr).max() <= 1e-12 * np.abs(xr).max()


def test_zero_bias_and_mna_rails(eec):
    # x = 0 (all gates at ground: the start of a DC solve), and rails as MNA unknowns
    for net in (netgen.ripple_adder(8), netgen.sram(6, 6)):
        rp, col, A, b = _system(net, zero_x=True)
        x, _, _ = eec.eec_lu_check_host(rp, col, A, b)
        M = sp.csr_matrix((A, col, rp), shape=(len(rp) - 1,) * 2)
        assert np.abs(M @ x - b).max() <= 64 * np.finfo(float).eps * (
            np.abs(A).max() * np.abs(x).max() + np.abs(b).max())
    net = netgen.ripple_adder(4)
    o = oracle.Oracle(net, CARDS, rail_mode=1)
    rp, col, _ = o.pattern()
    xm = np.concatenate([netgen.Rng(7, 8).uniform(net.n_nodes - 1),
                         1e-4 * netgen.Rng(7, 9).normal(o.n - net.n_nodes + 1)])
    r = o.eval_stamp(xm)
    x, _, _ = eec.eec_lu_check_host(rp, col, r["A"], r["b"])
    M = sp.csr_matrix((r["A"], col, rp), shape=(o.n, o.n))
    assert np.abs(M @ x - r["b"]).max() <= 64 * np.finfo(float).eps * (
        np.abs(r["A"]).max() * np.abs(x).max() + np.abs(r["b"]).max())


def test_singular_and_malformed_inputs_are_rejected(eec):
    # row 1 has no entry at all: structurally singular
    rp = np.array([0, 2, 2, 4])
    col = np.array([0, 2, 0, 2])
    with pytest.raises(eec.EECError) as e:
        eec.eec_lu_check_host(rp, col, np.array([1.0, 2.0, 3.0, 4.0]), np.ones(3))
    assert e.value.code == eec.EEC_ENUMERIC
    with pytest.raises(eec.EECError) as e:
        eec.eec_lu_check_host(np.array([0, 1, 2]), np.array([0, 5]), np.ones(2), np.ones(2))
    assert e.value.code == eec.EEC_EINVAL


def test_too_much_fill_is_refused_before_memory_runs_out(eec):
    # randomly wired logic has no good elimination order: its factor would fill towards a dense
    # matrix (a 20,000-gate netlist: ~36,000 unknowns). The analysis stops at its entry budget
    # and reports EEC_ENOMEM within a second instead of exhausting host memory.
    import time
    rp, col, A, b = _system(netgen.random_logic(20_000, seed=3))
    t0 = time.perf_counter()
    with pytest.raises(eec.EECError) as e:
        eec.eec_lu_check_host(rp, col, A, b)
    assert e.value.code == eec.EEC_ENOMEM
    assert time.perf_counter() - t0 < 30


def _dc_pruned(net, seed=2, shift=0.0):
    """The DC system at random node voltages, with the pattern's entries that no DC stamp writes
    dropped (the gate rows: in DC only their diagonal's gshunt is nonzero)."""
    import scipy.sparse as sp
    rp, col, A, b = _system(net, seed=seed, shift=shift)
    n = len(rp) - 1
    M = sp.csr_matrix((A, col, rp), shape=(n, n))
    full = M.copy()
    M.eliminate_zeros()
    M.sort_indices()
    return full, M, b


def _backward_error(M, x, b):
    return np.abs(M @ x - b).max() / (np.abs(M.data).max() * np.abs(x).max() + np.abs(b).max())


def test_dc_pruned_pattern_shortens_the_lu_chains(eec):
    # The symmetric pattern keeps the gate rows, which DC never writes. Symbolically the word
    # lines then couple every bit line through the cells, and the factor's last columns form
    # a chain as long as the array is wide. Without those entries, the same minimum-degree
    # order leaves short chains in the refactorisation and in both substitutions.
    full, M, b = _dc_pruned(netgen.sram(64, 64))
    _, _, nnz_full, bad_f, d_full = eec.eec_lu_check_host_ex(full.indptr, full.indices, full.data, b)
    x, _, nnz_dc, bad_d, d_dc = eec.eec_lu_check_host_ex(M.indptr, M.indices, M.data, b)
    assert min(d_full) >= 60 and max(d_dc) <= 8, (d_full, d_dc)
    assert nnz_dc < 0.8 * nnz_full and bad_f == bad_d == -1
    assert _backward_error(M, x, b) <= 64 * np.finfo(float).eps


def test_dc_pruned_pattern_of_random_logic_factors(eec):
    # randomly wired logic: the full pattern's fill is refused; without the gate rows it factors
    full, M, b = _dc_pruned(netgen.random_logic(2000, seed=3))
    with pytest.raises(eec.EECError) as e:
        eec.eec_lu_check_host_ex(full.indptr, full.indices, full.data, b)
    assert e.value.code == eec.EEC_ENOMEM
    x, _, nnz, bad, _ = eec.eec_lu_check_host_ex(M.indptr, M.indices, M.data, b)
    assert nnz <= 8 * M.nnz and bad == -1
    assert _backward_error(M, x, b) <= 64 * np.finfo(float).eps


@pytest.mark.parametrize("make", [lambda: netgen.random_logic(600, seed=3),
                                  lambda: netgen.sram(12, 10), lambda: netgen.ripple_adder(8),
                                  lambda: netgen.concat(netgen.batch_circuits(16))])
def test_block_triangular_order(eec, make):
    # the order lists the strongly connected components of A's directed graph, each after every
    # component its edges reach: A(q, q) is block lower triangular
    from scipy.sparse.csgraph import connected_components
    _, M, b = _dc_pruned(make(), shift=1e-3)   # a shunt keeps long chains well conditioned
    x, q, nnz, bad, depth = eec.eec_lu_check_host_ex(M.indptr, M.indices, M.data, b,
                                                     order=eec.EEC_LU_ORDER_BTF)
    n = M.shape[0]
    assert np.array_equal(np.sort(q), np.arange(n))
    _, lab = connected_components(M, directed=True, connection="strong")
    pos = np.empty(n, np.int64)
    pos[q] = np.arange(n)
    first = {}
    for k in range(n):                      # each component's columns are consecutive in q
        first.setdefault(lab[q[k]], k)
    comp_pos = np.array([first[lab[i]] for i in range(n)])
    sizes = np.bincount(lab)
    for c, k0 in first.items():
        assert set(lab[q[k0:k0 + sizes[c]]]) == {c}
    C = M.tocoo()
    assert np.all(comp_pos[C.col] <= comp_pos[C.row])   # row i's columns in earlier components
    assert bad == -1 and _backward_error(M, x, b) <= 64 * np.finfo(float).eps


def test_unknown_order_is_rejected(eec):
    _, M, b = _dc_pruned(netgen.inverter_chain(8))
    with pytest.raises(eec.EECError) as e:
        eec.eec_lu_check_host_ex(M.indptr, M.indices, M.data, b, order=7)
    assert e.value.code == eec.EEC_EINVAL
