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
