"""The DC Newton loop on the GPU (eec_newton_dc: the library's evaluate-and-stamp, a sparse solve
-- cuSOLVER's QR, or the library's own sparse LU (EEC_SOLVER_LU) -- and a damped update) against
the oracle's DC operating point (dense LU Newton with the same damping and stopping rules). Both
loops stop at |dx| <= 1e-12 + 1e-9 |x| with a KCL residual below 1e-12 A, so their solutions
agree far inside 1e-8 relative. The library's sparse LU is also checked on its own (eec_lu_solve)
against its host check (the same plan and operations on the CPU)."""
import numpy as np
import pytest

import netgen
import oracle

pytestmark = pytest.mark.gpu
CARDS = netgen.default_cards()


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


# circuits on which the oracle's uniformly damped Newton converges from x = 0
CASES = [lambda: netgen.inverter_chain(64), lambda: netgen.inverter_chain(64, vin=0.45),
         netgen.ota5t, lambda: netgen.ring_oscillator(11), lambda: netgen.ripple_adder(4)]


@pytest.mark.parametrize("make", CASES)
@pytest.mark.parametrize("variant,rule,solver", [(2, 0, 0), (0, 0, 0), (2, 1, 0), (2, 0, 1),
                                                 (2, 0, 2), (2, 1, 2), (5, 1, 2)])
def test_gpu_newton_reaches_the_oracle_operating_point(eec, make, variant, rule, solver):
    import torch
    net = make()
    ref, _ = oracle.Oracle(net, CARDS).dc_solve()
    circ = eec.Circuit(net, CARDS, variant=variant)
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    A, b, _ = circ.new_outputs(want_q=False)
    it = eec.eec_newton_dc(circ.ctx, x, A, b, step_rule=rule, solver=solver)
    assert 1 <= it <= 200
    assert circ.status() == 0
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=1e-8, atol=1e-10)
    # A, b come back formed at the returned x: its KCL residual A x - b is below 1e-12 A
    rp, col, _ = circ.pattern()
    Ah = A.cpu().numpy()
    xh = x.cpu().numpy()
    r = np.array([Ah[rp[i]:rp[i + 1]] @ xh[col[rp[i]:rp[i + 1]]] for i in range(circ.n)])
    assert np.abs(r - b.cpu().numpy()).max() <= 1e-12


def test_gpu_newton_reports_non_convergence_without_a_device_error(eec):
    # one solve per stage: plain Newton, gshunt stepping, and Newton after the relaxation start
    # all stop short (the ring's Jacobi sweeps oscillate instead of settling)
    import torch
    net = netgen.ring_oscillator(11)
    circ = eec.Circuit(net, CARDS)
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    A, b, _ = circ.new_outputs(want_q=False)
    with pytest.raises(eec.EECError) as e:
        eec.eec_newton_dc(circ.ctx, x, A, b, max_iter=1)
    assert e.value.code == eec.EEC_ENOCONV
    assert circ.status() == 0
    assert eec.eec_newton_info(circ.ctx)["path"] == 3
    it = eec.eec_newton_dc(circ.ctx, x, A, b)    # continues from the last iterate
    assert it >= 1


@pytest.mark.parametrize("solver", [0, 2])
@pytest.mark.parametrize("make,rail_mode,max_iter", [(lambda: netgen.inverter_chain(64), 0, 150),
                                                     (lambda: netgen.inverter_chain(64), 1, 300)])
def test_gshunt_stepping_where_plain_newton_fails(eec, make, rail_mode, max_iter, solver):
    # plain damped Newton does not converge on these from the start below (the oracle needs its
    # gshunt-stepping fallback too); the GPU loop falls back the same way and reaches the
    # oracle's operating point. Solves needed (whole-step scaling, counted with the oracle's
    # stamps and a sparse LU): rails eliminated, plain Newton 170 and the stages at most 120;
    # rails as unknowns, plain Newton none within 600 and the 1e-4 S stage 194-207 depending on
    # the rounding of A and b -- so that case gets 300 solves per stage, not a limit inside that
    # spread (the atomic schedule's rounding varies from run to run).
    import torch
    net = make()
    o = oracle.Oracle(net, CARDS, rail_mode=rail_mode)
    x0 = np.zeros(o.n)
    if rail_mode:
        R = [i for i in range(1, net.n_nodes) if net.node_fixed[i]]
        x0[np.array(R) - 1] = net.node_vfix[R]
    ref, _ = o.dc_solve(x0=x0, max_iter=max_iter)
    circ = eec.Circuit(net, CARDS, variant=2, rail_mode=rail_mode)
    x = torch.as_tensor(x0, device="cuda")
    A, b, _ = circ.new_outputs(want_q=False)
    it = eec.eec_newton_dc(circ.ctx, x, A, b, max_iter=max_iter, solver=solver)
    if solver == 0:
        assert it > max_iter            # the plain run used its solves, then the stages
    assert circ.status() == 0
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("make", [lambda: netgen.ripple_adder(16), lambda: netgen.sram(12, 10),
                                  lambda: netgen.random_logic(600, seed=3),
                                  lambda: netgen.inverter_chain(200), lambda: netgen.sram(64, 64)])
def test_sparse_lu_solve_matches_its_host_check(eec, make):
    # the GPU kernels (refactorisation, triangular solves) against the same plan and operations
    # executed on the host, on matrices stamped by the GPU; backward stability as the host LU.
    # The 64 x 64 SRAM's factor (78,080 entries) does not fit in shared memory: the kernel's
    # global-memory form.
    import torch
    import scipy.sparse as sp
    net = make()
    circ = eec.Circuit(net, CARDS, variant=2)
    rp, col, _ = circ.pattern()
    for seed in (2, 3):
        xv = torch.as_tensor(netgen.random_x(net, seed=seed), device="cuda")
        A, b, _ = circ.eval_stamp(xv, want_q=False)
        x = torch.empty_like(b)
        eec.eec_lu_solve(circ.ctx, A, b, x)
        Ah, bh, xg = A.cpu().numpy(), b.cpu().numpy(), x.cpu().numpy()
        M = sp.csr_matrix((Ah, col, rp), shape=(circ.n, circ.n))
        be = np.abs(M @ xg - bh).max() / (np.abs(Ah).max() * np.abs(xg).max() + np.abs(bh).max())
        assert be <= 64 * np.finfo(float).eps, be
        xh, nnz_lu, _ = eec.eec_lu_check_host(rp, col, Ah, bh)
        if np.linalg.cond(M.toarray()) < 1e8:
            assert np.abs(xg - xh).max() <= 1e-10 * np.abs(xh).max()
    nnz_lu_ctx, analyses = eec.eec_lu_stats(circ.ctx)
    assert nnz_lu_ctx >= circ.nnz and analyses >= 1


def test_sparse_lu_newton_on_the_64_bit_adder(eec):
    # NEXT-2 with the library's sparse LU: the 64-bit adder of Table II (896 unknowns) reaches
    # the oracle's operating point; its per-iteration time is reported by bench.py --newton
    import torch
    net = netgen.ripple_adder(64)
    ref, _ = oracle.Oracle(net, CARDS).dc_solve(max_iter=400)
    for rule in (0, 1):
        circ = eec.Circuit(net, CARDS, variant=2)
        x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
        A, b, _ = circ.new_outputs(want_q=False)
        it = eec.eec_newton_dc(circ.ctx, x, A, b, max_iter=400, step_rule=rule,
                               solver=eec.EEC_SOLVER_LU)
        assert it >= 1 and circ.status() == 0
        np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("n_stages,rail_mode", [(1024, 0), (4096, 0), (1024, 1)])
def test_long_chain_converges_through_the_relaxation_start(eec, n_stages, rail_mode):
    # From x = 0 the exact Newton step of a long inverter chain grows like the stage gain to the
    # power of the chain length (inf in doubles beyond a few hundred stages); plain Newton and
    # gshunt stepping both fail, and the relaxation start (Jacobi sweeps, one stage settled per
    # sweep) hands Newton a start from which it converges. The oracle's own DC solve fails on
    # these chains (its dense LU meets a zero pivot at 4096 stages), so its model checks the
    # result instead: the oracle's KCL residual at the returned x is at the level of rounding,
    # and the chain's unique operating point alternates between the rails (input at 0 V).
    import torch
    net = netgen.inverter_chain(n_stages)
    o = oracle.Oracle(net, CARDS, rail_mode=rail_mode)
    x0 = np.zeros(o.n)
    circ = eec.Circuit(net, CARDS, variant=2, rail_mode=rail_mode)
    x = torch.as_tensor(x0, device="cuda")
    A, b, _ = circ.new_outputs(want_q=False)
    it = eec.eec_newton_dc(circ.ctx, x, A, b, max_iter=100, step_rule=1, solver=eec.EEC_SOLVER_LU)
    info = eec.eec_newton_info(circ.ctx)
    assert circ.status() == 0 and it == info["solves"] >= 1
    if rail_mode == 0:
        assert info["path"] >= 2 and n_stages <= info["sweeps"] <= 4 * o.n + 1024
    xh = x.cpu().numpy()
    assert np.abs(o.kcl_residual(xh)).max() <= 1e-11
    _, _, unk = circ.pattern()
    v = xh[unk[3:3 + n_stages]]            # stage outputs: nodes 3, 4, ... (0 ground, 1 vdd, 2 in)
    assert np.abs(v - (np.arange(n_stages) % 2 == 0)).max() < 0.05


def test_sram_dc_point_through_the_multi_block_lu(eec):
    # the 64 x 64 SRAM's factor (78,080 entries) does not fit in one block's shared memory, so
    # every solve runs the cooperative kernel over all SMs; plain Newton and gshunt stepping from
    # x = 0 fail on the array of bistable cells and the relaxation start hands Newton a point
    # from which it converges. The oracle's dense LU is too slow at 8,384 unknowns, so its
    # model checks the result: its KCL residual at the returned point is at rounding level.
    import torch
    net = netgen.sram(64, 64)
    circ = eec.Circuit(net, CARDS, variant=2)
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    A, b, _ = circ.new_outputs(want_q=False)
    it = eec.eec_newton_dc(circ.ctx, x, A, b, max_iter=100, step_rule=1, solver=eec.EEC_SOLVER_LU)
    info = eec.eec_newton_info(circ.ctx)
    assert circ.status() == 0 and it == info["solves"] >= 1
    nnz_lu, _ = eec.eec_lu_stats(circ.ctx)
    assert 8 * nnz_lu > 227 * 1024            # the factor lives in global memory
    F = oracle.Oracle(net, CARDS).kcl_residual(x.cpu().numpy())
    assert np.abs(F).max() <= 1e-11


def test_batch_of_circuits_dc_points_in_one_newton_loop(eec):
    # 48 circuits of config 4's mix as one block-diagonal system: one Newton loop (its tests take
    # the maximum over every circuit's nodes) reaches every circuit's operating point. Each block
    # is checked with the oracle's model on its own circuit: the KCL residual of its nodes at the
    # returned point is at rounding level.
    import torch
    nets = netgen.batch_circuits(48, seed=11)
    circ = eec.Circuit(None, CARDS, color=True, batch=nets)
    x = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    A, b, _ = circ.new_outputs(want_q=False)
    it = eec.eec_newton_dc(circ.ctx, x, A, b, max_iter=300, step_rule=1, solver=eec.EEC_SOLVER_LU)
    assert it >= 1 and circ.status() == 0
    ro, _, _ = eec.eec_get_batch_offsets(circ.ctx, len(nets))
    xh = x.cpu().numpy()
    for k, net in enumerate(nets):
        F = oracle.Oracle(net, CARDS).kcl_residual(xh[ro[k]:ro[k + 1]])
        assert np.abs(F).max() <= 1e-11, k
