"""Pins of the oracle's EES-L1 device model (CPU only).

Each test checks a property that the model definition fixes independently of how the oracle
codes it: exact symmetries, conservation, limits in which the level reduces to the textbook
bulk-charge square law, one-term-at-a-time ratios, asymptotic slopes, and the dual-number
Jacobian against central differences.
"""
import math

import numpy as np
import pytest

import netgen
import oracle

KB, QE, EPS0 = 1.380649e-23, 1.602176634e-19, 8.8541878128e-12
VT = KB * 300.15 / QE
W0, L0 = 2e-6, 0.5e-6


def ev(card, p, V, W=W0, L=L0):
    return oracle.device_eval(card, p, W, L, np.asarray(V, float))


def chan_card(**kw):
    """Card with the junctions switched off so I_d is the channel current alone."""
    return netgen.card(JS=0.0, GMIN=0.0, **kw)


def ideal_card(**kw):
    """Card in which EES-L1 reduces to the bulk-charge square law: no velocity saturation,
    mobility degradation, DIBL, length modulation, Vdseff smoothing or phis smoothing."""
    base = dict(VSAT=1e30, UA=0.0, UB=0.0, ETA0=0.0, LAMBDA=0.0, DELTA=0.0, D1=0.0)
    base.update(kw)
    return chan_card(**base)


def cox(card):
    return 3.9 * EPS0 / card[netgen.CARD_FIELDS.index("TOX")]


def f(card, name):
    return float(card[netgen.CARD_FIELDS.index(name)])


def test_zero_vds_gives_zero_channel_current_exactly():
    c = chan_card()
    for vg in (-0.3, 0.2, 0.7, 1.2):
        for vs in (0.0, 0.3, 0.9):
            I, G, Q = ev(c, 1, [vs, vg, vs, 0.0])
            assert I[0] == 0.0 and I[2] == 0.0 and I[3] == 0.0
            assert np.all(np.isfinite(G))


def test_gate_current_and_gate_row_are_zero():
    rng = np.random.default_rng(1)
    for _ in range(20):
        V = rng.uniform(-0.2, 1.2, 4)
        I, G, Q = ev(netgen.card(), 1, V)
        assert I[1] == 0.0 and np.all(G[1] == 0.0)


@pytest.mark.parametrize("p", [1, -1])
def test_source_drain_swap_is_exact(p):
    rng = np.random.default_rng(2)
    c = netgen.default_cards()[0 if p > 0 else 1]
    for _ in range(50):
        V = rng.uniform(-0.1, 1.1, 4)
        if V[0] == V[2]:
            continue
        I, G, Q = ev(c, p, V)
        Is, Gs, Qs = ev(c, p, [V[2], V[1], V[0], V[3]])
        assert Is[0] == I[2] and Is[2] == I[0] and Is[3] == I[3]
        # Jacobian rows/columns swap accordingly
        perm = [2, 1, 0, 3]
        np.testing.assert_allclose(Gs, G[np.ix_(perm, perm)], rtol=1e-13, atol=1e-30)
        np.testing.assert_allclose(Qs, Q[perm], rtol=1e-13, atol=1e-30)


def test_pmos_is_the_mirror_of_nmos_with_the_same_card():
    rng = np.random.default_rng(3)
    c = netgen.card()
    for _ in range(50):
        V = rng.uniform(-1.2, 1.2, 4)
        In, Gn, Qn = ev(c, 1, V)
        Ip, Gp, Qp = ev(c, -1, -V)
        assert np.array_equal(Ip, -In)
        assert np.array_equal(Qp, -Qn)
        np.testing.assert_array_equal(Gp, Gn)   # dI/dV is even under the mirror


def test_terminal_currents_and_charges_sum_to_zero():
    rng = np.random.default_rng(4)
    for p, c in ((1, netgen.default_cards()[0]), (-1, netgen.default_cards()[1])):
        coxt = cox(c) * W0 * L0
        for _ in range(100):
            V = rng.uniform(-0.2, 1.2, 4)
            I, G, Q = ev(c, p, V)
            assert abs(I.sum()) <= 1e-15 * max(np.abs(I).max(), 1e-18)
            assert abs(Q.sum()) <= 1e-15 * coxt
            np.testing.assert_allclose(G.sum(axis=0), 0.0, atol=1e-15 * np.abs(G).max())


def test_square_law_limit_saturation_and_linear():
    c = ideal_card()
    vth0, k1, phi = f(c, "VTH0"), f(c, "K1"), f(c, "PHI")
    beta = f(c, "U0") * cox(c) * W0 / L0
    abulk = 1.0 + k1 / (2.0 * math.sqrt(phi))
    vgs = 1.5
    vg = vgs - vth0                      # Vgsteff in strong inversion (error ~ nVt e^-30)
    vgst2 = vg + 2 * VT
    vdsat = vgst2 / abulk
    I, _, _ = ev(c, 1, [2.0, vgs, 0.0, 0.0])
    np.testing.assert_allclose(I[0], beta * vg * vgst2 / (2 * abulk), rtol=1e-12)
    for vds in (0.05, 0.2, 0.5):
        assert vds < vdsat
        I, _, _ = ev(c, 1, [vds, vgs, 0.0, 0.0])
        np.testing.assert_allclose(I[0], beta * vg * vds * (1 - abulk * vds / (2 * vgst2)),
                                   rtol=1e-12)


def test_body_effect_limit():
    # D1 = 0: phis = PHI - vbs, Vth = VTH0 + K1 (sqrt(PHI - vbs) - sqrt(PHI)).
    c = ideal_card()
    vth0, k1, phi = f(c, "VTH0"), f(c, "K1"), f(c, "PHI")
    beta = f(c, "U0") * cox(c) * W0 / L0
    vbs, vgs = -0.5, 1.6
    sq = math.sqrt(phi - vbs)
    vth = vth0 + k1 * (sq - math.sqrt(phi))
    abulk = 1 + k1 / (2 * sq)
    vg = vgs - vth
    vgst2 = vg + 2 * VT
    I, _, _ = ev(c, 1, [2.5, vgs, 0.0, vbs])
    np.testing.assert_allclose(I[0], beta * vg * vgst2 / (2 * abulk), rtol=1e-12)
    Q = ev(c, 1, [2.5, vgs, 0.0, vbs])[2]
    np.testing.assert_allclose(Q[3], -cox(c) * W0 * L0 * k1 * sq, rtol=1e-13)


def test_mobility_degradation_ratio():
    ua, ub = 0.3, 0.04
    vgs, vds = 1.5, 0.1
    I0, _, _ = ev(ideal_card(), 1, [vds, vgs, 0.0, 0.0])
    I1, _, _ = ev(ideal_card(UA=ua, UB=ub), 1, [vds, vgs, 0.0, 0.0])
    vg = vgs - f(ideal_card(), "VTH0")
    np.testing.assert_allclose(I1[0] / I0[0], 1 / (1 + ua * vg + ub * vg * vg), rtol=1e-12)


def test_velocity_saturation_ratio_in_linear_region():
    vsat, vgs, vds = 1.1e5, 1.5, 0.05
    I0, _, _ = ev(ideal_card(), 1, [vds, vgs, 0.0, 0.0])
    I1, _, _ = ev(ideal_card(VSAT=vsat), 1, [vds, vgs, 0.0, 0.0])
    esatl = 2 * vsat * L0 / f(ideal_card(), "U0")
    np.testing.assert_allclose(I1[0] / I0[0], 1 / (1 + vds / esatl), rtol=1e-12)


def test_channel_length_modulation_ratio_in_saturation():
    lam, vgs, vds = 0.08, 1.5, 2.0
    c0, c1 = ideal_card(), ideal_card(LAMBDA=lam)
    I0, _, _ = ev(c0, 1, [vds, vgs, 0.0, 0.0])
    I1, _, _ = ev(c1, 1, [vds, vgs, 0.0, 0.0])
    abulk = 1 + f(c0, "K1") / (2 * math.sqrt(f(c0, "PHI")))
    vdsat = (vgs - f(c0, "VTH0") + 2 * VT) / abulk
    np.testing.assert_allclose(I1[0] / I0[0], 1 + lam * (f(c0, "LREF") / L0) * (vds - vdsat),
                               rtol=1e-12)


def test_smooth_vdseff_limits():
    # DELTA > 0: Vdseff -> vds for vds -> 0 with slope Vdsat / (Vdsat + DELTA); -> Vdsat deep in
    # saturation. Checked through the current ratio against the DELTA = 0 model.
    delta = 0.01
    c0, c1 = ideal_card(), ideal_card(DELTA=delta)
    vgs = 1.5
    abulk = 1 + f(c0, "K1") / (2 * math.sqrt(f(c0, "PHI")))
    vdsat = (vgs - f(c0, "VTH0") + 2 * VT) / abulk
    vds = 1e-7
    I0 = ev(c0, 1, [vds, vgs, 0, 0])[0][0]
    I1 = ev(c1, 1, [vds, vgs, 0, 0])[0][0]
    np.testing.assert_allclose(I1 / I0, vdsat / (vdsat + delta), rtol=1e-6)
    I0 = ev(c0, 1, [50.0, vgs, 0, 0])[0][0]
    I1 = ev(c1, 1, [50.0, vgs, 0, 0])[0][0]
    np.testing.assert_allclose(I1 / I0, 1.0, rtol=1e-5)


def test_subthreshold_slope():
    c = chan_card()
    nvt = f(c, "NFACT") * VT
    for vgs in (-0.5, -0.4):
        I, G, _ = ev(c, 1, [0.6, vgs, 0.0, 0.0])
        np.testing.assert_allclose(G[0, 1] / I[0], 1 / nvt, rtol=1e-6)


def test_dibl_ratio_in_deep_subthreshold():
    c = chan_card(LAMBDA=0.0, DELTA=1e-9)
    eta, nvt = f(c, "ETA0"), f(c, "NFACT") * VT
    I1 = ev(c, 1, [1.0, -0.5, 0.0, 0.0])[0][0]
    I2 = ev(c, 1, [2.0, -0.5, 0.0, 0.0])[0][0]
    np.testing.assert_allclose(I2 / I1, math.exp(eta / nvt), rtol=1e-6)


def test_junction_limiting_is_linear_above_40_vt():
    c = netgen.card()
    isat = f(c, "JS") * W0 * f(c, "HDIF")
    # NMOS with d = s = g = 0 V, body forward biased beyond 40 Vt: both junctions conduct.
    for z in (41.0, 55.0):
        vb = z * VT
        I, G, _ = ev(c, 1, [0.0, 0.0, 0.0, vb])
        ij = isat * (math.exp(40.0) * (1 + z - 40) - 1) + f(c, "GMIN") * vb
        np.testing.assert_allclose(I[3], 2 * ij, rtol=1e-13)
        np.testing.assert_allclose(G[3, 3], 2 * (isat * math.exp(40.0) / VT + f(c, "GMIN")),
                                   rtol=1e-13)


@pytest.mark.parametrize("p", [1, -1])
def test_jacobian_matches_central_differences(p):
    rng = np.random.default_rng(5 + p)
    c = netgen.default_cards()[0 if p > 0 else 1]
    h = 1e-6
    for _ in range(40):
        V = rng.uniform(-0.1, 1.1, 4)
        if abs(V[0] - V[2]) < 1e-3:
            continue
        I, G, _ = ev(c, p, V)
        Gfd = np.zeros((4, 4))
        for u in range(4):
            Vp, Vm = V.copy(), V.copy()
            Vp[u] += h
            Vm[u] -= h
            Gfd[:, u] = (ev(c, p, Vp)[0] - ev(c, p, Vm)[0]) / (2 * h)
        scale = np.abs(G).max()
        np.testing.assert_allclose(G, Gfd, rtol=1e-5, atol=1e-6 * scale)


def _intrinsic_split(V, p=1, **kw):
    """Drain and source charges with the overlaps switched off (forward mode: the mode drain is
    the physical drain)."""
    c = netgen.card(CGSO=0.0, CGDO=0.0, **kw)
    _, _, Q = ev(c, p, V)
    return Q[0], Q[2], f(c, "XPART")


def test_charge_partition_is_half_at_zero_vds():
    # fD = 1/2 - (1/2 - XPART) Vdseff / Vdsat with Vdseff = 0 at vds = 0: an even split
    for vg in (0.3, 0.7, 1.2):
        qd, qs, _ = _intrinsic_split([0.4, vg, 0.4, 0.0])
        assert qd != 0.0 and abs(qd - qs) <= 1e-15 * abs(qd)


def test_charge_partition_reaches_xpart_in_deep_saturation():
    # Vdseff -> Vdsat as vds grows, so the drain share of the inversion charge tends to XPART
    prev = None
    for vd in (1.0, 4.0, 16.0, 64.0):
        qd, qs, xpart = _intrinsic_split([vd, 1.0, 0.0, 0.0], JS=0.0)
        share = qd / (qd + qs)
        err = abs(share - xpart)
        if prev is not None:
            assert err < prev          # monotone approach
        prev = err
    assert prev < 1e-3


def test_charges_are_continuous_across_the_source_drain_swap():
    # the mode swap at vds = 0 moves no charge: with the partition above the terminal charges
    # are continuous in vds (a constant XPART split would jump by (1/2 - XPART) Qinv)
    c = netgen.default_cards()[0]
    for vg in (0.4, 0.9):
        for eps in (1e-6, 1e-8):
            _, _, qa = ev(c, 1, [0.5 + eps, vg, 0.5, 0.0])
            _, _, qb = ev(c, 1, [0.5 - eps, vg, 0.5, 0.0])
            coxt = cox(c) * W0 * L0
            assert np.abs(qa - qb).max() <= 10.0 * eps * coxt


def test_junctions_zero_bias_and_reverse_saturation():
    # d = g = s = ground, body at v: the two body junctions carry the whole current. It is
    # exactly zero at zero bias and saturates at -2 JS W HDIF in deep reverse bias (GMIN off).
    c = netgen.card(GMIN=0.0)
    I0, _, _ = ev(c, 1, [0.0, 0.0, 0.0, 0.0])
    assert np.all(I0 == 0.0)
    isat = f(c, "JS") * W0 * f(c, "HDIF")
    for v in (-2.0, -5.0):
        I, _, _ = ev(c, 1, [0.0, 0.0, 0.0, v])
        np.testing.assert_allclose(I[3], -2.0 * isat, rtol=1e-15)


def test_algorithmic_work_per_device():
    # the model's transcendental structure, counted by evaluating it on an operation-counting
    # scalar: softplus (one exp, one log1p), two junction expm1, and three square roots (the
    # body-effect smoothing and its square root, the smooth min of Vdseff); with source and
    # body held, the body-effect terms and the source junction are per-device constants
    c = netgen.default_cards()[0]
    V = np.array([0.8, 0.9, 0.1, 0.0])
    full = oracle.count_ops(c, 1, W0, L0, V)
    assert (full["exp"], full["log1p"], full["expm1"], full["sqrt"]) == (1, 1, 2, 3)
    held = oracle.count_ops(c, 1, W0, L0, V, free_mask=0b0011)
    assert (held["exp"], held["log1p"], held["expm1"], held["sqrt"]) == (1, 1, 1, 1)
    for k in ("add", "mul", "div"):
        assert 0 < held[k] < full[k]
    # a device with every terminal held does no voltage-dependent work
    assert sum(oracle.count_ops(c, 1, W0, L0, V, free_mask=0).values()) == 0
