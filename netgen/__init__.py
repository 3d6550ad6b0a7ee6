"""Seeded synthetic netlist generators shared by the oracle tests, the GPU tests and the bench.

This module holds inputs only: circuit topologies, device sizes, model-card data and random
node voltages. It contains none of the method's arithmetic (no model evaluation, no colouring,
no MNA pattern or stamping); both the oracle and the CUDA path derive those from the arrays
produced here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) in its counter form, so every stream is reproducible bit for bit on any
machine: draw i of a stream with key k is mix64(k + (i + 1) * 0x9E3779B97F4A7C15). A uniform is
(r >> 11) * 2^-53. Poisson draws use Knuth's product-of-uniforms method, normals Box-Muller.

Netlist conventions (the same arrays feed the C-ABI and the oracle):
  * node 0 is ground; ``node_fixed[i] == 1`` marks a node held by an ideal source at
    ``node_vfix[i]`` volts (ground is fixed at 0 V);
  * ``dev_nodes[k] = (d, g, s, b)``; ``dev_type[k]`` is +1 for NMOS, -1 for PMOS;
    ``model_id[k]`` indexes the model-card table;
  * resistors ``res_nodes[r] = (i, j)`` with conductance ``res_G[r]``;
  * current sources ``isrc_nodes[c] = (a, b)`` drive ``isrc_val[c]`` amperes from a to b
    through the source (out of node a, into node b).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

DEFAULT_SEED = 0x260403079
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = 0xD1B54A32D192ED03
_MASK64 = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based SplitMix64 stream; ``Rng(seed, stream)`` streams are independent."""

    _BLOCK = 1 << 14

    def __init__(self, seed: int = DEFAULT_SEED, stream: int = 0):
        self.key = np.uint64((seed ^ (stream * _STREAM_MUL)) & _MASK64)
        self.ctr = 0                 # draws consumed so far
        self._buf: List[float] = []  # pre-drawn uniforms for uniform1(), in stream order
        self._pos = 0

    def _raw_at(self, start: int, n: int) -> np.ndarray:
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return _mix64(self.key + i * _GOLDEN)

    def _sync(self) -> None:
        # Drop the unread part of the uniform1() buffer so bulk draws continue the stream.
        if self._pos < len(self._buf):
            self.ctr -= len(self._buf) - self._pos
        self._buf, self._pos = [], 0

    def raw(self, n: int) -> np.ndarray:
        self._sync()
        r = self._raw_at(self.ctr, n)
        self.ctr += n
        return r

    def uniform(self, n: int) -> np.ndarray:
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def uniform1(self) -> float:
        if self._pos == len(self._buf):
            self._buf = ((self._raw_at(self.ctr, self._BLOCK) >> np.uint64(11)).astype(np.float64)
                         * (1.0 / 9007199254740992.0)).tolist()
            self._pos = 0
            self.ctr += self._BLOCK
        v = self._buf[self._pos]
        self._pos += 1
        return v

    def poisson(self, lam: float) -> int:
        limit = math.exp(-lam)
        k, p = 0, 1.0
        while True:
            k += 1
            p *= self.uniform1()
            if p <= limit:
                return k - 1

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))          # 1 - u1 lies in (0, 1]
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]


# ---------------------------------------------------------------------------------------------
# Model cards of the EES-L1 level (data only; field order is the card layout of the C-ABI).
CARD_FIELDS = ("VTH0", "K1", "PHI", "NFACT", "U0", "UA", "UB", "VSAT", "TOX", "ETA0", "DELTA",
               "LAMBDA", "LREF", "JS", "HDIF", "CGSO", "CGDO", "XPART", "D1", "GMIN", "TEMP")
CARD_LEN = len(CARD_FIELDS)

_NMOS = dict(VTH0=0.40, K1=0.45, PHI=0.85, NFACT=1.40, U0=0.040, UA=0.30, UB=0.04, VSAT=1.1e5,
             TOX=1.8e-9, ETA0=0.06, DELTA=0.01, LAMBDA=0.08, LREF=1e-7, JS=1e-4, HDIF=2e-7,
             CGSO=2e-10, CGDO=2e-10, XPART=0.4, D1=0.01, GMIN=1e-12, TEMP=300.15)
_PMOS = dict(_NMOS, VTH0=0.42, K1=0.40, NFACT=1.45, U0=0.012, UA=0.25, UB=0.03, VSAT=0.9e5,
             ETA0=0.05, LAMBDA=0.10)


def card(**kw) -> np.ndarray:
    """One card as a float64 vector; ``kw`` overrides fields of the NMOS defaults."""
    d = dict(_NMOS, **kw)
    return np.array([d[f] for f in CARD_FIELDS], dtype=np.float64)


def default_cards() -> np.ndarray:
    """Card table [2, CARD_LEN]: row 0 NMOS, row 1 PMOS (PMOS values are in the p-frame)."""
    return np.stack([np.array([_NMOS[f] for f in CARD_FIELDS]),
                     np.array([_PMOS[f] for f in CARD_FIELDS])]).astype(np.float64)


# ---------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Netlist:
    name: str
    node_fixed: np.ndarray      # uint8 [n_nodes]
    node_vfix: np.ndarray       # float64 [n_nodes]
    dev_nodes: np.ndarray       # int32 [n_dev, 4]  (d, g, s, b)
    dev_type: np.ndarray        # int8 [n_dev]
    W: np.ndarray               # float64 [n_dev] metres
    L: np.ndarray               # float64 [n_dev] metres
    model_id: np.ndarray        # int32 [n_dev]
    res_nodes: np.ndarray       # int32 [n_res, 2]
    res_G: np.ndarray           # float64 [n_res]
    isrc_nodes: np.ndarray      # int32 [n_isrc, 2]
    isrc_val: np.ndarray        # float64 [n_isrc]
    gshunt: float = 1e-12       # conductance from every free node to ground
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.node_fixed.shape[0])

    @property
    def n_dev(self) -> int:
        return int(self.dev_nodes.shape[0])

    @property
    def n_free(self) -> int:
        return int(np.count_nonzero(self.node_fixed == 0))

    def free_nodes(self) -> np.ndarray:
        return np.nonzero(self.node_fixed == 0)[0].astype(np.int32)

    def with_sizes(self, W: np.ndarray, L: np.ndarray) -> "Netlist":
        return dataclasses.replace(self, W=np.ascontiguousarray(W, np.float64),
                                   L=np.ascontiguousarray(L, np.float64))


class _Builder:
    def __init__(self, name: str):
        self.name = name
        self.fixed: List[int] = []
        self.vfix: List[float] = []
        self.dev: List[tuple] = []
        self.typ: List[int] = []
        self.res: List[tuple] = []
        self.resG: List[float] = []
        self.isrc: List[tuple] = []
        self.ival: List[float] = []
        self.node(fixed=True, v=0.0)            # node 0 = ground

    def node(self, fixed: bool = False, v: float = 0.0) -> int:
        self.fixed.append(1 if fixed else 0)
        self.vfix.append(float(v) if fixed else 0.0)
        return len(self.fixed) - 1

    def nodes(self, n: int) -> np.ndarray:
        first = len(self.fixed)
        self.fixed.extend([0] * n)
        self.vfix.extend([0.0] * n)
        return np.arange(first, first + n, dtype=np.int64)

    def fet(self, typ: int, d: int, g: int, s: int, b: int):
        self.dev.append((d, g, s, b))
        self.typ.append(typ)

    def resistor(self, i: int, j: int, G: float):
        self.res.append((i, j))
        self.resG.append(G)

    def build(self, W: np.ndarray, L: np.ndarray, meta: Optional[dict] = None) -> Netlist:
        typ = np.asarray(self.typ, dtype=np.int8)
        dev = np.asarray(self.dev, dtype=np.int32).reshape(-1, 4)
        return Netlist(
            name=self.name,
            node_fixed=np.asarray(self.fixed, dtype=np.uint8),
            node_vfix=np.asarray(self.vfix, dtype=np.float64),
            dev_nodes=dev, dev_type=typ,
            W=np.ascontiguousarray(W, np.float64), L=np.ascontiguousarray(L, np.float64),
            model_id=np.where(typ > 0, 0, 1).astype(np.int32),
            res_nodes=np.asarray(self.res, dtype=np.int32).reshape(-1, 2),
            res_G=np.asarray(self.resG, dtype=np.float64),
            isrc_nodes=np.asarray(self.isrc, dtype=np.int32).reshape(-1, 2),
            isrc_val=np.asarray(self.ival, dtype=np.float64),
            meta=meta or {})


def _draw_wl(rng: Rng, n: int):
    """W ~ U[0.5, 5] um and L ~ U[0.1, 1] um: all W draws first, then all L draws."""
    W = 0.5e-6 + 4.5e-6 * rng.uniform(n)
    L = 0.1e-6 + 0.9e-6 * rng.uniform(n)
    return W, L


def _inverter_stages(b: _Builder, vdd: int, inp: int, outs) -> None:
    """Stage i: NMOS then PMOS, both driving outs[i] from the previous output."""
    prev = inp
    for o in outs:
        o = int(o)
        b.fet(+1, o, prev, 0, 0)
        b.fet(-1, o, prev, vdd, vdd)
        prev = o


def inverter_chain(n_stages: int = 64, seed: int = DEFAULT_SEED, vin: float = 0.0,
                   vdd: float = 1.0) -> Netlist:
    """CMOS inverter chain, stage-major device order (N_i, P_i); nodes 0 GND, 1 VDD, 2 VIN."""
    b = _Builder(f"inverter_chain_{n_stages}")
    nvdd = b.node(True, vdd)
    nin = b.node(True, vin)
    outs = b.nodes(n_stages)
    _inverter_stages(b, nvdd, nin, outs)
    W, L = _draw_wl(Rng(seed, 1), 2 * n_stages)
    return b.build(W, L, dict(vdd=vdd, vin=vin, in_node=nin, out_node=int(outs[-1])))


def ring_oscillator(n_stages: int = 11, seed: int = DEFAULT_SEED, vdd: float = 1.0) -> Netlist:
    """Ring of inverters: stage 0's input is the last stage's output."""
    b = _Builder(f"ring_{n_stages}")
    nvdd = b.node(True, vdd)
    outs = b.nodes(n_stages)
    _inverter_stages(b, nvdd, int(outs[-1]), outs)
    W, L = _draw_wl(Rng(seed, 2), 2 * n_stages)
    return b.build(W, L, dict(vdd=vdd, out_node=int(outs[-1])))


def ota5t(seed: int = DEFAULT_SEED, vdd: float = 1.0, vcm: float = 0.6, vbias: float = 0.5,
          sizes=None) -> Netlist:
    """Five-transistor OTA with a current-mirror load (M1..M5 in that order).

    M1/M2 NMOS differential pair (gates INP/INN, common source TAIL), M3/M4 PMOS mirror
    (M3 diode-connected at N1), M5 NMOS tail source (gate VBIAS)."""
    b = _Builder("ota5t")
    nvdd = b.node(True, vdd)
    inp = b.node(True, vcm)
    inn = b.node(True, vcm)
    vb = b.node(True, vbias)
    n1, out, tail = (int(v) for v in b.nodes(3))
    b.fet(+1, n1, inp, tail, 0)      # M1
    b.fet(+1, out, inn, tail, 0)     # M2
    b.fet(-1, n1, n1, nvdd, nvdd)    # M3
    b.fet(-1, out, n1, nvdd, nvdd)   # M4
    b.fet(+1, tail, vb, 0, 0)        # M5
    if sizes is None:
        W, L = _draw_wl(Rng(seed, 3), 5)
    else:
        W, L = sizes
    return b.build(W, L, dict(vdd=vdd, out_node=out))


def sram(rows: int = 256, cols: int = 256, seed: int = DEFAULT_SEED, vdd: float = 1.0,
         r_driver: float = 1e3) -> Netlist:
    """6T SRAM array; cells row-major, devices per cell PU1, PD1, PU2, PD2, AX1, AX2.

    Word lines and bit lines are free nodes, each driven through ``r_driver`` ohms from a fixed
    driver node (VWL, VBL). Node order: GND, VDD, VBL, VWL, WL[rows], (BL, BLB)[cols],
    (Q, QB)[rows*cols]."""
    b = _Builder(f"sram_{rows}x{cols}")
    nvdd = b.node(True, vdd)
    vbl = b.node(True, vdd)
    vwl = b.node(True, vdd)
    wl = b.nodes(rows)
    blp = b.nodes(2 * cols)
    qq = b.nodes(2 * rows * cols)
    G = 1.0 / r_driver
    for r in range(rows):
        b.resistor(int(wl[r]), vwl, G)
    for c in range(cols):
        b.resistor(int(blp[2 * c]), vbl, G)
        b.resistor(int(blp[2 * c + 1]), vbl, G)
    # Vectorised device table (same order as a row-major loop over cells).
    cell = np.arange(rows * cols)
    r = cell // cols
    c = cell % cols
    q = qq[2 * cell]
    qb = qq[2 * cell + 1]
    w = wl[r]
    bl = blp[2 * c]
    blb = blp[2 * c + 1]
    z = np.zeros_like(q)
    v = np.full_like(q, nvdd)
    per_cell = np.stack([
        np.stack([q, qb, v, v], 1),      # PU1
        np.stack([q, qb, z, z], 1),      # PD1
        np.stack([qb, q, v, v], 1),      # PU2
        np.stack([qb, q, z, z], 1),      # PD2
        np.stack([bl, w, q, z], 1),      # AX1
        np.stack([blb, w, qb, z], 1),    # AX2
    ], 1).reshape(-1, 4)
    types = np.tile(np.array([-1, 1, -1, 1, 1, 1], dtype=np.int8), rows * cols)
    b.dev = [tuple(x) for x in per_cell.tolist()]
    b.typ = types.tolist()
    W, L = _draw_wl(Rng(seed, 4), per_cell.shape[0])
    return b.build(W, L, dict(rows=rows, cols=cols, vdd=vdd))


_GATE_INV, _GATE_NAND2, _GATE_NOR2 = 0, 1, 2


def random_logic(n_gates: int = 200_000, seed: int = DEFAULT_SEED, n_pi: int = 64,
                 vdd: float = 1.0, fanout_mean: float = 3.0, fanout_cap: int = 8) -> Netlist:
    """Random DAG of INV/NAND2/NOR2 gates drawn 1:2:2.

    Each gate gets a fanout budget min(Poisson(fanout_mean), fanout_cap). Each gate input picks
    its driver among earlier gates with budget left, weighted by that budget (one token per unit
    of budget; the picked token is consumed); with no token left the input goes to one of
    ``n_pi`` fixed primary inputs. Gate templates (device order inside a gate):
      INV  : N(out, a, GND), P(out, a, VDD)
      NAND2: N1(out, a, x), N2(x, b, GND), P1(out, a, VDD), P2(out, b, VDD)
      NOR2 : P1(x, a, VDD), P2(out, b, x), N1(out, a, GND), N2(out, b, GND)
    NMOS bodies sit at GND and PMOS bodies at VDD."""
    rng = Rng(seed, 5)
    b = _Builder(f"random_logic_{n_gates}")
    nvdd = b.node(True, vdd)
    pi_v = (rng.uniform(n_pi) < 0.5) * vdd
    pis = [b.node(True, float(v)) for v in pi_v]
    pool: List[int] = []
    dev: List[tuple] = []
    typ: List[int] = []
    n_node = len(b.fixed)
    n_fixed = n_node
    counts = [0, 0, 0]
    for _ in range(n_gates):
        u = rng.uniform1()
        g = _GATE_INV if u < 0.2 else (_GATE_NAND2 if u < 0.6 else _GATE_NOR2)
        counts[g] += 1
        budget = min(rng.poisson(fanout_mean), fanout_cap)
        n_in = 1 if g == _GATE_INV else 2
        ins = []
        for _k in range(n_in):
            if pool:
                j = int(rng.uniform1() * len(pool))
                ins.append(pool[j])
                pool[j] = pool[-1]
                pool.pop()
            else:
                ins.append(pis[int(rng.uniform1() * n_pi)])
        out = n_node
        n_node += 1
        if g == _GATE_INV:
            a = ins[0]
            dev += [(out, a, 0, 0), (out, a, nvdd, nvdd)]
            typ += [1, -1]
        elif g == _GATE_NAND2:
            a, bb = ins
            x = n_node
            n_node += 1
            dev += [(out, a, x, 0), (x, bb, 0, 0), (out, a, nvdd, nvdd), (out, bb, nvdd, nvdd)]
            typ += [1, 1, -1, -1]
        else:
            a, bb = ins
            x = n_node
            n_node += 1
            dev += [(x, a, nvdd, nvdd), (out, bb, x, nvdd), (out, a, 0, 0), (out, bb, 0, 0)]
            typ += [-1, -1, 1, 1]
        pool.extend([out] * budget)
    b.fixed.extend([0] * (n_node - n_fixed))
    b.vfix.extend([0.0] * (n_node - n_fixed))
    b.dev = dev
    b.typ = typ
    W, L = _draw_wl(Rng(seed, 6), len(dev))
    return b.build(W, L, dict(n_gates=n_gates, gate_counts=dict(inv=counts[0], nand2=counts[1],
                                                                  nor2=counts[2])))


def _mirror_adder(b: _Builder, vdd: int, a: int, bb: int, cin: int):
    """Textbook 28-transistor mirror full adder (14 PMOS, 14 NMOS); returns (cout, sum) nodes.
    Carry: Coutb = NOT(maj(A, B, Cin)) by the mirror network; sum: Sb = NOT(sum) from Coutb;
    two output inverters. NMOS bodies at GND, PMOS bodies at VDD."""
    x1, x2, x3, x4, x5, y1, y2, y3, y4, y5, coutb, sb, cout, sm = (int(v) for v in b.nodes(14))
    P, N = (lambda d, g, s_: b.fet(-1, d, g, s_, vdd)), (lambda d, g, s_: b.fet(+1, d, g, s_, 0))
    # carry mirror
    P(x1, a, vdd); P(x1, bb, vdd); P(coutb, cin, x1); P(x2, a, vdd); P(coutb, bb, x2)
    N(y1, a, 0); N(y1, bb, 0); N(coutb, cin, y1); N(y2, a, 0); N(coutb, bb, y2)
    # sum mirror
    P(x3, a, vdd); P(x3, bb, vdd); P(x3, cin, vdd); P(sb, coutb, x3)
    P(x4, a, vdd); P(x5, bb, x4); P(sb, cin, x5)
    N(y3, a, 0); N(y3, bb, 0); N(y3, cin, 0); N(sb, coutb, y3)
    N(y4, a, 0); N(y5, bb, y4); N(sb, cin, y5)
    # output inverters
    P(cout, coutb, vdd); N(cout, coutb, 0)
    P(sm, sb, vdd); N(sm, sb, 0)
    return cout, sm


def ripple_adder(n_bits: int = 64, seed: int = DEFAULT_SEED, vdd: float = 1.0) -> Netlist:
    """n-bit ripple-carry adder of 28T mirror full adders (28 n MOSFETs). Operand bits A_k, B_k
    and the carry-in are fixed sources with seeded random 0/1 levels; bit k's carry-in is bit
    k-1's carry-out. Devices bit-major, in the order of _mirror_adder."""
    rng = Rng(seed, 9)
    b = _Builder(f"ripple_adder_{n_bits}")
    nvdd = b.node(True, vdd)
    lv = (rng.uniform(2 * n_bits + 1) < 0.5) * vdd
    ins = [b.node(True, float(v)) for v in lv]
    cin = ins[-1]
    sums = []
    for k in range(n_bits):
        cin, sm = _mirror_adder(b, nvdd, ins[2 * k], ins[2 * k + 1], cin)
        sums.append(sm)
    W, L = _draw_wl(Rng(seed, 10), len(b.dev))
    return b.build(W, L, dict(n_bits=n_bits, cout=cin, sums=sums))


def transistor_connections(net: Netlist) -> np.ndarray:
    """(device, terminal) pairs on a free node that at least two devices touch: the
    transistor-to-transistor connections where a series resistor can split a net."""
    nodes = net.dev_nodes
    free = net.node_fixed == 0
    devs_at = {}
    for k in range(net.n_dev):
        for t in range(4):
            v = int(nodes[k, t])
            if free[v]:
                devs_at.setdefault(v, set()).add(k)
    out = [(k, t) for k in range(net.n_dev) for t in range(4)
           if free[int(nodes[k, t])] and len(devs_at[int(nodes[k, t])]) >= 2]
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def insert_series_resistors(net: Netlist, per_group: Optional[int] = None, group_size: int = 28,
                            r_ohm: float = 1e-3, seed: int = DEFAULT_SEED) -> Netlist:
    """Move transistor terminals off shared nets through small series resistors (the paper's
    R14 / R89 netlists, Sec. II Benchmark 2): each selected (device, terminal) connection gets
    a new node tied to the original net by r_ohm. per_group None selects every connection;
    otherwise per_group connections drawn at random within each group of group_size devices
    (one full adder = 28 devices)."""
    conns = transistor_connections(net)
    if per_group is not None:
        rng = Rng(seed, 11)
        pick = []
        grp = conns[:, 0] // group_size
        for g in np.unique(grp):
            idx = np.nonzero(grp == g)[0]
            order = np.argsort(rng.uniform(len(idx)), kind="stable")
            pick.extend(idx[order[:per_group]].tolist())
        conns = conns[np.sort(np.asarray(pick, dtype=np.int64))]
    dev_nodes = net.dev_nodes.copy()
    n0 = net.n_nodes
    new = np.arange(n0, n0 + len(conns))
    res = np.stack([new, dev_nodes[conns[:, 0], conns[:, 1]]], 1)
    dev_nodes[conns[:, 0], conns[:, 1]] = new
    out = dataclasses.replace(
        net, name=f"{net.name}_R{len(conns)}",
        node_fixed=np.concatenate([net.node_fixed, np.zeros(len(conns), np.uint8)]),
        node_vfix=np.concatenate([net.node_vfix, np.zeros(len(conns))]),
        dev_nodes=dev_nodes.astype(np.int32),
        res_nodes=np.concatenate([net.res_nodes, res.astype(np.int32)]).reshape(-1, 2),
        res_G=np.concatenate([net.res_G, np.full(len(conns), 1.0 / r_ohm)]),
        meta=dict(net.meta, inserted=len(conns)))
    return out


def batch_circuits(n_circ: int = 4096, seed: int = DEFAULT_SEED) -> List[Netlist]:
    """Uneven sizing-candidate batch: 55% inverter chains (16..512 stages), 22.5% 11-stage
    rings, 22.5% 5T OTAs. Each circuit draws template sizes (W ~ U[0.5,5] um, L ~ U[0.1,1] um,
    separately for NMOS and PMOS) and scales every device's W and L by U[0.7, 1.3]."""
    rng = Rng(seed, 7)
    out: List[Netlist] = []
    for k in range(n_circ):
        u = rng.uniform1()
        if u < 0.55:
            stages = 16 + int(rng.uniform1() * 497)
            net = inverter_chain(stages, seed=seed + 1000 + k)
        elif u < 0.775:
            net = ring_oscillator(11, seed=seed + 1000 + k)
        else:
            net = ota5t(seed=seed + 1000 + k)
        t = rng.uniform(4)
        wn, ln_ = 0.5e-6 + 4.5e-6 * t[0], 0.1e-6 + 0.9e-6 * t[1]
        wp, lp = 0.5e-6 + 4.5e-6 * t[2], 0.1e-6 + 0.9e-6 * t[3]
        n = net.n_dev
        sw = 0.7 + 0.6 * rng.uniform(n)
        sl = 0.7 + 0.6 * rng.uniform(n)
        is_n = net.dev_type > 0
        W = np.where(is_n, wn, wp) * sw
        L = np.where(is_n, ln_, lp) * sl
        net = net.with_sizes(W, L)
        net.name = f"batch{k}_{net.name}"
        out.append(net)
    return out


def concat(nets: List[Netlist], name: str = "batch") -> Netlist:
    """Disjoint union of netlists: every circuit keeps its own nodes (ground of each circuit
    maps to the shared node 0). Returns the merged netlist; ``meta['node_off']`` holds the
    first node of each circuit (its ground excluded)."""
    fixed = [np.zeros(1, np.uint8) + 1]
    vfix = [np.zeros(1)]
    dev, typ, W, L, mid, res, resG, isn, isv, node_off = [], [], [], [], [], [], [], [], [], []
    nxt = 1
    for net in nets:
        m = np.arange(net.n_nodes, dtype=np.int64) - 1 + nxt
        m[0] = 0
        node_off.append(nxt)
        fixed.append(net.node_fixed[1:])
        vfix.append(net.node_vfix[1:])
        dev.append(m[net.dev_nodes])
        typ.append(net.dev_type)
        W.append(net.W)
        L.append(net.L)
        mid.append(net.model_id)
        res.append(m[net.res_nodes])
        resG.append(net.res_G)
        isn.append(m[net.isrc_nodes])
        isv.append(net.isrc_val)
        nxt += net.n_nodes - 1
    return Netlist(
        name=name, node_fixed=np.concatenate(fixed).astype(np.uint8),
        node_vfix=np.concatenate(vfix), dev_nodes=np.concatenate(dev).astype(np.int32),
        dev_type=np.concatenate(typ).astype(np.int8), W=np.concatenate(W), L=np.concatenate(L),
        model_id=np.concatenate(mid).astype(np.int32),
        res_nodes=np.concatenate(res).astype(np.int32).reshape(-1, 2),
        res_G=np.concatenate(resG), isrc_nodes=np.concatenate(isn).astype(np.int32).reshape(-1, 2),
        isrc_val=np.concatenate(isv), gshunt=nets[0].gshunt if nets else 1e-12,
        meta=dict(node_off=node_off, n_circ=len(nets)))


def shard(items, world: int, rank: int) -> list:
    """The share of rank `rank` among `world` ranks: every world-th item starting at `rank`
    (round robin, so circuits of uneven size spread evenly). The shares of the ranks partition
    the items; item i belongs to rank i % world, at position i // world of its share."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(items[rank::world])


def partition_rows(net: Netlist, k: int) -> List[Tuple[Netlist, np.ndarray]]:
    """Split the free nodes (in increasing order) into k contiguous blocks; part i keeps every
    node, so the unknowns keep their numbering, and every device, resistor and current source
    that touches one of its owned nodes. Each owned row of part i then receives all of its
    contributions: the rows a rank owning that block would stamp, after a halo exchange of the
    voltages of the other nodes its devices touch. Returns [(sub-netlist, owned node ids)]."""
    free = net.free_nodes()
    bounds = [len(free) * i // k for i in range(k + 1)]
    parts = []
    for i in range(k):
        owned = free[bounds[i]:bounds[i + 1]]
        mask = np.zeros(net.n_nodes, bool)
        mask[owned] = True
        d = mask[net.dev_nodes].any(axis=1)
        r = mask[net.res_nodes].any(axis=1) if len(net.res_nodes) else np.zeros(0, bool)
        c = mask[net.isrc_nodes].any(axis=1) if len(net.isrc_nodes) else np.zeros(0, bool)
        sub = dataclasses.replace(
            net, name=f"{net.name}_part{i}of{k}", dev_nodes=net.dev_nodes[d],
            dev_type=net.dev_type[d], W=net.W[d], L=net.L[d], model_id=net.model_id[d],
            res_nodes=net.res_nodes[r].reshape(-1, 2), res_G=net.res_G[r],
            isrc_nodes=net.isrc_nodes[c].reshape(-1, 2), isrc_val=net.isrc_val[c],
            meta=dict(net.meta, owned=owned))
        parts.append((sub, owned))
    return parts


def random_x(net: Netlist, seed: int = DEFAULT_SEED, lo: float = 0.0, hi: float = 1.0,
             stream: int = 8) -> np.ndarray:
    """Free-node voltages ~ U[lo, hi], one per free node in increasing node order."""
    return lo + (hi - lo) * Rng(seed, stream).uniform(net.n_free)


def config(k: int, seed: int = DEFAULT_SEED) -> Netlist:
    """The five workloads: 1 chain-64, 2 SRAM 256x256, 3 random logic 200k gates,
    4 batch of 4096 (merged), 5 = the SRAM of 2 (used with random upstream gradients)."""
    if k == 1:
        return inverter_chain(64, seed)
    if k in (2, 5):
        return sram(256, 256, seed)
    if k == 3:
        return random_logic(200_000, seed)
    if k == 4:
        return concat(batch_circuits(4096, seed))
    raise ValueError(k)
