"""Small test-only helpers: netlist builders for hand-checkable circuits and a conflict-graph
brute force written independently of both the oracle and the CUDA library."""
from __future__ import annotations

import itertools

import numpy as np

import netgen


def tiny_net(name, fixed, vfix, devs, types, W=None, L=None, res=(), resG=(), isrc=(), ival=(),
             gshunt=1e-12):
    n = len(devs)
    W = np.full(n, 2e-6) if W is None else np.asarray(W, float)
    L = np.full(n, 0.5e-6) if L is None else np.asarray(L, float)
    types = np.asarray(types, np.int8)
    return netgen.Netlist(
        name=name, node_fixed=np.asarray(fixed, np.uint8), node_vfix=np.asarray(vfix, float),
        dev_nodes=np.asarray(devs, np.int32).reshape(-1, 4), dev_type=types, W=W, L=L,
        model_id=np.where(types > 0, 0, 1).astype(np.int32),
        res_nodes=np.asarray(res, np.int32).reshape(-1, 2), res_G=np.asarray(resG, float),
        isrc_nodes=np.asarray(isrc, np.int32).reshape(-1, 2), isrc_val=np.asarray(ival, float),
        gshunt=gshunt)


def conflict_adjacency(net, rule=0):
    """Adjacency sets of the device conflict graph, by brute force over device pairs."""
    n = net.n_dev
    sets = []
    for k in range(n):
        s = set()
        for t, node in enumerate(net.dev_nodes[k]):
            node = int(node)
            if rule == 1:
                ok = node != 0
            else:
                ok = net.node_fixed[node] == 0
            if rule == 2 and t == 1:
                ok = False
            if ok:
                s.add(node)
        sets.append(s)
    adj = [set() for _ in range(n)]
    for a, b in itertools.combinations(range(n), 2):
        if sets[a] & sets[b]:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def chromatic_number(adj):
    """Exact chromatic number by trying k = 1, 2, ... with backtracking (tiny graphs only)."""
    n = len(adj)
    if n == 0:
        return 0
    order = sorted(range(n), key=lambda v: -len(adj[v]))
    for k in range(1, n + 1):
        col = [-1] * n

        def bt(i):
            if i == n:
                return True
            v = order[i]
            for c in range(k):
                if all(col[w] != c for w in adj[v]):
                    col[v] = c
                    if bt(i + 1):
                        return True
                    col[v] = -1
            return False

        if bt(0):
            return k
    return n


# Parity records of this test session: per check, the cancellation-aware error, the plain
# relative error and how much the entries cancel (printed by conftest at the end of the run).
PARITY_LOG = []


def rel_err(got, ref, scale):
    """Cancellation-aware per-entry error |got - ref| / max(|ref|, scale). Also records, for the
    session summary, the plain relative error |got - ref| / |ref| (entries with ref != 0) and the
    ratio scale / |ref| (how far the entry's contributions cancel)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), scale)
    den = np.where(den == 0, 1.0, den)
    err = np.abs(got - ref) / den
    _record(got, ref, scale, err)
    return err


def _record(got, ref, scale, err):
    import os
    nz = ref != 0
    rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "n": int(ref.size),
           "max_err": float(err.max()) if err.size else 0.0}
    if nz.any():
        plain = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
        ratio = np.asarray(scale, np.float64)[nz] / np.abs(ref[nz]) if np.ndim(scale) else \
            np.full(int(nz.sum()), float(scale)) / np.abs(ref[nz])
        well = ratio <= 10.0
        rec.update(max_plain=float(plain.max()), p99_plain=float(np.quantile(plain, 0.99)),
                   p99_ratio=float(np.quantile(ratio, 0.99)), max_ratio=float(ratio.max()),
                   frac_ratio_gt10=float(1.0 - well.mean()),
                   max_plain_well=float(plain[well].max()) if well.any() else 0.0)
    PARITY_LOG.append(rec)
