"""ctypes front end of the serial CPU oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers. The product library never imports this package.

Every function mirrors the C symbol of the same name with ``ora_`` dropped; arrays are numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

ENOCONV = -6


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (portable flags: it runs on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                        _SRC],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.ora_create.restype = P
            lib.ora_create.argtypes = [i32, P, P, i32, P, P, P, P, P, i32, P, P, i32, P, P, f64,
                                       i32, P, i32]
            lib.ora_destroy.argtypes = [P]
            lib.ora_n_unknowns.restype = i32
            lib.ora_n_unknowns.argtypes = [P]
            lib.ora_nnz.restype = i64
            lib.ora_nnz.argtypes = [P]
            lib.ora_pattern.argtypes = [P, P, P, P]
            lib.ora_set_sizes.argtypes = [P, P, P]
            lib.ora_eval_stamp.argtypes = [P, P, P, P, P, P, P]
            lib.ora_kcl_residual.argtypes = [P, P, P]
            lib.ora_color_greedy.argtypes = [P, i32, P, P, P]
            lib.ora_dc_solve.argtypes = [P, P, i32, P, P]
            lib.ora_adjoint.argtypes = [P, P, i32, P]
            lib.ora_eval_stamp_grad.argtypes = [P, P, P, P, P, P, P]
            lib.ora_device_eval.argtypes = [P, i32, f64, f64, P, P, P, P]
            lib.ora_card_len.restype = i32
            lib.ora_eval_stamp_tran.argtypes = [P, P, P, P, f64, f64, P, P, P, P, P, P]
            lib.ora_device_charge.argtypes = [P, i32, f64, f64, P, P, P]
            lib.ora_tran_solve.argtypes = [P, P, f64, i32, i32, P, P]
            lib.ora_count_ops.argtypes = [P, i32, f64, f64, P, i32, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Oracle:
    """Oracle context for one netlist (see ``netgen.Netlist``) and a card table.

    ``rail_mode`` 0 eliminates the held nodes; 1 is modified nodal analysis: every non-ground
    node is an unknown, followed by one source-current unknown per held node in node order."""

    def __init__(self, net, cards, rail_mode=0):
        lib = _load()
        self._keep = dict(
            fixed=_c(net.node_fixed, np.uint8), vfix=_c(net.node_vfix, np.float64),
            dev=_c(net.dev_nodes, np.int32), typ=_c(net.dev_type, np.int8),
            W=_c(net.W, np.float64), L=_c(net.L, np.float64), mid=_c(net.model_id, np.int32),
            rn=_c(net.res_nodes, np.int32), rG=_c(net.res_G, np.float64),
            sn=_c(net.isrc_nodes, np.int32), sI=_c(net.isrc_val, np.float64),
            cards=_c(cards, np.float64))
        k = self._keep
        self.n_dev = int(k["dev"].shape[0])
        self.h = lib.ora_create(
            int(k["fixed"].shape[0]), _p(k["fixed"]), _p(k["vfix"]), self.n_dev, _p(k["dev"]),
            _p(k["typ"]), _p(k["W"]), _p(k["L"]), _p(k["mid"]), int(k["rG"].shape[0]),
            _p(k["rn"]), _p(k["rG"]), int(k["sI"].shape[0]), _p(k["sn"]), _p(k["sI"]),
            float(net.gshunt), int(k["cards"].shape[0]), _p(k["cards"]), int(rail_mode))
        if not self.h:
            raise ValueError("oracle rejected the netlist")
        self.lib = lib
        self.n = int(lib.ora_n_unknowns(self.h))
        self.nnz = int(lib.ora_nnz(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.ora_destroy(self.h)
            self.h = None

    def pattern(self):
        rp = np.zeros(self.n + 1, np.int32)
        col = np.zeros(self.nnz, np.int32)
        unk = np.zeros(self._keep["fixed"].shape[0], np.int32)
        self.lib.ora_pattern(self.h, _p(rp), _p(col), _p(unk))
        return rp, col, unk

    def set_sizes(self, W, L):
        self._keep["W"] = _c(W, np.float64)
        self._keep["L"] = _c(L, np.float64)
        self.lib.ora_set_sizes(self.h, _p(self._keep["W"]), _p(self._keep["L"]))

    def eval_stamp(self, x, want_q=False, want_scale=False):
        x = _c(x, np.float64)
        A = np.zeros(self.nnz)
        b = np.zeros(self.n)
        q = np.zeros(4 * self.n_dev) if want_q else None
        As = np.zeros(self.nnz) if want_scale else None
        bs = np.zeros(self.n) if want_scale else None
        self.lib.ora_eval_stamp(self.h, _p(x), _p(A), _p(b), _p(q), _p(As), _p(bs))
        out = dict(A=A, b=b)
        if want_q:
            out["q"] = q.reshape(4, self.n_dev)
        if want_scale:
            out["A_scale"], out["b_scale"] = As, bs
        return out

    def kcl_residual(self, x):
        x = _c(x, np.float64)
        F = np.zeros(self.n)
        self.lib.ora_kcl_residual(self.h, _p(x), _p(F))
        return F

    def color_greedy(self, rule=0, order=None):
        col = np.zeros(self.n_dev, np.int32)
        C = ctypes.c_int32(0)
        o = None if order is None else _c(order, np.int32)
        rc = self.lib.ora_color_greedy(self.h, int(rule), _p(o), _p(col), ctypes.byref(C))
        if rc != 0:
            raise ValueError("bad colouring arguments")
        return col, int(C.value)

    def dc_solve(self, x0=None, max_iter=200, history=False):
        x = np.zeros(self.n) if x0 is None else _c(x0, np.float64).copy()
        hist = np.zeros((max_iter + 1) * self.n) if history else None
        nh = ctypes.c_int32(0)
        it = self.lib.ora_dc_solve(self.h, _p(x), int(max_iter), _p(hist), ctypes.byref(nh))
        if it == ENOCONV:
            raise RuntimeError("oracle DC Newton did not converge")
        if history:
            return x, int(it), hist[: nh.value * self.n].reshape(nh.value, self.n)
        return x, int(it)

    def adjoint(self, x, out_unknown):
        lam = np.zeros(self.n)
        rc = self.lib.ora_adjoint(self.h, _p(_c(x, np.float64)), int(out_unknown), _p(lam))
        if rc != 0:
            raise ValueError("adjoint solve failed")
        return lam

    def eval_stamp_tran(self, x, qprev, iprev, alpha, beta, want_scale=False):
        """Transient companion stamp at x; returns A, b, q (charges at x), i (capacitive
        currents at x) and, on request, the |contribution| scales."""
        x = _c(x, np.float64)
        qp = _c(qprev, np.float64).reshape(-1)
        ip = None if iprev is None else _c(iprev, np.float64).reshape(-1)
        A = np.zeros(self.nnz)
        b = np.zeros(self.n)
        q = np.zeros(4 * self.n_dev)
        i = np.zeros(4 * self.n_dev)
        As = np.zeros(self.nnz) if want_scale else None
        bs = np.zeros(self.n) if want_scale else None
        self.lib.ora_eval_stamp_tran(self.h, _p(x), _p(qp), _p(ip), float(alpha), float(beta),
                                     _p(A), _p(b), _p(q), _p(i), _p(As), _p(bs))
        out = dict(A=A, b=b, q=q.reshape(4, self.n_dev), i=i.reshape(4, self.n_dev))
        if want_scale:
            out["A_scale"], out["b_scale"] = As, bs
        return out

    def tran_solve(self, x0, h, n_steps, method=0, i0=None):
        x = _c(x0, np.float64).copy()
        traj = np.zeros((n_steps + 1) * self.n)
        ip = None if i0 is None else _c(i0, np.float64).reshape(-1)
        rc = self.lib.ora_tran_solve(self.h, _p(x), float(h), int(n_steps), int(method), _p(ip),
                                     _p(traj))
        if rc != 0:
            raise RuntimeError("oracle transient step did not converge")
        return traj.reshape(n_steps + 1, self.n)

    def eval_stamp_grad(self, x, gA, gb):
        gx = np.zeros(self.n)
        gW = np.zeros(self.n_dev)
        gL = np.zeros(self.n_dev)
        self.lib.ora_eval_stamp_grad(self.h, _p(_c(x, np.float64)), _p(_c(gA, np.float64)),
                                     _p(_c(gb, np.float64)), _p(gx), _p(gW), _p(gL))
        return gx, gW, gL


def device_charge(card, p, W, L, V):
    """Single device: returns (Q[4], C[4,4] = dQ/dV)."""
    lib = _load()
    card = _c(card, np.float64)
    V = _c(V, np.float64)
    Q = np.zeros(4)
    C = np.zeros(16)
    rc = lib.ora_device_charge(_p(card), int(p), float(W), float(L), _p(V), _p(Q), _p(C))
    if rc != 0:
        raise ValueError("bad device arguments")
    return Q, C.reshape(4, 4)


def device_eval(card, p, W, L, V):
    """Single device: returns (I[4], G[4,4], Q[4])."""
    lib = _load()
    card = _c(card, np.float64)
    V = _c(V, np.float64)
    I = np.zeros(4)
    G = np.zeros(16)
    Q = np.zeros(4)
    rc = lib.ora_device_eval(_p(card), int(p), float(W), float(L), _p(V), _p(I), _p(G), _p(Q))
    if rc != 0:
        raise ValueError("bad device arguments")
    return I, G.reshape(4, 4), Q


OP_CLASSES = ("add", "mul", "div", "exp", "expm1", "log1p", "sqrt")


def count_ops(card, p, W, L, V, free_mask=0b1111):
    """Floating-point operations of one device evaluation (currents and charges, values only)
    that depend on the free terminals (bit t of free_mask: terminal d, g, s, b on a free node),
    by class (see OP_CLASSES)."""
    lib = _load()
    out = np.zeros(len(OP_CLASSES), np.int64)
    rc = lib.ora_count_ops(_p(_c(card, np.float64)), int(p), float(W), float(L),
                           _p(_c(V, np.float64)), int(free_mask), _p(out))
    if rc != 0:
        raise ValueError("bad device arguments")
    return dict(zip(OP_CLASSES, (int(v) for v in out)))
