"""Python binding of the GB300 MOSFET evaluate-and-stamp library (``include/eec.h``).

The module-level ``eec_*`` functions carry the C names and only marshal arguments: numpy arrays
for host inputs, torch CUDA tensors for device buffers (float64, contiguous), the current torch
stream unless one is given. Every step of the path runs in the CUDA library ``_libeec.so``; there
is no Python or CPU fallback, and importing this package raises ``ImportError`` when the library
has not been built (``python -m paper_2604_03079_gb300.build``).

``Circuit`` bundles one context with its netlist and owns the output tensors; ``EvalStamp`` is the
``torch.autograd.Function`` whose backward is the library's gather-based adjoint kernel.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_libeec.so")

EEC_OK, EEC_EINVAL, EEC_ESTATE, EEC_ECUDA, EEC_ETIMEOUT, EEC_ENUMERIC, EEC_ENOMEM = 0, -1, -2, -3, -4, -5, -7
EEC_ENOCONV = -6
EEC_VARIANT_AUTO = -1
EEC_VARIANT_COLOR_FUSED = 0
EEC_VARIANT_PERSISTENT = 1
EEC_VARIANT_ATOMIC = 2
EEC_VARIANT_SEGREDUCE = 3
EEC_VARIANT_COLOR_BUFFERED = 4
EEC_VARIANT_COLOR_PIPELINED = 5
EEC_N_VARIANTS = 6
VARIANT_NAMES = {0: "color_fused", 1: "persistent", 2: "atomic", 3: "segreduce", 4: "color_buffered",
                 5: "color_pipelined"}
EEC_CONFLICT_FREE_NODE, EEC_CONFLICT_ANY_NONGROUND, EEC_CONFLICT_WRITE_ROWS = 0, 1, 2
EEC_COLOR_GREEDY_SEQ, EEC_COLOR_JP_INDEX, EEC_COLOR_JP_RANDOM = 0, 1, 2
EEC_RAIL_ELIMINATE, EEC_RAIL_MNA_BRANCH = 0, 1
EEC_SOLVER_LU = 2
EEC_LU_ORDER_MMD = 0   # column orders of eec_lu_check_host_ex
EEC_LU_ORDER_BTF = 1
EEC_CARD_LEN = 21
EEC_GATHER_WINDOW = 1024   # the gather plan's window and heavy-entry bound (eec.h)
EEC_GATHER_HEAVY = 32



class eec_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("block", ctypes.c_int32),
                ("conflict_rule", ctypes.c_int32), ("debug_checks", ctypes.c_int32),
                ("color_stamp", ctypes.c_int32), ("host_chunks", ctypes.c_int32),
                ("rail_mode", ctypes.c_int32)]


class eec_netlist(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("node_fixed", ctypes.c_void_p),
                ("node_vfix", ctypes.c_void_p), ("n_dev", ctypes.c_int32),
                ("dev_nodes", ctypes.c_void_p), ("dev_type", ctypes.c_void_p),
                ("W", ctypes.c_void_p), ("L", ctypes.c_void_p), ("model_id", ctypes.c_void_p),
                ("n_res", ctypes.c_int32), ("res_nodes", ctypes.c_void_p),
                ("res_G", ctypes.c_void_p), ("n_isrc", ctypes.c_int32),
                ("isrc_nodes", ctypes.c_void_p), ("isrc_val", ctypes.c_void_p)]


_P, _I32, _I64, _F64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIG = {
    "eec_default_options": (eec_options, []),
    "eec_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(eec_options)]),
    "eec_destroy": (None, [_P]),
    "eec_last_error": (ctypes.c_char_p, [_P]),
    "eec_upload_netlist": (ctypes.c_int, [_P, _I32, _P, _P, _I32, _P, _P, _P, _P, _P, _I32, _P, _P,
                                          _I32, _P, _P, _F64]),
    "eec_set_model_cards": (ctypes.c_int, [_P, _I32, _P]),
    "eec_color": (ctypes.c_int, [_P, _P, _I32, _P, ctypes.POINTER(_I32)]),
    "eec_build_scatter": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "eec_get_pattern": (ctypes.c_int, [_P, _P, _P, _P]),
    "eec_get_color_offsets": (ctypes.c_int, [_P, _P]),
    "eec_verify_coloring": (ctypes.c_int, [_P, _I32]),
    "eec_update_params": (ctypes.c_int, [_P, _P, _P, _P]),
    "eec_set_variant": (ctypes.c_int, [_P, _I32]),
    "eec_get_variant": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "eec_set_eval_order": (ctypes.c_int, [_P, _I32]),
    "eec_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                      ctypes.POINTER(_I32)]),
    "eec_eval_stamp": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "eec_eval_stamp_bwd": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "eec_eval_stamp_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "eec_newton_dc": (ctypes.c_int, [_P, _P, _P, _P, _I32, _F64, _I32, _I32, _F64, _F64, _F64,
                                     ctypes.POINTER(_I32), _P]),
    "eec_eval_stamp_tran": (ctypes.c_int, [_P, _P, _P, _P, _F64, _F64, _P, _P, _P, _P, _P]),
    "eec_newton_tran": (ctypes.c_int, [_P, _P, _P, _P, _F64, _F64, _P, _P, _P, _P, _I32, _F64,
                                       _I32, _I32, _F64, _F64, _F64, ctypes.POINTER(_I32), _P]),
    "eec_transient": (ctypes.c_int, [_P, _P, _F64, _I32, _I32, _P, _I32, _F64, _I32, _I32, _F64,
                                     _F64, _F64, ctypes.POINTER(_I32), _P]),
    "eec_eval_stamp_bwd_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "eec_graph_capture": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "eec_graph_launch": (ctypes.c_int, [_P, _P]),
    "eec_autotune": (ctypes.c_int, [_P, _P, _P, _P, _P, _I32, _P, _P]),
    "eec_status": (ctypes.c_int, [_P, _P]),
    "eec_get_sizes": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                     ctypes.POINTER(_I64), ctypes.POINTER(_I32)]),
    "eec_upload_batch": (ctypes.c_int, [_P, _I32, ctypes.POINTER(eec_netlist), _F64]),
    "eec_get_batch_offsets": (ctypes.c_int, [_P, _P, _P, _P]),
    "eec_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), _I32,
                                        ctypes.POINTER(ctypes.POINTER(eec_netlist)), _F64,
                                        ctypes.POINTER(eec_options)]),
    "eec_batch_capture_graph": (ctypes.c_int, [_P, _P]),
    "eec_fp64_peak": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(_F64)]),
    "eec_lu_stats": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I32)]),
    "eec_newton_info": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "eec_lu_solve": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "eec_lu_check_host": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P, ctypes.POINTER(_I64),
                                         ctypes.POINTER(_I32)]),
    "eec_lu_check_host_ex": (ctypes.c_int, [_I32, _P, _P, _P, _P, _I32, _P, _P,
                                            ctypes.POINTER(_I64), ctypes.POINTER(_I32), _P]),
    "eec_math_check": (ctypes.c_int, [_I32, _I64, _P, _P, _P, _P]),
    "eec_gather_plan_host": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_I64)]),
    "eec_test_barrier_timeout": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "eec_profile_enable": (ctypes.c_int, [_P, _I32]),
    "eec_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(_F64), ctypes.POINTER(_F64),
                                        ctypes.POINTER(_F64), ctypes.POINTER(_I64),
                                        ctypes.POINTER(_I64)]),
}
EXPORTED = tuple(_SIG)
_lib = None


def _load():
    """Load ``_libeec.so`` once; a missing library is an error (there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2604_03079_gb300.build` (there is no CPU fallback)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            f = getattr(handle, name)
            f.restype = res
            f.argtypes = args
        _lib = handle
    return _lib


def __getattr__(name):
    if name == "lib":
        return _load()
    if name == "EvalStamp":   # the torch.autograd.Function (built on first use: imports torch)
        global _EvalStamp
        if _EvalStamp is None:
            _EvalStamp = _autograd()
        return _EvalStamp
    raise AttributeError(name)


class EECError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"eec error {code}: {msg}")
        self.code = code


def _check(ctx, rc: int):
    if rc != EEC_OK:
        msg = _load().eec_last_error(ctx).decode() if ctx else ""
        raise EECError(rc, msg)


def _h(a, dt):
    """Host array -> (contiguous numpy array, pointer); keeps the array alive via the caller."""
    a = np.ascontiguousarray(a, dtype=dt)
    return a, (a.ctypes.data_as(_P) if a.size else None)


def _d(t, n=None, name="tensor"):
    """Device buffer pointer of a float64 contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return _P(t.data_ptr())


def _numel(t):
    return int(t.numel()) if hasattr(t, "numel") else int(np.asarray(t).size)


def _need(t, k, name):
    """The library reads and writes every buffer by the context's sizes (the C ABI takes bare
    pointers): a buffer of another length (None passes) is refused here, before the call."""
    if t is not None and _numel(t) != k:
        raise ValueError(f"{name} has {_numel(t)} elements, the context needs {k}")


def _sizes(ctx):
    """(devices, unknowns, nonzeros) of a context with its scatter map built."""
    nd, n, nnz, _ = eec_get_sizes(ctx)
    return nd, n, nnz


def _need_step(ctx, x, A, b, q=None):
    nd, n, nnz = _sizes(ctx)
    _need(x, n, "x")
    _need(A, nnz, "A")
    _need(b, n, "b")
    _need(q, 4 * nd, "q")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _P(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---- the C entry points ---------------------------------------------------------------------
def eec_default_options() -> eec_options:
    return _load().eec_default_options()


def eec_create(opt: Optional[eec_options] = None, **kw):
    o = eec_default_options() if opt is None else opt
    for k, v in kw.items():
        setattr(o, k, int(v))
    h = _P()
    rc = _load().eec_create(ctypes.byref(h), ctypes.byref(o))
    if rc != EEC_OK:
        raise EECError(rc, "eec_create failed")
    return h


def eec_destroy(ctx):
    _load().eec_destroy(ctx)


def eec_last_error(ctx) -> str:
    return _load().eec_last_error(ctx).decode()


def eec_upload_netlist(ctx, node_fixed, node_vfix, dev_nodes, dev_type, W, L, model_id,
                       res_nodes=(), res_G=(), isrc_nodes=(), isrc_val=(), gshunt=1e-12):
    keep = [_h(node_fixed, np.uint8), _h(node_vfix, np.float64), _h(dev_nodes, np.int32),
            _h(dev_type, np.int8), _h(W, np.float64), _h(L, np.float64), _h(model_id, np.int32),
            _h(res_nodes, np.int32), _h(res_G, np.float64), _h(isrc_nodes, np.int32),
            _h(isrc_val, np.float64)]
    (nf, pf), (_, pv), (dn, pdn), (_, pt), (_, pW), (_, pL), (_, pm), (_, prn), (rg, prg), \
        (_, psn), (sv, psv) = keep
    _check(ctx, _load().eec_upload_netlist(ctx, nf.size, pf, pv, dn.size // 4, pdn, pt, pW, pL, pm,
                                       rg.size, prn, prg, sv.size, psn, psv, float(gshunt)))


def _netlist_array(nets: Sequence):
    """ctypes array of eec_netlist over the circuits' arrays (returned with the arrays it
    points into, which must stay alive for the call)."""
    keep, arr = [], (eec_netlist * len(nets))()
    for i, net in enumerate(nets):
        parts = [_h(net.node_fixed, np.uint8), _h(net.node_vfix, np.float64),
                 _h(net.dev_nodes, np.int32), _h(net.dev_type, np.int8), _h(net.W, np.float64),
                 _h(net.L, np.float64), _h(net.model_id, np.int32), _h(net.res_nodes, np.int32),
                 _h(net.res_G, np.float64), _h(net.isrc_nodes, np.int32),
                 _h(net.isrc_val, np.float64)]
        keep.append(parts)
        m = arr[i]
        m.n_nodes = parts[0][0].size
        m.node_fixed, m.node_vfix = parts[0][1], parts[1][1]
        m.n_dev = parts[2][0].size // 4
        m.dev_nodes, m.dev_type, m.W, m.L, m.model_id = (p[1] for p in parts[2:7])
        m.n_res = parts[8][0].size
        m.res_nodes, m.res_G = parts[7][1], parts[8][1]
        m.n_isrc = parts[10][0].size
        m.isrc_nodes, m.isrc_val = parts[9][1], parts[10][1]
    return arr, keep


def eec_upload_batch(ctx, nets: Sequence, gshunt=1e-12):
    arr, keep = _netlist_array(nets)
    _check(ctx, _load().eec_upload_batch(ctx, len(nets), arr, float(gshunt)))


def eec_batch_create(nets: Sequence, gshunt=1e-12, opt: Optional[eec_options] = None, **kw):
    """Batched context in one call (eec_create + eec_upload_batch); options as eec_create."""
    o = eec_default_options() if opt is None else opt
    for k, v in kw.items():
        setattr(o, k, int(v))
    arr, keep = _netlist_array(nets)
    ptrs = (ctypes.POINTER(eec_netlist) * len(nets))(*[ctypes.pointer(arr[i])
                                                        for i in range(len(nets))])
    h = _P()
    rc = _load().eec_batch_create(ctypes.byref(h), len(nets), ptrs, float(gshunt),
                                  ctypes.byref(o))
    if rc != EEC_OK:
        raise EECError(rc, "eec_batch_create failed")
    return h


def eec_batch_capture_graph(ctx, stream=None):
    _check(ctx, _load().eec_batch_capture_graph(ctx, _stream(stream)))


def eec_set_model_cards(ctx, cards):
    c, pc = _h(cards, np.float64)
    if c.size % EEC_CARD_LEN:
        raise ValueError("card table size must be a multiple of EEC_CARD_LEN")
    _check(ctx, _load().eec_set_model_cards(ctx, c.size // EEC_CARD_LEN, pc))


def eec_color(ctx, order=None, algo=EEC_COLOR_GREEDY_SEQ, n_dev=None):
    C = _I32(0)
    po, o = None, None
    if order is not None:
        o, po = _h(order, np.int32)
        n_dev = o.size
    if n_dev is None:
        raise ValueError("eec_color needs n_dev (or an order) to size the colour array")
    col = np.zeros(n_dev, np.int32)
    _check(ctx, _load().eec_color(ctx, po, int(algo), col.ctypes.data_as(_P), ctypes.byref(C)))
    return col, int(C.value)


def eec_build_scatter(ctx):
    n, nnz = _I32(0), _I64(0)
    _check(ctx, _load().eec_build_scatter(ctx, ctypes.byref(n), ctypes.byref(nnz)))
    return int(n.value), int(nnz.value)


def eec_get_sizes(ctx):
    nd, n, nnz, C = _I32(0), _I32(0), _I64(0), _I32(0)
    _check(ctx, _load().eec_get_sizes(ctx, ctypes.byref(nd), ctypes.byref(n), ctypes.byref(nnz),
                                  ctypes.byref(C)))
    return int(nd.value), int(n.value), int(nnz.value), int(C.value)


def eec_get_pattern(ctx, n_nodes):
    _, n, nnz, _ = eec_get_sizes(ctx)
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    unk = np.zeros(n_nodes, np.int32)
    _check(ctx, _load().eec_get_pattern(ctx, rp.ctypes.data_as(_P), col.ctypes.data_as(_P),
                                    unk.ctypes.data_as(_P)))
    return rp, col, unk


def eec_verify_coloring(ctx, with_gate_rows=False):
    _check(ctx, _load().eec_verify_coloring(ctx, int(bool(with_gate_rows))))


def eec_get_color_offsets(ctx):
    C = eec_get_sizes(ctx)[3]
    off = np.zeros(C + 1, np.int32)
    _check(ctx, _load().eec_get_color_offsets(ctx, off.ctypes.data_as(_P)))
    return off


def eec_get_batch_offsets(ctx, n_circ):
    ro = np.zeros(n_circ + 1, np.int32)
    no = np.zeros(n_circ + 1, np.int64)
    do = np.zeros(n_circ + 1, np.int32)
    _check(ctx, _load().eec_get_batch_offsets(ctx, ro.ctypes.data_as(_P), no.ctypes.data_as(_P),
                                          do.ctypes.data_as(_P)))
    return ro, no, do


def eec_update_params(ctx, W, L, stream=None):
    nd = _sizes(ctx)[0]
    _need(W, nd, "W")
    _need(L, nd, "L")
    _check(ctx, _load().eec_update_params(ctx, _d(W, name="W"), _d(L, name="L"), _stream(stream)))


def eec_set_variant(ctx, variant: int):
    _check(ctx, _load().eec_set_variant(ctx, int(variant)))


def eec_set_eval_order(ctx, cost_order: int):
    _check(ctx, _load().eec_set_eval_order(ctx, int(cost_order)))


def eec_get_variant(ctx) -> int:
    v = _I32(0)
    _check(ctx, _load().eec_get_variant(ctx, ctypes.byref(v)))
    return int(v.value)


def eec_get_tuning(ctx):
    """-> (variant, block, eval_order) that eec_eval_stamp uses."""
    v, blk, od = _I32(0), _I32(0), _I32(0)
    _check(ctx, _load().eec_get_tuning(ctx, ctypes.byref(v), ctypes.byref(blk), ctypes.byref(od)))
    return int(v.value), int(blk.value), int(od.value)


def _eval_stamp(ctx, x, A, b, q, stream):
    _check(ctx, _load().eec_eval_stamp(ctx, _d(x, name="x"), _d(A, name="A"), _d(b, name="b"),
                                   _d(q, name="q"), _stream(stream)))


def eec_eval_stamp(ctx, x, A, b, q=None, stream=None):
    _need_step(ctx, x, A, b, q)
    _eval_stamp(ctx, x, A, b, q, stream)


def eec_lu_solve(ctx, A, b, x, stream=None):
    """x = A^-1 b (device tensors) with the library's sparse LU on the context's pattern."""
    _check(ctx, _load().eec_lu_solve(ctx, _d(A, name="A"), _d(b, name="b"), _d(x, name="x"),
                                     _stream(stream)))


def eec_lu_stats(ctx):
    """-> (entries of L and U of the current sparse-LU plan, host analyses so far)."""
    nnz = _I64(0)
    an = _I32(0)
    _check(ctx, _load().eec_lu_stats(ctx, ctypes.byref(nnz), ctypes.byref(an)))
    return int(nnz.value), int(an.value)


NEWTON_PATHS = ("plain Newton", "gshunt stepping", "relaxation start then Newton",
                "relaxation start then gshunt stepping")


def eec_newton_info(ctx):
    """The last eec_newton_dc call: -> dict(solves, stages (gshunt stepping), sweeps
    (relaxation), path (index into NEWTON_PATHS))."""
    info = (_I32 * 4)()
    _check(ctx, _load().eec_newton_info(ctx, info))
    return {"solves": int(info[0]), "stages": int(info[1]), "sweeps": int(info[2]),
            "path": int(info[3])}


def eec_gather_plan_host(cnt):
    """Host check of the segmented reduction's gather plan (no GPU) for entries with cnt[e]
    contributions: -> dict of item_of, step_of, woff [n_win, 33], loc [n_win, 1024], heavy
    [n_heavy, 3] (entry, first item, items) and n_items."""
    import numpy as np
    c = np.ascontiguousarray(cnt, np.int32)
    E = c.size
    n_win = -(-E // EEC_GATHER_WINDOW)
    n_heavy = int(np.count_nonzero(c >= EEC_GATHER_HEAVY))
    item_of = np.zeros(E, np.int64)
    step_of = np.zeros(E, np.int32)
    woff = np.zeros((n_win, 33), np.int32)
    loc = np.zeros((n_win, EEC_GATHER_WINDOW), np.uint16)
    heavy = np.zeros((n_heavy, 3), np.int32)
    n_items = _I64(0)
    rc = _load().eec_gather_plan_host(E, c.ctypes.data, item_of.ctypes.data, step_of.ctypes.data,
                                      woff.ctypes.data, loc.ctypes.data, heavy.ctypes.data,
                                      ctypes.byref(n_items))
    if rc != EEC_OK:
        raise EECError(rc, "eec_gather_plan_host failed")
    return {"item_of": item_of, "step_of": step_of, "woff": woff, "loc": loc, "heavy": heavy,
            "n_items": n_items.value}


def eec_lu_check_host(row_ptr, col, a, b):
    """Host check of the sparse LU (no GPU): -> (x solving A x = b, entries of L and U, first
    column whose refactorised pivot degraded or -1)."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, np.int32)
    cl = np.ascontiguousarray(col, np.int32)
    av = np.ascontiguousarray(a, np.float64)
    bv = np.ascontiguousarray(b, np.float64)
    n = rp.size - 1
    if cl.size != rp[-1] or av.size != rp[-1] or bv.size != n:
        raise ValueError("eec_lu_check_host: inconsistent sizes")
    x = np.zeros(n)
    nnz = _I64(0)
    bad = _I32(0)
    rc = _load().eec_lu_check_host(n, rp.ctypes.data, cl.ctypes.data, av.ctypes.data,
                                   bv.ctypes.data, x.ctypes.data, ctypes.byref(nnz),
                                   ctypes.byref(bad))
    if rc != EEC_OK:
        raise EECError(rc, "eec_lu_check_host failed")
    return x, int(nnz.value), int(bad.value)


def eec_lu_check_host_ex(row_ptr, col, a, b, order=EEC_LU_ORDER_MMD):
    """Host check of the sparse LU with a choice of column order (no GPU): -> (x solving A x = b,
    the column order q, entries of L and U, first column whose refactorised pivot degraded or
    -1, the longest chains of dependent steps of the plan: (refactorisation, forward
    substitution, backward substitution))."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, np.int32)
    cl = np.ascontiguousarray(col, np.int32)
    av = np.ascontiguousarray(a, np.float64)
    bv = np.ascontiguousarray(b, np.float64)
    n = rp.size - 1
    if cl.size != rp[-1] or av.size != rp[-1] or bv.size != n:
        raise ValueError("eec_lu_check_host_ex: inconsistent sizes")
    x = np.zeros(n)
    q = np.zeros(n, np.int32)
    nnz = _I64(0)
    bad = _I32(0)
    depth = np.zeros(3, np.int32)
    rc = _load().eec_lu_check_host_ex(n, rp.ctypes.data, cl.ctypes.data, av.ctypes.data,
                                      bv.ctypes.data, int(order), x.ctypes.data, q.ctypes.data,
                                      ctypes.byref(nnz), ctypes.byref(bad), depth.ctypes.data)
    if rc != EEC_OK:
        raise EECError(rc, "eec_lu_check_host_ex failed")
    return x, q, int(nnz.value), int(bad.value), tuple(int(v) for v in depth)


def eec_newton_dc(ctx, x, A, b, max_iter=200, vstep=0.2, step_rule=0, solver=0, tol_abs=1e-12,
                  tol_rel=1e-9, tol_f=1e-12, stream=None) -> int:
    """DC Newton on the GPU from x (updated in place), with gshunt stepping when it does not
    converge and then a relaxation start (eec_newton_info tells which path converged); returns
    the number of solves.
    step_rule 0: the whole step scaled to vstep; 1: every node's move clipped to vstep.
    solver 0: batched sparse QR, analysis reused; 1: sparse QR after an AMD ordering;
    2 (EEC_SOLVER_LU): the library's sparse LU, host analysis once, GPU refactorisation."""
    _need_step(ctx, x, A, b)
    it = _I32(0)
    _check(ctx, _load().eec_newton_dc(ctx, _d(x, name="x"), _d(A, name="A"), _d(b, name="b"),
                                      int(max_iter), float(vstep), int(step_rule), int(solver),
                                      float(tol_abs), float(tol_rel), float(tol_f),
                                      ctypes.byref(it), _stream(stream)))
    return int(it.value)


def eec_newton_tran(ctx, x, q_prev, i_prev, alpha, beta, A, b, q, icap=None, max_iter=200,
                    vstep=0.2, step_rule=1, solver=EEC_SOLVER_LU, tol_abs=1e-12, tol_rel=1e-9,
                    tol_f=1e-9, stream=None) -> int:
    """One implicit time step (Newton on the transient companion system) from x (updated in
    place); q and icap receive the charges and capacitive currents at the new point. Returns the
    Newton iterations."""
    _need_step(ctx, x, A, b, q)
    nd = _sizes(ctx)[0]
    _need(q_prev, 4 * nd, "q_prev")
    _need(i_prev, 4 * nd, "i_prev")
    _need(icap, 4 * nd, "icap")
    it = _I32(0)
    _check(ctx, _load().eec_newton_tran(
        ctx, _d(x, name="x"), _d(q_prev, name="q_prev"), _d(i_prev, name="i_prev"),
        float(alpha), float(beta), _d(A, name="A"), _d(b, name="b"), _d(q, name="q"),
        _d(icap, name="icap"), int(max_iter), float(vstep), int(step_rule), int(solver),
        float(tol_abs), float(tol_rel), float(tol_f), ctypes.byref(it), _stream(stream)))
    return int(it.value)


def eec_transient(ctx, x, h, n_steps, method=1, traj=None, max_iter=200, vstep=0.2, step_rule=1,
                  solver=EEC_SOLVER_LU, tol_abs=1e-12, tol_rel=1e-9, tol_f=1e-9,
                  stream=None) -> int:
    """n_steps fixed time steps of h seconds from x (updated in place; method 0 backward Euler,
    1 trapezoidal); traj (nullable, [(n_steps + 1) * n] device) receives every time point.
    Returns the Newton iterations over all steps."""
    n = _sizes(ctx)[1]
    _need(x, n, "x")
    _need(traj, (int(n_steps) + 1) * n, "traj")
    it = _I32(0)
    _check(ctx, _load().eec_transient(
        ctx, _d(x, name="x"), float(h), int(n_steps), int(method), _d(traj, name="traj"),
        int(max_iter), float(vstep), int(step_rule), int(solver), float(tol_abs), float(tol_rel),
        float(tol_f), ctypes.byref(it), _stream(stream)))
    return int(it.value)


def _hp(t, name):
    """Host buffer pointer of a contiguous float64 CPU tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float64":
            raise TypeError(f"{name} must be a contiguous float64 host tensor")
        return _P(t.data_ptr())
    if t.dtype != np.float64 or not t.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{name} must be a contiguous float64 array")
    return t.ctypes.data_as(_P)


def eec_eval_stamp_host(ctx, x, A, b, q=None, stream=None):
    """eval_stamp with host buffers (torch CPU tensors, page-locked for async copies, or numpy)."""
    _need_step(ctx, x, A, b, q)
    _check(ctx, _load().eec_eval_stamp_host(ctx, _hp(x, "x"), _hp(A, "A"), _hp(b, "b"),
                                            _hp(q, "q"), _stream(stream)))


def eec_eval_stamp_tran(ctx, x, q_prev, i_prev, alpha, beta, A, b, q, i=None, stream=None):
    _need_step(ctx, x, A, b, q)
    nd = _sizes(ctx)[0]
    _need(q_prev, 4 * nd, "q_prev")
    _need(i_prev, 4 * nd, "i_prev")
    _need(i, 4 * nd, "i")
    _check(ctx, _load().eec_eval_stamp_tran(
        ctx, _d(x, name="x"), _d(q_prev, name="q_prev"), _d(i_prev, name="i_prev"),
        float(alpha), float(beta), _d(A, name="A"), _d(b, name="b"), _d(q, name="q"),
        _d(i, name="i"), _stream(stream)))


def _need_bwd(ctx, x, gA, gb, gx, gW, gL):
    nd, n, nnz = _sizes(ctx)
    for t, k, name in ((x, n, "x"), (gA, nnz, "gA"), (gb, n, "gb"), (gx, n, "gx"),
                       (gW, nd, "gW"), (gL, nd, "gL")):
        _need(t, k, name)


def eec_eval_stamp_bwd(ctx, x, gA, gb, gx, gW, gL, stream=None):
    _need_bwd(ctx, x, gA, gb, gx, gW, gL)
    _check(ctx, _load().eec_eval_stamp_bwd(ctx, _d(x, name="x"), _d(gA, name="gA"), _d(gb, name="gb"),
                                       _d(gx, name="gx"), _d(gW, name="gW"), _d(gL, name="gL"),
                                       _stream(stream)))


def eec_eval_stamp_bwd_noalloc(ctx, x, gA, gb, gx, gW, gL, stream=None):
    """Backward with the library's fixed scratch array: allocates nothing (see include/eec.h)."""
    _need_bwd(ctx, x, gA, gb, gx, gW, gL)
    _check(ctx, _load().eec_eval_stamp_bwd_noalloc(
        ctx, _d(x, name="x"), _d(gA, name="gA"), _d(gb, name="gb"), _d(gx, name="gx"),
        _d(gW, name="gW"), _d(gL, name="gL"), _stream(stream)))


EEC_NOALLOC_MAX_DEV = 524288


def eec_graph_capture(ctx, x, A, b, q=None, stream=None):
    _need_step(ctx, x, A, b, q)
    _check(ctx, _load().eec_graph_capture(ctx, _d(x), _d(A), _d(b), _d(q), _stream(stream)))


def eec_graph_launch(ctx, stream=None):
    _check(ctx, _load().eec_graph_launch(ctx, _stream(stream)))


def eec_autotune(ctx, x, A, b, q=None, reps=10, stream=None):
    _need_step(ctx, x, A, b, q)
    ms = (ctypes.c_float * EEC_N_VARIANTS)()
    _check(ctx, _load().eec_autotune(ctx, _d(x), _d(A), _d(b), _d(q), int(reps), _stream(stream), ms))
    return [float(v) for v in ms]


def eec_status(ctx, stream=None) -> int:
    """Synchronise and return the device status code (0, EEC_ETIMEOUT or EEC_ENUMERIC)."""
    return int(_load().eec_status(ctx, _stream(stream)))


def eec_profile_enable(ctx, enable=True):
    _check(ctx, _load().eec_profile_enable(ctx, int(bool(enable))))


def eec_profile_read(ctx):
    """-> dict(ms_init, ms_eval, ms_stamp, calls, kernels) since the last read (synchronises)."""
    a, b, c = _F64(0), _F64(0), _F64(0)
    n, k = _I64(0), _I64(0)
    _check(ctx, _load().eec_profile_read(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                     ctypes.byref(n), ctypes.byref(k)))
    return dict(ms_init=a.value, ms_eval=b.value, ms_stamp=c.value, calls=int(n.value),
                kernels=int(k.value))


def eec_test_barrier_timeout(ctx, x, A, b, stream=None):
    _need_step(ctx, x, A, b)
    _check(ctx, _load().eec_test_barrier_timeout(ctx, _d(x, name="x"), _d(A, name="A"),
                                                 _d(b, name="b"), _stream(stream)))


def eec_math_check(fn, x, stream=None):
    """-> (library result, CUDA result) of exp (0), expm1 (1), log1p on [0, 1] (2), the
    reciprocal (3) or the reciprocal square root (4) at x."""
    import torch
    ours = torch.empty_like(x)
    ref = torch.empty_like(x)
    rc = _load().eec_math_check(int(fn), x.numel(), _d(x, name="x"), _d(ours), _d(ref),
                                _stream(stream))
    if rc != EEC_OK:
        raise EECError(rc, "eec_math_check failed")
    return ours, ref


def eec_fp64_peak(iters=4096, blocks_per_sm=8) -> float:
    f = _F64(0.0)
    rc = _load().eec_fp64_peak(int(iters), int(blocks_per_sm), ctypes.byref(f))
    if rc != EEC_OK:
        raise EECError(rc, "eec_fp64_peak failed")
    return float(f.value)


# ---- convenience layer ----------------------------------------------------------------------
class Circuit:
    """One context: netlist upload, optional colouring, scatter map, device outputs.

    ``net`` is any object with the netlist arrays (node_fixed, node_vfix, dev_nodes, dev_type,
    W, L, model_id, res_nodes, res_G, isrc_nodes, isrc_val, gshunt)."""

    def __init__(self, net, cards, color: bool = True, variant: int = EEC_VARIANT_AUTO,
                 conflict_rule: int = EEC_CONFLICT_FREE_NODE, algo: int = EEC_COLOR_GREEDY_SEQ,
                 order=None, debug_checks: bool = False, batch: Optional[Sequence] = None,
                 host_chunks: int = 0, color_stamp: int = 0,
                 rail_mode: int = EEC_RAIL_ELIMINATE):
        import torch
        self.ctx = eec_create(variant=variant, conflict_rule=conflict_rule,
                              debug_checks=int(debug_checks), host_chunks=host_chunks,
                              color_stamp=color_stamp, rail_mode=rail_mode)
        self.batch = batch
        if batch is not None:
            eec_upload_batch(self.ctx, batch, gshunt=batch[0].gshunt if batch else 1e-12)
            n_dev = sum(int(m.dev_nodes.shape[0]) for m in batch)
            n_nodes = 1 + sum(int(m.node_fixed.shape[0]) - 1 for m in batch)
        else:
            eec_upload_netlist(self.ctx, net.node_fixed, net.node_vfix, net.dev_nodes,
                               net.dev_type, net.W, net.L, net.model_id, net.res_nodes,
                               net.res_G, net.isrc_nodes, net.isrc_val, net.gshunt)
            n_dev = int(net.dev_nodes.shape[0])
            n_nodes = int(net.node_fixed.shape[0])
        eec_set_model_cards(self.ctx, cards)
        self.colors, self.n_colors = (None, 0)
        if color:
            self.colors, self.n_colors = eec_color(self.ctx, order=order, algo=algo, n_dev=n_dev)
        self.n, self.nnz = eec_build_scatter(self.ctx)
        self.n_dev, self.n_nodes = n_dev, n_nodes
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def __del__(self):
        if getattr(self, "ctx", None):
            eec_destroy(self.ctx)
            self.ctx = None

    def pattern(self):
        return eec_get_pattern(self.ctx, self.n_nodes)

    def new_outputs(self, want_q=True):
        import torch
        A = torch.empty(self.nnz, dtype=torch.float64, device=self.dev)
        b = torch.empty(self.n, dtype=torch.float64, device=self.dev)
        q = torch.empty(4 * self.n_dev, dtype=torch.float64, device=self.dev) if want_q else None
        return A, b, q

    def eval_stamp(self, x, A=None, b=None, q=None, want_q=True, stream=None):
        if A is None:
            A, b, q = self.new_outputs(want_q)
        # lengths against the sizes this object holds (no query of the context per call)
        for t, k, name in ((x, self.n, "x"), (A, self.nnz, "A"), (b, self.n, "b"),
                           (q, 4 * self.n_dev, "q")):
            _need(t, k, name)
        _eval_stamp(self.ctx, x, A, b, q, stream)
        return A, b, q

    def bwd(self, x, gA, gb, stream=None):
        import torch
        gx = torch.empty(self.n, dtype=torch.float64, device=self.dev)
        gW = torch.empty(self.n_dev, dtype=torch.float64, device=self.dev)
        gL = torch.empty(self.n_dev, dtype=torch.float64, device=self.dev)
        eec_eval_stamp_bwd(self.ctx, x, gA, gb, gx, gW, gL, stream)
        return gx, gW, gL

    def status(self) -> int:
        return eec_status(self.ctx)


def _autograd():
    import torch

    class EvalStamp(torch.autograd.Function):
        """(x, W, L) -> (A.values, b) of one Newton iteration; backward -> (gx, gW, gL)."""

        @staticmethod
        def forward(fctx, circuit: Circuit, x, W, L):
            eec_update_params(circuit.ctx, W.detach().contiguous(), L.detach().contiguous())
            A, b, _ = circuit.eval_stamp(x.detach().contiguous(), want_q=False)
            fctx.circuit = circuit
            fctx.save_for_backward(x, W, L)
            return A, b

        @staticmethod
        def backward(fctx, gA, gb):
            x, W, L = fctx.saved_tensors
            c = fctx.circuit
            eec_update_params(c.ctx, W.detach().contiguous(), L.detach().contiguous())
            import torch
            gA = torch.zeros(c.nnz, dtype=torch.float64, device=x.device) if gA is None else gA.contiguous()
            gb = torch.zeros(c.n, dtype=torch.float64, device=x.device) if gb is None else gb.contiguous()
            gx, gW, gL = c.bwd(x.detach().contiguous(), gA, gb)
            return None, gx, gW, gL

    return EvalStamp


_EvalStamp = None


def eval_stamp_autograd(circuit: Circuit, x, W, L):
    """Differentiable eval_stamp: returns (A.values, b) with gradients to x, W and L."""
    global _EvalStamp
    if _EvalStamp is None:
        _EvalStamp = _autograd()
    return _EvalStamp.apply(circuit, x, W, L)
