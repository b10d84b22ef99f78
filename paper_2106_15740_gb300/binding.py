"""ctypes binding of the C ABI in include/qtensor.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of the method: graphs, angles and buffers are converted to plain
pointers and sizes, the C call runs, and a non-QT_OK status raises
``QTError`` with the library's message.  The shared library is built
in-tree; if it is missing the import fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "libqtensor_gb300.so"

QT_OK, QT_EINVAL, QT_ENOMEM, QT_EWIDTH, QT_ECUDA, QT_ETIMEOUT, QT_ESTATE = range(7)
QT_C128, QT_C64, QT_C64X2 = 0, 1, 2
QT_MODE_PER_BUCKET, QT_MODE_PERSISTENT = 0, 1
QT_REP_DEFAULT, QT_REP_DIAGONAL, QT_REP_ZZ, QT_REP_ZZ_DIAGONAL = range(4)
STATUS_NAMES = {0: "QT_OK", 1: "QT_EINVAL", 2: "QT_ENOMEM", 3: "QT_EWIDTH", 4: "QT_ECUDA",
                5: "QT_ETIMEOUT", 6: "QT_ESTATE"}

# Exported symbols (must match include/qtensor.h).
EXPORTS = [
    "qt_build_lightcone", "qt_network_info", "qt_network_tensor", "qt_order",
    "qt_contract_workspace_size", "qt_contract", "qt_network_free",
    "qt_plan_options_default", "qt_plan_create", "qt_plan_workspace_size", "qt_plan_stats",
    "qt_plan_edge_widths", "qt_plan_energy", "qt_plan_check", "qt_plan_energy_host",
    "qt_plan_free", "qt_energy_workspace_size", "qt_energy", "qt_last_error",
    "qt_plan_set_profiling", "qt_plan_kernel_times", "qt_plan_energy_static",
    "qt_static_scratch_bytes", "qt_plan_set_wait_limit", "qt_plan_inject_stall", "qt_plan_edge_slices",
    "qt_plan_edge_bytes", "qt_plan_trace_size", "qt_plan_set_trace", "qt_plan_tasks", "qt_plan_schedule",
    "qt_amplitude_plan_create", "qt_plan_amplitudes", "qt_representation_cost", "qt_plan_edge_order",
]


class QTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class qt_graph(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_edges", C.c_int32), ("edges", C.POINTER(C.c_int32))]


class qt_plan_options(C.Structure):
    _fields_ = [("batch", C.c_int32), ("dtype", C.c_int32), ("mode", C.c_int32),
                ("gradient", C.c_int32), ("max_width", C.c_int32), ("lane_items", C.c_int32),
                ("max_workspace", C.c_int64), ("group_rows", C.c_int32), ("edge_begin", C.c_int32),
                ("edge_end", C.c_int32), ("slice", C.c_int32),
                ("chunk_tiles", C.c_int32), ("order_trials", C.c_int32), ("order_seed", C.c_int32),
                ("order_tau", C.c_double), ("checkpoint_bytes", C.c_int64),
                ("chain_steps", C.c_int32), ("queue_order", C.c_int32),
                ("chunk_tiles_by_rank", C.c_int32 * 32), ("fuse_chains", C.c_int32)]


_lib = None


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise ImportError(f"{LIB_PATH.name} is not built; run __graft_entry__.build()")
        L = C.CDLL(str(LIB_PATH))
        vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        pi32, pd = C.POINTER(C.c_int32), C.POINTER(C.c_double)
        sig = {
            "qt_build_lightcone": [C.POINTER(qt_graph), i32, pd, pd, i32, C.POINTER(vp)],
            "qt_network_info": [vp, pi32, pi32],
            "qt_network_tensor": [vp, i32, pi32, pi32, pi32, pi32, pi32],
            "qt_order": [vp, pi32, pi32, pi32],
            "qt_contract_workspace_size": [vp, pi32, i32, C.POINTER(sz)],
            "qt_contract": [vp, pi32, i32, vp, vp, sz, pd],
            "qt_plan_create": [C.POINTER(qt_graph), i32, C.POINTER(qt_plan_options), C.POINTER(vp)],
            "qt_plan_workspace_size": [vp, C.POINTER(sz)],
            "qt_plan_stats": [vp, pi32, pi32, C.POINTER(i64), pd, pd],
            "qt_plan_edge_widths": [vp, pi32],
            "qt_plan_edge_slices": [vp, pi32],
            "qt_plan_edge_order": [vp, i32, pi32, pi32],
            "qt_plan_edge_bytes": [vp, C.POINTER(C.c_double)],
            "qt_plan_energy": [vp, vp, vp, vp, vp, vp, vp, sz, vp],
            "qt_plan_check": [vp, vp],
            "qt_plan_energy_host": [vp, pd, pd, pd, pd, pd, vp, sz, vp],
            "qt_energy_workspace_size": [C.POINTER(qt_graph), i32, i32, i32, i32, C.POINTER(sz)],
            "qt_energy": [C.POINTER(qt_graph), i32, pd, pd, i32, i32, vp, vp, sz, pd, pd],
            "qt_plan_set_profiling": [vp, i32],
            "qt_plan_kernel_times": [vp, C.POINTER(C.c_float), i32, pi32],
            "qt_plan_energy_static": [vp, vp, vp, vp, vp, vp],
            "qt_plan_set_wait_limit": [vp, i32],
            "qt_plan_inject_stall": [vp, i32],
            "qt_plan_trace_size": [vp, C.POINTER(sz)],
            "qt_amplitude_plan_create": [C.POINTER(qt_graph), i32, C.POINTER(C.c_uint8), i32,
                                         C.POINTER(qt_plan_options), C.POINTER(vp)],
            "qt_plan_amplitudes": [vp, vp, vp, vp, vp, sz, vp],
            "qt_representation_cost": [C.POINTER(qt_graph), i32, i32, i32, i32, pi32, pi32, pd],
            "qt_plan_set_trace": [vp, vp, sz],
            "qt_plan_tasks": [vp, pi32, pi32, pi32, pi32, pi32, pi32, pi32],
            "qt_plan_schedule": [vp, pi32, pi32, pi32, pi32, pi32, pi32, pi32,
                                 C.POINTER(C.c_int64), C.POINTER(C.c_int64), pi32, pi32],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.qt_last_error.restype = C.c_char_p
        L.qt_last_error.argtypes = []
        L.qt_network_free.argtypes = [vp]
        L.qt_network_free.restype = None
        L.qt_plan_free.argtypes = [vp]
        L.qt_plan_free.restype = None
        L.qt_plan_options_default.argtypes = [C.POINTER(qt_plan_options)]
        L.qt_plan_options_default.restype = None
        L.qt_static_scratch_bytes.argtypes = []
        L.qt_static_scratch_bytes.restype = C.c_size_t
        _lib = L
    return _lib


def _check(status):
    if status != QT_OK:
        raise QTError(status, lib().qt_last_error().decode())


def _graph(n_vertices, edges):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    g = qt_graph(int(n_vertices), int(e.shape[0]), e.ctypes.data_as(C.POINTER(C.c_int32)))
    return g, e  # keep the array alive with the struct


def _dptr(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _as_pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _as_pi32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


# ------------------------------------------------------------------ network

def qt_build_lightcone(n_vertices, edges, p, gamma, beta, edge):
    g, keep = _graph(n_vertices, edges)
    ga, be = _dptr(gamma), _dptr(beta)
    h = C.c_void_p()
    _check(lib().qt_build_lightcone(C.byref(g), int(p), _as_pd(ga), _as_pd(be), int(edge), C.byref(h)))
    return h


def qt_network_info(net):
    nv, nt = C.c_int32(), C.c_int32()
    _check(lib().qt_network_info(net, C.byref(nv), C.byref(nt)))
    return nv.value, nt.value


def qt_network_tensor(net, t):
    k, l, c, r = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    v = (C.c_int32 * 2)()
    _check(lib().qt_network_tensor(net, int(t), C.byref(k), C.byref(l), C.byref(c), C.byref(r), v))
    return k.value, l.value, c.value, r.value, (v[0], v[1])


def qt_order(net):
    nv, _ = qt_network_info(net)
    order = np.zeros(nv, dtype=np.int32)
    n, w = C.c_int32(), C.c_int32()
    _check(lib().qt_order(net, order.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n), C.byref(w)))
    return order, w.value


def qt_contract_workspace_size(net, order, dtype):
    o = np.ascontiguousarray(order, dtype=np.int32)
    b = C.c_size_t()
    _check(lib().qt_contract_workspace_size(net, o.ctypes.data_as(C.POINTER(C.c_int32)), int(dtype), C.byref(b)))
    return b.value


def qt_contract(net, order, dtype, stream, workspace_ptr, ws_bytes):
    o = np.ascontiguousarray(order, dtype=np.int32)
    out = (C.c_double * 2)()
    _check(lib().qt_contract(net, o.ctypes.data_as(C.POINTER(C.c_int32)), int(dtype), C.c_void_p(stream),
                             C.c_void_p(workspace_ptr), C.c_size_t(ws_bytes), out))
    return complex(out[0], out[1])


def qt_network_free(net):
    lib().qt_network_free(net)


# -------------------------------------------------------------------- plans

def qt_plan_options_default():
    o = qt_plan_options()
    lib().qt_plan_options_default(C.byref(o))
    return o


def qt_plan_create(n_vertices, edges, p, opt):
    g, keep = _graph(n_vertices, edges)
    h = C.c_void_p()
    _check(lib().qt_plan_create(C.byref(g), int(p), C.byref(opt), C.byref(h)))
    return h


def qt_amplitude_plan_create(n_vertices, edges, p, bits, opt):
    """bits: uint8 array [n_strings, n_vertices] of 0/1."""
    bits = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8).reshape(-1, int(n_vertices)))
    g, keep = _graph(n_vertices, edges)
    out = C.c_void_p()
    _check(lib().qt_amplitude_plan_create(C.byref(g), int(p), bits.ctypes.data_as(C.POINTER(C.c_uint8)),
                                          bits.shape[0], C.byref(opt), C.byref(out)))
    return out


def qt_plan_amplitudes(plan, gamma_ptr, beta_ptr, amp_ptr, ws_ptr, ws_bytes, stream):
    _check(lib().qt_plan_amplitudes(plan, gamma_ptr, beta_ptr, amp_ptr, ws_ptr, ws_bytes, stream))


def qt_representation_cost(n_vertices, edges, p, rep, order_trials=0, seed=0):
    """(n_vars, width, log2 cost) of the amplitude network in representation rep."""
    g, keep = _graph(n_vertices, edges)
    nv, w, c = C.c_int32(), C.c_int32(), C.c_double()
    _check(lib().qt_representation_cost(C.byref(g), int(p), int(rep), int(order_trials), int(seed), C.byref(nv),
                                        C.byref(w), C.byref(c)))
    return nv.value, w.value, c.value


def qt_plan_workspace_size(plan):
    b = C.c_size_t()
    _check(lib().qt_plan_workspace_size(plan, C.byref(b)))
    return b.value


def qt_plan_stats(plan):
    ne, mw, nb = C.c_int32(), C.c_int32(), C.c_int64()
    ab, fl = C.c_double(), C.c_double()
    _check(lib().qt_plan_stats(plan, C.byref(ne), C.byref(mw), C.byref(nb), C.byref(ab), C.byref(fl)))
    return dict(n_edges=ne.value, max_width=mw.value, n_buckets=nb.value, alg_bytes=ab.value, flops=fl.value)


def qt_plan_edge_widths(plan, n_edges):
    w = np.zeros(n_edges, dtype=np.int32)
    _check(lib().qt_plan_edge_widths(plan, w.ctypes.data_as(C.POINTER(C.c_int32))))
    return w


def qt_plan_edge_slices(plan, n_edges):
    sl = np.zeros(n_edges, dtype=np.int32)
    _check(lib().qt_plan_edge_slices(plan, sl.ctypes.data_as(C.POINTER(C.c_int32))))
    return sl


def qt_plan_edge_order(plan, unit):
    n = C.c_int32(0)
    _check(lib().qt_plan_edge_order(plan, int(unit), None, C.byref(n)))
    order = np.zeros(n.value, dtype=np.int32)
    _check(lib().qt_plan_edge_order(plan, int(unit), order.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)))
    return order


def qt_plan_edge_bytes(plan, n_edges):
    by = np.zeros(n_edges, dtype=np.float64)
    _check(lib().qt_plan_edge_bytes(plan, by.ctypes.data_as(C.POINTER(C.c_double))))
    return by


def qt_plan_energy(plan, gamma_ptr, beta_ptr, energy_ptr, edge_zz_ptr, grad_ptr, ws_ptr, ws_bytes, stream):
    """Device-pointer call (all pointers are integers; 0 means NULL)."""
    vp = C.c_void_p
    _check(lib().qt_plan_energy(plan, vp(gamma_ptr), vp(beta_ptr), vp(energy_ptr), vp(edge_zz_ptr or None),
                                vp(grad_ptr or None), vp(ws_ptr), C.c_size_t(ws_bytes), vp(stream)))


def qt_plan_check(plan, stream):
    _check(lib().qt_plan_check(plan, C.c_void_p(stream)))


def qt_plan_energy_host(plan, gamma, beta, energy, edge_zz, grad, ws_ptr, ws_bytes, stream):
    """Host-pointer call: numpy float64 arrays in and out (edge_zz/grad may be None)."""
    _check(lib().qt_plan_energy_host(plan, _as_pd(gamma), _as_pd(beta), _as_pd(energy), _as_pd(edge_zz),
                                     _as_pd(grad), C.c_void_p(ws_ptr), C.c_size_t(ws_bytes),
                                     C.c_void_p(stream)))


def qt_plan_set_profiling(plan, on):
    _check(lib().qt_plan_set_profiling(plan, int(bool(on))))


def qt_plan_kernel_times(plan, cap=4096):
    """Durations (ms) of the contraction launches recorded since the last read."""
    ms = (C.c_float * cap)()
    n = C.c_int32()
    _check(lib().qt_plan_kernel_times(plan, ms, int(cap), C.byref(n)))
    return [ms[i] for i in range(n.value)]


def qt_plan_energy_static(plan, gamma_ptr, beta_ptr, energy_ptr, edge_zz_ptr, stream):
    """Device-pointer call that uses the library's built-in scratch array
    instead of a caller workspace (allocates no device memory)."""
    vp = C.c_void_p
    _check(lib().qt_plan_energy_static(plan, vp(gamma_ptr), vp(beta_ptr), vp(energy_ptr),
                                       vp(edge_zz_ptr or None), vp(stream)))


def qt_static_scratch_bytes():
    return lib().qt_static_scratch_bytes()


def qt_plan_set_wait_limit(plan, polls):
    _check(lib().qt_plan_set_wait_limit(plan, int(polls)))


def qt_plan_inject_stall(plan, enable):
    _check(lib().qt_plan_inject_stall(plan, int(bool(enable))))


def qt_plan_trace_size(plan):
    n = C.c_size_t()
    _check(lib().qt_plan_trace_size(plan, C.byref(n)))
    return n.value


def qt_plan_set_trace(plan, trace_ptr, nbytes):
    _check(lib().qt_plan_set_trace(plan, trace_ptr or None, int(nbytes)))


def qt_plan_tasks(plan):
    """Queue tasks as a dict of int32 arrays: step, chunk, out_rank, edge, n_in, kind."""
    names = ("step", "chunk", "out_rank", "edge", "n_in", "kind")
    n = C.c_int32()
    _check(lib().qt_plan_tasks(plan, C.byref(n), None, None, None, None, None, None))
    cols = {k: np.empty(n.value, dtype=np.int32) for k in names}
    _check(lib().qt_plan_tasks(plan, C.byref(n), *(_as_pi32(cols[k]) for k in names)))
    return cols


def qt_plan_schedule(plan):
    """Schedule of a persistent plan as a dict of arrays (see the C header):
    dep_first, dep_count, deps, acc_first, acc_lo, acc_hi, acc_write, unit."""
    ns, nd, na = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().qt_plan_schedule(plan, C.byref(ns), C.byref(nd), C.byref(na), *([None] * 9)))
    n = ns.value
    out = {k: np.empty(n, dtype=np.int32) for k in ("dep_first", "dep_count", "unit")}
    out["deps"] = np.empty(max(nd.value, 1), dtype=np.int32)
    out["acc_first"] = np.empty(n + 1, dtype=np.int32)
    out["acc_lo"] = np.empty(max(na.value, 1), dtype=np.int64)
    out["acc_hi"] = np.empty(max(na.value, 1), dtype=np.int64)
    out["acc_write"] = np.empty(max(na.value, 1), dtype=np.int32)
    p64 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int64))
    _check(lib().qt_plan_schedule(plan, C.byref(ns), C.byref(nd), C.byref(na), _as_pi32(out["dep_first"]),
                                  _as_pi32(out["dep_count"]), _as_pi32(out["deps"]), _as_pi32(out["acc_first"]),
                                  p64(out["acc_lo"]), p64(out["acc_hi"]), _as_pi32(out["acc_write"]),
                                  _as_pi32(out["unit"])))
    for k, m in (("deps", nd.value), ("acc_lo", na.value), ("acc_hi", na.value), ("acc_write", na.value)):
        out[k] = out[k][:m]
    return out


def qt_plan_free(plan):
    lib().qt_plan_free(plan)


def qt_energy_workspace_size(n_vertices, edges, p, B, dtype, gradient):
    g, keep = _graph(n_vertices, edges)
    b = C.c_size_t()
    _check(lib().qt_energy_workspace_size(C.byref(g), int(p), int(B), int(dtype), int(gradient), C.byref(b)))
    return b.value


def qt_energy(n_vertices, edges, p, gamma, beta, B, dtype, stream, ws_ptr, ws_bytes, energy, grad=None):
    g, keep = _graph(n_vertices, edges)
    _check(lib().qt_energy(C.byref(g), int(p), _as_pd(gamma), _as_pd(beta), int(B), int(dtype),
                           C.c_void_p(stream), C.c_void_p(ws_ptr), C.c_size_t(ws_bytes), _as_pd(energy),
                           _as_pd(grad)))


def qt_last_error():
    return lib().qt_last_error().decode()
