"""CPU oracle for graphBpp / graphL (plain C in ``sb_oracle.c``, loaded with ctypes).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and this module imports nothing from the product
package.  The functions here only marshal numpy arrays; every step of the
method is computed in ``sb_oracle.c``, which cites the paper section it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsb_oracle.so")
_lib = None
_lock = threading.Lock()

LOAD_LCC = 1
LOAD_MERGE_DUP = 2

STATUS = {
    0: "ok", -1: "arg", -3: "oom", -4: "self_loop", -5: "bad_sign", -6: "inconsistent",
    -7: "duplicate", -8: "disconnected", -9: "range",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code} ({STATUS.get(code, '?')})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, so x86 and Arm agree)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, u64, i32, u32, f64, f32 = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32,
                                            ctypes.c_double, ctypes.c_float)
            sig = {
                "or_mix64": (u64, [u64]),
                "or_fmix32": (u32, [u32]),
                "or_tree_key": (u64, [u64, i64]),
                "or_tree_root": (i64, [u64, i64, i64]),
                "or_parent_key": (u64, [u64, i64, i64, i64]),
                "or_vertex_weight": (u64, [i64]),
                "or_clean_graph": (ctypes.c_int, [i64, i64, P, P, P, u32, P, P, P, P, P, P]),
                "or_build_csr": (ctypes.c_int, [i64, i64, P, P, P, P, P, P]),
                "or_tree": (i64, [i64, P, P, P, u64, i64, P, P, P]),
                "or_frustration": (i64, [i64, P, P, P, P]),
                "or_state_hash": (u64, [i64, P]),
                "or_sample": (ctypes.c_int, [i64, P, P, P, i64, P, P, P, u64, i64, i64, P, P, P, P]),
                "or_mst_weight": (u64, [u64, i64, i64, i64]),
                "or_mst_tree": (i64, [i64, i64, P, P, P, u64, i64, P, P]),
                "or_mst_sample": (ctypes.c_int, [i64, i64, P, P, P, u64, i64, i64, P, P, P, P]),
                "or_cloud": (i64, [i64, i64, i64, P, P, P, P, P, P]),
                "or_cloud_bounded": (i64, [i64, i64, i64, P, P, i64, P, P, P, P]),
                "or_graphl_loss_f64": (None, [i64, P, P, P, P, i64, P, P]),
                "or_graphl_grad_f64": (None, [i64, P, P, P, P, i64, P, P]),
                "or_graphl_grad_f32": (None, [i64, P, P, P, P, i64, P, P]),
                "or_graphl_descent_f64": (ctypes.c_int, [i64, P, P, P, i64, P, P, P, P, i64, f64, i64,
                                                         ctypes.c_int, P, P]),
                "or_graphl_descent_f32": (ctypes.c_int, [i64, P, P, P, P, i64, f32, i64, ctypes.c_int, P]),
                "or_graphl_round_f32": (None, [i64, P, P, P, P, i64, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Graph:
    """Cleaned graph held by the oracle: sorted edge list + CSR (numpy)."""

    def __init__(self, n, eu, ev, eneg, vmap=None):
        self.n = int(n)
        self.eu = _c(eu, np.int32)
        self.ev = _c(ev, np.int32)
        self.eneg = _c(eneg, np.int8)
        self.m = int(self.eu.shape[0])
        self.vmap = vmap
        self.rowptr = np.zeros(self.n + 1, np.int64)
        self.col = np.zeros(2 * self.m, np.int32)
        self.colneg = np.zeros(2 * self.m, np.int8)
        rc = lib().or_build_csr(self.n, self.m, _p(self.eu), _p(self.ev), _p(self.eneg), _p(self.rowptr),
                                _p(self.col), _p(self.colneg))
        if rc != 0:
            raise OracleError(rc)

    @property
    def csr(self):
        return self.rowptr, self.col, self.colneg


def clean_graph(n, src, dst, sign, flags=LOAD_LCC | LOAD_MERGE_DUP) -> Graph:
    src, dst, sign = _c(src, np.int32), _c(dst, np.int32), _c(sign, np.int8)
    m = src.shape[0]
    eu = np.zeros(max(m, 1), np.int32)
    ev = np.zeros(max(m, 1), np.int32)
    en = np.zeros(max(m, 1), np.int8)
    vmap = np.zeros(n, np.int32)
    n_out = ctypes.c_int64()
    m_out = ctypes.c_int64()
    rc = lib().or_clean_graph(n, m, _p(src), _p(dst), _p(sign), flags, ctypes.byref(n_out), ctypes.byref(m_out),
                              _p(eu), _p(ev), _p(en), _p(vmap))
    if rc != 0:
        raise OracleError(rc)
    mm = m_out.value
    return Graph(n_out.value, eu[:mm], ev[:mm], en[:mm], vmap)


def tree(g: Graph, seed: int, t: int):
    """(root, parent[n], canonical labels[n] uint8, level[n]) of tree t."""
    parent = np.zeros(g.n, np.int32)
    clab = np.zeros(g.n, np.uint8)
    level = np.zeros(g.n, np.int32)
    r = lib().or_tree(g.n, _p(g.rowptr), _p(g.col), _p(g.colneg), seed, t, _p(parent), _p(clab), _p(level))
    if r < 0:
        raise OracleError(int(r))
    return int(r), parent, clab, level


def sample(g: Graph, seed: int, t0: int, K: int, want_labels=True, want_parents=False):
    """Trees [t0, t0+K): dict with counts (int32[K]), hashes (uint64[K]),
    labels (uint8[K, n], canonical) and parents (int32[K, n]) when asked."""
    counts = np.zeros(K, np.int32)
    hashes = np.zeros(K, np.uint64)
    labels = np.zeros((K, g.n), np.uint8) if want_labels else None
    parents = np.zeros((K, g.n), np.int32) if want_parents else None
    rc = lib().or_sample(g.n, _p(g.rowptr), _p(g.col), _p(g.colneg), g.m, _p(g.eu), _p(g.ev), _p(g.eneg), seed,
                         t0, K, _p(labels), _p(parents), _p(counts), _p(hashes))
    if rc != 0:
        raise OracleError(rc)
    return {"counts": counts, "hashes": hashes, "labels": labels, "parents": parents}


def mst_tree(g: Graph, seed: int, t: int):
    """(tree edge count, in_tree[m] uint8, canonical labels[n] uint8) of
    randomized Kruskal tree t."""
    in_tree = np.zeros(max(g.m, 1), np.uint8)
    clab = np.zeros(g.n, np.uint8)
    r = lib().or_mst_tree(g.n, g.m, _p(g.eu), _p(g.ev), _p(g.eneg), seed, t, _p(in_tree), _p(clab))
    if r < 0:
        raise OracleError(int(r))
    return int(r), in_tree[: g.m], clab


def mst_sample(g: Graph, seed: int, t0: int, K: int, want_labels=True, want_in_tree=False):
    """Kruskal trees [t0, t0+K): dict with counts, hashes, labels (uint8[K, n])
    and in_tree (uint8[K, m]) when asked."""
    counts = np.zeros(K, np.int32)
    hashes = np.zeros(K, np.uint64)
    labels = np.zeros((K, g.n), np.uint8) if want_labels else None
    in_tree = np.zeros((K, g.m), np.uint8) if want_in_tree else None
    rc = lib().or_mst_sample(g.n, g.m, _p(g.eu), _p(g.ev), _p(g.eneg), seed, t0, K, _p(in_tree), _p(labels),
                             _p(counts), _p(hashes))
    if rc != 0:
        raise OracleError(rc)
    return {"counts": counts, "hashes": hashes, "labels": labels, "in_tree": in_tree}


def mst_weight(seed, t, u, v) -> int:
    return int(lib().or_mst_weight(seed, t, u, v))


def frustration(g: Graph, clab) -> int:
    clab = _c(clab, np.uint8)
    return int(lib().or_frustration(g.m, _p(g.eu), _p(g.ev), _p(g.eneg), _p(clab)))


def state_hash(clab) -> int:
    clab = _c(clab, np.uint8)
    return int(lib().or_state_hash(clab.shape[0], _p(clab)))


def cloud(labels, counts, t0=0):
    """Distinct states of a K x n canonical label matrix, first-seen order.
    Returns dict of arrays: first_tree, count, S, H."""
    labels = _c(labels, np.uint8)
    counts = _c(counts, np.int32)
    K, n = labels.shape
    first = np.zeros(max(K, 1), np.int64)
    cnt = np.zeros(max(K, 1), np.int32)
    S = np.zeros(max(K, 1), np.int32)
    H = np.zeros(max(K, 1), np.uint64)
    ns = lib().or_cloud(n, K, t0, _p(labels), _p(counts), _p(first), _p(cnt), _p(S), _p(H))
    if ns < 0:
        raise OracleError(int(ns))
    return {"first_tree": first[:ns], "count": cnt[:ns], "S": S[:ns], "H": H[:ns]}


def cloud_bounded(labels, counts, fmax, t0=0):
    """Cloud of the scalable variant (at most fmax states; see or_cloud_bounded)."""
    labels = _c(labels, np.uint8)
    counts = _c(counts, np.int32)
    K, n = labels.shape
    cap = max(1, min(int(fmax), K))
    first = np.zeros(cap, np.int64)
    cnt = np.zeros(cap, np.int32)
    S = np.zeros(cap, np.int32)
    H = np.zeros(cap, np.uint64)
    ns = lib().or_cloud_bounded(n, K, t0, _p(labels), _p(counts), int(fmax), _p(first), _p(cnt), _p(S), _p(H))
    if ns < 0:
        raise OracleError(int(ns))
    return {"first_tree": first[:ns], "count": cnt[:ns], "S": S[:ns], "H": H[:ns]}


def graphl_loss_f64(g: Graph, gamma):
    gamma = _c(gamma, np.float64)
    R = gamma.shape[1]
    loss = np.zeros(R, np.float64)
    F = np.zeros(R, np.int64)
    lib().or_graphl_loss_f64(g.m, _p(g.eu), _p(g.ev), _p(g.eneg), _p(gamma), R, _p(loss), _p(F))
    return loss, F


def graphl_grad_f64(g: Graph, gamma, gout=None):
    gamma = _c(gamma, np.float64)
    R = gamma.shape[1]
    gout = np.ones(R, np.float64) if gout is None else _c(gout, np.float64)
    out = np.zeros_like(gamma)
    lib().or_graphl_grad_f64(g.n, _p(g.rowptr), _p(g.col), _p(g.colneg), _p(gamma), R, _p(gout), _p(out))
    return out


def graphl_grad_f32(g: Graph, gamma, gout=None):
    gamma = _c(gamma, np.float32)
    R = gamma.shape[1]
    gout = np.ones(R, np.float32) if gout is None else _c(gout, np.float32)
    out = np.zeros_like(gamma)
    lib().or_graphl_grad_f32(g.n, _p(g.rowptr), _p(g.col), _p(g.colneg), _p(gamma), R, _p(gout), _p(out))
    return out


def graphl_descent_f64(g: Graph, gamma0, alpha, steps, renorm_log2=32, trace=False):
    gamma = np.array(gamma0, dtype=np.float64, order="C", copy=True)
    R = gamma.shape[1]
    exps = np.zeros(R, np.int32)
    F_trace = np.zeros((steps, R), np.int64) if trace else None
    rc = lib().or_graphl_descent_f64(g.n, _p(g.rowptr), _p(g.col), _p(g.colneg), g.m, _p(g.eu), _p(g.ev),
                                     _p(g.eneg), _p(gamma), R, float(alpha), steps, renorm_log2, _p(exps),
                                     _p(F_trace))
    if rc != 0:
        raise OracleError(rc)
    return gamma, exps, F_trace


def graphl_descent_f32(g: Graph, gamma0, alpha, steps, renorm_log2=32):
    gamma = np.array(gamma0, dtype=np.float32, order="C", copy=True)
    R = gamma.shape[1]
    exps = np.zeros(R, np.int32)
    rc = lib().or_graphl_descent_f32(g.n, _p(g.rowptr), _p(g.col), _p(g.colneg), _p(gamma), R,
                                     np.float32(alpha).item(), steps, renorm_log2, _p(exps))
    if rc != 0:
        raise OracleError(rc)
    return gamma, exps


def graphl_round_f32(g: Graph, gamma, want_flip=False):
    gamma = _c(gamma, np.float32)
    R = gamma.shape[1]
    F = np.zeros(R, np.int64)
    flip = np.zeros((R, g.m), np.uint8) if want_flip else None
    lib().or_graphl_round_f32(g.m, _p(g.eu), _p(g.ev), _p(g.eneg), _p(gamma), R, _p(F), _p(flip))
    return F, flip


def mix64(z: int) -> int:
    return int(lib().or_mix64(z & 0xFFFFFFFFFFFFFFFF))


def fmix32(h: int) -> int:
    return int(lib().or_fmix32(h & 0xFFFFFFFF))


def parent_key(seed, t, u, v) -> int:
    return int(lib().or_parent_key(seed, t, u, v))


def tree_root(seed, t, n) -> int:
    return int(lib().or_tree_root(seed, t, n))
