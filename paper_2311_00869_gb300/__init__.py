"""GB300-native graphBpp / graphL (arXiv 2311.00869) behind a C ABI.

The Python layer only marshals arguments: every step runs in the CUDA
kernels of libsignedbal.so (see include/signedbal.h).  PyTorch provides the
device memory (its caching allocator backs the library's own buffers) and the
stream.  There is no CPU fallback: without the built library or a CUDA device
the calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi

LOAD_LCC = 1
LOAD_MERGE_DUP = 2

STATUS_NAMES = {
    0: "SB_OK", -1: "SB_ERR_ARG", -2: "SB_ERR_CUDA", -3: "SB_ERR_OOM", -4: "SB_ERR_SELF_LOOP",
    -5: "SB_ERR_BAD_SIGN", -6: "SB_ERR_INCONSISTENT", -7: "SB_ERR_DUPLICATE", -8: "SB_ERR_DISCONNECTED",
    -9: "SB_ERR_RANGE", -10: "SB_ERR_STATE", -11: "SB_ERR_CLOUD_FULL", -12: "SB_ERR_TIMEOUT",
    -13: "SB_ERR_DEVICE_CHECK",
}


class SignedBalError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(type(t))


class SignedBal:
    """One library context (sb_ctx) on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, torch_allocator: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("signedbal needs a CUDA device (no CPU fallback)")
        self.lib = _abi.load()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = self.lib.sb_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise SignedBalError(rc, "sb_create failed")
        self.h = h
        self._keep = []
        if torch_allocator:
            dev = device

            def _alloc(size, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), dev, stream or 0)
                except Exception:
                    return None

            def _free(ptr, stream, user):
                try:
                    torch.cuda.caching_allocator_delete(ptr)
                except Exception:
                    pass

            fa, ff = _abi.ALLOC_FN(_alloc), _abi.FREE_FN(_free)
            self._keep += [fa, ff]
            self._check(self.lib.sb_set_allocator(self.h, fa, ff, None))
        self.n = self.m = 0

    def close(self):
        if getattr(self, "h", None) is not None:
            self.lib.sb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            msg = self.lib.sb_last_error(self.h).decode(errors="replace")
            raise SignedBalError(rc, msg)

    # ---------------------------------------------------------------- ingest
    def load_graph(self, n, src, dst, sign, flags=LOAD_LCC | LOAD_MERGE_DUP, want_vmap=False):
        """src/dst int32, sign int8 (+1/-1): numpy arrays, host tensors (pinned
        or not) or device tensors.  Returns (n, m, vmap or None)."""
        conv = []
        for a, dt in ((src, np.int32), (dst, np.int32), (sign, np.int8)):
            if isinstance(a, torch.Tensor):
                conv.append(a.contiguous())
            else:
                conv.append(np.ascontiguousarray(a, dtype=dt))
        m = int(conv[0].shape[0])
        n_out, m_out = ctypes.c_int64(), ctypes.c_int64()
        vmap = np.zeros(n, np.int32) if want_vmap else None
        self._check(self.lib.sb_load_graph(self.h, int(n), m, _ptr(conv[0]), _ptr(conv[1]), _ptr(conv[2]), flags,
                                           ctypes.byref(n_out), ctypes.byref(m_out), _ptr(vmap)))
        self.batch_G = 0
        self.n, self.m = n_out.value, m_out.value
        return self.n, self.m, vmap

    def load_batch(self, graphs, flags=LOAD_LCC | LOAD_MERGE_DUP):
        """graphs: list of (n, src, dst, sign) with local ids.  Returns the
        cleaned (n_g, m_g) arrays."""
        G = len(graphs)
        nv = np.array([g[0] for g in graphs], np.int64)
        eofs = np.zeros(G + 1, np.int64)
        eofs[1:] = np.cumsum([len(g[1]) for g in graphs])
        src = np.ascontiguousarray(np.concatenate([np.asarray(g[1], np.int32) for g in graphs]))
        dst = np.ascontiguousarray(np.concatenate([np.asarray(g[2], np.int32) for g in graphs]))
        sign = np.ascontiguousarray(np.concatenate([np.asarray(g[3], np.int8) for g in graphs]))
        nv_out = np.zeros(G, np.int64)
        m_out = np.zeros(G, np.int64)
        self._check(self.lib.sb_load_batch(self.h, G, _ptr(nv), _ptr(eofs), _ptr(src), _ptr(dst), _ptr(sign), flags,
                                           _ptr(nv_out), _ptr(m_out)))
        self.batch_G = G
        self.n, self.m = int(nv_out.sum()), int(m_out.sum())
        return nv_out, m_out

    def batch_frustration(self):
        """(G, K) counts and hashes of the last sample in a batch."""
        counts = torch.empty((self.batch_G, self.K), dtype=torch.int32, device=self.device)
        hashes = torch.empty((self.batch_G, self.K), dtype=torch.int64, device=self.device)
        self._check(self.lib.sb_frustration(self.h, _ptr(counts), _ptr(hashes)))
        return counts, hashes

    def batch_cloud(self, want_entries=True):
        G, K = self.batch_G, self.K
        ns = np.zeros(G, np.int32)
        fm = np.zeros(G, np.int32)
        ent = (_abi.CloudEntry * (G * K))() if want_entries else None
        self._check(self.lib.sb_batch_cloud(self.h, _ptr(ns), _ptr(fm),
                                            ctypes.cast(ent, ctypes.c_void_p) if want_entries else None))
        out = {"n_states": ns, "fr_min": fm}
        if want_entries:
            arr = np.ctypeslib.as_array(ent).reshape(G, K)
            out["entries"] = [{k: np.array(arr[g, : ns[g]][k]) for k in ("hash", "S", "count", "first_tree")}
                              for g in range(G)]
        return out

    def batch_steps(self, seed, tree_begin, K, steps, use_graph=True, fr_min=None, n_states=None):
        """`steps` graphBpp steps over the batch without host synchronisation
        (one step captured into a CUDA graph and replayed when use_graph);
        returns the device tensors (fr_min over all steps, n_states of the
        last step), G entries each, valid after sync()."""
        G = self.batch_G
        fr_min = torch.empty(G, dtype=torch.int32, device=self.device) if fr_min is None else fr_min
        n_states = torch.empty(G, dtype=torch.int32, device=self.device) if n_states is None else n_states
        self._check(self.lib.sb_batch_steps(self.h, seed, tree_begin, K, steps, 1 if use_graph else 0, _ptr(fr_min),
                                            _ptr(n_states)))
        self.K = K
        return fr_min, n_states

    def graph_edges(self):
        u = torch.empty(self.m, dtype=torch.int32, device=self.device)
        v = torch.empty_like(u)
        neg = torch.empty(self.m, dtype=torch.int8, device=self.device)
        self._check(self.lib.sb_graph_edges(self.h, _ptr(u), _ptr(v), _ptr(neg)))
        return u, v, neg

    def graph_csr(self):
        rp = torch.empty(self.n + 1, dtype=torch.int32, device=self.device)
        col = torch.empty(2 * self.m, dtype=torch.int32, device=self.device)
        neg = torch.empty(2 * self.m, dtype=torch.int8, device=self.device)
        self._check(self.lib.sb_graph_csr(self.h, _ptr(rp), _ptr(col), _ptr(neg)))
        return rp, col, neg

    # -------------------------------------------------------------- graphBpp
    def sample_trees(self, seed, tree_begin, K, want_parents=False):
        parents = torch.empty((K, self.n), dtype=torch.int32, device=self.device) if want_parents else None
        self.K = K
        self._check(self.lib.sb_sample_trees(self.h, seed, tree_begin, K, _ptr(parents)))
        return parents

    def sample_trees_kruskal(self, seed, tree_begin, K, want_in_tree=False):
        """Randomized Kruskal trees [tree_begin, tree_begin + K) in place of
        the BFS trees; with want_in_tree, a (K, m) uint8 membership matrix."""
        in_tree = torch.empty((K, self.m), dtype=torch.uint8, device=self.device) if want_in_tree else None
        self.K = K
        self._check(self.lib.sb_sample_trees_kruskal(self.h, seed, tree_begin, K, _ptr(in_tree)))
        return in_tree

    def label(self, out=None):
        """Canonical labels, (n, ceil(K/64)) int64 words (bit b of word w =
        tree 64w+b)."""
        W = (self.K + 63) // 64
        out = torch.empty((self.n, W), dtype=torch.int64, device=self.device) if out is None else out
        self._check(self.lib.sb_label(self.h, _ptr(out)))
        return out

    def frustration(self, counts=None, hashes=None):
        """Counts and hashes of the last sample: K each, or G x K in a batch."""
        shape = (self.batch_G, self.K) if getattr(self, "batch_G", 0) else (self.K,)
        need = int(np.prod(shape))
        counts = torch.empty(shape, dtype=torch.int32, device=self.device) if counts is None else counts
        hashes = torch.empty(shape, dtype=torch.int64, device=self.device) if hashes is None else hashes
        if counts.numel() < need or hashes.numel() < need:
            raise ValueError(f"counts / hashes need {need} entries")
        self._check(self.lib.sb_frustration(self.h, _ptr(counts), _ptr(hashes)))
        return counts, hashes

    def cloud_insert(self):
        """Inserts the last batch into the cloud (once); returns the number of states."""
        ns, fr = ctypes.c_int64(), ctypes.c_int32()
        self._check(self.lib.sb_cloud(self.h, None, 0, ctypes.byref(ns), None))
        return ns.value

    def cloud(self, cap=None):
        """Inserts the last batch (once) and returns (entries, fr_min): a dict of
        numpy arrays hash / S / count / first_tree in order of first appearance."""
        ns, fr = ctypes.c_int64(), ctypes.c_int32()
        if cap is None:
            cap = self.cloud_insert()
        buf = (_abi.CloudEntry * max(cap, 1))()
        self._check(self.lib.sb_cloud(self.h, ctypes.cast(buf, ctypes.c_void_p), cap, ctypes.byref(ns),
                                      ctypes.byref(fr)))
        arr = np.ctypeslib.as_array(buf)[: min(cap, ns.value)]
        out = {
            "hash": np.array(arr["hash"], dtype=np.uint64),
            "S": np.array(arr["S"], dtype=np.int32),
            "count": np.array(arr["count"], dtype=np.int32),
            "first_tree": np.array(arr["first_tree"], dtype=np.int64),
        }
        return out, fr.value

    def cloud_reset(self, max_states=0, hash_bits=0):
        self._check(self.lib.sb_cloud_reset(self.h, max_states, hash_bits))

    def cloud_reset_scalable(self, f_max):
        """Empties the cloud and keeps at most f_max states by the paper's
        scalable rule (see sb_cloud_reset_scalable)."""
        self._check(self.lib.sb_cloud_reset_scalable(self.h, int(f_max)))

    def cloud_switch(self, idx):
        """(bits, count): int64 words with bit e set for every edge (order of
        graph_edges) that cloud state `idx` switches, and their number (= S)."""
        out = torch.empty((self.m + 63) // 64, dtype=torch.int64, device=self.device)
        cnt = ctypes.c_int64()
        self._check(self.lib.sb_cloud_switch(self.h, idx, _ptr(out), ctypes.byref(cnt)))
        return out, cnt.value

    def cloud_state(self, idx):
        out = torch.empty((self.n + 63) // 64, dtype=torch.int64, device=self.device)
        self._check(self.lib.sb_cloud_state(self.h, idx, _ptr(out)))
        return out

    # ---------------------------------------------------------------- graphL
    def _per_graph(self):
        return getattr(self, "batch_G", 0) or 1

    def graphL_fwd(self, gamma):
        gamma = gamma.contiguous()
        R = gamma.shape[1]
        loss = torch.empty(self._per_graph() * R, dtype=torch.float32, device=self.device)
        F = torch.empty(self._per_graph() * R, dtype=torch.int32, device=self.device)
        self._check(self.lib.sb_graphL_fwd(self.h, _ptr(gamma), R, _ptr(loss), _ptr(F)))
        return loss, F

    def graphL_bwd(self, gamma, gout):
        gamma = gamma.contiguous()
        R = gamma.shape[1]
        grad = torch.empty_like(gamma)
        self._check(self.lib.sb_graphL_bwd(self.h, _ptr(gamma), R, _ptr(gout.contiguous()), _ptr(grad)))
        return grad

    def graphL_descent(self, gamma0, alpha, steps, renorm_log2=32, trace=False, out=None):
        gamma0 = gamma0.contiguous()
        R = gamma0.shape[1]
        out = torch.empty_like(gamma0) if out is None else out
        GR = self._per_graph() * R
        exps = torch.empty(GR, dtype=torch.int32, device=self.device)
        F_trace = torch.empty((steps, GR), dtype=torch.int32, device=self.device) if trace else None
        F_final = torch.empty(GR, dtype=torch.int32, device=self.device)
        self._check(self.lib.sb_graphL_descent(self.h, _ptr(gamma0), _ptr(out), R, float(alpha), steps, renorm_log2,
                                               _ptr(exps), _ptr(F_trace), _ptr(F_final)))
        return out, exps, F_trace, F_final

    def graphL_round(self, gamma, want_flip=False):
        gamma = gamma.contiguous()
        R = gamma.shape[1]
        F = torch.empty(self._per_graph() * R, dtype=torch.int32, device=self.device)
        flip = torch.empty((R, (self.m + 63) // 64), dtype=torch.int64, device=self.device) if want_flip else None
        self._check(self.lib.sb_graphL_round(self.h, _ptr(gamma), R, _ptr(F), _ptr(flip)))
        return F, flip

    def sync(self):
        self._check(self.lib.sb_sync(self.h))

    TUNE_KNOBS = {"bfs_words": 0, "score_blocks_sm": 1, "gl_lanes": 2, "bfs_group": 3, "wait_us": 4,
                  "stall_test": 5, "mst_words": 6}

    def set_tuning(self, **knobs):
        for k, v in knobs.items():
            self._check(self.lib.sb_set_tuning(self.h, self.TUNE_KNOBS[k], int(v)))

    def get_tuning(self):
        out = {}
        for k, i in self.TUNE_KNOBS.items():
            v = ctypes.c_int64()
            self._check(self.lib.sb_get_tuning(self.h, i, ctypes.byref(v)))
            out[k] = v.value
        return out

    def hash_peak(self, seconds=1.0):
        """Measured hashes/s of the BFS parent-key hash mix on this GPU."""
        out = ctypes.c_double()
        self._check(self.lib.sb_hash_peak(self.h, float(seconds), ctypes.byref(out)))
        return out.value

    def stats(self):
        """Work counters of the last sample_trees call."""
        out = np.zeros(6, np.int64)
        self._check(self.lib.sb_stats(self.h, _ptr(out), 6))
        return {"bfs_levels": int(out[0]), "bfs_launches": int(out[1]), "scan_entries": int(out[2]),
                "hashed_candidates": int(out[3]), "second_pass_entries": int(out[4]),
                "hashed_candidates_split_rows": int(out[5])}

    PROF_FAMILIES = ("bfs", "score", "hash", "cloud", "ingest", "gl_rows", "gl_fwd", "other")

    def profile(self, enable: bool):
        self._check(self.lib.sb_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{family: (device ms, launches)} since the last read (resets)."""
        ms = np.zeros(len(self.PROF_FAMILIES), np.float64)
        cnt = np.zeros(len(self.PROF_FAMILIES), np.int64)
        self._check(self.lib.sb_profile_read(self.h, _ptr(ms), _ptr(cnt)))
        return {f: (float(ms[i]), int(cnt[i])) for i, f in enumerate(self.PROF_FAMILIES)}


class GraphLLoss(torch.autograd.Function):
    """graphL relaxed loss (Eq. 3) per start point, with the hand-written
    deterministic CSR adjoint (Eq. 4) as its backward."""

    @staticmethod
    def forward(ctx, gamma, sb: SignedBal):
        loss, _ = sb.graphL_fwd(gamma)
        ctx.save_for_backward(gamma)
        ctx.sb = sb
        return loss

    @staticmethod
    def backward(ctx, gout):
        (gamma,) = ctx.saved_tensors
        return ctx.sb.graphL_bwd(gamma, gout.float()), None


def unpack_labels(words: torch.Tensor, K: int) -> np.ndarray:
    """(n, W) int64 label words -> (K, n) uint8 matrix (helper for checks)."""
    w = words.cpu().numpy().view(np.uint64)
    n, W = w.shape
    bits = ((w[:, :, None] >> np.arange(64, dtype=np.uint64)[None, None, :]) & np.uint64(1)).astype(np.uint8)
    return bits.reshape(n, W * 64)[:, :K].T.copy()
