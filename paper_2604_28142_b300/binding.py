"""ctypes binding of the C ABI in include/tachiom.h (argument marshalling only).

Every function of the header is exposed under its own name on `lib()`; the
`Index` class is a thin owner of a `tachiom_index*` whose methods take torch
CUDA tensors (for device pointers and the current stream) or numpy arrays (for
host buffers) and call those functions. No step of the search runs in Python.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))

TACHIOM_OK = 0
DTYPE_F32, DTYPE_BF16 = 0, 1
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
FLAG_TOPC_RESCUED, FLAG_SELECT_TIES, FLAG_CAPACITY, FLAG_BAD_INPUT = 1, 2, 4, 8

_STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "CAPACITY", 5: "TIMEOUT", 6: "BUSY"}


class TachiomError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tachiom {_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(ct.Structure):
    _fields_ = [
        ("dim", ct.c_int32), ("n_centroids", ct.c_int64), ("n_docs", ct.c_int64),
        ("n_tokens", ct.c_int64), ("pq_m", ct.c_int32), ("pq_nbits", ct.c_int32),
        ("centroid_dtype", ct.c_int32), ("centroids", ct.c_void_p), ("centroid_type", ct.c_void_p),
        ("doc_offsets", ct.c_void_p), ("token_centroid", ct.c_void_p),
        ("pq_codebooks", ct.c_void_p), ("pq_codes", ct.c_void_p), ("residual_norms", ct.c_void_p),
    ]


class SearchParams(ct.Structure):
    _fields_ = [("kappa_c", ct.c_int32), ("kappa_d", ct.c_int32), ("precision", ct.c_int32),
                ("plan_id", ct.c_int32), ("rescore_margin", ct.c_float)]

    def __init__(self, kappa_c=40, kappa_d=0, precision=PREC_FP32, plan_id=-1, rescore_margin=0.0):
        super().__init__(kappa_c, kappa_d, precision, plan_id, rescore_margin)


class ProfileEntry(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int32), ("total_ms", ct.c_double)]


def profile_enable(on: bool = True):
    _check(lib().tachiom_profile_enable(1 if on else 0))


def profile_read(stream=None) -> dict:
    """{launcher name: (launches, total device ms)} since the previous read (synchronises)."""
    buf = (ProfileEntry * 64)()
    n = ct.c_int32()
    _check(lib().tachiom_profile_read(_stream(stream), buf, 64, ct.byref(n)))
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(n.value)}


class TacParams(ct.Structure):
    _fields_ = [("mu", ct.c_int64), ("tau", ct.c_int64), ("eps", ct.c_int32), ("theta", ct.c_double),
                ("gemm_min_kappa", ct.c_int32)]


def tac_allot(n, s, budget: int, mu: int, tau: int, eps: int, theta: float) -> np.ndarray:
    """Centroids per token type by Token-Aware Clustering's allotment (tachiom_tac_allot): n int64
    occurrences and s float64 spreads per type; returns int32 [n_types] summing to budget."""
    n = np.ascontiguousarray(n, dtype=np.int64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    if n.shape != s.shape or n.ndim != 1:
        raise ValueError("n and s must be 1-d arrays of the same length")
    out = np.zeros(n.shape[0], np.int32)
    p = TacParams(int(mu), int(tau), int(eps), float(theta))
    _check(lib().tachiom_tac_allot(_hp(n), _hp(s), int(n.shape[0]), int(budget), ct.byref(p), _hp(out)))
    return out


def tac_cluster(vectors, types, n_types: int, budget: int, mu: int, tau: int, eps: int, theta: float,
                iters: int, gemm_min_kappa: int = 0, stream=None):
    """Token-Aware Clustering of device vectors (torch cuda fp32 [N, 128]) with device token types
    (torch cuda int32 [N]) through tachiom_tac_cluster. Returns (kappa int32 [n_types] numpy,
    spread float64 [n_types] numpy, centroids fp32 [budget, 128], centroid type int32 [budget],
    labels int32 [N]) - the last three torch cuda tensors."""
    import torch
    n = int(vectors.shape[0])
    kappa = np.zeros(n_types, np.int32)
    spread = np.zeros(n_types, np.float64)
    cents = torch.empty((budget, 128), dtype=torch.float32, device=vectors.device)
    ctype = torch.empty(budget, dtype=torch.int32, device=vectors.device)
    labels = torch.empty(n, dtype=torch.int32, device=vectors.device)
    p = TacParams(int(mu), int(tau), int(eps), float(theta), int(gemm_min_kappa))
    _check(lib().tachiom_tac_cluster(_dp(vectors), _dp(types), n, int(n_types), int(budget), ct.byref(p),
                                     int(iters), _hp(kappa), _hp(spread), _dp(cents), _dp(ctype), _dp(labels),
                                     _stream(stream)))
    return kappa, spread, cents, ctype, labels


def pq_encode(vectors, centroids, labels, codebooks, stream=None):
    """Residual PQ codes and fp16 residual norms (tachiom_pq_encode) of device vectors (torch cuda
    fp32 [N, 128]) given their centroids (fp32 [C, 128]), labels (int32 [N]) and codebooks (fp32
    [M, 256, 128 / M]). Returns (codes uint8 [N, M], rnorm fp16 bits as int16 [N]), torch cuda."""
    import torch
    n, m = int(vectors.shape[0]), int(codebooks.shape[0])
    codes = torch.empty((n, m), dtype=torch.uint8, device=vectors.device)
    rnorm = torch.empty(n, dtype=torch.int16, device=vectors.device)
    _check(lib().tachiom_pq_encode(_dp(vectors), _dp(centroids), _dp(labels), n, _dp(codebooks), m,
                                   _dp(codes), _dp(rnorm), _stream(stream)))
    return codes, rnorm


def pq_train(vectors, centroids, labels, pq_m: int, sample: int, iters: int, stream=None):
    """Residual PQ codebooks fp32 [pq_m, 256, 128 / pq_m] (torch cuda) trained on `sample` of the
    device vectors (tachiom_pq_train), given their centroids and labels."""
    import torch
    books = torch.empty((pq_m, 256, 128 // pq_m), dtype=torch.float32, device=vectors.device)
    _check(lib().tachiom_pq_train(_dp(vectors), _dp(centroids), _dp(labels), int(vectors.shape[0]), int(pq_m),
                                  int(sample), int(iters), _dp(books), _stream(stream)))
    return books


def tc_available() -> bool:
    """True when the current device runs the tensor-core step (a)."""
    return bool(lib().tachiom_tc_available())


class ServerConfig(ct.Structure):
    _fields_ = [("n_slots", ct.c_int32), ("max_batch_queries", ct.c_int32), ("max_batch_rows", ct.c_int32),
                ("max_wait_us", ct.c_int32), ("scratch_budget_bytes", ct.c_int64)]


class ServerStats(ct.Structure):
    _fields_ = [("completed", ct.c_int64), ("batches", ct.c_int64), ("mean_batch", ct.c_double),
                ("p50_ms", ct.c_double), ("p95_ms", ct.c_double), ("p99_ms", ct.c_double), ("qps", ct.c_double)]


def lib_path() -> str:
    return os.environ.get("TACHIOM_LIB", os.path.join(_HERE, "libtachiom.so"))


_LIB = None


def lib():
    """Load libtachiom.so (fails loudly when it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libtachiom.so not found at {path}: run paper_2604_28142_b300/build.py")
    L = ct.CDLL(path)
    P, I32, I64, U32p = ct.c_void_p, ct.c_int32, ct.c_int64, ct.POINTER(ct.c_uint32)
    sig = {
        "tachiom_index_load": ([ct.POINTER(_Desc), ct.c_int, ct.POINTER(ct.c_void_p)], ct.c_int),
        "tachiom_index_free": ([P], ct.c_int),
        "tachiom_index_info": ([P, P, P, P, P, P, P], ct.c_int),
        "tachiom_index_lists": ([P, P, P], ct.c_int),
        "tachiom_search": ([P, ct.POINTER(SearchParams), P, P, P, I32, P, P, P], ct.c_int),
        "tachiom_search_host": ([P, ct.POINTER(SearchParams), P, P, P, I32, P, P, P], ct.c_int),
        "tachiom_top_centroids": ([P, ct.POINTER(SearchParams), P, I32, P, P, P], ct.c_int),
        "tachiom_gather": ([P, ct.POINTER(SearchParams), P, P, I32, P, P, P, P, P], ct.c_int),
        "tachiom_refine": ([P, ct.POINTER(SearchParams), P, P, P, I32, P, P, P, P], ct.c_int),
        "tachiom_centroid_interaction": ([P, ct.POINTER(SearchParams), P, P, P, I32, P, P, P, P], ct.c_int),
        "tachiom_refine_noalloc": ([P, ct.POINTER(SearchParams), P, P, P, I32, P, P, P, P], ct.c_int),
        "tachiom_refine_noalloc_status": ([P, P, U32p], ct.c_int),
        "tachiom_stream_status": ([P, P, U32p], ct.c_int),
        "tachiom_debug_tc_scores": ([P, P, I32, P, P], ct.c_int),
        "tachiom_debug_tc_scores_fp8": ([P, P, I32, P, P, P], ct.c_int),
        "tachiom_debug_wait_timeout": ([P, I32, P], ct.c_int),
        "tachiom_exhaustive_topk": ([P, I32, P, P, I32, I32, P, P, P], ct.c_int),
        "tachiom_autotune_budgets": ([P, I32, P, P, I32, I32, P, I32, P, I32, ct.c_float, P, P, P, P, P, P],
                                     ct.c_int),
        "tachiom_tc_available": ([], ct.c_int),
        "tachiom_debug_topc_groups": ([P, ct.POINTER(SearchParams), P, I32, P], ct.c_int),
        "tachiom_debug_refine_scores": ([P, ct.POINTER(SearchParams), P, P, I32, P, P, P, P], ct.c_int),
        "tachiom_profile_enable": ([ct.c_int], ct.c_int),
        "tachiom_profile_read": ([P, ct.POINTER(ProfileEntry), I32, ct.POINTER(ct.c_int32)], ct.c_int),
        "tachiom_server_create": ([P, ct.POINTER(SearchParams), ct.POINTER(ServerConfig), ct.POINTER(ct.c_void_p)],
                                  ct.c_int),
        "tachiom_server_submit": ([P, P, I32, I32, ct.POINTER(ct.c_uint64)], ct.c_int),
        "tachiom_server_wait": ([P, ct.c_uint64, I32, P, P, ct.POINTER(ct.c_double)], ct.c_int),
        "tachiom_server_read_stats": ([P, ct.POINTER(ServerStats)], ct.c_int),
        "tachiom_server_destroy": ([P], ct.c_int),
        "tachiom_graph_create": ([P, ct.POINTER(SearchParams), P, P, I32, ct.POINTER(ct.c_void_p)], ct.c_int),
        "tachiom_graph_launch": ([P, P, P, P, P], ct.c_int),
        "tachiom_graph_destroy": ([P], ct.c_int),
        "tachiom_autotune": ([P, ct.POINTER(SearchParams), P, P, P, I32, ct.POINTER(ct.c_int32),
                              ct.POINTER(ct.c_float), P], ct.c_int),
        "tachiom_last_error": ([], ct.c_char_p),
        "tachiom_version": ([], ct.c_char_p),
        "tachiom_tac_allot": ([P, P, I32, I64, ct.POINTER(TacParams), P], ct.c_int),
        "tachiom_tac_cluster": ([P, P, I64, I32, I64, ct.POINTER(TacParams), I32, P, P, P, P, P, P], ct.c_int),
        "tachiom_pq_encode": ([P, P, P, I64, P, I32, P, P, P], ct.c_int),
        "tachiom_pq_train": ([P, P, P, I64, I32, I32, I32, P, P], ct.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _LIB = L
    return L


def _check(st: int):
    if st != TACHIOM_OK:
        raise TachiomError(st, lib().tachiom_last_error().decode(errors="replace"))


def _hp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _dp(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


class Index:
    """A loaded index (tachiom_index_load / tachiom_index_free)."""

    def __init__(self, ix: dict, device: int = 0):
        L = lib()
        cd = DTYPE_BF16 if ix.get("centroid_dtype") == "bf16" else DTYPE_F32
        self._keep = {
            "centroids": np.ascontiguousarray(ix["centroids"]),
            "doc_offsets": np.ascontiguousarray(ix["doc_offsets"], dtype=np.int64),
            "token_centroid": np.ascontiguousarray(ix["token_centroid"], dtype=np.int32),
            "pq_codebooks": np.ascontiguousarray(ix["pq_codebooks"], dtype=np.float32),
            "pq_codes": np.ascontiguousarray(ix["pq_codes"], dtype=np.uint8),
        }
        ct_ = ix.get("centroid_type")
        rn = ix.get("residual_norms")
        self._keep["centroid_type"] = None if ct_ is None else np.ascontiguousarray(ct_, dtype=np.int32)
        self._keep["residual_norms"] = None if rn is None else np.ascontiguousarray(rn, dtype=np.uint16)
        k = self._keep
        C = k["centroids"].shape[0]
        D = k["doc_offsets"].shape[0] - 1
        T = k["token_centroid"].shape[0]
        M = k["pq_codebooks"].shape[0]
        d = _Desc(128, C, D, T, M, 8, cd, _hp(k["centroids"]), _hp(k["centroid_type"]),
                  _hp(k["doc_offsets"]), _hp(k["token_centroid"]), _hp(k["pq_codebooks"]),
                  _hp(k["pq_codes"]), _hp(k["residual_norms"]))
        h = ct.c_void_p()
        _check(L.tachiom_index_load(ct.byref(d), device, ct.byref(h)))
        self.h = h
        self.device = device
        self.C, self.D, self.T, self.M = C, D, T, M
        self._keep = None  # the library holds its own copies

    def close(self):
        if getattr(self, "h", None):
            lib().tachiom_index_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        v = [ct.c_int64(), ct.c_int64(), ct.c_int64(), ct.c_int64(), ct.c_int32(), ct.c_int64()]
        _check(lib().tachiom_index_info(self.h, *[ct.byref(x) for x in v]))
        keys = ["n_centroids", "n_docs", "n_tokens", "n_list_entries", "pq_m", "device_bytes"]
        return {k: x.value for k, x in zip(keys, v)}

    def lists(self):
        n = self.info()["n_list_entries"]
        off = np.empty(self.C + 1, np.int64)
        docs = np.empty(max(n, 1), np.int32)
        _check(lib().tachiom_index_lists(self.h, _hp(off), _hp(docs)))
        return off, docs[:n]

    # ---- the calls that take device tensors (torch) -----------------------------
    def search(self, params: SearchParams, queries, ntok: np.ndarray, k: np.ndarray, out_ids,
               out_scores, stream=None):
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        _check(lib().tachiom_search(self.h, ct.byref(params), _dp(queries), _hp(ntok), _hp(k),
                                    int(ntok.shape[0]), _dp(out_ids), _dp(out_scores), _stream(stream)))

    def search_host(self, params: SearchParams, queries: np.ndarray, ntok, k, stream=None):
        queries = np.ascontiguousarray(queries, dtype=np.float32)
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        tot = int(k.sum())
        ids = np.empty(max(tot, 1), np.int32)
        sc = np.empty(max(tot, 1), np.float32)
        _check(lib().tachiom_search_host(self.h, ct.byref(params), _hp(queries), _hp(ntok), _hp(k),
                                         int(ntok.shape[0]), _hp(ids), _hp(sc), _stream(stream)))
        return ids[:tot], sc[:tot]

    def top_centroids(self, params: SearchParams, rows, top_ids, top_scores, stream=None):
        _check(lib().tachiom_top_centroids(self.h, ct.byref(params), _dp(rows), int(rows.shape[0]),
                                           _dp(top_ids), _dp(top_scores), _stream(stream)))

    def gather(self, params: SearchParams, queries, ntok, top_ids, cand_ids, cand_scores, ncand,
               stream=None):
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        _check(lib().tachiom_gather(self.h, ct.byref(params), _dp(queries), _hp(ntok),
                                    int(ntok.shape[0]), _dp(top_ids), _dp(cand_ids), _dp(cand_scores),
                                    _dp(ncand), _stream(stream)))

    def refine(self, params: SearchParams, queries, ntok, k, cand_ids, out_ids, out_scores, stream=None):
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        _check(lib().tachiom_refine(self.h, ct.byref(params), _dp(queries), _hp(ntok), _hp(k),
                                    int(ntok.shape[0]), _dp(cand_ids), _dp(out_ids), _dp(out_scores),
                                    _stream(stream)))

    def centroid_interaction(self, params: SearchParams, queries, ntok, k, cand_ids, out_ids, out_scores,
                             stream=None):
        """Full centroid interaction of given candidate lists (tachiom_centroid_interaction)."""
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        _check(lib().tachiom_centroid_interaction(self.h, ct.byref(params), _dp(queries), _hp(ntok), _hp(k),
                                                  int(ntok.shape[0]), _dp(cand_ids), _dp(out_ids),
                                                  _dp(out_scores), _stream(stream)))

    def debug_tc_scores(self, rows, out, stream=None):
        _check(lib().tachiom_debug_tc_scores(self.h, _dp(rows), int(rows.shape[0]), _dp(out), _stream(stream)))

    def exhaustive_topk(self, precision, queries, ntok, k, stream=None):
        """(ids int32 [nq x k], scores fp32 [nq x k]) of the whole collection (host arrays)."""
        ntok = np.ascontiguousarray(ntok, np.int32)
        nq = len(ntok)
        ids = np.empty((nq, k), np.int32)
        sc = np.empty((nq, k), np.float32)
        _check(lib().tachiom_exhaustive_topk(self.h, int(precision), _dp(queries), _hp(ntok), nq, int(k), _hp(ids),
                                             _hp(sc), _stream(stream)))
        return ids, sc

    def autotune_budgets(self, precision, queries, ntok, k, grid_kc, grid_kd, min_recall=0.95, stream=None):
        """((kappa_c, kappa_d), recall, ms, table [n_kc x n_kd x 4]) of the budget autotuner."""
        ntok = np.ascontiguousarray(ntok, np.int32)
        gc = np.ascontiguousarray(grid_kc, np.int32)
        gd = np.ascontiguousarray(grid_kd, np.int32)
        bkc, bkd = ct.c_int32(0), ct.c_int32(0)
        rec, ms = ct.c_float(0), ct.c_float(0)
        table = np.zeros((len(gc), len(gd), 4), np.float32)
        _check(lib().tachiom_autotune_budgets(self.h, int(precision), _dp(queries), _hp(ntok), len(ntok), int(k),
                                              _hp(gc), len(gc), _hp(gd), len(gd), ct.c_float(min_recall),
                                              ct.byref(bkc), ct.byref(bkd), ct.byref(rec), ct.byref(ms), _hp(table),
                                              _stream(stream)))
        return (bkc.value, bkd.value), rec.value, ms.value, table

    def debug_wait_timeout(self, timeout_us, stream=None):
        _check(lib().tachiom_debug_wait_timeout(self.h, int(timeout_us), _stream(stream)))

    def debug_tc_scores_fp8(self, rows, out, margins=None, stream=None):
        _check(lib().tachiom_debug_tc_scores_fp8(self.h, _dp(rows), int(rows.shape[0]), _dp(out),
                                                 _dp(margins) if margins is not None else None, _stream(stream)))

    def debug_refine_scores(self, params: SearchParams, queries, ntok, cand_ids, out, bounds=None, stream=None):
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        _check(lib().tachiom_debug_refine_scores(self.h, ct.byref(params), _dp(queries), _hp(ntok),
                                                 int(ntok.shape[0]), _dp(cand_ids), _dp(out), _dp(bounds),
                                                 _stream(stream)))

    def autotune(self, params: SearchParams, queries, ntok, k, stream=None):
        """(best plan id, its median ms) for this batch (tachiom_autotune)."""
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        plan = ct.c_int32()
        ms = ct.c_float()
        _check(lib().tachiom_autotune(self.h, ct.byref(params), _dp(queries), _hp(ntok), _hp(k), int(ntok.shape[0]),
                                      ct.byref(plan), ct.byref(ms), _stream(stream)))
        return plan.value, ms.value

    def graph(self, params: SearchParams, ntok, k) -> "Graph":
        return Graph(self, params, ntok, k)

    def debug_topc_groups(self, params: SearchParams, rows) -> np.ndarray:
        out = np.empty(int(rows.shape[0]), np.int32)
        _check(lib().tachiom_debug_topc_groups(self.h, ct.byref(params), _dp(rows), int(rows.shape[0]), _hp(out)))
        return out

    def stream_status(self, stream=None) -> int:
        f = ct.c_uint32()
        _check(lib().tachiom_stream_status(self.h, _stream(stream), ct.byref(f)))
        return f.value


class Server:
    """Continuous-batching request loop (tachiom_server_*) over a loaded Index."""

    def __init__(self, index: Index, params: SearchParams, n_slots: int = 3, max_batch_queries: int = 64,
                 max_batch_rows: int = 2048, max_wait_us: int = 200, scratch_budget_bytes: int = 0):
        self.index = index  # keeps the index alive
        cfg = ServerConfig(n_slots, max_batch_queries, max_batch_rows, max_wait_us, scratch_budget_bytes)
        h = ct.c_void_p()
        _check(lib().tachiom_server_create(index.h, ct.byref(params), ct.byref(cfg), ct.byref(h)))
        self.h = h

    def submit(self, query: np.ndarray, k: int) -> int:
        q = np.ascontiguousarray(query, dtype=np.float32)
        rid = ct.c_uint64()
        _check(lib().tachiom_server_submit(self.h, _hp(q), int(q.shape[0]), int(k), ct.byref(rid)))
        return rid.value

    def wait(self, rid: int, k: int, timeout_ms: int = -1):
        ids = np.empty(k, np.int32)
        sc = np.empty(k, np.float32)
        lat = ct.c_double()
        _check(lib().tachiom_server_wait(self.h, ct.c_uint64(rid), int(timeout_ms), _hp(ids), _hp(sc),
                                         ct.byref(lat)))
        return ids, sc, lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().tachiom_server_read_stats(self.h, ct.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().tachiom_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured search of one batch shape (tachiom_graph_*)."""

    def __init__(self, index: Index, params: SearchParams, ntok, k):
        self.index = index
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        h = ct.c_void_p()
        _check(lib().tachiom_graph_create(index.h, ct.byref(params), _hp(ntok), _hp(k), int(ntok.shape[0]),
                                          ct.byref(h)))
        self.h = h

    def launch(self, queries, out_ids, out_scores, stream=None):
        _check(lib().tachiom_graph_launch(self.h, _dp(queries), _dp(out_ids), _dp(out_scores), _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().tachiom_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
