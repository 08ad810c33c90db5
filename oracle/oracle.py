"""ctypes wrapper over the plain-C FP64 oracle (test infrastructure only).

Each method cites the passage of the paper it follows; the arithmetic lives in
oracle.c. Function names mirror the steps of Sec. 2.2.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.environ.get("TACHIOM_ORACLE_LIB", os.path.join(_HERE, "liboracle.so"))


def build(force: bool = False, src: str | None = None, out: str | None = None,
          extra=()) -> str:
    """Compile oracle.c with gcc (-O2, OpenMP, strict IEEE: no fast-math)."""
    src = src or os.path.join(_HERE, "oracle.c")
    out = out or os.path.join(_HERE, "liboracle.so")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           *extra, src, "-o", out, "-lm"]
    subprocess.check_call(cmd)
    return out


_P = ct.c_void_p
_I64 = ct.c_int64
_I32 = ct.c_int32


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


class Oracle:
    """Holds one index (host arrays) and the oracle's own inverted lists."""

    def __init__(self, ix: dict, dim: int = 128, lib: str | None = None):
        path = lib or lib_path()
        if lib is None and not os.path.exists(path):
            build()
        self.L = ct.CDLL(path)
        L = self.L
        L.oracle_index_new.restype = _P
        L.oracle_index_new.argtypes = [ct.c_int, _I64, _I64, _I64, ct.c_int, ct.c_int,
                                       _P, _P, _P, _P, _P, _P]
        L.oracle_index_free.argtypes = [_P]
        L.oracle_list_total.restype = _I64
        L.oracle_list_total.argtypes = [_P]
        L.oracle_lists.argtypes = [_P, _P, _P]
        L.oracle_top_centroids.restype = ct.c_int
        L.oracle_top_centroids.argtypes = [_P, _P, _I64, ct.c_int, _P, _P]
        L.oracle_gather.restype = _I64
        L.oracle_gather.argtypes = [_P, _P, ct.c_int, _P, ct.c_int, _P, _P]
        L.oracle_gather_docroute.restype = _I64
        L.oracle_gather_docroute.argtypes = [_P, _P, ct.c_int, _P, ct.c_int, _P, _P]
        L.oracle_select.restype = _I64
        L.oracle_select.argtypes = [_P, _P, _I64, _I64, _P, _P]
        L.oracle_refine.restype = ct.c_int
        L.oracle_refine.argtypes = [_P, _P, ct.c_int, _P, _I64, _P]
        L.oracle_search.restype = ct.c_int
        L.oracle_search.argtypes = [_P, _P, _P, _P, _I32, ct.c_int, ct.c_int, _P, _P, _P, _P, _P, _P]

        self.dim = dim
        cd = ix.get("centroid_dtype", "f32")
        self.cdtype = 1 if cd == "bf16" else 0
        self.cents = np.ascontiguousarray(ix["centroids"])
        self.doc_off = np.ascontiguousarray(ix["doc_offsets"], dtype=np.int64)
        self.tok_cid = np.ascontiguousarray(ix["token_centroid"], dtype=np.int32)
        self.codebooks = np.ascontiguousarray(ix["pq_codebooks"], dtype=np.float32)
        self.codes = np.ascontiguousarray(ix["pq_codes"], dtype=np.uint8)
        rn = ix.get("residual_norms")
        self.rnorm = None if rn is None else np.ascontiguousarray(rn, dtype=np.uint16)
        self.C = self.cents.shape[0]
        self.D = self.doc_off.shape[0] - 1
        self.T = self.tok_cid.shape[0]
        self.M = self.codebooks.shape[0]
        h = L.oracle_index_new(dim, self.C, self.D, self.T, self.M, self.cdtype, _ptr(self.cents),
                               _ptr(self.doc_off), _ptr(self.tok_cid), _ptr(self.codebooks),
                               _ptr(self.codes), _ptr(self.rnorm))
        if not h:
            raise ValueError("oracle: invalid index")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            self.L.oracle_index_free(self.h)
            self.h = None

    def lists(self):
        """The oracle's inverted lists L_j (Sec. 2.2, Index Structure): CSR (off, docs)."""
        n = self.L.oracle_list_total(self.h)
        off = np.empty(self.C + 1, np.int64)
        docs = np.empty(max(n, 1), np.int32)
        self.L.oracle_lists(self.h, _ptr(off), _ptr(docs))
        return off, docs[:n]

    def top_centroids(self, q: np.ndarray, kc: int):
        """Step 1 (Sec. 2.2 Gather 1): exact top-kc centroids per row, (score desc, id asc)."""
        q = np.ascontiguousarray(q, dtype=np.float32)
        n = q.shape[0]
        ids = np.empty((n, kc), np.int32)
        s = np.empty((n, kc), np.float64)
        if self.L.oracle_top_centroids(self.h, _ptr(q), n, kc, _ptr(ids), _ptr(s)):
            raise ValueError("oracle_top_centroids failed")
        return ids, s

    def gather(self, q: np.ndarray, top_ids: np.ndarray, doc_route: bool = False):
        """Steps 2-4 (Sec. 2.2 Gather 2-4) for one query: (docs asc, S~) of every reached doc."""
        q = np.ascontiguousarray(q, dtype=np.float32)
        top_ids = np.ascontiguousarray(top_ids, dtype=np.int32)
        nt, kc = top_ids.shape
        docs = np.empty(max(self.D, 1), np.int32)
        s = np.empty(max(self.D, 1), np.float64)
        f = self.L.oracle_gather_docroute if doc_route else self.L.oracle_gather
        n = f(self.h, _ptr(q), nt, _ptr(top_ids), kc, _ptr(docs), _ptr(s))
        return docs[:n].copy(), s[:n].copy()

    def select(self, docs: np.ndarray, s: np.ndarray, k: int):
        """First k by (score desc, doc asc): Sec. 2.2 truncation to kappa_d, and the final top-k."""
        docs = np.ascontiguousarray(docs, dtype=np.int32)
        s = np.ascontiguousarray(s, dtype=np.float64)
        od = np.empty(max(k, 1), np.int32)
        os_ = np.empty(max(k, 1), np.float64)
        m = self.L.oracle_select(_ptr(docs), _ptr(s), docs.shape[0], k, _ptr(od), _ptr(os_))
        return od[:m].copy(), os_[:m].copy()

    def refine(self, q: np.ndarray, docs: np.ndarray):
        """Step 6 (Sec. 2.2 Refine): S(q,d) = sum_i max_t <q_i, c_a(t) + rho_t r^_t>."""
        q = np.ascontiguousarray(q, dtype=np.float32)
        docs = np.ascontiguousarray(docs, dtype=np.int32)
        out = np.empty(max(docs.shape[0], 1), np.float64)
        if self.L.oracle_refine(self.h, _ptr(q), q.shape[0], _ptr(docs), docs.shape[0], _ptr(out)):
            raise ValueError("oracle_refine: doc id out of range")
        return out[:docs.shape[0]].copy()

    def search(self, queries: np.ndarray, ntok: np.ndarray, k, kc: int, kd: int, stages=False):
        """The whole cascade (Sec. 2.2) for a batch; rows padded with (-1, -inf)."""
        queries = np.ascontiguousarray(queries, dtype=np.float32)
        ntok = np.ascontiguousarray(ntok, dtype=np.int32)
        nq = ntok.shape[0]
        kk = np.full(nq, k, np.int32) if np.isscalar(k) else np.ascontiguousarray(k, dtype=np.int32)
        tot = int(kk.sum())
        od = np.empty(tot, np.int32)
        os_ = np.empty(tot, np.float64)
        tid = ts = cd = cs = None
        if stages:
            R = int(ntok.sum())
            tid = np.empty((R, kc), np.int32)
            ts = np.empty((R, kc), np.float64)
            cd = np.empty((nq, kd), np.int32)
            cs = np.empty((nq, kd), np.float64)
        rc = self.L.oracle_search(self.h, _ptr(queries), _ptr(ntok), _ptr(kk), nq, kc, kd,
                                  _ptr(od), _ptr(os_), _ptr(tid), _ptr(ts), _ptr(cd), _ptr(cs))
        if rc:
            raise ValueError("oracle_search failed")
        res = {"ids": od, "scores": os_, "k": kk}
        if stages:
            res.update(top_ids=tid, top_s=ts, cand_ids=cd, cand_s=cs)
        return res
