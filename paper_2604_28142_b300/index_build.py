"""Build a searchable index from raw token vectors with the library's own kernels (Sec. 2.1):
Token-Aware Clustering (tachiom_tac_cluster), residual codebook training (tachiom_pq_train) and
residual encoding (tachiom_pq_encode). The result is the index dictionary `Index` loads.

    ix = build_index(vectors, types, doc_offsets, n_types=30000, n_centroids=262144,
                     mu=4, tau=32, eps=2, theta=64.0)
    G = Index(ix)
"""
from __future__ import annotations

import numpy as np

from .binding import pq_encode, pq_train, tac_cluster


def build_index(vectors, types, doc_offsets, n_types: int, n_centroids: int, mu: int, tau: int, eps: int,
                theta: float, iters: int = 10, pq_m: int = 16, pq_sample: int | None = None, pq_iters: int = 10,
                centroid_dtype: str = "f32") -> dict:
    """vectors: torch cuda fp32 [T, 128], the collection's token vectors in document order;
    types: torch cuda int32 [T] token type ids in [0, n_types); doc_offsets: int64 [D + 1] CSR of the
    documents over the tokens. eps must be >= 1 so every token type present gets a centroid.
    centroid_dtype "bf16" stores the centroids rounded to bf16 and encodes the residuals against the
    rounded values (what the index decodes with); "f32" keeps them as computed."""
    import torch
    if eps < 1:
        raise ValueError("build_index needs eps >= 1: every token must have a centroid")
    if centroid_dtype not in ("f32", "bf16"):
        raise ValueError("centroid_dtype must be 'f32' or 'bf16'")
    doc_offsets = np.ascontiguousarray(doc_offsets, dtype=np.int64)
    T = int(vectors.shape[0])
    if doc_offsets[0] != 0 or doc_offsets[-1] != T or np.any(np.diff(doc_offsets) < 0):
        raise ValueError("doc_offsets must run from 0 to the number of vectors, non-decreasing")
    kappa, spread, cents, ctype, labels = tac_cluster(vectors, types, n_types, n_centroids, mu, tau, eps, theta,
                                                      iters)
    if bool((labels < 0).any()):
        raise ValueError("a token type received no centroid")
    if centroid_dtype == "bf16":
        stored = cents.to(torch.bfloat16)
        used = stored.to(torch.float32).contiguous()
        cnp = stored.view(torch.int16).cpu().numpy().view(np.uint16)
    else:
        used = cents
        cnp = cents.cpu().numpy()
    sample = min(T, 1 << 18) if pq_sample is None else pq_sample
    books = pq_train(vectors, used, labels, pq_m, sample, pq_iters)
    codes, rnorm = pq_encode(vectors, used, labels, books)
    torch.cuda.synchronize()
    return {
        "name": "built",
        "centroid_dtype": centroid_dtype,
        "centroids": np.ascontiguousarray(cnp),
        "centroid_type": ctype.cpu().numpy().astype(np.int32),
        "doc_offsets": doc_offsets,
        "token_centroid": labels.cpu().numpy().astype(np.int32),
        "pq_codebooks": books.cpu().numpy().astype(np.float32),
        "pq_codes": np.ascontiguousarray(codes.cpu().numpy()),
        "residual_norms": rnorm.cpu().numpy().view(np.uint16),
        "kappa": kappa,
        "spread": spread,
    }
