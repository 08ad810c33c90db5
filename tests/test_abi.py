"""The C ABI on the CPU: the library loads, exports every declared symbol, and
rejects malformed arguments on the host before any device work (no GPU needed)."""
import ctypes as ct
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2604_28142_b300 as T
from paper_2604_28142_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "tachiom.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(tachiom_[a-z_0-9]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_28142_b300 import build
    build.build()
    return T.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10, names
    out = subprocess.check_output(["nm", "-D", "--defined-only", T.lib_path()]).decode()
    exported = set(re.findall(r"\bT (tachiom_[a-z_0-9]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_version_and_empty_error(lib):
    assert b"sm_103a" in lib.tachiom_version()
    assert isinstance(lib.tachiom_last_error(), bytes)


def _desc(**over):
    C, D = 4, 2
    arrs = {
        "centroids": np.zeros((C, 128), np.float32),
        "doc_offsets": np.array([0, 2, 3], np.int64),
        "token_centroid": np.array([0, 1, 3], np.int32),
        "pq_codebooks": np.zeros((16, 256, 8), np.float32),
        "pq_codes": np.zeros((3, 16), np.uint8),
    }
    arrs.update({k: v for k, v in over.items() if isinstance(v, np.ndarray)})
    f = dict(dim=128, n_centroids=arrs["centroids"].shape[0], n_docs=arrs["doc_offsets"].shape[0] - 1,
             n_tokens=arrs["token_centroid"].shape[0], pq_m=16, pq_nbits=8, centroid_dtype=0)
    f.update({k: v for k, v in over.items() if not isinstance(v, np.ndarray)})
    d = B._Desc(f["dim"], f["n_centroids"], f["n_docs"], f["n_tokens"], f["pq_m"], f["pq_nbits"],
                f["centroid_dtype"], B._hp(arrs["centroids"]), None, B._hp(arrs["doc_offsets"]),
                B._hp(arrs["token_centroid"]), B._hp(arrs["pq_codebooks"]), B._hp(arrs["pq_codes"]), None)
    return d, arrs


@pytest.mark.parametrize("over,msg", [
    (dict(dim=64), b"dim"),
    (dict(pq_m=12), b"pq_m"),
    (dict(pq_nbits=4), b"pq_nbits"),
    (dict(centroid_dtype=7), b"centroid_dtype"),
    (dict(doc_offsets=np.array([0, 3, 2], np.int64)), b"monotone"),
    (dict(doc_offsets=np.array([1, 2, 3], np.int64)), b"doc_offsets[0]"),
    (dict(token_centroid=np.array([0, 4, 1], np.int32)), b"out of [0, C)"),
    (dict(token_centroid=np.array([0, -1, 1], np.int32)), b"out of [0, C)"),
    (dict(n_tokens=5), b"n_tokens"),
    (dict(n_centroids=0), b"n_centroids"),
])
def test_index_load_rejects_malformed(lib, over, msg):
    d, keep = _desc(**over)
    h = ct.c_void_p()
    st = lib.tachiom_index_load(ct.byref(d), 0, ct.byref(h))
    assert st == 1, st
    assert not h.value
    assert msg in lib.tachiom_last_error()


def test_null_arguments(lib):
    h = ct.c_void_p()
    assert lib.tachiom_index_load(None, 0, ct.byref(h)) == 1
    p = B.SearchParams()
    assert lib.tachiom_search(None, ct.byref(p), None, None, None, 0, None, None, None) == 1
    assert lib.tachiom_index_free(None) == 0
    f = ct.c_uint32()
    assert lib.tachiom_stream_status(None, None, ct.byref(f)) == 1
