"""The index-construction benchmark's host side: arguments and the synthetic collection (CPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_28142_b300 import tac_bench as B  # noqa: E402


def test_defaults_are_the_passage_ranking_shape():
    a = B.parse([])
    assert (a.vectors, a.types, a.zipf, a.budget) == (70_000_000, 30_000, 1.1, 262_144)
    assert a.iters > 0 and a.theta > 0 and a.pq_m in (8, 16, 32)


def test_collection_recipe_on_cpu():
    x, t = B.make_collection(5000, 300, 1.1, seed=3, device="cpu")
    assert x.shape == (5000, 128) and x.dtype == torch.float32 and t.dtype == torch.int32
    assert torch.allclose(x.norm(dim=1), torch.ones(5000), atol=1e-5)
    tn = t.numpy()
    assert tn.min() >= 0 and tn.max() < 300
    counts = np.bincount(tn, minlength=300)
    assert counts[0] > counts[10] > counts[200]  # Zipfian: the first types dominate
    x2, t2 = B.make_collection(5000, 300, 1.1, seed=3, device="cpu")
    assert torch.equal(x, x2) and torch.equal(t, t2)  # seeded


def test_unit_codebooks():
    for m in (8, 16, 32):
        cb = B.unit_codebooks(m, seed=1, device="cpu")
        assert cb.shape == (m, 256, 128 // m)
        assert torch.allclose(cb.norm(dim=-1), torch.full((m, 256), 1.0 / np.sqrt(m)), atol=1e-6)
