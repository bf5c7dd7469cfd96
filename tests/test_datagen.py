"""The seeded input generators: deterministic per seed, the shapes and value
ranges the workloads state, and well-formed set rows."""
import numpy as np

from paper_1908_00814_gb300 import datagen


def test_generators_are_deterministic_and_shaped():
    cases = [
        (lambda s: datagen.sift_like(300, 128, seed=s), (300, 128)),
        (lambda s: datagen.sift_manifold(300, 128, seed=s), (300, 128)),
        (lambda s: datagen.bovw_like(300, 500, seed=s), (300, 500)),
        (lambda s: datagen.gist_like(200, 960, seed=s), (200, 960)),
        (lambda s: datagen.clustered_mixture(300, 96, seed=s, normalize=True), (300, 96)),
        (lambda s: datagen.gaussian_mixture(300, 32, seed=s), (300, 32)),
    ]
    for gen, shape in cases:
        a, b, c = gen(1), gen(1), gen(2)
        assert a.shape == shape and a.dtype == np.float32
        assert np.array_equal(a, b) and not np.array_equal(a, c)
        assert np.isfinite(a).all()


def test_value_ranges():
    for X in (datagen.sift_like(500, 128, seed=3), datagen.sift_manifold(500, 128, seed=3)):
        assert X.min() >= 0 and X.max() <= 255 and np.array_equal(X, np.round(X))
    B = datagen.bovw_like(500, 500, seed=3)
    assert B.min() >= 0 and np.array_equal(B, np.round(B)) and (B == 0).mean() > 0.5
    C = datagen.clustered_mixture(200, 96, seed=3, normalize=True)
    assert np.allclose(np.linalg.norm(C, axis=1), 1.0, atol=1e-5)


def test_itemsets_are_valid_csr():
    off, items = datagen.itemsets(2000, 5000, n_types=50, seed=4)
    assert off[0] == 0 and off[-1] == len(items) and (np.diff(off) >= 1).all()
    assert items.dtype == np.int32 and items.min() >= 0 and items.max() < 5000
    for i in range(0, 2000, 37):
        row = items[off[i]:off[i + 1]]
        assert (np.diff(row) > 0).all()                 # ascending, no repeats
    X = datagen.sets_to_rows(off, items, 5000)
    assert np.array_equal(X.sum(1), np.diff(off))
    o2, i2 = datagen.itemsets(2000, 5000, n_types=50, seed=4)
    assert np.array_equal(off, o2) and np.array_equal(items, i2)


def test_workload_table_generates_every_dense_workload():
    for name, w in datagen.WORKLOADS.items():
        if w["kind"] == "sets":
            continue
        X = datagen.generate(name, n=64)
        assert X.shape == (64, w["d"]) and X.dtype == np.float32


def test_sample_nodes_and_batches():
    q = datagen.sample_nodes(1000, 100, seed=0)
    assert len(q) == 100 and len(set(q.tolist())) == 100 and (np.diff(q) > 0).all()
    sizes = datagen.serve_batch_sizes(200, seed=1)
    assert sizes.min() >= 1000 and sizes.max() <= 64000
