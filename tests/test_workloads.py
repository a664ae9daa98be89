"""The seeded input recipe: chunk-local regeneration, the shapes and value
ranges each synthetic workload promises, and the uneven query batches."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("kind,d", [("gauss", 16), ("sift", 16), ("latent", 24), ("sphere", 8)])
def test_rows_regenerate_from_their_chunk_alone(kind, d):
    n = workloads.CHUNK + 1000
    X = workloads.generate(kind, n, d, seed=3, stream=0)
    rows = np.array([0, 5, workloads.CHUNK - 1, workloads.CHUNK, n - 1])
    np.testing.assert_array_equal(workloads.generate(kind, n, d, 3, 0, rows=rows), X[rows])
    # a whole-chunk prefix is the same rows as the longer draw; another
    # stream or seed differs
    C = workloads.CHUNK
    np.testing.assert_array_equal(workloads.generate(kind, C, d, 3, 0), X[:C])
    assert not np.array_equal(workloads.generate(kind, C, d, 3, 1), X[:C])
    assert not np.array_equal(workloads.generate(kind, C, d, 4, 0), X[:C])


def test_sift_like_rows_are_integers_in_byte_range():
    X = workloads.generate("sift", 5000, 32, seed=1, stream=0)
    assert X.dtype == np.float32
    assert X.min() >= 0 and X.max() <= 255
    np.testing.assert_array_equal(X, np.rint(X))


def test_sphere_rows_have_unit_norm():
    X = workloads.generate("sphere", 5000, 96, seed=3, stream=0).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-6)


def test_latent_rows_have_low_intrinsic_dimension():
    # a 64-d latent mixture mapped into d = 200: beyond 64 components only the
    # sigma = 0.05 noise is left
    X = workloads.generate("latent", 4000, 200, seed=2, stream=0).astype(np.float64)
    s = np.linalg.svd(X - X.mean(0), compute_uv=False)
    assert s[64] / s[0] < 0.01


def test_named_configs_have_their_shapes():
    X, Q, k = workloads.workload("c1", n=1000, m=7)
    assert X.shape == (1000, 128) and Q.shape == (7, 128) and k == 10
    X, Q, k = workloads.workload("c3", n=10, m=50)
    assert X.shape == (10, 960) and set(np.unique(k)) <= {10, 20, 50, 100}


def test_batch_sizes_cover_the_stream_with_uneven_batches():
    sizes = workloads.batch_sizes(100_000)
    assert sum(sizes) == 100_000
    assert min(sizes) >= 1 and max(sizes) <= 4096
    assert len(set(sizes)) > 50  # uneven
