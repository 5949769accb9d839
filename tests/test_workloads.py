"""The seeded input generators: deterministic per seed, and the shapes,
ranges and structure the workload recipes state."""
import numpy as np

from paper_1403_7394_gb300 import workloads as W


def test_generators_are_deterministic_per_seed():
    for gen in (lambda s: W.gmm_points(300, 5, 7, 0.5, seed=s), lambda s: W.texture_patches(300, 16, seed=s),
                lambda s: W.tiny_instance(9, 3, seed=s)):
        a, la = gen(4)
        b, lb = gen(4)
        c, _ = gen(5)
        assert np.array_equal(a, b) and np.array_equal(la, lb)
        assert not np.array_equal(a, c)


def test_workload_shapes_and_ranges():
    X0, l0 = W.config0()
    assert X0.shape == (500, 2) and X0.dtype == np.float64 and set(np.unique(l0)) <= set(range(10))
    X1, l1 = W.config1()
    assert X1.shape == (8192, 64) and len(np.unique(l1)) == 64
    X2, l2 = W.config2()
    assert X2.shape == (32768, 192) and X2.min() >= 0.0 and X2.max() <= 1.0
    assert len(np.unique(l2)) == 256
    X4, l4 = W.config4()
    assert X4.shape == (262144, 32) and len(np.unique(l4)) == 1024
    # means ~ N(0, 4 I) and unit noise: per-coordinate variance close to 4 + 1
    assert abs(X4.var(axis=0).mean() - 5.0) < 0.5


def test_tiny_instances_use_every_component():
    for s in range(10):
        X, lab = W.tiny_instance(8, 3, seed=s)
        assert X.shape == (8, 2) and set(lab) == {0, 1, 2}


def test_batch_instances_ranges():
    inst = W.batch_instances(count=40, seed=1)
    assert len(inst) == 40
    for b in inst:
        n, d = b["X"].shape
        assert 200 <= n <= 4000 and d == 32 and b["L"] in (2, 3, 4)
        assert 5 <= len(np.unique(b["labels"])) <= 50
    # one seed per instance
    assert len({b["seed"] for b in inst}) == 40


def test_sample_pairs_are_off_diagonal():
    i, j = W.sample_pairs(1000, 100000, seed=3)
    assert np.all(i != j) and i.min() >= 0 and j.min() >= 0 and i.max() < 1000 and j.max() < 1000
    # every ordered off-diagonal pair is equally likely: j is not biased towards i + 1
    assert abs(np.mean(j > i) - 0.5) < 0.01
