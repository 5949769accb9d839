"""Seeded synthetic inputs shaped like the paper's workloads.

Only point sets are generated here (no similarities, preferences or any other
part of the clustering method), so the CUDA library and the FP64 reference
can both consume them without sharing arithmetic.  All generators use numpy's
PCG64 ``default_rng(seed)`` and return float64 arrays.

The paper's own data (the 788-point "Aggregation" shape set and the Mandrill
and Buttons images of §4) are not available; these stand in for them:
  * ``gmm_points``: isotropic Gaussian mixtures (2-D point data of §4.2 and
    higher-dimensional feature vectors),
  * ``texture_patches``: 8x8x3 image patches drawn from procedural textures
    (the image-segmentation workloads of §4.1, which cluster RGB pixels).
"""
from __future__ import annotations

import numpy as np


def gmm_points(n: int, d: int, k: int, sigma: float, seed: int = 0,
               means: str = "uniform", mean_scale: float = 10.0):
    """n points in d dimensions from a k-component isotropic Gaussian mixture.

    means="uniform": component means uniform in [-mean_scale, mean_scale]^d;
    means="normal":  component means ~ N(0, mean_scale^2 I).
    Labels are uniform over the components.  Returns (X, labels)."""
    rng = np.random.default_rng(seed)
    if means == "uniform":
        mu = rng.uniform(-mean_scale, mean_scale, size=(k, d))
    elif means == "normal":
        mu = rng.normal(0.0, mean_scale, size=(k, d))
    else:
        raise ValueError(f"unknown means={means!r}")
    labels = rng.integers(0, k, size=n)
    X = mu[labels] + rng.normal(0.0, sigma, size=(n, d))
    return X, labels


def texture_patches(n: int, n_prototypes: int = 256, patch: int = 8,
                    noise: float = 0.05, seed: int = 0):
    """n flattened patch x patch x 3 image patches with values in [0, 1].

    Each prototype is, per channel, a base colour plus two or three random
    oriented sinusoids (random frequency and phase), clipped to [0, 1].  Patch
    i uses prototype perm[i mod n_prototypes] (a seeded shuffle) with Gaussian
    noise of std ``noise`` added and clipped again.  Returns (X, labels)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(patch), np.arange(patch), indexing="ij")
    protos = np.empty((n_prototypes, patch, patch, 3))
    for p in range(n_prototypes):
        for ch in range(3):
            img = np.full((patch, patch), rng.uniform(0.2, 0.8))
            for _ in range(int(rng.integers(2, 4))):
                theta = rng.uniform(0.0, np.pi)
                freq = rng.uniform(0.05, 0.45)
                phase = rng.uniform(0.0, 2.0 * np.pi)
                amp = rng.uniform(0.05, 0.25)
                img = img + amp * np.sin(2.0 * np.pi * freq *
                                         (np.cos(theta) * xx + np.sin(theta) * yy) + phase)
            protos[p, :, :, ch] = np.clip(img, 0.0, 1.0)
    perm = rng.permutation(n_prototypes)
    labels = perm[np.arange(n) % n_prototypes]
    X = protos[labels].reshape(n, -1) + rng.normal(0.0, noise, size=(n, patch * patch * 3))
    return np.clip(X, 0.0, 1.0), labels


def tiny_instance(n: int, k: int, sigma: float = 0.3, seed: int = 0):
    """A tiny 2-D mixture (n <= 10) for exhaustive checks: k means uniform in
    [-3, 3]^2, every component used at least once."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-3.0, 3.0, size=(k, 2))
    labels = np.concatenate([np.arange(k), rng.integers(0, k, size=n - k)])
    rng.shuffle(labels)
    X = mu[labels] + rng.normal(0.0, sigma, size=(n, 2))
    return X, labels


def batch_instances(count: int = 256, n_range=(200, 4000), levels=(2, 3, 4),
                    d: int = 32, k_range=(5, 50), seed: int = 0):
    """``count`` independent mixtures with N uniform in n_range, L uniform in
    ``levels`` and 5-50 components each (means ~ N(0, 4 I), sigma = 1), one
    seed per instance.  Returns a list of dicts {X, labels, L, seed}."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        L = int(rng.choice(levels))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        s = int(rng.integers(0, 2**31 - 1))
        X, lab = gmm_points(n, d, k, sigma=1.0, seed=s, means="normal", mean_scale=2.0)
        out.append({"X": X, "labels": lab, "L": L, "seed": s})
    return out


def sample_pairs(n: int, count: int, seed: int = 0):
    """``count`` seeded (i, j) index pairs with i != j, for sampled statistics
    of an n x n similarity matrix."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, size=count)
    j = rng.integers(0, n - 1, size=count)
    j = j + (j >= i)
    return i, j


# The five workload families (sizes of the benchmark configurations).
def config0(seed: int = 0):
    """N = 500 points in 2-D, 10 components, means uniform in [-10, 10]^2,
    sigma = 0.5 (stands in for the 788-point 2-D shape set of §4.2)."""
    return gmm_points(500, 2, 10, sigma=0.5, seed=seed, means="uniform", mean_scale=10.0)


def config1(seed: int = 0):
    """N = 8192 points in 64-D, 64 components, means ~ N(0, 4 I), sigma = 1."""
    return gmm_points(8192, 64, 64, sigma=1.0, seed=seed, means="normal", mean_scale=2.0)


def config2(seed: int = 0):
    """N = 32768 8x8x3 texture patches (d = 192) from 256 prototypes."""
    return texture_patches(32768, 256, 8, 0.05, seed=seed)


def config4(seed: int = 0):
    """N = 262144 points in 32-D, 1024 components, means ~ N(0, 4 I)."""
    return gmm_points(262144, 32, 1024, sigma=1.0, seed=seed, means="normal", mean_scale=2.0)
