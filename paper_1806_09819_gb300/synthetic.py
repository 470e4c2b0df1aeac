"""Seeded synthetic MNIST-shaped inputs (stand-in for the paper's MNIST, Section 4).

This module holds input generation only -- none of the method's arithmetic --
and is the one piece both the CUDA path and the oracle are fed from.

Recipe: 28x28 = 784 pixels, 10 classes.  Each class has a smooth template,
the sum of 3-5 isotropic Gaussian blobs (random centres, widths 2-5 px,
amplitudes 0.5-1), scaled to [0, 1].  An image of class y is
round(clip(T_y + N(0, 0.2^2), 0, 1) * 255) / 255; labels are uniform over the
10 classes.  Train 60k / test 10k images from data seed 1234; minibatch
indices come from their own seed (5678), sampled without replacement within a
batch and independently per generation.
"""
from __future__ import annotations

import numpy as np

SIDE = 28
PIXELS = SIDE * SIDE
CLASSES = 10
DATA_SEED = 1234
BATCH_SEED = 5678


def templates(seed: int = DATA_SEED) -> np.ndarray:
    """float64[10, 784] smooth class templates in [0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:SIDE, 0:SIDE].astype(np.float64)
    out = np.empty((CLASSES, PIXELS), dtype=np.float64)
    for k in range(CLASSES):
        img = np.zeros((SIDE, SIDE))
        for _ in range(int(rng.integers(3, 6))):
            cy, cx = rng.uniform(4.0, SIDE - 4.0, size=2)
            width = rng.uniform(2.0, 5.0)
            amp = rng.uniform(0.5, 1.0)
            img += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * width * width))
        img -= img.min()
        img /= max(img.max(), 1e-12)
        out[k] = img.reshape(-1)
    return out


def make_split(n: int, seed: int, tmpl: np.ndarray | None = None, noise: float = 0.2):
    """(x float32[n, 784] with values k/255, y int32[n])."""
    tmpl = templates() if tmpl is None else tmpl
    rng = np.random.Generator(np.random.PCG64(seed))
    y = rng.integers(0, CLASSES, size=n).astype(np.int32)
    x = tmpl[y] + rng.normal(0.0, noise, size=(n, PIXELS))
    x = np.rint(np.clip(x, 0.0, 1.0) * 255.0) / 255.0
    return x.astype(np.float32), y


def to_levels(x: np.ndarray) -> np.ndarray:
    """The 8-bit levels k of images x = k / 255 (uint8, same shape)."""
    k = np.rint(np.asarray(x, dtype=np.float64) * 255.0)
    assert np.all((k >= 0) & (k <= 255)) and np.all(np.float32(k / 255.0) == np.asarray(x, dtype=np.float32))
    return k.astype(np.uint8)


def dataset(n_train: int = 60000, n_test: int = 10000, seed: int = DATA_SEED):
    """((x_train, y_train), (x_test, y_test)) of the synthetic stand-in."""
    tmpl = templates(seed)
    train = make_split(n_train, seed + 1, tmpl)
    test = make_split(n_test, seed + 2, tmpl)
    return train, test


def batch_indices(n_items: int, batch: int, generations: int, seed: int = BATCH_SEED) -> np.ndarray:
    """int64[generations, batch]: per generation, a batch drawn without replacement."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((generations, batch), dtype=np.int64)
    for g in range(generations):
        out[g] = rng.choice(n_items, size=batch, replace=False)
    return out


def tiny_problem(d_in: int, d_out: int, batch: int, seed: int):
    """Small seeded inputs for brute-force cases (e.g. 2-2-2 nets): x ~ U(-1, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(-1.0, 1.0, size=(batch, d_in)).astype(np.float32)
    y = rng.integers(0, d_out, size=batch).astype(np.int32)
    return x, y


def random_population(pop: int, c: int, seed: int, scale: float = 0.1) -> np.ndarray:
    """float32[pop, c] of seeded N(0, scale^2) genes (a state to start lock-step tests from)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.normal(0.0, scale, size=(pop, c))).astype(np.float32)
