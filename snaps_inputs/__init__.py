"""Seeded synthetic asteroid populations shaped like the paper's 15-feature catalogue.

This module is shared input plumbing: the CPU oracle, the tests, the smoke
check and the benchmark all draw their populations from here, so both sides of
every parity check see the same bytes.  It holds none of the outlier method's
arithmetic (no distances, joins, scores or rankings) and imports neither the
oracle nor the CUDA package.

Recipe (the paper's SNAPShot1 / LSST5M catalogues are not available, so this
stands in for them with the same shape: N objects x 15 float32 features):

* features 1-5   ~ Normal(0.5, 0.12)
* features 6-9   ~ LogNormal(0, 0.5)
* features 10-12 ~ Beta(2, 5)
* features 13-15 ~ 0.6 Normal(0.3, 0.08) + 0.4 Normal(0.7, 0.08)
* every column is affinely mapped onto [0, 1] by its own sample range
  (part of the recipe, not the library's normalisation step, which the
  library and the oracle each redo independently), then
* 0.5 % of the rows (chosen by a seeded permutation) are replaced by
  Uniform[0, 1]^15 outliers.

Draw order is fixed so a (n, seed) pair always yields the same bytes:
normal block, lognormal block, beta block, mixture selector, mixture normal,
permutation, outlier values.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 15
OUTLIER_FRACTION = 0.005


def population(n: int, seed: int) -> np.ndarray:
    """Return an (n, 15) C-contiguous float32 population for ``seed``."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    x = np.empty((n, N_FEATURES), dtype=np.float64)
    x[:, 0:5] = rng.normal(0.5, 0.12, size=(n, 5))
    x[:, 5:9] = rng.lognormal(0.0, 0.5, size=(n, 4))
    x[:, 9:12] = rng.beta(2.0, 5.0, size=(n, 3))
    pick_high = rng.random(size=(n, 3)) < 0.4
    mix = rng.normal(0.0, 0.08, size=(n, 3))
    x[:, 12:15] = np.where(pick_high, 0.7, 0.3) + mix
    lo = x.min(axis=0)
    span = x.max(axis=0) - lo
    span[span == 0.0] = 1.0
    x = (x - lo) / span
    n_out = int(round(OUTLIER_FRACTION * n))
    rows = rng.permutation(n)[:n_out]
    x[rows] = rng.random(size=(n_out, N_FEATURES))
    return np.ascontiguousarray(x.astype(np.float32))


def all_masks(f: int = N_FEATURES) -> np.ndarray:
    """Every feature subset of 2..f of ``f`` features as a bitmask (bit j =
    feature j), in ascending mask value; 32,752 masks for f = 15 (Eq. 1)."""
    m = np.arange(1 << f, dtype=np.int64)
    pc = np.array([bin(int(v)).count("1") for v in m])
    return m[pc >= 2].astype(np.uint16)


def mask_sample(count: int, seed: int, f: int = N_FEATURES) -> np.ndarray:
    """A seeded sample of ``count`` distinct masks from :func:`all_masks`,
    returned in ascending mask value."""
    m = all_masks(f)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(m.size, size=min(count, m.size), replace=False))
    return m[pick]


def chunk_sample(count: int, seed: int, f: int = N_FEATURES) -> np.ndarray:
    """``count`` whole blocks of 32 masks (h << 5) | l, l = 0..31, that share a
    high part h over features 5.. of at least two features (so each block holds
    all 32 of its masks), h drawn with ``seed``; ascending mask value."""
    highs = np.array([h for h in range(1 << (f - 5)) if bin(h).count("1") >= 2])
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(highs, size=min(count, highs.size), replace=False))
    return np.array([(int(h) << 5) | low for h in pick for low in range(32)], dtype=np.uint16)


def pairs_and_full(f: int = N_FEATURES) -> np.ndarray:
    """The full f-feature mask plus every two-feature mask (106 for f = 15)."""
    two = [(1 << a) | (1 << b) for a in range(f) for b in range(a + 1, f)]
    return np.array(sorted(two + [(1 << f) - 1]), dtype=np.uint16)
