"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA library's
callers.  This module holds no arithmetic of the method: only random parameter
streams and the fixed parameter lists of the test problems.

SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) produces the hump parameters, so that any consumer
can regenerate the same list from the seed.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        # 53 random bits -> [0, 1)
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def dambreak_params(x0=0.5, y0=0.5, r2=0.04, h_in=2.0, h_out=1.0):
    """Radial dam break: h = h_in where (x-x0)^2 + (y-y0)^2 < r2, else h_out."""
    return np.array([x0, y0, r2, h_in, h_out], dtype=np.float64)


def humps_params(n_humps=64, seed=1, amp=(0.1, 0.5), width=(0.01, 0.05), base=1.0):
    """Random Gaussian humps on depth `base`: per hump (A, w, cx, cy) drawn in that
    order from SplitMix64(seed); h = base + sum A exp(-|x - c|^2 / w^2)."""
    g = SplitMix64(seed)
    p = [base]
    for _ in range(n_humps):
        A = g.uniform(*amp)
        w = g.uniform(*width)
        cx = g.uniform()
        cy = g.uniform()
        p += [A, w, cx, cy]
    return np.array(p, dtype=np.float64)


def random_forest_flags(n: int, seed: int, p_refine=0.3, p_coarsen=0.3) -> np.ndarray:
    """Random per-leaf flags in {-1, 0, +1} for topology tests."""
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    f = np.zeros(n, np.int8)
    f[u < p_refine] = 1
    f[(u >= p_refine) & (u < p_refine + p_coarsen)] = -1
    return f


def random_swe_state(n_patches: int, m: int, seed: int, h0=1.0, dh=0.3, vel=0.2) -> np.ndarray:
    """Smooth-ish random shallow-water state [n][3][m][m] with h > 0."""
    rng = np.random.default_rng(seed)
    h = h0 + dh * rng.random((n_patches, m, m))
    hu = h * vel * (2 * rng.random((n_patches, m, m)) - 1)
    hv = h * vel * (2 * rng.random((n_patches, m, m)) - 1)
    return np.stack([h, hu, hv], axis=1)


def random_unbalanced_leaves(seed: int, max_level: int = 5, ntrees: int = 1, p_split: float = 0.35):
    """Leaves (tree, level, x, y) of a random forest built by random splits,
    not balanced; for topology tests."""
    rng = np.random.default_rng(seed)
    leaves = [(t, 0, 0, 0) for t in range(ntrees)]
    for _ in range(max_level):
        new = []
        for (t, l, x, y) in leaves:
            if l < max_level and rng.random() < p_split:
                new += [(t, l + 1, 2 * x + (c & 1), 2 * y + (c >> 1)) for c in range(4)]
            else:
                new.append((t, l, x, y))
        leaves = new
    return leaves
