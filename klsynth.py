"""Seeded synthetic inputs for the indexed limit-set renderer.

This module is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark.  It holds random numbers and workload descriptions only: no part of
the rendering method's arithmetic (generators, seeds, word decode, maps,
pixel binning) lives here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a 64-bit Weyl sequence with
increment 0x9E3779B97F4A7C15 followed by the published 64-bit finaliser.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 stream.  ``next()`` returns the k-th 64-bit draw x_k."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1): the top 53 bits of the next draw times 2^-53."""
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)


def splitmix64_array(seed: int, n: int) -> np.ndarray:
    """First n draws of SplitMix64(seed) as uint64, vectorised (same values as
    calling ``SplitMix64(seed).next()`` n times)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def word_count(depth: int) -> int:
    """Number of reduced words of length ``depth`` over four letters whose
    only relations are the inverse pairs: 4 * 3^(depth-1)."""
    return 4 * 3 ** (depth - 1) if depth >= 1 else 0


def index_sample(seed: int, n: int, depth: int) -> np.ndarray:
    """n word indices i_k = x_k mod N_depth (uint64), from SplitMix64(seed)."""
    x = splitmix64_array(seed, n)
    return (x % np.uint64(word_count(depth))).astype(np.uint64)


@dataclass(frozen=True)
class Group:
    """Trace pair (ta, tb) of a once-punctured-torus group, as complex."""
    ta: complex
    tb: complex


@dataclass(frozen=True)
class RenderConfig:
    """One render: group, word length, view window and image size."""
    name: str
    group: Group
    depth: int
    window: Tuple[float, float, float, float]  # x0, x1, y0, y1
    width: int
    height: int
    precision: str = "fp64"          # "fp64" or "mixed"
    renorm_every: int = 8

    @property
    def n_words(self) -> int:
        return word_count(self.depth)


GASKET = Group(2.0 + 0.0j, 2.0 + 0.0j)
NEAR_CUSP = Group(1.91 + 0.05j, 1.91 + 0.05j)
FUCHSIAN = Group(3.0 + 0.0j, 3.0 + 0.0j)

# Plain FP64 gasket, all 78,732 reduced words of length 10, 1024^2.
C1 = RenderConfig("gasket-d10-1024", GASKET, 10, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, "fp64")
# Same group, length 18 (516,560,652 words), 4096^2; run both plain and mixed.
C2 = RenderConfig("gasket-d18-4096", GASKET, 18, (-1.5, 1.5, -1.5, 1.5), 4096, 4096, "mixed")
C2_FP64 = RenderConfig("gasket-d18-4096-fp64", GASKET, 18, (-1.5, 1.5, -1.5, 1.5), 4096, 4096, "fp64")
# Near-cusp quasi-Fuchsian group, length 20 (4,649,045,868 words), 8192^2.
C3 = RenderConfig("nearcusp-d20-8192", NEAR_CUSP, 20, (-2.0, 2.0, -2.0, 2.0), 8192, 8192, "mixed")

SAMPLE_SEED = 1709
BATCH_SEED = 1709
LOD_TRAIN_SEED = 1710
LOD_HELDOUT_SEED = 1711
# Validation groups for choosing the pruning setting, apart from both the
# training and the held-out groups.
LOD_VALID_SEED = 1712


def draw_groups(seed: int, n: int, depth_lo: int = 12, depth_hi: int = 18
                ) -> List[Tuple[Group, int]]:
    """n (group, depth) pairs: per group, in order, Re ta, Im ta, Re tb, Im tb
    and the depth.  Real parts uniform in [2, 3], imaginary parts uniform in
    [-0.05, 0.05], depth uniform on depth_lo..depth_hi."""
    rng = SplitMix64(seed)
    out = []
    span = depth_hi - depth_lo + 1
    for _ in range(n):
        tar = 2.0 + rng.uniform()
        tai = -0.05 + 0.1 * rng.uniform()
        tbr = 2.0 + rng.uniform()
        tbi = -0.05 + 0.1 * rng.uniform()
        dep = depth_lo + rng.next() % span
        out.append((Group(complex(tar, tai), complex(tbr, tbi)), int(dep)))
    return out


def batch_configs(n_groups: int = 256, seed: int = BATCH_SEED) -> List[RenderConfig]:
    """The batched sweep: n_groups groups, depth 12..18, 1024^2 each over
    [-1.5, 1.5]^2."""
    return [RenderConfig(f"batch-{k}", g, d, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, "mixed")
            for k, (g, d) in enumerate(draw_groups(seed, n_groups))]
