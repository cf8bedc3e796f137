"""Comparison of a GPU hit image with an oracle render.

Word values of the GPU path and of the oracle agree up to rounding
(different association: prefix matrix times suffix point against a chain of
point maps).  A word decides the same pixel on both sides unless one of its
pixel coordinates lies within the rounding tolerance `eta` of a pixel edge;
the oracle logs every such "edge word" with its coordinates.  The check is
then exact for all other words and bounded for edge words: removing the edge
words from the oracle image must leave an image S with GPU - S >= 0, every
extra hit at a pixel that is a candidate (floor(c +- eta)) of some edge word,
and the number of extra hits between the number of edge words that must land
and the number of edge words.
"""
import numpy as np


def candidates(c: float, eta: float, n: int):
    opts = {int(np.floor(c - eta)), int(np.floor(c + eta)), int(np.floor(c))}
    inside = sorted(k for k in opts if 0 <= k < n)
    may_drop = any(k < 0 or k >= n for k in opts)
    return inside, may_drop


def check_fp64_image(got: np.ndarray, ref, eta: float, max_edge_frac: float = 1e-3):
    """got: (H, W) integer image from the GPU; ref: oracle.Render with edge
    words logged at band eta.  Raises AssertionError on any inconsistency."""
    H, W = ref.image.shape
    assert got.shape == (H, W)
    n_words = ref.in_window + ref.dropped
    assert ref.edge_total == len(ref.edge_idx), "edge log overflowed"
    assert ref.edge_total <= max_edge_frac * n_words + 100, (ref.edge_total, n_words)
    S = ref.image.astype(np.int64).copy()
    cap = np.zeros((H, W), dtype=np.int64)
    must_land = 0
    for u, v in ref.edge_uv:
        if 0 <= u < W and 0 <= v < H:
            S[int(np.floor(v)), int(np.floor(u))] -= 1
        cols, drop_c = candidates(u, eta, W)
        rows, drop_r = candidates(v, eta, H)
        for r in rows:
            for c in cols:
                cap[r, c] += 1
        if not (drop_c or drop_r):
            must_land += 1
    assert (S >= 0).all()
    D = got.astype(np.int64) - S
    bad = np.argwhere(D < 0)
    assert bad.size == 0, f"GPU misses hits at {bad[:10].tolist()} (non-edge words)"
    over = np.argwhere(D > cap)
    assert over.size == 0, f"GPU extra hits at {over[:10].tolist()} (non-edge words)"
    extra = int(D.sum())
    assert must_land <= extra <= ref.edge_total, (must_land, extra, ref.edge_total)
    return extra


def iou(a: np.ndarray, b: np.ndarray) -> float:
    oa, ob = a > 0, b > 0
    union = np.logical_or(oa, ob).sum()
    return 1.0 if union == 0 else float(np.logical_and(oa, ob).sum()) / float(union)
