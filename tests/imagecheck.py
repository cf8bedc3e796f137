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


def check_band_image(got: np.ndarray, ref, eta: float):
    """check_fp64_image for large edge logs (vectorised), same rules: with
    S = the oracle image less its edge words, GPU - S must be >= 0, at most
    the number of edge words whose candidate pixels (floor(c +- eta) in each
    coordinate) include the pixel, and its total between the edge words that
    cannot leave the window and all edge words.  eta < 1/2.  Returns the
    number of edge-word hits the GPU image holds."""
    assert eta < 0.5
    H, W = ref.image.shape
    assert got.shape == (H, W)
    assert ref.edge_total == len(ref.edge_idx), "edge log overflowed"
    u = ref.edge_uv[:, 0]
    v = ref.edge_uv[:, 1]
    S = ref.image.astype(np.int64).ravel().copy()
    ins = (u >= 0) & (u < W) & (v >= 0) & (v < H)
    own = np.floor(v[ins]).astype(np.int64) * W + np.floor(u[ins]).astype(np.int64)
    S -= np.bincount(own, minlength=H * W)
    assert (S >= 0).all()
    c_lo, c_hi = np.floor(u - eta), np.floor(u + eta)
    r_lo, r_hi = np.floor(v - eta), np.floor(v + eta)
    cap = np.zeros(H * W, dtype=np.int64)
    for r, rok in ((r_lo, np.ones_like(u, dtype=bool)), (r_hi, r_hi != r_lo)):
        for c, cok in ((c_lo, np.ones_like(u, dtype=bool)), (c_hi, c_hi != c_lo)):
            sel = rok & cok & (r >= 0) & (r < H) & (c >= 0) & (c < W)
            cap += np.bincount(r[sel].astype(np.int64) * W + c[sel].astype(np.int64),
                               minlength=H * W)
    may_drop = (c_lo < 0) | (c_hi >= W) | (r_lo < 0) | (r_hi >= H)
    must_land = int((~may_drop).sum())
    D = got.astype(np.int64).ravel() - S
    assert (D >= 0).all(), f"GPU misses hits at {np.argwhere(D < 0)[:10].ravel().tolist()}"
    assert (D <= cap).all(), f"GPU extra hits at {np.argwhere(D > cap)[:10].ravel().tolist()}"
    extra = int(D.sum())
    assert must_land <= extra <= ref.edge_total, (must_land, extra, ref.edge_total)
    return extra
