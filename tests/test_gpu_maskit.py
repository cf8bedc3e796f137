"""Maskit's slice at the paper's example mu = -0.097 + 1.838i (b parabolic,
z -> z + 2): limit set and tiling renders, FP64 and mixed, and the paper's
scan with the torus table, against the oracle's renders of the oracle's own
Maskit generators.  Bars as for the other groups: FP64 exact up to edge
words, mixed exact up to words within the mixed tolerance of a pixel edge
(and IoU >= 0.999 for the limit set)."""
import numpy as np
import pytest

import oracle
from conftest import golden_table
from imagecheck import check_fp64_image, iou

pytestmark = pytest.mark.gpu

MU = -0.097 + 1.838j
WINDOW = (-1.0, 1.0, -0.08, 1.92)   # one period of the limit set (b translates by 2)
TOL = {"fp64": 1e-9, "mixed": 2e-5}


@pytest.fixture(scope="module")
def kl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


def tolerance(prec, W, H):
    sx = max(W / (WINDOW[1] - WINDOW[0]), H / (WINDOW[3] - WINDOW[2]))
    zmax = max(1.0, max(abs(complex(x, y)) for x in WINDOW[:2] for y in WINDOW[2:]))
    return TOL[prec] * zmax * sx


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mode,d,W", [("limit", 12, 1024), ("tiling", 10, 768)])
def test_maskit_renders(kl, prec, mode, d, W):
    gl, sl = kl.maskit(MU)
    p = kl.params_group(gl, sl, d, W, W, WINDOW, kl.FP64 if prec == "fp64" else kl.MIXED,
                        mode=kl.TILING if mode == "tiling" else kl.LIMIT_SET)
    img, cnt = kl.render(p)
    img = img.cpu().numpy().view(np.uint32)
    cnt = cnt.cpu().numpy()
    words = 2 * (3 ** d - 1) if mode == "tiling" else oracle.word_count(d)
    assert int(cnt[0]) + int(cnt[1]) == words
    assert int(cnt[0]) == int(img.astype(np.int64).sum())
    g, s = oracle.maskit(MU)
    tol = tolerance(prec, W, W)
    render = oracle.render_tiling if mode == "tiling" else oracle.render
    ref = render(g, s, d, WINDOW, W, W, eta=tol, edge_cap=1 << 22)
    check_fp64_image(img, ref, tol, max_edge_frac=4.0 * tol + 1e-2)
    if prec == "mixed" and mode == "limit":
        assert iou(img, ref.image) >= 0.999


def test_maskit_paper_scan(kl):
    t11 = golden_table("t11_indexed_cayley.txt")
    gl, sl = kl.maskit(MU)
    d, W = 9, 512
    p = kl.params_group(gl, sl, d, W, W, WINDOW, kl.FP64)
    f = kl.fsa_from_params(t11, p)
    img, cnt = kl.render_fsa(f, p)
    img = img.cpu().numpy().view(np.uint32)
    g, s = oracle.maskit(MU)
    tol = tolerance("fp64", W, W)
    ref = oracle.render_fsa(4, t11, oracle.as_matrices(g), oracle.as_points(s), d, WINDOW, W, W,
                            eta=tol, edge_cap=1 << 22)
    assert int(cnt[2].item()) == oracle.word_count(d)
    check_fp64_image(img, ref, tol, max_edge_frac=1e-2)
