"""Tiling mode (every node of the word tree, all lengths 1 .. d) through the
C ABI against the oracle's tiling render.  Every node is counted:
in-window + dropped = 2 (3^d - 1).  FP64 images are exact up to edge words
(words within 1e-9 max(1, |z|) of a pixel edge).  Mixed images are held to
the same check at the mixed tolerance, 2e-5 max(1, |z|): every word farther
than that from a pixel edge must land in the oracle's pixel.  (Occupancy IoU
is a weaker bar here: the short words of the gasket sit on exact rational
points such as 0 and +-i, on pixel edges of these grids, and each of them may
be the only hit of its pixel.)"""
import numpy as np
import pytest

import klsynth
import oracle
from imagecheck import check_fp64_image, iou

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 2e-5


@pytest.fixture(scope="module")
def kl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


CASES = [
    (klsynth.GASKET, 10, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, {}),
    (klsynth.NEAR_CUSP, 12, (-2.0, 2.0, -2.0, 2.0), 768, 512, {}),
    (klsynth.draw_groups(klsynth.BATCH_SEED, 3)[2][0], 11, (-1.5, 1.5, -1.5, 1.5), 600, 600,
     {"prefix_len": 4}),
]


@pytest.mark.parametrize("group,d,window,W,H,fields", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tiling_image(kl, group, d, window, W, H, fields, precision):
    prec = kl.FP64 if precision == "fp64" else kl.MIXED
    p = kl.params_init(group.ta, group.tb, d, W, H, window, prec, mode=kl.TILING, **fields)
    img, cnt = kl.render(p)
    img = img.cpu().numpy().view(np.uint32)
    cnt = cnt.cpu().numpy()
    assert int(cnt[0]) + int(cnt[1]) == 2 * (3 ** d - 1)
    assert int(cnt[0]) == int(img.astype(np.int64).sum())
    g, s = oracle.group(group.ta, group.tb)
    sx = max(W / (window[1] - window[0]), H / (window[3] - window[2]))
    zmax = max(1.0, max(abs(complex(x, y)) for x in window[:2] for y in window[2:]))
    tol = (TOL64 if prec == kl.FP64 else TOL32) * zmax * sx
    ref = oracle.render_tiling(g, s, d, window, W, H, eta=tol, edge_cap=1 << 22)
    # about 4 tol of the words fall within tol of a pixel edge (two coordinates,
    # two sides), plus the exact rational points of the short words: the
    # sanity bound on their number
    check_fp64_image(img, ref, tol, max_edge_frac=4.0 * tol + 1e-2)
    if prec == kl.MIXED:
        assert iou(img, ref.image) >= 0.998


def test_tiling_is_the_sum_of_the_lengths_and_accumulates(kl):
    import torch
    g = klsynth.NEAR_CUSP
    d, W, H, window = 9, 256, 256, (-2.0, 2.0, -2.0, 2.0)
    total = np.zeros((H, W), dtype=np.int64)
    for k in range(1, d + 1):
        p = kl.params_init(g.ta, g.tb, k, W, H, window, kl.FP64)
        img, _ = kl.render(p)
        total += img.cpu().numpy().view(np.uint32).astype(np.int64)
    p = kl.params_init(g.ta, g.tb, d, W, H, window, kl.FP64, mode=kl.TILING)
    img, cnt = kl.render(p)
    assert np.array_equal(img.cpu().numpy().view(np.uint32).astype(np.int64), total)
    p.accumulate = 1
    kl.render(p, img, cnt)
    assert np.array_equal(img.cpu().numpy().view(np.uint32).astype(np.int64), 2 * total)
    assert int(cnt.cpu()[0]) + int(cnt.cpu()[1]) == 4 * (3 ** d - 1)
    torch.cuda.synchronize()
