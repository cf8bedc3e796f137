"""Batched render (kl_batch_*): many groups of uneven depth in one persistent
launch, eagerly or replayed from a captured CUDA graph.

With the same prefix length a group's words are evaluated by the same
arithmetic in a batch as in a single kl_render, so images and counters must
match exactly; a sample of the 256-group sweep is checked against the oracle.
"""
import ctypes

import numpy as np
import pytest

import klsynth
import oracle
from imagecheck import iou

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


def group_params(kl, groups, depths, size, window, precision, **fields):
    return [kl.params_init(g.ta, g.tb, d, size, size, window, precision, **fields)
            for g, d in zip(groups, depths)]


def batch_split(d):
    s = min(8, max(1, d - 7))
    return d - s


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("bt", [64, 128, 256])
def test_batch_equals_single_renders(kl, precision, bt):
    prec = kl.MIXED if precision == "mixed" else kl.FP64
    drawn = klsynth.draw_groups(klsynth.BATCH_SEED, 7)
    groups = [g for g, _ in drawn] + [klsynth.GASKET, klsynth.NEAR_CUSP]
    depths = [8, 13, 9, 12, 2, 11, 10, 12, 11]
    ps = group_params(kl, groups, depths, 384, (-1.5, 1.5, -1.5, 1.5), prec, block_threads=bt)
    for p, d in zip(ps, depths):
        p.prefix_len = batch_split(d)
    b = kl.Batch(ps)
    imgs, cnts = b.render()
    imgs = imgs.cpu().numpy().view(np.uint32)
    cnts = cnts.cpu().numpy()
    for k, p in enumerate(ps):
        img, cnt = kl.render(p)
        assert np.array_equal(imgs[k], img.cpu().numpy().view(np.uint32)), k
        c = cnt.cpu().numpy()
        # in-window, dropped and FP64 words; the atomics counter depends on
        # how the work is cut into items
        assert np.array_equal(cnts[k][:3], c[:3]), (k, cnts[k], c)
        assert int(c[0]) + int(c[1]) == kl.word_count(depths[k])


def test_batch_graph_replays_equal_eager(kl):
    groups = [g for g, _ in klsynth.draw_groups(klsynth.BATCH_SEED, 12)]
    depths = [12, 13, 9, 14, 11, 10, 13, 12, 9, 14, 10, 11]
    ps = group_params(kl, groups, depths, 512, (-1.5, 1.5, -1.5, 1.5), kl.MIXED)
    b = kl.Batch(ps)
    ref_img, ref_cnt = [t.cpu().numpy().copy() for t in b.render()]
    b.capture()
    for _ in range(2):
        b.images.fill_(5)
        img, cnt = b.replay()
        assert np.array_equal(img.cpu().numpy(), ref_img)
        assert np.array_equal(cnt.cpu().numpy(), ref_cnt)


def test_batch_rejects_mixed_frames(kl):
    a = kl.params_init(2 + 0j, 2 + 0j, 8, 256, 256, (-1.5, 1.5, -1.5, 1.5), kl.MIXED)
    c = kl.params_init(2 + 0j, 2 + 0j, 8, 128, 256, (-1.5, 1.5, -1.5, 1.5), kl.MIXED)
    with pytest.raises(kl.KlError) as e:
        kl.Batch([a, c])
    assert e.value.status == 1
    h = ctypes.c_void_p()
    assert kl.lib().kl_batch_create((kl.Params * 1)(a), 0, ctypes.byref(h)) == 1


def test_sweep_sample_against_oracle(kl):
    """16 groups of the seeded 256-group sweep (depth 12..18, 1024^2), rendered
    in one batch, each against its own oracle render."""
    cfgs = klsynth.batch_configs(16)
    ps = [kl.params_init(c.group.ta, c.group.tb, c.depth, c.width, c.height, c.window, kl.MIXED)
          for c in cfgs]
    b = kl.Batch(ps)
    b.capture()
    imgs, cnts = b.replay()
    imgs = imgs.cpu().numpy().view(np.uint32)
    cnts = cnts.cpu().numpy()
    for k, c in enumerate(cfgs):
        g, s = oracle.group(c.group.ta, c.group.tb)
        ref = oracle.render(g, s, c.depth, c.window, c.width, c.height)
        assert int(cnts[k][0]) + int(cnts[k][1]) == c.n_words
        assert abs(int(cnts[k][0]) - ref.in_window) <= max(10, 1e-4 * ref.in_window)
        v = iou(imgs[k], ref.image)
        assert v >= 0.999, (k, c.depth, v)
