"""Sharded render on the GPU (kl_params.shard_index / shard_count), through
the C ABI, on one GPU: every shard of a job is rendered in turn, as the ranks
of a multi-GPU job would render theirs.

  - each FP64 shard image equals the oracle's render of the same shard
    (prefix-slot partition written separately in oracle/kl_oracle.c), exactly
    up to edge words (tests/imagecheck.py);
  - for every precision and for culled renders, the shards' images and
    counters sum bit for bit to the whole render's (same tables, same
    arithmetic per word);
  - degenerate splits: more shards than prefix slots (empty shards), words
    of length 1.
"""
import numpy as np
import pytest

import klsynth
import oracle
from imagecheck import check_fp64_image

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module")
def kl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


def shard_renders(kl, group, d, W, window, prec, n, **f):
    """Images (uint32) and counters of shards 0 .. n-1 and of the whole job."""
    parts = []
    for k in range(n):
        p = kl.params_init(group.ta, group.tb, d, W, W, window, prec, shard_index=k,
                           shard_count=n, **f)
        img, cnt = kl.render(p)
        parts.append((as_u32(img).copy(), cnt.cpu().numpy().copy()))
    p = kl.params_init(group.ta, group.tb, d, W, W, window, prec, **f)
    img, cnt = kl.render(p)
    return parts, (as_u32(img).copy(), cnt.cpu().numpy().copy())


CASES = [(klsynth.GASKET, 12, 512, (-1.5, 1.5, -1.5, 1.5)),
         (klsynth.NEAR_CUSP, 11, 640, (-2.0, 2.0, -2.0, 2.0)),
         (klsynth.draw_groups(klsynth.BATCH_SEED, 4)[3][0], 13, 384, (-1.5, 1.5, -1.5, 1.5))]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("n,pl", [(2, 7), (3, 8), (5, 6)])
def test_fp64_shards_match_the_oracle_shards(kl, case, n, pl):
    group, d, W, window = CASES[case]
    g, s = oracle.group(group.ta, group.tb)
    sx = W / (window[1] - window[0])
    parts, _ = shard_renders(kl, group, d, W, window, kl.FP64, n, prefix_len=pl)
    for k, (img, cnt) in enumerate(parts):
        ref = oracle.render_shard(g, s, d, window, W, W, pl, k, n, eta=TOL64 * sx)
        check_fp64_image(img, ref, TOL64 * sx, max_edge_frac=1e-3)
        assert int(cnt[0]) + int(cnt[1]) == ref.in_window + ref.dropped
        assert int(cnt[0]) == ref.in_window


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cull", [0, 1])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("n", [2, 3, 8])
def test_shards_sum_to_the_whole_render(kl, prec, cull, case, n):
    group, d, W, window = CASES[case]
    parts, (whole, wcnt) = shard_renders(kl, group, d, W, window,
                                         kl.FP64 if prec == "fp64" else kl.MIXED, n, cull=cull)
    img = np.zeros_like(whole)
    cnt = np.zeros_like(wcnt)
    for pi, pc in parts:
        img += pi
        cnt += pc
    assert np.array_equal(img, whole)
    assert np.array_equal(cnt[:3], wcnt[:3])   # in-window, dropped, FP64 words
    words = [int(pc[0]) + int(pc[1]) for _, pc in parts]
    assert sum(words) == kl.word_count(d)


@pytest.mark.parametrize("d,n", [(3, 5), (2, 4), (1, 3), (4, 2)])
def test_empty_shards_and_short_words(kl, d, n):
    """More shards than prefix slots leaves some shards empty; length 1 has
    one prefix slot, held by the last shard."""
    parts, (whole, wcnt) = shard_renders(kl, klsynth.NEAR_CUSP, d, 128, (-2.0, 2.0, -2.0, 2.0),
                                         kl.FP64, n)
    img = sum(pi.astype(np.uint64) for pi, _ in parts)
    cnt = sum(pc for _, pc in parts)
    assert np.array_equal(img, whole.astype(np.uint64))
    assert np.array_equal(cnt[:3], wcnt[:3])


def test_full_size_fp64_shards_sum_to_the_whole(kl):
    """The bench workload's split at 4 and 8 ranks: the near-cusp group at
    length 20, 8192^2, FP64 (the whole render checked against the oracle in
    tests/test_gpu_fullsize.py)."""
    import torch
    c = klsynth.C3
    p = kl.params_init(c.group.ta, c.group.tb, c.depth, c.width, c.height, c.window, kl.FP64)
    r = kl.Renderer(p)
    r()
    whole = r.image.clone()
    wcnt = r.counters.clone()
    for n in (4, 8):
        acc = torch.zeros_like(whole)
        cnt = torch.zeros_like(wcnt)
        for k in range(n):
            q = kl.Params.from_buffer_copy(p)
            q.shard_index, q.shard_count = k, n
            kl.render(q, r.image, r.counters, r.workspace)
            acc += r.image            # int32 addition wraps as uint32 does
            cnt += r.counters
        assert torch.equal(acc, whole)
        assert torch.equal(cnt[:3], wcnt[:3])
