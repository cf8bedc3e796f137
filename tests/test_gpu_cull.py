"""Culled renders (kl_params.cull = 1) through the C ABI.

A certified block is tallied without evaluating its words, so the culled
image must be the per-word image itself: bit for bit, with the same
in-window, dropped and FP64-word counts, against the per-word render that
uses the same prefix/suffix split (the split fixes the FP32 rounding).  Both
precisions are also checked against the oracle with the per-word renders'
tolerances: FP64 exact up to edge words, mixed exact for words farther than
the mixed tolerance from a pixel edge.
"""
import numpy as np
import pytest

import klsynth
import oracle
from imagecheck import check_fp64_image, iou

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 2e-5

def cull_suffix(d):
    """Suffix letters of the culled render's own split: d - 1 up to 9, then
    about half the word plus one, 9 .. 12."""
    return d - 1 if d - 1 <= 9 else min(12, max(9, d // 2 + 1))


GROUPS = {
    "gasket": klsynth.GASKET,
    "nearcusp": klsynth.NEAR_CUSP,
    "fuchsian": klsynth.FUCHSIAN,
    "batch0": klsynth.draw_groups(klsynth.BATCH_SEED, 1)[0][0],
    "batch7": klsynth.draw_groups(klsynth.BATCH_SEED, 8)[7][0],
}


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


def culled_and_per_word(kl, group, d, window, W, H, precision, **fields):
    """(culled image, counters), (per-word image, counters) on one split:
    the caller's prefix length if given, else the culled render's own."""
    plen = fields.pop("prefix_len", 0)
    pc = kl.params_init(group.ta, group.tb, d, W, H, window, precision, cull=1,
                        prefix_len=plen, **fields)
    pw = kl.params_init(group.ta, group.tb, d, W, H, window, precision,
                        prefix_len=plen or d - cull_suffix(d), **fields)
    ic, cc = kl.render(pc)
    iw, cw = kl.render(pw)
    return (as_u32(ic), cc.cpu().numpy()), (as_u32(iw), cw.cpu().numpy())


def assert_same(c, w, n_words):
    (ic, cc), (iw, cw) = c, w
    assert int(cc[0]) + int(cc[1]) == n_words
    assert np.array_equal(cc[:3], cw[:3])
    diff = np.flatnonzero(ic != iw)
    assert diff.size == 0, f"{diff.size} pixels differ, first {diff[:5]}"


CASES = [
    ("gasket", 10, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, {}),
    ("gasket", 13, (-1.5, 1.5, -1.5, 1.5), 2048, 2048, {}),
    ("nearcusp", 12, (-2.0, 2.0, -2.0, 2.0), 1536, 1024, {}),
    ("batch0", 12, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, {}),
    ("fuchsian", 11, (-1.1, 1.1, -1.1, 1.1), 777, 513, {}),
    ("batch7", 11, (-1.5, 1.5, -1.5, 1.5), 1000, 1000, {"prefix_len": 3}),
    ("nearcusp", 9, (-0.7, 0.4, -1.2, 0.3), 300, 200, {"prefix_len": 7}),
    ("gasket", 14, (0.1, 0.35, -0.2, 0.05), 4096, 4096, {}),
]


@pytest.mark.parametrize("name,d,window,W,H,fields", CASES)
def test_cull_fp64_equals_per_word_and_oracle(kl, name, d, window, W, H, fields):
    c, w = culled_and_per_word(kl, GROUPS[name], d, window, W, H, kl.FP64, **dict(fields))
    assert_same(c, w, oracle.word_count(d))
    g, s = oracle.group(GROUPS[name].ta, GROUPS[name].tb)
    sx = max(W / (window[1] - window[0]), H / (window[3] - window[2]))
    ref = oracle.render(g, s, d, window, W, H, eta=TOL64 * sx, edge_cap=1 << 22)
    check_fp64_image(c[0], ref, TOL64 * sx)


@pytest.mark.parametrize("name,d,window,W,H,fields", CASES)
def test_cull_mixed_equals_per_word_and_oracle(kl, name, d, window, W, H, fields):
    c, w = culled_and_per_word(kl, GROUPS[name], d, window, W, H, kl.MIXED, **dict(fields))
    assert_same(c, w, oracle.word_count(d))
    g, s = oracle.group(GROUPS[name].ta, GROUPS[name].tb)
    zmax = max(1.0, max(abs(complex(x, y)) for x in window[:2] for y in window[2:]))
    sx = max(W / (window[1] - window[0]), H / (window[3] - window[2]))
    tol = TOL32 * zmax * sx
    ref = oracle.render(g, s, d, window, W, H, eta=tol, edge_cap=1 << 22)
    check_fp64_image(c[0], ref, tol, max_edge_frac=4.0 * tol + 1e-2)
    assert iou(c[0], ref.image) >= 0.999


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cull_degenerate(kl, prec):
    """Short words (suffixes of one letter: blocks of one point), a window
    away from the limit set (every block outside), one-pixel images."""
    P = kl.FP64 if prec == "fp64" else kl.MIXED
    g = GROUPS["nearcusp"]
    for d, W, H, window in [(1, 16, 16, (-8.0, 8.0, -8.0, 8.0)), (2, 1, 1, (-2.0, 2.0, -2.0, 2.0)),
                            (3, 3, 7, (-2.0, 2.0, -2.0, 2.0)),
                            (7, 64, 64, (10.0, 11.0, 10.0, 11.0)),
                            (12, 1, 1, (-2.0, 2.0, -2.0, 2.0))]:
        c, w = culled_and_per_word(kl, g, d, window, W, H, P)
        assert_same(c, w, oracle.word_count(d))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cull_full_size_gasket(kl, prec):
    """Gasket, length 18 (516,560,652 words), 4096^2: culled = per-word."""
    c = klsynth.C2
    P = kl.FP64 if prec == "fp64" else kl.MIXED
    a, b = culled_and_per_word(kl, c.group, c.depth, c.window, c.width, c.height, P)
    assert_same(a, b, c.n_words)


def test_cull_full_size_near_cusp(kl):
    """Near-cusp group, length 20 (4.65e9 words), 8192^2, mixed: culled =
    per-word."""
    c = klsynth.C3
    a, b = culled_and_per_word(kl, c.group, c.depth, c.window, c.width, c.height, kl.MIXED)
    assert_same(a, b, c.n_words)


def test_cull_fp64_fallback_blocks(kl):
    """Gasket length 18 on the per-word render's own split (10 prefix
    letters), where near-parabolic prefixes send 3.2e6 words to the FP64 path:
    their blocks are culled by the FP64 test inside the mixed render."""
    c = klsynth.C2
    a, b = culled_and_per_word(kl, c.group, c.depth, c.window, c.width, c.height, kl.MIXED,
                               prefix_len=10)
    assert_same(a, b, c.n_words)
    assert int(a[1][2]) > 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cull_tiling_and_accumulate(kl, prec):
    """Tiling mode (every length 1..d; lengths above 9 culled) against the
    oracle, and accumulation: two culled renders add up to twice one."""
    import torch
    P = kl.FP64 if prec == "fp64" else kl.MIXED
    grp, d, W, window = GROUPS["gasket"], 12, 1024, (-1.5, 1.5, -1.5, 1.5)
    p = kl.params_init(grp.ta, grp.tb, d, W, W, window, P, cull=1, mode=kl.TILING)
    img, cnt = kl.render(p)
    g, s = oracle.group(grp.ta, grp.tb)
    sx = W / 3.0
    tol = (TOL64 if prec == "fp64" else TOL32 * 2.2) * sx
    ref = oracle.render_tiling(g, s, d, window, W, W, eta=tol, edge_cap=1 << 22)
    cnt = cnt.cpu().numpy()
    assert int(cnt[0]) + int(cnt[1]) == 2 * (3 ** d - 1)
    check_fp64_image(as_u32(img), ref, tol, max_edge_frac=4.0 * tol + 1e-2)
    q = kl.params_init(grp.ta, grp.tb, 13, W, W, window, P, cull=1)
    one, c1 = kl.render(q)
    one = one.clone()
    q.accumulate = 1
    two, c2 = kl.render(q, one.clone(), c1.clone())
    assert torch.equal(two, 2 * one)
    assert torch.equal(c2[:3], 2 * c1[:3])


def test_cull_rejections(kl):
    g = GROUPS["gasket"]
    p = kl.params_init(g.ta, g.tb, 12, 64, 64, (-1.5, 1.5, -1.5, 1.5), kl.MIXED, cull=2)
    with pytest.raises(RuntimeError):
        kl.render(p)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cull_through_noalloc(kl, prec):
    """The culled render through kl_render_noalloc (the library's static
    scratch array) gives the culled image of kl_render."""
    import torch
    P = kl.FP64 if prec == "fp64" else kl.MIXED
    g = GROUPS["gasket"]
    p = kl.params_init(g.ta, g.tb, 16, 2048, 2048, (-1.5, 1.5, -1.5, 1.5), P, cull=1)
    assert kl.workspace_bytes(p) <= kl.KL_STATIC_SCRATCH_BYTES
    a, ca = kl.render(p)
    b = torch.empty_like(a)
    cb = torch.zeros_like(ca)
    kl.render_noalloc(p, b, cb)
    assert torch.equal(a, b) and torch.equal(ca[:3], cb[:3])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("bt", [64, 128, 256])
def test_culled_batch_equals_culled_single_renders(kl, prec, bt):
    """A culled batch (one persistent launch over groups of uneven depth)
    gives each group's culled single render, image and counts, eagerly and
    from a captured graph."""
    import torch
    P = kl.FP64 if prec == "fp64" else kl.MIXED
    drawn = klsynth.draw_groups(klsynth.BATCH_SEED, 7)
    groups = [g for g, _ in drawn] + [GROUPS["gasket"], GROUPS["nearcusp"]]
    depths = [8, 14, 9, 12, 2, 11, 10, 15, 13]
    ps = [kl.params_init(g.ta, g.tb, d, 384, 384, (-1.5, 1.5, -1.5, 1.5), P, cull=1,
                         block_threads=bt) for g, d in zip(groups, depths)]
    b = kl.Batch(ps)
    imgs, cnts = b.render()
    eager_imgs, eager_cnts = imgs.clone(), cnts.clone()
    for k, p in enumerate(ps):
        img, cnt = kl.render(p)
        assert torch.equal(imgs[k], img), k
        assert torch.equal(cnts[k][:3], cnt[:3]), (k, cnts[k], cnt)
        assert int(cnt[0]) + int(cnt[1]) == oracle.word_count(depths[k])
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.images, eager_imgs)
    assert torch.equal(b.counters[:, :3], eager_cnts[:, :3])
