"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Tolerances (from the arithmetic and the required accuracy):
  - decode: bit-exact letters;
  - FP64 word values: |dz| <= 1e-9 max(1, |z|);
  - mixed word values: |dz| <= 2e-5 max(1, |z|);
  - FP64 images: exact for every word not within 1e-9 (in z) of a pixel edge,
    edge words only between their candidate pixels (tests/imagecheck.py);
  - mixed images: exact for every word farther than the mixed tolerance from
    a pixel edge (edge words among their candidate pixels), occupancy IoU >=
    0.999, hits + drops = N_d exactly.
"""
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


def dev_index(idx):
    import torch
    return torch.from_numpy(np.ascontiguousarray(idx, dtype=np.uint64).view(np.int64)).cuda()


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


# ---------------------------------------------------------------------------
# decode

@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 12])
def test_decode_all_indices(kl, d):
    n = oracle.word_count(d)
    idx = np.arange(n, dtype=np.uint64)
    got = kl.decode_words(d, dev_index(idx)).cpu().numpy()
    assert np.array_equal(got, oracle.decode(d, idx))


@pytest.mark.parametrize("d", [18, 20, 22, 31, 40])
def test_decode_sampled_and_out_of_range(kl, d):
    n = oracle.word_count(d)
    idx = np.concatenate([klsynth.index_sample(klsynth.SAMPLE_SEED, 200_000, d),
                          np.array([0, n - 1, n, n + 7, 2 ** 64 - 1], dtype=np.uint64)])
    got = kl.decode_words(d, dev_index(idx)).cpu().numpy()
    assert np.array_equal(got, oracle.decode(d, idx, strict=False))
    assert (got[-3:] == 0xFF).all()


# ---------------------------------------------------------------------------
# word values

GROUPS = {
    "gasket": klsynth.GASKET,
    "nearcusp": klsynth.NEAR_CUSP,
    "fuchsian": klsynth.FUCHSIAN,
    "batch0": klsynth.draw_groups(klsynth.BATCH_SEED, 1)[0][0],
    "batch7": klsynth.draw_groups(klsynth.BATCH_SEED, 8)[7][0],
}


def oracle_uv(g, s, d, idx, window, W, H):
    z = oracle.evaluate(g, s, d, idx)
    x0, x1, y0, y1 = window
    return z, (z.real - x0) * (W / (x1 - x0)), (y1 - z.imag) * (H / (y1 - y0))


def compare_values(kl, group, d, idx, window, W, H, precision, tol, **fields):
    p = kl.params_init(group.ta, group.tb, d, W, H, window, precision, **fields)
    uv = kl.eval_words(p, dev_index(idx)).cpu().numpy()
    g, s = oracle.group(group.ta, group.tb)
    z, u, v = oracle_uv(g, s, d, idx, window, W, H)
    sx, sy = W / (window[1] - window[0]), H / (window[3] - window[2])
    fin = np.isfinite(z) & (np.abs(z) < 1e12)
    assert np.isfinite(uv[fin]).all()
    zg = (window[0] + uv[:, 0] / sx) + 1j * (window[3] - uv[:, 1] / sy)
    err = np.abs(zg[fin] - z[fin]) / np.maximum(1.0, np.abs(z[fin]))
    # compare in pixel units too (what decides the pixel)
    du = np.abs(uv[fin, 0] - u[fin]) / sx / np.maximum(1.0, np.abs(z[fin]))
    dv = np.abs(uv[fin, 1] - v[fin]) / sy / np.maximum(1.0, np.abs(z[fin]))
    worst = max(err.max(), du.max(), dv.max())
    assert worst <= tol, worst
    return worst


CASES = [("gasket", 10, None), ("gasket", 18, None), ("nearcusp", 20, None),
         ("nearcusp", 13, 4), ("fuchsian", 12, None), ("batch0", 15, None), ("batch7", 17, 11),
         ("gasket", 2, None), ("nearcusp", 1, None)]


@pytest.mark.parametrize("name,d,plen", CASES)
def test_eval_fp64(kl, name, d, plen):
    n = oracle.word_count(d)
    idx = (np.arange(n, dtype=np.uint64) if n <= 100_000 else
           klsynth.index_sample(klsynth.SAMPLE_SEED, 100_000, d))
    fields = {"prefix_len": plen} if plen else {}
    compare_values(kl, GROUPS[name], d, idx, (-2.0, 2.0, -2.0, 2.0), 1024, 1024,
                   kl.FP64, TOL64, **fields)


@pytest.mark.parametrize("name,d,plen", CASES)
def test_eval_mixed(kl, name, d, plen):
    n = oracle.word_count(d)
    idx = (np.arange(n, dtype=np.uint64) if n <= 100_000 else
           klsynth.index_sample(klsynth.SAMPLE_SEED, 100_000, d))
    fields = {"prefix_len": plen} if plen else {}
    compare_values(kl, GROUPS[name], d, idx, (-2.0, 2.0, -2.0, 2.0), 1024, 1024,
                   kl.MIXED, TOL32, **fields)


def test_eval_rejects_out_of_range_index(kl):
    g = GROUPS["gasket"]
    p = kl.params_init(g.ta, g.tb, 6, 64, 64, (-2.0, 2.0, -2.0, 2.0))
    uv = kl.eval_words(p, dev_index([0, oracle.word_count(6), 5])).cpu().numpy()
    assert np.isfinite(uv[0]).all() and np.isnan(uv[1]).all() and np.isfinite(uv[2]).all()


# ---------------------------------------------------------------------------
# images

def render_both(kl, group, d, window, W, H, precision, eta_z=TOL64, **fields):
    p = kl.params_init(group.ta, group.tb, d, W, H, window, precision, **fields)
    img, cnt = kl.render(p)
    g, s = oracle.group(group.ta, group.tb)
    sx = max(W / (window[1] - window[0]), H / (window[3] - window[2]))
    ref = oracle.render(g, s, d, window, W, H, eta=eta_z * sx, edge_cap=1 << 22)
    cnt = cnt.cpu().numpy()
    assert int(cnt[0]) + int(cnt[1]) == oracle.word_count(d)
    return as_u32(img), cnt, ref


IMAGE_CASES = [
    ("gasket", 10, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, {}),
    ("gasket", 13, (-1.5, 1.5, -1.5, 1.5), 2048, 2048, {}),
    ("nearcusp", 12, (-2.0, 2.0, -2.0, 2.0), 1536, 1024, {}),
    ("batch0", 12, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, {}),
    ("fuchsian", 11, (-1.1, 1.1, -1.1, 1.1), 777, 513, {}),
    ("batch7", 11, (-1.5, 1.5, -1.5, 1.5), 1000, 1000, {"prefix_len": 3}),
    ("nearcusp", 9, (-0.7, 0.4, -1.2, 0.3), 300, 200, {"prefix_len": 7}),
]


@pytest.mark.parametrize("name,d,window,W,H,fields", IMAGE_CASES)
def test_render_fp64_image(kl, name, d, window, W, H, fields):
    img, cnt, ref = render_both(kl, GROUPS[name], d, window, W, H, kl.FP64, **fields)
    check_fp64_image(img, ref, TOL64 * max(W / (window[1] - window[0]),
                                           H / (window[3] - window[2])))
    assert int(cnt[0]) == int(img.astype(np.int64).sum())
    assert 0 < int(cnt[3]) <= int(cnt[0]) or int(cnt[0]) == 0


@pytest.mark.parametrize("name,d,window,W,H,fields", IMAGE_CASES)
def test_render_mixed_image(kl, name, d, window, W, H, fields):
    # every word farther than the mixed tolerance, 2e-5 max(1, |z|), from a
    # pixel edge must land in the oracle's pixel; the rest among their
    # candidate pixels
    zmax = max(1.0, max(abs(complex(x, y)) for x in window[:2] for y in window[2:]))
    img, cnt, ref = render_both(kl, GROUPS[name], d, window, W, H, kl.MIXED,
                                eta_z=TOL32 * zmax, **fields)
    sx = max(W / (window[1] - window[0]), H / (window[3] - window[2]))
    tol = TOL32 * zmax * sx
    check_fp64_image(img, ref, tol, max_edge_frac=4.0 * tol + 1e-2)
    assert iou(img, ref.image) >= 0.999
    assert int(cnt[0]) == int(img.astype(np.int64).sum())
    assert abs(int(cnt[0]) - ref.in_window) <= max(10, 1e-4 * ref.in_window)


def test_render_degenerate_sizes(kl):
    g = GROUPS["nearcusp"]
    for d, W, H, window in [(1, 16, 16, (-8.0, 8.0, -8.0, 8.0)), (2, 1, 1, (-2.0, 2.0, -2.0, 2.0)),
                            (3, 3, 7, (-2.0, 2.0, -2.0, 2.0)),
                            (7, 64, 64, (10.0, 11.0, 10.0, 11.0))]:
        for prec in (kl.FP64, kl.MIXED):
            img, cnt, ref = render_both(kl, g, d, window, W, H, prec)
            if prec == kl.FP64:
                check_fp64_image(img, ref, TOL64 * max(W / (window[1] - window[0]),
                                                       H / (window[3] - window[2])))
            else:
                assert iou(img, ref.image) >= 0.999 or ref.in_window == 0
    # a window away from the limit set drops every word
    assert int(cnt[0]) == 0 and int(cnt[1]) == oracle.word_count(7)


@pytest.mark.parametrize("prec,tol", [("MIXED", 2e-5), ("DF64", 1e-9)])
def test_render_at_the_maximum_depth(kl, prec, tol):
    """The deepest render a plan allows (length 24: 4 3^23 = 1.1e11 words,
    above 2^32): every word counted once in the 64-bit counters, the image
    holding every in-window word, and word values on a seeded sample against
    the oracle."""
    g, d, W, window = GROUPS["nearcusp"], 24, 1024, (-2.0, 2.0, -2.0, 2.0)
    p = kl.params_init(g.ta, g.tb, d, W, W, window, getattr(kl, prec))
    img, cnt = kl.render(p)
    c = cnt.cpu().numpy()
    n = oracle.word_count(d)
    assert n > 2 ** 32 and int(c[0]) + int(c[1]) == n
    assert int(as_u32(img).astype(np.uint64).sum()) == int(c[0])
    idx = klsynth.index_sample(klsynth.SAMPLE_SEED, 100_000, d)
    compare_values(kl, g, d, idx, window, W, W, getattr(kl, prec), tol)
    p.depth = d + 1
    with pytest.raises(kl.KlError):
        kl.render(p)


def test_render_accumulate_and_errors(kl):
    import torch
    g = GROUPS["gasket"]
    p = kl.params_init(g.ta, g.tb, 9, 512, 512, (-1.5, 1.5, -1.5, 1.5))
    img, cnt = kl.render(p)
    once = as_u32(img).astype(np.int64)
    p.accumulate = 1
    kl.render(p, img, cnt)
    assert np.array_equal(as_u32(img).astype(np.int64), 2 * once)
    assert int(cnt.cpu()[0]) + int(cnt.cpu()[1]) == 2 * oracle.word_count(9)
    p.accumulate = 0
    need = kl.workspace_bytes(p)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(kl.KlError) as e:
        kl.render(p, img, cnt, small)
    assert e.value.status == 4
    big = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(kl.KlError) as e:
        kl.render(p, img, cnt, big[1:])
    assert e.value.status == 1
    p.depth = 25
    with pytest.raises(kl.KlError) as e:
        kl.render(p, img, cnt, big)
    assert e.value.status in (1, 2)


@pytest.mark.parametrize("prec,mode", [("FP64", "LIMIT_SET"), ("MIXED", "LIMIT_SET"),
                                       ("DF64", "LIMIT_SET"), ("MIXED", "TILING")])
def test_render_replayed_from_a_graph(kl, prec, mode):
    """A kl_render captured in a CUDA graph and replayed gives the image and
    counters of the direct call, bit for bit, replay after replay."""
    import torch
    g = GROUPS["gasket"]
    p = kl.params_init(g.ta, g.tb, 12, 1024, 1024, (-1.5, 1.5, -1.5, 1.5), getattr(kl, prec),
                       mode=getattr(kl, mode))
    img, cnt = kl.render(p)
    r = kl.Renderer(p)
    r.capture()
    for _ in range(3):
        gi, gc = r.replay()
        torch.cuda.synchronize()
        assert torch.equal(gi, img) and torch.equal(gc[:3], cnt[:3])
