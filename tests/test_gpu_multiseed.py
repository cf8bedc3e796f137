"""Multi-seed feeding (the paper's loop over a list of fixed points): every
reduced word drawn once per seed point of kl_cusp_seeds, against the
oracle's multi-seed render of the oracle's own seed list.  FP64 exact up to
edge words; mixed exact for words farther than the mixed tolerance from a
pixel edge; every word counted once per point."""
import numpy as np
import pytest

import klsynth
import oracle
from imagecheck import check_fp64_image

pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("group,d,W,window", [
    (klsynth.GASKET, 10, 1024, (-1.5, 1.5, -1.5, 1.5)),
    (klsynth.NEAR_CUSP, 11, 768, (-2.0, 2.0, -2.0, 2.0)),
])
def test_multiseed_render(kl, prec, group, d, W, window):
    p = kl.params_init(group.ta, group.tb, d, W, W, window,
                       kl.FP64 if prec == "fp64" else kl.MIXED)
    s16 = kl.cusp_seeds(np.array(list(p.gens)))
    points = [complex(s16[2 * i], s16[2 * i + 1]) for i in range(8)]
    img, cnt = kl.render_multiseed(p, points)
    img = img.cpu().numpy().view(np.uint32)
    cnt = cnt.cpu().numpy()
    assert int(cnt[0]) + int(cnt[1]) == 8 * oracle.word_count(d)
    assert int(cnt[0]) == int(img.astype(np.int64).sum())
    g, _ = oracle.group(group.ta, group.tb)
    o16 = oracle.cusp_seeds(g)
    opts = [complex(o16[2 * i], o16[2 * i + 1]) for i in range(8)]
    sx = max(W / (window[1] - window[0]), W / (window[3] - window[2]))
    zmax = max(1.0, max(abs(complex(x, y)) for x in window[:2] for y in window[2:]))
    tol = TOL[prec] * zmax * sx
    ref = oracle.render_multiseed(g, opts, d, window, W, W, eta=tol, edge_cap=1 << 22)
    check_fp64_image(img, ref, tol, max_edge_frac=4.0 * tol + 1e-2)


@pytest.mark.parametrize("group,d,W,window", [
    (klsynth.GASKET, 10, 1024, (-1.5, 1.5, -1.5, 1.5)),
    (klsynth.NEAR_CUSP, 11, 768, (-2.0, 2.0, -2.0, 2.0)),
])
def test_repetend_render(kl, group, d, W, window):
    """The repetend points (render_repetends: every word at the four
    commutator fixed points) against the oracle's multi-seed render of its
    own four points, FP64, exact up to edge words."""
    p = kl.params_init(group.ta, group.tb, d, W, W, window, kl.FP64)
    img, cnt = kl.render_repetends(p)
    img = img.cpu().numpy().view(np.uint32)
    cnt = cnt.cpu().numpy()
    assert int(cnt[0]) + int(cnt[1]) == 4 * oracle.word_count(d)
    g, _ = oracle.group(group.ta, group.tb)
    o16 = oracle.cusp_seeds(g)
    opts = [complex(o16[2 * i], o16[2 * i + 1]) for i in range(4, 8)]
    sx = W / (window[1] - window[0])
    zmax = max(1.0, max(abs(complex(x, y)) for x in window[:2] for y in window[2:]))
    tol = TOL["fp64"] * zmax * sx
    ref = oracle.render_multiseed(g, opts, d, window, W, W, eta=tol, edge_cap=1 << 22)
    check_fp64_image(img, ref, tol, max_edge_frac=1e-2)


def test_repetends_catch_cusp_detail(kl):
    """What the repetends gain: at length 11 the near-cusp group's render
    misses pixels that a length-16 render reaches (the slow orbits near the
    cusps); adding the repetend points of the same length-11 words covers
    more of the deep render, and most pixels they add lie on it (within one
    pixel; measured 96.5%).  The rest are true limit points next to the cusps
    that even the length-16 render has not reached: there the orbits close in
    like 1/n, which is why the repetends are drawn at all.""" 
    import torch
    g = klsynth.NEAR_CUSP
    W, window = 1024, (-2.0, 2.0, -2.0, 2.0)
    deep = kl.render(kl.params_init(g.ta, g.tb, 16, W, W, window, kl.FP64))[0] != 0
    p = kl.params_init(g.ta, g.tb, 11, W, W, window, kl.FP64)
    base = kl.render(p)[0] != 0
    rep = kl.render_repetends(p)[0] != 0
    both = base | rep
    near = torch.nn.functional.max_pool2d(deep[None, None].float(), 3, stride=1,
                                          padding=1)[0, 0] > 0
    recall_base = float((base & deep).sum()) / float(deep.sum())
    recall_both = float((both & deep).sum()) / float(deep.sum())
    added = rep & ~base
    on_deep = float((added & near).sum()) / max(1.0, float(added.sum()))
    print(f"\nrecall of the length-16 render: length 11 {recall_base:.4f}, with repetends "
          f"{recall_both:.4f}; added pixels {int(added.sum())}, on it {on_deep:.4f}")
    assert recall_both > recall_base + 0.01
    assert on_deep > 0.9


@pytest.mark.parametrize("prec", ["FP64", "MIXED", "DF64"])
@pytest.mark.parametrize("mode", ["LIMIT_SET", "TILING"])
def test_multiseed_equals_single_seed_renders(kl, prec, mode):
    """kl_render_multiseed builds the prefix tables once for all points: its
    image and counters are those of one kl_render per point (all four seeds
    set to the point), summed, bit for bit."""
    import torch
    g = klsynth.NEAR_CUSP
    p = kl.params_init(g.ta, g.tb, 13, 512, 384, (-2.0, 2.0, -1.5, 1.5), getattr(kl, prec),
                       mode=getattr(kl, mode))
    s16 = kl.cusp_seeds(list(p.gens))
    points = [complex(s16[2 * i], s16[2 * i + 1]) for i in range(8)]
    img, cnt = kl.render_multiseed(p, points)
    acc = torch.zeros_like(img)
    acc_c = torch.zeros_like(cnt)
    q = kl.Params.from_buffer_copy(p)
    for z in points:
        for x in range(4):
            q.seeds[2 * x], q.seeds[2 * x + 1] = z.real, z.imag
        one, c1 = kl.render(q)
        acc += one
        acc_c += c1
    assert torch.equal(img, acc)
    assert torch.equal(cnt[:3], acc_c[:3])


def test_multiseed_refuses_bad_points(kl):
    g = klsynth.GASKET
    p = kl.params_init(g.ta, g.tb, 8, 64, 64, (-1.5, 1.5, -1.5, 1.5), kl.MIXED)
    for pts in ([], [complex(float("nan"), 0.0)], [0.1 + 0.2j, complex(0.0, float("inf"))]):
        with pytest.raises(kl.KlError) as e:
            kl.render_multiseed(p, pts)
        assert e.value.status == 1
