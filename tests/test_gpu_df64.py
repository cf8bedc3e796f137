"""The double-float path (KL_DF64) against the FP64 oracle, held to the FP64
gates: word values within 1e-9 max(1, |z|) and images exact up to edge words
(the oracle logs every word within 1e-9 in z of a pixel edge; tests/imagecheck.py).

The per-word map runs in double-float arithmetic (hi + lo pairs of floats,
about 48 significant bits) on the FP32 pipe; prefixes whose pole form is
invalid or out of float range take the FP64 path, as in the mixed render.
"""
import numpy as np
import pytest

import klsynth
import oracle
from imagecheck import check_fp64_image

pytestmark = pytest.mark.gpu

TOL64 = 1e-9

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


def dev_index(idx):
    import torch
    return torch.from_numpy(np.ascontiguousarray(idx, dtype=np.uint64).view(np.int64)).cuda()


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


CASES = [("gasket", 10, None), ("gasket", 18, None), ("nearcusp", 20, None),
         ("nearcusp", 13, 4), ("fuchsian", 12, None), ("batch0", 15, None), ("batch7", 17, 11),
         ("gasket", 2, None), ("nearcusp", 1, None)]


@pytest.mark.parametrize("name,d,plen", CASES)
def test_eval_df64(kl, name, d, plen):
    group = GROUPS[name]
    n = oracle.word_count(d)
    idx = (np.arange(n, dtype=np.uint64) if n <= 100_000 else
           klsynth.index_sample(klsynth.SAMPLE_SEED, 100_000, d))
    window, W, H = (-2.0, 2.0, -2.0, 2.0), 1024, 1024
    fields = {"prefix_len": plen} if plen else {}
    p = kl.params_init(group.ta, group.tb, d, W, H, window, kl.DF64, **fields)
    uv = kl.eval_words(p, dev_index(idx)).cpu().numpy()
    g, s = oracle.group(group.ta, group.tb)
    z = oracle.evaluate(g, s, d, idx)
    sx = W / (window[1] - window[0])
    fin = np.isfinite(z) & (np.abs(z) < 1e12)
    assert np.isfinite(uv[fin]).all()
    zg = (window[0] + uv[:, 0] / sx) + 1j * (window[3] - uv[:, 1] / sx)
    err = np.abs(zg[fin] - z[fin]) / np.maximum(1.0, np.abs(z[fin]))
    print(f"\n{name} d={d}: max rel |dz| {err.max():.3e}")
    assert err.max() <= TOL64


IMAGE_CASES = [
    ("gasket", 10, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, {}),
    ("gasket", 13, (-1.5, 1.5, -1.5, 1.5), 2048, 2048, {}),
    ("nearcusp", 12, (-2.0, 2.0, -2.0, 2.0), 1536, 1024, {}),
    ("batch0", 12, (-1.5, 1.5, -1.5, 1.5), 1024, 1024, {}),
    ("fuchsian", 11, (-1.1, 1.1, -1.1, 1.1), 777, 513, {}),
    ("batch7", 11, (-1.5, 1.5, -1.5, 1.5), 1000, 1000, {"prefix_len": 3}),
    ("nearcusp", 9, (-0.7, 0.4, -1.2, 0.3), 300, 200, {"prefix_len": 7}),
    ("nearcusp", 1, (-8.0, 8.0, -8.0, 8.0), 16, 16, {}),
    ("nearcusp", 7, (10.0, 11.0, 10.0, 11.0), 64, 64, {}),
]


@pytest.mark.parametrize("name,d,window,W,H,fields", IMAGE_CASES)
def test_render_df64_image(kl, name, d, window, W, H, fields):
    group = GROUPS[name]
    p = kl.params_init(group.ta, group.tb, d, W, H, window, kl.DF64, **fields)
    img, cnt = kl.render(p)
    g, s = oracle.group(group.ta, group.tb)
    sx = max(W / (window[1] - window[0]), H / (window[3] - window[2]))
    ref = oracle.render(g, s, d, window, W, H, eta=TOL64 * sx, edge_cap=1 << 22)
    cnt = cnt.cpu().numpy()
    img = as_u32(img)
    assert int(cnt[0]) + int(cnt[1]) == oracle.word_count(d)
    check_fp64_image(img, ref, TOL64 * sx)
    assert int(cnt[0]) == int(img.astype(np.int64).sum())


@pytest.mark.parametrize("cfg", [klsynth.C2, klsynth.C3], ids=["gasket-d18", "nearcusp-d20"])
def test_full_size_df64_image(kl, cfg):
    """The benchmark's workloads at full size: the double-float image is the
    oracle's up to edge words, as the FP64 render's is."""
    g, s = oracle.group(cfg.group.ta, cfg.group.tb)
    sx = cfg.width / (cfg.window[1] - cfg.window[0])
    ref = oracle.render(g, s, cfg.depth, cfg.window, cfg.width, cfg.height,
                        eta=TOL64 * sx, edge_cap=1 << 22)
    p = kl.params_init(cfg.group.ta, cfg.group.tb, cfg.depth, cfg.width, cfg.height,
                       cfg.window, kl.DF64)
    img, cnt = kl.render(p)
    got = as_u32(img)
    c = cnt.cpu().numpy()
    assert int(c[0]) + int(c[1]) == cfg.n_words
    extra = check_fp64_image(got, ref, TOL64 * sx, max_edge_frac=1e-4)
    print(f"\n{cfg.name} df64: edge words {ref.edge_total}, their hits {extra}, "
          f"fp64 fallback words {int(c[2])}")


def test_df64_tiling_and_shards(kl):
    """Tiling mode (every length 1..d) and a 3-way shard split in double-float."""
    import torch
    group, d, W, window = GROUPS["batch0"], 11, 512, (-1.5, 1.5, -1.5, 1.5)
    p = kl.params_init(group.ta, group.tb, d, W, W, window, kl.DF64, mode=kl.TILING)
    img, cnt = kl.render(p)
    g, s = oracle.group(group.ta, group.tb)
    sx = W / (window[1] - window[0])
    ref = oracle.render_tiling(g, s, d, window, W, W, eta=TOL64 * sx, edge_cap=1 << 20)
    check_fp64_image(as_u32(img), ref, TOL64 * sx)
    q = kl.params_init(group.ta, group.tb, 13, W, W, window, kl.DF64)
    whole, wcnt = kl.render(q)
    acc = torch.zeros_like(whole)
    ccount = torch.zeros_like(wcnt)
    for k in range(3):
        q.shard_index, q.shard_count = k, 3
        part, pc = kl.render(q)
        acc += part
        ccount += pc
    assert torch.equal(acc, whole) and torch.equal(ccount[:3], wcnt[:3])


def test_df64_is_refused_where_unsupported(kl):
    g = GROUPS["gasket"]
    p = kl.params_init(g.ta, g.tb, 12, 256, 256, (-1.5, 1.5, -1.5, 1.5), kl.DF64, cull=1)
    with pytest.raises(kl.KlError) as e:
        kl.render(p)
    assert e.value.status == 1
    p.cull = 0
    with pytest.raises(kl.KlError) as e:
        kl.Batch([p])
    assert e.value.status == 1
