"""Parity at full size, in the launch configuration the benchmark times.

  - gasket, length 18 (516,560,652 words), 4096^2 over [-1.5, 1.5]^2;
  - near-cusp group ta = tb = 1.91 + 0.05i, length 20 (4,649,045,868 words),
    8192^2 over [-2, 2]^2.
Full oracle renders (tree walk on all host cores) against both GPU paths, and
word values on the seeded 1e6-index sample against the oracle's per-word
definition.
"""
import numpy as np
import pytest

import klsynth
import oracle
from imagecheck import check_band_image, check_fp64_image, iou

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


def sample_errors(kl, cfg, precision):
    idx = klsynth.index_sample(klsynth.SAMPLE_SEED, 1_000_000, cfg.depth)
    p = kl.params_init(cfg.group.ta, cfg.group.tb, cfg.depth, cfg.width, cfg.height,
                       cfg.window, precision)
    uv = kl.eval_words(p, dev_index(idx)).cpu().numpy()
    g, s = oracle.group(cfg.group.ta, cfg.group.tb)
    z = oracle.evaluate(g, s, cfg.depth, idx)
    x0, x1, y0, y1 = cfg.window
    sx, sy = cfg.width / (x1 - x0), cfg.height / (y1 - y0)
    zg = (x0 + uv[:, 0] / sx) + 1j * (y1 - uv[:, 1] / sy)
    fin = np.isfinite(z) & (np.abs(z) < 1e12)
    err = np.abs(zg[fin] - z[fin]) / np.maximum(1.0, np.abs(z[fin]))
    return float(err.max()), float(np.abs(zg[fin] - z[fin]).max())


@pytest.fixture(scope="module")
def c2_oracle():
    cfg = klsynth.C2
    g, s = oracle.group(cfg.group.ta, cfg.group.tb)
    sx = cfg.width / (cfg.window[1] - cfg.window[0])
    return oracle.render(g, s, cfg.depth, cfg.window, cfg.width, cfg.height,
                         eta=TOL64 * sx, edge_cap=1 << 22)


def test_gasket_d18_fp64_image(kl, c2_oracle):
    cfg = klsynth.C2
    p = kl.params_init(cfg.group.ta, cfg.group.tb, cfg.depth, cfg.width, cfg.height,
                       cfg.window, kl.FP64)
    img, cnt = kl.render(p)
    got = img.cpu().numpy().view(np.uint32)
    extra = check_fp64_image(got, c2_oracle, TOL64 * cfg.width / 3.0, max_edge_frac=1e-4)
    c = cnt.cpu().numpy()
    assert int(c[0]) + int(c[1]) == cfg.n_words and int(c[0]) == c2_oracle.in_window
    print(f"\ngasket d18 fp64: edge words {c2_oracle.edge_total}, moved {extra}")


def test_gasket_d18_mixed_image(kl, c2_oracle):
    cfg = klsynth.C2
    p = kl.params_init(cfg.group.ta, cfg.group.tb, cfg.depth, cfg.width, cfg.height,
                       cfg.window, kl.MIXED)
    img, cnt = kl.render(p)
    got = img.cpu().numpy().view(np.uint32)
    v = iou(got, c2_oracle.image)
    c = cnt.cpu().numpy()
    assert int(c[0]) + int(c[1]) == cfg.n_words
    assert v >= 0.999
    diff = np.abs(got.astype(np.int64) - c2_oracle.image.astype(np.int64)).sum()
    print(f"\ngasket d18 mixed: IoU {v:.6f}, L1 hit difference {diff} of {cfg.n_words}, "
          f"fp64 words {int(c[2])}")


def test_gasket_d18_mixed_image_band(kl):
    """The mixed image pixel by pixel at the mixed tolerance: every word whose
    value lies farther than 2e-5 max(1, |z|) from a pixel edge lands in the
    oracle's pixel (the gasket's limit set has |z| <= 1.4, so the band is
    2e-5 x 1.4 in z, 0.038 px), and every other word in one of its candidate
    pixels.  The split is the one the benchmark times (prefix 10, suffix 8)."""
    cfg = klsynth.C2
    g, s = oracle.group(cfg.group.ta, cfg.group.tb)
    sx = cfg.width / (cfg.window[1] - cfg.window[0])
    eta = TOL32 * 1.4 * sx
    ref = oracle.render(g, s, cfg.depth, cfg.window, cfg.width, cfg.height, eta=eta,
                        edge_cap=1 << 27)
    p = kl.params_init(cfg.group.ta, cfg.group.tb, cfg.depth, cfg.width, cfg.height,
                       cfg.window, kl.MIXED)
    img, cnt = kl.render(p)
    got = img.cpu().numpy().view(np.uint32)
    extra = check_band_image(got, ref, eta)
    c = cnt.cpu().numpy()
    assert int(c[0]) + int(c[1]) == cfg.n_words
    print(f"\ngasket d18 mixed, band {eta:.4f} px: edge words {ref.edge_total}, "
          f"their hits in the image {extra}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cfg", [klsynth.C2, klsynth.C3], ids=["gasket-d18", "nearcusp-d20"])
def test_sample_1e6_value_errors(kl, cfg, prec):
    rel, absmax = sample_errors(kl, cfg, kl.FP64 if prec == "fp64" else kl.MIXED)
    print(f"\n{cfg.name} {prec}: max rel |dz| {rel:.3e}, max |dz| {absmax:.3e} on 1e6 words")
    assert rel <= (TOL64 if prec == "fp64" else TOL32)


def test_nearcusp_d20_images(kl):
    cfg = klsynth.C3
    g, s = oracle.group(cfg.group.ta, cfg.group.tb)
    sx = cfg.width / (cfg.window[1] - cfg.window[0])
    ref = oracle.render(g, s, cfg.depth, cfg.window, cfg.width, cfg.height,
                        eta=TOL64 * sx, edge_cap=1 << 22)
    for prec in ("mixed", "fp64"):
        p = kl.params_init(cfg.group.ta, cfg.group.tb, cfg.depth, cfg.width, cfg.height,
                           cfg.window, kl.MIXED if prec == "mixed" else kl.FP64)
        img, cnt = kl.render(p)
        got = img.cpu().numpy().view(np.uint32)
        c = cnt.cpu().numpy()
        assert int(c[0]) + int(c[1]) == cfg.n_words
        if prec == "fp64":
            extra = check_fp64_image(got, ref, TOL64 * sx, max_edge_frac=1e-4)
            assert int(c[0]) == ref.in_window
            print(f"\nnear-cusp d20 fp64: edge words {ref.edge_total}, moved {extra}")
        else:
            v = iou(got, ref.image)
            print(f"\nnear-cusp d20 mixed: IoU {v:.6f}, in-window {int(c[0])} "
                  f"(oracle {ref.in_window}), fp64 words {int(c[2])}")
            assert v >= 0.999
        del img, got
