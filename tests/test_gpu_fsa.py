"""General presentations: the paper's scan of the unpruned m-ary tree with an
indexed Cayley table (kl_render_fsa) against the oracle's scan render.
FP64 images exact up to edge words; kept words = the count of the table run;
with the once-punctured-torus table the scan keeps exactly the reduced words,
so its image equals the reduced-index render's."""
import numpy as np
import pytest

import klsynth
import oracle
from conftest import golden_table
from imagecheck import check_fp64_image

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
KLEIN = [[[1j, 0], [0, -1j]], [[0, 1j], [1j, 0]], [[0, -1], [1, 0]]]


@pytest.fixture(scope="module")
def kl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


def run(kl, table, gens, seeds, d, window, W, H):
    m = len(gens)
    f = kl.fsa(table, gens, seeds)
    p = kl.params_init(2 + 0j, 2 + 0j, d, W, H, window, kl.FP64)
    img, cnt = kl.render_fsa(f, p)
    img = img.cpu().numpy().view(np.uint32)
    cnt = cnt.cpu().numpy()
    sx = max(W / (window[1] - window[0]), H / (window[3] - window[2]))
    zmax = max(1.0, max(abs(complex(x, y)) for x in window[:2] for y in window[2:]))
    ref = oracle.render_fsa(m, table, gens, seeds, d, window, W, H, eta=TOL64 * zmax * sx,
                            edge_cap=1 << 22)
    kept = kl.fsa_count(f, d)
    assert int(cnt[0]) + int(cnt[1]) == kept == int(cnt[2])
    assert int(cnt[0]) == int(img.astype(np.int64).sum())
    check_fp64_image(img, ref, TOL64 * zmax * sx, max_edge_frac=1e-2)
    return img, cnt


@pytest.mark.parametrize("d", [1, 2, 7, 13])
def test_klein_four_group(kl, d):
    k4 = golden_table("klein4_indexed_cayley.txt")
    seeds = [0.31 + 0.17j, -0.43 + 0.29j, 0.12 - 0.61j]
    run(kl, k4, KLEIN, seeds, d, (-4.1, 3.9, -3.7, 4.3), 257, 199)


@pytest.mark.parametrize("group,d,W", [(klsynth.GASKET, 9, 512), (klsynth.NEAR_CUSP, 11, 768),
                                       (klsynth.draw_groups(klsynth.BATCH_SEED, 2)[1][0], 12,
                                        640)])
def test_torus_table_equals_the_reduced_index_render(kl, group, d, W):
    t11 = golden_table("t11_indexed_cayley.txt")
    g, s = oracle.group(group.ta, group.tb)
    gens = [m.tolist() for m in oracle.as_matrices(g)]
    window = (-2.0, 2.0, -2.0, 2.0)
    img, cnt = run(kl, t11, gens, oracle.as_points(s), d, window, W, W)
    assert int(cnt[2]) == oracle.word_count(d)
    # the reduced-index render of the same group: the same words; both are
    # exact up to edge words against their oracles, so they agree up to them
    p = kl.params_init(group.ta, group.tb, d, W, W, window, kl.FP64)
    img2, cnt2 = kl.render(p)
    img2 = img2.cpu().numpy().view(np.uint32).astype(np.int64)
    diff = np.abs(img.astype(np.int64) - img2).sum()
    assert diff <= 2 * 1e-3 * oracle.word_count(d) + 10, diff
    assert int(cnt2[0].item()) + int(cnt2[1].item()) == int(cnt[0]) + int(cnt[1])


def test_accumulate_and_single_letter(kl):
    """m = 1 with a table that lets the letter repeat: one string per depth."""
    f = kl.fsa([[0, 1], [0, 1]], [[[1, 0.5], [0, 1]]], [0.25 + 0.1j])
    p = kl.params_init(2 + 0j, 2 + 0j, 6, 64, 64, (-1.0, 7.0, -4.0, 4.0), kl.FP64)
    img, cnt = kl.render_fsa(f, p)
    # z -> z + 1/2 applied six times to 0.25 + 0.1i
    z = 0.25 + 0.1j + 3.0
    col = int(np.floor((z.real + 1.0) * 8)), int(np.floor((4.0 - z.imag) * 8))
    a = img.cpu().numpy()
    assert a[col[1], col[0]] == 1 and a.sum() == 1
    p.accumulate = 1
    kl.render_fsa(f, p, img, cnt)
    assert img.cpu().numpy()[col[1], col[0]] == 2 and int(cnt[2].item()) == 2
