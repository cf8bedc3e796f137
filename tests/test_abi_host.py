"""The C-ABI library without a GPU: it loads, exports every declared entry
point, and its host-side arithmetic (recipe, seeds, counts, validation) agrees
with the oracle.  No device call is made here."""
import os
import re

import numpy as np
import pytest

import klsynth
import oracle
from conftest import ROOT


@pytest.fixture(scope="module")
def kl():
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^KL_API\b[^;(]*?\b(kl_\w+)\s*\(", text, flags=re.M)
    return names


def test_every_declared_symbol_is_exported(kl):
    names = declared_functions()
    assert len(names) >= 9
    assert set(names) == set(kl.binding.API)
    assert set(kl.exported_symbols()) == set(names)


def test_word_count(kl):
    for d in range(0, 43):
        assert kl.word_count(d) == oracle.word_count(d)


def test_status_strings(kl):
    assert kl.status_string(0) == "ok"
    assert kl.status_string(4) == "workspace too small"
    assert kl.status_string(99) == "unknown status"


TRACES = [(2 + 0j, 2 + 0j), (1.91 + 0.05j, 1.91 + 0.05j), (3 + 0j, 3 + 0j)] + [
    (g.ta, g.tb) for g, _ in klsynth.draw_groups(klsynth.BATCH_SEED, 8)]


@pytest.mark.parametrize("ta,tb", TRACES)
def test_grandma_and_seeds_agree_with_oracle(kl, ta, tb):
    g_lib, g_or = kl.grandma(ta, tb), oracle.grandma(ta, tb)
    assert np.allclose(g_lib, g_or, rtol=1e-14, atol=1e-15)
    s_lib, s_or = kl.seeds(g_lib), oracle.seeds(g_or)
    assert np.allclose(s_lib, s_or, rtol=1e-12, atol=1e-13)


def test_grandma_rejects_bad_traces(kl):
    with pytest.raises(kl.KlError) as e:
        kl.grandma(float("nan") + 0j, 2 + 0j)
    assert e.value.status == 1
    # ta = tb = 0 makes the recipe's z0 denominator vanish
    with pytest.raises(kl.KlError):
        kl.grandma(0j, 0j)


def test_params_init_defaults(kl):
    p = kl.params_init(2 + 0j, 2 + 0j, 10, 1024, 768, (-1.5, 1.5, -1.0, 1.0))
    assert (p.depth, p.width, p.height) == (10, 1024, 768)
    assert (p.x0, p.x1, p.y0, p.y1) == (-1.5, 1.5, -1.0, 1.0)
    assert p.precision == kl.FP64 and p.renorm_every == 8 and p.parabolic_tol == 1e-6
    assert p.prefix_len == 0 and p.accumulate == 0
    assert p.mode == kl.LIMIT_SET and p.cull == 0
    assert np.allclose(list(p.gens), oracle.grandma(2, 2), atol=1e-15)


def test_workspace_validation(kl):
    good = kl.params_init(2 + 0j, 2 + 0j, 18, 4096, 4096, (-1.5, 1.5, -1.5, 1.5))
    n = kl.workspace_bytes(good)
    assert n > 0 and n % 256 == 0
    # suffix of 8 letters: 4 * 3^7 points; prefix of 10 letters: 4 * 3^9 slots
    assert n >= 4 * 3 ** 9 * (64 + 48 + 4) + 4 * 3 ** 7 * 24
    for field, bad in [("depth", 0), ("depth", 25), ("width", 0), ("height", 70000),
                       ("x1", -2.0), ("y0", float("nan")), ("prefix_len", 18)]:
        p = kl.params_init(2 + 0j, 2 + 0j, 18, 4096, 4096, (-1.5, 1.5, -1.5, 1.5))
        setattr(p, field, bad)
        assert kl.workspace_bytes(p) == 0, field


def test_autotuner_default_split_matches_library(kl):
    """The tuner's idea of the library's default prefix length gives the same
    workspace as letting the library choose (prefix_len = 0)."""
    from paper_1709_08018_gb300 import autotune
    for d in range(2, 24):
        p = kl.params_init(2 + 0j, 2 + 0j, d, 512, 512, (-1.5, 1.5, -1.5, 1.5))
        auto = kl.workspace_bytes(p)
        p.prefix_len = autotune.default_prefix_len(d, False)
        assert kl.workspace_bytes(p) == auto, d


def test_pruned_render_rejects_bad_edge(kl):
    """The edge guard must lie in [0, 1/2); the check comes before any device
    call (the pointers below are never dereferenced)."""
    import ctypes
    p = kl.params_init(2 + 0j, 2 + 0j, 22, 8192, 8192, (-2.0, 2.0, -2.0, 2.0), kl.MIXED)
    fake = 0x1000
    L = kl.binding.lib()
    for edge in (-0.01, 0.5, 0.7, float("nan")):
        st = L.kl_render_lod(ctypes.byref(p), 8, 15, fake, 0.0, edge, fake, fake, fake, fake,
                             1 << 30, None)
        assert st == 1, edge  # KL_EINVAL
        st = L.kl_render_lod_labels(ctypes.byref(p), 8, 15, fake, edge, fake, fake, fake, fake,
                                    1 << 30, None)
        assert st == 1, edge


def test_tiling_workspace_and_rejections(kl):
    """Tiling takes the largest table of its lengths; the batch and the
    level-of-detail calls take limit-set parameters only (checked before any
    device call)."""
    import ctypes
    for d in (1, 2, 9, 10, 11, 18, 20):
        p = kl.params_init(2 + 0j, 2 + 0j, d, 512, 512, (-1.5, 1.5, -1.5, 1.5))
        one = kl.workspace_bytes(p)
        p.mode = kl.TILING
        most = max(kl.workspace_bytes(kl.params_init(2 + 0j, 2 + 0j, k, 512, 512,
                                                     (-1.5, 1.5, -1.5, 1.5)))
                   for k in range(1, d + 1))
        assert kl.workspace_bytes(p) == max(one, most)
    p.mode = 2
    assert kl.workspace_bytes(p) == 0
    L = kl.binding.lib()
    p = kl.params_init(2 + 0j, 2 + 0j, 12, 64, 64, (-1.5, 1.5, -1.5, 1.5), mode=kl.TILING)
    h = ctypes.c_void_p()
    assert L.kl_batch_create(ctypes.byref(p), 1, ctypes.byref(h)) == 1
    assert L.kl_lod_label_bytes(ctypes.byref(p), 3, 8) == 0


def test_cull_workspace_and_rejections(kl):
    """Culled renders take their own split (long suffix tables: d - 1 letters
    up to 9, then about half the word plus one, at most 12), so their
    workspace differs; a caller's prefix length may leave up to 12 suffix
    letters; cull values above 1, and culled level-of-detail calls, are
    refused before any device call."""
    import ctypes
    win = (-1.5, 1.5, -1.5, 1.5)
    for d in (2, 9, 10, 11, 18, 20, 22, 24):
        sl = d - 1 if d - 1 <= 9 else min(12, max(9, d // 2 + 1))
        c = kl.params_init(2 + 0j, 2 + 0j, d, 512, 512, win, cull=1)
        w = kl.params_init(2 + 0j, 2 + 0j, d, 512, 512, win, cull=1, prefix_len=d - sl)
        assert kl.workspace_bytes(c) == kl.workspace_bytes(w) > 0
    for d, plen, ok in ((20, 8, True), (20, 7, False), (24, 12, True), (24, 11, False)):
        p = kl.params_init(2 + 0j, 2 + 0j, d, 512, 512, win, prefix_len=plen)
        assert (kl.workspace_bytes(p) > 0) == ok
    p = kl.params_init(2 + 0j, 2 + 0j, 25, 512, 512, win, cull=1)
    assert kl.workspace_bytes(p) == 0
    L = kl.binding.lib()
    p = kl.params_init(2 + 0j, 2 + 0j, 12, 64, 64, win, kl.MIXED, cull=2)
    assert L.kl_render(ctypes.byref(p), ctypes.c_void_p(16), None, ctypes.c_void_p(256),
                       ctypes.c_size_t(1 << 30), None) == 1
    h = ctypes.c_void_p()
    assert L.kl_batch_create(ctypes.byref(p), 1, ctypes.byref(h)) == 1  # cull = 2
    p.cull = 1
    assert L.kl_lod_label_bytes(ctypes.byref(p), 3, 8) == 0


def _klein():
    return [[[1j, 0], [0, -1j]], [[0, 1j], [1j, 0]], [[0, -1], [1, 0]]]


def test_fsa_count_agrees_with_the_oracle_scan(kl):
    from conftest import golden_table
    t11 = golden_table("t11_indexed_cayley.txt")
    k4 = golden_table("klein4_indexed_cayley.txt")
    g, s = oracle.group(2 + 0j, 2 + 0j)
    torus = kl.fsa(t11, [m.tolist() for m in oracle.as_matrices(g)], oracle.as_points(s))
    klein = kl.fsa(k4, _klein(), [0.3 + 0.2j, -0.4 + 0.3j, 0.1 - 0.6j])
    for d in range(1, 9):
        assert kl.fsa_count(torus, d) == oracle.fsa_count(4, t11, d) == 4 * 3 ** (d - 1)
        assert kl.fsa_count(klein, d) == oracle.fsa_count(3, k4, d)
    assert kl.fsa_count(torus, 20) == 4 * 3 ** 19          # beyond any scan
    # a table with a free letter: every string of length d survives
    free = kl.fsa([[0, 1], [0, 1]], [[[1, 1], [0, 1]]], [0j])
    assert kl.fsa_count(free, 12) == 1
    free2 = kl.fsa([[0, 1, 2], [0, 1, 2], [0, 1, 2]], _klein()[:2], [0j, 0j])
    assert kl.fsa_count(free2, 10) == 2 ** 10


def test_fsa_rejects_bad_input(kl):
    from conftest import golden_table
    k4 = golden_table("klein4_indexed_cayley.txt")
    f = kl.fsa(k4, _klein(), [0j, 0j, 0j])
    for d, status in [(0, 2), (33, 2), (26, 2)]:     # 3^26 > 2^40
        with pytest.raises(kl.KlError) as e:
            kl.fsa_count(f, d)
        assert e.value.status == status
    f.table[1 * 10 + 2] = 7                            # entry > m
    with pytest.raises(kl.KlError):
        kl.fsa_count(f, 4)
    f = kl.fsa(k4, _klein(), [0j, 0j, 0j])
    f.m = 10
    with pytest.raises(kl.KlError):
        kl.fsa_count(f, 4)
    f.m = 3
    f.gens[5] = float("nan")
    with pytest.raises(kl.KlError):
        kl.fsa_count(f, 4)


def test_fsa_from_params_carries_the_group(kl):
    from conftest import golden_table
    t11 = golden_table("t11_indexed_cayley.txt")
    p = kl.params_init(1.91 + 0.05j, 1.91 + 0.05j, 10, 64, 64, (-2.0, 2.0, -2.0, 2.0))
    f = kl.fsa_from_params(t11, p)
    g, s = oracle.group(1.91 + 0.05j, 1.91 + 0.05j)
    h = kl.fsa(t11, [m.tolist() for m in oracle.as_matrices(g)], oracle.as_points(s))
    assert f.m == h.m == 4 and bytes(f.table) == bytes(h.table)
    assert np.allclose(list(f.gens)[:32], list(h.gens)[:32], rtol=1e-14, atol=1e-15)
    assert np.allclose(list(f.seeds)[:8], list(h.seeds)[:8], rtol=1e-12, atol=1e-13)
    assert kl.fsa_count(f, 10) == oracle.word_count(10)


def test_maskit_agrees_with_the_oracle(kl):
    for mu in (-0.097 + 1.838j, 2j):
        g_lib, s_lib = kl.maskit(mu)
        g_or, s_or = oracle.maskit(mu)
        # the same maps: the matrices may differ by an overall sign
        for x in range(4):
            u, v = g_lib[8 * x: 8 * x + 8], g_or[8 * x: 8 * x + 8]
            assert np.allclose(u, v, atol=1e-15) or np.allclose(u, -v, atol=1e-15)
        assert np.allclose(s_lib, s_or, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("ta,tb", TRACES[:6])
def test_cusp_seeds_agree_with_the_oracle(kl, ta, tb):
    g = kl.grandma(ta, tb)
    assert np.allclose(kl.cusp_seeds(g), oracle.cusp_seeds(oracle.grandma(ta, tb)),
                       rtol=1e-9, atol=1e-12)


def test_multiseed_argument_checks_need_no_gpu(kl):
    """kl_render_multiseed refuses a missing, empty or non-finite point list
    before any device call (the pointers below are never dereferenced)."""
    import ctypes
    p = kl.params_init(2 + 0j, 2 + 0j, 10, 256, 256, (-1.5, 1.5, -1.5, 1.5), kl.MIXED)
    ws_bytes = kl.workspace_bytes(p)
    fake_img, fake_ws = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 24)
    L = kl.lib()
    ok_pts = np.array([0.1, 0.2, 0.3, 0.4])
    bad_pts = np.array([0.1, float("nan"), 0.3, 0.4])
    cases = [(None, 2), (ok_pts.ctypes.data, 0), (bad_pts.ctypes.data, 2)]
    for pts, n in cases:
        st = L.kl_render_multiseed(ctypes.byref(p), pts, n, fake_img, None, fake_ws, ws_bytes,
                                   None)
        assert st == 1, (pts, n, st)
    # and the render's own checks come first: a workspace that is too small
    st = L.kl_render_multiseed(ctypes.byref(p), ok_pts.ctypes.data, 2, fake_img, None, fake_ws,
                               ws_bytes - 256, None)
    assert st == 4
