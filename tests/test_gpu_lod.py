"""Level-of-detail labels and the network-pruned render.

  - with pruning switched off (margin +inf) the pruned render is the exact
    render of the level-hi prefixes: the same image, bit for bit;
  - with everything pruned at level lo, every word is still counted once;
  - the labels obey their recursion, and level-hi labels agree with the
    oracle's own test "the subtree's image is under `extent` pixels, or
    misses the window";
  - a network trained on 64 groups, with its pruning setting chosen on
    separate validation groups, renders 16 held-out groups faster than both
    exact methods without it (the per-word render, which evaluates every
    word, and the culled render) at occupancy IoU >= 0.999; pruning by the
    true labels with the edge guard at the label extent keeps IoU >= 0.9999.
"""
import numpy as np
import pytest

import klsynth
import oracle

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


def group_params(kl, g, d, size, window=(-2.0, 2.0, -2.0, 2.0), **fields):
    return kl.params_init(g.ta, g.tb, d, size, size, window, kl.MIXED, **fields)


def test_unpruned_equals_exact_and_full_pruning_conserves(kl):
    import torch
    from paper_1709_08018_gb300 import lod
    mlp = lod.init_params(1)
    for g, d in [(klsynth.NEAR_CUSP, 14), (klsynth.draw_groups(1710, 1)[0][0], 13)]:
        lo, hi = 4, 9
        p = group_params(kl, g, d, 1024, prefix_len=hi)
        img, cnt = kl.render(p)
        ref = img.cpu().numpy().copy()
        ref_c = cnt.cpu().numpy().copy()
        r = kl.LodRenderer(p, lo, hi)
        out, c, st = r(mlp, margin=1e30)       # never prune
        assert np.array_equal(out.cpu().numpy(), ref)
        assert np.array_equal(c.cpu().numpy()[:3], ref_c[:3])
        st = st.cpu().numpy()
        assert st[1] == 0 and st[2] == 4 * 3 ** (hi - 1)
        out, c, st = r(mlp, margin=-1e30)      # every score says "prune"
        c = c.cpu().numpy()
        assert int(c[0]) + int(c[1]) == kl.word_count(d)
        assert int(out.cpu().numpy().view(np.uint32).astype(np.int64).sum()) == int(c[0])
        # nodes whose three representative words share a pixel are pruned at once
        st = st.cpu().numpy()
        assert st[1] > 0 and st[0] >= 4 * 3 ** (lo - 1)
        torch.cuda.synchronize()


def subtree_pixels(g, s, d, k, slot, window, size):
    """Oracle pixel coordinates of all words of node `slot` at level k."""
    nk = 3 ** (k - 1)
    x, r = slot // nk, slot % nk
    digits = []
    for _ in range(k - 1):
        digits.append(r % 3)
        r //= 3
    digits = digits[::-1]             # most significant first: w_{k-1} .. w_1
    letters = [x]
    for dg in digits:
        ban = (letters[-1] + 2) % 4
        letters.append([y for y in range(4) if y != ban][dg])
    prefix = letters[::-1]            # w_1 .. w_k
    # word index: mixed radix of the prefix, then all suffix digits
    idx = prefix[0]
    for j in range(1, k):
        ban = (prefix[j - 1] + 2) % 4
        idx = idx * 3 + [y for y in range(4) if y != ban].index(prefix[j])
    m = d - k
    base = idx * 3 ** m
    ids = np.arange(base, base + 3 ** m, dtype=np.uint64)
    z = oracle.evaluate(g, s, d, ids)
    x0, x1, y0, y1 = window
    u = (z.real - x0) * size / (x1 - x0)
    v = (y1 - z.imag) * size / (y1 - y0)
    return u, v


def test_labels_recursion_and_oracle(kl):
    group = klsynth.draw_groups(1710, 2)[1][0]
    d, lo, hi, size, window = 12, 3, 8, 256, (-2.0, 2.0, -2.0, 2.0)
    p = group_params(kl, group, d, size, window)
    _, _, feats, labels = kl.lod_labels(p, lo, hi)
    labels = labels.cpu().numpy().astype(int)
    assert np.isfinite(feats.cpu().numpy()).all()
    base = {}
    acc = 0
    for k in range(lo, hi + 1):
        base[k] = acc
        acc += 4 * 3 ** (k - 1)
    assert acc == len(labels)
    for k in range(lo, hi):
        nk = 3 ** (k - 1)
        for slot in range(4 * nk):
            x, r = slot // nk, slot % nk
            ch = []
            for q in range(3):
                y = [t for t in range(4) if t != (x + 2) % 4][q]
                rk = x - (1 if x > (y + 2) % 4 else 0)
                ch.append(labels[base[k + 1] + y * 3 * nk + rk * nk + r])
            lab = labels[base[k] + slot]
            if max(ch) > 0:
                assert lab == 1 + max(ch)
            else:
                assert lab in (0, 1)
    # Level-hi labels, exactly: the label kernel bins each word at the value
    # the render computes (the mixed FP32 local frame, or FP64 for fallback
    # prefixes) into 1/256-pixel fixed point.  kl_eval_words returns those same
    # values for the same plan (prefix length hi), so boxes built from them
    # must give the same resolved / unresolved decision for every node.
    g, s = oracle.group(group.ta, group.tb)
    nh = 4 * 3 ** (hi - 1)
    ext = 256  # extent 1 pixel, in 1/256-pixel fixed point
    q = kl.Params.from_buffer_copy(p)
    q.prefix_len = hi
    sat = float(1 << 30)

    def resolved_of(u, v):
        fin = np.isfinite(u) & np.isfinite(v)
        if not fin.any():
            return True
        # floor(256 u), saturated as the kernel saturates far words
        cu = np.clip(np.floor(256.0 * u[fin]), -sat, sat).astype(np.int64)
        cv = np.clip(np.floor(256.0 * v[fin]), -sat, sat).astype(np.int64)
        far_u, far_v = np.abs(u[fin]) >= 2.0 ** 20, np.abs(v[fin]) >= 2.0 ** 20
        cu[far_u] = np.sign(u[fin][far_u]).astype(np.int64) * (1 << 30)
        cv[far_v] = np.sign(v[fin][far_v]).astype(np.int64) * (1 << 30)
        outside = cu.max() < 0 or cu.min() >= 256 * size or cv.max() < 0 or \
            cv.min() >= 256 * size
        small = cu.max() - cu.min() < ext and cv.max() - cv.min() < ext
        return outside or small

    ids_all = [node_word_ids(d, hi, slot) for slot in range(nh)]
    uv = kl.eval_words(q, dev_index(np.concatenate(ids_all))).cpu().numpy()
    same, agree_oracle, off = 0, 0, 0
    for slot in range(nh):
        n_w = len(ids_all[slot])
        mine = resolved_of(uv[off:off + n_w, 0], uv[off:off + n_w, 1])
        off += n_w
        same += (labels[base[hi] + slot] == 0) == mine
        u, v = subtree_pixels(g, s, d, hi, slot, window, size)
        agree_oracle += (labels[base[hi] + slot] == 0) == resolved_of(u, v)
    assert same == nh, (same, nh)
    # against the oracle's FP64 values the decisions may differ only where a
    # box side lies within rounding of the one-pixel extent or of the window
    # border (the mixed words differ from the oracle's by ~1e-8 relative)
    assert agree_oracle >= 0.995 * nh, (agree_oracle, nh)


def dev_index(idx):
    import torch
    return torch.from_numpy(np.ascontiguousarray(idx, dtype=np.uint64).view(np.int64)).cuda()


def node_word_ids(d, k, slot):
    """Word indices of the 3^(d-k) words below level-k node `slot`."""
    prefix = node_letters(k, slot)
    idx = prefix[0]
    for j in range(1, k):
        ban = (prefix[j - 1] + 2) % 4
        idx = idx * 3 + [y for y in range(4) if y != ban].index(prefix[j])
    m = d - k
    return np.arange(idx * 3 ** m, (idx + 1) * 3 ** m, dtype=np.uint64)


def node_letters(k, slot):
    """w_1 .. w_k of level-k node `slot` (x = w_k, ranks of w_{k-1} .. w_1)."""
    nk = 3 ** (k - 1)
    x, r = slot // nk, slot % nk
    digits = []
    for _ in range(k - 1):
        digits.append(r % 3)
        r //= 3
    letters = [x]
    for dg in digits[::-1]:
        ban = (letters[-1] + 2) % 4
        letters.append([y for y in range(4) if y != ban][dg])
    return letters[::-1]


def test_features_against_oracle(kl):
    """Features of sampled nodes of every level: the product of the oracle's
    generator matrices over the node's letters, divided by the principal root
    of its determinant, sign-canonicalised (Re tr > 0), then sign(v) log1p|v|."""
    group = klsynth.draw_groups(1710, 3)[2][0]
    d, lo, hi = 14, 3, 10
    p = group_params(kl, group, d, 512)
    _, _, feats, _ = kl.lod_labels(p, lo, hi)
    feats = feats.cpu().numpy()
    g, _ = oracle.group(group.ta, group.tb)
    M = oracle.as_matrices(g)
    rng = np.random.default_rng(7)
    base = 0
    for k in range(lo, hi + 1):
        n = 4 * 3 ** (k - 1)
        for slot in sorted(set(rng.integers(0, n, 64).tolist()) | {0, n - 1}):
            P = np.eye(2, dtype=complex)
            for w in node_letters(k, slot):
                P = P @ M[w]
            P = P / np.sqrt(np.linalg.det(P))
            v = np.array([P[0, 0].real, P[0, 0].imag, P[0, 1].real, P[0, 1].imag,
                          P[1, 0].real, P[1, 0].imag, P[1, 1].real, P[1, 1].imag])
            if v[0] + v[6] < 0:
                v = -v
            want = np.sign(v) * np.log1p(np.abs(v))
            np.testing.assert_allclose(feats[base + slot], want, rtol=1e-5, atol=1e-5,
                                       err_msg=f"level {k} slot {slot}")
        base += n
    assert base == feats.shape[0]


@pytest.mark.parametrize("prec,tol", [("MIXED", 2e-5), ("FP64", 1e-9), ("DF64", 1e-9)])
def test_depth22_word_values(kl, prec, tol):
    """The exact depth-22 render the pruned render is judged against (8192^2
    over [-2,2]^2, held-out groups): its word values on a seeded sample of
    1e5 indices against the oracle's per-word definition."""
    d, size, window = 22, 8192, (-2.0, 2.0, -2.0, 2.0)
    for g, _ in klsynth.draw_groups(klsynth.LOD_HELDOUT_SEED, 2):
        p = kl.params_init(g.ta, g.tb, d, size, size, window, getattr(kl, prec))
        idx = klsynth.index_sample(klsynth.SAMPLE_SEED, 100_000, d)
        uv = kl.eval_words(p, dev_index(idx)).cpu().numpy()
        go, so = oracle.group(g.ta, g.tb)
        z = oracle.evaluate(go, so, d, idx)
        sx = size / (window[1] - window[0])
        zg = (window[0] + uv[:, 0] / sx) + 1j * (window[3] - uv[:, 1] / sx)
        fin = np.isfinite(z) & (np.abs(z) < 1e12)
        assert np.isfinite(uv[fin]).all()
        err = np.abs(zg[fin] - z[fin]) / np.maximum(1.0, np.abs(z[fin]))
        print(f"\n{prec} d=22 group {g.ta:.4f}: max rel |dz| {err.max():.3e}")
        assert err.max() <= tol


def test_trained_network_gain(kl):
    """The benchmark's setting: a network trained on 64 groups, its pruning
    setting (margin, edge, last level) chosen on 8 validation groups, judged
    on the 16 held-out groups at depth 22, 8192^2.  Against the method
    without it, both ways: the per-word render (every word evaluated) and the
    exact culled render (kl_params.cull), which certifies sub-pixel blocks
    without the network's losses."""
    from paper_1709_08018_gb300 import lod
    d, lo, hi, size, extent = 22, 8, 15, 8192, 1.0 / 32
    train_groups = [g for g, _ in klsynth.draw_groups(klsynth.LOD_TRAIN_SEED, 64)]
    valid_groups = [g for g, _ in klsynth.draw_groups(klsynth.LOD_VALID_SEED, 8)]
    test_groups = [g for g, _ in klsynth.draw_groups(klsynth.LOD_HELDOUT_SEED, 16)]
    ptrain = [group_params(kl, g, d, size) for g in train_groups]
    x, t = lod.make_dataset(ptrain, lo, hi, per_level=60_000, seed=3, extent=extent)
    mlp, losses = lod.train(x, t, steps=10000, batch=16384, lr=2e-3, seed=5, under=32.0)
    assert losses[-1] < 0.01 * losses[0]
    tuned = lod.tune_prune([group_params(kl, g, d, size) for g in valid_groups], mlp, lo, hi,
                           target=0.9995)
    pruned_ms = exact_ms = culled_ms = 0.0
    iou_min = 1.0
    for n, g in enumerate(test_groups):
        p = group_params(kl, g, d, size)
        if n < 2:
            # true labels with the edge guard at the label extent: no word may
            # leave its pixel, up to the rounding of the mixed words
            floor = lod.evaluate_labels(p, lo, hi, extent)
            assert floor.words == kl.word_count(d) and floor.iou >= 0.9999, floor
        e = lod.evaluate(p, mlp, lo, tuned["hi"], tuned["margin"], tuned["edge"], repeats=2)
        assert e.words == kl.word_count(d)
        iou_min = min(iou_min, e.iou)
        pruned_ms += e.pruned_ms
        exact_ms += e.exact_ms
        q = kl.Params.from_buffer_copy(p)
        q.cull = 1
        rc = kl.Renderer(q)
        culled_ms += lod.time_ms(lambda: rc(), 2)
        del rc
    print(f"\n16 held-out groups: per-word {exact_ms:.2f} ms, pruned {pruned_ms:.2f} ms "
          f"(IoU min {iou_min:.5f}; margin {tuned['margin']}, edge {tuned['edge']}, "
          f"levels {lo}..{tuned['hi']}), culled exact {culled_ms:.2f} ms")
    assert iou_min >= 0.999, tuned
    # the gain over the per-word render
    assert pruned_ms < 0.2 * exact_ms
    # and over the exact culled render
    assert pruned_ms < culled_ms
