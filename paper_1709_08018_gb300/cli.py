"""Render one of the named workloads (or a custom group) from the command line.

  python -m paper_1709_08018_gb300.cli --config gasket-d18-4096 --precision mixed \
      [--repeat N] [--out image.npy]
  python -m paper_1709_08018_gb300.cli --batch 32 [--repeat N]
  python -m paper_1709_08018_gb300.cli --lod [--train-groups 4] [--train-steps 300]
      [--per-level 20000] [--held-out 1] [--repeat N]
  python -m paper_1709_08018_gb300.cli --scan [--depth 14] [--repeat N]
  python -m paper_1709_08018_gb300.cli --mlp ROWS [--repeat N]

Prints the counters and the device time of the last render.  With --repeat N
the render runs N times (the first ones serve as warm-up for profilers).
--batch G renders the first G groups of the seeded 256-group sweep (depth
12..18, 1024^2 each) in one batched launch.  --lod trains the pruning network
briefly on a few seeded groups (labels, gradient and Adam kernels) and runs
the pruned depth-22 render of one held-out group at 8192^2.  --mlp ROWS
times the network's training step (gradient and Adam kernels) on ROWS seeded
random rows, N steps after 3 untimed ones.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import numpy as np
    import torch

    import klsynth
    import paper_1709_08018_gb300 as kl

    named = {c.name: c for c in (klsynth.C1, klsynth.C2, klsynth.C3)}
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default=klsynth.C2.name, choices=sorted(named))
    ap.add_argument("--ta", type=complex)
    ap.add_argument("--tb", type=complex)
    ap.add_argument("--depth", type=int)
    ap.add_argument("--size", type=int)
    ap.add_argument("--precision", choices=["fp64", "mixed", "df64"], default="mixed")
    ap.add_argument("--prefix-len", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--out")
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--lod", action="store_true")
    ap.add_argument("--train-groups", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--per-level", type=int, default=20_000)
    ap.add_argument("--held-out", type=int, default=1)
    ap.add_argument("--margin", type=float, default=-1.4, help="pruning margin (--lod)")
    ap.add_argument("--edge", type=float, default=1.0 / 128, help="edge guard in px (--lod)")
    ap.add_argument("--last-level", type=int, default=0,
                    help="last expanded level of the pruned render (--lod; default hi - 2)")
    ap.add_argument("--scan", action="store_true")
    ap.add_argument("--mlp", type=int, default=0, help="rows of a training-step timing")
    ap.add_argument("--tiling", action="store_true")
    ap.add_argument("--cull", action="store_true", help="place certified blocks of words at once")
    ap.add_argument("--seeds", choices=["one", "cusp", "repetends"], default="one",
                    help="one seed per first letter (default), the 8-point multi-seed list, or "
                         "its 4 repetend (commutator) points")
    a = ap.parse_args(argv)
    if a.batch:
        return run_batch(a, kl, klsynth, torch)
    if a.lod:
        return run_lod(a, kl, klsynth, torch)
    if a.scan:
        return run_scan(a, kl, klsynth, torch)
    if a.mlp:
        return run_mlp(a, kl, torch)
    c = named[a.config]
    ta = a.ta if a.ta is not None else c.group.ta
    tb = a.tb if a.tb is not None else c.group.tb
    depth = a.depth or c.depth
    W = H = a.size or c.width
    p = kl.params_init(ta, tb, depth, W, H, c.window,
                       {"mixed": kl.MIXED, "fp64": kl.FP64, "df64": kl.DF64}[a.precision],
                       prefix_len=a.prefix_len, mode=kl.TILING if a.tiling else kl.LIMIT_SET,
                       cull=int(a.cull))
    r = kl.Renderer(p)
    points = None
    if a.seeds != "one":
        s16 = kl.cusp_seeds(list(p.gens))
        first = 0 if a.seeds == "cusp" else 4
        points = [complex(s16[2 * i], s16[2 * i + 1]) for i in range(first, 8)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(a.repeat):
        e0.record()
        if points is None:
            r()
        else:
            kl.render_multiseed(p, points, r.image, r.counters, r.workspace)
        e1.record()
    torch.cuda.synchronize()
    cnt = r.counters.cpu().tolist()
    n = 1 if points is None else len(points)
    print(f"{a.config} {a.precision} d={depth} {W}x{H}: words {n * kl.word_count(depth)}, "
          f"in-window {cnt[0]}, dropped {cnt[1]}, fp64 words {cnt[2]}, atomics {cnt[3]}, "
          f"{e0.elapsed_time(e1):.3f} ms")
    if a.out:
        np.save(a.out, r.image.cpu().numpy().view(np.uint32))


def run_batch(a, kl, klsynth, torch):
    cfgs = klsynth.batch_configs(256)[:a.batch]
    ps = [kl.params_init(c.group.ta, c.group.tb, c.depth, c.width, c.height, c.window, kl.MIXED,
                         cull=int(a.cull)) for c in cfgs]
    b = kl.Batch(ps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(a.repeat):
        b.counters.zero_()
        e0.record()
        b.render()
        e1.record()
    torch.cuda.synchronize()
    cnt = b.counters.sum(0).cpu().tolist()
    words = sum(c.n_words for c in cfgs)
    print(f"batch of {a.batch} groups: words {words}, in-window {cnt[0]}, dropped {cnt[1]}, "
          f"fp64 words {cnt[2]}, atomics {cnt[3]}, {e0.elapsed_time(e1):.3f} ms")


def run_scan(a, kl, klsynth, torch):
    """The paper's scan (kl_render_fsa) of the gasket group with the torus
    table: all 4^d strings of depth d (default 14), FP64, 4096^2."""
    d = a.depth or 14
    W = a.size or 4096
    table = [[0, 1, 2, 3, 4], [1, 1, 2, 0, 4], [2, 1, 2, 3, 0], [3, 0, 2, 3, 4], [4, 1, 0, 3, 4]]
    p = kl.params_init(klsynth.GASKET.ta, klsynth.GASKET.tb, d, W, W, (-1.5, 1.5, -1.5, 1.5),
                       kl.FP64)
    f = kl.fsa_from_params(table, p)
    img = torch.empty((W, W), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(kl.KL_N_COUNTERS, dtype=torch.int64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(a.repeat):
        e0.record()
        kl.render_fsa(f, p, img, cnt)
        e1.record()
    torch.cuda.synchronize()
    c = cnt.cpu().tolist()
    print(f"scan d={d}: strings {4 ** d}, kept {c[2]}, in-window {c[0]}, "
          f"{e0.elapsed_time(e1):.3f} ms")


def run_mlp(a, kl, torch):
    """Training steps of the network (kl_mlp_grad + kl_mlp_adam) on --mlp
    seeded random rows; the per-step time of the last --repeat steps."""
    g = torch.Generator(device="cuda")
    g.manual_seed(1709)
    params = 0.1 * torch.randn(kl.KL_MLP_NPARAMS, device="cuda", generator=g)
    x = torch.randn(a.mlp, 8, device="cuda", generator=g)
    t = torch.randn(a.mlp, device="cuda", generator=g)
    tr = kl.MlpTrainer(params, lr=1e-3)
    for _ in range(3):
        tr.step(x, t)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.repeat):
        tr.step(x, t)
    e1.record()
    torch.cuda.synchronize()
    print(f"mlp training: {a.mlp} rows, {a.repeat} steps, "
          f"{1000.0 * e0.elapsed_time(e1) / a.repeat:.1f} us per step, "
          f"loss {float(tr.loss.item()):.4f}")


def run_lod(a, kl, klsynth, torch):
    """Train the pruning network on --train-groups groups (--per-level nodes
    per level, --train-steps steps; bench.py's setting is 64, 60000, 10000)
    and run the pruned render (--margin, --edge px, levels lo..--last-level)
    of the first --held-out held-out groups, --repeat times each, at depth
    --depth (22) and --size (8192) pixels.  The defaults are the setting
    bench.py's validation groups select (margin -1.4, edge 1/128 px, last
    level hi - 2)."""
    from paper_1709_08018_gb300 import lod
    # bench.py's setting by default; --depth and --size give a smaller case
    # (levels lo..hi follow the depth: hi = d - 7, lo = hi - 7)
    d, size, extent = a.depth or 22, a.size or 8192, 1.0 / 32
    hi = min(15, d - 7)
    lo = max(1, hi - 7)
    W = (-2.0, 2.0, -2.0, 2.0)
    mk = lambda g: kl.params_init(g.ta, g.tb, d, size, size, W, kl.MIXED)
    tr = [mk(g) for g, _ in klsynth.draw_groups(klsynth.LOD_TRAIN_SEED, a.train_groups)]
    x, t = lod.make_dataset(tr, lo, hi, per_level=a.per_level, seed=3, extent=extent)
    mlp, losses = lod.train(x, t, steps=a.train_steps, batch=16384, lr=2e-3, seed=5, under=32.0)
    last = a.last_level or max(lo, hi - 2)
    for g, _ in klsynth.draw_groups(klsynth.LOD_HELDOUT_SEED, a.held_out):
        L = kl.LodRenderer(mk(g), lo, last)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(a.repeat):
            e0.record()
            img, cnt, st = L(mlp, a.margin, a.edge)
            e1.record()
        torch.cuda.synchronize()
        st, cnt = st.cpu().tolist(), cnt.cpu().tolist()
        print(f"lod d={d} {size}^2 levels {lo}..{last}: loss {losses[0]:.3g} -> {losses[-1]:.3g}, "
              f"nodes {st[0]}, pruned {st[1]}, deferred {st[2]}, words {cnt[0] + cnt[1]}, "
              f"{e0.elapsed_time(e1):.3f} ms")
        del L

if __name__ == "__main__":
    main()
