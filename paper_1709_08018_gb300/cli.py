"""Render one of the named workloads (or a custom group) from the command line.

  python -m paper_1709_08018_gb300.cli --config gasket-d18-4096 --precision mixed \
      [--repeat N] [--out image.npy]

Prints the counters and the device time of the last render.  With --repeat N
the render runs N times (the first ones serve as warm-up for profilers).
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
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--prefix-len", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--out")
    a = ap.parse_args(argv)
    c = named[a.config]
    ta = a.ta if a.ta is not None else c.group.ta
    tb = a.tb if a.tb is not None else c.group.tb
    depth = a.depth or c.depth
    W = H = a.size or c.width
    p = kl.params_init(ta, tb, depth, W, H, c.window,
                       kl.MIXED if a.precision == "mixed" else kl.FP64,
                       prefix_len=a.prefix_len)
    r = kl.Renderer(p)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(a.repeat):
        e0.record()
        r()
        e1.record()
    torch.cuda.synchronize()
    cnt = r.counters.cpu().tolist()
    print(f"{a.config} {a.precision} d={depth} {W}x{H}: words {kl.word_count(depth)}, "
          f"in-window {cnt[0]}, dropped {cnt[1]}, fp64 words {cnt[2]}, atomics {cnt[3]}, "
          f"{e0.elapsed_time(e1):.3f} ms")
    if a.out:
        np.save(a.out, r.image.cpu().numpy().view(np.uint32))


if __name__ == "__main__":
    main()
