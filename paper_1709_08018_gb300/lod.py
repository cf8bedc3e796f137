"""Learned level-of-detail pruning, end to end: training data from the exact
renderer, training with the library's tensor-core MLP kernels, and the
pruned render compared with the exact one.

All arithmetic runs in the library (kl_lod_labels, kl_mlp_grad, kl_mlp_adam,
kl_render_lod, kl_render); this module only selects samples and batches,
keeps the training loop and reports metrics.
"""
from dataclasses import dataclass
from typing import Dict, List, Sequence

import numpy as np

from . import binding as kb


def init_params(seed: int):
    """He-initialised network parameters (KL_MLP_NPARAMS floats, CUDA)."""
    import torch
    rng = np.random.default_rng(seed)
    p = np.zeros(kb.KL_MLP_NPARAMS, dtype=np.float32)
    p[0:512] = rng.normal(0.0, np.sqrt(2.0 / 8), 512)
    p[512:576] = 0.01
    p[576:4672] = rng.normal(0.0, np.sqrt(2.0 / 64), 4096)
    p[4672:4736] = 0.01
    p[4736:4800] = rng.normal(0.0, np.sqrt(1.0 / 64), 64)
    p[4800] = 1.0
    return torch.tensor(p, device="cuda")


def level_bounds(lo: int, hi: int):
    """(level, first node, node count) of each level in the node arrays."""
    out, base = [], 0
    for k in range(lo, hi + 1):
        n = 4 * 3 ** (k - 1)
        out.append((k, base, n))
        base += n
    return out


def make_dataset(params: Sequence[kb.Params], lo: int, hi: int, per_level: int, seed: int,
                 extent: float = 1.0, clip: float = 3.0):
    """Features and targets from every group: per level, `per_level` nodes
    drawn without replacement (all of a level's nodes when it has fewer), so
    that shallow levels, where a prune saves the most, are represented as
    well as deep ones.  Target: the label clipped to `clip` (the prune
    decision only needs to tell 0 from the rest)."""
    import ctypes
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    xs, ts = [], []
    ws = None
    for p in params:
        need = int(kb.lib().kl_lod_label_bytes(ctypes.byref(p), lo, hi))
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        _, _, f, lab = kb.lod_labels(p, lo, hi, extent=extent, workspace=ws)
        for _, base, n in level_bounds(lo, hi):
            if per_level < n:
                idx = base + torch.randperm(n, generator=gen, device="cuda")[:per_level]
            else:
                idx = torch.arange(base, base + n, device="cuda")
            xs.append(f[idx])
            ts.append(torch.clamp(lab[idx].float(), max=clip))
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous()


def train(x, t, steps: int, batch: int, lr: float, seed: int, init=None, under: float = 1.0):
    """Adam on the (weighted) mean squared error of the label, random
    mini-batches, learning rate decayed from `lr` to 0 along a half cosine
    (so that the final parameters do not carry the mini-batch noise of a
    constant rate); `under` > 1 weighs predictions below the label (too-early
    prunes) more."""
    import math
    import torch
    params = init_params(seed) if init is None else init.clone()
    tr = kb.MlpTrainer(params, lr=lr, under_weight=under)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 1)
    n = x.shape[0]
    losses = []
    for s in range(steps):
        tr.lr = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
        idx = torch.randint(0, n, (min(batch, n),), generator=gen, device="cuda")
        loss = tr.step(x[idx].contiguous(), t[idx].contiguous())
        if s % 50 == 0 or s == steps - 1:
            losses.append(float(loss.item()))
    return params, losses


@dataclass
class Eval:
    iou: float
    missed: int          # pixels hit by the exact render, empty in the pruned one
    extra: int           # pixels hit only by the pruned render
    occupied: int        # pixels hit by the exact render
    exact_ms: float
    pruned_ms: float
    nodes: int           # nodes scored by the network
    pruned_nodes: int
    deferred: int        # level-hi nodes rendered exactly
    words: int


def time_ms(fn, repeats: int = 3) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _compare(exact, img, cnt, st, exact_ms, pruned_ms) -> Eval:
    a, b = exact != 0, img != 0
    inter, union = int((a & b).sum()), int((a | b).sum())
    st, c = st.cpu().tolist(), cnt.cpu().tolist()
    return Eval(iou=inter / union if union else 1.0, missed=int((a & ~b).sum()),
                extra=int((b & ~a).sum()), occupied=int(a.sum()), exact_ms=exact_ms,
                pruned_ms=pruned_ms, nodes=st[0], pruned_nodes=st[1], deferred=st[2],
                words=c[0] + c[1])


def evaluate(p: kb.Params, mlp, lo: int, hi: int, margin: float, edge: float = 0.0,
             repeats: int = 3) -> Eval:
    """Pruned against exact render of one group (both timed with CUDA events)."""
    r = kb.Renderer(p)
    exact_ms = time_ms(lambda: r(), repeats)
    exact = r.image.clone()
    lod = kb.LodRenderer(p, lo, hi)
    pruned_ms = time_ms(lambda: lod(mlp, margin, edge), repeats)
    img, cnt, st = lod(mlp, margin, edge)
    return _compare(exact, img, cnt, st, exact_ms, pruned_ms)


def evaluate_labels(p: kb.Params, lo: int, hi: int, extent: float = 1.0) -> Eval:
    """Pruning by the true labels (edge guard = the label extent) against the
    exact render: what the splat loses when every prune decision is right."""
    r = kb.Renderer(p)
    exact_ms = time_ms(lambda: r(), 1)
    exact = r.image.clone()
    _, _, _, labels = kb.lod_labels(p, lo, hi, extent=extent)
    lod = kb.LodRenderer(p, lo, hi)
    pruned_ms = time_ms(lambda: lod.with_labels(labels, extent), 1)
    img, cnt, st = lod.with_labels(labels, extent)
    return _compare(exact, img, cnt, st, exact_ms, pruned_ms)


# Pruning settings tried by tune_prune: margin (added to the score before the
# 1/2 threshold; negative prunes more) x edge guard in pixels (larger sends
# more near-edge nodes down the tree).
PRUNE_MARGINS = (-1.4, -1.2, -1.0, -0.8, -0.6, -0.4, -0.2, 0.0)
PRUNE_EDGES = (0.0, 1 / 512, 1 / 128)


def tune_prune(params: Sequence[kb.Params], mlp, lo: int, hi: int, target: float = 0.9995,
               margins=PRUNE_MARGINS, edges=PRUNE_EDGES, his=None) -> Dict:
    """The fastest (margin, edge, hi) setting whose pruned renders of
    `params` all reach occupancy IoU >= target against their exact renders
    (the setting with the best worst-case IoU if none does).  hi is the last
    level the render expands (the network is trained on levels lo..hi; a
    smaller hi hands the remaining nodes to the exact render sooner); by
    default hi - 2 .. hi.  `params` are validation groups, apart from both the
    training and the held-out groups.  Returns {"margin", "edge", "hi",
    "tried": [(margin, edge, hi, worst IoU, ms)]}."""
    if his is None:
        his = [h for h in (hi - 2, hi - 1, hi) if h >= lo]
    exact = []
    for p in params:
        r = kb.Renderer(p)
        r()
        exact.append(r.image != 0)
        del r
    tried = []
    for h in his:
        lods = [kb.LodRenderer(p, lo, h) for p in params]
        for margin in margins:
            for edge in edges:
                worst, ms = 1.0, 0.0
                for occ, L in zip(exact, lods):
                    ms += time_ms(lambda: L(mlp, margin, edge), 1)
                    img, _, _ = L(mlp, margin, edge)
                    b = img != 0
                    union = int((occ | b).sum())
                    worst = min(worst, int((occ & b).sum()) / union if union else 1.0)
                tried.append((margin, edge, h, worst, ms))
        del lods
    ok = [t for t in tried if t[3] >= target]
    best = min(ok, key=lambda t: t[4]) if ok else max(tried, key=lambda t: t[3])
    return {"margin": best[0], "edge": best[1], "hi": best[2], "tried": tried}


def summarize(evals: List[Eval]) -> Dict:
    return {"groups": len(evals),
            "iou_min": min(e.iou for e in evals),
            "iou_mean": float(np.mean([e.iou for e in evals])),
            "missed_pixels": int(sum(e.missed for e in evals)),
            "extra_pixels": int(sum(e.extra for e in evals)),
            "occupied_pixels": int(sum(e.occupied for e in evals)),
            "exact_ms": float(sum(e.exact_ms for e in evals)),
            "pruned_ms": float(sum(e.pruned_ms for e in evals)),
            "speedup": float(sum(e.exact_ms for e in evals) / sum(e.pruned_ms for e in evals)),
            "nodes_scored": int(sum(e.nodes for e in evals)),
            "nodes_pruned": int(sum(e.pruned_nodes for e in evals)),
            "deferred_nodes": int(sum(e.deferred for e in evals)),
            "per_group": [{"iou": round(e.iou, 6), "exact_ms": round(e.exact_ms, 3),
                           "pruned_ms": round(e.pruned_ms, 3), "nodes": e.nodes,
                           "pruned": e.pruned_nodes, "deferred": e.deferred} for e in evals]}
