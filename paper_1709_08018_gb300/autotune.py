"""Autotuner for the render kernels' launch shapes.

The knobs change how work is cut, never which words are counted:
  block_threads  threads per block of the render kernel (64, 128, 256);
  chunk_pairs    suffix-point pairs per work item (the tile along the suffix
                 dimension; 0 lets the library size items to ~12 per block);
  prefix_len     letters per cached prefix matrix, i.e. the split of each
                 word into a prefix tile and a suffix tile (changes only the
                 rounding association, within the tested tolerances).
Each candidate is timed with CUDA events on the current stream (single
renders: kl_render; batches: replays of the captured graph), the fastest is
returned and cached in a JSON file keyed by GPU name and workload.
"""
import itertools
import json
import os
import time
from typing import Dict, List, Optional, Sequence

from . import binding as kb

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuned.json")


def _gpu_name():
    import torch
    return torch.cuda.get_device_name()


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, rec):
    data = _load()
    data[key] = rec
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time_ms(fn, repeats: int) -> float:
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


def _apply(p: kb.Params, knobs: Dict[str, int]) -> kb.Params:
    q = kb.Params()
    import ctypes
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
    for k, v in knobs.items():
        setattr(q, k, v)
    return q


def default_prefix_len(depth: int, batched: bool) -> int:
    """The library's own split (kl_plan.cuh make_plan) for a depth."""
    if depth <= 1:
        return 1
    if batched:
        s = min(8, max(1, depth - 7))
    elif depth <= 10:
        s = 1
    else:
        s = min(9 if depth > 20 else 8, depth - 9)
    return depth - s


def tune_render(p: kb.Params, key: str, blocks: Sequence[int] = (64, 128, 256),
                chunks: Sequence[int] = (0, 32, 128), prefix_shifts: Sequence[int] = (0, -1, 1),
                repeats: int = 3, budget_s: float = 30.0, use_cache: bool = True) -> Dict:
    """Fastest knobs for a single render of p (words/s), cached under key."""
    full = f"{_gpu_name()}|render|{key}"
    if use_cache and full in _load():
        return _load()[full]
    base_p = default_prefix_len(p.depth, False)
    r = kb.Renderer(p)
    results: List[Dict] = []
    t0 = time.time()
    for bt, ch, sh in itertools.product(blocks, chunks, prefix_shifts):
        pl = base_p + sh
        if pl < 1 or p.depth - pl < 1 or pl > 15 or p.depth - pl > 9:
            continue
        q = _apply(p, {"block_threads": bt, "chunk_pairs": ch, "prefix_len": pl})
        need = kb.workspace_bytes(q)
        if need == 0:
            continue
        if need > r.workspace.numel():
            import torch
            r.workspace = torch.empty(need, dtype=torch.uint8, device=r.image.device)
        ms = _time_ms(lambda: kb.render(q, r.image, r.counters, r.workspace), repeats)
        results.append({"block_threads": bt, "chunk_pairs": ch, "prefix_len": pl, "ms": ms})
        if time.time() - t0 > budget_s:
            break
    best = min(results, key=lambda x: x["ms"])
    rec = {"best": best, "tried": results}
    _store(full, rec)
    return rec


def tune_batch(params: List[kb.Params], key: str, blocks: Sequence[int] = (64, 128, 256),
               chunks: Sequence[int] = (32, 64, 128), prefix_shifts: Sequence[int] = (0, -1),
               repeats: int = 3, budget_s: float = 60.0, use_cache: bool = True) -> Dict:
    """Fastest knobs for a batch (graph replays), cached under key."""
    import torch
    full = f"{_gpu_name()}|batch|{key}"
    if use_cache and full in _load():
        return _load()[full]
    results: List[Dict] = []
    t0 = time.time()
    for bt, ch, sh in itertools.product(blocks, chunks, prefix_shifts):
        ps = []
        for p in params:
            pl = default_prefix_len(p.depth, True) + sh
            pl = max(1, min(pl, p.depth - 1, 15))
            ps.append(_apply(p, {"block_threads": bt, "chunk_pairs": ch, "prefix_len": pl}))
        b = kb.Batch(ps)
        b.capture()
        ms = _time_ms(lambda: b.replay(), repeats)
        results.append({"block_threads": bt, "chunk_pairs": ch, "prefix_shift": sh, "ms": ms})
        del b
        torch.cuda.synchronize()
        if time.time() - t0 > budget_s:
            break
    best = min(results, key=lambda x: x["ms"])
    rec = {"best": best, "tried": results}
    _store(full, rec)
    return rec


def apply_batch(params: List[kb.Params], best: Dict) -> List[kb.Params]:
    """The batch's parameter sets with the tuned knobs."""
    out = []
    for p in params:
        pl = default_prefix_len(p.depth, True) + best.get("prefix_shift", 0)
        pl = max(1, min(pl, p.depth - 1, 15))
        out.append(_apply(p, {"block_threads": best["block_threads"],
                              "chunk_pairs": best["chunk_pairs"], "prefix_len": pl}))
    return out


def apply_render(p: kb.Params, best: Dict) -> kb.Params:
    return _apply(p, {"block_threads": best["block_threads"], "chunk_pairs": best["chunk_pairs"],
                      "prefix_len": best["prefix_len"]})
