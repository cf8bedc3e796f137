"""ctypes front end of the C oracle (``kl_oracle.c``).

TEST INFRASTRUCTURE: see the package docstring.
"""
import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        D, U64, I, P = ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        L.or_grandma.argtypes = [D, D, D, D, P]
        L.or_grandma.restype = I
        L.or_seeds.argtypes = [P, P]
        L.or_seeds.restype = I
        L.or_word_count.argtypes = [I]
        L.or_word_count.restype = U64
        L.or_decode.argtypes = [I, U64, P]
        L.or_decode.restype = I
        L.or_decode_many.argtypes = [I, P, U64, P]
        L.or_decode_many.restype = I
        L.or_eval.argtypes = [P, P, I, P, U64, P]
        L.or_eval.restype = I
        L.or_render_indexed.argtypes = [P, P, I, P, I, I, U64, U64, P, P, D, P, P, U64, P]
        L.or_render_indexed.restype = I
        L.or_render_tree.argtypes = [P, P, I, P, I, I, I, I, I, P, P, D, P, P, U64, P]
        L.or_cusp_seeds.argtypes = [P, P]
        L.or_cusp_seeds.restype = I
        L.or_maskit.argtypes = [D, D, P, P]
        L.or_maskit.restype = I
        L.or_fsa_count.argtypes = [I, P, I, P]
        L.or_fsa_count.restype = I
        L.or_render_fsa.argtypes = [I, P, P, P, I, P, I, I, U64, U64, P, P, D, P, P, U64, P]
        L.or_render_fsa.restype = I
        L.or_prefix_rank.argtypes = [I, I, P, U64, P]
        L.or_prefix_rank.restype = I
        L.or_render_shard.argtypes = [P, P, I, P, I, I, I, I, I, P, P, D, P, P, U64, P]
        L.or_render_shard.restype = I
        L.or_tree_jobs.argtypes = [I]
        L.or_tree_jobs.restype = I
        L.or_render_tree.restype = I
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def grandma(ta: complex, tb: complex) -> np.ndarray:
    """Generators a, b, A, B from traces: 32 doubles, per matrix p, q, r, s as
    (re, im)."""
    out = np.zeros(32, dtype=np.float64)
    rc = lib().or_grandma(ta.real, ta.imag, tb.real, tb.imag, _ptr(out))
    if rc != 0:
        raise ValueError("degenerate traces for the recipe")
    return out


def seeds(gens: np.ndarray) -> np.ndarray:
    """Attracting fixed points of a, b, A, B: 8 doubles (re, im)."""
    g = np.ascontiguousarray(gens, dtype=np.float64)
    out = np.zeros(8, dtype=np.float64)
    if lib().or_seeds(_ptr(g), _ptr(out)) != 0:
        raise ValueError("a generator has no attracting finite fixed point")
    return out


def group(ta: complex, tb: complex) -> Tuple[np.ndarray, np.ndarray]:
    g = grandma(ta, tb)
    return g, seeds(g)


def as_matrices(gens: np.ndarray):
    """32 doubles -> list of four 2x2 complex128 matrices [[p, q], [r, s]]."""
    g = np.asarray(gens, dtype=np.float64).reshape(4, 4, 2)
    c = g[..., 0] + 1j * g[..., 1]
    return [c[k].reshape(2, 2) for k in range(4)]


def as_points(seeds8: np.ndarray):
    s = np.asarray(seeds8, dtype=np.float64).reshape(4, 2)
    return [complex(s[k, 0], s[k, 1]) for k in range(4)]


def word_count(d: int) -> int:
    return int(lib().or_word_count(d))


def decode(d: int, indices, strict: bool = True) -> np.ndarray:
    """Letter codes (n, d) uint8 of the given word indices.  An index outside
    [0, N_d) raises (strict) or decodes to letters 0xFF."""
    idx = np.ascontiguousarray(indices, dtype=np.uint64).ravel()
    out = np.zeros((idx.size, d), dtype=np.uint8)
    if lib().or_decode_many(d, _ptr(idx), idx.size, _ptr(out)) != 0:
        raise IndexError(f"bad depth {d}")
    if strict and idx.size and (out[:, 0] == 0xFF).any():
        raise IndexError(f"index outside [0, N_{d})")
    return out


def evaluate(gens, seeds8, d: int, indices) -> np.ndarray:
    """Word values (complex128) of the given indices, one sequential orbit per word."""
    idx = np.ascontiguousarray(indices, dtype=np.uint64).ravel()
    g = np.ascontiguousarray(gens, dtype=np.float64)
    s = np.ascontiguousarray(seeds8, dtype=np.float64)
    out = np.zeros(2 * idx.size, dtype=np.float64)
    if lib().or_eval(_ptr(g), _ptr(s), d, _ptr(idx), idx.size, _ptr(out)) != 0:
        raise IndexError("bad depth or index")
    return out[0::2] + 1j * out[1::2]


def tree_jobs(d: int) -> int:
    """Number of equal-size jobs the tree walk splits depth d into."""
    return int(lib().or_tree_jobs(d))


@dataclass
class Render:
    image: np.ndarray        # uint32 (H, W)
    in_window: int
    dropped: int
    edge_idx: np.ndarray     # uint64 (k,) indices of edge words
    edge_uv: np.ndarray      # float64 (k, 2) their pixel coordinates (u, v)
    edge_total: int          # edge words found (may exceed the stored k)


def render_tiling(gens, seeds8, d: int, window: Sequence[float], width: int, height: int,
                  mode: str = "tree", threads: Optional[int] = None, eta: float = 0.0,
                  edge_cap: int = 1 << 16) -> Render:
    """Tiling mode (Sec. "Implementation", the second drawing mode): every node
    of the word tree drawn at its own value, i.e. the words of every length
    1 .. d; the sum of the renders of each length (edge words of all lengths
    logged together, their indices relative to their own length)."""
    parts = [render(gens, seeds8, k, window, width, height, mode=mode, threads=threads, eta=eta,
                    edge_cap=edge_cap) for k in range(1, d + 1)]
    img = np.zeros((height, width), dtype=np.uint32)
    for r in parts:
        img += r.image
    return Render(img, sum(r.in_window for r in parts), sum(r.dropped for r in parts),
                  np.concatenate([r.edge_idx for r in parts]),
                  np.concatenate([r.edge_uv for r in parts]).reshape(-1, 2),
                  sum(r.edge_total for r in parts))


def render(gens, seeds8, d: int, window: Sequence[float], width: int, height: int,
           mode: str = "tree", threads: Optional[int] = None, eta: float = 0.0,
           edge_cap: int = 1 << 16, i0: int = 0, i1: Optional[int] = None,
           jobs: Optional[Tuple[int, int]] = None) -> Render:
    """Hit image of all reduced words of length d (mode "tree": tree walk,
    multi-threaded, optionally only the equal-size jobs [j0, j1) of
    ``tree_jobs(d)``; mode "indexed": per word over [i0, i1), single thread).
    Words whose pixel coordinates lie within ``eta`` pixels of a pixel edge are
    logged as edge words."""
    g = np.ascontiguousarray(gens, dtype=np.float64)
    s = np.ascontiguousarray(seeds8, dtype=np.float64)
    win = np.ascontiguousarray(window, dtype=np.float64)
    img = np.zeros((height, width), dtype=np.uint32)
    cnt = np.zeros(2, dtype=np.uint64)
    cap = edge_cap if eta > 0 else 0
    eidx = np.zeros(max(cap, 1), dtype=np.uint64)
    euv = np.zeros(2 * max(cap, 1), dtype=np.float64)
    ecount = np.zeros(1, dtype=np.uint64)
    L = lib()
    if mode == "tree":
        if threads is None:
            threads = os.cpu_count() or 1
        j0, j1 = jobs if jobs is not None else (0, tree_jobs(d))
        rc = L.or_render_tree(_ptr(g), _ptr(s), d, _ptr(win), width, height, threads, j0, j1,
                              _ptr(img), _ptr(cnt), eta, _ptr(eidx), _ptr(euv), cap, _ptr(ecount))
    elif mode == "indexed":
        n = word_count(d)
        i1 = n if i1 is None else i1
        rc = L.or_render_indexed(_ptr(g), _ptr(s), d, _ptr(win), width, height, i0, i1,
                                 _ptr(img), _ptr(cnt), eta, _ptr(eidx), _ptr(euv), cap,
                                 _ptr(ecount))
    else:
        raise ValueError(mode)
    if rc != 0:
        raise ValueError("bad render arguments")
    k = int(min(int(ecount[0]), cap))
    return Render(img, int(cnt[0]), int(cnt[1]), eidx[:k].copy(),
                  euv[:2 * k].reshape(k, 2).copy(), int(ecount[0]))


def prefix_rank(d: int, p: int, indices) -> np.ndarray:
    """Prefix slot ranks r (uint64) of the given words at prefix length p:
    the ranks of w_{p-1}, ..., w_1 among the letters other than the inverse of
    their right neighbour, base 3, w_{p-1} most significant (see
    or_render_shard)."""
    idx = np.ascontiguousarray(indices, dtype=np.uint64).ravel()
    out = np.zeros(idx.size, dtype=np.uint64)
    if lib().or_prefix_rank(d, p, _ptr(idx), idx.size, _ptr(out)) != 0:
        raise ValueError("bad depth, prefix length or index")
    return out


def render_shard(gens, seeds8, d: int, window: Sequence[float], width: int, height: int,
                 p: int, shard: int, n_shards: int, eta: float = 0.0,
                 edge_cap: int = 1 << 16) -> Render:
    """Per-word render of shard `shard` of `n_shards` at prefix length p: the
    words whose prefix slot rank r lies in [floor(k 3^(p-1)/n), floor((k+1)
    3^(p-1)/n)) (see or_render_shard)."""
    g = np.ascontiguousarray(gens, dtype=np.float64)
    s = np.ascontiguousarray(seeds8, dtype=np.float64)
    win = np.ascontiguousarray(window, dtype=np.float64)
    img = np.zeros((height, width), dtype=np.uint32)
    cnt = np.zeros(2, dtype=np.uint64)
    cap = edge_cap if eta > 0 else 0
    eidx = np.zeros(max(cap, 1), dtype=np.uint64)
    euv = np.zeros(2 * max(cap, 1), dtype=np.float64)
    ecount = np.zeros(1, dtype=np.uint64)
    rc = lib().or_render_shard(_ptr(g), _ptr(s), d, _ptr(win), width, height, p, shard,
                               n_shards, _ptr(img), _ptr(cnt), eta, _ptr(eidx), _ptr(euv), cap,
                               _ptr(ecount))
    if rc != 0:
        raise ValueError("bad shard render arguments")
    k = int(min(int(ecount[0]), cap))
    return Render(img, int(cnt[0]), int(cnt[1]), eidx[:k].copy(),
                  euv[:2 * k].reshape(k, 2).copy(), int(ecount[0]))


# ---------------------------------------------------------------------------
# general presentations (the paper's scan of the unpruned m-ary tree)

def fsa_count(m: int, table, d: int) -> int:
    """Strings of d symbols (1..m) that survive the run of the indexed table
    (rows = states 0..m, columns = symbols 0..m), counted by the scan."""
    t = np.ascontiguousarray(np.asarray(table, dtype=np.uint8).reshape(m + 1, m + 1))
    out = np.zeros(1, dtype=np.uint64)
    if lib().or_fsa_count(m, _ptr(t), d, _ptr(out)) != 0:
        raise ValueError("bad table or depth")
    return int(out[0])


def render_fsa(m: int, table, gens, seeds, d: int, window: Sequence[float], width: int,
               height: int, eta: float = 0.0, edge_cap: int = 1 << 16, i0: int = 0,
               i1: Optional[int] = None) -> Render:
    """Hit image of the kept strings of the scan of [i0, i1) (Sec.
    "Implementation"): gens = m matrices [[p, q], [r, s]] (complex), seeds = m
    points; edge words logged with their scan index."""
    t = np.ascontiguousarray(np.asarray(table, dtype=np.uint8).reshape(m + 1, m + 1))
    g = np.zeros((m, 8))
    for x in range(m):
        M = np.asarray(gens[x], dtype=complex).reshape(2, 2)
        g[x] = [M[0, 0].real, M[0, 0].imag, M[0, 1].real, M[0, 1].imag,
                M[1, 0].real, M[1, 0].imag, M[1, 1].real, M[1, 1].imag]
    sd = np.array([[complex(z).real, complex(z).imag] for z in seeds], dtype=np.float64)
    win = np.ascontiguousarray(window, dtype=np.float64)
    img = np.zeros((height, width), dtype=np.uint32)
    cnt = np.zeros(2, dtype=np.uint64)
    cap = edge_cap if eta > 0 else 0
    eidx = np.zeros(max(cap, 1), dtype=np.uint64)
    euv = np.zeros(2 * max(cap, 1), dtype=np.float64)
    ecount = np.zeros(1, dtype=np.uint64)
    i1 = m ** d if i1 is None else i1
    rc = lib().or_render_fsa(m, _ptr(t), _ptr(np.ascontiguousarray(g)), _ptr(sd), d, _ptr(win),
                             width, height, i0, i1, _ptr(img), _ptr(cnt), eta, _ptr(eidx),
                             _ptr(euv), cap, _ptr(ecount))
    if rc != 0:
        raise ValueError("bad render arguments")
    k = int(min(int(ecount[0]), cap))
    return Render(img, int(cnt[0]), int(cnt[1]), eidx[:k].copy(),
                  euv[:2 * k].reshape(k, 2).copy(), int(ecount[0]))


def maskit(mu: complex) -> Tuple[np.ndarray, np.ndarray]:
    """Maskit's slice group a(z) = mu + 1/z, b(z) = z + 2: (32 generator
    doubles, 8 seed doubles); see or_maskit."""
    g = np.zeros(32)
    s = np.zeros(8)
    if lib().or_maskit(mu.real, mu.imag, _ptr(g), _ptr(s)) != 0:
        raise ValueError("degenerate Maskit group")
    return g, s


# ---------------------------------------------------------------------------
# multi-seed feeding (the paper's loop over a list of fixed points)

def cusp_seeds(gens) -> np.ndarray:
    """8 seed points (16 doubles): the attracting fixed points of a, b, A, B,
    then the fixed points of abAB, bABa, ABab, BabA (see or_cusp_seeds)."""
    g = np.ascontiguousarray(gens, dtype=np.float64)
    out = np.zeros(16)
    if lib().or_cusp_seeds(_ptr(g), _ptr(out)) != 0:
        raise ValueError("degenerate group")
    return out


def render_multiseed(gens, points, d: int, window: Sequence[float], width: int, height: int,
                     threads: Optional[int] = None, eta: float = 0.0,
                     edge_cap: int = 1 << 16) -> Render:
    """Every reduced word of length d drawn once per seed point: the word's
    maps applied to each point of the list in turn, whatever its first
    letter (the paper's loop over fixed points).  points: k complex."""
    img = np.zeros((height, width), dtype=np.uint32)
    parts = []
    for z in points:
        s8 = np.array([complex(z).real, complex(z).imag] * 4, dtype=np.float64)
        r = render(gens, s8, d, window, width, height, threads=threads, eta=eta, edge_cap=edge_cap)
        img += r.image
        parts.append(r)
    return Render(img, sum(r.in_window for r in parts), sum(r.dropped for r in parts),
                  np.concatenate([r.edge_idx for r in parts]),
                  np.concatenate([r.edge_uv for r in parts]).reshape(-1, 2),
                  sum(r.edge_total for r in parts))
