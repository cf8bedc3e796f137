"""ctypes binding of ``include/kl.h`` (argument marshalling only)."""
import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libkl.so")

FP64, MIXED, DF64 = 0, 1, 2
LIMIT_SET, TILING = 0, 1  # kl_mode
KL_CNT_IN_WINDOW, KL_CNT_DROPPED, KL_CNT_FP64_WORDS, KL_CNT_ATOMICS, KL_N_COUNTERS = 0, 1, 2, 3, 4

# Every function include/kl.h declares, in declaration order.
API = ("kl_status_string", "kl_word_count", "kl_grandma", "kl_seeds", "kl_maskit",
       "kl_cusp_seeds",
       "kl_params_init",
       "kl_decode_words", "kl_workspace_bytes", "kl_eval_words", "kl_render",
       "kl_render_multiseed",
       "kl_batch_create", "kl_batch_workspace_bytes", "kl_batch_render", "kl_batch_capture",
       "kl_batch_replay", "kl_batch_destroy", "kl_mlp_forward", "kl_mlp_scratch_bytes",
       "kl_mlp_grad", "kl_mlp_adam", "kl_mlp_train_step", "kl_wait_selftest",
       "kl_lod_node_count", "kl_lod_label_bytes", "kl_lod_labels",
       "kl_lod_render_bytes", "kl_render_lod", "kl_render_lod_labels", "kl_fsa_count",
       "kl_render_fsa", "kl_render_noalloc", "kl_set_profile_events")
KL_MLP_NPARAMS = 4801
KL_STATIC_SCRATCH_BYTES = 32 << 20


class Params(ctypes.Structure):
    """Mirror of ``kl_params``."""
    _fields_ = [
        ("gens", ctypes.c_double * 32),
        ("seeds", ctypes.c_double * 8),
        ("depth", ctypes.c_uint32),
        ("width", ctypes.c_uint32),
        ("height", ctypes.c_uint32),
        ("x0", ctypes.c_double),
        ("x1", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("y1", ctypes.c_double),
        ("precision", ctypes.c_uint32),
        ("renorm_every", ctypes.c_uint32),
        ("parabolic_tol", ctypes.c_double),
        ("prefix_len", ctypes.c_uint32),
        ("accumulate", ctypes.c_uint32),
        ("block_threads", ctypes.c_uint32),
        ("chunk_pairs", ctypes.c_uint32),
        ("mode", ctypes.c_uint32),
        ("cull", ctypes.c_uint32),
        ("shard_index", ctypes.c_uint32),
        ("shard_count", ctypes.c_uint32),
    ]


KL_FSA_MAX_LETTERS = 9
KL_FSA_WORKSPACE_BYTES = 256


class Fsa(ctypes.Structure):
    """Mirror of ``kl_fsa``: a group given by m Moebius generators, seeds and
    an indexed Cayley table (row stride KL_FSA_MAX_LETTERS + 1)."""
    _fields_ = [
        ("m", ctypes.c_uint32),
        ("table", ctypes.c_uint8 * ((KL_FSA_MAX_LETTERS + 1) ** 2)),
        ("gens", ctypes.c_double * (KL_FSA_MAX_LETTERS * 8)),
        ("seeds", ctypes.c_double * (KL_FSA_MAX_LETTERS * 2)),
    ]


def fsa(table, gens, seeds) -> Fsa:
    """A kl_fsa from an (m+1) x (m+1) table, m 2x2 complex matrices and m seeds."""
    m = len(gens)
    f = Fsa()
    f.m = m
    for r, row in enumerate(table):
        for c, v in enumerate(row):
            f.table[r * (KL_FSA_MAX_LETTERS + 1) + c] = int(v)
    for x, M in enumerate(gens):
        vals = [M[0][0], M[0][1], M[1][0], M[1][1]]
        for k, z in enumerate(vals):
            f.gens[8 * x + 2 * k] = complex(z).real
            f.gens[8 * x + 2 * k + 1] = complex(z).imag
    for x, z in enumerate(seeds):
        f.seeds[2 * x] = complex(z).real
        f.seeds[2 * x + 1] = complex(z).imag
    return f


def fsa_from_params(table, p: "Params") -> Fsa:
    """A kl_fsa with the four letters a, b, A, B of p (its generators and
    seeds) and the given (5 x 5) indexed table."""
    f = Fsa()
    f.m = 4
    for r, row in enumerate(table):
        for c, v in enumerate(row):
            f.table[r * (KL_FSA_MAX_LETTERS + 1) + c] = int(v)
    for k in range(32):
        f.gens[k] = p.gens[k]
    for k in range(8):
        f.seeds[k] = p.seeds[k]
    return f


def fsa_count(f: Fsa, depth: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().kl_fsa_count(ctypes.byref(f), depth, ctypes.byref(out)), "kl_fsa_count")
    return int(out.value)


def render_fsa(f: Fsa, p: "Params", image=None, counters=None, stream=None, device="cuda"):
    """kl_render_fsa with the view, size, depth and accumulate flag of p."""
    torch = _torch()
    if image is None:
        image = torch.empty((p.height, p.width), dtype=torch.int32, device=device)
    if counters is None:
        counters = torch.zeros(KL_N_COUNTERS, dtype=torch.int64, device=image.device)
    ws = torch.empty(KL_FSA_WORKSPACE_BYTES, dtype=torch.uint8, device=image.device)
    _check(lib().kl_render_fsa(ctypes.byref(f), ctypes.byref(p), image.data_ptr(),
                               counters.data_ptr(), ws.data_ptr(), ws.numel(),
                               _stream_handle(stream)), "kl_render_fsa")
    return image, counters


class KlError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"CUDA library {LIB_PATH} is missing: build it with __graft_entry__.build() "
                "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        P, U32, U64, I, D, SZ = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_size_t)
        L.kl_status_string.argtypes = [I]
        L.kl_status_string.restype = ctypes.c_char_p
        L.kl_word_count.argtypes = [U32]
        L.kl_word_count.restype = U64
        L.kl_grandma.argtypes = [D, D, D, D, P]
        L.kl_grandma.restype = I
        L.kl_seeds.argtypes = [P, P]
        L.kl_seeds.restype = I
        L.kl_maskit.argtypes = [D, D, P, P]
        L.kl_maskit.restype = I
        L.kl_cusp_seeds.argtypes = [P, P]
        L.kl_cusp_seeds.restype = I
        L.kl_params_init.argtypes = [ctypes.POINTER(Params), D, D, D, D, U32, U32, U32, D, D, D, D]
        L.kl_params_init.restype = I
        L.kl_decode_words.argtypes = [U32, P, U64, P, P]
        L.kl_decode_words.restype = I
        L.kl_workspace_bytes.argtypes = [ctypes.POINTER(Params)]
        L.kl_workspace_bytes.restype = SZ
        L.kl_eval_words.argtypes = [ctypes.POINTER(Params), P, U64, P, P, SZ, P]
        L.kl_eval_words.restype = I
        L.kl_render.argtypes = [ctypes.POINTER(Params), P, P, P, SZ, P]
        L.kl_render.restype = I
        L.kl_render_multiseed.argtypes = [ctypes.POINTER(Params), P, U32, P, P, P, SZ, P]
        L.kl_render_multiseed.restype = I
        L.kl_batch_create.argtypes = [ctypes.POINTER(Params), U32, ctypes.POINTER(P)]
        L.kl_batch_create.restype = I
        L.kl_batch_workspace_bytes.argtypes = [P]
        L.kl_batch_workspace_bytes.restype = SZ
        for fn in (L.kl_batch_render, L.kl_batch_capture):
            fn.argtypes = [P, P, P, P, SZ, P]
            fn.restype = I
        L.kl_batch_replay.argtypes = [P, P]
        L.kl_batch_replay.restype = I
        L.kl_batch_destroy.argtypes = [P]
        L.kl_batch_destroy.restype = None
        L.kl_mlp_forward.argtypes = [P, P, U64, P, P]
        L.kl_mlp_forward.restype = I
        L.kl_mlp_scratch_bytes.argtypes = [U64]
        L.kl_mlp_scratch_bytes.restype = SZ
        L.kl_mlp_grad.argtypes = [P, P, P, U64, ctypes.c_float, P, P, P, SZ, P]
        L.kl_mlp_grad.restype = I
        L.kl_mlp_adam.argtypes = [P, P, P, P, U32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, P]
        L.kl_mlp_adam.restype = I
        L.kl_mlp_train_step.argtypes = [P, P, P, P, P, U64, ctypes.c_float, U32, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P, P,
                                        SZ, P]
        L.kl_mlp_train_step.restype = I
        L.kl_wait_selftest.argtypes = [U64, P, P]
        L.kl_wait_selftest.restype = I
        L.kl_lod_node_count.argtypes = [U32, U32]
        L.kl_lod_node_count.restype = U64
        L.kl_lod_label_bytes.argtypes = [ctypes.POINTER(Params), U32, U32]
        L.kl_lod_label_bytes.restype = SZ
        L.kl_lod_labels.argtypes = [ctypes.POINTER(Params), U32, U32, ctypes.c_float, P, P, P, P,
                                    P, SZ, P]
        L.kl_lod_labels.restype = I
        L.kl_lod_render_bytes.argtypes = [ctypes.POINTER(Params), U32, U32]
        L.kl_lod_render_bytes.restype = SZ
        L.kl_render_lod.argtypes = [ctypes.POINTER(Params), U32, U32, P, ctypes.c_float,
                                    ctypes.c_float, P, P, P,
                                    P, SZ, P]
        L.kl_render_lod.restype = I
        L.kl_render_lod_labels.argtypes = [ctypes.POINTER(Params), U32, U32, P, ctypes.c_float, P,
                                           P, P, P, SZ, P]
        L.kl_render_lod_labels.restype = I
        L.kl_fsa_count.argtypes = [ctypes.POINTER(Fsa), U32, ctypes.POINTER(ctypes.c_uint64)]
        L.kl_fsa_count.restype = I
        L.kl_render_fsa.argtypes = [ctypes.POINTER(Fsa), ctypes.POINTER(Params), P, P, P, SZ, P]
        L.kl_render_fsa.restype = I
        L.kl_render_noalloc.argtypes = [ctypes.POINTER(Params), P, P, P]
        L.kl_render_noalloc.restype = I
        L.kl_set_profile_events.argtypes = [P, P]
        L.kl_set_profile_events.restype = I
        _lib = L
    return _lib


def exported_symbols() -> Tuple[str, ...]:
    """Names of API that the loaded library exports."""
    L = lib()
    return tuple(n for n in API if hasattr(L, n))


def status_string(status: int) -> str:
    return lib().kl_status_string(status).decode()


def _check(status: int, what: str):
    if status != 0:
        raise KlError(status, what)


def word_count(depth: int) -> int:
    return int(lib().kl_word_count(depth))


def grandma(ta: complex, tb: complex) -> np.ndarray:
    out = np.zeros(32, dtype=np.float64)
    _check(lib().kl_grandma(ta.real, ta.imag, tb.real, tb.imag, out.ctypes.data), "kl_grandma")
    return out


def seeds(gens) -> np.ndarray:
    g = np.ascontiguousarray(gens, dtype=np.float64)
    out = np.zeros(8, dtype=np.float64)
    _check(lib().kl_seeds(g.ctypes.data, out.ctypes.data), "kl_seeds")
    return out


def maskit(mu: complex):
    """Maskit's slice group a(z) = mu + 1/z, b(z) = z + 2 (kl_maskit):
    (32 generator doubles, 8 seed doubles)."""
    g = np.zeros(32, dtype=np.float64)
    s = np.zeros(8, dtype=np.float64)
    _check(lib().kl_maskit(mu.real, mu.imag, g.ctypes.data, s.ctypes.data), "kl_maskit")
    return g, s


def cusp_seeds(gens) -> np.ndarray:
    """kl_cusp_seeds: 8 seed points (16 doubles) for multi-seed feeding."""
    g = np.ascontiguousarray(gens, dtype=np.float64)
    out = np.zeros(16, dtype=np.float64)
    _check(lib().kl_cusp_seeds(g.ctypes.data, out.ctypes.data), "kl_cusp_seeds")
    return out


def render_multiseed(p: "Params", points, image=None, counters=None, workspace=None,
                     stream=None, device="cuda"):
    """kl_render_multiseed: every word of p drawn once per seed point (all four
    seeds set to it), into one image and one set of counters.  points:
    complex seed points."""
    torch = _torch()
    pts = np.array([[complex(z).real, complex(z).imag] for z in points], dtype=np.float64)
    if image is None:
        image = torch.empty((p.height, p.width), dtype=torch.int32, device=device)
    if counters is None:
        counters = torch.zeros(KL_N_COUNTERS, dtype=torch.int64, device=image.device)
    workspace = _workspace(p, image.device, workspace)
    _check(lib().kl_render_multiseed(ctypes.byref(p), pts.ctypes.data, len(pts),
                                     image.data_ptr(), counters.data_ptr(),
                                     workspace.data_ptr(), workspace.numel(),
                                     _stream_handle(stream)), "kl_render_multiseed")
    return image, counters


def render_repetends(p: "Params", image=None, counters=None, workspace=None, stream=None,
                     device="cuda"):
    """Repetend points: every word w of p drawn at w(fix t) for the parabolic
    tails t, the limits of the infinite words w t t t ... (near a cusp the
    orbit w t^n(z) reaches that limit only like 1/n, so a fixed-depth render
    leaves it out).  The parabolic tails are the cyclic permutations of the
    commutator abAB and of its inverse; their fixed points are the four
    commutator points of kl_cusp_seeds (entries 4..7), and after any last
    letter of w some reduced tail reaches each of them, so this is the
    multi-seed render over those four points (4 N_d words drawn).  Add it to
    p's ordinary render (accumulate = 1) to fill in the cusps."""
    s16 = cusp_seeds(list(p.gens))
    points = [complex(s16[2 * i], s16[2 * i + 1]) for i in range(4, 8)]
    return render_multiseed(p, points, image, counters, workspace, stream, device)


def params_group(gens, seeds8, depth: int, width: int, height: int, window: Sequence[float],
                 precision: int = FP64, **fields) -> Params:
    """Parameters for the caller's own generators and seeds (32 and 8
    doubles), with the same defaults as params_init."""
    p = params_init(2 + 0j, 2 + 0j, depth, width, height, window, precision, **fields)
    for k in range(32):
        p.gens[k] = float(gens[k])
    for k in range(8):
        p.seeds[k] = float(seeds8[k])
    return p


def params_init(ta: complex, tb: complex, depth: int, width: int, height: int,
                window: Sequence[float], precision: int = FP64, **fields) -> Params:
    p = Params()
    x0, x1, y0, y1 = window
    _check(lib().kl_params_init(ctypes.byref(p), ta.real, ta.imag, tb.real, tb.imag, depth,
                                width, height, x0, x1, y0, y1), "kl_params_init")
    p.precision = precision
    for k, v in fields.items():
        setattr(p, k, v)
    return p


def workspace_bytes(p: Params) -> int:
    return int(lib().kl_workspace_bytes(ctypes.byref(p)))


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _index_ptr(index):
    torch = _torch()
    if not index.is_cuda or not index.is_contiguous():
        raise ValueError("indices must be a contiguous CUDA tensor")
    if index.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise ValueError("indices must be int64 or uint64")
    return index.data_ptr()


def decode_words(depth: int, index, stream=None):
    """Letters (n, depth) uint8 of a CUDA tensor of word indices."""
    torch = _torch()
    n = index.numel()
    out = torch.empty((n, depth), dtype=torch.uint8, device=index.device)
    _check(lib().kl_decode_words(depth, _index_ptr(index), n, out.data_ptr(),
                                 _stream_handle(stream)), "kl_decode_words")
    return out


def _workspace(p: Params, device, workspace=None):
    """The caller's workspace as given (the library checks its size and
    alignment), or a new one of kl_workspace_bytes(p) bytes."""
    if workspace is not None:
        return workspace
    need = workspace_bytes(p)
    if need == 0:
        raise KlError(1, "kl_workspace_bytes")
    return _torch().empty(need, dtype=torch_uint8(), device=device)


def torch_uint8():
    return _torch().uint8


def eval_words(p: Params, index, workspace=None, stream=None):
    """Pixel coordinates (n, 2) float64 of the given words, computed exactly as
    kl_render computes them."""
    torch = _torch()
    n = index.numel()
    ws = _workspace(p, index.device, workspace)
    out = torch.empty((n, 2), dtype=torch.float64, device=index.device)
    _check(lib().kl_eval_words(ctypes.byref(p), _index_ptr(index), n, out.data_ptr(),
                               ws.data_ptr(), ws.numel(), _stream_handle(stream)),
           "kl_eval_words")
    return out


def render(p: Params, image=None, counters=None, workspace=None, stream=None, device="cuda"):
    """Render into a (height, width) uint32 CUDA image; returns (image, counters)."""
    torch = _torch()
    if image is None:
        image = torch.empty((p.height, p.width), dtype=torch.int32, device=device)
    if counters is None:
        counters = torch.zeros(KL_N_COUNTERS, dtype=torch.int64, device=image.device)
    if image.numel() != p.width * p.height or image.element_size() != 4 or not image.is_cuda:
        raise ValueError("image must be a CUDA tensor of width*height 32-bit elements")
    ws = _workspace(p, image.device, workspace)
    _check(lib().kl_render(ctypes.byref(p), image.data_ptr(), counters.data_ptr(), ws.data_ptr(),
                           ws.numel(), _stream_handle(stream)), "kl_render")
    return image, counters


def render_noalloc(p: Params, image, counters, stream=None):
    """kl_render_noalloc: render into caller-provided image and counters using
    the library's own static scratch array (no allocation anywhere)."""
    if image.numel() != p.width * p.height or image.element_size() != 4 or not image.is_cuda:
        raise ValueError("image must be a CUDA tensor of width*height 32-bit elements")
    _check(lib().kl_render_noalloc(ctypes.byref(p), image.data_ptr(), counters.data_ptr(),
                                   _stream_handle(stream)), "kl_render_noalloc")
    return image, counters


class Batch:
    """A batched render of many groups (kl_batch_*): one persistent launch,
    optionally captured once in a CUDA graph and replayed."""

    def __init__(self, params, device="cuda"):
        torch = _torch()
        n = len(params)
        arr = (Params * n)(*params)
        h = ctypes.c_void_p()
        _check(lib().kl_batch_create(arr, n, ctypes.byref(h)), "kl_batch_create")
        self.handle = h
        self.n = n
        self.width, self.height = params[0].width, params[0].height
        need = int(lib().kl_batch_workspace_bytes(h))
        self.workspace = torch.empty(need, dtype=torch.uint8, device=device)
        self.images = torch.empty((n, self.height, self.width), dtype=torch.int32, device=device)
        self.counters = torch.zeros((n, KL_N_COUNTERS), dtype=torch.int64, device=device)
        self.captured = False

    def _args(self):
        return (self.handle, self.images.data_ptr(), self.counters.data_ptr(),
                self.workspace.data_ptr(), self.workspace.numel())

    def render(self, stream=None):
        _check(lib().kl_batch_render(*self._args(), _stream_handle(stream)), "kl_batch_render")
        return self.images, self.counters

    def capture(self):
        """Capture the batch into a CUDA graph (on a side stream: the legacy
        default stream cannot be captured)."""
        torch = _torch()
        side = torch.cuda.Stream(device=self.images.device)
        side.wait_stream(torch.cuda.current_stream(self.images.device))
        _check(lib().kl_batch_capture(*self._args(), side.cuda_stream), "kl_batch_capture")
        torch.cuda.current_stream(self.images.device).wait_stream(side)
        self.captured = True

    def replay(self, stream=None):
        _check(lib().kl_batch_replay(self.handle, _stream_handle(stream)), "kl_batch_replay")
        return self.images, self.counters

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            try:
                _torch().cuda.synchronize()
            except Exception:
                pass
            _lib.kl_batch_destroy(h)
            self.handle = None


def mlp_forward(params, x, stream=None):
    """y = MLP(x): params (KL_MLP_NPARAMS,) float32, x (n, 8) float32, CUDA."""
    torch = _torch()
    n = x.shape[0]
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    _check(lib().kl_mlp_forward(params.data_ptr(), x.data_ptr(), n, y.data_ptr(),
                                _stream_handle(stream)), "kl_mlp_forward")
    return y


def wait_selftest(limit_cycles: int, stream=None):
    """kl_wait_selftest: (gave up, completed, cycles the give-up took)."""
    torch = _torch()
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    _check(lib().kl_wait_selftest(limit_cycles, out.data_ptr(), _stream_handle(stream)),
           "kl_wait_selftest")
    r = out.cpu().numpy().view(np.uint32)
    return bool(r[0]), bool(r[1]), int(r[2])


class MlpTrainer:
    """Adam training of the MLP with the library's kernels (kl_mlp_grad +
    kl_mlp_adam); params is updated in place."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, under_weight=1.0):
        torch = _torch()
        self.params = params
        self.under_weight = under_weight
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.grad = torch.zeros_like(params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=params.device)
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.step_no = 0
        self.scratch = None

    def gradient(self, x, t, stream=None):
        torch = _torch()
        n = x.shape[0]
        need = int(lib().kl_mlp_scratch_bytes(n))
        if self.scratch is None or self.scratch.numel() < need:
            self.scratch = torch.empty(need, dtype=torch.uint8, device=x.device)
        _check(lib().kl_mlp_grad(self.params.data_ptr(), x.data_ptr(), t.data_ptr(), n,
                                 self.under_weight, self.grad.data_ptr(), self.loss.data_ptr(),
                                 self.scratch.data_ptr(), self.scratch.numel(),
                                 _stream_handle(stream)), "kl_mlp_grad")
        return self.grad, self.loss

    def step(self, x, t, stream=None):
        """One Adam step on rows x, targets t (kl_mlp_train_step: gradient,
        fixed-order sum and Adam update); returns the loss before the step."""
        torch = _torch()
        n = x.shape[0]
        need = int(lib().kl_mlp_scratch_bytes(n))
        if self.scratch is None or self.scratch.numel() < need:
            self.scratch = torch.empty(need, dtype=torch.uint8, device=x.device)
        self.step_no += 1
        _check(lib().kl_mlp_train_step(self.params.data_ptr(), self.m.data_ptr(),
                                       self.v.data_ptr(), x.data_ptr(), t.data_ptr(), n,
                                       self.under_weight, self.step_no, self.lr, self.b1, self.b2,
                                       self.eps, self.loss.data_ptr(), self.grad.data_ptr(),
                                       self.scratch.data_ptr(), self.scratch.numel(),
                                       _stream_handle(stream)), "kl_mlp_train_step")
        return self.loss

    def step_separate(self, x, t, stream=None):
        """The same step as two calls, kl_mlp_grad then kl_mlp_adam."""
        self.gradient(x, t, stream)
        self.step_no += 1
        _check(lib().kl_mlp_adam(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                 self.grad.data_ptr(), self.step_no, self.lr, self.b1, self.b2,
                                 self.eps, _stream_handle(stream)), "kl_mlp_adam")
        return self.loss


def lod_node_count(lo: int, hi: int) -> int:
    return int(lib().kl_lod_node_count(lo, hi))


def lod_labels(p: Params, lo: int, hi: int, extent: float = 1.0, workspace=None, stream=None,
               device="cuda"):
    """Exact render plus per-node labels (uint8) and features (n, 8) of levels
    lo..hi (kl_lod_labels).  Returns (image, counters, features, labels)."""
    torch = _torch()
    n = lod_node_count(lo, hi)
    need = int(lib().kl_lod_label_bytes(ctypes.byref(p), lo, hi))
    if n == 0 or need == 0:
        raise KlError(2, "kl_lod_label_bytes")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=device)
    image = torch.empty((p.height, p.width), dtype=torch.int32, device=device)
    counters = torch.zeros(KL_N_COUNTERS, dtype=torch.int64, device=device)
    feats = torch.empty((n, 8), dtype=torch.float32, device=device)
    labels = torch.empty(n, dtype=torch.uint8, device=device)
    _check(lib().kl_lod_labels(ctypes.byref(p), lo, hi, extent, image.data_ptr(),
                               counters.data_ptr(),
                               feats.data_ptr(), labels.data_ptr(), workspace.data_ptr(),
                               workspace.numel(), _stream_handle(stream)), "kl_lod_labels")
    return image, counters, feats, labels


class LodRenderer:
    """Holds the workspace and outputs of kl_render_lod for repeated renders."""

    def __init__(self, p: Params, lo: int, hi: int, device="cuda"):
        torch = _torch()
        self.p, self.lo, self.hi = p, lo, hi
        need = int(lib().kl_lod_render_bytes(ctypes.byref(p), lo, hi))
        if need == 0:
            raise KlError(2, "kl_lod_render_bytes")
        self.workspace = torch.empty(need, dtype=torch.uint8, device=device)
        self.image = torch.empty((p.height, p.width), dtype=torch.int32, device=device)
        self.counters = torch.zeros(KL_N_COUNTERS, dtype=torch.int64, device=device)
        self.stats = torch.zeros(4, dtype=torch.int64, device=device)

    def __call__(self, mlp_params, margin: float = 0.0, edge: float = 0.0, stream=None):
        """Pruned render; `edge`: the distance in pixels a pruned node's
        representative words must keep from their pixel's sides."""
        _check(lib().kl_render_lod(ctypes.byref(self.p), self.lo, self.hi, mlp_params.data_ptr(),
                                   margin, edge, self.image.data_ptr(), self.counters.data_ptr(),
                                   self.stats.data_ptr(), self.workspace.data_ptr(),
                                   self.workspace.numel(), _stream_handle(stream)),
               "kl_render_lod")
        return self.image, self.counters, self.stats

    def with_labels(self, labels, edge: float = 0.0, stream=None):
        """The same render pruned by the true labels (kl_render_lod_labels)."""
        _check(lib().kl_render_lod_labels(ctypes.byref(self.p), self.lo, self.hi,
                                          labels.data_ptr(), edge, self.image.data_ptr(),
                                          self.counters.data_ptr(), self.stats.data_ptr(),
                                          self.workspace.data_ptr(), self.workspace.numel(),
                                          _stream_handle(stream)), "kl_render_lod_labels")
        return self.image, self.counters, self.stats


def set_profile_events(start=None, stop=None):
    """Record two torch.cuda.Event objects (already recorded once, so that
    they exist) around the main per-word kernel of every following render;
    no arguments switches it off."""
    a = start.cuda_event if start is not None else None
    b = stop.cuda_event if stop is not None else None
    _check(lib().kl_set_profile_events(a, b), "kl_set_profile_events")


class Renderer:
    """Holds parameters, workspace, image and counters for repeated renders."""

    def __init__(self, p: Params, device="cuda"):
        torch = _torch()
        self.p = p
        self.image = torch.empty((p.height, p.width), dtype=torch.int32, device=device)
        self.counters = torch.zeros(KL_N_COUNTERS, dtype=torch.int64, device=device)
        self.workspace = _workspace(p, device)

    def __call__(self, stream=None):
        return render(self.p, self.image, self.counters, self.workspace, stream)

    def capture(self):
        """Record one kl_render of p (its three launches: parts, combine and
        the per-word kernel) in a CUDA graph, after one render outside the
        capture; replay() then repeats it with one launch from the host."""
        torch = _torch()
        dev = self.image.device
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self()
        torch.cuda.current_stream(dev).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self()
        self.graph = g

    def replay(self):
        self.graph.replay()
        return self.image, self.counters
