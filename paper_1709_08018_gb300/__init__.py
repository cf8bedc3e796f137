"""GB300 indexed renderer of once-punctured-torus limit sets (arXiv:1709.08018).

Thin Python binding of the C ABI declared in ``include/kl.h``: every call
marshals arguments (torch CUDA tensors -> device pointers, the current torch
stream -> cudaStream_t) and calls the CUDA library ``_build/libkl.so``.  No
step of the method runs in Python.  Importing the package loads the library
and fails loudly if it has not been built (``__graft_entry__.build()`` or
``python -m paper_1709_08018_gb300.build``).
"""
from .binding import (  # noqa: F401
    DF64, FP64, KL_CNT_ATOMICS, KL_CNT_DROPPED, KL_CNT_FP64_WORDS, KL_CNT_IN_WINDOW, KL_MLP_NPARAMS,
    KL_N_COUNTERS, KL_STATIC_SCRATCH_BYTES, LIMIT_SET, MIXED, TILING, Batch, KlError,
    LodRenderer, MlpTrainer, Params, Renderer, lod_labels, lod_node_count, Fsa, fsa, fsa_count,
    fsa_from_params, maskit, params_group, cusp_seeds, render_multiseed, render_repetends,
    render_fsa,
    decode_words, eval_words, exported_symbols, grandma, lib, mlp_forward, params_init, render,
    render_noalloc, seeds, set_profile_events, status_string, word_count, workspace_bytes,
)
