"""FP64 CPU oracle for the indexed limit-set renderer (arXiv:1709.08018).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_1709_08018_gb300``) and never imports it.

Parity status per function (what pins it is in ``tests/test_oracle_pins.py``):
  grandma        pinned: trace, determinant and commutator-trace invariants,
                 the closed-form gasket matrices at ta = tb = 2
  seeds          pinned: fixed-point equation, attraction, gasket closed form
  decode         pinned: brute-force scan of all 4^d base-4 strings filtered
                 by the paper's indexed Cayley table (order and set), counts
  eval           pinned: the paper's abA orbit order, independent matrix
                 products, the Fuchsian circle, tree walk = per-word bitwise
  render         pinned: brute-force render from the scan, hit conservation
  render_tiling  pinned: brute-force scan over every length 1 .. d, the node
                 count 2 (3^d - 1)
  fsa_count,     pinned: the paper's scan written out in Python (set and
  render_fsa     image), the closed-form counts 4 3^(d-1) (once-punctured
                 torus table) and 3 2^(d-1) (Klein four-group table)
  cusp_seeds,    pinned: each commutator permutation has trace -2 and fixes
  render_multiseed its point; consecutive points are images under the
                 generators (conjugation); brute-force scan with fixed seeds
  mlp (numpy)    pinned: central finite differences, closed-form tiny nets
  prefix_rank,   pinned: (w_p, r) is a bijection of the prefixes onto
  render_shard   4 x 3^(p-1) slots (brute force); the shards' images and
                 counters sum to the whole per-word render; shard word counts
                 equal the closed form 4 3^(d-p) (slots of the shard)
"""
from .oracle import *  # noqa: F401,F403
