/*
 * kl.h -- C ABI of the GB300 indexed limit-set renderer.
 *
 * The library renders the limit set (attractor) of a once-punctured-torus
 * group generated by four linear-fractional maps a, b, A = a^-1, B = b^-1,
 * following A. Rosa, "A new indexed approach to render the attractors of
 * Kleinian groups" (arXiv:1709.08018): every reduced word of length d over
 * {a, b, A, B} is pulled out of an integer index instead of being stored
 * (Sec. "The revised deterministic approach"), its maps are applied to a seed
 * point right to left (Sec. "Introduction"), and the resulting word value is
 * drawn into a hit image (Sec. "Implementation", the index-search loop).
 *
 * Conventions shared by every entry point:
 *  - Letters have codes a = 0, b = 1, A = 2, B = 3 (the row order of the
 *    paper's Cayley table, Sec. "Once-punctured torus groups", minus one), so
 *    the inverse of x is (x + 2) mod 4.
 *  - A word w_1 .. w_d is applied right to left: w_d first, w_1 last.
 *  - Word index i in [0, N_d), N_d = 4 * 3^(d-1): w_1 = floor(i / 3^(d-1)),
 *    then each base-3 digit c_k of the rest (most significant first) selects
 *    the c_k-th smallest letter other than inv(w_{k-1}).  This is the order
 *    in which the paper's base-4 scan filtered by the indexed Cayley table
 *    (Sec. "Cayley Multiplication Tables", "Implementation") meets reduced
 *    words.
 *  - Complex numbers are pairs of doubles (re, im).  A matrix [[p, q], [r, s]]
 *    acting as z -> (p z + q)/(r z + s) is stored as 8 doubles
 *    p.re p.im q.re q.im r.re r.im s.re s.im.
 *  - Pointers named d_* are device pointers (cudaMalloc'd, or torch CUDA
 *    tensors); all others are host pointers.  The caller owns every buffer;
 *    the library never allocates, frees or retains caller memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    work is enqueued asynchronously; argument errors are returned before
 *    anything is enqueued.  A CUDA launch error is returned as KL_ECUDA.
 *  - Return values are kl_status codes; no C++ exception crosses the ABI.
 */
#ifndef KL_H
#define KL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KL_API __attribute__((visibility("default")))
#else
#define KL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  KL_OK = 0,
  KL_EINVAL = 1,      /* a null pointer, a bad size, window or depth */
  KL_ERANGE = 2,      /* a value outside the representable range (e.g. N_d > 2^64) */
  KL_ECUDA = 3,       /* the CUDA runtime reported an error */
  KL_ENOSPACE = 4,    /* the workspace passed is smaller than required */
  KL_EDEGENERATE = 5  /* degenerate traces or generators (recipe or fixed point undefined) */
} kl_status;

/* Arithmetic of the per-word work. */
typedef enum {
  KL_FP64 = 0,   /* every step in FP64 */
  KL_MIXED = 1,  /* prefix products, renormalisation and near-parabolic words in
                    FP64; the per-word map in FP32 in a per-prefix local frame */
  KL_DF64 = 2    /* prefix products, tables and pole-form constants in FP64; the
                    per-word map in double-float arithmetic on the FP32 pipe (each
                    value an unevaluated sum of two floats, about 48 significant bits,
                    error-free sums and products built from FP32 adds and fused
                    multiply-adds), giving word values within the FP64 tolerance
                    (1e-9 relative) at FP32-pipe speed, 117 FP32 operations per word.  Prefixes whose pole form is
                    invalid or out of float range (P10 ~ 0, pixel offsets >= 2^20,
                    constants outside [1e-30, 1e30]) run in FP64.  kl_render (limit
                    set and tiling), kl_render_noalloc and kl_eval_words only; not
                    with cull = 1 */
} kl_precision;

/* Which words a render draws (Sec. "Implementation": the two drawing modes). */
typedef enum {
  KL_LIMIT_SET = 0,  /* the words of length exactly d: N_d = 4 3^(d-1) */
  KL_TILING = 1      /* every node of the word tree: all lengths 1 .. d,
                        sum_k N_k = 2 (3^d - 1) words, each drawn at its own value */
} kl_mode;

#define KL_MAX_DEPTH 40          /* N_40 = 4 * 3^39 < 2^64 */
#define KL_MAX_IMAGE_SIDE 65536  /* width and height limit */

/* Everything one render needs: the group (generators and seeds), the word
 * length, the view window and the image size.  Fill with kl_params_init, or
 * set the fields directly (gens and seeds from kl_grandma / kl_seeds or from
 * the caller's own matrices of determinant one). */
typedef struct {
  double gens[32];         /* a, b, A, B (8 doubles each, layout above) */
  double seeds[8];         /* seed point of each first-applied letter a, b, A, B */
  uint32_t depth;          /* word length d, 1 .. KL_MAX_DEPTH */
  uint32_t width, height;  /* image size in pixels, 1 .. KL_MAX_IMAGE_SIDE */
  double x0, x1, y0, y1;   /* window: x0 < x1, y0 < y1; pixel (row, col) covers
                              [x0 + col/sx, x0 + (col+1)/sx) x (y1 - (row+1)/sy, y1 - row/sy],
                              sx = width/(x1-x0), sy = height/(y1-y0); row 0 is the top */
  uint32_t precision;      /* kl_precision */
  uint32_t renorm_every;   /* prefix products are divided by sqrt(det) every this many
                              letters (0 = never); 8 by default */
  double parabolic_tol;    /* KL_MIXED: a prefix matrix P with
                              |tr(P)^2 - 4 det P| < tol * max(1, |tr P|^2) is near-parabolic
                              and its words are evaluated in FP64; default 1e-6 */
  uint32_t prefix_len;     /* letters per cached prefix matrix, 1 .. 15 leaving 1 .. 12
                              suffix letters (0 = choose) */
  uint32_t accumulate;     /* 0: kl_render zeroes the image and counters first;
                              1: it adds to them */
  uint32_t block_threads;  /* threads per block of the render kernels: 64, 128 or 256
                              (0 = 128); a tuning knob, results do not depend on it */
  uint32_t chunk_pairs;    /* suffix-point pairs per work item (FP64: twice as many points;
                              culled renders: culling blocks per item); 0 = choose; a
                              tuning knob, results do not depend on it */
  uint32_t mode;           /* kl_mode: KL_LIMIT_SET (default) or KL_TILING; kl_render and
                              kl_render_noalloc only (the batch and level-of-detail calls
                              take KL_LIMIT_SET; kl_eval_words evaluates length-d words) */
  uint32_t cull;           /* kl_render, kl_render_noalloc and batches (the level-of-detail
                              calls take 0; their exact render of deferred nodes culls
                              anyway, with the same image): 0 (default)
                              evaluates every word; 1 places whole blocks of words at once.
                              The suffix points of one subtree (blocks of 9 .. 729 points,
                              fewer for short words, each block's children being the three
                              blocks of a third its size inside it) are bounded by a disk; a
                              prefix map sends that disk onto a disk in closed form, and when
                              the image disk, widened by a rounding margin, lies inside one
                              pixel or wholly outside the window, every word of the block
                              lands there and is tallied without being evaluated.  Otherwise
                              the block's children are tested, and a failing 9-point block is
                              evaluated word by word.  The image and the in-window, dropped
                              and FP64-word counters are those of the per-word render on the
                              same prefix/suffix split (the margin exceeds the per-word
                              rounding error); KL_CNT_ATOMICS differs.  The split differs from
                              the per-word default (suffixes of d-1 letters up to 9, then
                              d/2+1, at most 12), so kl_workspace_bytes depends on this
                              field. */
  uint32_t shard_index;    /* Sharded render, one process per GPU: kl_render (and
                              kl_render_noalloc) with shard_count = n > 1 draws only the
                              words of shard shard_index (0 .. n-1): those whose prefix
                              slot r lies in [floor(k np / n), floor((k+1) np / n)), k =
                              shard_index, np = 3^(p-1), p = the render's prefix length
                              (prefix_len, or the length the render chooses for 0).  The
                              prefix slot of a word w_1 .. w_d is r = the base-3 ranks of
                              w_{p-1}, ..., w_1, most significant first, each among the
                              three letters other than the inverse of its right
                              neighbour.  Every word of a prefix slot is in the same shard,
                              so the n shards partition the words, with 4 * 3^(d-p) times
                              the shard's slot count each (equal to within one slot); each
                              shard's image and counters are exactly the part of the whole
                              render that its words make, so the element-wise sums (uint32,
                              modulo 2^32) of the n shards' images and counters are the
                              whole render's.  Limit-set mode only; kl_eval_words ignores
                              the shard fields; batches and the level-of-detail calls
                              return KL_EINVAL for shard_count > 1.  The paper's loop is
                              one index range on one machine; independent index ranges
                              are what makes this split possible (Sec. "The revised
                              deterministic approach": the words are in the integers). */
  uint32_t shard_count;    /* 0 or 1: the whole render (default); n > 1: n shards, with
                              shard_index < n (else KL_EINVAL) */
} kl_params;

/* Counters written by kl_render (uint64 each). */
enum {
  KL_CNT_IN_WINDOW = 0,    /* words drawn into the image */
  KL_CNT_DROPPED = 1,      /* words outside the window or non-finite */
  KL_CNT_FP64_WORDS = 2,   /* KL_MIXED, KL_DF64: words evaluated on the FP64 path */
  KL_CNT_ATOMICS = 3,      /* image atomics issued (after run-length merging) */
  KL_N_COUNTERS = 4
};

/* Human-readable name of a status code (static string). */
KL_API const char* kl_status_string(int status);

/* Number of reduced words of length `depth`: 4 * 3^(depth-1); 0 when depth is
 * 0 or above KL_MAX_DEPTH.  Sec. "Once-punctured torus groups": the pruned tree
 * drops the children aA, Aa, bB, Bb, leaving three children per node. */
KL_API uint64_t kl_word_count(uint32_t depth);

/* Grandma's two-generator recipe (Mumford, Series, Wright, "Indra's Pearls",
 * ch. 8; the paper cites the book for its groups): from tr a = ta and
 * tr b = tb it builds a, b of determinant one with tr(a b a^-1 b^-1) = -2, and
 * A, B as their inverses.  gens_out: 32 doubles (host).  Returns KL_EINVAL on a
 * null pointer or non-finite trace, KL_EDEGENERATE if a denominator of the
 * recipe vanishes.  Host only; needs no GPU. */
KL_API int kl_grandma(double ta_re, double ta_im, double tb_re, double tb_im, double* gens_out);

/* Seeds: the attracting fixed point of each generator (the orbit of a word
 * starts at the fixed point of its first-applied letter; Sec. "Implementation"
 * feeds fixed points as orbit starts).  Ties between the two fixed points
 * (parabolic maps) take ((p - s) + sqrt((p - s)^2 + 4 q r)) / (2 r).  gens: 32
 * doubles, seeds_out: 8 doubles (host).  KL_EDEGENERATE if a generator has no
 * attracting finite fixed point.  Host only. */
KL_API int kl_seeds(const double* gens, double* seeds_out);

/* Maskit's slice (the once-punctured torus groups with b parabolic): a(z) =
 * mu + 1/z, b(z) = z + 2, written as matrices of determinant one, and their
 * inverses, into gens_out (32 doubles); tr(a b A B) = -2 for every mu.  The
 * group of the paper's example is mu = -0.097 + 1.838 i.  seeds_out (8
 * doubles): the attracting fixed points of a and A; b and B fix only
 * infinity, so they get the fixed point of the parabolic commutator a b A B,
 * a finite limit point.  Host only.  KL_EDEGENERATE if a fixed point is not
 * finite. */
KL_API int kl_maskit(double mu_re, double mu_im, double* gens_out, double* seeds_out);

/* Seed list for multi-seed feeding (Sec. "Implementation" loops the scan
 * over a list of fixed points that the paper does not print): 8 points into
 * seeds_out (16 doubles): the attracting fixed points of a, b, A, B (as
 * kl_seeds), then the fixed points of the commutator a b A B and of its
 * cyclic permutations b A B a, A B a b, B a b A, parabolic maps whose fixed
 * points are the cusps of the limit set.  A multi-seed render draws every
 * word once per point: kl_render with all four seeds set to that point,
 * accumulating over the list.  Host only.  KL_EDEGENERATE if a point is not
 * finite. */
KL_API int kl_cusp_seeds(const double* gens, double* seeds_out);

/* Fill *p: generators and seeds from the traces, the given depth, image and
 * window, and defaults for the rest (precision KL_FP64, renorm_every 8,
 * parabolic_tol 1e-6, prefix_len 0, accumulate 0).  Host only. */
KL_API int kl_params_init(kl_params* p, double ta_re, double ta_im, double tb_re, double tb_im,
                   uint32_t depth, uint32_t width, uint32_t height,
                   double x0, double x1, double y0, double y1);

/* Index decode (Sec. "The revised deterministic approach": words are pulled
 * out of integers instead of being stored).  For each of the n indices in
 * d_index, writes its `depth` letter codes to d_letters[t*depth .. t*depth +
 * depth - 1] (w_1 first).  An index >= N_depth gets letters 0xFF.  Device
 * pointers; asynchronous on `stream`. */
KL_API int kl_decode_words(uint32_t depth, const uint64_t* d_index, uint64_t n, uint8_t* d_letters,
                    void* stream);

/* Bytes of device workspace kl_render and kl_eval_words need for *p
 * (prefix-matrix and suffix-point tables; in KL_TILING mode the largest
 * over the lengths 1 .. d).  0 on invalid parameters. */
KL_API size_t kl_workspace_bytes(const kl_params* p);

/* Word values, computed with exactly the arithmetic kl_render uses for *p (its
 * precision, prefix length and tables), returned as pixel coordinates:
 * d_uv[2t] = (Re z - x0) * sx, d_uv[2t+1] = (y1 - Im z) * sy (so that the pixel is
 * (floor(d_uv[2t+1]), floor(d_uv[2t])) when inside).  Non-finite values are
 * returned as NaN; an index >= N_d gives NaN.  d_workspace: at least
 * kl_workspace_bytes(p) bytes, 256-byte aligned; it is overwritten.  Sec.
 * "Introduction" (word value = last orbit element). */
KL_API int kl_eval_words(const kl_params* p, const uint64_t* d_index, uint64_t n, double* d_uv,
                  void* d_workspace, size_t workspace_bytes, void* stream);

/* Render: every reduced word of length p->depth is decoded from its index,
 * evaluated and counted into the pixel it falls in (Sec. "Implementation",
 * "limit set" mode: words of length exactly d).  In KL_TILING mode the words
 * of every length 1 .. d are drawn, each length as a render of its own into
 * the same image and counters (the prefix length field applies to length d;
 * shorter lengths choose their own).  d_image: width*height uint32,
 * row-major, row 0 at y1; counts wrap modulo 2^32.  d_counters: KL_N_COUNTERS
 * uint64 (may be NULL).  Unless p->accumulate, the image and counters are
 * zeroed first (on `stream`).  d_workspace as for kl_eval_words.  Words whose
 * value is outside the window or not finite are dropped and counted. */
KL_API int kl_render(const kl_params* p, uint32_t* d_image, uint64_t* d_counters, void* d_workspace,
              size_t workspace_bytes, void* stream);

/* Multi-seed feeding (Sec. "Implementation": the drawing loop runs over a list
 * of fixed points): every word of *p drawn once per point, i.e. the render of
 * *p with all four seeds set to points[2i] + i points[2i+1], for i = 0 ..
 * n_points - 1, into one image and one set of counters (zeroed first unless
 * p->accumulate; the counters add up to n_points N_d).  The points' renders
 * differ only in their suffix tables, so the prefix tables are built once
 * (limit-set mode; a KL_TILING render shares them per point across its
 * lengths).  kl_cusp_seeds gives the paper's list; its last four points are
 * the repetend points of the cusps.  points: host array of 2 n_points
 * doubles.  KL_EINVAL if n_points is 0 or a point is not finite; otherwise
 * the arguments and errors of kl_render. */
KL_API int kl_render_multiseed(const kl_params* p, const double* points, uint32_t n_points,
                               uint32_t* d_image, uint64_t* d_counters, void* d_workspace,
                               size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Batched render: a sweep over many groups in one persistent launch.
 *
 * n_groups parameter sets with their own traces/generators, seeds, depth and
 * prefix_len, sharing precision, cull, image size, window, renorm_every,
 * parabolic_tol and the tuning knobs of params[0].  Every group's words are
 * rendered exactly as kl_render would render them, into its own image (with
 * cull = 1, a culled batch: one persistent launch of the culling over all
 * groups, each image that of the group's culled kl_render):
 * d_images holds n_groups images of width*height uint32, group k at offset
 * k*width*height; d_counters holds n_groups * KL_N_COUNTERS uint64.  All
 * groups' work items share one device queue (FP64 fallback items first), so
 * groups of uneven depth balance across the GPU in a single launch of the
 * render kernel.  Images and counters are zeroed by each render (accumulate
 * is ignored).
 *
 * A kl_batch is a host-side handle (it owns host memory and, after
 * kl_batch_capture, a CUDA graph); all device memory is the caller's.
 */
typedef struct kl_batch kl_batch;

/* Validate the parameter sets and plan the batch on the current device.
 * *out receives a handle to free with kl_batch_destroy.  KL_EINVAL if the sets
 * do not share precision, cull, image size and window, or a set has cull > 1;
 * other codes as kl_render. */
KL_API int kl_batch_create(const kl_params* params, uint32_t n_groups, kl_batch** out);

/* Device workspace bytes the batch needs (256-byte aligned), 0 on a null handle. */
KL_API size_t kl_batch_workspace_bytes(const kl_batch* b);

/* Enqueue the whole batch on `stream`: upload of the group descriptors (from
 * host memory owned by the handle), zeroing, the table passes and the one
 * persistent render launch. */
KL_API int kl_batch_render(kl_batch* b, uint32_t* d_images, uint64_t* d_counters,
                           void* d_workspace, size_t workspace_bytes, void* stream);

/* Capture the batch into a CUDA graph held by the handle (the descriptors are
 * uploaded first, outside the graph; the graph holds the zeroing, the table
 * passes and the render launch).  The buffers must stay valid while the graph
 * is replayed.  `stream` must not be capturing already. */
KL_API int kl_batch_capture(kl_batch* b, uint32_t* d_images, uint64_t* d_counters,
                            void* d_workspace, size_t workspace_bytes, void* stream);

/* Launch the captured graph on `stream`.  KL_EINVAL if nothing was captured. */
KL_API int kl_batch_replay(kl_batch* b, void* stream);

/* Free the handle and its graph (after the work using it has finished). */
KL_API void kl_batch_destroy(kl_batch* b);

/* ---------------------------------------------------------------------------
 * Level-of-detail network.  The paper's closing remark is that both rendering
 * approaches need tricks to be accelerated (Sec. "Conclusions"); this library's
 * trick is a small MLP that reads a prefix's normalised matrix and predicts how
 * many more letters its subtree needs before its image falls into a single
 * pixel, so that the enumeration can stop early (kl_render_lod).
 *
 * Model: 8 -> 64 -> 64 -> 1, ReLU after both hidden layers, BF16 weights and
 * activations on the tensor cores with FP32 accumulation.  Parameters: one
 * FP32 vector of KL_MLP_NPARAMS floats,
 *   W1 [8][64] | b1 [64] | W2 [64][64] | b2 [64] | w3 [64] | b3
 * with h_out = sum_in x_in W[in][out] + b_out.  Inputs x: [n][8] FP32 rows.
 */
#define KL_MLP_NPARAMS 4801

/* y[i] = MLP(x[i]) for n rows (device pointers). */
KL_API int kl_mlp_forward(const float* d_params, const float* d_x, uint64_t n, float* d_y,
                          void* stream);

/* Scratch bytes kl_mlp_grad needs for n rows. */
KL_API size_t kl_mlp_scratch_bytes(uint64_t n);

/* Loss and gradient of the weighted mean squared error over n rows with
 * targets t: *d_loss = mean w_i (y_i - t_i)^2 with w_i = under_weight where
 * y_i < t_i and 1 elsewhere (under_weight > 1 penalises predicting too few
 * levels, the direction that prunes too early); d_grad = its gradient
 * (KL_MLP_NPARAMS floats, same layout as the parameters).  Both are
 * overwritten.  The partial sums are added in a fixed order (no floating-
 * point atomics), so equal inputs give bit-identical results on one GPU
 * model. */
KL_API int kl_mlp_grad(const float* d_params, const float* d_x, const float* d_t, uint64_t n,
                       float under_weight, float* d_grad, float* d_loss, void* d_scratch,
                       size_t scratch_bytes, void* stream);

/* One Adam step (Kingma and Ba, 2015) with bias correction for `step` >= 1,
 * then d_grad is zeroed.  d_m, d_v: first and second moments (start at 0). */
KL_API int kl_mlp_adam(float* d_params, float* d_m, float* d_v, float* d_grad, uint32_t step,
                       float lr, float beta1, float beta2, float eps, void* stream);

/* One training step: the gradient of kl_mlp_grad, then, in the same pass that
 * sums the partials (in the same fixed order), the Adam step of kl_mlp_adam
 * applied to d_params, d_m and d_v.  The parameters that result are bit for bit
 * those of kl_mlp_grad followed by kl_mlp_adam, one launch fewer.  d_loss: the
 * loss before the step; d_grad: receives the gradient if not null.  d_scratch
 * as for kl_mlp_grad. */
KL_API int kl_mlp_train_step(float* d_params, float* d_m, float* d_v, const float* d_x,
                             const float* d_t, uint64_t n, float under_weight, uint32_t step,
                             float lr, float beta1, float beta2, float eps, float* d_loss,
                             float* d_grad, void* d_scratch, size_t scratch_bytes, void* stream);

/* Self-test of the bounded waits the tensor-core kernels use (their MMA
 * completions are waited for on an mbarrier, for at most about a second; on
 * a timeout a kernel marks its results and returns instead of hanging).  One
 * warp waits on an mbarrier that nothing completes, for at most limit_cycles
 * clock cycles, then on one it completes itself.  d_result (4 uint32, device):
 * [0] 1 if the first wait gave up, [1] 1 if the second completed, [2] the
 * cycles the first wait took, capped at 2^32 - 1, [3] 0.  KL_EINVAL if
 * limit_cycles is 0 or above 2^31. */
KL_API int kl_wait_selftest(uint64_t limit_cycles, uint32_t* d_result, void* stream);

/* Level-of-detail labels and pruned render.
 *
 * Tree levels: a node at level k is a reduced prefix w_1 .. w_k (the letters
 * applied last), numbered by its prefix slot: x = w_k, then the base-3 ranks
 * of w_{k-1} .. w_1 (each among the letters other than the inverse of its
 * right neighbour), most significant first: slot = x 3^(k-1) + r.  Its
 * subtree is its 3^(d-k) words of length d (Sec. "Basic setup": the tree of
 * words; the pruned tree of Sec. "Once-punctured torus groups").
 * A node is resolved when the image of its subtree falls under one pixel
 * (its words' bounding box narrower and lower than `extent` pixels, 1 by
 * default), or no word falls inside the window.  Its label is 0 if resolved, else
 * 1 + the largest label of its three children; at the deepest level hi an
 * unresolved node has label 1.  Node arrays list levels lo..hi in order, each
 * level in slot order (kl_lod_node_count(lo, hi) nodes).
 * Requirements: 1 <= lo <= hi < depth, hi <= 15, depth - hi <= 9. */
KL_API uint64_t kl_lod_node_count(uint32_t lo, uint32_t hi);

/* Workspace bytes of kl_lod_labels (0 on invalid arguments). */
KL_API size_t kl_lod_label_bytes(const kl_params* p, uint32_t lo, uint32_t hi);

/* Exact render of *p (into d_image, d_counters as kl_render, prefix length
 * hi) and, from the same pass, the labels (uint8) and the network input
 * features (8 FP32 per node) of every node of levels lo..hi.  Features: the
 * prefix matrix (a product of generators of determinant one, so already of
 * determinant one up to rounding: the division by the principal square root
 * of its determinant changes no feature and is left out), negated if needed
 * so that Re tr > 0, then sign(v) log(1 + |v|) of the real and imaginary
 * parts of p, q, r, s. */
KL_API int kl_lod_labels(const kl_params* p, uint32_t lo, uint32_t hi, float extent,
                         uint32_t* d_image, uint64_t* d_counters, float* d_features,
                         uint8_t* d_labels, void* d_workspace, size_t workspace_bytes,
                         void* stream);

/* Workspace bytes of kl_render_lod (0 on invalid arguments). */
KL_API size_t kl_lod_render_bytes(const kl_params* p, uint32_t lo, uint32_t hi);

/* Render with the network pruning the enumeration (p->precision must be
 * KL_MIXED).  From level lo to hi each active node is scored by the network
 * (d_mlp: KL_MLP_NPARAMS floats).  A node with score + margin < 1/2 whose
 * first, middle and last words in index order (the words taking the allowed
 * letter of rank 0, 1, 2 at every step) fall into one pixel, each at least
 * `edge` pixels from that pixel's sides, adds all 3^(d-k) words of its
 * subtree to that pixel (all three at least `edge` outside the window: counts
 * them dropped); the others expand; nodes still active at level hi are
 * rendered exactly.  With edge = the label extent the network was trained
 * for (kl_lod_labels), a right prediction keeps every word in its own pixel.
 * Every word is counted once (in d_counters, as kl_render).  d_stats (4
 * uint64): nodes scored, nodes pruned, level-hi nodes rendered exactly, 0.
 * The scores come from the same tensor-core forward pass as kl_mlp_forward,
 * 128 nodes per tile; if a tensor-core wait runs out (bounded at about a
 * second), the affected scores are NaN, which prunes nothing, so those nodes
 * are still drawn exactly.  KL_EINVAL unless 0 <= edge < 1/2. */
KL_API int kl_render_lod(const kl_params* p, uint32_t lo, uint32_t hi, const float* d_mlp,
                         float margin, float edge, uint32_t* d_image, uint64_t* d_counters,
                         uint64_t* d_stats, void* d_workspace, size_t workspace_bytes,
                         void* stream);

/* As kl_render_lod, with the true labels of kl_lod_labels (same p, lo, hi)
 * taking the network's place: a node is pruned when its label is 0 and the
 * edge test passes.  It measures what the pruned render loses by its splat
 * alone, separately from the network's errors. */
KL_API int kl_render_lod_labels(const kl_params* p, uint32_t lo, uint32_t hi,
                                const uint8_t* d_labels, float edge, uint32_t* d_image,
                                uint64_t* d_counters, uint64_t* d_stats, void* d_workspace,
                                size_t workspace_bytes, void* stream);

/* General presentations (Sec. "Cayley Multiplication Tables" and Sec.
 * "Implementation"): the paper's own enumeration, for any group given by an
 * indexed Cayley table.  Every index n in [0, m^d) of the unpruned m-ary tree
 * is written as d base-m digits, each plus one (symbols 1..m; 0 is the
 * identity), the first digit most significant; the string is kept when the
 * run of the table over it, read right to left from state 0, never reaches
 * the crash state 0.  A kept string w_1 .. w_d (letter = symbol - 1) is drawn
 * at its word value: the seed of w_d, then the maps of w_d, ..., w_1. */
#define KL_FSA_MAX_LETTERS 9
#define KL_FSA_WORKSPACE_BYTES 256u

typedef struct {
  uint32_t m;   /* letters (symbols 1..m), 1 .. KL_FSA_MAX_LETTERS */
  uint8_t table[(KL_FSA_MAX_LETTERS + 1) * (KL_FSA_MAX_LETTERS + 1)];
                /* indexed table, row-major with row stride KL_FSA_MAX_LETTERS + 1:
                   table[state * 10 + symbol] = next state (0..m, 0 = crash) for
                   states and symbols 0..m; the run starts in state 0 */
  double gens[KL_FSA_MAX_LETTERS * 8];  /* letter k's matrix (p, q, r, s as re, im) */
  double seeds[KL_FSA_MAX_LETTERS * 2]; /* seed point of each first-applied letter */
} kl_fsa;

/* Strings of length `depth` kept by the table run (host only, no GPU):
 * counted by the states of the run, not by scanning.  KL_ERANGE unless
 * 1 <= depth <= 32 and m^depth <= 2^40; KL_EINVAL on a table entry > m. */
KL_API int kl_fsa_count(const kl_fsa* f, uint32_t depth, uint64_t* count);

/* Render of the kept strings of depth p->depth with the view, image size and
 * accumulate flag of *p (its gens, seeds and mode are not used; precision
 * must be KL_FP64).  Counters as kl_render (KL_CNT_FP64_WORDS = kept words).
 * d_workspace: at least KL_FSA_WORKSPACE_BYTES, 256-byte aligned. */
KL_API int kl_render_fsa(const kl_fsa* f, const kl_params* p, uint32_t* d_image,
                         uint64_t* d_counters, void* d_workspace, size_t workspace_bytes,
                         void* stream);

/* Size of the library's own device scratch array used by kl_render_noalloc. */
#define KL_STATIC_SCRATCH_BYTES (32u << 20)

/* kl_render for callers that cannot allocate device memory: the same render,
 * with the prefix and suffix tables placed in a scratch array compiled into
 * the library instead of a caller-provided workspace.  Some callers cannot call
 * cudaMalloc at render time: code embedded in a host application that owns
 * the whole device heap through its own pool, or a render loop that must run
 * within a fixed device-memory budget and cannot risk an allocation failure
 * mid-frame.  They pass only the image and the counters.
 * There is no counterpart of this call in the paper.
 *  - The scratch array holds KL_STATIC_SCRATCH_BYTES (32 MiB) on every GPU that
 *    loads the library, until the process exits, whether or not this call is
 *    used.  A request whose kl_workspace_bytes(p) exceeds it returns
 *    KL_ENOSPACE before anything is enqueued.
 *  - Every call whose stream is not capturing looks up the array's device
 *    address with the calling device current (cudaGetSymbolAddress, which
 *    allocates nothing), so the address always belongs to the current
 *    context, also after a device reset.  A call on a capturing stream uses
 *    the address the last uncaptured call on that device found, and returns
 *    KL_EINVAL if there was none: make one uncaptured call on each device
 *    before any stream capture.
 *  - All calls share the one array, which keeps the last call's tables; the
 *    render rebuilds and re-zeroes what it needs on every call.  Calls that
 *    overlap on the GPU (concurrent streams, or several host threads) race on
 *    the array and give wrong images: serialise them.
 *  - Neither this call nor anything it calls allocates or frees memory. */
KL_API int kl_render_noalloc(const kl_params* p, uint32_t* d_image, uint64_t* d_counters,
                             void* stream);

/* Instrumentation: when set, kl_render records the CUDA events ev_start and
 * ev_stop (cudaEvent_t, created by the caller) on its stream immediately
 * before and after its main per-word kernel (the FP64 or mixed render
 * kernel), so that the caller can time that kernel alone with
 * cudaEventElapsedTime.  NULL, NULL switches it off.  The setting belongs to
 * the calling host thread and applies to every following kl_render call made
 * from that thread (other threads are not affected).  This is an
 * addition of this library (the paper reports no timings); it changes no
 * result. */
KL_API int kl_set_profile_events(void* ev_start, void* ev_stop);

#ifdef __cplusplus
}
#endif

#endif /* KL_H */
