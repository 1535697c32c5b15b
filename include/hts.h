/*
 * hts.h -- C ABI of libhts: the per-iteration gradient of hyperbolic t-SNE
 * ("Accelerating hyperbolic t-SNE", arXiv 2401.13708) on one NVIDIA GB300.
 *
 * One context holds one embedding problem on one device: the sparse
 * symmetric affinity matrix P (CSR), the embedding Y in the Poincare disk
 * (n x 2, float64 master copy), the optimiser state (velocity, gains) and
 * all device work buffers.  Every iteration runs on the device:
 *
 *   polar keys -> radix sort -> polar-quadtree build (Sec. 4.1)
 *   -> attractive sum over P      (first sum of Eq. KlGradientHyperbolicSplit)
 *   -> Barnes-Hut repulsion + Z   (second sum, Eq. CellApproximation, Sec. 4.2)
 *   -> gradient and Riemannian step (Eq. PoincareMetric rescale, exp map,
 *      Eq. HyperbolicProjection; momentum / exaggeration of Sec. 5.1)
 *
 * Conventions
 *   - Return value: HTS_OK (0) or a negative HTS_E* code.  No C++ exception
 *     or process exit crosses this boundary.  hts_last_error() gives a
 *     human-readable message for the last failing call on a context.
 *   - Ownership: inputs are copied into the context; the caller keeps its
 *     buffers and may free them after the call returns.  Outputs are written
 *     into caller buffers.  `where` says whether a pointer is host memory
 *     (HTS_HOST) or device memory of the context's device (HTS_DEVICE).
 *     Host buffers may be pageable or pinned.
 *   - Streams: all work is queued on the stream given in hts_config (NULL =
 *     the legacy default stream).  Calls that return data to the host
 *     (host outputs, hts_kl, Z_out) synchronise that stream before returning;
 *     device outputs are ready in stream order.
 *   - Layout: y and gradients are n x 2 row-major float64 (x0, y0, x1, y1, ...).
 *     CSR: indptr int64[n+1] (indptr[0] = 0, non-decreasing, indptr[n] = nnz),
 *     indices int32[nnz] in [0, n), no diagonal entries; values float32 or
 *     float64[nnz], finite and >= 0.  P is used as given (the caller
 *     symmetrises and normalises it, Eq. HighDimensionalProbability).
 *   - Threads: a context is not thread-safe; use one context per thread.
 *   - theta == 0 means "no approximation" (Sec. 5.2.3): the exact O(n^2)
 *     repulsion kernel replaces the tree walk.
 */
#ifndef HTS_H
#define HTS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HTS_API __attribute__((visibility("default")))
#else
#define HTS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define HTS_OK 0
#define HTS_EINVAL (-1)   /* invalid argument: NULL pointer, unknown enum, bad theta/lr */
#define HTS_ESHAPE (-2)   /* inconsistent sizes: n mismatch between P and Y, malformed CSR */
#define HTS_ENOTSET (-3)  /* P or Y has not been set on this context */
#define HTS_EDOMAIN (-4)  /* a point with |y| >= 1 or a non-finite coordinate/value */
#define HTS_ECUDA (-5)    /* a CUDA runtime call failed (message has the CUDA error) */
#define HTS_EOOM (-6)     /* device allocation failed */
#define HTS_ENUMERIC (-7) /* device check tripped: non-finite gradient/position or tree overflow */
#define HTS_ETIMEOUT (-9) /* a bounded device-side wait gave up (the results of that call are invalid;
                             the context stays usable) */

/* ---- enums ------------------------------------------------------------ */
#define HTS_FP64 0        /* every step in float64 */
#define HTS_FP32_MIXED 1  /* pair forces in float32 (hi/lo point pairs, conformal
                             factors from float64); Z, sums and the step in float64 */

#define HTS_EQUAL_LENGTH 0 /* radial split at (max_r + min_r)/2, Eq. EqualEmbeddingLengthsSplitting */
#define HTS_EQUAL_AREA 1   /* radial split at acosh((cosh max + cosh min)/2), Eq. EqualAreaSplitting */

#define HTS_EXACT_KL 0     /* gradient 4 sum (p - q) w d dd/dy: the derivative of KL */
#define HTS_PAPER_EQ 1     /* the form printed in Eq. KLGradientHyperbolic (without d) */

#define HTS_HOST 0
#define HTS_DEVICE 1

#define HTS_F32 0
#define HTS_F64 1

#define HTS_TREE_LEVELS 29 /* depth cap of the polar quadtree (29 radial + 29 angular key bits) */

typedef struct hts_ctx hts_ctx;

typedef struct {
    int precision;   /* HTS_FP64 | HTS_FP32_MIXED (default HTS_FP32_MIXED) */
    int split_rule;  /* HTS_EQUAL_LENGTH (default) | HTS_EQUAL_AREA */
    int grad_form;   /* HTS_EXACT_KL (default) | HTS_PAPER_EQ */
    int metric_pow;  /* step rescale lambda^-metric_pow: 1 (default, "product of lambda^-1
                        with the variation", Sec. 4.2) or 2 (Riemannian gradient) */
    double eps;      /* projection margin of Eq. HyperbolicProjection: points that reach
                        |y| >= 1 - eps/2 are put back at radius 1 - eps (default 1e-5) */
    int use_gains;   /* per-coordinate gains (Sec. 5.1): +0.2 on sign disagreement of
                        gradient and velocity, *0.8 otherwise, floor 0.01 (default 0) */
    int device;      /* CUDA device ordinal (default 0) */
    void *stream;    /* cudaStream_t to queue work on (default NULL) */
} hts_config;

/* Fill *cfg with the defaults listed above.  Never fails. */
HTS_API void hts_default_config(hts_config *cfg);

/* Create a context on cfg->device.  *out receives the handle (NULL on error).
 * Allocates only host memory; device buffers are allocated by hts_set_P /
 * hts_set_Y.  Errors: HTS_EINVAL (NULL out, bad enum, eps not in (0, 0.5)),
 * HTS_ECUDA (device not usable). */
HTS_API int hts_create(hts_ctx **out, const hts_config *cfg);

/* Free every buffer of the context.  NULL is ignored. */
HTS_API void hts_destroy(hts_ctx *ctx);

/* Copy the affinity matrix P (n x n, CSR, see Conventions) into the context.
 * dtype HTS_F32 | HTS_F64; in HTS_FP32_MIXED the values are kept as float32,
 * in HTS_FP64 as float64.  Host inputs are validated (monotone indptr,
 * indices in range and off-diagonal, finite non-negative values); device
 * inputs are validated on the device.  After an error past the argument
 * checks the context holds no P until the next successful call.  Errors:
 * HTS_EINVAL, HTS_ESHAPE (bad CSR or n differs from a Y already set),
 * HTS_EDOMAIN (bad values), HTS_EOOM, HTS_ECUDA. */
HTS_API int hts_set_P(hts_ctx *ctx, int64_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
              const void *values, int dtype, int where);

/* Copy the embedding Y (n x 2 float64) into the context and reset the
 * velocity to 0 and the gains to 1.  Every point must satisfy |y| < 1 and be
 * finite; this is checked on the device after the copy (host and device
 * inputs alike), and the call returns once the copy is complete.  On
 * HTS_EDOMAIN the context holds no Y until the next successful call.
 * Errors: HTS_EINVAL, HTS_ESHAPE (n differs from P), HTS_EDOMAIN, HTS_EOOM,
 * HTS_ECUDA. */
HTS_API int hts_set_Y(hts_ctx *ctx, int64_t n, const double *y, int where);

/* Overwrite the positions of the current Y (n x 2 float64, the n already
 * set) and keep the optimiser state -- velocity, gains, iteration count --
 * for a caller that holds Y in its own memory between steps or edits it
 * (re-centring, constraints).  Checked on the device like hts_set_Y; returns
 * once the copy is complete.  Errors: HTS_EINVAL, HTS_ENOTSET (no Y yet),
 * HTS_EDOMAIN (then the context holds no Y), HTS_ECUDA. */
HTS_API int hts_update_Y(hts_ctx *ctx, const double *y, int where);

/* Run n_iter gradient-descent iterations (Sec. 5.1): each builds the tree
 * from the current Y, computes g = 4 (exaggeration * F_attr - F_rep / Z) with
 * the Barnes-Hut repulsion at `theta` (exact when theta == 0), and updates
 *   v <- momentum * v - lr * gains * lambda^-metric_pow * g,
 *   y <- proj(exp_y(v)).
 * theta in [0, 1], exaggeration > 0, lr >= 0, momentum in [0, 1].
 * Synchronises once at the end to read the device status word.
 * Errors: HTS_ENOTSET, HTS_EINVAL, HTS_ENUMERIC, HTS_ECUDA. */
HTS_API int hts_step(hts_ctx *ctx, int n_iter, double theta, double exaggeration, double lr, double momentum);

/* Copy Y (n x 2 float64) out.  Errors: HTS_ENOTSET, HTS_EINVAL, HTS_ECUDA. */
HTS_API int hts_get_Y(hts_ctx *ctx, double *y_out, int where);

/* Euclidean gradient of KL at the current Y (no step, no rescale):
 * g = 4 (exaggeration * F_attr - F_rep / Z), the split form of Eq.
 * KlGradientHyperbolicSplit, with Z the Barnes-Hut (theta > 0) or exact
 * (theta == 0) normalisation.  g_out (n x 2, may be NULL) in `where`
 * memory; Z_out (host double, may be NULL).  Errors: HTS_ENOTSET,
 * HTS_EINVAL, HTS_ENUMERIC, HTS_ECUDA. */
HTS_API int hts_grad(hts_ctx *ctx, double theta, double exaggeration, double *g_out, double *Z_out, int where);

/* KL(P || Q^H) at the current Y (Eq. KLDivergence with the hyperbolic q of
 * Eq. LowDimensionalProbabilityHyperbolic), without exaggeration:
 *   sum p log p - sum p log w + (sum p) log Z,
 * Z from the tree (theta > 0) or exact (theta == 0).  *kl_out is a host
 * double.  Errors: HTS_ENOTSET, HTS_EINVAL, HTS_ECUDA. */
HTS_API int hts_kl(hts_ctx *ctx, double theta, double *kl_out);

/* Message for the last failing call on ctx ("" if none; a static string
 * when ctx is NULL).  Valid until the next call on ctx. */
HTS_API const char *hts_last_error(const hts_ctx *ctx);

/* ---- inspection and checkpointing ---------------------------------------- */

/* Polar keys (Sec. 4.1, reading R5) of the current Y in point order:
 * digit l (l = 1 most significant, bits 2(29-l)+1..2(29-l)) is
 * 2 * radial_bit + angular_bit of the depth-l cell.  keys_out: uint64[n];
 * bounds_out (host double[2], may be NULL): the root annulus [lo, hi] in the
 * radial split coordinate.  Errors: HTS_ENOTSET, HTS_EINVAL, HTS_ECUDA. */
HTS_API int hts_get_keys(hts_ctx *ctx, uint64_t *keys_out, double *bounds_out, int where);

/* Build the tree for the current Y and export its nodes in pre-order
 * (children in key order, chains of one-child cells collapsed to the
 * deepest cell).  Call with cap = 0 (arrays may be NULL) to get the node
 * count in *count_out; then with cap >= count.  Arrays are host memory:
 * depth int32[cap], prefix uint64[cap] (top 2*depth key bits), count
 * int64[cap] (N_cell), first int64[cap] (point index of a single-point leaf,
 * smallest point index of a depth-29 bucket, -1 for internal cells), ycell
 * double[2*cap] (Einstein midpoint of Eq. EinsteinMidpoint in disk
 * coordinates, or the point), rcell double[cap] (longest internal distance
 * of the cell, +inf for the root and for single-point leaves).
 * Errors: HTS_ENOTSET, HTS_EINVAL (cap too small), HTS_ECUDA. */
HTS_API int hts_get_tree(hts_ctx *ctx, int64_t cap, int64_t *count_out, int32_t *depth, uint64_t *prefix,
                 int64_t *count, int64_t *first, double *ycell, double *rcell);

/* Counters (host int64[5]): [0..3] summed over the tree walks run while
 * counting is on -- accepted cells, leaf pair interactions, warp node
 * visits, query points (the walk then runs a counting variant; switching
 * counting on resets them); [4] the number of CUDA kernels this context
 * has launched. */
HTS_API int hts_get_counters(hts_ctx *ctx, int64_t *out5);
HTS_API int hts_set_counters(hts_ctx *ctx, int enable);

/* Acceptance tests of Sec. 4.2 (r_cell / d < theta at an internal cell)
 * made by the counted walks, one per (query point, cell) pair the walk
 * reached with the point still open -- the criterion work itself, where
 * warp node visits (hts_get_counters [2]) also count the lanes of a warp
 * that had already accepted an ancestor.  Reset with the other counters.
 * *out: host int64.  Errors: HTS_EINVAL, HTS_ECUDA. */
HTS_API int hts_get_criterion_count(hts_ctx *ctx, int64_t *out);

/* Per-phase timing.  While profiling is on, hts_step records CUDA events at
 * the phase boundaries of every iteration (up to 4096 per call).
 * hts_get_profile returns the accumulated milliseconds of the six phases --
 * keys, sort, tree build, tree walk (or exact kernel), attractive sum, Z +
 * update -- and the number of iterations they cover, then resets them.
 * enable = 1 times the iteration as it normally runs (the attractive sum
 * overlapped on its side stream, so its interval spans the stages it shares
 * the GPU with); enable = 2 runs the attractive sum on the main stream
 * between the walk and the Z reduction, so that each phase is timed alone.
 * ms6: host double[6]. */
HTS_API int hts_set_profiling(hts_ctx *ctx, int enable);
HTS_API int hts_get_profile(hts_ctx *ctx, double *ms6, int64_t *iters);

/* Optimiser state for checkpoint/resume: velocity and gains (n x 2 float64
 * each, in `where` memory) and the number of iterations run.  get: outputs
 * may be NULL.  set: NULL leaves a part unchanged; iters >= 0.  Errors:
 * HTS_ENOTSET, HTS_EINVAL (bad `where`, negative iters, or a pointer given as
 * HTS_DEVICE that is not device memory of the context's device), HTS_ECUDA. */
HTS_API int hts_get_state(hts_ctx *ctx, double *vel, double *gains, int64_t *iters, int where);
HTS_API int hts_set_state(hts_ctx *ctx, const double *vel, const double *gains, int64_t iters, int where);

/* CO-SNE objective (Sec. 4.3): lambda1 KL + lambda2 H with
 * H = (1/n) sum_i (|x_i|^2 - |y_i|^2)^2, x_i the high-dimensional points.
 * With x_sqnorm (n doubles |x_i|^2, in `where` memory) set, hts_grad and
 * hts_step use lambda1 g_KL,i - (4 lambda2 / n)(|x_i|^2 - |y_i|^2) y_i -- the
 * derivative of that cost (the variation printed in the paper has the
 * opposite sign on the second term).  x_sqnorm == NULL switches the term off.
 * hts_kl still returns KL alone.  Set Y first; a later hts_set_Y with another
 * n switches the term off.  Errors: HTS_ENOTSET, HTS_EINVAL, HTS_EDOMAIN
 * (negative or non-finite |x|^2), HTS_EOOM, HTS_ECUDA. */
HTS_API int hts_set_cosne(hts_ctx *ctx, double lambda1, double lambda2, const double *x_sqnorm, int where);

/* ---- batched embeddings ---------------------------------------------------
 * Up to HTS_MAX_SEGMENTS independent embeddings (different data sets,
 * perplexities or seeds) share one context: the n points are split into
 * nseg consecutive ranges [offsets[s], offsets[s+1]) (host int64[nseg+1],
 * offsets[0] = 0, offsets[nseg] = n, every range non-empty), and P must be
 * block diagonal (each row indexes only points of its own segment; checked
 * on the device).  Every segment gets its own root annulus and polar
 * quadtree (Sec. 4.1; the segment id is the top 6 key bits, so the trees form
 * one forest built by the same launches), its own Z, and its own learning
 * rate lr * lr_scale[s] in hts_step (lr_scale: host double[nseg], NULL = all
 * 1; the paper's lr = n_s / 12000 is lr = 1/12000 with lr_scale[s] = n_s).
 * All segments advance in the same kernel launches.  nseg = 1 restores the
 * single-embedding behaviour (lr_scale is then ignored); hts_set_Y with
 * another n resets to nseg = 1, and so does hts_set_P with another n.  With
 * segments, the CO-SNE term of hts_set_cosne uses the segment's size n_s in
 * place of n.
 * Errors (each leaves the context with nseg = 1): HTS_ENOTSET (set P and Y
 * first), HTS_EINVAL, HTS_ESHAPE (bad offsets or P not block diagonal),
 * HTS_EOOM, HTS_ECUDA. */
#define HTS_MAX_SEGMENTS 64
HTS_API int hts_set_segments(hts_ctx *ctx, int nseg, const int64_t *offsets, const double *lr_scale);

/* Per-segment Z of the last hts_grad / hts_step / hts_kl (host double[nseg]). */
HTS_API int hts_get_segment_Z(hts_ctx *ctx, double *Z_out);

/* Per-segment KL (host double[nseg]), Z from the tree (theta > 0) or exact
 * (theta == 0) within each segment.  hts_kl returns their sum. */
HTS_API int hts_kl_segments(hts_ctx *ctx, double theta, double *kl_out);

/* Replay each hts_step iteration as one CUDA graph (captured on a private
 * stream ordered after the context's stream by events; re-captured when
 * theta, exaggeration, lr, momentum or the problem changes).  Saves launch
 * overhead at small n; results are identical.  Off by default. */
HTS_API int hts_set_graphs(hts_ctx *ctx, int enable);

/* ---- launch-shape autotuner ------------------------------------------------
 * (No counterpart in the paper, whose implementation is a CPU program.)  Two
 * launch shapes of the hot path depend on the problem: the BH walk's threads
 * per block (32, 64, 128 or 256; each warp walks 32 key-adjacent points, and
 * small blocks spread a small problem over more SMs) and the float32
 * attraction's lanes per row of P (4, 8, 16 or 32; matched to the row
 * lengths).  hts_autotune builds the tree for the current Y once (theta > 0),
 * times `reps` launches of every candidate of each kernel on the context's
 * stream with CUDA events, keeps the fastest and writes the choice to
 * tuning[2] = {walk threads per block, attraction lanes per row} (may be
 * NULL); for a small problem it also picks the split walk's cut depth
 * (hts_get_walk_split).  A smaller walk block is kept only if it is 3% faster
 * than the larger ones.  It changes no result of the walk (the work split per warp does not
 * depend on the block size); lanes per row change only the float32 summation
 * order inside a row.  hts_set_tuning sets them directly (0 keeps a value),
 * hts_get_tuning reads them.  Defaults: {256, 8}.  Errors: HTS_ENOTSET,
 * HTS_EINVAL (theta outside [0, 1], reps outside [1, 1000], a value not in
 * the lists), HTS_ECUDA. */
HTS_API int hts_autotune(hts_ctx *ctx, double theta, int reps, int *tuning);

/* Split walk for small problems (one embedding; no counterpart in the
 * paper).  With few 32-point chunks the walk cannot fill the GPU, so each
 * chunk is walked by up to 4^depth warps, one per subtree of the tree cut at
 * `depth` (0..3) below the root, which is never accepted; a warp first
 * evaluates the criterion at its subtree's ancestors, and the interaction
 * with an accepted ancestor is counted by one warp only, so every point gets
 * exactly the interactions of its own walk (the partial sums are added in a
 * fixed order).  depth = -1 (default) picks the shallowest cut that gives
 * about 2048 warps, within a partial-sum buffer of
 * min(64 n, 2^22) entries for n <= 524288 (no split above).  Errors: HTS_EINVAL (depth < -1 or > 3). */
HTS_API int hts_set_walk_split(hts_ctx *ctx, int depth);
/* The cut depth in use (the automatic choice resolved; 0 with segments).
 * hts_autotune also times every depth the buffer allows on the current
 * problem and keeps the fastest.  Errors: HTS_EINVAL. */
HTS_API int hts_get_walk_split(const hts_ctx *ctx, int *depth);
HTS_API int hts_set_tuning(hts_ctx *ctx, int walk_block, int attract_lanes);
HTS_API int hts_get_tuning(const hts_ctx *ctx, int *tuning);

/* ---- roofline denominators ---------------------------------------------------
 * (No counterpart in the paper.)  Measures, on `device`, the sustained issue
 * rates that bound the hot path: out3[0] float32 FMA (TFLOP/s, 2 flop per
 * FMA), out3[1] special-function reciprocal square roots (Tops/s), out3[2]
 * float64 FMA (TFLOP/s).  Each is one ~5-10 ms kernel of independent chains
 * over 64 warps per SM.  Allocates 4 bytes of device memory for the duration.
 * Errors: HTS_EINVAL, HTS_ECUDA, HTS_EOOM. */
HTS_API int hts_measure_peaks(int device, double *out3);

/* Test of the bounded device-side waits (no counterpart in the paper).  The
 * one-sweep sort passes (problems of more than 4096 points) wait, per tile,
 * for the digit counts of earlier tiles; every such wait gives up after a
 * bounded number of polls (~0.3 s), sets a status bit and writes no key out
 * of range, so that a lost publication can never hang the GPU.  With
 * spin_limit > 0 the first tile of every pass withholds its publication and
 * the waits give up after spin_limit polls (microseconds): hts_step and
 * hts_grad then return HTS_ETIMEOUT, and the failed iteration and the rest of
 * that call leave Y, velocity and gains unchanged.  spin_limit = 0 (the
 * default) restores normal operation; the context stays usable.  For tests
 * only.  Errors: HTS_EINVAL (spin_limit outside [0, 4096]). */
HTS_API int hts_set_wait_test(hts_ctx *ctx, int spin_limit);

/* Number of points n and non-zeros nnz currently set (either may be NULL). */
HTS_API int hts_get_sizes(const hts_ctx *ctx, int64_t *n, int64_t *nnz);

/* ---- allocation-free exact gradient ---------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory: a plug-in inside a framework or inference
 * server whose own allocator owns the device memory budget (a cudaMalloc
 * behind its back can fail or starve it), or code on a latency-critical path
 * that cannot take the implicit device synchronisation of cudaMalloc and
 * cudaFree.
 *
 * hts_exact_grad_noalloc computes what hts_grad computes with theta = 0 in
 * HTS_FP64: g = 4 (exaggeration * F_attr - F_rep / Z) with the exact
 * repulsion over all pairs, and Z.  It needs no context.  Every pointer is
 * device memory of the current device: y (n x 2 float64), the CSR matrix
 * (int64 indptr[n+1], int32 indices[nnz], float64 values[nnz], laid out as
 * for hts_set_P; not validated, but out-of-range entries are skipped), g_out
 * (n x 2 float64) and Z_out (one float64, may be NULL).  Every point must lie
 * inside the open unit disk and be finite; the call does not read y back to
 * the host to check, so a point outside gives NaN in every element of g_out
 * and in *Z_out (the return value is still HTS_OK).  The work is queued on
 * `stream` (a cudaStream_t; NULL = legacy default stream) and is complete in
 * stream order; nothing is copied to the host.
 *
 * Work arrays live in one fixed file-scope device array sized for
 * HTS_NOALLOC_MAX_N points (about 4.5 MB); every device that loads the
 * library holds it until the process exits.  n > HTS_NOALLOC_MAX_N returns
 * HTS_ETOOLARGE.  No cudaMalloc, cudaFree or allocating library call is
 * made.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, which may make the driver load this library's
 * device code on that device); make that first call before any stream
 * capture.  All calls share the array; each call clears the one flag that
 * must start at zero and overwrites everything else it reads -- but calls
 * whose kernels overlap on the GPU (other streams, other host threads on the
 * same device) race on it: serialise them.
 * Errors: HTS_EINVAL (negative sizes, NULL pointers, bad grad_form or
 * exaggeration), HTS_ETOOLARGE, HTS_ECUDA (address lookup or launch failed). */
#define HTS_NOALLOC_MAX_N 65536
#define HTS_ETOOLARGE (-8) /* size beyond the fixed capacity of an allocation-free entry point */
HTS_API int hts_exact_grad_noalloc(int64_t n, int64_t nnz, const double *y, const int64_t *indptr,
                                   const int32_t *indices, const double *values, double exaggeration,
                                   int grad_form, double *g_out, double *Z_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HTS_H */
