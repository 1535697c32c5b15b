// hts_internal.cuh -- data layout, context and device helpers of libhts.
//
// Every array lives in HBM of one GB300 and is allocated once per problem
// size (hts_set_P / hts_set_Y); an iteration allocates nothing.
//
// Per point (n), original order:  y, vel, gains (double2), fattr, frep
//   (double2), zi (double), pts32 / pts64 (32-byte point records: position
//   as float hi/lo pairs or double, and il = 1 / (1 - |y|^2) taken from
//   float64), apts32 (16-byte records of the float32 attractive sum),
//   radial (double, split coordinate of the point).
// Per point, key order:  keys / idx (uint64 / uint32, sort ping-pong),
//   spts32 / spts64 (gathered records), terms (Einstein terms, 3 doubles).
// Binary radix tree over the sorted keys (n - 1 internal nodes): children,
//   parents, ranges, prefix lengths, per-point quad-level masks; exclusive
//   prefix sums of the Einstein terms over the sorted points (3 x 128-bit
//   fixed point, 48 B per point).
// Polar quadtree (<= 2n - 1 nodes), pre-order with skip indices:
//   NodeF (32 B) or NodeD (48 B).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hts.h"
#include "bits.cuh"

namespace hts {

constexpr int kLevels = HTS_TREE_LEVELS;  // 29 levels: 58 key bits
constexpr int kMaxSegments = HTS_MAX_SEGMENTS;  // segment id in the top 6 key bits
constexpr int kSegShift = 2 * kLevels;          // 58
constexpr double kTwoPi = 6.283185307179586476925286766559;

// Point record, float32 mode: position as hi + lo float pairs (the pair
// carries ~48 bits, enough to form |y_i - y_j| of nearby points near the
// rim without cancellation) and il = 1 / (1 - |y|^2) rounded from float64.
struct __align__(16) PointF {
    float xh, yh, xl, yl;
    float il, pad0, pad1, pad2;
};

// Point record of the float32 attractive sum (16 bytes: the neighbour
// gather moves half the bytes of a PointF): hi floats and il as in PointF,
// and the lo floats scaled by 2^24 and rounded to half precision, packed in
// one word (lo | hi << 16).  For |y| < 1 a lo float is at most 2^-25, so the
// packed value is at most 0.5 and the position keeps an absolute error
// below 2^-36 -- relative 1e-6 of a neighbour distance of 1e-5 at the rim.
struct __align__(16) PointA {
    float xh, yh, il;
    unsigned lo;
};

// Point record, float64 mode.
struct __align__(16) PointD {
    double x, y, il, pad;
};

// Tree node, float32 mode (one 32-byte sector; count is a float holding an
// integer, so the walk multiplies by it without a conversion).
//   count >= 2 : internal cell; (xh, yh, xl, yl) Einstein midpoint, il of the
//                midpoint, thr = cosh(r_cell / theta) - 1 (accept iff the
//                pair's delta = cosh(d) - 1 exceeds it), skip = pre-order
//                index after the subtree.
//   count == 1 : single-point leaf; the point itself, thr holds the point's
//                sorted position (int bits), skip = index + 1.
//   count <  0 : depth-29 bucket of -count points; thr holds the sorted
//                position of its first point (int bits).
struct __align__(16) NodeF {
    float xh, yh, xl, yl;
    float il, thr;
    float count;
    int skip;
};
// Empty float32 node slots the tree build writes after its last node (the
// walk visits up to three past its last node: four visits per loop test).
constexpr int kWalkOverrun = 4;

// Tree node, float64 mode (same meaning; pos = sorted position for leaves
// and buckets).
struct __align__(16) NodeD {
    double x, y, il, thr;
    int count, skip, pos, pad;
};

struct TreeExport {  // optional host-visible copy of the tree (device arrays)
    int32_t *depth;
    uint64_t *prefix;
    int64_t *count, *first;
    double *ycell, *rcell;
};

}  // namespace hts

struct hts_ctx {
    hts_config cfg;
    cudaStream_t stream = nullptr;
    // side stream for the attractive sum, which needs only the point records
    // and so overlaps the key / sort / tree / walk stages
    cudaStream_t astream = nullptr;
    cudaEvent_t aev_fork = nullptr, aev_join = nullptr;
    // hts_step runs its iterations on pstream (highest priority), ordered
    // after and before the context's stream by events; astream has the
    // lowest priority, so attraction blocks take only SM slots that the
    // key / sort / tree / walk kernels leave free
    cudaStream_t pstream = nullptr;
    cudaEvent_t pev_in = nullptr, pev_out = nullptr;
    // the tree build's two independent chains (sorted records + fixed-point
    // sums; radix tree + layout) run side by side: tstream (highest
    // priority) takes the first, forked and joined by events
    cudaStream_t tstream = nullptr;
    cudaEvent_t tev_fork = nullptr, tev_join = nullptr;
    int sm_count = 0;
    std::string err;

    int64_t n = 0, nnz = 0;
    bool have_P = false, have_Y = false;
    int64_t cap_n = 0, cap_nnz = 0;  // allocated capacities
    int values_f64 = 0;             // stored dtype of P values
    int64_t iters = 0;
    int counters_on = 0;

    // CSR
    int64_t *indptr = nullptr;
    int32_t *indices = nullptr;
    void *values = nullptr;

    // per point, original order
    double2 *y = nullptr, *vel = nullptr, *gains = nullptr, *fattr = nullptr, *frep = nullptr;
    double *zi = nullptr, *radial = nullptr;
    hts::PointF *pts32 = nullptr;
    hts::PointA *apts32 = nullptr;   // float32 attraction records
    hts::PointD *pts64 = nullptr;

    // per point, key order
    uint64_t *keys = nullptr, *keys_alt = nullptr;
    uint32_t *idx = nullptr, *idx_alt = nullptr;
    hts::PointF *spts32 = nullptr;
    hts::PointD *spts64 = nullptr;
    double *terms = nullptr;  // 3 per point

    // binary radix tree
    int *bn_left = nullptr, *bn_right = nullptr, *bn_parent = nullptr, *leaf_parent = nullptr;
    int *bn_lo = nullptr, *bn_hi = nullptr, *bn_pref = nullptr, *bn_flag = nullptr, *bn_quad = nullptr;
    double *bn_sum = nullptr;  // n + 1 prefix sums of S_gamma, S_ux, S_uy (3 x 128-bit fixed point)
    int *cnt = nullptr, *pre = nullptr;  // n + 1 each

    // quadtree
    hts::NodeF *nodes32 = nullptr;
    hts::NodeD *nodes64 = nullptr;

    // scratch
    unsigned long long *sort_scratch = nullptr;  // digit offsets, tile counters, look-back status words
    double *exact_part = nullptr;    // exact kernel chunk sums (4 doubles x exact_split(n) x n)
    int *scan_tmp = nullptr;
    int64_t scan_tmp_len = 0;
    double *red_tmp = nullptr;        // reduction partials
    unsigned long long *minmax = nullptr;  // [2s] min bits, [2s+1] max bits of segment s; then the largest gamma
    double *dscal = nullptr;          // [0] Z, [1] sum p log p, [2] sum p log w, [3] sum p
    int *status = nullptr;
    unsigned long long *counters = nullptr;  // 5: accepted cells, leaf pairs, warp visits, queries, criterion tests
    int *n_nodes = nullptr;          // device scalar: number of tree nodes
    double *h_pinned = nullptr;      // 8 doubles of pinned host scratch

    // batched embeddings: nseg independent problems in consecutive point ranges
    int nseg = 1;
    int64_t *seg_off = nullptr;      // device, nseg + 1 offsets
    unsigned char *seg_of = nullptr; // device, segment of each point (original order)
    double *seg_lr = nullptr;        // device, per-segment learning-rate factor
    double *seg_z = nullptr;         // device, per-segment Z (nseg > 1)
    int64_t seg_off_h[HTS_MAX_SEGMENTS + 1] = {0};

    // CUDA graph of one iteration (replayed by hts_step when enabled)
    int use_graphs = 0;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double gkey[5] = {-1, -1, -1, -1, -1};  // theta, exag, lr, momentum, layout version
    int64_t layout_version = 0;
    int64_t graph_launches = 0;      // kernels in one captured iteration

    // launch shapes (hts_autotune / hts_set_tuning)
    int walk_block = 256;            // walk threads per block: 32, 64, 128 or 256
    int attract_group = 8;           // float32 attraction lanes per row of P: 4, 8, 16 or 32
    int walk_split = -1;             // cut depth of the split walk (-1: by problem size)
    int attract_background = 0;      // set while the attraction is launched beside the walk
    unsigned *walk_cost = nullptr;   // per walk block: cycles of the last walk (launch-order input)
    int *walk_order = nullptr;       // [0] grid size, then the launch order of the walk's blocks
    void *split_frontier = nullptr;  // frontier table + entry count
    void *split_part = nullptr;      // partial sums of the split walk

    // CO-SNE term (Sec. 4.3): lambda1 KL + lambda2 (1/n) sum (|x|^2 - |y|^2)^2
    double cosne_l1 = 1.0, cosne_l2 = 0.0;
    double *xsq = nullptr;           // |x_i|^2, n doubles (nullptr: term off)

    // wait test (hts_set_wait_test): > 0 = the look-back spin limit while the
    // first tile of every sort pass withholds its status; 0 = off
    int wait_test = 0;

    // instrumentation
    int64_t launches = 0;            // kernels launched since creation
    int profiling = 0;               // record phase events every iteration
    cudaEvent_t *events = nullptr;   // kPhases + 3 per iteration slot
    int event_slots = 0;
    double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t phase_iters = 0;
};

namespace hts {

// ---- host launchers (one translation unit each) -------------------------
// keys.cu
void launch_prep_points(hts_ctx *c);
void launch_make_keys(hts_ctx *c);
// sort.cu
void launch_sort_pairs(hts_ctx *c);
int scan_exclusive(const int *in, int *out, int64_t len, int *tmp, cudaStream_t s);  // returns kernels launched
int64_t scan_tmp_size(int64_t len);
size_t sort_status_words(int64_t n);
// tree.cu
void launch_build_tree(hts_ctx *c, double theta, const TreeExport *ex);
// traverse.cu
void launch_walk(hts_ctx *c);
void launch_exact(hts_ctx *c);
// j-chunks of the exact kernel for n points (1 when the i-blocks alone fill
// the GPU); the partial sums take exact_split(n) * n double4 when it is > 1
int exact_split(int64_t n);
// split walk: buffer capacity (frontier entries) for n points, the depth used,
// and the bytes of the frontier table
int walk_split_capacity(int64_t n);
int walk_split_depth(int64_t n, int want, bool fp64);
size_t walk_split_frontier_bytes();
// attract.cu
void launch_attract(hts_ctx *c);
void launch_kl_terms(hts_ctx *c);
void launch_validate_csr(hts_ctx *c, int n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                         const void *values, int f64);
void launch_kl_rows(hts_ctx *c, double *a, double *b, double *p);
void launch_segments_setup(hts_ctx *c);
// update.cu
void launch_reduce_z(hts_ctx *c);
void launch_update(hts_ctx *c, double exag, double lr, double mom, double2 *g_out, int do_step);
void launch_check_y(hts_ctx *c);
void launch_segment_sums(hts_ctx *c, const double *v, double *out);

}  // namespace hts

// ---- device helpers ------------------------------------------------------
#ifdef __CUDACC__
namespace hts {

// Pair term of the repulsive and attractive sums for y_i and a point or
// cell midpoint c, written in terms of delta = cosh(d) - 1 =
// 2 |y_i - c|^2 il_i il_c (Eq. PoincareDistance).  With t = sinh(d) =
// sqrt(delta (delta + 2)), d = log1p(delta + t), w = 1 / (1 + d^2)
// and r1 = 1 / (t (1 + d^2)):
//   w          = t r1
//   w^2 d / t  = w d r1          (repulsion, exact KL form)
//   w d / t    = d r1            (attraction, exact KL form)
// and Eq. PoincareDistanceDerivative reads
//   dd/dy_i = 4 il_i il_c (Delta + s il_i y_i) / t,   s = |Delta|^2,
// so every pair adds a scalar times (Delta, s); the common 4 il_i factor
// and the il_i s y_i term are applied once per point at the end.
// delta is clamped below by a tiny positive number so that coincident
// points give w = 1 and zero force (the limit of w^2 d dd/dy as d -> 0).
// Float64 position and 1 / (1 - |y|^2) of a point record.
__device__ __forceinline__ void point_xy_il(const PointF &q, double &x, double &y, double &il)
{
    x = (double)q.xh + (double)q.xl;
    y = (double)q.yh + (double)q.yl;
    il = (double)q.il;
}
__device__ __forceinline__ void point_xy_il(const PointD &q, double &x, double &y, double &il)
{
    x = q.x;
    y = q.y;
    il = q.il;
}

struct PairF {
    float w, rep, att;  // w, w^2 d / t (or w^2 / t), w d / t (or w / t)
};
// (t = sinh(d) = sqrt(delta (delta + 2)); both forms below return these.)

// Float32 pair term with three special-function-unit operations (rsqrt,
// log2, reciprocal).  d = acosh(1 + delta) and the ratio f = d / sinh(d) are
// taken, for delta < 0.02, from the Taylor series
//   acosh(1 + x) / sqrt(x (2 + x)) = sum_k (-1)^k 2^k (k!)^2 / (2k + 1)! x^k
// (four terms: relative truncation error < 5e-9 at x = 0.02), and otherwise
// from d = log(1 + delta + sinh d) with the hardware log (absolute error
// ~2^-21.4 for arguments in [0.5, 2]), small against d >= 0.2 there.
// Relative error of every returned term stays below ~2e-6.  (Six terms up to
// 0.1 measured 2.5% slower in the walk for ~1e-6.)
// delta is held in [1e-30, 1e18]: the top keeps delta (delta + 2) finite in
// float32 for points within 1e-9 of the rim (there d ~ 42 and the pair's
// force is ~1e-3 of a unit-distance pair's).
template <int GF>
__device__ __forceinline__ PairF pair_terms_f32(float delta)
{
    delta = fminf(fmaxf(delta, 1e-30f), 1e18f);
    const float x = delta * (delta + 2.0f);  // sinh(d)^2
    const float rs = rsqrtf(x);              // 1 / sinh(d)
    const float t = x * rs;                  // sinh(d)
    float fs = -2.0f / 35.0f;
    fs = fmaf(fs, delta, 2.0f / 15.0f);
    fs = fmaf(fs, delta, -1.0f / 3.0f);
    fs = fmaf(fs, delta, 1.0f);
    const float lg = __logf(1.0f + delta + t);
    const bool small = delta < 0.02f;
    const float2 ld = __fmul2_rn(make_float2(lg, t), make_float2(rs, fs));  // (lg / t, t fs): one paired multiply
    const float f = small ? fs : ld.x;       // d / sinh(d)
    const float d = small ? ld.y : lg;       // acosh(1 + delta)
    PairF p;
    p.w = __fdividef(1.0f, fmaf(d, d, 1.0f));
    if (GF == 0) {
        p.att = p.w * f;
        p.rep = p.w * p.att;
    } else {
        p.att = p.w * rs;
        p.rep = p.w * p.att;
    }
    return p;
}

// Paired float32 arithmetic (one instruction for both components, each
// rounded as the scalar operation): a - b and the compensated difference of
// two hi/lo pairs, (ah - bh) + (al - bl) per component.
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);  // -b + a, exact like a - b
}
__device__ __forceinline__ float2 delta2(float2 ah, float2 al, float2 bh, float2 bl)
{
    return __fadd2_rn(sub2(ah, bh), sub2(al, bl));
}

struct PairD {
    double w, rep, att;
};

template <int GF>
__device__ __forceinline__ PairD pair_terms_f64(double delta)
{
    delta = fmax(delta, 1e-300);
    double t = sqrt(delta * (delta + 2.0));
    double d = log1p(delta + t);
    double u = fma(d, d, 1.0);
    double r1 = 1.0 / (t * u);
    PairD p;
    p.w = t * r1;
    if (GF == 0) {
        p.att = d * r1;
        p.rep = p.w * p.att;
    } else {
        p.att = r1;
        p.rep = p.w * r1;
    }
    return p;
}

// Quadtree level of a binary-radix-tree node from its common-prefix length
// (Karras' delta: clz of the key xor, or 64 + clz of the index xor for equal
// keys).  Keys occupy the low 58 bits, so distinct keys have delta in [6, 63].
__device__ __forceinline__ int quad_level(int pref)
{
    if (pref >= 64) return kLevels;
    if (pref < 6) return -1;  // keys of different segments: above every segment's root
    int l = (pref - 6) >> 1;
    return l < kLevels ? l : kLevels;
}

}  // namespace hts
#endif
