// tree.cu -- device build of the modified polar quadtree (Sec. 4.1).
//
// Input: keys sorted with their point indices (sort.cu).  Steps:
//  1. gather      sorted point records for the walk, and the per-point
//                 Einstein terms gamma_j, gamma_j v_j (Eq. EinsteinMidpoint in
//                 Klein coordinates, gamma_j v_j = 2 y_j / (1 - |y_j|^2)).
//  2. radix tree  binary radix tree over the sorted keys (Karras, "Maximizing
//                 parallelism in the construction of BVHs, octrees and k-d
//                 trees", HPG 2012): one thread per internal node finds its
//                 key range and split by binary search on common-prefix
//                 lengths; equal keys are ordered by index.
//  3. sums        bottom-up over the binary tree: the second thread to reach
//                 a node adds its two children in fixed (left, right) order
//                 in double-double, so every cell's sums are exact to ~1e-30
//                 and independent of scheduling; rounding them once gives the
//                 correctly rounded float64 sums.
//  4. quad nodes  a binary node is a quadtree cell iff its quad level
//                 floor(prefix_bits / 2) exceeds its parent's; that is the
//                 deepest cell of a chain of one-child cells (chains collapse:
//                 the cell diameter shrinks along a chain while the summary
//                 stays the same, so accepting the deepest cell is accepting
//                 the chain).  Level-29 cells with several points are buckets.
//  5. layout      nodes in pre-order (children in key order): order by first
//                 point, then by depth, so per first point p the count of
//                 nodes starting at p is scanned into pre[]; a cell's position
//                 is pre[lo] + (its ancestors starting at lo) and the index
//                 after its subtree is pre[hi + 1].
//  6. emit        midpoint y_cell = m / (1 + sqrt(1 - |m|^2)), m = S_u / S_gamma,
//                 il = 1 / (1 - |y_cell|^2), r_cell (longest internal distance:
//                 max of diagonal, radial edge and outer-arc chord, Sec. 4.1)
//                 and the acceptance threshold cosh(r_cell / theta) - 1, which
//                 turns the criterion r_cell / d < theta into delta > thr.
#include <math.h>

#include <cuda/atomic>

#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kBlock = 256;

__global__ void gather_kernel(int n, const uint32_t *__restrict__ idx, const double2 *__restrict__ y,
                              const PointF *__restrict__ pts32, const PointD *__restrict__ pts64, PointF *spts32,
                              PointD *spts64, double *terms)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t i = idx[p];
    if (spts32) spts32[p] = pts32[i];
    if (spts64) spts64[p] = pts64[i];
    double2 q = y[i];
    double n2 = __dadd_rn(__dmul_rn(q.x, q.x), __dmul_rn(q.y, q.y));
    double a = __dsub_rn(1.0, n2);
    terms[3 * p + 0] = __ddiv_rn(__dadd_rn(1.0, n2), a);
    terms[3 * p + 1] = __ddiv_rn(__dmul_rn(2.0, q.x), a);
    terms[3 * p + 2] = __ddiv_rn(__dmul_rn(2.0, q.y), a);
}

__device__ __forceinline__ int prefix_len(const uint64_t *__restrict__ keys, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    uint64_t a = keys[i], b = keys[j];
    if (a == b) return 64 + __clz((unsigned)(i ^ j));
    return __clzll((long long)(a ^ b));
}

// Children are encoded as >= 0 (internal node) or ~leaf (sorted position).
__global__ void radix_tree_kernel(int n, const uint64_t *__restrict__ keys, int *left, int *right, int *parent,
                                  int *leaf_parent, int *lo_arr, int *hi_arr, int *pref_arr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (prefix_len(keys, n, i, i + 1) - prefix_len(keys, n, i, i - 1)) > 0 ? 1 : -1;
    int dmin = prefix_len(keys, n, i, i - d);
    int lmax = 2;
    while (prefix_len(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (prefix_len(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = prefix_len(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (prefix_len(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int split = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int lc = (lo == split) ? ~split : split;
    int rc = (hi == split + 1) ? ~(split + 1) : split + 1;
    left[i] = lc;
    right[i] = rc;
    if (lc < 0) leaf_parent[~lc] = i; else parent[lc] = i;
    if (rc < 0) leaf_parent[~rc] = i; else parent[rc] = i;
    lo_arr[i] = lo;
    hi_arr[i] = hi;
    pref_arr[i] = dnode;
    if (i == 0) parent[0] = -1;
}

__device__ __forceinline__ void load_child(int c, const double *__restrict__ terms, const double *sums, DD out[3])
{
    if (c < 0) {
        int p = ~c;
        out[0] = DD{terms[3 * p], 0.0};
        out[1] = DD{terms[3 * p + 1], 0.0};
        out[2] = DD{terms[3 * p + 2], 0.0};
    } else {
        const double *s = sums + 6 * (size_t)c;
        out[0] = DD{__ldcg(s + 0), __ldcg(s + 1)};
        out[1] = DD{__ldcg(s + 2), __ldcg(s + 3)};
        out[2] = DD{__ldcg(s + 4), __ldcg(s + 5)};
    }
}

__global__ void bottom_up_kernel(int n, const double *__restrict__ terms, const int *__restrict__ left,
                                 const int *__restrict__ right, const int *__restrict__ parent,
                                 const int *__restrict__ leaf_parent, int *flags, double *sums)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || n < 2) return;
    int node = leaf_parent[j];
    // The walk climbs at most n - 1 nodes; the bound only guards corrupt input.
    for (int guard = 0; node >= 0 && guard < n; ++guard) {
        // acquire-release: this thread's stored sums are visible to whoever
        // arrives second, and the second arrival sees its sibling's sums
        cuda::atomic_ref<int, cuda::thread_scope_device> flag(flags[node]);
        if (flag.fetch_add(1, cuda::memory_order_acq_rel) == 0) return;  // first arrival
        DD a[3], b[3];
        load_child(left[node], terms, sums, a);
        load_child(right[node], terms, sums, b);
        double *s = sums + 6 * (size_t)node;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            DD r = dd_add(a[k], b[k]);
            __stcg(s + 2 * k, r.hi);
            __stcg(s + 2 * k + 1, r.lo);
        }
        node = parent[node];
    }
}

__global__ void quad_mark_kernel(int n, const int *__restrict__ parent, const int *__restrict__ leaf_parent,
                                 const int *__restrict__ lo_arr, const int *__restrict__ pref, int *quad, int *cnt)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n - 1) {  // binary internal node k
        int lv = quad_level(pref[k]);
        int pl = k == 0 ? -1 : quad_level(pref[parent[k]]);
        int q = lv > pl;
        quad[k] = q;
        if (q) atomicAdd(&cnt[lo_arr[k]], 1);
    }
    if (k < n) {  // point k: a node of its own unless it sits in a bucket
        bool leaf = n == 1 || quad_level(pref[leaf_parent[k]]) < kLevels;
        if (leaf) atomicAdd(&cnt[k], 1);
    }
}

// Hyperbolic distance between the polar points (ra, 0) and (rb, dphi) with
// exact radial gap drr = rb - ra: |p - q|^2 = drr^2 + 4 ra rb sin^2(dphi/2),
// 1 - r^2 = (1 - r)(1 + r) -- no cancellation for small cells.  Explicitly
// rounded operations keep the cell geometry free of fused multiply-adds.
__device__ __forceinline__ double polar_dist(double ra, double rb, double drr, double sh)
{
    double s = __dadd_rn(__dmul_rn(drr, drr), __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(4.0, ra), rb), sh), sh));
    double den = __dmul_rn(__dmul_rn(__dsub_rn(1.0, ra), __dadd_rn(1.0, ra)),
                           __dmul_rn(__dsub_rn(1.0, rb), __dadd_rn(1.0, rb)));
    double delta = __ddiv_rn(__dmul_rn(2.0, s), den);
    return log1p(__dadd_rn(delta, __dsqrt_rn(__dmul_rn(delta, __dadd_rn(delta, 2.0)))));
}

__device__ __forceinline__ double radius_of(double c, int rule)
{
    return rule == HTS_EQUAL_AREA ? __dsqrt_rn(__ddiv_rn(__dsub_rn(c, 1.0), __dadd_rn(c, 1.0))) : c;
}

// Longest internal distance of the depth-`ell` polar quad with radial index a:
// max of diagonal, radial edge and outer-arc chord (Sec. 4.1).  The gap in the
// split coordinate is span * 2^-ell exactly; for equal-area splitting
// r1 - r0 = 2 dc / ((c0 + 1)(c1 + 1)(r0 + r1)) since r^2 = 1 - 2 / (c + 1).
__device__ double cell_size(double lo, double hi, uint64_t a, int ell, int rule)
{
    double scale = ldexp(1.0, -ell);
    double span = __dsub_rn(hi, lo);
    double c0 = __dadd_rn(lo, __dmul_rn(span, __dmul_rn((double)a, scale)));
    double c1 = __dadd_rn(lo, __dmul_rn(span, __dmul_rn((double)(a + 1), scale)));
    double dc = __dmul_rn(span, scale);
    double r0 = radius_of(c0, rule), r1 = radius_of(c1, rule);
    double dr = dc;
    if (rule == HTS_EQUAL_AREA) {
        double rs = __dadd_rn(r0, r1);
        dr = rs > 0.0 ? __ddiv_rn(__dmul_rn(2.0, dc), __dmul_rn(__dmul_rn(__dadd_rn(c0, 1.0), __dadd_rn(c1, 1.0)), rs))
                      : 0.0;
    }
    double sh = sin(__dmul_rn(kTwoPi, scale) / 2.0);
    double diag = polar_dist(r0, r1, dr, sh);
    double radial = polar_dist(r0, r1, dr, 0.0);
    double arc = polar_dist(r1, r1, 0.0, sh);
    return fmax(fmax(diag, radial), arc);
}

// Float32 version of the cell size and acceptance threshold, used when the
// tree serves the float32 walk (its thresholds are float32 anyway).  The
// radii, their gap and the conformal terms 1 - r^2 are formed in float64;
// the distances use the float32 acosh of pair_terms_f32 (series below 0.1).
__device__ __forceinline__ float acosh1p_f32(float delta)
{
    delta = fmaxf(delta, 0.0f);
    const float x = delta * (delta + 2.0f);
    const float t = sqrtf(x);
    float fs = -8.0f / 693.0f;
    fs = fmaf(fs, delta, 8.0f / 315.0f);
    fs = fmaf(fs, delta, -2.0f / 35.0f);
    fs = fmaf(fs, delta, 2.0f / 15.0f);
    fs = fmaf(fs, delta, -1.0f / 3.0f);
    fs = fmaf(fs, delta, 1.0f);
    return delta < 0.1f ? t * fs : __logf(1.0f + delta + t);
}

__device__ float cell_threshold_f32(double lo, double hi, uint64_t a, int ell, int rule, double theta)
{
    double scale = ldexp(1.0, -ell);
    double span = hi - lo;
    double c0 = lo + span * ((double)a * scale);
    double c1 = lo + span * ((double)(a + 1) * scale);
    double dc = span * scale;
    double r0 = radius_of(c0, rule), r1 = radius_of(c1, rule);
    double dr = rule == HTS_EQUAL_AREA ? (r0 + r1 > 0.0 ? 2.0 * dc / ((c0 + 1.0) * (c1 + 1.0) * (r0 + r1)) : 0.0)
                                       : dc;
    const float a0 = (float)((1.0 - r0) * (1.0 + r0)), a1 = (float)((1.0 - r1) * (1.0 + r1));
    const float f0 = (float)r0, f1 = (float)r1, fdr = (float)dr;
    const float sh = sinpif(ldexpf(1.0f, -ell));  // sin(dphi / 2), dphi = 2 pi 2^-ell: relative accuracy
    const float sh2 = sh * sh;
    const float diag = acosh1p_f32(2.0f * (fdr * fdr + 4.0f * f0 * f1 * sh2) / (a0 * a1));
    const float radial = acosh1p_f32(2.0f * (fdr * fdr) / (a0 * a1));
    const float arc = acosh1p_f32(2.0f * (4.0f * f1 * f1 * sh2) / (a1 * a1));
    const float rc = fmaxf(fmaxf(diag, radial), arc);
    // cosh(rc / theta) - 1 = 2 sinh(x)^2 with x = rc / (2 theta); series below 0.5
    const float x = rc / (float)(2.0 * theta);
    float sx;
    if (x < 0.5f) {
        const float x2 = x * x;
        sx = x * fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 5040.0f, 1.0f / 120.0f), 1.0f / 6.0f), 1.0f);
    } else {
        const float e = __expf(x);
        sx = 0.5f * (e - 1.0f / e);
    }
    return 2.0f * sx * sx;
}

__device__ __forceinline__ uint64_t radial_index(uint64_t prefix, int ell)
{
    uint64_t a = 0;
    for (int b = 0; b < ell; ++b) a |= ((prefix >> (2 * b + 1)) & 1ull) << b;
    return a;
}

struct EmitArgs {
    int n;
    double theta;
    int rule;
    const uint64_t *keys;
    const uint32_t *idx;
    const double2 *y;
    const PointF *spts32;
    const PointD *spts64;
    const int *left, *parent, *leaf_parent, *lo_arr, *hi_arr, *pref, *quad, *cnt, *pre;
    const double *sums;
    const unsigned long long *mm;
    NodeF *nodes32;
    NodeD *nodes64;
    TreeExport ex;
    int capacity;
    int *status;
};

__global__ void emit_kernel(EmitArgs A)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = A.n;
    if (k < n - 1 && A.quad[k]) {
        int lo = A.lo_arr[k], hi = A.hi_arr[k];
        int rank = 0;
        for (int a = A.parent[k]; a >= 0 && A.lo_arr[a] == lo; a = A.parent[a]) rank += A.quad[a];
        int pos = A.pre[lo] + rank;
        int skip = A.pre[hi + 1];
        int ell = quad_level(A.pref[k]);
        const double *s = A.sums + 6 * (size_t)k;
        double sg = s[0], sux = s[2], suy = s[4];
        double mx = __ddiv_rn(sux, sg), my = __ddiv_rn(suy, sg);
        double sq = __dsqrt_rn(__dsub_rn(1.0, __dadd_rn(__dmul_rn(mx, mx), __dmul_rn(my, my))));
        double cx = __ddiv_rn(mx, __dadd_rn(1.0, sq)), cy = __ddiv_rn(my, __dadd_rn(1.0, sq));
        double beta = __dsub_rn(1.0, __dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)));
        double il = 1.0 / beta;
        double lob = __longlong_as_double((long long)A.mm[0]);
        double hib = __longlong_as_double((long long)A.mm[1]);
        uint64_t prefix = ell > 0 ? (A.keys[lo] >> (2 * (kLevels - ell))) : 0ull;
        // float64 geometry for the float64 walk and for exports; float32 otherwise
        const bool geo64 = A.nodes64 != nullptr || A.ex.depth != nullptr;
        double rc = HUGE_VAL, thr = HUGE_VAL;
        float thr32 = INFINITY;
        if (ell > 0 && geo64) {
            rc = cell_size(lob, hib, radial_index(prefix, ell), ell, A.rule);
            if (A.theta > 0.0) {
                double sh = sinh(rc / (2.0 * A.theta));
                thr = 2.0 * sh * sh;
            }
            thr32 = (float)thr;
        } else if (ell > 0 && A.theta > 0.0) {
            thr32 = cell_threshold_f32(lob, hib, radial_index(prefix, ell), ell, A.rule, A.theta);
        }
        int count = hi - lo + 1;
        bool bucket = ell == kLevels;
        if (pos < 0 || pos >= A.capacity || skip <= pos || skip > A.capacity) {
            atomicOr(A.status, 2);
            return;
        }
        if (A.nodes32) {
            NodeF nd;
            nd.xh = (float)cx;
            nd.yh = (float)cy;
            nd.xl = (float)(cx - (double)nd.xh);
            nd.yl = (float)(cy - (double)nd.yh);
            nd.il = (float)il;
            nd.thr = bucket ? __int_as_float(lo) : thr32;
            nd.count = bucket ? -count : count;
            nd.skip = skip;
            A.nodes32[pos] = nd;
        }
        if (A.nodes64) {
            NodeD nd;
            nd.x = cx;
            nd.y = cy;
            nd.il = il;
            nd.thr = thr;
            nd.count = bucket ? -count : count;
            nd.skip = skip;
            nd.pos = lo;
            nd.pad = 0;
            A.nodes64[pos] = nd;
        }
        if (A.ex.depth) {
            int64_t first = -1;
            if (bucket) {
                first = A.idx[lo];
                for (int p = lo + 1; p <= hi; ++p) first = min(first, (int64_t)A.idx[p]);
            }
            A.ex.depth[pos] = ell;
            A.ex.prefix[pos] = prefix;
            A.ex.count[pos] = count;
            A.ex.first[pos] = first;
            A.ex.ycell[2 * pos] = cx;
            A.ex.ycell[2 * pos + 1] = cy;
            A.ex.rcell[pos] = rc;
        }
    }
    if (k < n) {
        bool leaf = n == 1 || quad_level(A.pref[A.leaf_parent[k]]) < kLevels;
        if (!leaf) return;
        int pos = A.pre[k] + A.cnt[k] - 1;
        if (pos < 0 || pos >= A.capacity) {
            atomicOr(A.status, 2);
            return;
        }
        if (A.nodes32) {
            PointF q = A.spts32[k];
            NodeF nd;
            nd.xh = q.xh;
            nd.yh = q.yh;
            nd.xl = q.xl;
            nd.yl = q.yl;
            nd.il = q.il;
            nd.thr = __int_as_float(k);
            nd.count = 1;
            nd.skip = pos + 1;
            A.nodes32[pos] = nd;
        }
        if (A.nodes64) {
            PointD q = A.spts64[k];
            NodeD nd;
            nd.x = q.x;
            nd.y = q.y;
            nd.il = q.il;
            nd.thr = HUGE_VAL;
            nd.count = 1;
            nd.skip = pos + 1;
            nd.pos = k;
            nd.pad = 0;
            A.nodes64[pos] = nd;
        }
        if (A.ex.depth) {
            int depth = n == 1 ? 0 : quad_level(A.pref[A.leaf_parent[k]]) + 1;
            uint32_t i = A.idx[k];
            double2 q = A.y[i];
            A.ex.depth[pos] = depth;
            A.ex.prefix[pos] = depth > 0 ? (A.keys[k] >> (2 * (kLevels - depth))) : 0ull;
            A.ex.count[pos] = 1;
            A.ex.first[pos] = i;
            A.ex.ycell[2 * pos] = q.x;
            A.ex.ycell[2 * pos + 1] = q.y;
            A.ex.rcell[pos] = HUGE_VAL;
        }
    }
}

}  // namespace

void launch_build_tree(hts_ctx *c, double theta, const TreeExport *ex)
{
    const int n = (int)c->n;
    cudaStream_t s = c->stream;
    const bool f32 = c->cfg.precision == HTS_FP32_MIXED;
    const int gp = (n + kBlock - 1) / kBlock;
    gather_kernel<<<gp, kBlock, 0, s>>>(n, c->idx, c->y, c->pts32, c->pts64, f32 ? c->spts32 : nullptr,
                                        f32 ? nullptr : c->spts64, c->terms);
    c->launches += 3;  // gather, quad_mark, emit
    if (n > 1) {
        const int gi = (n - 1 + kBlock - 1) / kBlock;
        radix_tree_kernel<<<gi, kBlock, 0, s>>>(n, c->keys, c->bn_left, c->bn_right, c->bn_parent, c->leaf_parent,
                                                c->bn_lo, c->bn_hi, c->bn_pref);
        cudaMemsetAsync(c->bn_flag, 0, sizeof(int) * (size_t)(n - 1), s);
        bottom_up_kernel<<<gp, kBlock, 0, s>>>(n, c->terms, c->bn_left, c->bn_right, c->bn_parent, c->leaf_parent,
                                               c->bn_flag, c->bn_sum);
        c->launches += 2;
    }
    cudaMemsetAsync(c->cnt, 0, sizeof(int) * (size_t)(n + 1), s);
    quad_mark_kernel<<<gp, kBlock, 0, s>>>(n, c->bn_parent, c->leaf_parent, c->bn_lo, c->bn_pref, c->bn_quad,
                                           c->cnt);
    c->launches += scan_exclusive(c->cnt, c->pre, (int64_t)n + 1, c->scan_tmp, s);
    EmitArgs A;
    A.n = n;
    A.theta = theta;
    A.rule = c->cfg.split_rule;
    A.keys = c->keys;
    A.idx = c->idx;
    A.y = c->y;
    A.spts32 = c->spts32;
    A.spts64 = c->spts64;
    A.left = c->bn_left;
    A.parent = c->bn_parent;
    A.leaf_parent = c->leaf_parent;
    A.lo_arr = c->bn_lo;
    A.hi_arr = c->bn_hi;
    A.pref = c->bn_pref;
    A.quad = c->bn_quad;
    A.cnt = c->cnt;
    A.pre = c->pre;
    A.sums = c->bn_sum;
    A.mm = c->minmax;
    A.nodes32 = f32 ? c->nodes32 : nullptr;
    A.nodes64 = f32 ? nullptr : c->nodes64;
    A.ex = ex ? *ex : TreeExport{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    A.capacity = 2 * n;
    A.status = c->status;
    emit_kernel<<<gp, kBlock, 0, s>>>(A);
}

}  // namespace hts
