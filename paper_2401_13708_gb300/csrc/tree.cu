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
//  3. sums        exclusive prefix sums of the Einstein terms over the sorted
//                 points in 128-bit fixed point: each float64 term is scaled
//                 by 2^E (E from the largest term and n, so no prefix can
//                 overflow) and kept as an exact integer, the scan adds
//                 integers (exact, any order), and a cell's sums
//                 P[hi + 1] - P[lo] are exact; one correctly rounded
//                 conversion gives the float64 sums the oracle rounds from its
//                 128-bit accumulation.  Terms above 2^(52 - E) convert
//                 exactly (E >= ~90 for 1M points within 1 - 1e-4 of the rim);
//                 smaller ones are truncated at 2^-E.  Integer adds keep the
//                 scan off the float64 pipe, which is narrow on this GPU.
//  4. quad nodes  a binary node is a quadtree cell iff its quad level
//                 floor(prefix_bits / 2) exceeds its parent's; that is the
//                 deepest cell of a chain of one-child cells (chains collapse:
//                 the cell diameter shrinks along a chain while the summary
//                 stays the same, so accepting the deepest cell is accepting
//                 the chain).  Level-29 cells with several points are buckets.
//  5. layout      nodes in pre-order (children in key order): order by first
//                 point, then by depth, so per first point p the count of
//                 nodes starting at p is scanned into pre[]; a cell's position
//                 is pre[lo] + (number of shallower cells starting at lo, a
//                 popcount of a per-point bit set of quad levels) and the index
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

// Sorted point records and the Einstein terms; *gmax receives the largest
// gamma (bits of a positive double order like the double), which bounds every
// term (|gamma v| <= gamma).
// exact: the oracle's correctly rounded divisions (float64 nodes, exports);
// otherwise one reciprocal (the float32 nodes round the result to float).
__global__ void gather_kernel(int n, const uint32_t *__restrict__ idx, const double2 *__restrict__ y,
                              const PointF *__restrict__ pts32, const PointD *__restrict__ pts64, PointF *spts32,
                              PointD *spts64, double *terms, unsigned long long *gmax, int exact)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long gb = 0;
    if (p < n) {
        uint32_t i = idx[p];
        if (spts32) spts32[p] = pts32[i];
        if (spts64) spts64[p] = pts64[i];
        double2 q = y[i];
        double n2 = __dadd_rn(__dmul_rn(q.x, q.x), __dmul_rn(q.y, q.y));
        double a = __dsub_rn(1.0, n2);
        double g;
        if (exact) {
            g = __ddiv_rn(__dadd_rn(1.0, n2), a);
            terms[3 * p + 1] = __ddiv_rn(__dmul_rn(2.0, q.x), a);
            terms[3 * p + 2] = __ddiv_rn(__dmul_rn(2.0, q.y), a);
        } else {
            const double ia = 1.0 / a;
            g = (1.0 + n2) * ia;
            terms[3 * p + 1] = 2.0 * q.x * ia;
            terms[3 * p + 2] = 2.0 * q.y * ia;
        }
        terms[3 * p + 0] = g;
        gb = (unsigned long long)__double_as_longlong(g);
    }
    for (int o = 16; o > 0; o >>= 1) gb = max(gb, __shfl_xor_sync(0xffffffffu, gb, o));
    if ((threadIdx.x & 31) == 0 && gb) atomicMax(gmax, gb);
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

// ---- exclusive prefix sums of the Einstein terms in 128-bit fixed point -----
// P[p] = sum of terms of sorted points 0 .. p-1 (three quantities), so the
// sums of any cell [lo, hi] are P[hi + 1] - P[lo].
constexpr int kScanT = 256;            // threads per scan block
constexpr int kScanI = 4;              // elements per thread
constexpr int kScanB = kScanT * kScanI;

typedef __int128 fx_t;

struct FX3 {
    fx_t g, x, y;
};

__device__ __forceinline__ FX3 fx3_add(const FX3 &a, const FX3 &b) { return FX3{a.g + b.g, a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ FX3 fx3_zero() { return FX3{0, 0, 0}; }

__device__ __forceinline__ fx_t fx_shfl_up(fx_t v, int o)
{
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    const unsigned long long l2 = __shfl_up_sync(0xffffffffu, lo, o), h2 = __shfl_up_sync(0xffffffffu, hi, o);
    return (fx_t)(((unsigned __int128)h2 << 64) | l2);
}

__device__ __forceinline__ FX3 fx3_shfl_up(const FX3 &v, int o)
{
    return FX3{fx_shfl_up(v.g, o), fx_shfl_up(v.x, o), fx_shfl_up(v.y, o)};
}

// Scale exponent E with n * gmax * 2^E < 2^125: no prefix sum can overflow.
__device__ __forceinline__ int fx_exponent(unsigned long long gmax_bits, int n)
{
    const int e = (int)((gmax_bits >> 52) & 0x7ff) - 1022;  // gmax >= 1 is normal: gmax < 2^e
    const int lg = 32 - __clz(max(n, 1));                    // n < 2^lg
    return 125 - e - lg;
}

// 2^k for -1022 <= k <= 1023 (a normal float64 built from its exponent bits).
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// floor(x * 2^E) and a cell sum as a float64 without the 2^-E scale (float32
// nodes: the scale cancels in the ratios), both from bit patterns with integer
// operations (bits.cuh), off the float64 pipe that runs the conversions.
__device__ __forceinline__ fx_t fx_from_double(double x, int E) { return fixed_from_double(x, E); }
__device__ __forceinline__ double fx_to_double_unscaled(fx_t v) { return fixed_to_double_trunc(v); }

// v * 2^-E correctly rounded to float64: the top 64 significant bits, with a
// sticky bit for the rest, go through one round-to-nearest conversion.
__device__ __forceinline__ double fx_to_double(fx_t v, int E)
{
    const bool neg = v < 0;
    const unsigned __int128 m = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
    const unsigned long long top = (unsigned long long)(m >> 64), low = (unsigned long long)m;
    double d;
    if (top == 0) {
        d = __ull2double_rn(low);
    } else {
        const int sh = 64 - __clzll((long long)top);  // 1 .. 64
        const unsigned long long lowmask = sh >= 64 ? ~0ull : ((1ull << sh) - 1ull);
        const unsigned long long t = (unsigned long long)(m >> sh) | ((low & lowmask) ? 1ull : 0ull);
        d = __ull2double_rn(t) * pow2(sh);
    }
    d = d * pow2(-E);
    return neg ? -d : d;
}

// One block scans kScanB consecutive elements: out[i] = exclusive prefix within
// the block, tot[block] = block total.  Input: float64 terms (3 per point,
// converted with the exponent from *gmax) when `terms` is given, otherwise
// FX3 values.
__global__ void __launch_bounds__(kScanT) fx_scan_block_kernel(int len, const double *__restrict__ terms,
                                                              const unsigned long long *__restrict__ gmax, int n,
                                                              const FX3 *__restrict__ in, FX3 *out, FX3 *tot)
{
    __shared__ FX3 wsum[kScanT / 32];
    const int E = terms ? fx_exponent(*gmax, n) : 0;
    const int base = blockIdx.x * kScanB + threadIdx.x * kScanI;
    FX3 v[kScanI];
    FX3 t = fx3_zero();
#pragma unroll
    for (int k = 0; k < kScanI; ++k) {
        const int i = base + k;
        if (i < len) {
            if (terms) {
                v[k] = FX3{fx_from_double(terms[3 * i], E), fx_from_double(terms[3 * i + 1], E),
                           fx_from_double(terms[3 * i + 2], E)};
            } else {
                v[k] = in[i];
            }
        } else {
            v[k] = fx3_zero();
        }
        t = fx3_add(t, v[k]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    FX3 inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        FX3 u = fx3_shfl_up(inc, o);
        if (lane >= o) inc = fx3_add(u, inc);
    }
    FX3 excl = fx3_shfl_up(inc, 1);
    if (lane == 0) excl = fx3_zero();
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    FX3 run = excl;
    for (int k = 0; k < w; ++k) run = fx3_add(run, wsum[k]);
#pragma unroll
    for (int k = 0; k < kScanI; ++k) {
        const int i = base + k;
        if (i < len) out[i] = run;
        run = fx3_add(run, v[k]);
    }
    if (threadIdx.x == kScanT - 1) tot[blockIdx.x] = run;
}

__global__ void fx_scan_add_kernel(int len, FX3 *out, const FX3 *__restrict__ off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = fx3_add(off[i / kScanB], out[i]);
}

// Exclusive scan of len elements into out[0 .. len-1]; the grand total goes to
// *total.  tmp holds the block totals of every recursion level.
void fx_scan(int len, const double *terms, const unsigned long long *gmax, int n, const FX3 *in, FX3 *out,
             FX3 *total, FX3 *tmp, cudaStream_t s, int64_t *launches)
{
    const int blocks = (len + kScanB - 1) / kScanB;
    FX3 *tot = tmp;
    fx_scan_block_kernel<<<blocks, kScanT, 0, s>>>(len, terms, gmax, n, in, out, tot);
    *launches += 1;
    if (blocks == 1) {
        cudaMemcpyAsync(total, tot, sizeof(FX3), cudaMemcpyDeviceToDevice, s);
        return;
    }
    fx_scan(blocks, nullptr, nullptr, 0, tot, tot, total, tmp + blocks, s, launches);
    fx_scan_add_kernel<<<(len + 255) / 256, 256, 0, s>>>(len, out, tot);
    *launches += 1;
}

// Quad levels present among the cells whose first sorted point is p, one bit
// per level (cells with a common first point are nested, at distinct levels),
// so a cell's rank among them is a popcount.  Points outside buckets are
// leaves of their own.
__global__ void quad_mark_kernel(int n, const int *__restrict__ parent, const int *__restrict__ leaf_parent,
                                 const int *__restrict__ lo_arr, const int *__restrict__ pref, int *quad,
                                 unsigned *mask)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n - 1) {  // binary internal node k
        int lv = quad_level(pref[k]);
        int pl = k == 0 ? -1 : quad_level(pref[parent[k]]);
        int q = lv > pl;
        quad[k] = q;
        if (q) atomicOr(&mask[lo_arr[k]], 1u << lv);
    }
}

__global__ void count_kernel(int n, const int *__restrict__ leaf_parent, const int *__restrict__ pref,
                             const unsigned *__restrict__ mask, int *cnt)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        bool leaf = n == 1 || quad_level(pref[leaf_parent[k]]) < kLevels;
        cnt[k] = __popc(mask[k]) + (leaf ? 1 : 0);
    } else if (k == n) {
        cnt[n] = 0;
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
    const unsigned *mask;
    const FX3 *prefix;  // n + 1 exclusive prefix sums of the Einstein terms (fixed point)
    const unsigned long long *gmax;  // largest gamma (bits): the fixed-point exponent
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
    if (k == 0 && A.nodes32) {  // four empty slots after the last node: the float32 walk's overrun
        const int m = min(A.pre[n], A.capacity);
        for (int e = 0; e < kWalkOverrun; ++e) A.nodes32[m + e] = NodeF{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
    }
    if (k < n - 1 && A.quad[k]) {
        int lo = A.lo_arr[k], hi = A.hi_arr[k];
        int ell = quad_level(A.pref[k]);
        int rank = __popc(A.mask[lo] & ((1u << ell) - 1u));  // shallower cells starting at lo
        int pos = A.pre[lo] + rank;
        int skip = A.pre[hi + 1];
        const FX3 p1 = A.prefix[hi + 1], p0 = A.prefix[lo];
        double cx, cy, beta;
        if (A.nodes64 || A.ex.depth) {  // float64 walk / export: the oracle's correctly rounded steps
            const int E = fx_exponent(*A.gmax, n);
            const double sg = fx_to_double(p1.g - p0.g, E);
            const double sux = fx_to_double(p1.x - p0.x, E);
            const double suy = fx_to_double(p1.y - p0.y, E);
            const double mx = __ddiv_rn(sux, sg);
            const double my = __ddiv_rn(suy, sg);
            const double sq = __dsqrt_rn(__dsub_rn(1.0, __dadd_rn(__dmul_rn(mx, mx), __dmul_rn(my, my))));
            cx = __ddiv_rn(mx, __dadd_rn(1.0, sq));
            cy = __ddiv_rn(my, __dadd_rn(1.0, sq));
            beta = __dsub_rn(1.0, __dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)));
        } else {
            // float32 nodes: the sums stay scaled by 2^E (it cancels), and
            // with m = S_u / S_g and R = sqrt(S_g^2 - |S_u|^2) = S_g sq,
            //   y_cell = m / (1 + sq) = S_u / (S_g + R),
            //   1 - |y_cell|^2 = 2 sq / (1 + sq) = 2 R / (S_g + R):
            // one reciprocal instead of two
            const double sg = fx_to_double_unscaled(p1.g - p0.g);
            const double sux = fx_to_double_unscaled(p1.x - p0.x), suy = fx_to_double_unscaled(p1.y - p0.y);
            const double R = sqrt(fmax(sg * sg - (sux * sux + suy * suy), 0.0));
            const double rd = 1.0 / (sg + R);
            cx = sux * rd;
            cy = suy * rd;
            beta = 2.0 * R * rd;
        }
        // 1 / beta: a float64 division for float64 nodes; float32 nodes store a
        // float, taken as the float reciprocal of beta (off the float64 pipe)
        const double il = A.nodes64 ? 1.0 / beta : 0.0;
        const uint64_t key = A.keys[lo];
        const int seg = (int)(key >> kSegShift);  // segment: its own root annulus
        double lob = __longlong_as_double((long long)A.mm[2 * seg]);
        double hib = __longlong_as_double((long long)A.mm[2 * seg + 1]);
        const uint64_t kb = key & ((1ull << kSegShift) - 1);
        uint64_t prefix = ell > 0 ? (kb >> (2 * (kLevels - ell))) : 0ull;
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
            float b32, unused;
            split_f32(cx, nd.xh, nd.xl);
            split_f32(cy, nd.yh, nd.yl);
            split_f32(beta, b32, unused);  // (float)beta
            nd.il = __frcp_rn(b32);
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
            A.ex.prefix[pos] = depth > 0 ? ((A.keys[k] & ((1ull << kSegShift) - 1)) >> (2 * (kLevels - depth))) : 0ull;
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
    unsigned long long *gmax = c->minmax + 2 * kMaxSegments;
    FX3 *prefix = reinterpret_cast<FX3 *>(c->bn_sum);  // n + 1 entries
    unsigned *mask = reinterpret_cast<unsigned *>(c->bn_flag);
    cudaMemsetAsync(gmax, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(mask, 0, sizeof(unsigned) * (size_t)n, s);
    // two independent chains, joined before emit: on the side stream the
    // sorted point records and the fixed-point prefix sums of the Einstein
    // terms; here the radix tree, the quad-level marks and the node layout
    // (they need only the sorted keys)
    cudaStream_t ts = c->tstream;
    cudaEventRecord(c->tev_fork, s);
    cudaStreamWaitEvent(ts, c->tev_fork, 0);
    gather_kernel<<<gp, kBlock, 0, ts>>>(n, c->idx, c->y, c->pts32, c->pts64, f32 ? c->spts32 : nullptr,
                                         f32 ? nullptr : c->spts64, c->terms, gmax, (!f32 || ex) ? 1 : 0);
    c->launches += 4;  // gather, quad_mark, count, emit
    if (n > 1)
        fx_scan(n, c->terms, gmax, n, nullptr, prefix, prefix + n, reinterpret_cast<FX3 *>(c->red_tmp), ts,
                &c->launches);
    cudaEventRecord(c->tev_join, ts);
    if (n > 1) {
        const int gi = (n - 1 + kBlock - 1) / kBlock;
        radix_tree_kernel<<<gi, kBlock, 0, s>>>(n, c->keys, c->bn_left, c->bn_right, c->bn_parent, c->leaf_parent,
                                                c->bn_lo, c->bn_hi, c->bn_pref);
        c->launches += 1;
        quad_mark_kernel<<<gp, kBlock, 0, s>>>(n, c->bn_parent, c->leaf_parent, c->bn_lo, c->bn_pref, c->bn_quad,
                                               mask);
    }
    count_kernel<<<(n + 1 + kBlock - 1) / kBlock, kBlock, 0, s>>>(n, c->leaf_parent, c->bn_pref, mask, c->cnt);
    c->launches += scan_exclusive(c->cnt, c->pre, (int64_t)n + 1, c->scan_tmp, s);
    cudaStreamWaitEvent(s, c->tev_join, 0);
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
    A.mask = mask;
    A.prefix = prefix;
    A.mm = c->minmax;
    A.gmax = gmax;
    A.nodes32 = f32 ? c->nodes32 : nullptr;
    A.nodes64 = f32 ? nullptr : c->nodes64;
    A.ex = ex ? *ex : TreeExport{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    A.capacity = 2 * n;
    A.status = c->status;
    emit_kernel<<<gp, kBlock, 0, s>>>(A);
}

}  // namespace hts
