// traverse.cu -- Barnes-Hut repulsion (Sec. 4.2, Eq. CellApproximation) and
// the exact O(n^2) repulsion (Eq. KlGradientHyperbolicSplit, second sum).
//
// Warp-cooperative tree walk.  A warp takes 32 consecutive points in key
// order (neighbouring cells, so the lanes' walks overlap) and visits the
// pre-order node array with one warp-uniform cursor:
//   - at an internal cell every active lane tests its own criterion
//     r_cell / d(y_i, y_cell) < theta, written as delta_i,cell > thr_cell
//     with thr = cosh(r_cell / theta) - 1 (cosh is increasing, so the test is
//     exact and needs no transcendental);  a lane that accepts adds the cell
//     term N_cell w^2 d dd/dy_i and becomes inactive until the cursor leaves
//     the cell's subtree (pre-order index >= skip);
//   - the warp descends (cursor + 1) if any active lane rejected the cell,
//     otherwise it jumps to skip;
//   - leaves add the exact pair term for every active lane, except the lane
//     whose own point it is; depth-29 buckets add each of their points.
// Each lane therefore accumulates exactly the terms of its own depth-first
// walk; the warp visits the union of the 32 walks.  Node loads are
// warp-uniform (one sector, broadcast) and stay in L1/L2.
//
// Per lane the pair term is reduced to a scalar times (Delta, s) and a w
// for Z (see pair_terms_* in hts_internal.cuh); the result per point is
//   F_rep,i = 4 il_i (R_Delta + il_i R_s y_i),   Z_i = sum N w,
// written to the point's original index.
#include <limits.h>

#include <algorithm>

#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kWalkBlock = 256;
constexpr bool kWalkPairs = true;  // float32 walk with two queries per lane
constexpr int kExactBlock = 256;

__device__ __forceinline__ NodeF load_node(const NodeF *__restrict__ nodes, int k)
{
    const float4 *p = reinterpret_cast<const float4 *>(nodes + k);
    float4 a = __ldg(p), b = __ldg(p + 1);
    NodeF r;
    r.xh = a.x;
    r.yh = a.y;
    r.xl = a.z;
    r.yl = a.w;
    r.il = b.x;
    r.thr = b.y;
    r.count = __float_as_int(b.z);
    r.skip = __float_as_int(b.w);
    return r;
}

// One warp walks for the 32 sorted points of chunk `warp`.
template <int GF, bool COUNT>
__device__ __forceinline__ void walk_f32_chunk(int warp, int n, const NodeF *__restrict__ nodes,
                                                const int *__restrict__ n_nodes,
                                                const PointF *__restrict__ spts,
                                                const uint32_t *__restrict__ idx, double2 *frep, double *zi,
                                                unsigned long long *counters, int *status)
{
    const int lane = threadIdx.x & 31;
    const int p = warp * 32 + lane;
    const bool valid = p < n;
    const PointF q = spts[valid ? p : n - 1];
    const float twoil = 2.0f * q.il;
    float rx = 0.f, ry = 0.f, rs = 0.f, z = 0.f;
    const int m = min(*n_nodes, 2 * n);
    int resume = valid ? 0 : INT_MAX;
    int node = 0;
    unsigned long long c_acc = 0, c_pair = 0, c_visit = 0;
    while (node < m) {
        const NodeF c = load_node(nodes, node);
        const bool active = node >= resume;
        int next = node + 1;
        if (c.count >= 2) {
            float dx = (q.xh - c.xh) + (q.xl - c.xl);
            float dy = (q.yh - c.yh) + (q.yl - c.yl);
            float s = fmaf(dx, dx, dy * dy);
            float delta = s * twoil * c.il;
            bool acc = active && delta > c.thr;
            if (acc) {
                PairF t = pair_terms_f32<GF>(delta);
                float mult = (float)c.count;
                float k = mult * t.rep * c.il;
                rx = fmaf(k, dx, rx);
                ry = fmaf(k, dy, ry);
                rs = fmaf(k, s, rs);
                z = fmaf(mult, t.w, z);
                resume = c.skip;
                if (COUNT) ++c_acc;
            }
            if (!__any_sync(0xffffffffu, active && !acc)) next = c.skip;
        } else if (c.count == 1) {
            if (active && __float_as_int(c.thr) != p) {
                float dx = (q.xh - c.xh) + (q.xl - c.xl);
                float dy = (q.yh - c.yh) + (q.yl - c.yl);
                float s = fmaf(dx, dx, dy * dy);
                PairF t = pair_terms_f32<GF>(s * twoil * c.il);
                float k = t.rep * c.il;
                rx = fmaf(k, dx, rx);
                ry = fmaf(k, dy, ry);
                rs = fmaf(k, s, rs);
                z += t.w;
                if (COUNT) ++c_pair;
            }
        } else {
            const int lo = __float_as_int(c.thr), cnt = -c.count;
            if (active && lo >= 0 && cnt > 0 && lo + cnt <= n) {
                for (int k2 = 0; k2 < cnt; ++k2) {
                    if (lo + k2 == p) continue;
                    PointF o = spts[lo + k2];
                    float dx = (q.xh - o.xh) + (q.xl - o.xl);
                    float dy = (q.yh - o.yh) + (q.yl - o.yl);
                    float s = fmaf(dx, dx, dy * dy);
                    PairF t = pair_terms_f32<GF>(s * twoil * o.il);
                    float k = t.rep * o.il;
                    rx = fmaf(k, dx, rx);
                    ry = fmaf(k, dy, ry);
                    rs = fmaf(k, s, rs);
                    z += t.w;
                    if (COUNT) ++c_pair;
                }
            }
        }
        if (COUNT && lane == 0) ++c_visit;
        node = max(next, node + 1);  // always advances: the loop ends within m visits
    }
    if (valid) {
        const uint32_t i = idx[p];
        double x = (double)q.xh + (double)q.xl, y = (double)q.yh + (double)q.yl;
        double il = (double)q.il;
        double rsd = il * (double)rs;
        frep[i] = make_double2(4.0 * il * ((double)rx + rsd * x), 4.0 * il * ((double)ry + rsd * y));
        zi[i] = (double)z;
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            c_acc += __shfl_xor_sync(0xffffffffu, c_acc, o);
            c_pair += __shfl_xor_sync(0xffffffffu, c_pair, o);
        }
        if (lane == 0) {
            atomicAdd(&counters[0], c_acc);
            atomicAdd(&counters[1], c_pair);
            atomicAdd(&counters[2], c_visit);
            atomicAdd(&counters[3], (unsigned long long)min(32, n - warp * 32));
        }
    }
}

// One warp per chunk of 32 sorted points; the 8 warps of a block take
// consecutive chunks, so their walks share node data in L1.
template <int GF, bool COUNT>
__global__ void __launch_bounds__(kWalkBlock) walk_f32_kernel(int n, const NodeF *__restrict__ nodes,
                                                              const int *__restrict__ n_nodes,
                                                              const PointF *__restrict__ spts,
                                                              const uint32_t *__restrict__ idx, double2 *frep,
                                                              double *zi, unsigned long long *counters,
                                                              int *status)
{
    const int warp = (blockIdx.x * kWalkBlock + threadIdx.x) >> 5;
    if (warp * 32 >= n) return;
    walk_f32_chunk<GF, COUNT>(warp, n, nodes, n_nodes, spts, idx, frep, zi, counters, status);
}

// ---- float32 walk with two queries per lane -------------------------------
// A warp takes 64 consecutive sorted points; lane l holds points 2l and 2l+1
// (neighbours in key order, so their walks almost coincide).  The two queries'
// coordinates, accumulators and pair terms live in the two halves of float2
// registers and use the paired float32 instructions (add / mul / fma on
// f32x2), so node loads, votes, loop control and most arithmetic are shared by
// two queries; only the special-function operations stay scalar.  Each query
// keeps its own resume index, so it still accumulates exactly its own walk.
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }

template <int GF>
__device__ __forceinline__ void pair_terms_f32x2(float2 D, float2 &W, float2 &REP)
{
    D = make_float2(fmaxf(D.x, 1e-30f), fmaxf(D.y, 1e-30f));
    const float2 X = __fmul2_rn(D, __fadd2_rn(D, bc2(2.0f)));          // sinh(d)^2
    const float2 RS = make_float2(rsqrtf(X.x), rsqrtf(X.y));            // 1 / sinh(d)
    const float2 T = __fmul2_rn(X, RS);                                 // sinh(d)
    float2 FS = bc2(-8.0f / 693.0f);                                    // d / sinh(d), series
    FS = __ffma2_rn(FS, D, bc2(8.0f / 315.0f));
    FS = __ffma2_rn(FS, D, bc2(-2.0f / 35.0f));
    FS = __ffma2_rn(FS, D, bc2(2.0f / 15.0f));
    FS = __ffma2_rn(FS, D, bc2(-1.0f / 3.0f));
    FS = __ffma2_rn(FS, D, bc2(1.0f));
    const float2 A = __fadd2_rn(__fadd2_rn(bc2(1.0f), D), T);
    const float2 L = __fmul2_rn(make_float2(__log2f(A.x), __log2f(A.y)), bc2(0.69314718f));  // log = log2 * ln 2
    const float2 LR = __fmul2_rn(L, RS);
    const float2 TF = __fmul2_rn(T, FS);
    const bool s0 = D.x < 0.1f, s1 = D.y < 0.1f;
    const float2 F = make_float2(s0 ? FS.x : LR.x, s1 ? FS.y : LR.y);   // d / sinh(d)
    const float2 Dd = make_float2(s0 ? TF.x : L.x, s1 ? TF.y : L.y);    // d
    const float2 U = __ffma2_rn(Dd, Dd, bc2(1.0f));
    W = make_float2(__fdividef(1.0f, U.x), __fdividef(1.0f, U.y));
    const float2 ATT = __fmul2_rn(W, GF == 0 ? F : RS);
    REP = __fmul2_rn(W, ATT);
}

template <int GF, bool COUNT>
__device__ __forceinline__ void walk_f32x2_chunk(int warp, int n, const NodeF *__restrict__ nodes,
                                                  const int *__restrict__ n_nodes,
                                                  const PointF *__restrict__ spts,
                                                  const uint32_t *__restrict__ idx, double2 *frep, double *zi,
                                                  unsigned long long *counters)
{
    const int lane = threadIdx.x & 31;
    const int p0 = warp * 64 + 2 * lane, p1 = p0 + 1;
    const bool v0 = p0 < n, v1 = p1 < n;
    const PointF q0 = spts[v0 ? p0 : n - 1], q1 = spts[v1 ? p1 : n - 1];
    const float2 QXH = make_float2(q0.xh, q1.xh), QYH = make_float2(q0.yh, q1.yh);
    const float2 QXL = make_float2(q0.xl, q1.xl), QYL = make_float2(q0.yl, q1.yl);
    const float2 TWOIL = make_float2(2.0f * q0.il, 2.0f * q1.il);
    float2 RX = bc2(0.f), RY = bc2(0.f), RS = bc2(0.f), Z = bc2(0.f);
    const int m = min(*n_nodes, 2 * n);
    int res0 = v0 ? 0 : INT_MAX, res1 = v1 ? 0 : INT_MAX;
    int node = 0;
    unsigned long long c_acc = 0, c_pair = 0, c_visit = 0;
    while (node < m) {
        const NodeF c = load_node(nodes, node);
        const bool a0 = node >= res0, a1 = node >= res1;
        int next = node + 1;
        if (c.count >= 2) {
            const float2 DX = __fadd2_rn(__fadd2_rn(QXH, bc2(-c.xh)), __fadd2_rn(QXL, bc2(-c.xl)));
            const float2 DY = __fadd2_rn(__fadd2_rn(QYH, bc2(-c.yh)), __fadd2_rn(QYL, bc2(-c.yl)));
            const float2 S = __ffma2_rn(DX, DX, __fmul2_rn(DY, DY));
            const float2 D = __fmul2_rn(S, __fmul2_rn(TWOIL, bc2(c.il)));
            const bool acc0 = a0 && D.x > c.thr, acc1 = a1 && D.y > c.thr;
            if (acc0 || acc1) {
                float2 W, REP;
                pair_terms_f32x2<GF>(D, W, REP);
                const float N = (float)c.count;
                const float2 M = make_float2(acc0 ? N : 0.0f, acc1 ? N : 0.0f);
                const float2 K = __fmul2_rn(__fmul2_rn(M, REP), bc2(c.il));
                RX = __ffma2_rn(K, DX, RX);
                RY = __ffma2_rn(K, DY, RY);
                RS = __ffma2_rn(K, S, RS);
                Z = __ffma2_rn(M, W, Z);
                if (acc0) res0 = c.skip;
                if (acc1) res1 = c.skip;
                if (COUNT) c_acc += (unsigned)acc0 + (unsigned)acc1;
            }
            if (!__any_sync(0xffffffffu, (a0 && !acc0) || (a1 && !acc1))) next = c.skip;
        } else if (c.count == 1) {
            const int pos = __float_as_int(c.thr);
            const bool i0 = a0 && pos != p0, i1 = a1 && pos != p1;
            if (i0 || i1) {
                const float2 DX = __fadd2_rn(__fadd2_rn(QXH, bc2(-c.xh)), __fadd2_rn(QXL, bc2(-c.xl)));
                const float2 DY = __fadd2_rn(__fadd2_rn(QYH, bc2(-c.yh)), __fadd2_rn(QYL, bc2(-c.yl)));
                const float2 S = __ffma2_rn(DX, DX, __fmul2_rn(DY, DY));
                const float2 D = __fmul2_rn(S, __fmul2_rn(TWOIL, bc2(c.il)));
                float2 W, REP;
                pair_terms_f32x2<GF>(D, W, REP);
                const float2 M = make_float2(i0 ? 1.0f : 0.0f, i1 ? 1.0f : 0.0f);
                const float2 K = __fmul2_rn(__fmul2_rn(M, REP), bc2(c.il));
                RX = __ffma2_rn(K, DX, RX);
                RY = __ffma2_rn(K, DY, RY);
                RS = __ffma2_rn(K, S, RS);
                Z = __fadd2_rn(Z, __fmul2_rn(M, W));
                if (COUNT) c_pair += (unsigned)i0 + (unsigned)i1;
            }
        } else {
            const int lo = __float_as_int(c.thr), cnt = -c.count;
            if ((a0 || a1) && lo >= 0 && cnt > 0 && lo + cnt <= n) {
                for (int k2 = 0; k2 < cnt; ++k2) {
                    const int pj = lo + k2;
                    const bool i0 = a0 && pj != p0, i1 = a1 && pj != p1;
                    const PointF o = spts[pj];
                    const float2 DX = __fadd2_rn(__fadd2_rn(QXH, bc2(-o.xh)), __fadd2_rn(QXL, bc2(-o.xl)));
                    const float2 DY = __fadd2_rn(__fadd2_rn(QYH, bc2(-o.yh)), __fadd2_rn(QYL, bc2(-o.yl)));
                    const float2 S = __ffma2_rn(DX, DX, __fmul2_rn(DY, DY));
                    const float2 D = __fmul2_rn(S, __fmul2_rn(TWOIL, bc2(o.il)));
                    float2 W, REP;
                    pair_terms_f32x2<GF>(D, W, REP);
                    const float2 M = make_float2(i0 ? 1.0f : 0.0f, i1 ? 1.0f : 0.0f);
                    const float2 K = __fmul2_rn(__fmul2_rn(M, REP), bc2(o.il));
                    RX = __ffma2_rn(K, DX, RX);
                    RY = __ffma2_rn(K, DY, RY);
                    RS = __ffma2_rn(K, S, RS);
                    Z = __fadd2_rn(Z, __fmul2_rn(M, W));
                    if (COUNT) c_pair += (unsigned)i0 + (unsigned)i1;
                }
            }
        }
        if (COUNT && lane == 0) ++c_visit;
        node = max(next, node + 1);  // always advances: the loop ends within m visits
    }
    auto finish = [&](int p, const PointF &q, float rx, float ry, float rs, float z) {
        const uint32_t i = idx[p];
        double x = (double)q.xh + (double)q.xl, y = (double)q.yh + (double)q.yl;
        double il = (double)q.il;
        double rsd = il * (double)rs;
        frep[i] = make_double2(4.0 * il * ((double)rx + rsd * x), 4.0 * il * ((double)ry + rsd * y));
        zi[i] = (double)z;
    };
    if (v0) finish(p0, q0, RX.x, RY.x, RS.x, Z.x);
    if (v1) finish(p1, q1, RX.y, RY.y, RS.y, Z.y);
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            c_acc += __shfl_xor_sync(0xffffffffu, c_acc, o);
            c_pair += __shfl_xor_sync(0xffffffffu, c_pair, o);
        }
        if (lane == 0) {
            atomicAdd(&counters[0], c_acc);
            atomicAdd(&counters[1], c_pair);
            atomicAdd(&counters[2], c_visit);
            atomicAdd(&counters[3], (unsigned long long)min(64, n - warp * 64));
        }
    }
}

template <int GF, bool COUNT>
__global__ void __launch_bounds__(kWalkBlock) walk_f32x2_kernel(int n, const NodeF *__restrict__ nodes,
                                                                const int *__restrict__ n_nodes,
                                                                const PointF *__restrict__ spts,
                                                                const uint32_t *__restrict__ idx, double2 *frep,
                                                                double *zi, unsigned long long *counters)
{
    const int warp = (blockIdx.x * kWalkBlock + threadIdx.x) >> 5;
    if (warp * 64 >= n) return;
    walk_f32x2_chunk<GF, COUNT>(warp, n, nodes, n_nodes, spts, idx, frep, zi, counters);
}


// One warp walks for the 32 sorted points of chunk `warp`.
template <int GF, bool COUNT>
__device__ __forceinline__ void walk_f64_chunk(int warp, int n, const NodeD *__restrict__ nodes,
                                                const int *__restrict__ n_nodes,
                                                const PointD *__restrict__ spts,
                                                const uint32_t *__restrict__ idx, double2 *frep, double *zi,
                                                unsigned long long *counters, int *status)
{
    const int lane = threadIdx.x & 31;
    const int p = warp * 32 + lane;
    const bool valid = p < n;
    const PointD q = spts[valid ? p : n - 1];
    const double twoil = 2.0 * q.il;
    double rx = 0, ry = 0, rs = 0, z = 0;
    const int m = min(*n_nodes, 2 * n);
    int resume = valid ? 0 : INT_MAX;
    int node = 0;
    unsigned long long c_acc = 0, c_pair = 0, c_visit = 0;
    while (node < m) {
        const NodeD c = nodes[node];
        const bool active = node >= resume;
        int next = node + 1;
        if (c.count >= 2) {
            double dx = q.x - c.x, dy = q.y - c.y;
            double s = fma(dx, dx, dy * dy);
            double delta = s * twoil * c.il;
            bool acc = active && delta > c.thr;
            if (acc) {
                PairD t = pair_terms_f64<GF>(delta);
                double mult = (double)c.count;
                double k = mult * t.rep * c.il;
                rx = fma(k, dx, rx);
                ry = fma(k, dy, ry);
                rs = fma(k, s, rs);
                z = fma(mult, t.w, z);
                resume = c.skip;
                if (COUNT) ++c_acc;
            }
            if (!__any_sync(0xffffffffu, active && !acc)) next = c.skip;
        } else if (c.count == 1) {
            if (active && c.pos != p) {
                double dx = q.x - c.x, dy = q.y - c.y;
                double s = fma(dx, dx, dy * dy);
                PairD t = pair_terms_f64<GF>(s * twoil * c.il);
                double k = t.rep * c.il;
                rx = fma(k, dx, rx);
                ry = fma(k, dy, ry);
                rs = fma(k, s, rs);
                z += t.w;
                if (COUNT) ++c_pair;
            }
        } else {
            const int lo = c.pos, cnt = -c.count;
            if (active && lo >= 0 && cnt > 0 && lo + cnt <= n) {
                for (int k2 = 0; k2 < cnt; ++k2) {
                    if (lo + k2 == p) continue;
                    PointD o = spts[lo + k2];
                    double dx = q.x - o.x, dy = q.y - o.y;
                    double s = fma(dx, dx, dy * dy);
                    PairD t = pair_terms_f64<GF>(s * twoil * o.il);
                    double k = t.rep * o.il;
                    rx = fma(k, dx, rx);
                    ry = fma(k, dy, ry);
                    rs = fma(k, s, rs);
                    z += t.w;
                    if (COUNT) ++c_pair;
                }
            }
        }
        if (COUNT && lane == 0) ++c_visit;
        node = max(next, node + 1);
    }
    if (valid) {
        const uint32_t i = idx[p];
        double rsd = q.il * rs;
        frep[i] = make_double2(4.0 * q.il * (rx + rsd * q.x), 4.0 * q.il * (ry + rsd * q.y));
        zi[i] = z;
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            c_acc += __shfl_xor_sync(0xffffffffu, c_acc, o);
            c_pair += __shfl_xor_sync(0xffffffffu, c_pair, o);
        }
        if (lane == 0) {
            atomicAdd(&counters[0], c_acc);
            atomicAdd(&counters[1], c_pair);
            atomicAdd(&counters[2], c_visit);
            atomicAdd(&counters[3], (unsigned long long)min(32, n - warp * 32));
        }
    }
}

// One warp per chunk of 32 sorted points; the 8 warps of a block take
// consecutive chunks, so their walks share node data in L1.
template <int GF, bool COUNT>
__global__ void __launch_bounds__(kWalkBlock) walk_f64_kernel(int n, const NodeD *__restrict__ nodes,
                                                              const int *__restrict__ n_nodes,
                                                              const PointD *__restrict__ spts,
                                                              const uint32_t *__restrict__ idx, double2 *frep,
                                                              double *zi, unsigned long long *counters,
                                                              int *status)
{
    const int warp = (blockIdx.x * kWalkBlock + threadIdx.x) >> 5;
    if (warp * 32 >= n) return;
    walk_f64_chunk<GF, COUNT>(warp, n, nodes, n_nodes, spts, idx, frep, zi, counters, status);
}


// Exact repulsion: one thread per point i, tiles of 256 points j staged in
// shared memory, every pair j != i.
template <int GF>
__global__ void __launch_bounds__(kExactBlock) exact_f32_kernel(int n, const PointF *__restrict__ pts, double2 *frep,
                                                                double *zi)
{
    __shared__ PointF tile[kExactBlock];
    const int i = blockIdx.x * kExactBlock + threadIdx.x;
    const PointF q = pts[i < n ? i : n - 1];
    const float twoil = 2.0f * q.il;
    float rx = 0.f, ry = 0.f, rs = 0.f, z = 0.f;
    for (int base = 0; base < n; base += kExactBlock) {
        int j = base + threadIdx.x;
        if (j < n) tile[threadIdx.x] = pts[j];
        __syncthreads();
        const int cnt = min(kExactBlock, n - base);
        for (int k = 0; k < cnt; ++k) {
            if (base + k == i) continue;
            const PointF o = tile[k];
            float dx = (q.xh - o.xh) + (q.xl - o.xl);
            float dy = (q.yh - o.yh) + (q.yl - o.yl);
            float s = fmaf(dx, dx, dy * dy);
            PairF t = pair_terms_f32<GF>(s * twoil * o.il);
            float kk = t.rep * o.il;
            rx = fmaf(kk, dx, rx);
            ry = fmaf(kk, dy, ry);
            rs = fmaf(kk, s, rs);
            z += t.w;
        }
        __syncthreads();
    }
    if (i < n) {
        double x = (double)q.xh + (double)q.xl, y = (double)q.yh + (double)q.yl;
        double il = (double)q.il;
        double rsd = il * (double)rs;
        frep[i] = make_double2(4.0 * il * ((double)rx + rsd * x), 4.0 * il * ((double)ry + rsd * y));
        zi[i] = (double)z;
    }
}

template <int GF>
__global__ void __launch_bounds__(kExactBlock) exact_f64_kernel(int n, const PointD *__restrict__ pts, double2 *frep,
                                                                double *zi)
{
    __shared__ PointD tile[kExactBlock];
    const int i = blockIdx.x * kExactBlock + threadIdx.x;
    const PointD q = pts[i < n ? i : n - 1];
    const double twoil = 2.0 * q.il;
    double rx = 0, ry = 0, rs = 0, z = 0;
    for (int base = 0; base < n; base += kExactBlock) {
        int j = base + threadIdx.x;
        if (j < n) tile[threadIdx.x] = pts[j];
        __syncthreads();
        const int cnt = min(kExactBlock, n - base);
        for (int k = 0; k < cnt; ++k) {
            if (base + k == i) continue;
            const PointD o = tile[k];
            double dx = q.x - o.x, dy = q.y - o.y;
            double s = fma(dx, dx, dy * dy);
            PairD t = pair_terms_f64<GF>(s * twoil * o.il);
            double kk = t.rep * o.il;
            rx = fma(kk, dx, rx);
            ry = fma(kk, dy, ry);
            rs = fma(kk, s, rs);
            z += t.w;
        }
        __syncthreads();
    }
    if (i < n) {
        double rsd = q.il * rs;
        frep[i] = make_double2(4.0 * q.il * (rx + rsd * q.x), 4.0 * q.il * (ry + rsd * q.y));
        zi[i] = z;
    }
}

}  // namespace

void launch_walk(hts_ctx *c)
{
    const int n = (int)c->n;
    const int warps = (n + 31) / 32;
    const int blocks = (warps * 32 + kWalkBlock - 1) / kWalkBlock;
    const bool cnt = c->counters_on != 0;  // counters accumulate while enabled
    c->launches += 1;
    if (c->cfg.precision == HTS_FP32_MIXED && kWalkPairs) {
        const int blocks2 = ((n + 63) / 64 * 32 + kWalkBlock - 1) / kWalkBlock;
#define HTS_WALK(GF, CT) \
    walk_f32x2_kernel<GF, CT><<<blocks2, kWalkBlock, 0, c->stream>>>(n, c->nodes32, c->n_nodes, c->spts32, \
                                                                     c->idx, c->frep, c->zi, c->counters)
        if (c->cfg.grad_form == HTS_EXACT_KL) {
            if (cnt) HTS_WALK(0, true); else HTS_WALK(0, false);
        } else {
            if (cnt) HTS_WALK(1, true); else HTS_WALK(1, false);
        }
#undef HTS_WALK
    } else if (c->cfg.precision == HTS_FP32_MIXED) {
#define HTS_WALK(GF, CT) \
    walk_f32_kernel<GF, CT><<<blocks, kWalkBlock, 0, c->stream>>>(n, c->nodes32, c->n_nodes, c->spts32, c->idx, \
                                                                  c->frep, c->zi, c->counters, c->status)
        if (c->cfg.grad_form == HTS_EXACT_KL) {
            if (cnt) HTS_WALK(0, true); else HTS_WALK(0, false);
        } else {
            if (cnt) HTS_WALK(1, true); else HTS_WALK(1, false);
        }
#undef HTS_WALK
    } else {
#define HTS_WALK(GF, CT) \
    walk_f64_kernel<GF, CT><<<blocks, kWalkBlock, 0, c->stream>>>(n, c->nodes64, c->n_nodes, c->spts64, c->idx, \
                                                                  c->frep, c->zi, c->counters, c->status)
        if (c->cfg.grad_form == HTS_EXACT_KL) {
            if (cnt) HTS_WALK(0, true); else HTS_WALK(0, false);
        } else {
            if (cnt) HTS_WALK(1, true); else HTS_WALK(1, false);
        }
#undef HTS_WALK
    }
}

void launch_exact(hts_ctx *c)
{
    const int n = (int)c->n;
    const int blocks = (n + kExactBlock - 1) / kExactBlock;
    c->launches += 1;
    if (c->cfg.precision == HTS_FP32_MIXED) {
        if (c->cfg.grad_form == HTS_EXACT_KL)
            exact_f32_kernel<0><<<blocks, kExactBlock, 0, c->stream>>>(n, c->pts32, c->frep, c->zi);
        else
            exact_f32_kernel<1><<<blocks, kExactBlock, 0, c->stream>>>(n, c->pts32, c->frep, c->zi);
    } else {
        if (c->cfg.grad_form == HTS_EXACT_KL)
            exact_f64_kernel<0><<<blocks, kExactBlock, 0, c->stream>>>(n, c->pts64, c->frep, c->zi);
        else
            exact_f64_kernel<1><<<blocks, kExactBlock, 0, c->stream>>>(n, c->pts64, c->frep, c->zi);
    }
}

}  // namespace hts
