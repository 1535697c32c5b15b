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
constexpr int kExactBlock = 64;

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

// Batched embeddings: the sorted points of segment s occupy positions
// [off[s], off[s+1]) (sorting keeps segments in order), so its tree is the
// pre-order range [pre[off[s]], pre[off[s+1]]).  A lane is active only inside
// its own segment's range; lanes of a warp that straddles two segments walk
// their own trees under the same cursor.
struct SegView {
    const uint64_t *keys;   // sorted keys (segment id in the top bits)
    const int64_t *off;     // segment offsets
    const int *pre;         // pre-order start position per first point
};

__device__ __forceinline__ void segment_range(const SegView &sv, int p, int m, int &root, int &end)
{
    const int sg = (int)(sv.keys[p] >> kSegShift);
    root = sv.pre[sv.off[sg]];
    end = min(sv.pre[sv.off[sg + 1]], m);
}

// One warp walks for the 32 sorted points of chunk `warp`.
template <int GF, bool COUNT, bool SEG>
__device__ __forceinline__ void walk_f32_chunk(int warp, int n, const NodeF *__restrict__ nodes,
                                                const int *__restrict__ n_nodes,
                                                const PointF *__restrict__ spts,
                                                const uint32_t *__restrict__ idx, double2 *frep, double *zi,
                                                unsigned long long *counters, const SegView sv)
{
    const int lane = threadIdx.x & 31;
    const int p = warp * 32 + lane;
    const bool valid = p < n;
    const PointF q = spts[valid ? p : n - 1];
    const float twoil = 2.0f * q.il;
    float rx = 0.f, ry = 0.f, rs = 0.f, z = 0.f;
    const int m = min(*n_nodes, 2 * n);
    int root = 0, end = m;
    if (SEG) segment_range(sv, valid ? p : n - 1, m, root, end);
    int resume = valid ? root : INT_MAX;
    int node = SEG ? __shfl_sync(0xffffffffu, root, 0) : 0;  // lane 0 holds the first segment
    const int stop = SEG ? __reduce_max_sync(0xffffffffu, valid ? end : 0) : m;
    unsigned long long c_acc = 0, c_pair = 0, c_visit = 0;
    while (node < stop) {
        const NodeF c = load_node(nodes, node);
        const bool active = node >= resume && (!SEG || node < end);
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
        // next > node always: a cell's skip exceeds its position (emit writes
        // no cell otherwise) and unwritten slots are zero (empty buckets)
        node = next;
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

// One warp per chunk of 32 sorted points; the warps of a block (blockDim.x /
// 32 <= kWalkBlock / 32, picked by the autotuner) take consecutive chunks, so
// their walks share node data in L1.  The block size does not change results.
template <int GF, bool COUNT, bool SEG>
__global__ void __launch_bounds__(kWalkBlock) walk_f32_kernel(int n, const NodeF *__restrict__ nodes,
                                                              const int *__restrict__ n_nodes,
                                                              const PointF *__restrict__ spts,
                                                              const uint32_t *__restrict__ idx, double2 *frep,
                                                              double *zi, unsigned long long *counters,
                                                              const SegView sv)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp * 32 >= n) return;
    walk_f32_chunk<GF, COUNT, SEG>(warp, n, nodes, n_nodes, spts, idx, frep, zi, counters, sv);
}

template <int GF, bool COUNT, bool SEG>
__device__ __forceinline__ void walk_f64_chunk(int warp, int n, const NodeD *__restrict__ nodes,
                                                const int *__restrict__ n_nodes,
                                                const PointD *__restrict__ spts,
                                                const uint32_t *__restrict__ idx, double2 *frep, double *zi,
                                                unsigned long long *counters, const SegView sv)
{
    const int lane = threadIdx.x & 31;
    const int p = warp * 32 + lane;
    const bool valid = p < n;
    const PointD q = spts[valid ? p : n - 1];
    const double twoil = 2.0 * q.il;
    double rx = 0, ry = 0, rs = 0, z = 0;
    const int m = min(*n_nodes, 2 * n);
    int root = 0, end = m;
    if (SEG) segment_range(sv, valid ? p : n - 1, m, root, end);
    int resume = valid ? root : INT_MAX;
    int node = SEG ? __shfl_sync(0xffffffffu, root, 0) : 0;
    const int stop = SEG ? __reduce_max_sync(0xffffffffu, valid ? end : 0) : m;
    unsigned long long c_acc = 0, c_pair = 0, c_visit = 0;
    while (node < stop) {
        const NodeD c = nodes[node];
        const bool active = node >= resume && (!SEG || node < end);
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
        node = next;  // as in the float32 walk
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

// As walk_f32_kernel, in float64.
template <int GF, bool COUNT, bool SEG>
__global__ void __launch_bounds__(kWalkBlock) walk_f64_kernel(int n, const NodeD *__restrict__ nodes,
                                                              const int *__restrict__ n_nodes,
                                                              const PointD *__restrict__ spts,
                                                              const uint32_t *__restrict__ idx, double2 *frep,
                                                              double *zi, unsigned long long *counters,
                                                              const SegView sv)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp * 32 >= n) return;
    walk_f64_chunk<GF, COUNT, SEG>(warp, n, nodes, n_nodes, spts, idx, frep, zi, counters, sv);
}


// Exact repulsion: one thread per point i, tiles of kExactBlock points j
// staged in shared memory, every pair j != i of the same segment.  A small
// problem has too few i-blocks to fill the GPU, so the j range of each
// i-block is cut into `split` chunks (grid.y): with split == 1 the block
// writes the finished force and Z_i, otherwise raw sums per chunk go to
// `part` and exact_combine_kernel adds them in chunk order (deterministic).
struct ExactArgs {
    int n, split;
    double2 *frep;
    double *zi;
    double4_32a *part;  // [split][n]: sums of k Delta_x, k Delta_y, k s, w
    const unsigned char *seg_of;
    const int64_t *seg_off;
};

__device__ __forceinline__ void exact_ranges(const ExactArgs &A, int i, int &jlo, int &jhi, int &cbeg, int &cend)
{
    // own segment [jlo, jhi); the union over the block's threads, cut into chunks
    int blo = 0, bhi = A.n;
    jlo = 0;
    jhi = A.n;
    if (A.seg_of) {
        const int first = blockIdx.x * kExactBlock, last = min(first + kExactBlock, A.n) - 1;
        const int si = A.seg_of[i < A.n ? i : A.n - 1];
        jlo = (int)A.seg_off[si];
        jhi = (int)A.seg_off[si + 1];
        blo = (int)A.seg_off[A.seg_of[first]];
        bhi = (int)A.seg_off[A.seg_of[last] + 1];
    }
    const int tiles = (bhi - blo + kExactBlock - 1) / kExactBlock;
    const int per = (tiles + A.split - 1) / A.split;
    cbeg = min(bhi, blo + (int)blockIdx.y * per * kExactBlock);
    cend = min(bhi, cbeg + per * kExactBlock);
}

template <int GF>
__global__ void __launch_bounds__(kExactBlock) exact_f32_kernel(const PointF *__restrict__ pts, ExactArgs A)
{
    __shared__ PointF tile[kExactBlock];
    const int n = A.n;
    const int i = blockIdx.x * kExactBlock + threadIdx.x;
    int jlo, jhi, cbeg, cend;
    exact_ranges(A, i, jlo, jhi, cbeg, cend);
    const PointF q = pts[i < n ? i : n - 1];
    const float twoil = 2.0f * q.il;
    float rx = 0.f, ry = 0.f, rs = 0.f, z = 0.f;
    for (int base = cbeg; base < cend; base += kExactBlock) {
        int j = base + threadIdx.x;
        if (j < cend) tile[threadIdx.x] = pts[j];
        __syncthreads();
        const int cnt = min(kExactBlock, cend - base);
        for (int k = 0; k < cnt; ++k) {
            const int jj = base + k;
            if (jj == i || jj < jlo || jj >= jhi) continue;
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
    if (i >= n) return;
    if (A.split > 1) {
        A.part[(size_t)blockIdx.y * n + i] = make_double4_32a(rx, ry, rs, z);
        return;
    }
    double x = (double)q.xh + (double)q.xl, y = (double)q.yh + (double)q.yl;
    double il = (double)q.il;
    double rsd = il * (double)rs;
    A.frep[i] = make_double2(4.0 * il * ((double)rx + rsd * x), 4.0 * il * ((double)ry + rsd * y));
    A.zi[i] = (double)z;
}

template <int GF>
__global__ void __launch_bounds__(kExactBlock) exact_f64_kernel(const PointD *__restrict__ pts, ExactArgs A)
{
    __shared__ PointD tile[kExactBlock];
    const int n = A.n;
    const int i = blockIdx.x * kExactBlock + threadIdx.x;
    int jlo, jhi, cbeg, cend;
    exact_ranges(A, i, jlo, jhi, cbeg, cend);
    const PointD q = pts[i < n ? i : n - 1];
    const double twoil = 2.0 * q.il;
    double rx = 0, ry = 0, rs = 0, z = 0;
    for (int base = cbeg; base < cend; base += kExactBlock) {
        int j = base + threadIdx.x;
        if (j < cend) tile[threadIdx.x] = pts[j];
        __syncthreads();
        const int cnt = min(kExactBlock, cend - base);
        for (int k = 0; k < cnt; ++k) {
            const int jj = base + k;
            if (jj == i || jj < jlo || jj >= jhi) continue;
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
    if (i >= n) return;
    if (A.split > 1) {
        A.part[(size_t)blockIdx.y * n + i] = make_double4_32a(rx, ry, rs, z);
        return;
    }
    double rsd = q.il * rs;
    A.frep[i] = make_double2(4.0 * q.il * (rx + rsd * q.x), 4.0 * q.il * (ry + rsd * q.y));
    A.zi[i] = z;
}

// Sums of the chunks of each point in chunk order, then the per-point factors.
template <typename PT>
__global__ void exact_combine_kernel(const PT *__restrict__ pts, ExactArgs A)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    double rx = 0, ry = 0, rs = 0, z = 0;
    for (int c = 0; c < A.split; ++c) {
        const double4_32a v = A.part[(size_t)c * A.n + i];
        rx += v.x;
        ry += v.y;
        rs += v.z;
        z += v.w;
    }
    const PT q = pts[i];
    double x, y, il;
    point_xy_il(q, x, y, il);
    const double rsd = il * rs;
    A.frep[i] = make_double2(4.0 * il * (rx + rsd * x), 4.0 * il * (ry + rsd * y));
    A.zi[i] = z;
}

}  // namespace

void launch_walk(hts_ctx *c)
{
    const int n = (int)c->n;
    const int warps = (n + 31) / 32;
    const int wb = c->walk_block;  // 32 .. kWalkBlock threads, a multiple of 32
    const int blocks = (warps * 32 + wb - 1) / wb;
    const bool cnt = c->counters_on != 0;  // counters accumulate while enabled
    const bool seg = c->nseg > 1;
    const SegView sv{c->keys, c->seg_off, c->pre};
    c->launches += 1;
#define HTS_WALK(P, NODES, SPTS, GF, CT, SG)                                                             \
    walk_##P##_kernel<GF, CT, SG><<<blocks, wb, 0, c->stream>>>(n, NODES, c->n_nodes, SPTS, c->idx, \
                                                                         c->frep, c->zi, c->counters, sv)
#define HTS_WALK_ALL(P, NODES, SPTS)                                                   \
    if (c->cfg.grad_form == HTS_EXACT_KL) {                                             \
        if (cnt) { if (seg) HTS_WALK(P, NODES, SPTS, 0, true, true); else HTS_WALK(P, NODES, SPTS, 0, true, false); } \
        else { if (seg) HTS_WALK(P, NODES, SPTS, 0, false, true); else HTS_WALK(P, NODES, SPTS, 0, false, false); } \
    } else {                                                                            \
        if (cnt) { if (seg) HTS_WALK(P, NODES, SPTS, 1, true, true); else HTS_WALK(P, NODES, SPTS, 1, true, false); } \
        else { if (seg) HTS_WALK(P, NODES, SPTS, 1, false, true); else HTS_WALK(P, NODES, SPTS, 1, false, false); } \
    }
    if (c->cfg.precision == HTS_FP32_MIXED) {
        HTS_WALK_ALL(f32, c->nodes32, c->spts32)
    } else {
        HTS_WALK_ALL(f64, c->nodes64, c->spts64)
    }
#undef HTS_WALK_ALL
#undef HTS_WALK
}

int exact_split(int64_t n)
{
    constexpr int64_t kTargetBlocks = 1216;  // 8 blocks of 64 threads on each of 152 SMs
    const int64_t blocks = (n + kExactBlock - 1) / kExactBlock;
    if (blocks <= 0 || blocks >= kTargetBlocks) return 1;
    return (int)std::min<int64_t>(blocks, (kTargetBlocks + blocks - 1) / blocks);
}

void launch_exact(hts_ctx *c)
{
    ExactArgs A;
    A.n = (int)c->n;
    A.split = exact_split(c->n);
    A.frep = c->frep;
    A.zi = c->zi;
    A.part = reinterpret_cast<double4_32a *>(c->exact_part);
    A.seg_of = c->nseg > 1 ? c->seg_of : nullptr;
    A.seg_off = c->seg_off;
    const dim3 grid((unsigned)((A.n + kExactBlock - 1) / kExactBlock), (unsigned)A.split);
    const int cb = (A.n + 255) / 256;
    c->launches += A.split > 1 ? 2 : 1;
    if (c->cfg.precision == HTS_FP32_MIXED) {
        if (c->cfg.grad_form == HTS_EXACT_KL)
            exact_f32_kernel<0><<<grid, kExactBlock, 0, c->stream>>>(c->pts32, A);
        else
            exact_f32_kernel<1><<<grid, kExactBlock, 0, c->stream>>>(c->pts32, A);
        if (A.split > 1) exact_combine_kernel<PointF><<<cb, 256, 0, c->stream>>>(c->pts32, A);
    } else {
        if (c->cfg.grad_form == HTS_EXACT_KL)
            exact_f64_kernel<0><<<grid, kExactBlock, 0, c->stream>>>(c->pts64, A);
        else
            exact_f64_kernel<1><<<grid, kExactBlock, 0, c->stream>>>(c->pts64, A);
        if (A.split > 1) exact_combine_kernel<PointD><<<cb, 256, 0, c->stream>>>(c->pts64, A);
    }
}

}  // namespace hts
