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

// One node, read through the non-coherent path: a single 256-bit load (the
// node array comes from cudaMalloc and a node is 32 bytes, so every node is
// 32-byte aligned); two 128-bit loads measured 2% slower.
__device__ __forceinline__ NodeF load_node(const NodeF *__restrict__ nodes, int k)
{
    NodeF r;
    float skipf;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r.xh), "=f"(r.yh), "=f"(r.xl), "=f"(r.yl), "=f"(r.il), "=f"(r.thr), "=f"(r.count), "=f"(skipf)
        : "l"(nodes + k));
    r.skip = __float_as_int(skipf);
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

// Launch order of the walk's blocks.  A walk's chunks differ in cost (dense
// regions have longer walks), and a grid of several waves whose costliest
// blocks start last ends with a tail of few busy SMs.  Every walk therefore
// records, per logical block, the cycles its warps took, and
// walk_order_kernel turns them into the launch order of the next walk:
// costliest first, the cheap blocks filling the end (longest-processing-time
// first).  The mapping of chunks to warps is unchanged, so results do not
// depend on the order.
struct BlockOrder {
    const int *order;  // [0]: grid size the order was made for; [1 + k]: logical block launched k-th
    unsigned *cost;    // per logical block: summed cycles / 64 of its warps (nullptr: not recorded)
};

__device__ __forceinline__ int logical_block(const BlockOrder &bo)
{
    int b = blockIdx.x;
    if (bo.order && bo.order[0] == (int)gridDim.x) {
        const int o = bo.order[1 + blockIdx.x];
        if (o >= 0 && o < (int)gridDim.x) b = o;
    }
    return b;
}

__device__ __forceinline__ void record_cost(const BlockOrder &bo, int b, long long t0)
{
    if (bo.cost && (threadIdx.x & 31) == 0)
        atomicAdd(&bo.cost[b], (unsigned)min((clock64() - t0) >> 6, 0xFFFFFll));
}

// Split walk (small problems, one embedding): the root is never accepted
// (every point lies inside it, and r_cell / d >= 1 > theta), so each point's
// walk is the union of its walks of the subtrees below a cut of the tree at
// depth D.  One warp takes one 32-point chunk and one subtree of the cut (a
// "frontier" entry): it first evaluates the criterion at the entry's
// ancestors (depth 1 .. D-1) -- a lane that accepts one is done with this
// subtree, and the interaction with that ancestor is counted by the first
// frontier entry below it only -- then walks the subtree.  The partial sums
// of the entries are added in entry order by walk_combine_kernel, so every
// lane gets exactly the interactions of its full walk.
constexpr int kMaxSplitDepth = 3;
constexpr int kMaxFrontier = 64;           // 4^3
constexpr int64_t kSplitMaxN = 1 << 19;    // above: chunks alone fill the GPU (a cut measured slower at 1M)
constexpr int64_t kSplitEntries = 1 << 22; // partial-sum buffer: entries x points

struct Frontier {
    int node;                         // subtree root
    int nanc;                         // ancestors below the root
    int anc[kMaxSplitDepth];
    int own;                          // bit k: this entry counts an accepted anc[k]
};

struct SplitView {
    const Frontier *fr;               // nullptr: no split
    const int *count;                 // frontier entries
    void *part;                       // [entry][n] partial sums (float4 / double4)
};

struct NodesF {  // float32 nodes: cell test and skip index
    const NodeF *nodes;
    __device__ bool cell(int k) const { return nodes[k].count >= 2.0f; }
    __device__ int skip(int k) const { return nodes[k].skip; }
};
struct NodesD {  // float64 nodes
    const NodeD *nodes;
    __device__ bool cell(int k) const { return nodes[k].count >= 2; }
    __device__ int skip(int k) const { return nodes[k].skip; }
};

// Per-lane state of the float32 walk: the query point (sorted position p),
// its running sums, and the pre-order index from which the lane is open
// again (a lane that accepts a cell skips the cell's subtree).
struct LaneF {
    float2 qh, ql;  // position as hi / lo float pairs
    float twoil;
    int p;
    float2 rxy, rsz;  // sums of k Delta and of (k s, mult w)
    int resume;
    unsigned long long c_acc, c_pair, c_crit;  // counting walk only
};

// Adds mult times the pair term of (Delta, s, delta) with conformal factor il
// of the other point: a cell's N_cell-weighted term (Eq. CellApproximation)
// or one exact pair (mult = 1).
// (The sums are paired: (rx, ry) += k Delta and (rs, z) += (k, mult) (s, w),
// one fused multiply-add per pair, rounded as the scalar ones.)
template <int GF>
__device__ __forceinline__ void add_pair_f32(LaneF &L, float2 d, float s, float delta, float mult, float il)
{
    const PairF t = pair_terms_f32<GF>(delta);
    const float k = mult * t.rep * il;
    L.rxy = __ffma2_rn(make_float2(k, k), d, L.rxy);
    L.rsz = __ffma2_rn(make_float2(k, mult), make_float2(s, t.w), L.rsz);
}

// The compensated difference y_i - y_j of two hi/lo float pairs and |y_i - y_j|^2.
__device__ __forceinline__ float2 delta_f32(const LaneF &L, float2 h, float2 l, float &s)
{
    const float2 d = delta2(L.qh, L.ql, h, l);
    s = fmaf(d.x, d.x, d.y * d.y);
    return d;
}

// One visit of the warp's cursor at `node` (the node is the same for every
// lane, so the branches on its kind are uniform).  Returns the next cursor:
// at a cell, node + 1 if some open lane rejected it (the warp descends),
// otherwise the index after its subtree; node + 1 after a leaf or bucket.
// BOUNDED: a lane is open only below its own `end` (segments, split walk).
template <int GF, bool COUNT, bool BOUNDED>
__device__ __forceinline__ int visit_f32(int node, int end, LaneF &L, const NodeF *__restrict__ nodes,
                                         const PointF *__restrict__ spts, int n)
{
    const NodeF c = load_node(nodes, node);
    const bool open = node >= L.resume && (!BOUNDED || node < end);
    int next = node + 1;
    if (c.count >= 2) {  // cell: r_cell / d < theta  <=>  delta > thr
        float s;
        const float2 d = delta_f32(L, make_float2(c.xh, c.yh), make_float2(c.xl, c.yl), s);
        const float delta = s * L.twoil * c.il;
        const bool acc = open && delta > c.thr;
        // the pair term runs on every lane when one accepts (no divergent
        // branch); a lane that rejects adds it with weight 0, which leaves its
        // sums unchanged (every term is finite: delta is clamped)
        if (__any_sync(0xffffffffu, acc)) {
            add_pair_f32<GF>(L, d, s, delta, acc ? c.count : 0.0f, c.il);
            L.resume = acc ? c.skip : L.resume;
        }
        if (COUNT) {
            L.c_crit += open ? 1 : 0;
            L.c_acc += acc ? 1 : 0;
        }
        if (!__any_sync(0xffffffffu, open && !acc)) next = c.skip;
    } else if (c.count == 1) {  // single-point leaf: the exact pair (not the lane's own point)
        const bool take = open && __float_as_int(c.thr) != L.p;
        if (__any_sync(0xffffffffu, take)) {  // as at a cell: weight 0 for the other lanes
            float s;
            const float2 d = delta_f32(L, make_float2(c.xh, c.yh), make_float2(c.xl, c.yl), s);
            add_pair_f32<GF>(L, d, s, s * L.twoil * c.il, take ? 1.0f : 0.0f, c.il);
            if (COUNT) L.c_pair += take ? 1 : 0;
        }
    } else {  // depth-29 bucket: each of its points exactly
        const int lo = __float_as_int(c.thr), cnt = (int)(-c.count);
        if (open && lo >= 0 && cnt > 0 && lo + cnt <= n) {
            for (int k2 = 0; k2 < cnt; ++k2) {
                if (lo + k2 == L.p) continue;
                const PointF o = spts[lo + k2];
                float s;
                const float2 d = delta_f32(L, make_float2(o.xh, o.yh), make_float2(o.xl, o.yl), s);
                add_pair_f32<GF>(L, d, s, s * L.twoil * o.il, 1.0f, o.il);
                if (COUNT) ++L.c_pair;
            }
        }
    }
    // next > node always: a cell's skip exceeds its position (emit writes no
    // cell otherwise) and unwritten slots are zero (empty buckets)
    return next;
}

// One warp walks for the 32 sorted points of chunk `warp` (and, split, the
// frontier entry `fi`).
template <int GF, bool COUNT, bool SEG, bool SPLIT>
__device__ __forceinline__ void walk_f32_chunk(int warp, int n, const NodeF *__restrict__ nodes,
                                                const int *__restrict__ n_nodes, const PointF *__restrict__ spts,
                                                const uint32_t *__restrict__ idx, double2 *frep, double *zi,
                                                unsigned long long *counters, const SegView sv,
                                                const SplitView sp, int fi)
{
    const int lane = threadIdx.x & 31;
    LaneF L;
    L.p = warp * 32 + lane;
    const bool valid = L.p < n;
    {
        const PointF q = spts[valid ? L.p : n - 1];
        L.qh = make_float2(q.xh, q.yh);
        L.ql = make_float2(q.xl, q.yl);
        L.twoil = 2.0f * q.il;
    }
    L.rxy = L.rsz = make_float2(0.f, 0.f);
    L.c_acc = L.c_pair = L.c_crit = 0;
    unsigned long long c_visit = 0;
    const int m = min(*n_nodes, 2 * n);
    int root = 0, end = m;
    if (SEG) segment_range(sv, valid ? L.p : n - 1, m, root, end);
    bool live = valid;
    if (SPLIT) {  // frontier entry: ancestors first, then the subtree [node, skip)
        const Frontier F = sp.fr[fi];
#pragma unroll
        for (int k = 0; k < kMaxSplitDepth; ++k) {
            if (k >= F.nanc) break;
            const NodeF a = load_node(nodes, F.anc[k]);
            const bool own = (F.own >> k) & 1;
            float s;
            const float2 d = delta_f32(L, make_float2(a.xh, a.yh), make_float2(a.xl, a.yl), s);
            const float delta = s * L.twoil * a.il;
            if (COUNT) L.c_crit += (live && own) ? 1 : 0;
            if (live && delta > a.thr) {
                if (own) {
                    add_pair_f32<GF>(L, d, s, delta, a.count, a.il);
                    if (COUNT) ++L.c_acc;
                }
                live = false;
            }
        }
        root = F.node;
        end = min(load_node(nodes, F.node).skip, m);
    }
    L.resume = live ? root : INT_MAX;
    int node = SEG ? __shfl_sync(0xffffffffu, root, 0) : root;  // lane 0 holds the first segment
    const int stop = SEG ? __reduce_max_sync(0xffffffffu, valid ? end : 0) : end;
    // four visits per trip and one test of the cursor: in this issue-bound
    // loop the loop-back branch and the cursor tests cost.  The cursor may run
    // up to three nodes past `stop`: past the last node the tree build leaves
    // four empty slots (visited as no-ops), and below it every lane's own
    // bound `end` closes it (BOUNDED).
    constexpr bool kBounded = SEG || SPLIT;
    while (node < stop) {
        if (COUNT && lane == 0) ++c_visit;  // (counted: visits below stop)
        node = visit_f32<GF, COUNT, kBounded>(node, end, L, nodes, spts, n);
        if (COUNT && lane == 0 && node < stop) ++c_visit;
        node = visit_f32<GF, COUNT, kBounded>(node, end, L, nodes, spts, n);
        if (COUNT && lane == 0 && node < stop) ++c_visit;
        node = visit_f32<GF, COUNT, kBounded>(node, end, L, nodes, spts, n);
        if (COUNT && lane == 0 && node < stop) ++c_visit;
        node = visit_f32<GF, COUNT, kBounded>(node, end, L, nodes, spts, n);
    }
    if (SPLIT && valid) {
        reinterpret_cast<float4 *>(sp.part)[(size_t)fi * n + L.p] = make_float4(L.rxy.x, L.rxy.y, L.rsz.x, L.rsz.y);
    } else if (valid) {
        const uint32_t i = idx[L.p];
        double x = (double)L.qh.x + (double)L.ql.x, y = (double)L.qh.y + (double)L.ql.y;
        double il = 0.5 * (double)L.twoil;
        double rsd = il * (double)L.rsz.x;
        frep[i] = make_double2(4.0 * il * ((double)L.rxy.x + rsd * x), 4.0 * il * ((double)L.rxy.y + rsd * y));
        zi[i] = (double)L.rsz.y;
    }
    if (COUNT) {
        unsigned long long c_acc = L.c_acc, c_pair = L.c_pair, c_crit = L.c_crit;
        for (int o = 16; o > 0; o >>= 1) {
            c_acc += __shfl_xor_sync(0xffffffffu, c_acc, o);
            c_pair += __shfl_xor_sync(0xffffffffu, c_pair, o);
            c_crit += __shfl_xor_sync(0xffffffffu, c_crit, o);
        }
        if (lane == 0) {
            atomicAdd(&counters[0], c_acc);
            atomicAdd(&counters[1], c_pair);
            atomicAdd(&counters[2], c_visit);
            atomicAdd(&counters[3], (unsigned long long)min(32, n - warp * 32));
            atomicAdd(&counters[4], c_crit);
        }
    }
}

// One warp per chunk of 32 sorted points; the warps of a block (blockDim.x /
// 32 <= kWalkBlock / 32, picked by the autotuner) take consecutive chunks, so
// their walks share node data in L1.  The block size does not change results.
template <int GF, bool COUNT, bool SEG, bool SPLIT>
__global__ void __launch_bounds__(kWalkBlock) walk_f32_kernel(int n, const NodesF nodes,
                                                              const int *__restrict__ n_nodes,
                                                              const PointF *__restrict__ spts,
                                                              const uint32_t *__restrict__ idx, double2 *frep,
                                                              double *zi, unsigned long long *counters,
                                                              const SegView sv, const SplitView sp,
                                                              const BlockOrder bo)
{
    const int b = logical_block(bo);
    const int warp = (b * blockDim.x + threadIdx.x) >> 5;
    if (warp * 32 >= n) return;
    if (SPLIT && (int)blockIdx.y >= *sp.count) return;
    const long long t0 = clock64();
    walk_f32_chunk<GF, COUNT, SEG, SPLIT>(warp, n, nodes.nodes, n_nodes, spts, idx, frep, zi, counters, sv, sp,
                                          blockIdx.y);
    record_cost(bo, b, t0);
}

template <int GF, bool COUNT, bool SEG, bool SPLIT>
__device__ __forceinline__ void walk_f64_chunk(int warp, int n, const NodeD *__restrict__ nodes,
                                                const int *__restrict__ n_nodes,
                                                const PointD *__restrict__ spts,
                                                const uint32_t *__restrict__ idx, double2 *frep, double *zi,
                                                unsigned long long *counters, const SegView sv,
                                                const SplitView sp, int fi)
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
    unsigned long long c_acc = 0, c_pair = 0, c_visit = 0;
    bool live = valid;
    if (SPLIT) {  // as in the float32 walk
        const Frontier F = sp.fr[fi];
#pragma unroll
        for (int k = 0; k < kMaxSplitDepth; ++k) {
            if (k >= F.nanc) break;
            const NodeD a = nodes[F.anc[k]];
            double dx = q.x - a.x, dy = q.y - a.y;
            double s = fma(dx, dx, dy * dy);
            double delta = s * twoil * a.il;
            if (live && delta > a.thr) {
                if ((F.own >> k) & 1) {
                    PairD t = pair_terms_f64<GF>(delta);
                    double mult = (double)a.count;
                    double kk = mult * t.rep * a.il;
                    rx = fma(kk, dx, rx);
                    ry = fma(kk, dy, ry);
                    rs = fma(kk, s, rs);
                    z = fma(mult, t.w, z);
                    if (COUNT) ++c_acc;
                }
                live = false;
            }
        }
        root = F.node;
        end = min(nodes[F.node].skip, m);
    }
    int resume = live ? root : INT_MAX;
    int node = SEG ? __shfl_sync(0xffffffffu, root, 0) : root;
    const int stop = SEG ? __reduce_max_sync(0xffffffffu, valid ? end : 0) : end;
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
    if (SPLIT && valid) {
        reinterpret_cast<double4_32a *>(sp.part)[(size_t)fi * n + p] = make_double4_32a(rx, ry, rs, z);
    } else if (valid) {
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
template <int GF, bool COUNT, bool SEG, bool SPLIT>
__global__ void __launch_bounds__(kWalkBlock) walk_f64_kernel(int n, const NodeD *__restrict__ nodes,
                                                              const int *__restrict__ n_nodes,
                                                              const PointD *__restrict__ spts,
                                                              const uint32_t *__restrict__ idx, double2 *frep,
                                                              double *zi, unsigned long long *counters,
                                                              const SegView sv, const SplitView sp,
                                                              const BlockOrder bo)
{
    const int b = logical_block(bo);
    const int warp = (b * blockDim.x + threadIdx.x) >> 5;
    if (warp * 32 >= n) return;
    if (SPLIT && (int)blockIdx.y >= *sp.count) return;
    const long long t0 = clock64();
    walk_f64_chunk<GF, COUNT, SEG, SPLIT>(warp, n, nodes, n_nodes, spts, idx, frep, zi, counters, sv, sp, blockIdx.y);
    record_cost(bo, b, t0);
}

// The next launch order from the recorded costs: a counting sort on 256
// levels of cost / (max + 1), costliest first (the order inside a level is
// arbitrary); then the costs are cleared for the next walk.  One block.
__global__ void __launch_bounds__(1024) walk_order_kernel(unsigned *cost, int nb, int *order)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned smax;
    if (threadIdx.x < 256) hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    unsigned m = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) m = max(m, cost[b]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&smax, m);
    __syncthreads();
    const unsigned long long top = (unsigned long long)smax + 1ull;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        atomicAdd(&hist[255 - (int)((unsigned long long)cost[b] * 256ull / top)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive scan over the 256 levels
        unsigned run = 0;
        for (int k = 0; k < 256; ++k) {
            const unsigned h = hist[k];
            hist[k] = run;
            run += h;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const unsigned pos = atomicAdd(&hist[255 - (int)((unsigned long long)cost[b] * 256ull / top)], 1u);
        order[1 + pos] = b;
        cost[b] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) order[0] = nb;
}

// The frontier of the cut at `depth` (single thread; at most 4^depth entries
// in pre-order).  A cell with more than 4 children or a skip that does not
// advance is a broken tree: status bit 2, no entries (the walk then does no
// work and the error is reported).
template <typename NV>
__global__ void frontier_kernel(const NV nodes, const int *__restrict__ n_nodes, int n, int depth, Frontier *fr,
                                int *count, int *status)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = min(*n_nodes, 2 * n);
    Frontier a[kMaxFrontier], b[kMaxFrontier];
    int na = 1;
    a[0].node = 0;
    a[0].nanc = 0;
    a[0].own = 0;
    bool bad = m <= 0;
    for (int d = 0; d < depth && !bad; ++d) {
        int nb = 0;
        for (int e = 0; e < na && !bad; ++e) {
            const Frontier &E = a[e];
            if (!nodes.cell(E.node)) {  // leaf or bucket: stays an entry
                if (nb >= kMaxFrontier) { bad = true; break; }
                b[nb++] = E;
                continue;
            }
            const int cskip = nodes.skip(E.node);
            bool first = true;
            int kids = 0;
            for (int ch = E.node + 1; ch < cskip && ch < m;) {
                if (++kids > 4 || nb >= kMaxFrontier) { bad = true; break; }
                Frontier F = E;
                F.node = ch;
                F.own = first ? E.own : 0;
                if (d >= 1) {  // E is below the root: an ancestor of its children
                    F.anc[F.nanc] = E.node;
                    if (first) F.own |= 1 << F.nanc;
                    F.nanc += 1;
                }
                b[nb++] = F;
                first = false;
                const int nx = nodes.skip(ch);
                if (nx <= ch) { bad = true; break; }
                ch = nx;
            }
        }
        for (int e = 0; e < nb; ++e) a[e] = b[e];
        na = nb;
    }
    if (bad) {
        atomicOr(status, 2);
        na = 0;
    }
    for (int e = 0; e < na; ++e) fr[e] = a[e];
    *count = na;
}

// Sorted point p: the frontier entries' partial sums in entry order, then the
// per-point factors.
template <typename PT, typename VT>
__global__ void walk_combine_kernel(int n, const PT *__restrict__ spts, const uint32_t *__restrict__ idx,
                                    const VT *__restrict__ part, const int *__restrict__ count, double2 *frep,
                                    double *zi)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int nf = *count;
    double rx = 0, ry = 0, rs = 0, z = 0;
    for (int e = 0; e < nf; ++e) {
        const VT v = part[(size_t)e * n + p];
        rx += (double)v.x;
        ry += (double)v.y;
        rs += (double)v.z;
        z += (double)v.w;
    }
    double x, y, il;
    point_xy_il(spts[p], x, y, il);
    const double rsd = il * rs;
    const uint32_t i = idx[p];
    frep[i] = make_double2(4.0 * il * (rx + rsd * x), 4.0 * il * (ry + rsd * y));
    zi[i] = z;
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
    const float2 qh = make_float2(q.xh, q.yh), ql = make_float2(q.xl, q.yl);
    const float twoil = 2.0f * q.il;
    float2 rxy = make_float2(0.f, 0.f), rsz = make_float2(0.f, 0.f);  // paired sums, as in the walk
    for (int base = cbeg; base < cend; base += kExactBlock) {
        int j = base + threadIdx.x;
        if (j < cend) tile[threadIdx.x] = pts[j];
        __syncthreads();
        const int cnt = min(kExactBlock, cend - base);
        for (int k = 0; k < cnt; ++k) {
            const int jj = base + k;
            if (jj == i || jj < jlo || jj >= jhi) continue;
            const PointF o = tile[k];
            const float2 d = delta2(qh, ql, make_float2(o.xh, o.yh), make_float2(o.xl, o.yl));
            const float s = fmaf(d.x, d.x, d.y * d.y);
            const PairF t = pair_terms_f32<GF>(s * twoil * o.il);
            const float kk = t.rep * o.il;
            rxy = __ffma2_rn(make_float2(kk, kk), d, rxy);
            rsz = __ffma2_rn(make_float2(kk, 1.0f), make_float2(s, t.w), rsz);
        }
        __syncthreads();
    }
    if (i >= n) return;
    if (A.split > 1) {
        A.part[(size_t)blockIdx.y * n + i] = make_double4_32a(rxy.x, rxy.y, rsz.x, rsz.y);
        return;
    }
    double x = (double)q.xh + (double)q.xl, y = (double)q.yh + (double)q.yl;
    double il = (double)q.il;
    double rsd = il * (double)rsz.x;
    A.frep[i] = make_double2(4.0 * il * ((double)rxy.x + rsd * x), 4.0 * il * ((double)rxy.y + rsd * y));
    A.zi[i] = (double)rsz.y;
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

int walk_split_capacity(int64_t n)
{
    // frontier entries x points of the partial-sum buffer (0: no split)
    if (n <= 0 || n > kSplitMaxN) return 0;
    return (int)std::min<int64_t>(kMaxFrontier, kSplitEntries / n);
}

// Cut depth for n points: the shallowest that gives about 2048 warps, within
// the buffer; `want` >= 0 overrides (clamped), -1 chooses.  (A deeper cut for
// the float64 walk measured slower at N = 20,000: there the float64 pipe, not
// the warp count, is the limit.)
int walk_split_depth(int64_t n, int want, bool fp64)
{
    (void)fp64;
    const int cap = walk_split_capacity(n);
    int dmax = 0;
    while (dmax < kMaxSplitDepth && (1 << (2 * (dmax + 1))) <= cap) ++dmax;
    if (want >= 0) return std::min(want, dmax);
    const int64_t chunks = (n + 31) / 32, target = 2048;
    int d = 0;
    while (d < dmax && chunks * (1 << (2 * d)) < target) ++d;
    return d;
}

void launch_walk(hts_ctx *c)
{
    const int n = (int)c->n;
    const int warps = (n + 31) / 32;
    const int wb = c->walk_block;  // 32 .. kWalkBlock threads, a multiple of 32
    const bool cnt = c->counters_on != 0;  // counters accumulate while enabled
    const bool seg = c->nseg > 1;
    const SegView sv{c->keys, c->seg_off, c->pre};
    const int depth = seg ? 0 : walk_split_depth(n, c->walk_split, c->cfg.precision == HTS_FP64);
    SplitView sp{nullptr, nullptr, nullptr};
    dim3 grid((unsigned)((warps * 32 + wb - 1) / wb), 1);
    if (depth > 0) {
        Frontier *fr = reinterpret_cast<Frontier *>(c->split_frontier);
        int *fcount = reinterpret_cast<int *>(fr + kMaxFrontier);
        if (c->cfg.precision == HTS_FP32_MIXED)
            frontier_kernel<<<1, 32, 0, c->stream>>>(NodesF{c->nodes32}, c->n_nodes, n, depth, fr, fcount, c->status);
        else
            frontier_kernel<<<1, 32, 0, c->stream>>>(NodesD{c->nodes64}, c->n_nodes, n, depth, fr, fcount, c->status);
        c->launches += 1;
        sp = SplitView{fr, fcount, c->split_part};
        grid.y = 1u << (2 * depth);
    }
    c->launches += 1;
    // blocks in order of their cost in the previous walk, when the grid is
    // more than one wave (resident threads per SM: 2048)
    const bool balance = depth == 0 && (int64_t)grid.x > (int64_t)c->sm_count * (2048 / wb);
    const BlockOrder bo{balance ? c->walk_order : nullptr, balance ? c->walk_cost : nullptr};
#define HTS_WALK(P, NODES, SPTS, GF, CT, SG, SPL)                                                    \
    walk_##P##_kernel<GF, CT, SG, SPL><<<grid, wb, 0, c->stream>>>(n, NODES, c->n_nodes, SPTS, c->idx,   \
                                                                   c->frep, c->zi, c->counters, sv, sp, bo)
#define HTS_WALK_GF(P, NODES, SPTS, GF)                                                                   \
    if (depth > 0) {                                                                                       \
        if (cnt) HTS_WALK(P, NODES, SPTS, GF, true, false, true); else HTS_WALK(P, NODES, SPTS, GF, false, false, true); \
    } else if (cnt) {                                                                                      \
        if (seg) HTS_WALK(P, NODES, SPTS, GF, true, true, false); else HTS_WALK(P, NODES, SPTS, GF, true, false, false); \
    } else {                                                                                               \
        if (seg) HTS_WALK(P, NODES, SPTS, GF, false, true, false); else HTS_WALK(P, NODES, SPTS, GF, false, false, false); \
    }
#define HTS_WALK_ALL(P, NODES, SPTS)                                \
    if (c->cfg.grad_form == HTS_EXACT_KL) {                          \
        HTS_WALK_GF(P, NODES, SPTS, 0)                               \
    } else {                                                         \
        HTS_WALK_GF(P, NODES, SPTS, 1)                               \
    }
    if (c->cfg.precision == HTS_FP32_MIXED) {
        const NodesF nf{c->nodes32};
        HTS_WALK_ALL(f32, nf, c->spts32)
    } else {
        HTS_WALK_ALL(f64, c->nodes64, c->spts64)
    }
#undef HTS_WALK_ALL
#undef HTS_WALK_GF
#undef HTS_WALK
    if (balance) {
        walk_order_kernel<<<1, 1024, 0, c->stream>>>(c->walk_cost, (int)grid.x, c->walk_order);
        c->launches += 1;
    }
    if (depth > 0) {
        const int cb = (n + 255) / 256;
        const int *fcount = reinterpret_cast<const int *>(reinterpret_cast<Frontier *>(c->split_frontier) +
                                                          kMaxFrontier);
        if (c->cfg.precision == HTS_FP32_MIXED)
            walk_combine_kernel<PointF, float4><<<cb, 256, 0, c->stream>>>(
                n, c->spts32, c->idx, reinterpret_cast<const float4 *>(c->split_part), fcount, c->frep, c->zi);
        else
            walk_combine_kernel<PointD, double4_32a><<<cb, 256, 0, c->stream>>>(
                n, c->spts64, c->idx, reinterpret_cast<const double4_32a *>(c->split_part), fcount, c->frep,
                c->zi);
        c->launches += 1;
    }
}

size_t walk_split_frontier_bytes() { return sizeof(Frontier) * kMaxFrontier + 64; }

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
