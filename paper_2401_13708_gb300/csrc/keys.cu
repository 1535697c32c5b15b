// keys.cu -- per-point preparation and polar keys (Sec. 4.1).
//
// prep_points: conformal factor il = 1 / (1 - |y|^2) (lambda / 2, Eq.
//   PoincareMetric), the 32-byte point records, and the radial split
//   coordinate (disk radius for Eq. EqualEmbeddingLengthsSplitting, cosh of
//   the hyperbolic radius, (1 + |y|^2) / (1 - |y|^2), for Eq.
//   EqualAreaSplitting) with the root annulus bounds of each segment reduced
//   by atomic min / max on the bit patterns (exact for non-negative doubles).
// make_keys: normalised coordinates rho^ = (c - c_min) / (c_max - c_min),
//   phi^ = atan2 / 2 pi in [0, 1], each quantised to 29 bits and
//   interleaved (digit l = 2 * radial bit + angular bit of level l, most
//   significant first), so that the depth-l cell of the equal-length tree is
//   the top 2l key bits below the 6-bit segment id (bits 58..63).  The float64 steps use explicitly rounded
//   intrinsics so no fused multiply-add changes a quantised bit.
#include <cuda_fp16.h>

#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kBlock = 256;

__global__ void init_minmax_kernel(unsigned long long *mm, int nseg)
{
    const int s = threadIdx.x;
    if (s < nseg) {
        mm[2 * s] = 0x7FF0000000000000ull;  // +inf
        mm[2 * s + 1] = 0ull;               // +0
    }
}

// Per point: records and radial coordinate; per segment: the root annulus
// [min, max] of the radial coordinate (warp-reduced when a warp's points lie
// in one segment, which is all but the warps straddling a boundary).
__global__ void prep_points_kernel(int n, const double2 *__restrict__ y, int split_rule, PointF *pts32,
                                   PointA *apts32, PointD *pts64, double *radial,
                                   const unsigned char *__restrict__ seg_of, unsigned long long *mm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double c = 0.0;
    bool ok = i < n;
    int sg = 0;
    if (ok) {
        double2 p = y[i];
        double n2 = __dadd_rn(__dmul_rn(p.x, p.x), __dmul_rn(p.y, p.y));
        if (pts32) {  // il as the float reciprocal of 1 - |y|^2 (off the float64 pipe)
            PointF r;
            float a32, unused;
            split_f32(p.x, r.xh, r.xl);
            split_f32(p.y, r.yh, r.yl);
            split_f32(__dsub_rn(1.0, n2), a32, unused);  // (float)(1 - |y|^2)
            r.il = __frcp_rn(a32);
            r.pad0 = r.pad1 = r.pad2 = 0.f;
            pts32[i] = r;
            const unsigned lx = __half_as_ushort(__float2half_rn(r.xl * 16777216.0f));  // lo * 2^24
            const unsigned ly = __half_as_ushort(__float2half_rn(r.yl * 16777216.0f));
            apts32[i] = PointA{r.xh, r.yh, r.il, lx | (ly << 16)};
        }
        if (pts64) pts64[i] = PointD{p.x, p.y, __ddiv_rn(1.0, __dsub_rn(1.0, n2)), 0.0};
        c = split_rule == HTS_EQUAL_AREA ? __ddiv_rn(__dadd_rn(1.0, n2), __dsub_rn(1.0, n2)) : __dsqrt_rn(n2);
        radial[i] = c;
        if (seg_of) sg = seg_of[i];
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(c);
    const int s0 = __shfl_sync(0xffffffffu, sg, 0);
    if (__all_sync(0xffffffffu, !ok || sg == s0)) {
        unsigned long long vmin = ok ? b : 0x7FF0000000000000ull;
        unsigned long long vmax = ok ? b : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long a = __shfl_xor_sync(0xffffffffu, vmin, o);
            unsigned long long z = __shfl_xor_sync(0xffffffffu, vmax, o);
            vmin = a < vmin ? a : vmin;
            vmax = z > vmax ? z : vmax;
        }
        if ((threadIdx.x & 31) == 0 && vmax >= vmin) {
            atomicMin(&mm[2 * s0], vmin);
            atomicMax(&mm[2 * s0 + 1], vmax);
        }
    } else if (ok) {
        atomicMin(&mm[2 * sg], b);
        atomicMax(&mm[2 * sg + 1], b);
    }
}

// Spread the low 29 bits of v to the odd/even positions of a 58-bit word.
__device__ __forceinline__ uint64_t spread_bits(uint64_t v)
{
    v &= 0x1FFFFFFFull;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

// floor(u 2^kLevels) clamped to [0, 2^kLevels - 1], from the bit pattern of u
// (bits.cuh): the float64 route (multiply, floor, convert) runs on the narrow
// float64 pipe.
__device__ __forceinline__ uint64_t quantise(double u) { return quantise_unit(u, kLevels); }

__global__ void make_keys_kernel(int n, const double2 *__restrict__ y, const double *__restrict__ radial,
                                 const unsigned char *__restrict__ seg_of, const unsigned long long *__restrict__ mm,
                                 uint64_t *keys, uint32_t *idx)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sg = seg_of ? seg_of[i] : 0;
    double lo = __longlong_as_double((long long)mm[2 * sg]);
    double hi = __longlong_as_double((long long)mm[2 * sg + 1]);
    double c = radial[i];
    double rh = hi > lo ? __ddiv_rn(__dsub_rn(c, lo), __dsub_rn(hi, lo)) : 0.0;
    double2 p = y[i];
    double phi = atan2(p.y, p.x);
    if (phi < 0.0) phi = __dadd_rn(phi, kTwoPi);
    double ph = __ddiv_rn(phi, kTwoPi);
    uint64_t qa = quantise(rh), qb = quantise(ph);
    keys[i] = ((uint64_t)sg << kSegShift) | (spread_bits(qa) << 1) | spread_bits(qb);
    idx[i] = (uint32_t)i;
}

}  // namespace

void launch_prep_points(hts_ctx *c)
{
    int n = (int)c->n;
    init_minmax_kernel<<<1, kMaxSegments, 0, c->stream>>>(c->minmax, c->nseg);
    bool f32 = c->cfg.precision == HTS_FP32_MIXED;
    prep_points_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>(
        n, c->y, c->cfg.split_rule, f32 ? c->pts32 : nullptr, f32 ? c->apts32 : nullptr, f32 ? nullptr : c->pts64,
        c->radial,
        c->nseg > 1 ? c->seg_of : nullptr, c->minmax);
    c->launches += 2;
}

void launch_make_keys(hts_ctx *c)
{
    int n = (int)c->n;
    make_keys_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>(
        n, c->y, c->radial, c->nseg > 1 ? c->seg_of : nullptr, c->minmax, c->keys, c->idx);
    c->launches += 1;
}

}  // namespace hts
