// attract.cu -- the attractive sum over P (first sum of Eq.
// KlGradientHyperbolicSplit), the KL cost terms (Eq. KLDivergence) and
// device-side validation of a CSR matrix.
//
// A group of lanes per row of P (8 in float32, a warp in float64) reads
// consecutive (index, value) entries (coalesced), gathers the neighbours'
// point records (16-byte PointA in float32, 32-byte PointD in float64;
// random, mostly L2 hits) and reduces three scalars by shuffles.
// Per point: F_attr,i = 4 il_i (A_Delta + il_i A_s y_i) with
//   A_Delta = sum_j p_ij (w d / t)_ij il_j Delta_ij,  A_s = same with s_ij.
// Bytes per non-zero: 4 (index) + 4 or 8 (value) + 16 or 32 (gathered record).
#include <cuda_fp16.h>

#include <algorithm>

#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kBlock = 256;

// Float32 path: a group of G lanes per row (kBlock / G rows per block; G in
// {4, 8, 16, 32}, picked by the autotuner, default 8), so short rows do not
// leave most of a warp idle; each lane keeps kUnroll index loads and gathers
// in flight before its arithmetic.
constexpr int kUnroll = 4;
// launched in the background: resident blocks per SM of the float32 (beside the
// tree build and the walk) and float64 (beside the walk) attraction
constexpr int kAttractBlocksPerSM32 = 2, kAttractBlocksPerSM64 = 8;

// Lo floats of a PointA (see hts_internal.cuh): the packed halves times 2^-24.
__device__ __forceinline__ float2 point_lo(unsigned lo)
{
    const float2 h = __half22float2(__halves2half2(__ushort_as_half((unsigned short)(lo & 0xFFFFu)),
                                                   __ushort_as_half((unsigned short)(lo >> 16))));
    return make_float2(h.x * 5.9604644775390625e-8f, h.y * 5.9604644775390625e-8f);
}

template <int GF, int kGroup>
__global__ void __launch_bounds__(kBlock) attract_f32_kernel(int n, const int64_t *__restrict__ indptr,
                                                             const int32_t *__restrict__ indices,
                                                             const float *__restrict__ vals,
                                                             const PointA *__restrict__ pts, double2 *fattr)
{
    // grid-stride over blocks of rows: one pass with the full grid, several
    // with the small grid of the background launch (kAttractBlocksPerSM32)
    const int64_t span = (int64_t)n * kGroup;
    for (int64_t base = (int64_t)blockIdx.x * kBlock; base < span; base += (int64_t)gridDim.x * kBlock) {
    const int row = (int)((base + threadIdx.x) / kGroup);
    const int lane = threadIdx.x & (kGroup - 1);
    const bool live = row < n;
    const int r = live ? row : n - 1;
    const PointA q = pts[r];
    const float2 ql = point_lo(q.lo);
    const float twoil = 2.0f * q.il;
    const int64_t e0 = indptr[r];
    const int len = live ? (int)(indptr[r + 1] - e0) : 0;  // a row is shorter than 2^31
    const int32_t *__restrict__ ir = indices + e0;
    const float *__restrict__ vr = vals + e0;
    float ax = 0.f, ay = 0.f, as = 0.f;
    for (int e = lane; e < len; e += kGroup * kUnroll) {
        int j[kUnroll];
        float pv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int eu = e + kGroup * u;
            const bool ok = eu < len;
            j[u] = ok ? __ldg(ir + eu) : r;
            pv[u] = ok ? __ldg(vr + eu) : 0.0f;
        }
        PointA o[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) o[u] = pts[j[u]];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const float2 ol = point_lo(o[u].lo);
            const float dx = (q.xh - o[u].xh) + (ql.x - ol.x);
            const float dy = (q.yh - o[u].yh) + (ql.y - ol.y);
            const float s = fmaf(dx, dx, dy * dy);
            const PairF t = pair_terms_f32<GF>(s * twoil * o[u].il);
            const float k = pv[u] * t.att * o[u].il;
            ax = fmaf(k, dx, ax);
            ay = fmaf(k, dy, ay);
            as = fmaf(k, s, as);
        }
    }
    for (int o = kGroup / 2; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        as += __shfl_xor_sync(0xffffffffu, as, o);
    }
    if (lane == 0 && live) {
        double x = (double)q.xh + (double)ql.x, y = (double)q.yh + (double)ql.y;
        double il = (double)q.il;
        double asd = il * (double)as;
        fattr[row] = make_double2(4.0 * il * ((double)ax + asd * x), 4.0 * il * ((double)ay + asd * y));
    }
    }
}

template <int GF>
__global__ void __launch_bounds__(kBlock) attract_f64_kernel(int n, const int64_t *__restrict__ indptr,
                                                             const int32_t *__restrict__ indices,
                                                             const double *__restrict__ vals,
                                                             const PointD *__restrict__ pts, double2 *fattr)
{
    const int lane = threadIdx.x & 31;
    // grid-stride over rows (a warp per row), as in the float32 kernel
    for (int row = (blockIdx.x * kBlock + threadIdx.x) >> 5; row < n; row += (gridDim.x * kBlock) >> 5) {
    const PointD q = pts[row];
    const double twoil = 2.0 * q.il;
    const int64_t e0 = indptr[row], e1 = indptr[row + 1];
    double ax = 0, ay = 0, as = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int j = __ldg(indices + e);
        const double pv = __ldg(vals + e);
        const PointD o = pts[j];
        double dx = q.x - o.x, dy = q.y - o.y;
        double s = fma(dx, dx, dy * dy);
        PairD t = pair_terms_f64<GF>(s * twoil * o.il);
        double k = pv * t.att * o.il;
        ax = fma(k, dx, ax);
        ay = fma(k, dy, ay);
        as = fma(k, s, as);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        as += __shfl_xor_sync(0xffffffffu, as, o);
    }
    if (lane == 0) {
        double asd = q.il * as;
        fattr[row] = make_double2(4.0 * q.il * (ax + asd * q.x), 4.0 * q.il * (ay + asd * q.y));
    }
    }
}

// KL terms in float64 from the float64 positions: per block partial sums of
// p log p, p log w = -p log1p(d^2) and p, combined in fixed order later.
template <typename VT>
__global__ void __launch_bounds__(kBlock) kl_terms_kernel(int n, const int64_t *__restrict__ indptr,
                                                          const int32_t *__restrict__ indices,
                                                          const VT *__restrict__ vals, const double2 *__restrict__ y,
                                                          double *partial)
{
    const int row = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double a = 0, b = 0, sp = 0;
    if (row < n) {
        const double2 q = y[row];
        const double ai = 1.0 - (q.x * q.x + q.y * q.y);
        for (int64_t e = indptr[row] + lane; e < indptr[row + 1]; e += 32) {
            const double pv = (double)vals[e];
            if (!(pv > 0.0)) continue;
            const double2 o = y[indices[e]];
            double dx = q.x - o.x, dy = q.y - o.y;
            double bj = 1.0 - (o.x * o.x + o.y * o.y);
            double delta = 2.0 * (dx * dx + dy * dy) / (ai * bj);
            double d = log1p(delta + sqrt(delta * (delta + 2.0)));
            a += pv * log(pv);
            b -= pv * log1p(d * d);
            sp += pv;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
    }
    __shared__ double sh[3][kBlock / 32];
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
        sh[2][w] = sp;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0;
        for (int k = 0; k < kBlock / 32; ++k) t += sh[threadIdx.x][k];
        partial[3 * blockIdx.x + threadIdx.x] = t;
    }
}

// Per-row KL terms (for per-segment sums): a[i] = sum p log p, b[i] = sum p log w,
// pp[i] = sum p over row i, all in float64 from the float64 positions.
template <typename VT>
__global__ void __launch_bounds__(kBlock) kl_rows_kernel(int n, const int64_t *__restrict__ indptr,
                                                         const int32_t *__restrict__ indices,
                                                         const VT *__restrict__ vals, const double2 *__restrict__ y,
                                                         double *a_out, double *b_out, double *p_out)
{
    const int row = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double a = 0, b = 0, sp = 0;
    const double2 q = y[row];
    const double ai = 1.0 - (q.x * q.x + q.y * q.y);
    for (int64_t e = indptr[row] + lane; e < indptr[row + 1]; e += 32) {
        const double pv = (double)vals[e];
        if (!(pv > 0.0)) continue;
        const double2 o = y[indices[e]];
        double dx = q.x - o.x, dy = q.y - o.y;
        double bj = 1.0 - (o.x * o.x + o.y * o.y);
        double delta = 2.0 * (dx * dx + dy * dy) / (ai * bj);
        double d = log1p(delta + sqrt(delta * (delta + 2.0)));
        a += pv * log(pv);
        b -= pv * log1p(d * d);
        sp += pv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
    }
    if (lane == 0) {
        a_out[row] = a;
        b_out[row] = b;
        p_out[row] = sp;
    }
}

// Rows of segment s may only index points of segment s (status bit 16).
__global__ void check_block_diagonal_kernel(int n, const int64_t *__restrict__ indptr,
                                            const int32_t *__restrict__ indices,
                                            const unsigned char *__restrict__ seg_of, int *status)
{
    const int row = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int s = seg_of[row];
    for (int64_t e = indptr[row] + lane; e < indptr[row + 1]; e += 32)
        if (seg_of[indices[e]] != s) atomicOr(status, 16);
}

__global__ void fill_segments_kernel(int n, int nseg, const int64_t *__restrict__ off, unsigned char *seg_of)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nseg - 1;  // last s with off[s] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    seg_of[i] = (unsigned char)lo;
}

__global__ void sum_partials_kernel(int blocks, const double *__restrict__ partial, double *out3)
{
    __shared__ double sh[3][256];
    double a = 0, b = 0, c = 0;
    for (int k = threadIdx.x; k < blocks; k += 256) {
        a += partial[3 * k];
        b += partial[3 * k + 1];
        c += partial[3 * k + 2];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3) out3[threadIdx.x] = sh[threadIdx.x][0];
}

// status bits: 8 bad indptr, 16 bad index / diagonal, 32 bad value
template <typename VT>
__global__ void validate_csr_kernel(int n, int64_t nnz, const int64_t *__restrict__ indptr,
                                    const int32_t *__restrict__ indices, const VT *__restrict__ vals, int *status)
{
    const int row = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int64_t e0 = indptr[row], e1 = indptr[row + 1];
    if (lane == 0) {
        if ((row == 0 && e0 != 0) || e1 < e0 || (row == n - 1 && e1 != nnz) || e1 > nnz || e0 < 0)
            atomicOr(status, 8);
    }
    if (e1 < e0 || e0 < 0 || e1 > nnz) return;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        int j = indices[e];
        if (j < 0 || j >= n || j == row) atomicOr(status, 16);
        double v = (double)vals[e];
        if (!(v >= 0.0) || !isfinite(v)) atomicOr(status, 32);
    }
}

}  // namespace

void launch_attract(hts_ctx *c)
{
    const int n = (int)c->n;
    const int blocks = (int)(((int64_t)n * 32 + kBlock - 1) / kBlock);
    const int G = c->attract_group;
    // in the background: a small resident grid that strides over the rows
    // instead of one block per 256 / G rows
    const int full = (int)(((int64_t)n * G + kBlock - 1) / kBlock);
    const int blocks32 = c->attract_background ? std::min(full, kAttractBlocksPerSM32 * c->sm_count) : full;
    const int blocks64 = c->attract_background ? std::min(blocks, kAttractBlocksPerSM64 * c->sm_count) : blocks;
    c->launches += 1;
    if (c->cfg.precision == HTS_FP32_MIXED) {
        const float *v = (const float *)c->values;
#define HTS_ATTRACT(GF, GG)                                                                             \
    attract_f32_kernel<GF, GG><<<blocks32, kBlock, 0, c->stream>>>(n, c->indptr, c->indices, v, c->apts32, \
                                                                    c->fattr)
#define HTS_ATTRACT_G(GF)                          \
    switch (G) {                                   \
    case 4: HTS_ATTRACT(GF, 4); break;             \
    case 16: HTS_ATTRACT(GF, 16); break;           \
    case 32: HTS_ATTRACT(GF, 32); break;           \
    default: HTS_ATTRACT(GF, 8); break;            \
    }
        if (c->cfg.grad_form == HTS_EXACT_KL) {
            HTS_ATTRACT_G(0)
        } else {
            HTS_ATTRACT_G(1)
        }
#undef HTS_ATTRACT_G
#undef HTS_ATTRACT
    } else {
        const double *v = (const double *)c->values;
        if (c->cfg.grad_form == HTS_EXACT_KL)
            attract_f64_kernel<0><<<blocks64, kBlock, 0, c->stream>>>(n, c->indptr, c->indices, v, c->pts64,
                                                                      c->fattr);
        else
            attract_f64_kernel<1><<<blocks64, kBlock, 0, c->stream>>>(n, c->indptr, c->indices, v, c->pts64,
                                                                      c->fattr);
    }
}

void launch_kl_terms(hts_ctx *c)
{
    const int n = (int)c->n;
    const int blocks = (int)(((int64_t)n * 32 + kBlock - 1) / kBlock);
    if (c->values_f64)
        kl_terms_kernel<double><<<blocks, kBlock, 0, c->stream>>>(n, c->indptr, c->indices,
                                                                  (const double *)c->values, c->y, c->red_tmp);
    else
        kl_terms_kernel<float><<<blocks, kBlock, 0, c->stream>>>(n, c->indptr, c->indices, (const float *)c->values,
                                                                 c->y, c->red_tmp);
    sum_partials_kernel<<<1, 256, 0, c->stream>>>(blocks, c->red_tmp, c->dscal + 1);
    c->launches += 2;
}

void launch_kl_rows(hts_ctx *c, double *a, double *b, double *p)
{
    const int n = (int)c->n;
    const int blocks = (int)(((int64_t)n * 32 + kBlock - 1) / kBlock);
    if (c->values_f64)
        kl_rows_kernel<double><<<blocks, kBlock, 0, c->stream>>>(n, c->indptr, c->indices, (const double *)c->values,
                                                                 c->y, a, b, p);
    else
        kl_rows_kernel<float><<<blocks, kBlock, 0, c->stream>>>(n, c->indptr, c->indices, (const float *)c->values,
                                                                c->y, a, b, p);
    c->launches += 1;
}

void launch_segments_setup(hts_ctx *c)
{
    const int n = (int)c->n;
    fill_segments_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->nseg, c->seg_off, c->seg_of);
    const int blocks = (int)(((int64_t)n * 32 + kBlock - 1) / kBlock);
    check_block_diagonal_kernel<<<blocks, kBlock, 0, c->stream>>>(n, c->indptr, c->indices, c->seg_of, c->status);
}

void launch_validate_csr(hts_ctx *c, int n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                         const void *values, int f64)
{
    const int blocks = (int)(((int64_t)n * 32 + kBlock - 1) / kBlock);
    if (f64)
        validate_csr_kernel<double><<<blocks, kBlock, 0, c->stream>>>(n, nnz, indptr, indices,
                                                                       (const double *)values, c->status);
    else
        validate_csr_kernel<float><<<blocks, kBlock, 0, c->stream>>>(n, nnz, indptr, indices, (const float *)values,
                                                                     c->status);
}

}  // namespace hts
