// noalloc.cu -- the exact float64 gradient without any device allocation.
//
// hts_exact_grad_noalloc computes the same quantity as hts_grad with
// theta = 0 in HTS_FP64 (exact repulsion over all pairs, attraction over P,
// Z, g = 4 (exag F_attr - F_rep / Z)), but keeps its work arrays in one
// file-scope __device__ array of fixed size instead of buffers from
// cudaMalloc.  It exists for callers that cannot allocate device memory
// themselves or through this library: a plug-in inside a framework or an
// inference server whose own allocator owns the whole device memory budget
// (a cudaMalloc behind its back can fail or starve it), and code on a
// latency-critical path where the implicit device synchronisation of
// cudaMalloc / cudaFree is not acceptable.  Such callers pass device
// pointers for every input and output.
//
// The array holds HTS_NOALLOC_MAX_N points (about 4.5 MB) and stays resident
// on every device that loads this library, until the process exits.  All
// calls share it: a call writes every element it later reads (the one flag
// that must start at zero is cleared at the start of each call), but two
// calls whose kernels overlap on the GPU (different streams, or different
// host threads on one device) race on it and must be serialised by the
// caller.
#include <mutex>

#include "hts_internal.cuh"

namespace {

using hts::PairD;
using hts::PointD;
using hts::pair_terms_f64;

constexpr int kMaxN = HTS_NOALLOC_MAX_N;
constexpr int kBlock = 256;
constexpr int kRedBlocks = 256;

struct Scratch {
    PointD pts[kMaxN];       // positions with il = 1 / (1 - |y|^2)
    double2 frep[kMaxN];     // repulsive sums
    double2 fattr[kMaxN];    // attractive sums
    double zi[kMaxN];        // per-point Z terms
    double partial[kRedBlocks];
    double Z;
    int bad;                 // set when a point is outside the open disk or not finite
};

static __device__ __align__(256) Scratch g_scratch;

// Device address of g_scratch, resolved once per device (host code must not
// use the symbol itself as a pointer).
constexpr int kMaxDevices = 64;
Scratch *g_addr[kMaxDevices] = {};
std::mutex g_mutex;

int scratch_address(int device, Scratch **out)
{
    if (device < 0 || device >= kMaxDevices) return HTS_EINVAL;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return HTS_ECUDA;
        }
        g_addr[device] = static_cast<Scratch *>(p);
    }
    *out = g_addr[device];
    return HTS_OK;
}

// Point records; a point with |y| >= 1 or a non-finite coordinate sets
// s->bad, which turns g and Z into NaN (na_final_z, na_combine).
__global__ void na_prep(int n, const double2 *__restrict__ y, Scratch *s)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    double2 p = y[i];
    double n2 = p.x * p.x + p.y * p.y;
    if (!isfinite(p.x) || !isfinite(p.y) || !(n2 < 1.0)) {
        atomicOr(&s->bad, 1);
        p = make_double2(0.0, 0.0);  // keeps the later kernels' arithmetic finite
        n2 = 0.0;
    }
    s->pts[i] = PointD{p.x, p.y, 1.0 / (1.0 - n2), 0.0};
}

template <int GF>
__global__ void __launch_bounds__(kBlock) na_repulsion(int n, Scratch *s)
{
    __shared__ PointD tile[kBlock];
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const PointD q = s->pts[i < n ? i : n - 1];
    const double twoil = 2.0 * q.il;
    double rx = 0, ry = 0, rs = 0, z = 0;
    for (int base = 0; base < n; base += kBlock) {
        if (base + threadIdx.x < n) tile[threadIdx.x] = s->pts[base + threadIdx.x];
        __syncthreads();
        const int cnt = min(kBlock, n - base);
        for (int k = 0; k < cnt; ++k) {
            if (base + k == i) continue;
            const PointD o = tile[k];
            double dx = q.x - o.x, dy = q.y - o.y;
            double sq = fma(dx, dx, dy * dy);
            PairD t = pair_terms_f64<GF>(sq * twoil * o.il);
            double kk = t.rep * o.il;
            rx = fma(kk, dx, rx);
            ry = fma(kk, dy, ry);
            rs = fma(kk, sq, rs);
            z += t.w;
        }
        __syncthreads();
    }
    if (i < n) {
        double rsd = q.il * rs;
        s->frep[i] = make_double2(4.0 * q.il * (rx + rsd * q.x), 4.0 * q.il * (ry + rsd * q.y));
        s->zi[i] = z;
    }
}

// Entries outside [0, nnz) and column indices outside [0, n) are skipped, so
// a malformed matrix cannot make the kernel read outside its buffers.
template <int GF>
__global__ void __launch_bounds__(kBlock) na_attraction(int n, int64_t nnz, const int64_t *__restrict__ indptr,
                                                        const int32_t *__restrict__ indices,
                                                        const double *__restrict__ vals, Scratch *s)
{
    const int row = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const PointD q = s->pts[row];
    const double twoil = 2.0 * q.il;
    double ax = 0, ay = 0, as = 0;
    const int64_t e0 = max(indptr[row], (int64_t)0), e1 = min(indptr[row + 1], nnz);
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int j = indices[e];
        if ((unsigned)j >= (unsigned)n) continue;
        const PointD o = s->pts[j];
        double dx = q.x - o.x, dy = q.y - o.y;
        double sq = fma(dx, dx, dy * dy);
        PairD t = pair_terms_f64<GF>(sq * twoil * o.il);
        double k = vals[e] * t.att * o.il;
        ax = fma(k, dx, ax);
        ay = fma(k, dy, ay);
        as = fma(k, sq, as);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        as += __shfl_xor_sync(0xffffffffu, as, o);
    }
    if (lane == 0) {
        double asd = q.il * as;
        s->fattr[row] = make_double2(4.0 * q.il * (ax + asd * q.x), 4.0 * q.il * (ay + asd * q.y));
    }
}

__global__ void __launch_bounds__(kBlock) na_partial_z(int n, Scratch *s)
{
    __shared__ double sh[kBlock];
    double a = 0;
    for (int k = blockIdx.x * kBlock + threadIdx.x; k < n; k += kRedBlocks * kBlock) a += s->zi[k];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) s->partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kRedBlocks) na_final_z(Scratch *s, double *Z_out)
{
    __shared__ double sh[kRedBlocks];
    sh[threadIdx.x] = s->partial[threadIdx.x];
    __syncthreads();
    for (int w = kRedBlocks / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double Z = s->bad ? __longlong_as_double(0x7FF8000000000000ll) : sh[0];  // NaN: a point out of range
        s->Z = Z;
        if (Z_out) *Z_out = Z;
    }
}

__global__ void na_combine(int n, double exag, const Scratch *s, double2 *g)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    if (s->bad) {  // a point outside the open disk: no gradient
        const double nan = __longlong_as_double(0x7FF8000000000000ll);
        g[i] = make_double2(nan, nan);
        return;
    }
    const double invZ = s->Z > 0.0 ? 1.0 / s->Z : 0.0;
    const double2 fa = s->fattr[i], fr = s->frep[i];
    g[i] = make_double2(4.0 * (exag * fa.x - fr.x * invZ), 4.0 * (exag * fa.y - fr.y * invZ));
}

}  // namespace

extern "C" int hts_exact_grad_noalloc(int64_t n, int64_t nnz, const double *y, const int64_t *indptr,
                                      const int32_t *indices, const double *values, double exaggeration,
                                      int grad_form, double *g_out, double *Z_out, void *stream)
{
    if (n < 0 || nnz < 0 || (n > 0 && (!y || !indptr || !g_out)) || (nnz > 0 && (!indices || !values)) ||
        (grad_form != HTS_EXACT_KL && grad_form != HTS_PAPER_EQ) || !(exaggeration > 0.0))
        return HTS_EINVAL;
    if (n > kMaxN) return HTS_ETOOLARGE;
    if (n == 0) return HTS_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HTS_ECUDA;
    }
    Scratch *s = nullptr;
    int r = scratch_address(dev, &s);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((n + kBlock - 1) / kBlock);
    const int rb = (int)((n * 32 + kBlock - 1) / kBlock);
    if (cudaMemsetAsync(&s->bad, 0, sizeof(int), st) != cudaSuccess) {  // not an allocation
        cudaGetLastError();
        return HTS_ECUDA;
    }
    na_prep<<<nb, kBlock, 0, st>>>((int)n, (const double2 *)y, s);
    if (grad_form == HTS_EXACT_KL) {
        na_repulsion<0><<<nb, kBlock, 0, st>>>((int)n, s);
        na_attraction<0><<<rb, kBlock, 0, st>>>((int)n, nnz, indptr, indices, values, s);
    } else {
        na_repulsion<1><<<nb, kBlock, 0, st>>>((int)n, s);
        na_attraction<1><<<rb, kBlock, 0, st>>>((int)n, nnz, indptr, indices, values, s);
    }
    na_partial_z<<<kRedBlocks, kBlock, 0, st>>>((int)n, s);
    na_final_z<<<1, kRedBlocks, 0, st>>>(s, Z_out);
    na_combine<<<nb, kBlock, 0, st>>>((int)n, exaggeration, s, (double2 *)g_out);
    if (cudaGetLastError() != cudaSuccess) return HTS_ECUDA;
    return HTS_OK;
}
