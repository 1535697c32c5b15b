// sort.cu -- LSD radix sort of (key, index) pairs and an exclusive int scan.
//
// The tree of Sec. 4.1 is a hierarchy over the keys, so sorting the points
// by key puts every cell's points in one contiguous run.  Eight stable
// passes of 8 bits each (keys use the low 58 bits).  Per pass:
//   hist     one 4096-key tile per block: 256-bin shared histogram,
//            written digit-major as counts[digit][tile];
//   scan     exclusive scan of the counts gives every (digit, tile) its
//            first output slot;
//   scatter  each warp owns 512 consecutive keys of the tile; warp
//            histograms (match_any + popc), a per-digit prefix over the 8
//            warps, then a second in-order pass ranks each key among equal
//            digits (match_any + popc of lower lanes) and writes it out.
// Traffic per pass: 8 B/key read (hist) + 12 B read + 12 B write (scatter).
#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kTile = 4096;
constexpr int kSortThreads = 256;
constexpr int kWarps = kSortThreads / 32;
constexpr int kPerWarp = kTile / kWarps;   // 512
constexpr int kRounds = kPerWarp / 32;     // 16
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kSortThreads) hist_kernel(const uint64_t *__restrict__ keys, int n, int shift,
                                                            int tiles, int *counts)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kTile;
#pragma unroll 4
    for (int k = threadIdx.x; k < kTile; k += kSortThreads) {
        int i = base + k;
        if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 0xFFu)], 1);
    }
    __syncthreads();
    counts[threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) scatter_kernel(const uint64_t *__restrict__ kin,
                                                               const uint32_t *__restrict__ vin,
                                                               uint64_t *__restrict__ kout,
                                                               uint32_t *__restrict__ vout, int n, int shift,
                                                               int tiles, const int *__restrict__ offsets)
{
    __shared__ int wh[kWarps][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wh[0][0])[k] = 0;
    __syncthreads();

    const int base = blockIdx.x * kTile + w * kPerWarp;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[kRounds];
    uint32_t val[kRounds];
    int dig[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int i = base + r * 32 + lane;
        bool ok = i < n;
        key[r] = ok ? kin[i] : 0ull;
        val[r] = ok ? vin[i] : 0u;
        dig[r] = ok ? (int)((key[r] >> shift) & 0xFFu) : 256 + lane;  // invalid lanes match only themselves
        unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
        if (ok && (peers & lt) == 0u) wh[w][dig[r]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        int d = threadIdx.x;  // 256 threads = 256 digits
        int run = offsets[d * tiles + blockIdx.x];
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            int t = wh[k][d];
            wh[k][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int i = base + r * 32 + lane;
        bool ok = i < n;
        unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
        int pos = 0;
        if (ok) pos = wh[w][dig[r]] + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0u) wh[w][dig[r]] += __popc(peers);
        __syncwarp();
        if (ok) {
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ---- exclusive scan --------------------------------------------------------

__global__ void __launch_bounds__(kScanThreads) scan_block_kernel(const int *__restrict__ in, int *out, int64_t len,
                                                                  int *block_sums)
{
    __shared__ int warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < len ? in[i] : 0;
        local += v[k];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int s = t;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = s - t;  // exclusive warp offsets
        if (lane == 31 && block_sums) block_sums[blockIdx.x] = s;
    }
    __syncthreads();
    int run = warp_tot[w] + incl - local;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < len) out[i] = run;
        run += v[k];
    }
}

__global__ void add_offsets_kernel(int *out, int64_t len, const int *__restrict__ offs)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += offs[i / kScanBlock];
}

}  // namespace

int64_t scan_tmp_size(int64_t len)
{
    int64_t total = 0;
    while (len > kScanBlock) {
        len = (len + kScanBlock - 1) / kScanBlock;
        total += len + 1;
    }
    return total + 1;
}

// Exclusive scan of len ints (in and out may alias only if equal).
// Returns the number of kernels launched.
int scan_exclusive(const int *in, int *out, int64_t len, int *tmp, cudaStream_t s)
{
    if (len <= 0) return 0;
    int64_t blocks = (len + kScanBlock - 1) / kScanBlock;
    if (blocks == 1) {
        scan_block_kernel<<<1, kScanThreads, 0, s>>>(in, out, len, nullptr);
        return 1;
    }
    int *sums = tmp;
    scan_block_kernel<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, len, sums);
    int k = scan_exclusive(sums, sums, blocks, tmp + blocks + 1, s);
    add_offsets_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(out, len, sums);
    return k + 2;
}

void launch_sort_pairs(hts_ctx *c)
{
    int n = (int)c->n;
    int tiles = (n + kTile - 1) / kTile;
    int *counts = (int *)c->sort_counts;
    uint64_t *ka = c->keys, *kb = c->keys_alt;
    uint32_t *va = c->idx, *vb = c->idx_alt;
    for (int shift = 0; shift < 64; shift += 8) {
        hist_kernel<<<tiles, kSortThreads, 0, c->stream>>>(ka, n, shift, tiles, counts);
        c->launches += 2 + scan_exclusive(counts, counts, (int64_t)256 * tiles, c->scan_tmp, c->stream);
        scatter_kernel<<<tiles, kSortThreads, 0, c->stream>>>(ka, va, kb, vb, n, shift, tiles, counts);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    // eight passes: the sorted pairs are back in c->keys / c->idx
}

}  // namespace hts
