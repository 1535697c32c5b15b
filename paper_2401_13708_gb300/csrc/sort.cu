// sort.cu -- LSD radix sort of (key, index) pairs and an exclusive int scan.
//
// The tree of Sec. 4.1 is a hierarchy over the keys, so sorting the points
// by key puts every cell's points in one contiguous run.  Eight stable
// passes of 8 bits each (58 key bits + 6 segment bits), one kernel per pass:
//   digit_hist  once per sort: the global histograms of all eight digits
//               (they do not depend on the order of the keys; shared-memory
//               atomics per key and digit), then an exclusive scan of each
//               gives every digit its first slot;
//   onesweep    per pass, one tile per block (1024, 2048 or 4096 keys of
//               256 threads, or 8192 keys of 512 threads, by problem size:
//               tile_keys), tiles taken in launch
//               order from an atomic counter: warp histograms (the lanes
//               sharing a digit from eight ballots, one per digit bit), the
//               tile's per-digit counts published to a status word, and a
//               decoupled look-back over earlier tiles (thread d for digit
//               d, kLookBack status words per round trip) adds up the keys
//               of digit d before this tile; then each key is ranked among
//               equal digits in order and written out.  Look-back spins are
//               bounded: a timeout sets a status bit (reported as an
//               error), and out-of-range positions are never written.
// Traffic per pass: 12 B read + 12 B write per key (+ 8 B read once for the
// histograms).
#include <cuda/atomic>

#include <algorithm>

#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kSmallMax = 4096;    // up to this many keys, one block sorts (small_sort_kernel)
constexpr int kMinTile = 1024;     // one-sweep tiles hold 1024, 2048, 4096 or 8192 keys (tile_keys)
constexpr int kSortThreads = 256;
constexpr int kWarps = kSortThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

constexpr int kPasses = 8;
constexpr unsigned long long kFlagAgg = 1ull << 62;   // tile count published
constexpr unsigned long long kFlagPre = 2ull << 62;   // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookBack = 8;  // status words loaded per look-back round trip
// above this, 8192-key tiles of 512 threads (4096-key tiles of 256 threads
// serve sizes between 524,288 and this bound when it is raised)
constexpr int64_t kBigTileFrom = 524288;

// Keys per one-sweep tile.  A pass is latency-bound: one block ranks and
// writes its tile in kTile / 256 sequential rounds, so smaller tiles finish
// sooner while there are SMs to spare; large problems take larger tiles
// (fewer look-back steps and status words: every tile of a pass is resident
// at once, so the last tile looks back over nearly all of them).  Measured
// sort times per iteration: 20,000 keys 156 / 110 / 87 us with 4096 / 2048 /
// 1024-key tiles, 262,145 keys 174 / 143 / 152 us, 1,000,000 keys 283 / 295 /
// 301 us (before the ballot ranking and the batched look-back); with them,
// 1,000,000 keys 198 us with 4096-key tiles and 185 us with 8192 keys of 512
// threads (700,000 keys: 181 / 180 us).
int tile_keys(int64_t n)
{
    return n <= 196608 ? 1024 : n <= 524288 ? 2048 : n <= kBigTileFrom ? 4096 : 8192;
}

// The lanes of the warp whose 8-bit digit equals this lane's, from eight
// ballots (one per digit bit); a lane that is not `ok` matches only itself.
// Every lane of the warp makes the call.
__device__ __forceinline__ unsigned digit_peers(int dg, bool ok, int lane)
{
    const unsigned valid = __ballot_sync(0xffffffffu, ok);
    unsigned m = ok ? valid : (1u << lane);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const unsigned bb = __ballot_sync(0xffffffffu, (dg >> b) & 1);
        m &= ((dg >> b) & 1) ? bb : ~bb;
    }
    return m;
}

// Global histograms of all eight digits; hist[pass][digit] (2048 ints).
template <int kTile>
__global__ void __launch_bounds__(kSortThreads) digit_hist_kernel(const uint64_t *__restrict__ keys, int n,
                                                                  int *hist)
{
    __shared__ int h[kPasses][256];
    for (int k = threadIdx.x; k < kPasses * 256; k += kSortThreads) (&h[0][0])[k] = 0;
    __syncthreads();
    const int base = blockIdx.x * kTile;
    for (int r = 0; r < kTile / kSortThreads; ++r) {
        const int i = base + r * kSortThreads + threadIdx.x;
        const bool ok = i < n;
        const uint64_t key = ok ? keys[i] : 0ull;
#pragma unroll
        for (int p = 0; p < kPasses; ++p) {
            if (ok) atomicAdd(&h[p][(int)((key >> (8 * p)) & 0xFFu)], 1);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kPasses * 256; k += kSortThreads) {
        const int v = (&h[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

// hist[pass][digit] -> exclusive prefix over digits (in place), one warp per pass.
__global__ void digit_offsets_kernel(int *hist)
{
    const int p = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (p >= kPasses) return;
    int *h = hist + p * 256;
    int v[8], local = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = h[lane * 8 + k];
        local += v[k];
    }
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    int run = incl - local;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        h[lane * 8 + k] = run;
        run += v[k];
    }
}

template <int kTile, int kThreads = kSortThreads>
__global__ void __launch_bounds__(kThreads) onesweep_kernel(const uint64_t *__restrict__ kin,
                                                                const uint32_t *__restrict__ vin,
                                                                uint64_t *__restrict__ kout,
                                                                uint32_t *__restrict__ vout, int n, int shift,
                                                                const int *__restrict__ digit_off,
                                                                unsigned long long *tile_status, int *tile_ctr,
                                                                int *status, int spin_limit, int withhold_first)
{
    constexpr int kW = kThreads / 32;  // warps per tile
    constexpr int kPerWarp = kTile / kW;
    constexpr int kRounds = kPerWarp / 32;
    __shared__ int wh[kW][256];
    __shared__ int s_tile;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < kW * 256; k += kThreads) (&wh[0][0])[k] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1);  // tiles in launch order
    __syncthreads();
    const int tile = s_tile;

    const int base = tile * kTile + w * kPerWarp;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[kRounds];
    uint32_t val[kRounds];
    unsigned peers[kRounds];  // lanes of the round with the same digit (kept for the scatter)
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int i = base + r * 32 + lane;
        bool ok = i < n;
        key[r] = ok ? kin[i] : 0ull;
        val[r] = ok ? vin[i] : 0u;
        const int dg = (int)((key[r] >> shift) & 0xFFu);
        const unsigned m = digit_peers(dg, ok, lane);
        peers[r] = m;
        if (ok && (m & lt) == 0u) wh[w][dg] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;  // the first 256 threads: one digit each
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            const int t = wh[k][d];
            wh[k][d] = cnt;  // exclusive prefix over the warps of this tile
            cnt += t;
        }
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> mine(tile_status[(size_t)tile * 256 + d]);
        long long excl = 0;
        if (tile == 0) {
            // (withhold_first: the wait test of hts_set_wait_test; the later
            // tiles' waits then run out)
            if (!withhold_first) mine.store(kFlagPre | (unsigned long long)cnt, cuda::memory_order_relaxed);
        } else {
            mine.store(kFlagAgg | (unsigned long long)cnt, cuda::memory_order_relaxed);
            // decoupled look-back: add tile counts until an inclusive prefix,
            // kLookBack earlier tiles per round trip (their loads are
            // independent; a tile whose word is not yet published is waited
            // for in order).  Tile 0 always holds an inclusive prefix, so the
            // walk ends there at the latest.
            bool done = false;
            for (int t = tile - 1; t >= 0 && !done; t -= kLookBack) {
                unsigned long long v[kLookBack];
#pragma unroll
                for (int j = 0; j < kLookBack; ++j)
                    v[j] = t - j >= 0 ? cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(
                                            tile_status[(size_t)(t - j) * 256 + d])
                                            .load(cuda::memory_order_relaxed)
                                      : 0ull;
#pragma unroll
                for (int j = 0; j < kLookBack; ++j) {
                    if (done || t - j < 0) break;
                    unsigned long long vj = v[j];
                    int spins = 0;
                    while ((vj >> 62) == 0ull && ++spins < spin_limit) {
                        __nanosleep(64);
                        vj = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(
                                 tile_status[(size_t)(t - j) * 256 + d])
                                 .load(cuda::memory_order_relaxed);
                    }
                    if ((vj >> 62) == 0ull) {  // gave up: report (HTS_ETIMEOUT), positions invalid
                        atomicOr(status, 128);
                        excl = (long long)n;
                        done = true;
                        break;
                    }
                    excl += (long long)(vj & kValMask);
                    done = (vj & kFlagPre) && !(vj & kFlagAgg);
                }
            }
            mine.store(kFlagPre | (unsigned long long)(excl + cnt), cuda::memory_order_relaxed);
        }
        const int off = digit_off[d] + (int)min(excl, (long long)n);
#pragma unroll
        for (int k = 0; k < kW; ++k) wh[k][d] += off;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int i = base + r * 32 + lane;
        bool ok = i < n;
        const int dg = (int)((key[r] >> shift) & 0xFFu);
        int pos = 0;
        if (ok) pos = wh[w][dg] + __popc(peers[r] & lt);
        __syncwarp();
        if (ok && (peers[r] & lt) == 0u) wh[w][dg] += __popc(peers[r]);
        __syncwarp();
        if (ok) {
            if (pos >= 0 && pos < n) {
                kout[pos] = key[r];
                vout[pos] = val[r];
            } else {
                atomicOr(status, 4);
            }
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

namespace {

// n <= kSmallMax: all eight passes in one block (no look-back: the block's own
// histogram is the global one), ping-ponging through the two key buffers.
// ROUNDS keys per lane: 256 * ROUNDS >= n (fewer rounds for fewer keys).
template <int ROUNDS>
__global__ void __launch_bounds__(kSortThreads) small_sort_kernel(uint64_t *ka, uint32_t *va, uint64_t *kb,
                                                                  uint32_t *vb, int n)
{
    constexpr int kRounds = ROUNDS;
    __shared__ int wh[kWarps][256];
    __shared__ int dsum[256];
    __shared__ int wtot[kWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int base = w * 32 * ROUNDS;
    for (int p = 0; p < kPasses; ++p) {
        const uint64_t *kin = (p & 1) ? kb : ka;
        const uint32_t *vin = (p & 1) ? vb : va;
        uint64_t *kout = (p & 1) ? ka : kb;
        uint32_t *vout = (p & 1) ? va : vb;
        const int shift = 8 * p;
        for (int k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wh[0][0])[k] = 0;
        __syncthreads();
        uint64_t key[kRounds];
        uint32_t val[kRounds];
        unsigned peers[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int i = base + r * 32 + lane;
            const bool ok = i < n;
            key[r] = ok ? kin[i] : 0ull;
            val[r] = ok ? vin[i] : 0u;
            const int dg = (int)((key[r] >> shift) & 0xFFu);
            peers[r] = digit_peers(dg, ok, lane);
            if (ok && (peers[r] & lt) == 0u) wh[w][dg] += __popc(peers[r]);
            __syncwarp();
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < kWarps; ++k) {
                const int t = wh[k][d];
                wh[k][d] = cnt;
                cnt += t;
            }
            // exclusive scan of the 256 digit counts: warp scans, then warp totals
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) wtot[w] = incl;
            dsum[d] = incl - cnt;
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            int off = dsum[d];
            for (int k = 0; k < w; ++k) off += wtot[k];
#pragma unroll
            for (int k = 0; k < kWarps; ++k) wh[k][d] += off;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int i = base + r * 32 + lane;
            const bool ok = i < n;
            const int dg = (int)((key[r] >> shift) & 0xFFu);
            int pos = 0;
            if (ok) pos = wh[w][dg] + __popc(peers[r] & lt);
            __syncwarp();
            if (ok && (peers[r] & lt) == 0u) wh[w][dg] += __popc(peers[r]);
            __syncwarp();
            if (ok && pos >= 0 && pos < n) {
                kout[pos] = key[r];
                vout[pos] = val[r];
            }
        }
        __syncthreads();  // this pass's output is the next pass's input
    }
}

}  // namespace

size_t sort_status_words(int64_t n)
{
    const int64_t tiles = (n + kMinTile - 1) / kMinTile;  // the most tiles any size up to n uses
    return (size_t)kPasses * 256 * (size_t)std::max<int64_t>(tiles, 1);
}

void launch_sort_pairs(hts_ctx *c)
{
    const int n = (int)c->n;
    const int tile = tile_keys(n);
    const int tiles = (n + tile - 1) / tile;
    static_assert(kSmallMax == kSortThreads * 16, "small_sort_kernel<16> covers kSmallMax keys");
    if (n <= kSmallMax) {  // one block does all eight passes
        if (n <= kSortThreads * 4)
            small_sort_kernel<4><<<1, kSortThreads, 0, c->stream>>>(c->keys, c->idx, c->keys_alt, c->idx_alt, n);
        else if (n <= kSortThreads * 8)
            small_sort_kernel<8><<<1, kSortThreads, 0, c->stream>>>(c->keys, c->idx, c->keys_alt, c->idx_alt, n);
        else
            small_sort_kernel<16><<<1, kSortThreads, 0, c->stream>>>(c->keys, c->idx, c->keys_alt, c->idx_alt, n);
        c->launches += 1;
        return;
    }
    // scratch: 2048 ints of digit offsets, 8 tile counters, then the status words
    int *hist = reinterpret_cast<int *>(c->sort_scratch);
    int *ctr = hist + kPasses * 256;
    unsigned long long *stat = reinterpret_cast<unsigned long long *>(c->sort_scratch + (kPasses * 256 + 64) / 2);
    cudaMemsetAsync(c->sort_scratch, 0, sizeof(unsigned long long) * ((kPasses * 256 + 64) / 2 +
                                                                      (size_t)kPasses * 256 * tiles), c->stream);
    // (the histograms do not depend on the pass tiles: at most 4096 keys per
    // block keeps enough blocks in flight)
    const int hblocks = (n + 4095) / 4096;
    if (tile == 1024)
        digit_hist_kernel<1024><<<tiles, kSortThreads, 0, c->stream>>>(c->keys, n, hist);
    else if (tile == 2048)
        digit_hist_kernel<2048><<<tiles, kSortThreads, 0, c->stream>>>(c->keys, n, hist);
    else
        digit_hist_kernel<4096><<<hblocks, kSortThreads, 0, c->stream>>>(c->keys, n, hist);
    digit_offsets_kernel<<<1, 32 * kPasses, 0, c->stream>>>(hist);
    c->launches += 2 + kPasses;
    uint64_t *ka = c->keys, *kb = c->keys_alt;
    uint32_t *va = c->idx, *vb = c->idx_alt;
    const int spin = c->wait_test > 0 ? c->wait_test : kSpinLimit;
    const int hold = c->wait_test > 0 ? 1 : 0;
    for (int p = 0; p < kPasses; ++p) {
        unsigned long long *sp = stat + (size_t)p * 256 * tiles;
        if (tile == 1024)
            onesweep_kernel<1024><<<tiles, kSortThreads, 0, c->stream>>>(ka, va, kb, vb, n, 8 * p, hist + p * 256,
                                                                         sp, ctr + p, c->status, spin, hold);
        else if (tile == 2048)
            onesweep_kernel<2048><<<tiles, kSortThreads, 0, c->stream>>>(ka, va, kb, vb, n, 8 * p, hist + p * 256,
                                                                         sp, ctr + p, c->status, spin, hold);
        else if (tile == 4096)
            onesweep_kernel<4096><<<tiles, kSortThreads, 0, c->stream>>>(ka, va, kb, vb, n, 8 * p, hist + p * 256,
                                                                         sp, ctr + p, c->status, spin, hold);
        else
            onesweep_kernel<8192, 2 * kSortThreads><<<tiles, 2 * kSortThreads, 0, c->stream>>>(
                ka, va, kb, vb, n, 8 * p, hist + p * 256, sp, ctr + p, c->status, spin, hold);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    // eight passes: the sorted pairs are back in c->keys / c->idx
}

}  // namespace hts
