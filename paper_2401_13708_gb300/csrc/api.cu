// api.cu -- the C ABI of libhts (declared in include/hts.h).
//
// One iteration (hts_step) queues, on the context's stream:
//   prep_points -> make_keys -> sort (8 passes) -> build_tree -> walk
//   -> attract -> reduce_z -> update
// or, for theta == 0, prep_points -> exact -> attract -> reduce_z -> update.
// Nothing is allocated and nothing is copied to the host inside the loop;
// the status word is read once after the last iteration.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hts_internal.cuh"

using namespace hts;

namespace {

int fail(hts_ctx *c, int code, const char *msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(hts_ctx *c, cudaError_t e, const char *where)
{
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    }
    return e == cudaErrorMemoryAllocation ? HTS_EOOM : HTS_ECUDA;
}

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

#define LAUNCHED(what)                                       \
    do {                                                     \
        cudaError_t e_ = cudaGetLastError();                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <typename T>
int dalloc(hts_ctx *c, T **p, size_t count)
{
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(c, e, "cudaMalloc");
    }
    return HTS_OK;
}

template <typename T>
void dfree(T **p)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
}

int set_device(hts_ctx *c)
{
    cudaError_t e = cudaSetDevice(c->cfg.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return HTS_OK;
}

// Check that a pointer given as HTS_DEVICE is device memory of our device.
int check_device_ptr(hts_ctx *c, const void *p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HTS_EINVAL, "pointer given as HTS_DEVICE is not CUDA memory");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(c, HTS_EINVAL, "pointer given as HTS_DEVICE is not device memory");
    if (a.type == cudaMemoryTypeDevice && a.device != c->cfg.device)
        return fail(c, HTS_EINVAL, "device pointer belongs to another device");
    return HTS_OK;
}

int ensure_points(hts_ctx *c, int64_t n)
{
    if (n == c->cap_n && (c->pts32 || c->pts64)) return HTS_OK;
    const size_t N = (size_t)std::max<int64_t>(n, 1);
    c->cap_n = -1;  // until every buffer below has its new size
    int r;
#define AL(ptr, cnt) \
    if ((r = dalloc(c, &(ptr), (cnt))) != HTS_OK) return r
    AL(c->y, N);
    AL(c->vel, N);
    AL(c->gains, N);
    AL(c->fattr, N);
    AL(c->frep, N);
    AL(c->zi, N);
    AL(c->radial, N);
    if (c->cfg.precision == HTS_FP32_MIXED) {
        AL(c->pts32, N);
        AL(c->apts32, N);
        AL(c->spts32, N);
        AL(c->nodes32, 2 * N + kWalkOverrun);
    } else {
        AL(c->pts64, N);
        AL(c->spts64, N);
        AL(c->nodes64, 2 * N);
    }
    // a node slot never written by a tree build reads as an empty bucket
    // (count 0), which the walk steps over
    if (c->nodes32 && cudaMemset(c->nodes32, 0, sizeof(NodeF) * (2 * N + kWalkOverrun)) != cudaSuccess)
        return HTS_ECUDA;
    if (c->nodes64 && cudaMemset(c->nodes64, 0, sizeof(NodeD) * 2 * N) != cudaSuccess) return HTS_ECUDA;
    AL(c->keys, N);
    AL(c->keys_alt, N);
    AL(c->idx, N);
    AL(c->idx_alt, N);
    AL(c->terms, 3 * N);
    AL(c->bn_left, N);
    AL(c->bn_right, N);
    AL(c->bn_parent, N);
    AL(c->leaf_parent, N);
    AL(c->bn_lo, N);
    AL(c->bn_hi, N);
    AL(c->bn_pref, N);
    AL(c->bn_flag, N);
    AL(c->bn_quad, N);
    AL(c->bn_sum, 6 * (N + 1));  // 3 x 128-bit fixed-point prefix sums (n + 1 entries, 48 B each)
    AL(c->cnt, N + 1);
    AL(c->pre, N + 1);
    AL(c->walk_cost, (N + 31) / 32);       // one per walk block (at most one per warp)
    AL(c->walk_order, (N + 31) / 32 + 1);
    if (cudaMemset(c->walk_cost, 0, sizeof(unsigned) * ((N + 31) / 32)) != cudaSuccess ||
        cudaMemset(c->walk_order, 0, sizeof(int) * ((N + 31) / 32 + 1)) != cudaSuccess)
        return HTS_ECUDA;
    const int64_t tiles = ((int64_t)N + 4095) / 4096;
    AL(c->sort_scratch, (8 * 256 + 64) / 2 + sort_status_words((int64_t)N));
    c->scan_tmp_len = scan_tmp_size(std::max<int64_t>(256 * tiles, (int64_t)N + 1));
    AL(c->scan_tmp, (size_t)c->scan_tmp_len);
    AL(c->red_tmp, std::max<size_t>(3 * ((size_t)N * 32 / 256 + 2), 512));  // also >= 6 (N / 1024 + 2)
    {
        const int sp = exact_split((int64_t)N);
        AL(c->exact_part, sp > 1 ? 4 * (size_t)sp * N : 4);
        const int cap = walk_split_capacity((int64_t)N);  // split walk partial sums (float4 / double4)
        double *part = (double *)c->split_part, *fr = (double *)c->split_frontier;
        c->split_part = nullptr;
        c->split_frontier = nullptr;
        if (part) cudaFree(part);
        if (fr) cudaFree(fr);
        if ((r = dalloc(c, &part, cap > 0 ? 4 * (size_t)cap * N : 4))) return r;
        if ((r = dalloc(c, &fr, walk_split_frontier_bytes() / sizeof(double) + 1))) {
            cudaFree(part);
            return r;
        }
        c->split_part = part;
        c->split_frontier = fr;
    }
#undef AL
    c->n_nodes = c->pre + n;
    c->cap_n = n;
    return HTS_OK;
}

int read_status(hts_ctx *c, int *out)
{
    CK(cudaMemcpyAsync(c->h_pinned, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    memcpy(out, c->h_pinned, sizeof(int));
    return HTS_OK;
}

int status_error(hts_ctx *c, int st)
{
    if (st & 128) return fail(c, HTS_ETIMEOUT, "a bounded device-side wait (sort look-back) ran out");
    if (st & 64) return fail(c, HTS_EDOMAIN, "a point has |y| >= 1 or a non-finite coordinate");
    if (st & (8 | 16)) return fail(c, HTS_ESHAPE, "malformed CSR (indptr, indices or diagonal entries)");
    if (st & 32) return fail(c, HTS_EDOMAIN, "P has a negative or non-finite value");
    if (st & 1) return fail(c, HTS_ENUMERIC, "non-finite gradient or position after a step");
    if (st & (2 | 4)) return fail(c, HTS_ENUMERIC, "tree build/walk consistency check failed");
    return HTS_OK;
}

constexpr int kPhases = 6;  // keys, sort, tree, walk/exact, attract, Z + update
constexpr int kEvents = kPhases + 3;  // per iteration: 6 marks on the main stream, 2 on the side stream
constexpr int kMaxSplitCut = 3;      // deepest cut the autotuner tries (hts_set_walk_split's range)
// stage after which the attraction forks (0 prep, 1 keys, 2 sort, 3 tree):
// float32 after the sort, float64 (a heavier attraction) after the tree build
constexpr int kAttractAfter32 = 2, kAttractAfter64 = 3;

// Repulsion, attraction and Z for the current Y (results in frep, zi, fattr,
// dscal[0] / seg_z).  The attractive sum needs only the point records, so it
// runs on the side stream (lowest priority) from the stage kAttractAfter32 /
// kAttractAfter64 to the Z reduction, as a small resident grid beside the
// latency-bound tree build and the walk (see launch_attract).  With `ev` (kEvents events)
// the stage boundaries are recorded: ev[0..4] and ev[6] on the main stream
// (start, after keys, sort, tree, walk / exact; ev[6] after the update is
// recorded by the caller), ev[7..8] around the attractive sum.
int run_gradient(hts_ctx *c, double theta, cudaEvent_t *ev = nullptr)
{
#define MARK(k) \
    if (ev) CK(cudaEventRecord(ev[k], c->stream))
    // every phase alone (timing), and the exact path: its kernel fills the GPU
    // by itself, and an attraction beside it only lengthens its tail
    const bool serial = c->profiling == 2 || theta == 0.0;
    const bool attract = c->nnz > 0 && !serial;
    const int fork_at = c->cfg.precision == HTS_FP32_MIXED ? kAttractAfter32 : kAttractAfter64;
    // fork: the side stream waits for the point records (and for the stages
    // before fork_at, so that it does not hold SMs they need)
    auto fork_attract = [&]() -> int {
        CK(cudaEventRecord(c->aev_fork, c->stream));
        CK(cudaStreamWaitEvent(c->astream, c->aev_fork, 0));
        cudaStream_t keep = c->stream;
        c->stream = c->astream;
        if (ev) CK(cudaEventRecord(ev[7], c->astream));
        c->attract_background = 1;
        launch_attract(c);
        c->attract_background = 0;
        c->stream = keep;
        LAUNCHED("attract");
        if (ev) CK(cudaEventRecord(ev[8], c->astream));
        CK(cudaEventRecord(c->aev_join, c->astream));
        return HTS_OK;
    };
    int r = HTS_OK;
    MARK(0);
    launch_prep_points(c);
    LAUNCHED("prep_points");
    if (c->nnz == 0) CK(cudaMemsetAsync(c->fattr, 0, sizeof(double2) * (size_t)c->n, c->stream));
    if (theta == 0.0) {
        MARK(1);
        MARK(2);
        MARK(3);
        launch_exact(c);
        LAUNCHED("exact");
    } else {
        if (attract && fork_at == 0 && (r = fork_attract())) return r;
        launch_make_keys(c);
        LAUNCHED("make_keys");
        MARK(1);
        if (attract && fork_at == 1 && (r = fork_attract())) return r;
        launch_sort_pairs(c);
        LAUNCHED("sort");
        MARK(2);
        if (attract && fork_at == 2 && (r = fork_attract())) return r;
        launch_build_tree(c, theta, nullptr);
        LAUNCHED("build_tree");
        MARK(3);
        if (attract && fork_at == 3 && (r = fork_attract())) return r;
        launch_walk(c);
        LAUNCHED("walk");
    }
    MARK(4);
    if (attract) CK(cudaStreamWaitEvent(c->stream, c->aev_join, 0));  // join
    if (serial && c->nnz > 0) {
        if (ev) CK(cudaEventRecord(ev[7], c->stream));
        launch_attract(c);
        LAUNCHED("attract");
        if (ev) CK(cudaEventRecord(ev[8], c->stream));
    }
    MARK(5);
    launch_reduce_z(c);
    LAUNCHED("reduce_z");
#undef MARK
    return HTS_OK;
}

int ensure_events(hts_ctx *c, int slots)
{
    if (slots <= c->event_slots) return HTS_OK;
    cudaEvent_t *ev = new cudaEvent_t[(size_t)slots * kEvents];
    for (int k = 0; k < c->event_slots * kEvents; ++k) ev[k] = c->events[k];
    for (int k = c->event_slots * kEvents; k < slots * kEvents; ++k) CK(cudaEventCreate(&ev[k]));
    delete[] c->events;
    c->events = ev;
    c->event_slots = slots;
    return HTS_OK;
}

int ready(hts_ctx *c)
{
    if (!c) return HTS_EINVAL;
    if (!c->have_P || !c->have_Y) return fail(c, HTS_ENOTSET, "P and Y must both be set");
    if (c->n != c->cap_n) return fail(c, HTS_ESHAPE, "P and Y sizes differ");
    int r = set_device(c);
    if (r) return r;
    c->err.clear();
    return HTS_OK;
}

int check_theta(hts_ctx *c, double theta)
{
    if (!(theta >= 0.0 && theta <= 1.0)) return fail(c, HTS_EINVAL, "theta must be in [0, 1]");
    return HTS_OK;
}

void free_segments(hts_ctx *c)
{
    dfree(&c->seg_off);
    dfree(&c->seg_of);
    dfree(&c->seg_lr);
    dfree(&c->seg_z);
    c->nseg = 1;
    c->seg_off_h[0] = 0;
    c->seg_off_h[1] = c->n;
}

void drop_graph(hts_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey[0] = -1.0;
}

// Capture one iteration (gradient + update) into c->gexec on the private
// stream, unless the cached graph already matches the arguments and layout.
int capture_iteration(hts_ctx *c, double theta, double exag, double lr, double mom)
{
    const double key[5] = {theta, exag, lr, mom, (double)c->layout_version};
    if (c->gexec && memcmp(key, c->gkey, sizeof(key)) == 0) return HTS_OK;
    drop_graph(c);
    if (!c->gstream) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&c->gstream, cudaStreamNonBlocking, greatest));
        CK(cudaEventCreateWithFlags(&c->gev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->gev_out, cudaEventDisableTiming));
    }
    cudaStream_t keep = c->stream;
    const int64_t l0 = c->launches;
    CK(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    c->stream = c->gstream;
    int r = run_gradient(c, theta);
    if (!r) {
        launch_update(c, exag, lr, mom, nullptr, 1);
        r = cudaGetLastError() == cudaSuccess ? HTS_OK : HTS_ECUDA;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
    c->stream = keep;
    c->graph_launches = c->launches - l0;
    c->launches = l0;
    if (r || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return r ? r : cuda_fail(c, e, "cudaStreamEndCapture");
    }
    // (kernel-node priorities as in eager launches -- attraction lowest -- measured
    // 8% slower on the 64-embedding batch than the graph's default scheduling)
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    memcpy(c->gkey, key, sizeof(key));
    return HTS_OK;
}

// Per-segment KL parts after run_gradient (Z only): kl[s] for s < nseg.
int kl_parts(hts_ctx *c, std::vector<double> &kl)
{
    const int ns = c->nseg;
    std::vector<double> h(4 * (size_t)ns, 0.0);  // Z, sum p log p, sum p log w, sum p
    const double *zsrc = ns > 1 ? c->seg_z : c->dscal;
    CK(cudaMemcpyAsync(h.data(), zsrc, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->stream));
    if (c->nnz > 0 && ns == 1) {
        launch_kl_terms(c);
        LAUNCHED("kl_terms");
        CK(cudaMemcpyAsync(h.data() + 1, c->dscal + 1, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    } else if (c->nnz > 0) {
        const size_t n = (size_t)c->n;
        double *a = c->terms, *b = c->terms + n, *pp = c->terms + 2 * n;  // 3n doubles of scratch
        launch_kl_rows(c, a, b, pp);
        LAUNCHED("kl_rows");
        double *out = c->red_tmp;  // >= 3 * HTS_MAX_SEGMENTS doubles
        launch_segment_sums(c, a, out);
        launch_segment_sums(c, b, out + HTS_MAX_SEGMENTS);
        launch_segment_sums(c, pp, out + 2 * HTS_MAX_SEGMENTS);
        LAUNCHED("segment_sums");
        for (int k = 0; k < 3; ++k)
            CK(cudaMemcpyAsync(h.data() + (size_t)(k + 1) * ns, out + k * HTS_MAX_SEGMENTS, sizeof(double) * ns,
                               cudaMemcpyDeviceToHost, c->stream));
    }
    int st = 0;
    int r = read_status(c, &st);  // synchronises the stream
    if (r) return r;
    if ((r = status_error(c, st))) return r;
    kl.assign((size_t)ns, 0.0);
    for (int s = 0; s < ns; ++s) {
        double Z, a, b, sp;
        if (ns == 1) {
            Z = h[0]; a = h[1]; b = h[2]; sp = h[3];
        } else {
            Z = h[s]; a = h[(size_t)ns + s]; b = h[2 * (size_t)ns + s]; sp = h[3 * (size_t)ns + s];
        }
        kl[s] = a - b + (sp > 0.0 ? sp * log(Z) : 0.0);
    }
    return HTS_OK;
}

__global__ void convert_values_kernel(int64_t nnz, const void *in, int in_f64, void *out, int out_f64)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    double v = in_f64 ? ((const double *)in)[e] : (double)((const float *)in)[e];
    if (out_f64) ((double *)out)[e] = v; else ((float *)out)[e] = (float)v;
}

__global__ void fill_state_kernel(int64_t n, double2 *vel, double2 *gains)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vel[i] = make_double2(0.0, 0.0);
    gains[i] = make_double2(1.0, 1.0);
}

}  // namespace

extern "C" {

void hts_default_config(hts_config *cfg)
{
    if (!cfg) return;
    cfg->precision = HTS_FP32_MIXED;
    cfg->split_rule = HTS_EQUAL_LENGTH;
    cfg->grad_form = HTS_EXACT_KL;
    cfg->metric_pow = 1;
    cfg->eps = 1e-5;
    cfg->use_gains = 0;
    cfg->device = 0;
    cfg->stream = nullptr;
}

int hts_create(hts_ctx **out, const hts_config *cfg)
{
    if (!out) return HTS_EINVAL;
    *out = nullptr;
    hts_config k;
    if (cfg) k = *cfg; else hts_default_config(&k);
    if ((k.precision != HTS_FP64 && k.precision != HTS_FP32_MIXED) ||
        (k.split_rule != HTS_EQUAL_LENGTH && k.split_rule != HTS_EQUAL_AREA) ||
        (k.grad_form != HTS_EXACT_KL && k.grad_form != HTS_PAPER_EQ) || (k.metric_pow != 1 && k.metric_pow != 2) ||
        !(k.eps > 0.0 && k.eps < 0.5) || k.device < 0)
        return HTS_EINVAL;
    hts_ctx *c = new hts_ctx();
    c->cfg = k;
    c->stream = (cudaStream_t)k.stream;
    int r = set_device(c);
    if (r) {
        delete c;
        return r;
    }
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, k.device);
    if (e != cudaSuccess) {
        delete c;
        return HTS_ECUDA;
    }
    c->sm_count = prop.multiProcessorCount;
    if (dalloc(c, &c->minmax, 2 * kMaxSegments + 2) || dalloc(c, &c->dscal, 8) || dalloc(c, &c->status, 1) ||
        dalloc(c, &c->counters, 5) || cudaMallocHost((void **)&c->h_pinned, 8 * sizeof(double)) != cudaSuccess) {
        hts_destroy(c);
        return HTS_EOOM;
    }
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (cudaStreamCreateWithPriority(&c->astream, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->pstream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->tstream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->tev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->tev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->aev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->aev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->pev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->pev_out, cudaEventDisableTiming) != cudaSuccess) {
        hts_destroy(c);
        return HTS_ECUDA;
    }
    cudaMemset(c->counters, 0, 5 * sizeof(unsigned long long));
    cudaMemset(c->status, 0, sizeof(int));
    *out = c;
    return HTS_OK;
}

void hts_destroy(hts_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->cfg.device);
    // every stream of the context is idle before a buffer is freed (a failed
    // call can leave work on a side stream that was never joined)
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    if (c->pstream) cudaStreamSynchronize(c->pstream);
    if (c->astream) cudaStreamSynchronize(c->astream);
    if (c->tstream) cudaStreamSynchronize(c->tstream);
    if (c->gstream) cudaStreamSynchronize(c->gstream);
    dfree(&c->indptr); dfree(&c->indices); dfree(&c->values);
    dfree(&c->y); dfree(&c->vel); dfree(&c->gains); dfree(&c->fattr); dfree(&c->frep);
    dfree(&c->zi); dfree(&c->radial); dfree(&c->pts32); dfree(&c->pts64);
    dfree(&c->keys); dfree(&c->keys_alt); dfree(&c->idx); dfree(&c->idx_alt);
    dfree(&c->spts32); dfree(&c->spts64); dfree(&c->terms);
    dfree(&c->bn_left); dfree(&c->bn_right); dfree(&c->bn_parent); dfree(&c->leaf_parent);
    dfree(&c->bn_lo); dfree(&c->bn_hi); dfree(&c->bn_pref); dfree(&c->bn_flag); dfree(&c->bn_quad);
    dfree(&c->bn_sum); dfree(&c->cnt); dfree(&c->pre); dfree(&c->nodes32); dfree(&c->apts32); dfree(&c->walk_cost); dfree(&c->walk_order); dfree(&c->nodes64);
    dfree(&c->sort_scratch); dfree(&c->scan_tmp); dfree(&c->exact_part);
    if (c->split_part) cudaFree(c->split_part);
    if (c->split_frontier) cudaFree(c->split_frontier); dfree(&c->red_tmp); dfree(&c->minmax);
    dfree(&c->dscal); dfree(&c->status); dfree(&c->counters); dfree(&c->xsq);
    dfree(&c->seg_off); dfree(&c->seg_of); dfree(&c->seg_lr); dfree(&c->seg_z);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->gev_in) cudaEventDestroy(c->gev_in);
    if (c->gev_out) cudaEventDestroy(c->gev_out);
    if (c->astream) cudaStreamDestroy(c->astream);
    if (c->pstream) cudaStreamDestroy(c->pstream);
    if (c->tstream) cudaStreamDestroy(c->tstream);
    if (c->tev_fork) cudaEventDestroy(c->tev_fork);
    if (c->tev_join) cudaEventDestroy(c->tev_join);
    if (c->aev_fork) cudaEventDestroy(c->aev_fork);
    if (c->aev_join) cudaEventDestroy(c->aev_join);
    if (c->pev_in) cudaEventDestroy(c->pev_in);
    if (c->pev_out) cudaEventDestroy(c->pev_out);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    for (int k = 0; k < c->event_slots * kEvents; ++k) cudaEventDestroy(c->events[k]);
    delete[] c->events;
    delete c;
}

const char *hts_last_error(const hts_ctx *c)
{
    if (!c) return "no context";
    return c->err.c_str();
}

int hts_set_P(hts_ctx *c, int64_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices, const void *values,
              int dtype, int where)
{
    if (!c) return HTS_EINVAL;
    c->err.clear();
    if (n < 0 || n > (1 << 30) || nnz < 0 || nnz > ((int64_t)1 << 40) || !indptr ||
        (nnz > 0 && (!indices || !values)) || (dtype != HTS_F32 && dtype != HTS_F64) ||
        (where != HTS_HOST && where != HTS_DEVICE))
        return fail(c, HTS_EINVAL, "hts_set_P: invalid argument");
    if (c->have_Y && n != c->n) return fail(c, HTS_ESHAPE, "hts_set_P: n differs from the n of Y");
    int r = set_device(c);
    if (r) return r;
    const int in_f64 = dtype == HTS_F64;
    const int out_f64 = c->cfg.precision == HTS_FP64;
    if (where == HTS_HOST) {
        if (indptr[0] != 0 || indptr[n] != nnz) return fail(c, HTS_ESHAPE, "hts_set_P: indptr[0] != 0 or indptr[n] != nnz");
        for (int64_t i = 0; i < n; ++i) {
            if (indptr[i + 1] < indptr[i]) return fail(c, HTS_ESHAPE, "hts_set_P: indptr decreases");
            for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e) {
                int32_t j = indices[e];
                if (j < 0 || j >= n || j == i) return fail(c, HTS_ESHAPE, "hts_set_P: index out of range or diagonal");
                double v = in_f64 ? ((const double *)values)[e] : (double)((const float *)values)[e];
                if (!(v >= 0.0) || !isfinite(v)) return fail(c, HTS_EDOMAIN, "hts_set_P: negative or non-finite value");
            }
        }
    } else {
        if ((r = check_device_ptr(c, indptr))) return r;
        if (nnz > 0 && ((r = check_device_ptr(c, indices)) || (r = check_device_ptr(c, values)))) return r;
    }
    c->have_P = false;  // the buffers change below: no P until this call succeeds
    c->layout_version += 1;
    if ((r = dalloc(c, &c->indptr, (size_t)n + 1))) return r;
    if ((r = dalloc(c, &c->indices, (size_t)nnz))) return r;
    if (out_f64) {
        double *v = nullptr;
        if ((r = dalloc(c, &v, (size_t)nnz))) return r;
        dfree(&c->values);
        c->values = v;
    } else {
        float *v = nullptr;
        if ((r = dalloc(c, &v, (size_t)nnz))) return r;
        dfree(&c->values);
        c->values = v;
    }
    cudaMemcpyKind kind = where == HTS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(c->indptr, indptr, sizeof(int64_t) * (size_t)(n + 1), kind, c->stream));
    if (nnz > 0) CK(cudaMemcpyAsync(c->indices, indices, sizeof(int32_t) * (size_t)nnz, kind, c->stream));
    if (nnz > 0) {
        if (in_f64 == out_f64) {
            CK(cudaMemcpyAsync(c->values, values, (size_t)nnz * (in_f64 ? 8 : 4), kind, c->stream));
        } else if (where == HTS_HOST) {
            if (out_f64) {
                std::vector<double> tmp((size_t)nnz);
                for (int64_t e = 0; e < nnz; ++e) tmp[e] = ((const float *)values)[e];
                CK(cudaMemcpy(c->values, tmp.data(), 8 * (size_t)nnz, cudaMemcpyHostToDevice));
            } else {
                std::vector<float> tmp((size_t)nnz);
                for (int64_t e = 0; e < nnz; ++e) tmp[e] = (float)((const double *)values)[e];
                CK(cudaMemcpy(c->values, tmp.data(), 4 * (size_t)nnz, cudaMemcpyHostToDevice));
            }
        } else {
            convert_values_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, c->stream>>>(nnz, values, in_f64,
                                                                                      c->values, out_f64);
            LAUNCHED("convert_values");
        }
    }
    if (where == HTS_DEVICE && n > 0) {
        CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        launch_validate_csr(c, (int)n, nnz, c->indptr, c->indices, c->values, out_f64);
        LAUNCHED("validate_csr");
        int st = 0;
        if ((r = read_status(c, &st))) return r;
        if (st) {
            c->have_P = false;
            return status_error(c, st);
        }
    }
    CK(cudaStreamSynchronize(c->stream));
    c->values_f64 = out_f64;
    c->nnz = nnz;
    c->layout_version += 1;
    if (c->nseg > 1 && n == c->n && n > 0) {  // segments stay: P must respect them
        CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        launch_segments_setup(c);
        LAUNCHED("segments_setup");
        int st = 0;
        if ((r = read_status(c, &st))) return r;
        if (st) {
            c->have_P = false;
            return fail(c, HTS_ESHAPE, "hts_set_P: P is not block diagonal over the segments");
        }
    } else if (c->nseg > 1) {
        free_segments(c);
    }
    c->n = n;
    c->seg_off_h[1] = c->nseg == 1 ? n : c->seg_off_h[1];
    c->have_P = true;
    return HTS_OK;
}

int hts_set_Y(hts_ctx *c, int64_t n, const double *y, int where)
{
    if (!c) return HTS_EINVAL;
    c->err.clear();
    if (n < 0 || n > (1 << 30) || (n > 0 && !y) || (where != HTS_HOST && where != HTS_DEVICE))
        return fail(c, HTS_EINVAL, "hts_set_Y: invalid argument");
    if (c->have_P && n != c->n) return fail(c, HTS_ESHAPE, "hts_set_Y: n differs from the n of P");
    int r = set_device(c);
    if (r) return r;
    if (where == HTS_DEVICE && n > 0 && (r = check_device_ptr(c, y))) return r;
    if (c->xsq && n != c->n) {
        dfree(&c->xsq);  // the per-point term no longer matches
        c->cosne_l1 = 1.0;
        c->cosne_l2 = 0.0;
    }
    if (n != c->n && c->nseg > 1) free_segments(c);
    // buffers move (and captured graphs go stale) only when the size changes
    if (n != c->n || n != c->cap_n || !(c->pts32 || c->pts64)) c->layout_version += 1;
    c->have_Y = false;  // until this call succeeds
    if ((r = ensure_points(c, n))) return r;
    if (n > 0) {
        CK(cudaMemcpyAsync(c->y, y, sizeof(double2) * (size_t)n,
                           where == HTS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
        fill_state_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->vel, c->gains);
        LAUNCHED("fill_state");
        // host and device inputs alike are checked on the device (one pass,
        // no host loop over the points); the status read also completes the copy
        CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        c->n = n;
        launch_check_y(c);
        LAUNCHED("check_y");
        int st = 0;
        if ((r = read_status(c, &st))) return r;
        if (st) {
            c->have_Y = false;
            return status_error(c, st);
        }
    }
    c->n = n;
    if (c->nseg == 1) c->seg_off_h[1] = n;
    c->iters = 0;
    c->have_Y = true;
    return HTS_OK;
}

int hts_update_Y(hts_ctx *c, const double *y, int where)
{
    if (!c) return HTS_EINVAL;
    c->err.clear();
    if (!c->have_Y) return fail(c, HTS_ENOTSET, "hts_update_Y: set Y first");
    if ((c->n > 0 && !y) || (where != HTS_HOST && where != HTS_DEVICE))
        return fail(c, HTS_EINVAL, "hts_update_Y: invalid argument");
    int r = set_device(c);
    if (r) return r;
    if (c->n == 0) return HTS_OK;
    if (where == HTS_DEVICE && (r = check_device_ptr(c, y))) return r;
    CK(cudaMemcpyAsync(c->y, y, sizeof(double2) * (size_t)c->n,
                       where == HTS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    launch_check_y(c);
    LAUNCHED("check_y");
    int st = 0;
    if ((r = read_status(c, &st))) return r;
    if (st) {
        c->have_Y = false;
        return status_error(c, st);
    }
    return HTS_OK;
}

int hts_step(hts_ctx *c, int n_iter, double theta, double exaggeration, double lr, double momentum)
{
    int r = ready(c);
    if (r) return r;
    if (n_iter < 0 || !(exaggeration > 0.0) || !(lr >= 0.0) || !(momentum >= 0.0 && momentum <= 1.0) ||
        !isfinite(exaggeration) || !isfinite(lr))
        return fail(c, HTS_EINVAL, "hts_step: invalid n_iter, exaggeration, lr or momentum");
    if ((r = check_theta(c, theta))) return r;
    if (c->n == 0 || n_iter == 0) return HTS_OK;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    const int prof = c->profiling ? std::min(n_iter, 4096) : 0;
    if (prof && (r = ensure_events(c, prof))) return r;
    if (c->use_graphs && !prof && !c->counters_on) {
        if ((r = capture_iteration(c, theta, exaggeration, lr, momentum))) return r;
        CK(cudaEventRecord(c->gev_in, c->stream));
        CK(cudaStreamWaitEvent(c->gstream, c->gev_in, 0));
        for (int it = 0; it < n_iter; ++it) CK(cudaGraphLaunch(c->gexec, c->gstream));
        CK(cudaEventRecord(c->gev_out, c->gstream));
        CK(cudaStreamWaitEvent(c->stream, c->gev_out, 0));
        c->launches += c->graph_launches * n_iter;
    } else {
        // the iterations run on the high-priority stream, between two events
        CK(cudaEventRecord(c->pev_in, c->stream));
        CK(cudaStreamWaitEvent(c->pstream, c->pev_in, 0));
        cudaStream_t user = c->stream;
        c->stream = c->pstream;
        for (int it = 0; it < n_iter && !r; ++it) {
            cudaEvent_t *ev = it < prof ? c->events + (size_t)it * kEvents : nullptr;
            if ((r = run_gradient(c, theta, ev))) break;
            launch_update(c, exaggeration, lr, momentum, nullptr, 1);
            if (cudaGetLastError() != cudaSuccess) r = fail(c, HTS_ECUDA, "update launch failed");
            if (!r && ev && cudaEventRecord(ev[6], c->stream) != cudaSuccess) r = fail(c, HTS_ECUDA, "event");
        }
        c->stream = user;
        if (r) {  // a failed iteration may have left the attraction unjoined
            CK(cudaEventRecord(c->aev_join, c->astream));
            CK(cudaStreamWaitEvent(c->pstream, c->aev_join, 0));
        }
        CK(cudaEventRecord(c->pev_out, c->pstream));
        CK(cudaStreamWaitEvent(c->stream, c->pev_out, 0));
        if (r) return r;
    }
    c->iters += n_iter;
    int st = 0;
    if ((r = read_status(c, &st))) return r;
    for (int it = 0; it < prof; ++it) {
        cudaEvent_t *ev = c->events + (size_t)it * kEvents;
        // keys, sort, tree, walk: consecutive main-stream marks; attract: its
        // own interval on the side stream (overlapping); Z + update: from the
        // join to the end of the update
        const int from[kPhases] = {0, 1, 2, 3, 7, 5}, to[kPhases] = {1, 2, 3, 4, 8, 6};
        for (int k = 0; k < kPhases; ++k) {
            if (k == 4 && c->nnz == 0) continue;
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[from[k]], ev[to[k]]));
            c->phase_ms[k] += ms;
        }
    }
    c->phase_iters += prof;
    return status_error(c, st);
}

int hts_get_Y(hts_ctx *c, double *y_out, int where)
{
    if (!c) return HTS_EINVAL;
    if (!c->have_Y) return fail(c, HTS_ENOTSET, "Y is not set");
    if (!y_out && c->n > 0) return fail(c, HTS_EINVAL, "hts_get_Y: NULL output");
    int r = set_device(c);
    if (r) return r;
    if (c->n == 0) return HTS_OK;
    if (where == HTS_DEVICE && (r = check_device_ptr(c, y_out))) return r;
    CK(cudaMemcpyAsync(y_out, c->y, sizeof(double2) * (size_t)c->n,
                       where == HTS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
    if (where == HTS_HOST) CK(cudaStreamSynchronize(c->stream));
    return HTS_OK;
}

int hts_grad(hts_ctx *c, double theta, double exaggeration, double *g_out, double *Z_out, int where)
{
    int r = ready(c);
    if (r) return r;
    if (!(exaggeration > 0.0) || !isfinite(exaggeration)) return fail(c, HTS_EINVAL, "hts_grad: bad exaggeration");
    if ((r = check_theta(c, theta))) return r;
    if (where != HTS_HOST && where != HTS_DEVICE) return fail(c, HTS_EINVAL, "hts_grad: bad where");
    if (c->n == 0) {
        if (Z_out) *Z_out = 0.0;
        return HTS_OK;
    }
    if (g_out && where == HTS_DEVICE && (r = check_device_ptr(c, g_out))) return r;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    if ((r = run_gradient(c, theta))) return r;
    // a host output is staged in the tree-build scratch `terms` (3n doubles)
    double2 *dst = nullptr;
    if (g_out) dst = where == HTS_DEVICE ? (double2 *)g_out : (double2 *)c->terms;
    launch_update(c, exaggeration, 0.0, 0.0, dst, 0);
    LAUNCHED("combine");
    if (g_out && where == HTS_HOST)
        CK(cudaMemcpyAsync(g_out, c->terms, sizeof(double2) * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->h_pinned + 1, c->dscal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    int st = 0;
    if ((r = read_status(c, &st))) return r;
    if (Z_out) *Z_out = c->h_pinned[1];
    return status_error(c, st);
}

int hts_kl(hts_ctx *c, double theta, double *kl_out)
{
    int r = ready(c);
    if (r) return r;
    if (!kl_out) return fail(c, HTS_EINVAL, "hts_kl: NULL output");
    if ((r = check_theta(c, theta))) return r;
    if (c->n == 0) {
        *kl_out = 0.0;
        return HTS_OK;
    }
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    int64_t keep = c->nnz;
    c->nnz = 0;  // Z only: skip the attractive sum
    r = run_gradient(c, theta);
    c->nnz = keep;
    if (r) return r;
    std::vector<double> kl;
    if ((r = kl_parts(c, kl))) return r;
    double t = 0.0;
    for (double v : kl) t += v;
    *kl_out = t;
    return HTS_OK;
}

int hts_get_keys(hts_ctx *c, uint64_t *keys_out, double *bounds_out, int where)
{
    if (!c) return HTS_EINVAL;
    if (!c->have_Y) return fail(c, HTS_ENOTSET, "Y is not set");
    int r = set_device(c);
    if (r) return r;
    if (c->n == 0) return HTS_OK;
    if (!keys_out) return fail(c, HTS_EINVAL, "hts_get_keys: NULL output");
    if (where == HTS_DEVICE && (r = check_device_ptr(c, keys_out))) return r;
    launch_prep_points(c);
    LAUNCHED("prep_points");
    launch_make_keys(c);
    LAUNCHED("make_keys");
    CK(cudaMemcpyAsync(keys_out, c->keys, sizeof(uint64_t) * (size_t)c->n,
                       where == HTS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
    unsigned long long mm[2];
    CK(cudaMemcpyAsync(mm, c->minmax, sizeof(mm), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (bounds_out) {
        memcpy(&bounds_out[0], &mm[0], 8);
        memcpy(&bounds_out[1], &mm[1], 8);
    }
    return HTS_OK;
}

int hts_get_tree(hts_ctx *c, int64_t cap, int64_t *count_out, int32_t *depth, uint64_t *prefix, int64_t *count,
                 int64_t *first, double *ycell, double *rcell)
{
    if (!c) return HTS_EINVAL;
    if (!c->have_Y) return fail(c, HTS_ENOTSET, "Y is not set");
    int r = set_device(c);
    if (r) return r;
    const int64_t n = c->n;
    if (n == 0) {
        if (count_out) *count_out = 0;
        return HTS_OK;
    }
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    const size_t M = 2 * (size_t)n;
    // export arrays, freed on every return path
    struct Owned {
        TreeExport ex{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        ~Owned()
        {
            cudaFree(ex.depth); cudaFree(ex.prefix); cudaFree(ex.count); cudaFree(ex.first);
            cudaFree(ex.ycell); cudaFree(ex.rcell);
        }
    } own;
    TreeExport &ex = own.ex;
    bool want = cap > 0;
    if (want) {
        CK(cudaMalloc((void **)&ex.depth, M * sizeof(int32_t)));
        CK(cudaMalloc((void **)&ex.prefix, M * sizeof(uint64_t)));
        CK(cudaMalloc((void **)&ex.count, M * sizeof(int64_t)));
        CK(cudaMalloc((void **)&ex.first, M * sizeof(int64_t)));
        CK(cudaMalloc((void **)&ex.ycell, 2 * M * sizeof(double)));
        CK(cudaMalloc((void **)&ex.rcell, M * sizeof(double)));
    }
    launch_prep_points(c);
    launch_make_keys(c);
    launch_sort_pairs(c);
    launch_build_tree(c, 0.5, want ? &ex : nullptr);
    LAUNCHED("tree export");
    int m = 0;
    CK(cudaMemcpyAsync(&m, c->n_nodes, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (m < 0 || m > (int64_t)M) return fail(c, HTS_ENUMERIC, "hts_get_tree: node count out of range");
    if (count_out) *count_out = m;
    int st = 0;
    if ((r = read_status(c, &st))) return r;
    if (want) {
        int rc = HTS_OK;
        if (cap < m) {
            rc = fail(c, HTS_EINVAL, "hts_get_tree: cap smaller than the node count");
        } else {
            if (depth) CK(cudaMemcpy(depth, ex.depth, m * sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (prefix) CK(cudaMemcpy(prefix, ex.prefix, m * sizeof(uint64_t), cudaMemcpyDeviceToHost));
            if (count) CK(cudaMemcpy(count, ex.count, m * sizeof(int64_t), cudaMemcpyDeviceToHost));
            if (first) CK(cudaMemcpy(first, ex.first, m * sizeof(int64_t), cudaMemcpyDeviceToHost));
            if (ycell) CK(cudaMemcpy(ycell, ex.ycell, 2 * m * sizeof(double), cudaMemcpyDeviceToHost));
            if (rcell) CK(cudaMemcpy(rcell, ex.rcell, m * sizeof(double), cudaMemcpyDeviceToHost));
        }
        if (rc) return rc;
    }
    return status_error(c, st);
}

int hts_set_counters(hts_ctx *c, int enable)
{
    if (!c) return HTS_EINVAL;
    int r = set_device(c);
    if (r) return r;
    if (enable && !c->counters_on) CK(cudaMemsetAsync(c->counters, 0, 5 * sizeof(unsigned long long), c->stream));
    c->counters_on = enable ? 1 : 0;
    c->layout_version += 1;
    return HTS_OK;
}

int hts_get_counters(hts_ctx *c, int64_t *out5)
{
    if (!c || !out5) return HTS_EINVAL;
    int r = set_device(c);
    if (r) return r;
    unsigned long long v[4];
    CK(cudaMemcpyAsync(v, c->counters, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 4; ++k) out5[k] = (int64_t)v[k];
    out5[4] = c->launches;
    return HTS_OK;
}

int hts_set_wait_test(hts_ctx *c, int spin_limit)
{
    if (!c) return HTS_EINVAL;
    if (spin_limit < 0 || spin_limit > 4096) return fail(c, HTS_EINVAL, "hts_set_wait_test: spin_limit in [0, 4096]");
    c->wait_test = spin_limit;
    c->layout_version += 1;  // captured graphs hold the sort's arguments
    return HTS_OK;
}

int hts_get_criterion_count(hts_ctx *c, int64_t *out)
{
    if (!c || !out) return HTS_EINVAL;
    int r = set_device(c);
    if (r) return r;
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, c->counters + 4, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out = (int64_t)v;
    return HTS_OK;
}

int hts_set_profiling(hts_ctx *c, int enable)
{
    if (!c) return HTS_EINVAL;
    if (enable < 0 || enable > 2) return fail(c, HTS_EINVAL, "hts_set_profiling: enable is 0, 1 or 2");
    c->profiling = enable;
    return HTS_OK;
}

int hts_get_profile(hts_ctx *c, double *ms6, int64_t *iters)
{
    if (!c || !ms6) return HTS_EINVAL;
    for (int k = 0; k < kPhases; ++k) {
        ms6[k] = c->phase_ms[k];
        c->phase_ms[k] = 0.0;
    }
    if (iters) *iters = c->phase_iters;
    c->phase_iters = 0;
    return HTS_OK;
}

int hts_get_state(hts_ctx *c, double *vel, double *gains, int64_t *iters, int where)
{
    if (!c) return HTS_EINVAL;
    if (!c->have_Y) return fail(c, HTS_ENOTSET, "Y is not set");
    if (where != HTS_HOST && where != HTS_DEVICE) return fail(c, HTS_EINVAL, "hts_get_state: bad where");
    int r = set_device(c);
    if (r) return r;
    if (where == HTS_DEVICE && c->n &&
        ((vel && (r = check_device_ptr(c, vel))) || (gains && (r = check_device_ptr(c, gains)))))
        return r;
    cudaMemcpyKind k = where == HTS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (vel && c->n) CK(cudaMemcpyAsync(vel, c->vel, sizeof(double2) * (size_t)c->n, k, c->stream));
    if (gains && c->n) CK(cudaMemcpyAsync(gains, c->gains, sizeof(double2) * (size_t)c->n, k, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (iters) *iters = c->iters;
    return HTS_OK;
}

int hts_set_state(hts_ctx *c, const double *vel, const double *gains, int64_t iters, int where)
{
    if (!c) return HTS_EINVAL;
    if (!c->have_Y) return fail(c, HTS_ENOTSET, "Y is not set");
    if (where != HTS_HOST && where != HTS_DEVICE) return fail(c, HTS_EINVAL, "hts_set_state: bad where");
    if (iters < 0) return fail(c, HTS_EINVAL, "hts_set_state: negative iteration count");
    int r = set_device(c);
    if (r) return r;
    if (where == HTS_DEVICE && c->n &&
        ((vel && (r = check_device_ptr(c, vel))) || (gains && (r = check_device_ptr(c, gains)))))
        return r;
    cudaMemcpyKind k = where == HTS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (vel && c->n) CK(cudaMemcpyAsync(c->vel, vel, sizeof(double2) * (size_t)c->n, k, c->stream));
    if (gains && c->n) CK(cudaMemcpyAsync(c->gains, gains, sizeof(double2) * (size_t)c->n, k, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->iters = iters;
    return HTS_OK;
}

int hts_set_cosne(hts_ctx *c, double lambda1, double lambda2, const double *x_sqnorm, int where)
{
    if (!c) return HTS_EINVAL;
    c->err.clear();
    if (!x_sqnorm) {
        dfree(&c->xsq);
        c->cosne_l1 = 1.0;
        c->cosne_l2 = 0.0;
        c->layout_version += 1;
        return HTS_OK;
    }
    if (!c->have_Y) return fail(c, HTS_ENOTSET, "hts_set_cosne: set Y first (the term is per point)");
    if (!isfinite(lambda1) || !isfinite(lambda2) || (where != HTS_HOST && where != HTS_DEVICE))
        return fail(c, HTS_EINVAL, "hts_set_cosne: invalid argument");
    int r = set_device(c);
    if (r) return r;
    if (where == HTS_HOST) {
        for (int64_t i = 0; i < c->n; ++i)
            if (!(x_sqnorm[i] >= 0.0) || !isfinite(x_sqnorm[i]))
                return fail(c, HTS_EDOMAIN, "hts_set_cosne: |x_i|^2 must be finite and >= 0");
    } else if ((r = check_device_ptr(c, x_sqnorm))) {
        return r;
    }
    if ((r = dalloc(c, &c->xsq, (size_t)std::max<int64_t>(c->n, 1)))) return r;
    if (c->n > 0)
        CK(cudaMemcpyAsync(c->xsq, x_sqnorm, sizeof(double) * (size_t)c->n,
                           where == HTS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->cosne_l1 = lambda1;
    c->cosne_l2 = lambda2;
    c->layout_version += 1;
    return HTS_OK;
}

int hts_set_segments(hts_ctx *c, int nseg, const int64_t *offsets, const double *lr_scale)
{
    if (!c) return HTS_EINVAL;
    c->err.clear();
    int r = set_device(c);
    if (r) return r;
    CK(cudaStreamSynchronize(c->stream));
    free_segments(c);  // every error below leaves one segment
    c->layout_version += 1;
    if (!c->have_P || !c->have_Y) return fail(c, HTS_ENOTSET, "hts_set_segments: set P and Y first");
    if (nseg < 1 || nseg > HTS_MAX_SEGMENTS || !offsets) return fail(c, HTS_EINVAL, "hts_set_segments: bad nseg");
    if (offsets[0] != 0 || offsets[nseg] != c->n)
        return fail(c, HTS_ESHAPE, "hts_set_segments: offsets must start at 0 and end at n");
    for (int s = 0; s < nseg; ++s)
        if (offsets[s + 1] <= offsets[s]) return fail(c, HTS_ESHAPE, "hts_set_segments: empty or decreasing range");
    if (lr_scale)
        for (int s = 0; s < nseg; ++s)
            if (!(lr_scale[s] >= 0.0) || !isfinite(lr_scale[s]))
                return fail(c, HTS_EINVAL, "hts_set_segments: lr_scale must be finite and >= 0");
    if (nseg == 1) return HTS_OK;
    if ((r = dalloc(c, &c->seg_off, HTS_MAX_SEGMENTS + 1)) || (r = dalloc(c, &c->seg_of, (size_t)c->n)) ||
        (r = dalloc(c, &c->seg_lr, HTS_MAX_SEGMENTS)) || (r = dalloc(c, &c->seg_z, HTS_MAX_SEGMENTS))) {
        free_segments(c);
        return r;
    }
    std::vector<double> lr((size_t)nseg, 1.0);
    if (lr_scale) lr.assign(lr_scale, lr_scale + nseg);
    cudaError_t e = cudaMemcpy(c->seg_off, offsets, sizeof(int64_t) * (size_t)(nseg + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->seg_lr, lr.data(), sizeof(double) * (size_t)nseg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) {
        free_segments(c);
        return cuda_fail(c, e, "hts_set_segments: copy");
    }
    c->nseg = nseg;
    launch_segments_setup(c);
    int st = 0;
    e = cudaGetLastError();
    if (e != cudaSuccess || (r = read_status(c, &st)) || st) {
        free_segments(c);
        if (e != cudaSuccess) return cuda_fail(c, e, "segments_setup");
        return r ? r : fail(c, HTS_ESHAPE, "hts_set_segments: P is not block diagonal over the segments");
    }
    for (int s = 0; s <= nseg; ++s) c->seg_off_h[s] = offsets[s];
    return HTS_OK;
}

int hts_get_segment_Z(hts_ctx *c, double *Z_out)
{
    if (!c || !Z_out) return HTS_EINVAL;
    int r = set_device(c);
    if (r) return r;
    CK(cudaMemcpyAsync(c->h_pinned, c->nseg > 1 ? c->seg_z : c->dscal, sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    if (c->nseg > 1)
        CK(cudaMemcpyAsync(Z_out, c->seg_z, sizeof(double) * (size_t)c->nseg, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->nseg == 1) Z_out[0] = c->h_pinned[0];
    return HTS_OK;
}

int hts_kl_segments(hts_ctx *c, double theta, double *kl_out)
{
    int r = ready(c);
    if (r) return r;
    if (!kl_out) return fail(c, HTS_EINVAL, "hts_kl_segments: NULL output");
    if ((r = check_theta(c, theta))) return r;
    if (c->n == 0) {
        kl_out[0] = 0.0;
        return HTS_OK;
    }
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    int64_t keep = c->nnz;
    c->nnz = 0;
    r = run_gradient(c, theta);
    c->nnz = keep;
    if (r) return r;
    std::vector<double> kl;
    if ((r = kl_parts(c, kl))) return r;
    for (int s = 0; s < c->nseg; ++s) kl_out[s] = kl[s];
    return HTS_OK;
}

int hts_set_graphs(hts_ctx *c, int enable)
{
    if (!c) return HTS_EINVAL;
    int r = set_device(c);
    if (r) return r;
    c->use_graphs = enable ? 1 : 0;
    if (!enable) {
        if (c->gstream) CK(cudaStreamSynchronize(c->gstream));
        drop_graph(c);
    }
    return HTS_OK;
}

int hts_autotune(hts_ctx *c, double theta, int reps, int *tuning)
{
    int r = ready(c);
    if (r) return r;
    if ((r = check_theta(c, theta))) return r;
    if (reps < 1 || reps > 1000) return fail(c, HTS_EINVAL, "hts_autotune: reps must be in [1, 1000]");
    if (c->n > 0) {
        CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        if ((r = ensure_events(c, 1))) return r;
        cudaEvent_t a = c->events[0], b = c->events[1];
        launch_prep_points(c);
        LAUNCHED("prep_points");
        auto time_it = [&](auto launch, float *ms) -> int {
            launch();  // warm
            CK(cudaEventRecord(a, c->stream));
            for (int k = 0; k < reps; ++k) launch();
            CK(cudaEventRecord(b, c->stream));
            CK(cudaEventSynchronize(b));
            LAUNCHED("autotune");
            CK(cudaEventElapsedTime(ms, a, b));
            return HTS_OK;
        };
        if (theta > 0.0) {
            launch_make_keys(c);
            launch_sort_pairs(c);
            launch_build_tree(c, theta, nullptr);
            LAUNCHED("build_tree");
            // largest first; a smaller block must win by 3%: its edge at the
            // tuning state (balance of the cost-ordered launches) tends to turn
            // into a loss as the embedding spreads, where larger blocks share
            // node data in L1 across more warps (N = 1M over the protocol: 128
            // and 256 threads 3-8% ahead of 64, though 64 can win at Y0)
            const int cand[4] = {256, 128, 64, 32};
            float best = INFINITY;
            int pick = c->walk_block;
            for (int wb : cand) {
                c->walk_block = wb;
                float ms = 0.f;
                if ((r = time_it([&] { launch_walk(c); }, &ms))) return r;
                if (ms < 0.97f * best) {
                    best = ms;
                    pick = wb;
                }
            }
            c->walk_block = pick;
            // warps per chunk: the cut depth of the split walk (small problems)
            const int dmax = walk_split_depth(c->n, kMaxSplitCut, c->cfg.precision == HTS_FP64);
            if (c->nseg == 1 && dmax > 0) {
                float bestd = INFINITY;
                int pickd = 0;
                for (int d = 0; d <= dmax; ++d) {
                    c->walk_split = d;
                    float ms = 0.f;
                    if ((r = time_it([&] { launch_walk(c); }, &ms))) return r;
                    if (ms < bestd) {
                        bestd = ms;
                        pickd = d;
                    }
                }
                c->walk_split = pickd;
            }
        }
        if (c->nnz > 0 && c->cfg.precision == HTS_FP32_MIXED) {
            const int cand[4] = {4, 8, 16, 32};
            float best = INFINITY;
            int pick = c->attract_group;
            for (int g : cand) {
                c->attract_group = g;
                float ms = 0.f;
                if ((r = time_it([&] { launch_attract(c); }, &ms))) return r;
                if (ms < best) {
                    best = ms;
                    pick = g;
                }
            }
            c->attract_group = pick;
        }
        int st = 0;
        if ((r = read_status(c, &st))) return r;
        if ((r = status_error(c, st))) return r;
        c->layout_version += 1;
    }
    if (tuning) {
        tuning[0] = c->walk_block;
        tuning[1] = c->attract_group;
    }
    return HTS_OK;
}

int hts_set_tuning(hts_ctx *c, int walk_block, int attract_lanes)
{
    if (!c) return HTS_EINVAL;
    c->err.clear();
    auto in = [](int v, int a, int b, int d, int e) { return v == a || v == b || v == d || v == e; };
    if ((walk_block && !in(walk_block, 32, 64, 128, 256)) || (attract_lanes && !in(attract_lanes, 4, 8, 16, 32)))
        return fail(c, HTS_EINVAL, "hts_set_tuning: walk_block in {32,64,128,256}, attract_lanes in {4,8,16,32}");
    if (walk_block) c->walk_block = walk_block;
    if (attract_lanes) c->attract_group = attract_lanes;
    c->layout_version += 1;
    return HTS_OK;
}

int hts_set_walk_split(hts_ctx *c, int depth)
{
    if (!c) return HTS_EINVAL;
    c->err.clear();
    if (depth < -1 || depth > 3) return fail(c, HTS_EINVAL, "hts_set_walk_split: depth in -1 .. 3");
    c->walk_split = depth;
    c->layout_version += 1;
    return HTS_OK;
}

int hts_get_walk_split(const hts_ctx *c, int *depth)
{
    if (!c || !depth) return HTS_EINVAL;
    *depth = c->nseg > 1 ? 0 : walk_split_depth(c->n, c->walk_split, c->cfg.precision == HTS_FP64);
    return HTS_OK;
}

int hts_get_tuning(const hts_ctx *c, int *tuning)
{
    if (!c || !tuning) return HTS_EINVAL;
    tuning[0] = c->walk_block;
    tuning[1] = c->attract_group;
    return HTS_OK;
}

int hts_get_sizes(const hts_ctx *c, int64_t *n, int64_t *nnz)
{
    if (!c) return HTS_EINVAL;
    if (n) *n = c->n;
    if (nnz) *nnz = c->nnz;
    return HTS_OK;
}

}  // extern "C"
