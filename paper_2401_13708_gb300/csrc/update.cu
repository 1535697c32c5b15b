// update.cu -- Z, the gradient and the Riemannian step, all in float64.
//
// reduce_z   Z = sum_i Z_i in a fixed order (256 fixed block partials, then
//            one block), so the value is reproducible.
// update     g_i = 4 (exag F_attr,i - F_rep,i / Z)  (Eq. KlGradientHyperbolicSplit
//            with the exaggeration of Sec. 5.1), then
//              r_i = lambda_i^-metric_pow g_i  ("product of lambda^-1 with the
//                    variation", Sec. 4.2; lambda = 2 / (1 - |y|^2), Eq. PoincareMetric)
//              optional gains (+0.2 on sign disagreement of g and v, *0.8
//                    otherwise, floor 0.01),
//              v_i <- momentum v_i - lr gains r_i,
//              y_i <- proj(exp_{y_i}(v_i)),  exp_y(v) = y (+) tanh(lambda |v| / 2) v / |v|
//                    with Moebius addition (+) (Sec. 4.2), proj of Eq.
//                    HyperbolicProjection: radius 1 - eps once |y| >= 1 - eps/2.
//            With the CO-SNE term on (Sec. 4.3), g_i becomes
//              lambda1 g_i - (4 lambda2 / n)(|x_i|^2 - |y_i|^2) y_i,
//            the derivative of lambda1 KL + (lambda2 / n) sum (|x|^2 - |y|^2)^2.
//            A non-finite result sets bit 1 of the status word.
#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kBlock = 256;
// status bits that void an iteration's gradient: tree node out of range (2),
// sort position out of range (4), a bounded look-back wait ran out (128)
constexpr int kStepBlockingStatus = 2 | 4 | 128;

// Fixed-shape two-pass sum: kRedBlocks blocks reduce grid-strided slices,
// one block adds the partials in order -- reproducible for a given n.
constexpr int kRedBlocks = 256;

__global__ void __launch_bounds__(kBlock) partial_sum_kernel(int n, const double *__restrict__ v, double *partial)
{
    __shared__ double sh[kBlock];
    double a = 0;
    for (int k = blockIdx.x * kBlock + threadIdx.x; k < n; k += kRedBlocks * kBlock) a += v[k];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kRedBlocks) final_sum_kernel(const double *__restrict__ partial, double *out)
{
    __shared__ double sh[kRedBlocks];
    sh[threadIdx.x] = partial[threadIdx.x];
    __syncthreads();
    for (int s = kRedBlocks / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Per-segment sum of v over [off[s], off[s+1]), one block per segment.
__global__ void __launch_bounds__(1024) segment_sum_kernel(const double *__restrict__ v,
                                                          const int64_t *__restrict__ off, double *out)
{
    __shared__ double sh[1024];
    const int64_t lo = off[blockIdx.x], hi = off[blockIdx.x + 1];
    double a = 0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += 1024) a += v[k];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

struct UpdateArgs {
    int n;
    double2 *y, *vel, *gains;
    const double2 *fattr, *frep;
    const double *Z;
    double exag, lr, mom, eps;
    int metric_pow, use_gains, do_step;
    double2 *g_out;
    int *status;
    const double *xsq;  // CO-SNE |x_i|^2 (nullptr: off)
    double l1, l2;
    const unsigned char *seg_of;  // batched: segment of each point (nullptr: one problem)
    const double *seg_lr;         // batched: learning-rate factor per segment
    const int64_t *seg_off;       // batched: segment offsets (CO-SNE uses the segment's n)
};

// tanh for the exp map's argument lambda |v| / 2 >= 0, which is small for the
// steps of the optimiser: below 2^-5 the Taylor series
//   tanh x = x - x^3/3 + 2 x^5/15 - 17 x^7/315 + 62 x^9/2835 - ...
// to the x^9 term (truncation below 1e-17 relative there), else tanh.
__device__ __forceinline__ double tanh_step(double x)
{
    if (x < 0.03125) {
        const double t = x * x;
        double p = 62.0 / 2835.0;
        p = fma(p, t, -17.0 / 315.0);
        p = fma(p, t, 2.0 / 15.0);
        p = fma(p, t, -1.0 / 3.0);
        return fma(x * t, p, x);
    }
    return tanh(x);
}

__global__ void __launch_bounds__(kBlock) update_kernel(UpdateArgs A)
{
    __shared__ double s_invz;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (!A.seg_of) {  // one problem: 1 / Z once per block (float64 division is costly here)
        if (threadIdx.x == 0) {
            const double Z0 = A.Z[0];
            s_invz = Z0 > 0.0 ? 1.0 / Z0 : 0.0;
        }
        __syncthreads();
    }
    if (i >= A.n) return;
    const int sg = A.seg_of ? A.seg_of[i] : 0;
    double invZ;
    if (A.seg_of) {
        const double Z = A.Z[sg];
        invZ = Z > 0.0 ? 1.0 / Z : 0.0;
    } else {
        invZ = s_invz;
    }
    const double2 fa = A.fattr[i], fr = A.frep[i];
    double gx = 4.0 * (A.exag * fa.x - fr.x * invZ);
    double gy = 4.0 * (A.exag * fa.y - fr.y * invZ);
    double2 p = A.y[i];
    const double n2 = p.x * p.x + p.y * p.y;
    if (A.xsq) {  // CO-SNE: lambda1 g_KL - (4 lambda2 / n)(|x|^2 - |y|^2) y
        const double ns = A.seg_of ? (double)(A.seg_off[sg + 1] - A.seg_off[sg]) : (double)A.n;
        const double c = 4.0 * A.l2 / ns * (A.xsq[i] - n2);
        gx = A.l1 * gx - c * p.x;
        gy = A.l1 * gy - c * p.y;
    }
    if (A.g_out) A.g_out[i] = make_double2(gx, gy);
    if (!A.do_step) return;
    // an iteration whose sort or tree build failed (a bounded wait ran out,
    // a position or node out of range) leaves Y and the optimiser state as
    // they were, so the context stays usable after the error is reported
    if (*(volatile const int *)A.status & kStepBlockingStatus) return;
    double2 v = A.vel[i];
    const double a = 1.0 - n2;  // 2 / lambda (Eq. PoincareMetric)
    const double hl = 0.5 * a;  // 1 / lambda
    const double sc = A.metric_pow == 2 ? hl * hl : hl;
    double kx = 1.0, ky = 1.0;
    if (A.use_gains) {
        double2 gn = A.gains[i];
        gn.x = ((gx > 0.0) == (v.x > 0.0)) ? gn.x * 0.8 : gn.x + 0.2;
        gn.y = ((gy > 0.0) == (v.y > 0.0)) ? gn.y * 0.8 : gn.y + 0.2;
        gn.x = fmax(gn.x, 0.01);
        gn.y = fmax(gn.y, 0.01);
        A.gains[i] = gn;
        kx = gn.x;
        ky = gn.y;
    }
    const double lr = A.seg_of ? A.lr * A.seg_lr[sg] : A.lr;
    v.x = A.mom * v.x - lr * kx * (gx * sc);
    v.y = A.mom * v.y - lr * ky * (gy * sc);
    const double vv = v.x * v.x + v.y * v.y;
    double2 q = p;
    if (vv > 0.0) {
        // exp map: p (+) tanh(lambda |v| / 2) v / |v|, lambda |v| / 2 = |v| / a;
        // 1 / |v| from one reciprocal square root (no square root and division)
        const double rn = rsqrt(vv), nv = vv * rn;
        const double f = tanh_step(nv / a) * rn;
        const double ux = f * v.x, uy = f * v.y;
        const double pu = p.x * ux + p.y * uy;
        const double nu = ux * ux + uy * uy;
        const double ca = 1.0 + 2.0 * pu + nu;
        const double rden = 1.0 / (1.0 + 2.0 * pu + n2 * nu);
        q.x = (ca * p.x + a * ux) * rden;
        q.y = (ca * p.y + a * uy) * rden;
    }
    const double q2 = q.x * q.x + q.y * q.y;
    const double lim = 1.0 - A.eps / 2.0;
    if (q2 >= lim * lim) {  // |q| >= 1 - eps/2 (Eq. HyperbolicProjection): back to radius 1 - eps
        const double f = (1.0 - A.eps) / sqrt(q2);
        q.x *= f;
        q.y *= f;
    }
    if (!isfinite(q.x) || !isfinite(q.y) || !isfinite(v.x) || !isfinite(v.y)) atomicOr(A.status, 1);
    A.y[i] = q;
    A.vel[i] = v;
}

// status bit 64: a point outside the open disk or non-finite
__global__ void check_y_kernel(int n, const double2 *__restrict__ y, int *status)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    double2 p = y[i];
    double n2 = p.x * p.x + p.y * p.y;
    if (!isfinite(p.x) || !isfinite(p.y) || !(n2 < 1.0)) atomicOr(status, 64);
}

}  // namespace

void launch_reduce_z(hts_ctx *c)
{
    if (c->nseg > 1) {  // one block per segment, fixed order
        segment_sum_kernel<<<c->nseg, 1024, 0, c->stream>>>(c->zi, c->seg_off, c->seg_z);
        c->launches += 1;
        return;
    }
    double *partial = c->red_tmp;  // >= kRedBlocks doubles
    partial_sum_kernel<<<kRedBlocks, kBlock, 0, c->stream>>>((int)c->n, c->zi, partial);
    final_sum_kernel<<<1, kRedBlocks, 0, c->stream>>>(partial, c->dscal);
    c->launches += 2;
}

void launch_update(hts_ctx *c, double exag, double lr, double mom, double2 *g_out, int do_step)
{
    UpdateArgs A;
    A.n = (int)c->n;
    A.y = c->y;
    A.vel = c->vel;
    A.gains = c->gains;
    A.fattr = c->fattr;
    A.frep = c->frep;
    A.Z = c->nseg > 1 ? c->seg_z : c->dscal;
    A.seg_of = c->nseg > 1 ? c->seg_of : nullptr;
    A.seg_lr = c->seg_lr;
    A.seg_off = c->seg_off;
    A.exag = exag;
    A.lr = lr;
    A.mom = mom;
    A.eps = c->cfg.eps;
    A.metric_pow = c->cfg.metric_pow;
    A.use_gains = c->cfg.use_gains;
    A.do_step = do_step;
    A.g_out = g_out;
    A.status = c->status;
    A.xsq = c->xsq;
    A.l1 = c->cosne_l1;
    A.l2 = c->cosne_l2;
    update_kernel<<<(A.n + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>(A);
    c->launches += 1;
}

void launch_segment_sums(hts_ctx *c, const double *v, double *out)
{
    segment_sum_kernel<<<c->nseg, 1024, 0, c->stream>>>(v, c->seg_off, out);
    c->launches += 1;
}

void launch_check_y(hts_ctx *c)
{
    check_y_kernel<<<((int)c->n + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>((int)c->n, c->y, c->status);
}

}  // namespace hts
