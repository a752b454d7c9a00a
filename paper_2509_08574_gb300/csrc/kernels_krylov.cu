// Krylov (CGLS) vector work for sm_103a: the fused vector updates, the
// FP64 reductions and the scalar recurrences of one CGLS step on the
// augmented IRN-PICCS system (Sec. 2.3; CGLS is the inner solver the paper
// uses, mathematically equivalent to LSQR).
//
// The scalars (gamma, delta, step, beta) live in device memory and are read
// by the vector kernels directly, so one reconstruction enqueues its whole
// iteration sequence without a host round trip.  Reductions are two-level and
// deterministic: each kernel writes one FP64 partial per CTA, and a one-CTA
// finalize kernel adds the partials in a fixed order.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace piccs {

namespace {

constexpr int kThreads = 256;
constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kThreads)
p_update_kernel(long long M, const float *__restrict__ s, float *__restrict__ p,
                const KrylovScalars *__restrict__ k)
{
    const float beta = (float)k->beta;
    const long long n4 = M >> 2;
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
    float4 *p4 = reinterpret_cast<float4 *>(p);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (beta == 0.f) {  // restart: p = s (p may hold garbage)
        for (long long i = t0; i < n4; i += stride) p4[i] = s4[i];
        for (long long i = (n4 << 2) + t0; i < M; i += stride) p[i] = s[i];
        return;
    }
    for (long long i = t0; i < n4; i += stride) {
        const float4 a = s4[i];
        float4 b = p4[i];
        b.x = fmaf(beta, b.x, a.x);
        b.y = fmaf(beta, b.y, a.y);
        b.z = fmaf(beta, b.z, a.z);
        b.w = fmaf(beta, b.w, a.w);
        p4[i] = b;
    }
    for (long long i = (n4 << 2) + t0; i < M; i += stride) p[i] = fmaf(beta, p[i], s[i]);
}

// x += a p; g -= a t; s = g (the adjoint then adds A^T r to s); r -= a q
__global__ void __launch_bounds__(kThreads)
x_update_kernel(long long M, long long N, float *__restrict__ x, const float *__restrict__ p,
                float *__restrict__ g, const float *__restrict__ t, float *__restrict__ s,
                float *__restrict__ r, const float *__restrict__ q,
                const KrylovScalars *__restrict__ k)
{
    const float a = (float)k->a;
    const long long m4 = M >> 2, n4 = N >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float4 *x4 = reinterpret_cast<float4 *>(x);
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
    float4 *g4 = reinterpret_cast<float4 *>(g);
    const float4 *t4 = reinterpret_cast<const float4 *>(t);
    float4 *s4 = reinterpret_cast<float4 *>(s);
    for (long long i = t0; i < m4; i += stride) {
        const float4 pp = p4[i], tt = t4[i];
        float4 xx = x4[i], gg = g4[i];
        xx.x = fmaf(a, pp.x, xx.x); xx.y = fmaf(a, pp.y, xx.y);
        xx.z = fmaf(a, pp.z, xx.z); xx.w = fmaf(a, pp.w, xx.w);
        gg.x = fmaf(-a, tt.x, gg.x); gg.y = fmaf(-a, tt.y, gg.y);
        gg.z = fmaf(-a, tt.z, gg.z); gg.w = fmaf(-a, tt.w, gg.w);
        x4[i] = xx;
        g4[i] = gg;
        s4[i] = gg;
    }
    for (long long i = (m4 << 2) + t0; i < M; i += stride) {
        x[i] = fmaf(a, p[i], x[i]);
        const float gg = fmaf(-a, t[i], g[i]);
        g[i] = gg;
        s[i] = gg;
    }
    float4 *r4 = reinterpret_cast<float4 *>(r);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    for (long long i = t0; i < n4; i += stride) {
        const float4 qq = q4[i];
        float4 rr = r4[i];
        rr.x = fmaf(-a, qq.x, rr.x); rr.y = fmaf(-a, qq.y, rr.y);
        rr.z = fmaf(-a, qq.z, rr.z); rr.w = fmaf(-a, qq.w, rr.w);
        r4[i] = rr;
    }
    for (long long i = (n4 << 2) + t0; i < N; i += stride) r[i] = fmaf(-a, q[i], r[i]);
}

__device__ __forceinline__ void block_sum_store(double v, double *partials)
{
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// ||v||^2: each float4 is squared and summed in FP32, then accumulated in FP64
__global__ void __launch_bounds__(kThreads)
norm2_kernel(long long n, const float *__restrict__ v, double *__restrict__ partials)
{
    const long long n4 = n >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
    double acc = 0.0;
    for (long long i = t0; i < n4; i += stride) {
        const float4 a = v4[i];
        acc += (double)fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w)));
    }
    for (long long i = (n4 << 2) + t0; i < n; i += stride) acc += (double)v[i] * (double)v[i];
    block_sum_store(acc, partials);
}

// Fixed-order sum of partials by one CTA (deterministic).
__device__ double cta_sum(const double *p, int n)
{
    __shared__ double red[kFinThreads / 32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kFinThreads)
finalize_delta_kernel(KrylovScalars *k, const double *pa, int na, const double *pb, int nb)
{
    const double da = cta_sum(pa, na);
    const double db = (pb && nb > 0) ? cta_sum(pb, nb) : 0.0;
    if (threadIdx.x != 0) return;
    const double delta = da + db;
    k->delta = delta;
    double a = 0.0;
    if (k->status == 0 && !k->stopped) {
        if (!(delta > 0.0) || !isfinite(delta)) {
            k->status = -4;  // PICCS_EBREAKDOWN
        } else {
            a = k->gamma / delta;
            if (!isfinite(a)) { k->status = -4; a = 0.0; }
        }
    }
    k->a = a;
    if (a != 0.0) k->iters_run += 1;
}

__global__ void __launch_bounds__(kFinThreads)
finalize_gamma_kernel(KrylovScalars *k, const double *p, int n, int restart)
{
    const double gnew = cta_sum(p, n);
    if (threadIdx.x != 0) return;
    if (!isfinite(gnew)) {
        if (k->status == 0) k->status = -4;
        k->a = 0.0;
        k->beta = 0.0;
    } else if (restart) {
        k->gamma = gnew;
        k->gamma0 = gnew;
        k->beta = 0.0;
        k->stopped = !(gnew > 0.0);
    } else if (k->a != 0.0) {
        const double gold = k->gamma;
        k->beta = gold > 0.0 ? gnew / gold : 0.0;
        k->gamma = gnew;
        // same stopping rule as a textbook CGLS: ||s|| below 1e-13 of its start
        if (!(gnew > 1e-26 * k->gamma0)) k->stopped = 1;
    }
    if (k->n_hist < 512) k->hist[k->n_hist++] = gnew;
}

__global__ void reset_scalars_kernel(KrylovScalars *k)
{
    k->gamma = k->gamma0 = k->delta = k->a = k->beta = 0.0;
    k->status = 0;
    k->iters_run = 0;
    k->n_hist = 0;
    k->stopped = 0;
    k->nonfinite = 0;
}

__global__ void __launch_bounds__(kThreads)
count_nonfinite_kernel(long long n, const float *__restrict__ v, int *__restrict__ flag)
{
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(v[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void __launch_bounds__(kFinThreads)
sum_partials_kernel(const double *p, int n, double *out)
{
    const double t = cta_sum(p, n);
    if (threadIdx.x == 0) *out = t;
}

}  // namespace

int vector_blocks() { return 152 * 8; }

cudaError_t launch_p_update(long long M, const float *s, float *p, const KrylovScalars *k,
                            cudaStream_t st)
{
    p_update_kernel<<<vector_blocks(), kThreads, 0, st>>>(M, s, p, k);
    return cudaGetLastError();
}

cudaError_t launch_x_update(long long M, long long N, float *x, const float *p, float *g,
                            const float *t, float *s, float *r, const float *q,
                            const KrylovScalars *k, cudaStream_t st)
{
    x_update_kernel<<<vector_blocks(), kThreads, 0, st>>>(M, N, x, p, g, t, s, r, q, k);
    return cudaGetLastError();
}

cudaError_t launch_norm2(long long n, const float *v, double *partials, cudaStream_t st)
{
    norm2_kernel<<<vector_blocks(), kThreads, 0, st>>>(n, v, partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize_delta(KrylovScalars *k, const double *pa, int na, const double *pb,
                                  int nb, cudaStream_t st)
{
    finalize_delta_kernel<<<1, kFinThreads, 0, st>>>(k, pa, na, pb, nb);
    return cudaGetLastError();
}

cudaError_t launch_finalize_gamma(KrylovScalars *k, const double *p, int n, int restart,
                                  cudaStream_t st)
{
    finalize_gamma_kernel<<<1, kFinThreads, 0, st>>>(k, p, n, restart);
    return cudaGetLastError();
}

cudaError_t launch_reset_scalars(KrylovScalars *k, cudaStream_t st)
{
    reset_scalars_kernel<<<1, 1, 0, st>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(long long n, const float *v, int *flag, cudaStream_t st)
{
    count_nonfinite_kernel<<<vector_blocks(), kThreads, 0, st>>>(n, v, flag);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double *p, int n, double *out, cudaStream_t st)
{
    sum_partials_kernel<<<1, kFinThreads, 0, st>>>(p, n, out);
    return cudaGetLastError();
}

}  // namespace piccs
