// Krylov vector work for sm_103a: the fused vector updates, the FP64
// reductions and the scalar recurrences of one step of CGLS or of LSQR
// (Golub-Kahan bidiagonalisation with the Givens QR update, optionally
// re-orthogonalised) on the augmented IRN-PICCS system (Sec. 2.3 names both,
// as mathematically equivalent).
//
// The scalars (CGLS: gamma, delta, step, beta; LSQR: see LsqrScalars in
// internal.h) live in device memory and are read
// by the vector kernels directly, so one reconstruction enqueues its whole
// iteration sequence without a host round trip.  Reductions are two-level and
// deterministic: each kernel writes one FP64 partial per CTA, and a one-CTA
// finalize kernel adds the partials in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace piccs {

namespace {

constexpr int kThreads = 256;
constexpr int kFinThreads = 1024;

// Four consecutive basis values (FP32, or BF16 when stored at reduced
// precision), i counted in groups of four.
__device__ __forceinline__ float4 ld4(const float *p, long long i)
{
    return reinterpret_cast<const float4 *>(p)[i];
}
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p, long long i)
{
    const uint2 u = reinterpret_cast<const uint2 *>(p)[i];
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&u.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ void st4(float *p, long long i, float4 v)
{
    reinterpret_cast<float4 *>(p)[i] = v;
}
__device__ __forceinline__ void st4(__nv_bfloat16 *p, long long i, float4 v)
{
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned *>(&a);
    u.y = *reinterpret_cast<const unsigned *>(&b);
    reinterpret_cast<uint2 *>(p)[i] = u;
}
__device__ __forceinline__ float ld1(const float *p, long long i) { return p[i]; }
__device__ __forceinline__ float ld1(const __nv_bfloat16 *p, long long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void st1(float *p, long long i, float v) { p[i] = v; }
__device__ __forceinline__ void st1(__nv_bfloat16 *p, long long i, float v) { p[i] = __float2bfloat16_rn(v); }

__global__ void __launch_bounds__(kThreads)
p_update_kernel(long long M, const float *__restrict__ s, float *__restrict__ p,
                const KrylovScalars *__restrict__ k, long long sstride)
{
    const long long so = blockIdx.y * sstride;
    s = slot_ptr(s, so);
    p = slot_ptr(p, so);
    k = slot_ptr(k, so);
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
                const KrylovScalars *__restrict__ k, long long sstride)
{
    {
        const long long so = blockIdx.y * sstride;
        x = slot_ptr(x, so);
        p = slot_ptr(p, so);
        g = slot_ptr(g, so);
        t = slot_ptr(t, so);
        s = slot_ptr(s, so);
        r = slot_ptr(r, so);
        q = slot_ptr(q, so);
        k = slot_ptr(k, so);
    }
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
norm2_kernel(long long n, const float *__restrict__ v, double *__restrict__ partials,
             long long sstride)
{
    v = slot_ptr(v, blockIdx.y * sstride);
    partials = slot_ptr(partials, blockIdx.y * sstride);
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
finalize_delta_kernel(KrylovScalars *k, const double *pa, int na, const double *pb, int nb,
                      long long sstride)
{
    const long long so = blockIdx.x * sstride;  // one CTA per slot
    k = slot_ptr(k, so);
    pa = slot_ptr(pa, so);
    pb = slot_ptr(pb, so);
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
finalize_gamma_kernel(KrylovScalars *k, const double *p, int n, int restart, long long sstride)
{
    k = slot_ptr(k, blockIdx.x * sstride);
    p = slot_ptr(p, blockIdx.x * sstride);
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

__global__ void reset_scalars_kernel(KrylovScalars *k, long long sstride)
{
    k = slot_ptr(k, blockIdx.x * sstride);
    k->gamma = k->gamma0 = k->delta = k->a = k->beta = 0.0;
    k->status = 0;
    k->iters_run = 0;
    k->n_hist = 0;
    k->stopped = 0;
    k->nonfinite = 0;
}

__global__ void __launch_bounds__(kThreads)
count_nonfinite_kernel(long long n, const float *__restrict__ v, int *__restrict__ flag,
                       long long sstride)
{
    v = slot_ptr(v, blockIdx.y * sstride);
    flag = slot_ptr(flag, blockIdx.y * sstride);
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

// ---------------------------------------------------------------------------
// LSQR (Golub-Kahan bidiagonalisation with the Givens QR update, the Krylov
// method Sec. 2.3 names as equivalent to CGLS).  State and notation:
// LsqrScalars in internal.h.  Per step i the host enqueues: the forward in
// FWD_LSQR mode (uA <- A vhat / alpha_i - (alpha_i / beta_i) uA), the z-step
// stencil (kernels_reg.cu), finalize_beta (beta_{i+1}, rho_i, c_i, s_i, phi_i,
// phibar_{i+1}), the adjoint (s += A^T uA), lsqr_vx (w, x and the next vhat),
// optionally the re-orthogonalisation, and finalize_alpha (alpha_{i+1},
// theta_{i+1}, rhobar_{i+1}, the stop test).

__global__ void lsqr_reset_kernel(LsqrScalars *l, long long sstride)
{
    l = slot_ptr(l, blockIdx.x * sstride);
    l->alpha = l->beta = l->rhobar = l->phibar = l->c = l->s = l->rho = 0.0;
    l->sigma = l->sigma_next = l->bR2 = l->normar0 = 0.0;
    l->stopped = 0;
    l->nbasis = 0;
    for (int i = 0; i < 4; ++i) l->ureg[i] = 0.f;
    for (int i = 0; i < 8; ++i) l->fwd[i] = l->vx[i] = 0.f;
}

// rA -= pending * Aw (update; skipped when nothing is pending, so Aw may be
// unset), U = rA, |U|^2
__global__ void __launch_bounds__(kThreads)
lsqr_rinit_kernel(long long N, int update, float *__restrict__ ra, const float *__restrict__ aw,
                  float *__restrict__ u, const LsqrScalars *__restrict__ l,
                  double *__restrict__ partials, long long sstride)
{
    {
        const long long so = blockIdx.y * sstride;
        ra = slot_ptr(ra, so);
        aw = slot_ptr(aw, so);
        u = slot_ptr(u, so);
        l = slot_ptr(l, so);
        partials = slot_ptr(partials, so);
    }
    const float pend = update ? l->fwd[4] : 0.f;
    const long long n4 = N >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float4 *r4 = reinterpret_cast<float4 *>(ra);
    const float4 *a4 = reinterpret_cast<const float4 *>(aw);
    float4 *u4 = reinterpret_cast<float4 *>(u);
    double acc = 0.0;
    for (long long i = t0; i < n4; i += stride) {
        float4 r = r4[i];
        if (pend != 0.f) {
            const float4 a = a4[i];
            r.x = fmaf(-pend, a.x, r.x);
            r.y = fmaf(-pend, a.y, r.y);
            r.z = fmaf(-pend, a.z, r.z);
            r.w = fmaf(-pend, a.w, r.w);
            r4[i] = r;
        }
        u4[i] = r;
        acc += (double)fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, r.w * r.w)));
    }
    for (long long i = (n4 << 2) + t0; i < N; i += stride) {
        float r = ra[i];
        if (pend != 0.f) {
            r = fmaf(-pend, aw[i], r);
            ra[i] = r;
        }
        u[i] = r;
        acc += (double)r * (double)r;
    }
    block_sum_store(acc, partials);
}

template <bool FIRST, bool LAST, class BT>
__global__ void __launch_bounds__(kThreads)
lsqr_vx_kernel(long long M, float *__restrict__ x, float *__restrict__ w,
               float *__restrict__ vhat, const float *__restrict__ s, BT *__restrict__ basis,
               const LsqrScalars *__restrict__ l, double *__restrict__ partials, long long sstride,
               long long bstride)
{
    {
        const long long so = blockIdx.y * sstride;
        x = slot_ptr(x, so);
        w = slot_ptr(w, so);
        vhat = slot_ptr(vhat, so);
        s = slot_ptr(s, so);
        l = slot_ptr(l, so);
        partials = slot_ptr(partials, so);
        basis = slot_ptr(basis, blockIdx.y * bstride);
    }
    const float ia = l->vx[0], tw = l->vx[1], tx = l->vx[2], ib = l->vx[3], bb = l->vx[4];
    if (!FIRST && l->vx[5] != 0.f) return;
    const bool wrestart = l->vx[6] != 0.f;  // first step of a cycle: w = v
    const long long n4 = M >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double acc = 0.0;
    auto one = [&](float vh, float si, float &xo, float &wo, float &vo, float &bo) -> float {
        if (FIRST) {
            vo = ib * si;
            return vo * vo;
        }
        const float v = ia * vh;
        const float wn = wrestart ? v : fmaf(-tw, wo, v);
        xo = fmaf(tx, wn, xo);
        wo = wn;
        bo = v;
        if (LAST) return 0.f;
        vo = fmaf(ib, si, -bb * v);
        return vo * vo;
    };
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
    float4 *x4 = reinterpret_cast<float4 *>(x);
    float4 *w4 = reinterpret_cast<float4 *>(w);
    float4 *v4 = reinterpret_cast<float4 *>(vhat);
    for (long long i = t0; i < n4; i += stride) {
        const float4 si = LAST ? make_float4(0.f, 0.f, 0.f, 0.f) : s4[i];
        float4 vh = FIRST ? make_float4(0.f, 0.f, 0.f, 0.f) : v4[i];
        float4 xo = make_float4(0.f, 0.f, 0.f, 0.f), wo = xo, bo = xo, vo = vh;
        if (!FIRST) {
            xo = x4[i];
            if (!wrestart) wo = w4[i];
        }
        float q = one(vh.x, si.x, xo.x, wo.x, vo.x, bo.x);
        q += one(vh.y, si.y, xo.y, wo.y, vo.y, bo.y);
        q += one(vh.z, si.z, xo.z, wo.z, vo.z, bo.z);
        q += one(vh.w, si.w, xo.w, wo.w, vo.w, bo.w);
        acc += (double)q;
        if (!FIRST) {
            x4[i] = xo;
            w4[i] = wo;
            if (basis) st4(basis, i, bo);
        }
        if (!LAST) v4[i] = vo;
    }
    for (long long i = (n4 << 2) + t0; i < M; i += stride) {
        float xo = FIRST ? 0.f : x[i], wo = (FIRST || wrestart) ? 0.f : w[i];
        float vo = 0.f, bo = 0.f;
        acc += (double)one(FIRST ? 0.f : vhat[i], LAST ? 0.f : s[i], xo, wo, vo, bo);
        if (!FIRST) {
            x[i] = xo;
            w[i] = wo;
            if (basis) st1(basis, i, bo);
        }
        if (!LAST) vhat[i] = vo;
    }
    if (!LAST) block_sum_store(acc, partials);
}

__global__ void __launch_bounds__(kFinThreads)
lsqr_finalize_beta_kernel(KrylovScalars *k, LsqrScalars *l, int init, const double *pu, int nu,
                          const double *pr, int nr, long long sstride)
{
    {
        const long long so = blockIdx.x * sstride;  // one CTA per slot
        k = slot_ptr(k, so);
        l = slot_ptr(l, so);
        pu = slot_ptr(pu, so);
        pr = slot_ptr(pr, so);
    }
    const double u2 = cta_sum(pu, nu);
    const double zkz = cta_sum(pr, nr);
    const double zc = cta_sum(pr + nr, nr);
    const double bR2 = init ? cta_sum(pr + 2 * (long long)nr, nr) : l->bR2;
    if (threadIdx.x != 0) return;
    if (!init && l->stopped) return;
    const double sigma = init ? 1.0 : l->sigma_next;
    double beta2 = u2 + zkz + 2.0 * sigma * zc + sigma * sigma * bR2;
    if (!isfinite(beta2)) {
        if (k->status == 0) k->status = -4;  // PICCS_EBREAKDOWN
        l->stopped = 1;
        l->vx[2] = 0.f;
        l->vx[5] = 1.f;
        l->fwd[4] = 0.f;
        return;
    }
    const double beta = sqrt(fmax(beta2, 0.0));
    l->sigma = sigma;
    l->beta = beta;
    l->vx[3] = beta > 0.0 ? (float)(1.0 / beta) : 0.f;
    l->vx[4] = (float)beta;
    if (init) {
        l->bR2 = bR2;
        l->phibar = beta;
        l->vx[2] = 0.f;
        l->fwd[4] = 0.f;
        return;
    }
    // one Givens rotation eliminates beta_{i+1} below rhobar_i
    const double rho = hypot(l->rhobar, beta);
    const double c = l->rhobar / rho, s = beta / rho;
    const double phi = c * l->phibar;
    l->phibar = s * l->phibar;
    l->rho = rho;
    l->c = c;
    l->s = s;
    const double tx = phi / rho;
    l->vx[2] = isfinite(tx) ? (float)tx : 0.f;
    l->fwd[4] = l->vx[2];  // applied to x by lsqr_vx, to rA by the next forward
    if (!isfinite(tx) && k->status == 0) k->status = -4;
    if (l->vx[2] != 0.f) k->iters_run += 1;
}

__global__ void __launch_bounds__(kFinThreads)
lsqr_finalize_alpha_kernel(KrylovScalars *k, LsqrScalars *l, int init, const double *p, int n,
                           long long sstride)
{
    {
        const long long so = blockIdx.x * sstride;
        k = slot_ptr(k, so);
        l = slot_ptr(l, so);
        p = slot_ptr(p, so);
    }
    const double a2 = cta_sum(p, n);
    if (threadIdx.x != 0) return;
    if (l->stopped) return;
    int stop = 0;
    double alpha = sqrt(fmax(a2, 0.0));
    if (!isfinite(alpha)) {
        if (k->status == 0) k->status = -4;
        alpha = 0.0;
        stop = 1;
    }
    double normar, tw = 0.0;
    if (init) {
        l->rhobar = alpha;
        normar = alpha * l->beta;
        l->normar0 = normar;
        stop |= !(normar > 0.0);
    } else {
        const double theta = l->s * alpha;
        l->rhobar = -l->c * alpha;
        tw = theta / l->rho;
        normar = l->phibar * alpha * fabs(l->c);
        // same rule as CGLS: |A~^T r~| down to 1e-13 of its start, or a
        // vanishing bidiagonal entry (the least-squares solution is reached)
        stop |= !(normar > 1e-13 * l->normar0) || !(alpha > 0.0) || !(l->beta > 0.0);
    }
    l->alpha = alpha;
    if (k->n_hist < 512) k->hist[k->n_hist++] = normar * normar;
    const double ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
    const double kb = l->beta > 0.0 ? alpha / l->beta : 0.0;
    l->sigma_next = -kb * l->sigma;
    l->stopped = stop;
    const float fs = stop ? 1.f : 0.f;
    l->fwd[0] = (float)ia;
    l->fwd[1] = (float)kb;
    l->fwd[2] = fs;
    l->fwd[3] = (float)tw;
    l->fwd[5] = init ? 1.f : 0.f;
    l->ureg[0] = (float)ia;
    l->ureg[1] = (float)kb;
    l->ureg[2] = (float)l->sigma_next;
    l->ureg[3] = fs;
    l->vx[0] = (float)ia;
    l->vx[1] = (float)tw;
    l->vx[5] = fs;
    l->vx[6] = init ? 1.f : 0.f;
}

// Gram-Schmidt coefficients h_j = <basis_j, vhat>, eight basis vectors per
// blockIdx.y; one FP64 partial per (j, block) at partials[j * gridDim.x + block]
constexpr int kDotVecs = 8;

template <class BT>
__global__ void __launch_bounds__(kThreads)
lsqr_dots_kernel(long long M, long long ldb, int nb, const BT *__restrict__ basis,
                 const float *__restrict__ vhat, const LsqrScalars *__restrict__ l,
                 double *__restrict__ partials, long long sstride, long long bstride)
{
    {
        const long long so = blockIdx.z * sstride, bo = blockIdx.z * bstride;
        vhat = slot_ptr(vhat, so);
        l = slot_ptr(l, so);
        basis = slot_ptr(basis, bo);
        partials = slot_ptr(partials, bo);
    }
    if (l->stopped) return;
    const int j0 = blockIdx.y * kDotVecs;
    const int nj = min(kDotVecs, nb - j0);
    double acc[kDotVecs];
#pragma unroll
    for (int q = 0; q < kDotVecs; ++q) acc[q] = 0.0;
    const long long n4 = M >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const float4 *v4 = reinterpret_cast<const float4 *>(vhat);
    for (long long i = t0; i < n4; i += stride) {
        const float4 a = v4[i];
#pragma unroll
        for (int q = 0; q < kDotVecs; ++q) {
            if (q < nj) {
                const float4 b = ld4(basis + (long long)(j0 + q) * ldb, i);
                acc[q] += (double)fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
            }
        }
    }
    for (long long i = (n4 << 2) + t0; i < M; i += stride) {
#pragma unroll
        for (int q = 0; q < kDotVecs; ++q)
            if (q < nj) acc[q] += (double)vhat[i] * (double)ld1(basis + (long long)(j0 + q) * ldb, i);
    }
    __shared__ double red[kDotVecs][kThreads / 32];
#pragma unroll
    for (int q = 0; q < kDotVecs; ++q) {
        double t = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x < nj) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) t += red[threadIdx.x][w];
        partials[(long long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kFinThreads)
lsqr_fin_dots_kernel(LsqrScalars *l, const double *partials, int nblk, long long sstride,
                     long long bstride)
{
    l = slot_ptr(l, blockIdx.y * sstride);
    partials = slot_ptr(partials, blockIdx.y * bstride);
    const double h = cta_sum(partials + (long long)blockIdx.x * nblk, nblk);
    if (threadIdx.x == 0) l->h[blockIdx.x] = l->stopped ? 0.0 : h;
}

// vhat -= sum_j h_j basis_j; partials (may be null) get |vhat|^2
template <class BT>
__global__ void __launch_bounds__(kThreads)
lsqr_sub_kernel(long long M, long long ldb, int nb, const BT *__restrict__ basis,
                float *__restrict__ vhat, const LsqrScalars *__restrict__ l,
                double *__restrict__ partials, long long sstride, long long bstride)
{
    {
        const long long so = blockIdx.y * sstride;
        vhat = slot_ptr(vhat, so);
        l = slot_ptr(l, so);
        partials = slot_ptr(partials, so);
        basis = slot_ptr(basis, blockIdx.y * bstride);
    }
    if (l->stopped) return;
    const long long n4 = M >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float4 *v4 = reinterpret_cast<float4 *>(vhat);
    double acc = 0.0;
    for (long long i = t0; i < n4; i += stride) {
        float4 a = v4[i];
        for (int j = 0; j < nb; ++j) {
            const float h = (float)l->h[j];
            const float4 b = ld4(basis + (long long)j * ldb, i);
            a.x = fmaf(-h, b.x, a.x);
            a.y = fmaf(-h, b.y, a.y);
            a.z = fmaf(-h, b.z, a.z);
            a.w = fmaf(-h, b.w, a.w);
        }
        v4[i] = a;
        acc += (double)fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w)));
    }
    for (long long i = (n4 << 2) + t0; i < M; i += stride) {
        float a = vhat[i];
        for (int j = 0; j < nb; ++j) a = fmaf(-(float)l->h[j], ld1(basis + (long long)j * ldb, i), a);
        vhat[i] = a;
        acc += (double)a * (double)a;
    }
    if (partials) block_sum_store(acc, partials);
}

}  // namespace

int vector_blocks() { return 152 * 8; }

cudaError_t launch_p_update(long long M, const float *s, float *p, const KrylovScalars *k,
                            cudaStream_t st, Slots sl)
{
    p_update_kernel<<<dim3(vector_blocks(), sl.n), kThreads, 0, st>>>(M, s, p, k, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_x_update(long long M, long long N, float *x, const float *p, float *g,
                            const float *t, float *s, float *r, const float *q,
                            const KrylovScalars *k, cudaStream_t st, Slots sl)
{
    x_update_kernel<<<dim3(vector_blocks(), sl.n), kThreads, 0, st>>>(M, N, x, p, g, t, s, r, q, k,
                                                                     sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_norm2(long long n, const float *v, double *partials, cudaStream_t st, Slots sl)
{
    norm2_kernel<<<dim3(vector_blocks(), sl.n), kThreads, 0, st>>>(n, v, partials, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_finalize_delta(KrylovScalars *k, const double *pa, int na, const double *pb,
                                  int nb, cudaStream_t st, Slots sl)
{
    finalize_delta_kernel<<<sl.n, kFinThreads, 0, st>>>(k, pa, na, pb, nb, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_finalize_gamma(KrylovScalars *k, const double *p, int n, int restart,
                                  cudaStream_t st, Slots sl)
{
    finalize_gamma_kernel<<<sl.n, kFinThreads, 0, st>>>(k, p, n, restart, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_reset_scalars(KrylovScalars *k, cudaStream_t st, Slots sl)
{
    reset_scalars_kernel<<<sl.n, 1, 0, st>>>(k, sl.stride);
    return cudaGetLastError();
}

// BF16 data: NaN/Inf have all exponent bits set
__global__ void __launch_bounds__(kThreads)
count_nonfinite16_kernel(long long n, const unsigned short *__restrict__ v, int *__restrict__ flag,
                         long long sstride)
{
    v = slot_ptr(v, blockIdx.y * sstride);
    flag = slot_ptr(flag, blockIdx.y * sstride);
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= (v[i] & 0x7F80u) == 0x7F80u;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_count_nonfinite16(long long n, const void *v, int *flag, cudaStream_t st,
                                     Slots sl)
{
    count_nonfinite16_kernel<<<dim3(vector_blocks(), sl.n), kThreads, 0, st>>>(
        n, static_cast<const unsigned short *>(v), flag, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(long long n, const float *v, int *flag, cudaStream_t st,
                                   Slots sl)
{
    count_nonfinite_kernel<<<dim3(vector_blocks(), sl.n), kThreads, 0, st>>>(n, v, flag,
                                                                            sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double *p, int n, double *out, cudaStream_t st)
{
    sum_partials_kernel<<<1, kFinThreads, 0, st>>>(p, n, out);
    return cudaGetLastError();
}

int lsqr_dot_blocks() { return 152 * 2; }

cudaError_t launch_lsqr_rinit(long long N, int update, float *rA, const float *Aw, float *U,
                              const LsqrScalars *l, double *partials, cudaStream_t st, Slots sl)
{
    lsqr_rinit_kernel<<<dim3(vector_blocks(), sl.n), kThreads, 0, st>>>(N, update, rA, Aw, U, l,
                                                                       partials, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_reset(KrylovScalars *, LsqrScalars *l, cudaStream_t st, Slots sl)
{
    lsqr_reset_kernel<<<sl.n, 1, 0, st>>>(l, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_vx(long long M, int first, int last, float *x, float *w, float *vhat,
                           const float *s, void *basis, const LsqrScalars *l, double *partials,
                           cudaStream_t st, Slots sl, long long bstride, bool basis_bf16)
{
    const dim3 grid(vector_blocks(), sl.n);
    if (first)
        lsqr_vx_kernel<true, false, float><<<grid, kThreads, 0, st>>>(M, x, w, vhat, s, nullptr, l,
                                                                     partials, sl.stride, 0);
    else if (last)
        lsqr_vx_kernel<false, true, float><<<grid, kThreads, 0, st>>>(M, x, w, vhat, s, nullptr, l,
                                                                     partials, sl.stride, 0);
    else if (basis_bf16)
        lsqr_vx_kernel<false, false, __nv_bfloat16><<<grid, kThreads, 0, st>>>(
            M, x, w, vhat, s, static_cast<__nv_bfloat16 *>(basis), l, partials, sl.stride, bstride);
    else
        lsqr_vx_kernel<false, false, float><<<grid, kThreads, 0, st>>>(
            M, x, w, vhat, s, static_cast<float *>(basis), l, partials, sl.stride, bstride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_finalize_beta(KrylovScalars *k, LsqrScalars *l, int init,
                                      const double *pu, int nu, const double *pr, int nr,
                                      cudaStream_t st, Slots sl)
{
    lsqr_finalize_beta_kernel<<<sl.n, kFinThreads, 0, st>>>(k, l, init, pu, nu, pr, nr,
                                                            sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_finalize_alpha(KrylovScalars *k, LsqrScalars *l, int init,
                                       const double *p, int n, cudaStream_t st, Slots sl)
{
    lsqr_finalize_alpha_kernel<<<sl.n, kFinThreads, 0, st>>>(k, l, init, p, n, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_dots(long long M, long long ldb, int nb, const void *basis,
                             const float *vhat, const LsqrScalars *l, double *partials,
                             cudaStream_t st, Slots sl, long long bstride, bool basis_bf16)
{
    const dim3 grid((unsigned)lsqr_dot_blocks(), (unsigned)((nb + kDotVecs - 1) / kDotVecs),
                    (unsigned)sl.n);
    if (basis_bf16)
        lsqr_dots_kernel<__nv_bfloat16><<<grid, kThreads, 0, st>>>(
            M, ldb, nb, static_cast<const __nv_bfloat16 *>(basis), vhat, l, partials, sl.stride,
            bstride);
    else
        lsqr_dots_kernel<float><<<grid, kThreads, 0, st>>>(M, ldb, nb, static_cast<const float *>(basis),
                                                           vhat, l, partials, sl.stride, bstride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_fin_dots(int nb, LsqrScalars *l, const double *partials, cudaStream_t st,
                                 Slots sl, long long bstride)
{
    lsqr_fin_dots_kernel<<<dim3(nb, sl.n), kFinThreads, 0, st>>>(l, partials, lsqr_dot_blocks(),
                                                                 sl.stride, bstride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_sub(long long M, long long ldb, int nb, const void *basis, float *vhat,
                            const LsqrScalars *l, double *norm_partials, cudaStream_t st, Slots sl,
                            long long bstride, bool basis_bf16)
{
    const dim3 grid(vector_blocks(), sl.n);
    if (basis_bf16)
        lsqr_sub_kernel<__nv_bfloat16><<<grid, kThreads, 0, st>>>(
            M, ldb, nb, static_cast<const __nv_bfloat16 *>(basis), vhat, l, norm_partials, sl.stride,
            bstride);
    else
        lsqr_sub_kernel<float><<<grid, kThreads, 0, st>>>(M, ldb, nb, static_cast<const float *>(basis),
                                                          vhat, l, norm_partials, sl.stride, bstride);
    return cudaGetLastError();
}

}  // namespace piccs
