// PICCS regularisation terms for sm_103a: IRN weights, the prior right-hand
// side and the regularisation block of the normal operator.
//
// D stacks the forward differences (D_d z)_i = z_i - z_{i+e_d} along x, y, z
// (D1 rows [1, -1], Sec. 2.2), each zero where i+e_d leaves the grid.  With
// the weights frozen per IRN cycle (Eqs. 10-11), the two regularisation blocks
// alpha W1 D and lambda W2 D of the augmented system enter the normal
// equations only through one combined per-voxel field
//   omega = alpha^2 w1^2 + lambda^2 w2^2,
// because W1 and W2 repeat the same value over the three directions:
//   [alpha W1 D; lambda W2 D]^T [alpha W1 D; lambda W2 D] = D^T diag(omega) D,
// and the right-hand side block is c = lambda^2 D^T W2^2 D x_p.  So the solver
// never stores the 6M augmented rows; each application is one 7-point stencil
// pass.  All kernels are memory-bound streaming passes over z-fastest volumes:
// blocks stride over the xy voxel columns and the threads of a block run
// along z, so no voxel index is ever divided; the +-1 and +-nz neighbours
// come from L1 and the +-ny*nz neighbours from L2.  Sums are kept per thread
// in compensated FP32 and combined in FP64 per block (FP64 arithmetic per
// voxel would cost more than the memory traffic on this GPU).
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace piccs {

namespace {

constexpr int kThreads = 256;

// Visits every voxel once.  The threads of a block form groups of nzr (nz /
// kPer, rounded up to whole warps, at most the block), one xy column
// (ix * ny + iy) per group, each thread kPer z layers nzr apart so that
// several voxels' loads are in flight; the block's groups take consecutive
// columns and the grid strides over them, stepping (ix, iy) without division.
// f(i, ix, iy, iz), i the flat index (32-bit: the volume has < 2^31 voxels).
template <int kPer, class F>
__device__ __forceinline__ void for_voxels(const VolDims &d, F &&f)
{
    const int nzr = min(((d.nz + kPer - 1) / kPer + 31) / 32 * 32, (int)blockDim.x);
    const int cpi = (int)blockDim.x / nzr;
    const int sub = (int)threadIdx.x / nzr, tz = (int)threadIdx.x - sub * nzr;
    if (sub >= cpi) return;
    const int ncol = d.nx * d.ny;
    const int step = (int)gridDim.x * cpi;
    const int step_x = step / d.ny, step_y = step - step_x * d.ny;
    int col = (int)blockIdx.x * cpi + sub;
    int ix = col / d.ny, iy = col - ix * d.ny;
    for (; col < ncol; col += step) {
        const int base = col * d.nz;
        for (int z0 = tz; z0 < d.nz; z0 += kPer * nzr) {
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int iz = z0 + k * nzr;
                if (iz < d.nz) f(base + iz, ix, iy, iz);
            }
        }
        ix += step_x;
        iy += step_y;
        if (iy >= d.ny) {
            iy -= d.ny;
            ++ix;
        }
    }
}

// Compensated (Kahan) FP32 sum of one thread's terms.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// w^2 for a gradient with squared Euclidean norm n2 (tau2 = tau^2):
// R1 1/(|g| + tau^2), R2 1/sqrt(|g|^2 + tau^2)
__device__ __forceinline__ float weight_sq(float n2, float tau2, int rule)
{
    if (rule == 0) return 1.f / (sqrtf(n2) + tau2);
    return rsqrtf(n2 + tau2);
}

__global__ void __launch_bounds__(kThreads)
weights_kernel(VolDims d, long long M, const float *__restrict__ x, const float *__restrict__ xp,
               float alpha2, float lambda2, float tau2, int rule, int variant,
               float *__restrict__ omega, float *__restrict__ w2sq, long long sstride)
{
    const long long so = blockIdx.y * sstride;
    x = slot_ptr(x, so);
    xp = slot_ptr(xp, so);
    omega = slot_ptr(omega, so);
    w2sq = slot_ptr(w2sq, so);
    const int sx = d.ny * d.nz, sy = d.nz;
    (void)M;
    for_voxels<1>(d, [&](int i, int ix, int iy, int iz) {
        const float xi = x[i];
        const float gx = (ix + 1 < d.nx) ? xi - x[i + sx] : 0.f;
        const float gy = (iy + 1 < d.ny) ? xi - x[i + sy] : 0.f;
        const float gz = (iz + 1 < d.nz) ? xi - x[i + 1] : 0.f;
        float om = 0.f;
        if (variant != 3) om = alpha2 * weight_sq(gx * gx + gy * gy + gz * gz, tau2, rule);
        if (variant == 0) {
            const float di = xi - xp[i];
            const float hx = (ix + 1 < d.nx) ? di - (x[i + sx] - xp[i + sx]) : 0.f;
            const float hy = (iy + 1 < d.ny) ? di - (x[i + sy] - xp[i + sy]) : 0.f;
            const float hz = (iz + 1 < d.nz) ? di - (x[i + 1] - xp[i + 1]) : 0.f;
            const float w2 = weight_sq(hx * hx + hy * hy + hz * hz, tau2, rule);
            om += lambda2 * w2;
            w2sq[i] = w2;
        }
        omega[i] = om;
    });
}

// c = lambda^2 D^T W2^2 D x_p (PICCS), lambda^2 x_p (PIPLE), 0 otherwise
__global__ void __launch_bounds__(kThreads)
prior_rhs_kernel(VolDims d, long long M, const float *__restrict__ xp,
                 const float *__restrict__ w2sq, float lambda2, int variant, float *__restrict__ c,
                 long long sstride)
{
    const long long so = blockIdx.y * sstride;
    xp = slot_ptr(xp, so);
    w2sq = slot_ptr(w2sq, so);
    c = slot_ptr(c, so);
    const int sx = d.ny * d.nz, sy = d.nz;
    (void)M;
    for_voxels<1>(d, [&](int i, int ix, int iy, int iz) {
        float out = 0.f;
        if (variant == 0) {
            const float pi = xp[i], wi = w2sq[i];
            float acc = 0.f;
            if (ix + 1 < d.nx) acc += wi * (pi - xp[i + sx]);
            if (iy + 1 < d.ny) acc += wi * (pi - xp[i + sy]);
            if (iz + 1 < d.nz) acc += wi * (pi - xp[i + 1]);
            if (ix >= 1) acc -= w2sq[i - sx] * (xp[i - sx] - pi);
            if (iy >= 1) acc -= w2sq[i - sy] * (xp[i - sy] - pi);
            if (iz >= 1) acc -= w2sq[i - 1] * (xp[i - 1] - pi);
            out = lambda2 * acc;
        } else if (variant == 1) {
            out = lambda2 * xp[i];
        }
        c[i] = out;
    });
}

// t = D^T diag(omega) D z (+ lam2 z) at voxel i, and omega |(Dz)_i|^2 (+ lam2 z_i^2)
__device__ __forceinline__ float stencil_at(const VolDims &d, int i, int ix, int iy, int iz,
                                            const float *__restrict__ z,
                                            const float *__restrict__ omega, float lam2,
                                            float &energy)
{
    const int sx = d.ny * d.nz, sy = d.nz;
    const float zi = z[i];
    const float w = omega[i];
    const float gx = (ix + 1 < d.nx) ? zi - z[i + sx] : 0.f;
    const float gy = (iy + 1 < d.ny) ? zi - z[i + sy] : 0.f;
    const float gz = (iz + 1 < d.nz) ? zi - z[i + 1] : 0.f;
    float t = w * (gx + gy + gz);
    if (ix >= 1) t -= omega[i - sx] * (z[i - sx] - zi);
    if (iy >= 1) t -= omega[i - sy] * (z[i - sy] - zi);
    if (iz >= 1) t -= omega[i - 1] * (z[i - 1] - zi);
    t = fmaf(lam2, zi, t);
    energy = w * (gx * gx + gy * gy + gz * gz) + lam2 * zi * zi;
    return t;
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

template <bool NORM>
__global__ void __launch_bounds__(kThreads)
reg_normal_kernel(VolDims d, long long M, const float *__restrict__ z,
                  const float *__restrict__ omega, float lam2, float *__restrict__ out,
                  double *__restrict__ partials, long long sstride)
{
    const long long so = blockIdx.y * sstride;
    z = slot_ptr(z, so);
    omega = slot_ptr(omega, so);
    out = slot_ptr(out, so);
    partials = slot_ptr(partials, so);
    KahanF acc;
    (void)M;
    for_voxels<2>(d, [&](int i, int ix, int iy, int iz) {
        float e;
        out[i] = stencil_at(d, i, ix, iy, iz, z, omega, lam2, e);
        if (NORM) acc.add(e);
    });
    if (NORM) block_sum_store(acc.value(), partials);
}

__global__ void __launch_bounds__(kThreads)
reg_restart_kernel(VolDims d, long long M, const float *__restrict__ x,
                   const float *__restrict__ omega, float lam2, const float *__restrict__ c,
                   float *__restrict__ g, float *__restrict__ s, int first,
                   double *__restrict__ partials, long long sstride)
{
    const long long so = blockIdx.y * sstride;
    x = slot_ptr(x, so);
    omega = slot_ptr(omega, so);
    c = slot_ptr(c, so);
    g = slot_ptr(g, so);
    s = slot_ptr(s, so);
    partials = slot_ptr(partials, so);
    KahanF acc;
    (void)M;
    for_voxels<2>(d, [&](int i, int ix, int iy, int iz) {
        float e;
        const float gn = c[i] - stencil_at(d, i, ix, iy, iz, x, omega, lam2, e);
        const float sn = first ? gn : s[i] + (gn - g[i]);
        g[i] = gn;
        s[i] = sn;
        acc.add(sn * sn);
    });
    if (partials) block_sum_store(acc.value(), partials);
}

// Block sums of up to three per-thread values, one partial per block each,
// at partials[a * gridDim.x + blockIdx.x].
template <int NV>
__device__ __forceinline__ void block_sums_store(const double (&v)[NV], double *partials)
{
    __shared__ double red[NV][kThreads / 32];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        double t = v[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) t += red[threadIdx.x][w];
        partials[(long long)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// Regularisation part of A~^T u for LSQR: s = K z + sigma c with K the
// regularisation normal operator, and the partial sums z.K z, <z, c> (and,
// in the first step of a cycle, <x_p, c> = |b_R|^2); z was formed by
// lsqr_zstep_kernel.
template <bool INIT>
__global__ void __launch_bounds__(kThreads)
lsqr_ureg_kernel(VolDims d, long long M, const float *__restrict__ z,
                 const float *__restrict__ omega, float lam2, const float *__restrict__ c,
                 const float *__restrict__ xp, float *__restrict__ s,
                 const float *__restrict__ co, double *__restrict__ partials, long long sstride)
{
    {
        const long long so = blockIdx.y * sstride;
        z = slot_ptr(z, so);
        omega = slot_ptr(omega, so);
        c = slot_ptr(c, so);
        xp = slot_ptr(xp, so);
        s = slot_ptr(s, so);
        co = slot_ptr(co, so);
        partials = slot_ptr(partials, so);
    }
    float sig = 1.f;
    if (!INIT) {
        if (co[3] != 0.f) return;
        sig = co[2];
    }
    KahanF k0, k1, k2;
    (void)M;
    for_voxels<2>(d, [&](int i, int ix, int iy, int iz) {
        float e;
        const float t = stencil_at(d, i, ix, iy, iz, z, omega, lam2, e);
        const float ci = c[i];
        s[i] = fmaf(sig, ci, t);
        k0.add(e);
        k1.add(z[i] * ci);
        if (INIT && xp) k2.add(xp[i] * ci);  // |b_R|^2 (no prior: b_R = 0)
    });
    const double acc[3] = {k0.value(), k1.value(), k2.value()};
    if (INIT) {
        block_sums_store<3>(acc, partials);
    } else {
        const double a2[2] = {acc[0], acc[1]};
        block_sums_store<2>(a2, partials);
    }
}

// LSQR z-step: z' = co[0] src - co[1] zold (init: z' = -src), four voxels a
// thread at a time.
template <bool INIT>
__global__ void __launch_bounds__(kThreads)
lsqr_zstep_kernel(long long M, const float *__restrict__ src, const float *__restrict__ zold,
                  float *__restrict__ znew, const float *__restrict__ co, long long sstride)
{
    {
        const long long so = blockIdx.y * sstride;
        src = slot_ptr(src, so);
        zold = slot_ptr(zold, so);
        znew = slot_ptr(znew, so);
        co = slot_ptr(co, so);
    }
    float ca = -1.f, cb = 0.f;
    if (!INIT) {
        if (co[3] != 0.f) return;
        ca = co[0];
        cb = co[1];
    }
    const long long n4 = M >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    const float4 *o4 = reinterpret_cast<const float4 *>(zold);
    float4 *n4p = reinterpret_cast<float4 *>(znew);
    for (long long i = t0; i < n4; i += stride) {
        const float4 a = s4[i];
        float4 r;
        if (INIT) {
            r = make_float4(-a.x, -a.y, -a.z, -a.w);
        } else {
            const float4 b = o4[i];
            r = make_float4(fmaf(ca, a.x, -cb * b.x), fmaf(ca, a.y, -cb * b.y),
                            fmaf(ca, a.z, -cb * b.z), fmaf(ca, a.w, -cb * b.w));
        }
        n4p[i] = r;
    }
    for (long long i = (n4 << 2) + t0; i < M; i += stride)
        znew[i] = INIT ? -src[i] : fmaf(ca, src[i], -cb * zold[i]);
}

}  // namespace

int stencil_blocks(long long M)
{
    // persistent-style grid: 152 SMs x 8 resident CTAs of 256 threads
    long long want = (M + kThreads - 1) / kThreads;
    const long long cap = kStencilMaxBlocks;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_weights(VolDims d, const float *x, const float *xp, float alpha2,
                           float lambda2, float tau2, int rule, int variant, float *omega,
                           float *w2sq, cudaStream_t st, Slots sl)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    weights_kernel<<<dim3(stencil_blocks(M), sl.n), kThreads, 0, st>>>(
        d, M, x, xp, alpha2, lambda2, tau2, rule, variant, omega, w2sq, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_prior_rhs(VolDims d, const float *xp, const float *w2sq, float lambda2,
                             int variant, float *c, cudaStream_t st, Slots sl)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    prior_rhs_kernel<<<dim3(stencil_blocks(M), sl.n), kThreads, 0, st>>>(d, M, xp, w2sq, lambda2,
                                                                        variant, c, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_reg_normal(VolDims d, const float *z, const float *omega, float lam2_piple,
                              float *out, double *partials, cudaStream_t st, Slots sl)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    const dim3 grid(stencil_blocks(M), sl.n);
    if (partials)
        reg_normal_kernel<true><<<grid, kThreads, 0, st>>>(d, M, z, omega, lam2_piple, out,
                                                           partials, sl.stride);
    else
        reg_normal_kernel<false><<<grid, kThreads, 0, st>>>(d, M, z, omega, lam2_piple, out,
                                                            partials, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_reg_restart(VolDims d, const float *x, const float *omega, float lam2_piple,
                               const float *c, float *g, float *s, int first, double *partials,
                               cudaStream_t st, Slots sl)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    reg_restart_kernel<<<dim3(stencil_blocks(M), sl.n), kThreads, 0, st>>>(
        d, M, x, omega, lam2_piple, c, g, s, first, partials, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_zstep(VolDims d, int init, const float *src, const float *zold, float *znew,
                              const float *co, cudaStream_t st, Slots sl)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    const dim3 grid(152 * 8, sl.n);
    if (init)
        lsqr_zstep_kernel<true><<<grid, kThreads, 0, st>>>(M, src, zold, znew, co, sl.stride);
    else
        lsqr_zstep_kernel<false><<<grid, kThreads, 0, st>>>(M, src, zold, znew, co, sl.stride);
    return cudaGetLastError();
}

cudaError_t launch_lsqr_ureg(VolDims d, int init, const float *z, const float *omega,
                             float lam2_piple, const float *c, const float *xp, float *s,
                             const float *co, double *partials, cudaStream_t st, Slots sl)
{
    const long long M = (long long)d.nx * d.ny * d.nz;
    const dim3 grid(stencil_blocks(M), sl.n);
    if (init)
        lsqr_ureg_kernel<true><<<grid, kThreads, 0, st>>>(d, M, z, omega, lam2_piple, c, xp, s, co,
                                                          partials, sl.stride);
    else
        lsqr_ureg_kernel<false><<<grid, kThreads, 0, st>>>(d, M, z, omega, lam2_piple, c, xp, s, co,
                                                           partials, sl.stride);
    return cudaGetLastError();
}

}  // namespace piccs
