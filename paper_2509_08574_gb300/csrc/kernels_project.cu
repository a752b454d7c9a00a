// Cone-beam projector A and its matched adjoint A^T for sm_103a.
//
// A_ij is the length (mm) of ray i inside voxel j (the linear model of
// Sec. 2.1, Eq. 1, with exact ray/voxel intersection lengths).  Krylov
// methods need one product with A and one with A^T per iteration (Sec. 2.3,
// the text after the augmented system), so these two kernels carry nearly all
// of the bytes of a reconstruction.
//
// Layout of the work: one warp = 32 consecutive detector rows of one detector
// column of one view; one CTA = 8 such warps of the same column (256 rows),
// so the column's cell list is fetched from DRAM once per CTA.  Because the detector v
// axis is parallel to the rotation axis and the source lies in z = 0, every
// ray of a column has the same xy path.  That path is walked once per
// geometry on the host (FP64, ray_tables.h) and stored as the column's cell
// list (voxel-column index and exit distance per cell); a warp streams it with
// one broadcast 16-byte load per two cells, so the xy part of the walk costs
// almost nothing and is warp-uniform.  Only the
// z crossings are per lane.  At every xy cell the 32 lanes touch neighbouring
// z voxels of one z-fastest voxel column, so the forward gathers coalesce into
// one or two 32-byte sectors.
//
// The adjoint is a gather over the transpose of the same tables: one thread
// per voxel (one CTA per xy voxel column) visits every detector column that
// crosses its voxel column and, for the two or three rows whose rays cross its
// z layer there, adds piece length x ray value -- no atomics, one store per
// voxel, deterministic.  Both kernels evaluate the same piece lengths
//   len = min(s_exit_xy, s_z(exit plane)) - max(s_enter_xy, s_z(entry plane))
// from the same FP32 cell boundaries and the same plane-crossing formula
// fma(kc, KD / v, -s0), with the exact plane coordinate kc (never an
// accumulated distance), so A^T applies bit-identical weights to A; only the
// order of the FP32 sums differs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace piccs {

namespace {

constexpr int kRowGroups = 8;    // warps per forward CTA: 8 x 32 rows of one column
constexpr int kGatherThreads = 64;
constexpr int kLayersPerThread = 4;
constexpr unsigned kFull = 0xffffffffu;

// per-ray factor: 3D length per unit of xy length
__device__ __forceinline__ float ray_sec(float v, float invD)
{
    const float m = v * invD;
    return __fsqrt_rn(fmaf(m, m, 1.f));
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// CTA = one detector column (j, iu) and kRowGroups groups of 32 rows
__device__ __forceinline__ void decode_block(const ProjGeom &G, int &col, int &iv)
{
    const int nrgb = (G.nv + 32 * kRowGroups - 1) / (32 * kRowGroups);
    const int b = blockIdx.x;
    col = b / nrgb;
    iv = ((b - col * nrgb) * kRowGroups + (threadIdx.x >> 5)) * 32 + (threadIdx.x & 31);
}

template <int MODE, bool NORM>
__global__ void __launch_bounds__(256)
fwd_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
           const int4 *__restrict__ cells, const float *__restrict__ vol,
           float *__restrict__ out, const float *__restrict__ b, double *__restrict__ partials,
           int *__restrict__ nonfinite)
{
    int col, iv;
    decode_block(G, col, iv);
    const bool ray_ok = iv < G.nv;
    float acc = 0.f, sec = 1.f;
    const ColParams cp = cols[col];
    if (cp.ncells > 0) {
        const float2 w = ray_ok ? __ldg(vr + iv) : make_float2(0.f, 1e30f);
        const float inv = cp.KD * w.y;  // xy distance per voxel of z (signed)
        sec = ray_sec(w.x, cp.invD);
        const bool up = w.y > 0.f;      // rv = 1e30 > 0 for v = 0
        const int stepz = up ? 1 : -1;
        const float stepf = up ? 1.f : -1.f;
        int iz = __float2int_rd(w.x * (cp.s0 * cp.rKD) + G.halfnz);
        bool act = ray_ok && iz >= 0 && iz < G.nz;
        if (!act) iz = 0;
        // centred coordinate of the plane the ray leaves layer iz through
        float kce = (float)(iz + (up ? 1 : 0)) - G.halfnz;
        // the FP32 layer index can disagree with the sign of a tiny z offset:
        // a first crossing "behind" the entry is taken at the entry
        float szn = fmaxf(fmaf(kce, inv, -cp.s0), 0.f);
        if (__any_sync(kFull, act)) {
            const int4 *t = cells + cp.start2;
            const int n2 = (cp.ncells + 1) >> 1;
            float s = 0.f;
            // one xy cell [s, se] of the voxel column at colbase: this ray's pieces
            auto cell = [&](int colbase, float se) {
                const float *cpv = vol + colbase;
                if (act) {
                    acc = fmaf(fminf(szn, se) - s, __ldg(cpv + iz), acc);
                    while (szn < se) {
                        const float sl = szn;
                        iz += stepz;
                        if ((unsigned)iz >= (unsigned)G.nz) { act = false; break; }
                        kce += stepf;
                        szn = fmaf(kce, inv, -cp.s0);
                        acc = fmaf(fminf(szn, se) - sl, __ldg(cpv + iz), acc);
                    }
                }
                s = se;
            };
            for (int c = 0; c < n2; ++c) {
                const int4 e = __ldg(t + c);
                cell(e.x, __int_as_float(e.y));
                cell(e.z, __int_as_float(e.w));
                if ((c & 1) && !__any_sync(kFull, act)) break;
            }
        }
    }

    float val = 0.f;
    if (ray_ok) {
        const int j = col / G.nu, iu = col - j * G.nu;
        const long long idx = (long long)j * G.sj + (long long)iu * G.su + (long long)iv * G.sv;
        const float q = sec * acc;
        if (MODE == FWD_RESID) {
            const float bb = b[idx];
            if (!isfinite(bb)) atomicOr(nonfinite, 1);
            val = bb - q;
        } else {
            val = q;
        }
        out[idx] = val;
    }
    if (NORM) {
        __shared__ double red[kRowGroups];
        float sq = val * val;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kRowGroups; ++w) t += red[w];
            partials[blockIdx.x] = t;
        }
    }
}

// rs = proj * sec, per ray (the adjoint's gather then needs no square root)
__global__ void __launch_bounds__(256)
scale_rays_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
                  const float *__restrict__ proj, float *__restrict__ rs)
{
    int col, iv;
    decode_block(G, col, iv);
    if (iv >= G.nv) return;
    const int j = col / G.nu, iu = col - j * G.nu;
    const long long idx = (long long)j * G.sj + (long long)iu * G.su + (long long)iv * G.sv;
    rs[idx] = proj[idx] * ray_sec(__ldg(vr + iv).x, cols[col].invD);
}

// Adjoint gather: CTA = one xy voxel column (ix, iy) and up to 256 z layers,
// thread = kLayersPerThread layers (k, k + 64, ...).  For every crossing
// (view j, detector column iu, xy interval [sa, sb]) of the voxel column, the
// rows whose rays pass through layer k inside [sa, sb] form a short interval
// of heights v (ray z = v * (s0 + s) * rKD, so v in [zl, zh] / ((s0 + s) rKD));
// each candidate row is checked with the exact piece length, the same
// expression the forward walk evaluates.
__global__ void __launch_bounds__(kGatherThreads)
adj_gather_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
                  const int *__restrict__ hit_ptr, const CellHit *__restrict__ hits,
                  const float *__restrict__ rs, float *__restrict__ vol)
{
    constexpr int L = kLayersPerThread;
    const int cell = blockIdx.x;
    const int kb = blockIdx.y * kGatherThreads * L + threadIdx.x;
    float zlo[L], acc[L];
    bool kok[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        const int k = kb + q * kGatherThreads;
        kok[q] = k < G.nz;
        zlo[q] = (float)k - G.halfnz;  // centred coordinate of the layer's lower plane
        acc[q] = 0.f;
    }
    const int h0 = __ldg(hit_ptr + cell), h1 = __ldg(hit_ptr + cell + 1);
    for (int h = h0; h < h1; ++h) {
        const CellHit e = __ldg(hits + h);
        const int j = e.x >> 16, iu = e.x & 0xffff;
        const float sa = __int_as_float(e.y), sb = __int_as_float(e.z);
        const float4 cz = __ldg(reinterpret_cast<const float4 *>(cols + (long long)j * G.nu + iu) + 1);
        const float s0 = cz.x, KD = cz.y, rKD = cz.w;
        // candidate bounds only: the rows are then checked exactly
        const float rGa = rcp_approx((s0 + sa) * rKD), rGb = rcp_approx((s0 + sb) * rKD);
        const float *rsc = rs + (long long)j * G.sj + (long long)iu * G.su;
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const float zl = zlo[q], zh = zl + 1.f;
            const float vlo = fminf(zl * rGa, zl * rGb), vhi = fmaxf(zh * rGa, zh * rGb);
            int ilo = __float2int_ru(fmaf(vlo, G.rdv, G.cv - 1e-3f));
            int ihi = __float2int_rd(fmaf(vhi, G.rdv, G.cv + 1e-3f));
            ilo = max(ilo, 0);
            ihi = kok[q] ? min(ihi, G.nv - 1) : -1;
            auto cand = [&](int iv) {
                const float inv = KD * __ldg(vr + iv).y;
                const float xl = fmaf(zl, inv, -s0), xh = fmaf(zh, inv, -s0);
                // the ray is inside the layer between its two plane crossings
                const float len = fminf(sb, fmaxf(xl, xh)) - fmaxf(sa, fminf(xl, xh));
                if (len > 0.f) acc[q] = fmaf(len, __ldg(rsc + iv * G.sv32), acc[q]);
            };
            if (ilo <= ihi) cand(ilo);
            if (ilo + 1 <= ihi) cand(ilo + 1);
            if (ilo + 2 <= ihi) cand(ilo + 2);
            for (int iv = ilo + 3; iv <= ihi; ++iv) cand(iv);
        }
    }
#pragma unroll
    for (int q = 0; q < L; ++q)
        if (kok[q]) vol[(long long)cell * G.nz + kb + q * kGatherThreads] += acc[q];
}

}  // namespace

int project_blocks(const ProjGeom &g)
{
    const int nrgb = (g.nv + 32 * kRowGroups - 1) / (32 * kRowGroups);
    return g.n_views * g.nu * nrgb;
}

cudaError_t launch_forward(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                           const int4 *cells, const float *vol, float *out, int mode,
                           const float *b, double *partials, int *nonfinite, cudaStream_t st)
{
    const int nb = project_blocks(g);
    if (nb <= 0) return cudaSuccess;
    if (mode == FWD_RESID) {
        if (partials)
            fwd_kernel<FWD_RESID, true><<<nb, 256, 0, st>>>(g, cols, vr, cells, vol, out, b,
                                                            partials, nonfinite);
        else
            fwd_kernel<FWD_RESID, false><<<nb, 256, 0, st>>>(g, cols, vr, cells, vol, out, b,
                                                             partials, nonfinite);
    } else {
        if (partials)
            fwd_kernel<FWD_PLAIN, true><<<nb, 256, 0, st>>>(g, cols, vr, cells, vol, out, b,
                                                            partials, nonfinite);
        else
            fwd_kernel<FWD_PLAIN, false><<<nb, 256, 0, st>>>(g, cols, vr, cells, vol, out, b,
                                                             partials, nonfinite);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                           const int *hit_ptr, const CellHit *hits, const float *proj, float *rs,
                           float *vol, cudaStream_t st)
{
    const int nb = project_blocks(g);
    if (nb <= 0) return cudaSuccess;
    scale_rays_kernel<<<nb, 256, 0, st>>>(g, cols, vr, proj, rs);
    const int per_cta = kGatherThreads * kLayersPerThread;
    const dim3 grid((unsigned)(g.nx * g.ny), (unsigned)((g.nz + per_cta - 1) / per_cta));
    adj_gather_kernel<<<grid, kGatherThreads, 0, st>>>(g, cols, vr, hit_ptr, hits, rs, vol);
    return cudaGetLastError();
}

}  // namespace piccs
