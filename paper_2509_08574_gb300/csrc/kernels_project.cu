// Cone-beam projector A and its matched adjoint A^T for sm_103a.
//
// A_ij is the length (mm) of ray i inside voxel j (the linear model of
// Sec. 2.1, Eq. 1, with exact ray/voxel intersection lengths).  Krylov
// methods need one product with A and one with A^T per iteration (Sec. 2.3,
// the text after the augmented system), so these two kernels carry nearly all
// of the bytes of a reconstruction.
//
// Layout of the work: one warp = 32 consecutive detector rows of one detector
// column of one view; one CTA = 8 adjacent columns.  Because the detector v
// axis is parallel to the rotation axis and the source lies in z = 0, every
// ray of a column has the same xy path.  That path is walked once per
// geometry on the host (FP64, ray_tables.h) and stored as the column's cell
// list; a warp streams it with one broadcast 16-byte load per four cells, so
// the xy part of the walk costs almost nothing and is warp-uniform.  Only the
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
// (never accumulated), so A^T applies bit-identical weights to A; only the
// order of the FP32 sums differs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace piccs {

namespace {

constexpr int kWarps = 8;        // detector columns per CTA
constexpr unsigned kFull = 0xffffffffu;

struct LaneRay {
    float zE;      // centred z (voxel units) at the entry point
    float inv_mz;  // xy distance per voxel of z (signed; +inf when v == 0)
    float sec;     // 3D length per unit xy length
    int stepz;
};

// per-ray factor: 3D length per unit of xy length
__device__ __forceinline__ float ray_sec(float v, float invD)
{
    const float m = v * invD;
    return __fsqrt_rn(fmaf(m, m, 1.f));
}

// v: row height; rv = 1/v (1e30 for v == 0, which never crosses a z plane)
__device__ __forceinline__ LaneRay lane_ray(const ColParams &cp, float v, float rv)
{
    LaneRay r;
    r.zE = v * cp.kE;
    r.inv_mz = cp.KD * rv;
    r.sec = ray_sec(v, cp.invD);
    r.stepz = (v >= 0.f) ? 1 : -1;
    return r;
}

// s at which the ray leaves voxel layer iz in its direction of travel
__device__ __forceinline__ float z_exit(int iz, const LaneRay &r, float halfnz)
{
    const float kc = (float)(iz + (r.stepz > 0)) - halfnz;  // centred plane coordinate
    return (kc - r.zE) * r.inv_mz;
}

__device__ __forceinline__ void decode_block(const ProjGeom &G, int &j, int &iu, int &iv)
{
    int b = blockIdx.x;
    const int ncg = (G.nu + kWarps - 1) / kWarps;
    const int cg = b % ncg;
    b /= ncg;
    j = b % G.n_views;
    const int rg = b / G.n_views;
    iu = cg * kWarps + (threadIdx.x >> 5);
    iv = rg * 32 + (threadIdx.x & 31);
}

// Per-lane state of the z part of the walk.
struct ZWalk {
    int iz;       // current voxel layer
    float szn;    // xy distance at which the ray leaves layer iz
    bool act;     // still inside the volume's z range
};

__device__ __forceinline__ ZWalk z_start(const LaneRay &r, bool ray_ok, const ProjGeom &G)
{
    ZWalk w;
    w.iz = __float2int_rd(r.zE + G.halfnz);
    w.act = ray_ok && w.iz >= 0 && w.iz < G.nz;
    // the FP32 layer index can disagree with the sign of a tiny z offset: a
    // first crossing "behind" the entry is taken at the entry
    w.szn = fmaxf(z_exit(w.iz, r, G.halfnz), 0.f);
    return w;
}

template <int MODE, bool NORM>
__global__ void __launch_bounds__(256)
fwd_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float *__restrict__ vrow,
           const float *__restrict__ rvrow, const float *__restrict__ cells,
           const float *__restrict__ vol,
           float *__restrict__ out, const float *__restrict__ b, double *__restrict__ partials,
           int *__restrict__ nonfinite)
{
    int j, iu, iv;
    decode_block(G, j, iu, iv);
    const bool col_ok = iu < G.nu;
    const bool ray_ok = col_ok && iv < G.nv;
    float acc = 0.f, sec = 1.f;

    if (col_ok) {
        const ColParams cp = cols[(long long)j * G.nu + iu];
        if (cp.ncells > 0) {
            const float v = ray_ok ? __ldg(vrow + iv) : 0.f;
            const float rv = ray_ok ? __ldg(rvrow + iv) : 1e30f;
            const LaneRay r = lane_ray(cp, v, rv);
            sec = r.sec;
            ZWalk z = z_start(r, ray_ok, G);
            if (__any_sync(kFull, z.act)) {
                const float4 *t4 = reinterpret_cast<const float4 *>(cells) + cp.start4;
                const int n = cp.ncells;
                const int dcx = cp.stepx * G.ny * G.nz, dcy = cp.stepy * G.nz;
                int colbase = (cp.ix0 * G.ny + cp.iy0) * G.nz;
                float s = 0.f;
                // one xy cell [s, |e|]: the pieces of this lane's ray in it
                auto cell = [&](float e) {
                    const float se = fabsf(e);
                    if (z.act) {
                        acc = fmaf(fminf(z.szn, se) - s, __ldg(vol + colbase + z.iz), acc);
                        while (z.szn < se) {
                            const float sl = z.szn;
                            z.iz += r.stepz;
                            if ((unsigned)z.iz >= (unsigned)G.nz) { z.act = false; break; }
                            z.szn = z_exit(z.iz, r, G.halfnz);
                            acc = fmaf(fminf(z.szn, se) - sl, __ldg(vol + colbase + z.iz), acc);
                        }
                    }
                    s = se;
                    colbase += (__float_as_int(e) < 0) ? dcy : dcx;
                };
                for (int c = 0; c < n; c += 4) {
                    const float4 e4 = __ldg(t4 + (c >> 2));
                    cell(e4.x);
                    if (c + 1 < n) cell(e4.y);
                    if (c + 2 < n) cell(e4.z);
                    if (c + 3 < n) cell(e4.w);
                    if (!__any_sync(kFull, z.act)) break;
                }
            }
        }
    }

    float val = 0.f;
    if (ray_ok) {
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
        __shared__ double red[kWarps];
        float sq = val * val;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) t += red[w];
            partials[blockIdx.x] = t;
        }
    }
}

// rs = proj * sec, per ray (the adjoint's gather then needs no square root)
__global__ void __launch_bounds__(256)
scale_rays_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float *__restrict__ vrow,
                  const float *__restrict__ proj, float *__restrict__ rs)
{
    int j, iu, iv;
    decode_block(G, j, iu, iv);
    if (iu >= G.nu || iv >= G.nv) return;
    const float invD = cols[(long long)j * G.nu + iu].invD;
    const long long idx = (long long)j * G.sj + (long long)iu * G.su + (long long)iv * G.sv;
    rs[idx] = proj[idx] * ray_sec(__ldg(vrow + iv), invD);
}

// Adjoint gather: CTA = one xy voxel column (ix, iy) and up to 256 z layers,
// thread = one voxel.  For every crossing (view j, detector column iu, xy
// interval [sa, sb]) of the voxel column, the rows whose rays pass through
// layer k within [sa, sb] form a short interval of v (ray height z = v*G(s),
// G(s) = kE + s*rKD); each is checked with the exact piece length.
__global__ void __launch_bounds__(256)
adj_gather_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float *__restrict__ vrow,
                  const float *__restrict__ rvrow, const int *__restrict__ hit_ptr,
                  const CellHit *__restrict__ hits, const float *__restrict__ rs,
                  float *__restrict__ vol)
{
    const int cell = blockIdx.x;
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    const bool kok = k < G.nz;
    const float zl = (float)k - G.halfnz;  // centred coordinate of the layer's lower plane
    const float zh = zl + 1.f;
    const int h0 = __ldg(hit_ptr + cell), h1 = __ldg(hit_ptr + cell + 1);
    float acc = 0.f;
    for (int h = h0; h < h1; ++h) {
        const CellHit e = __ldg(hits + h);
        const int j = e.x >> 16, iu = e.x & 0xffff;
        const float sa = __int_as_float(e.y), sb = __int_as_float(e.z);
        const float4 cz = __ldg(reinterpret_cast<const float4 *>(cols + (long long)j * G.nu + iu) + 2);
        const float kE = cz.x, KD = cz.y, rKD = cz.w;
        // rays with z in [zl, zh] somewhere in [sa, sb]: v in [vlo, vhi]
        const float rGa = __frcp_rn(fmaf(sa, rKD, kE)), rGb = __frcp_rn(fmaf(sb, rKD, kE));
        const float vlo = fminf(zl * rGa, zl * rGb), vhi = fmaxf(zh * rGa, zh * rGb);
        int ilo = (int)ceilf(fmaf(vlo, G.rdv, G.cv) - 1e-3f);
        int ihi = (int)floorf(fmaf(vhi, G.rdv, G.cv) + 1e-3f);
        ilo = max(ilo, 0);
        ihi = kok ? min(ihi, G.nv - 1) : -1;
        const long long rbase = (long long)j * G.sj + (long long)iu * G.su;
        for (int iv = ilo; iv <= ihi; ++iv) {
            const float v = __ldg(vrow + iv), rv = __ldg(rvrow + iv);
            const float zE = v * kE, inv = KD * rv;
            const bool up = v >= 0.f;
            // plane the ray leaves layer k through, and the one it enters through
            const float sx = ((up ? zh : zl) - zE) * inv;
            const float sn = ((up ? zl : zh) - zE) * inv;
            const float len = fminf(sb, sx) - fmaxf(sa, sn);
            if (len > 0.f) acc = fmaf(len, __ldg(rs + rbase + (long long)iv * G.sv), acc);
        }
    }
    if (kok) {
        const long long i = (long long)cell * G.nz + k;
        vol[i] += acc;
    }
}

}  // namespace

int project_blocks(const ProjGeom &g)
{
    const int ncg = (g.nu + kWarps - 1) / kWarps;
    const int nrg = (g.nv + 31) / 32;
    return ncg * nrg * g.n_views;
}

cudaError_t launch_forward(const ProjGeom &g, const ColParams *cols, const float *vrow,
                           const float *rvrow, const float *cells, const float *vol, float *out,
                           int mode, const float *b, double *partials, int *nonfinite,
                           cudaStream_t st)
{
    const int nb = project_blocks(g);
    if (nb <= 0) return cudaSuccess;
    if (mode == FWD_RESID) {
        if (partials)
            fwd_kernel<FWD_RESID, true><<<nb, 256, 0, st>>>(g, cols, vrow, rvrow, cells, vol, out, b, partials,
                                                            nonfinite);
        else
            fwd_kernel<FWD_RESID, false><<<nb, 256, 0, st>>>(g, cols, vrow, rvrow, cells, vol, out, b, partials,
                                                             nonfinite);
    } else {
        if (partials)
            fwd_kernel<FWD_PLAIN, true><<<nb, 256, 0, st>>>(g, cols, vrow, rvrow, cells, vol, out, b, partials,
                                                            nonfinite);
        else
            fwd_kernel<FWD_PLAIN, false><<<nb, 256, 0, st>>>(g, cols, vrow, rvrow, cells, vol, out, b, partials,
                                                             nonfinite);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const ProjGeom &g, const ColParams *cols, const float *vrow,
                           const float *rvrow, const int *hit_ptr, const CellHit *hits,
                           const float *proj, float *rs, float *vol, cudaStream_t st)
{
    const int nb = project_blocks(g);
    if (nb <= 0) return cudaSuccess;
    scale_rays_kernel<<<nb, 256, 0, st>>>(g, cols, vrow, proj, rs);
    const dim3 grid((unsigned)(g.nx * g.ny), (unsigned)((g.nz + 255) / 256));
    adj_gather_kernel<<<grid, 256, 0, st>>>(g, cols, vrow, rvrow, hit_ptr, hits, rs, vol);
    return cudaGetLastError();
}

}  // namespace piccs
