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
// ray of a column has the same xy path: the xy part of the Siddon walk is
// warp-uniform (no divergence, one broadcast table entry per warp) and only
// the z crossings are per lane.  At every xy cell the 32 lanes touch
// neighbouring z voxels of the same z-fastest voxel column, so the gathers of
// the forward projector coalesce into one or two 32-byte sectors.
//
// Both kernels run the same walk and evaluate the same piece lengths
//   len = min(s_exit_xy, s_z(k+1)) - max(s_enter_xy, s_z(k))
// with every plane crossing computed from its plane index (never
// accumulated), so A^T sees bit-identical piece lengths and the same per-ray
// factor sec as A; only the order of the FP32 sums differs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace piccs {

namespace {

constexpr int kWarps = 8;        // detector columns per CTA
constexpr int kWin = 128;        // adjoint staging window, voxels per warp
constexpr unsigned kFull = 0xffffffffu;

struct LaneRay {
    float zE;      // centred z (voxel units) at the entry point
    float inv_mz;  // xy distance per voxel of z (signed; +inf when v == 0)
    float sec;     // 3D length per unit xy length
    int stepz;
};

__device__ __forceinline__ LaneRay lane_ray(const ColParams &cp, float v)
{
    LaneRay r;
    r.zE = v * cp.kE;
    r.inv_mz = (v != 0.f) ? __fdiv_rn(cp.KD, v) : __int_as_float(0x7f800000);
    const float m = v * cp.invD;
    r.sec = __fsqrt_rn(fmaf(m, m, 1.f));
    r.stepz = (v >= 0.f) ? 1 : -1;  // v == 0: never crosses a z plane (inv_mz = +inf)
    return r;
}

// s at which the ray leaves voxel layer iz in its direction of travel
__device__ __forceinline__ float z_exit(int iz, const LaneRay &r, float halfnz)
{
    const float kc = (float)(iz + (r.stepz > 0)) - halfnz;  // centred plane coordinate
    return (kc - r.zE) * r.inv_mz;
}

// s at which the column leaves voxel ix (or iy) in its direction of travel
__device__ __forceinline__ float xy_exit(int i, int step, float e, float inv)
{
    return ((float)(i + (step > 0)) - e) * inv;
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

template <int MODE, bool NORM>
__global__ void __launch_bounds__(256)
fwd_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float *__restrict__ vrow,
           const float *__restrict__ vol, float *__restrict__ out, const float *__restrict__ b,
           double *__restrict__ partials, int *__restrict__ nonfinite)
{
    int j, iu, iv;
    decode_block(G, j, iu, iv);
    const bool col_ok = iu < G.nu;
    const bool ray_ok = col_ok && iv < G.nv;
    float acc = 0.f, sec = 1.f;

    if (col_ok) {
        const ColParams cp = cols[(long long)j * G.nu + iu];
        if (cp.L > 0.f) {
            const float v = ray_ok ? __ldg(vrow + iv) : 0.f;
            const LaneRay r = lane_ray(cp, v);
            sec = r.sec;
            int iz = __float2int_rd(r.zE + G.halfnz);
            bool act = ray_ok && iz >= 0 && iz < G.nz;
            // the FP32 layer index can disagree with the sign of a tiny z offset:
            // a first crossing "behind" the entry is taken at the entry
            float szn = fmaxf(z_exit(iz, r, G.halfnz), 0.f);

            int ix = cp.ix0, iy = cp.iy0;
            float sxn = xy_exit(ix, cp.stepx, cp.ex, cp.inv_dx);
            float syn = xy_exit(iy, cp.stepy, cp.ey, cp.inv_dy);
            int colbase = (ix * G.ny + iy) * G.nz;
            const int dcx = cp.stepx * G.ny * G.nz, dcy = cp.stepy * G.nz;
            float s = 0.f;
            if (__any_sync(kFull, act)) {
                for (;;) {
                    const float se = fminf(fminf(sxn, syn), cp.L);
                    if (act) {
                        float sl = s;
                        while (szn < se) {
                            acc = fmaf(szn - sl, __ldg(vol + colbase + iz), acc);
                            sl = szn;
                            iz += r.stepz;
                            if ((unsigned)iz >= (unsigned)G.nz) { act = false; break; }
                            szn = z_exit(iz, r, G.halfnz);
                        }
                        if (act) acc = fmaf(se - sl, __ldg(vol + colbase + iz), acc);
                    }
                    if (se >= cp.L) break;
                    if (sxn <= syn) {
                        ix += cp.stepx;
                        if ((unsigned)ix >= (unsigned)G.nx) break;
                        colbase += dcx;
                        sxn = xy_exit(ix, cp.stepx, cp.ex, cp.inv_dx);
                    } else {
                        iy += cp.stepy;
                        if ((unsigned)iy >= (unsigned)G.ny) break;
                        colbase += dcy;
                        syn = xy_exit(iy, cp.stepy, cp.ey, cp.inv_dy);
                    }
                    s = se;
                    if (!__any_sync(kFull, act)) break;
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

// Adjoint: every lane scatters w * len into the voxels its ray crosses.  Per
// xy cell the warp's contributions land in one voxel column within a short z
// range; they are summed in a per-warp shared-memory window (shared atomics
// resolve the lanes that hit the same voxel) and flushed with one 16-byte
// vector reduction per group of four voxels.
template <bool VEC>
__global__ void __launch_bounds__(256)
adj_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float *__restrict__ vrow,
           const float *__restrict__ proj, float *__restrict__ vol)
{
    __shared__ float4 win4[kWarps][kWin / 4];
    int j, iu, iv;
    decode_block(G, j, iu, iv);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *mywin4 = win4[warp];
    float *mywin = reinterpret_cast<float *>(mywin4);
    mywin4[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    if (iu >= G.nu) return;  // warp-uniform; no CTA-wide barrier follows
    const ColParams cp = cols[(long long)j * G.nu + iu];
    if (!(cp.L > 0.f)) return;
    const bool ray_ok = iv < G.nv;
    const float v = ray_ok ? __ldg(vrow + iv) : 0.f;
    const LaneRay r = lane_ray(cp, v);
    float w = 0.f;
    if (ray_ok)
        w = proj[(long long)j * G.sj + (long long)iu * G.su + (long long)iv * G.sv] * r.sec;
    int iz = __float2int_rd(r.zE + G.halfnz);
    bool act = ray_ok && w != 0.f && iz >= 0 && iz < G.nz;
    if (!__any_sync(kFull, act)) return;
    float szn = fmaxf(z_exit(iz, r, G.halfnz), 0.f);

    int ix = cp.ix0, iy = cp.iy0;
    float sxn = xy_exit(ix, cp.stepx, cp.ex, cp.inv_dx);
    float syn = xy_exit(iy, cp.stepy, cp.ey, cp.inv_dy);
    int colbase = (ix * G.ny + iy) * G.nz;
    const int dcx = cp.stepx * G.ny * G.nz, dcy = cp.stepy * G.nz;
    float s = 0.f;
    for (;;) {
        const float se = fminf(fminf(sxn, syn), cp.L);
        const int izmin = __reduce_min_sync(kFull, act ? iz : 0x7fffffff);
        if (izmin == 0x7fffffff) break;  // every lane has left the volume
        const int z0 = (izmin & ~3) - 4;
        if (act) {
            float sl = s;
            for (;;) {
                const bool cross = szn < se;
                const float seg = (cross ? szn : se) - sl;
                const int k = iz - z0;
                if ((unsigned)k < (unsigned)kWin) atomicAdd(mywin + k, seg * w);
                else atomicAdd(vol + colbase + iz, seg * w);
                if (!cross) break;
                sl = szn;
                iz += r.stepz;
                if ((unsigned)iz >= (unsigned)G.nz) { act = false; break; }
                szn = z_exit(iz, r, G.halfnz);
            }
        }
        __syncwarp();
        const float4 c4 = mywin4[lane];
        if (c4.x != 0.f || c4.y != 0.f || c4.z != 0.f || c4.w != 0.f) {
            const int zs = z0 + 4 * lane;
            float *dst = vol + colbase + zs;
            if (VEC && zs >= 0 && zs + 3 < G.nz) {
                atomicAdd(reinterpret_cast<float4 *>(dst), c4);
            } else {
                if (c4.x != 0.f && zs + 0 >= 0 && zs + 0 < G.nz) atomicAdd(dst + 0, c4.x);
                if (c4.y != 0.f && zs + 1 >= 0 && zs + 1 < G.nz) atomicAdd(dst + 1, c4.y);
                if (c4.z != 0.f && zs + 2 >= 0 && zs + 2 < G.nz) atomicAdd(dst + 2, c4.z);
                if (c4.w != 0.f && zs + 3 >= 0 && zs + 3 < G.nz) atomicAdd(dst + 3, c4.w);
            }
            mywin4[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        if (se >= cp.L) break;
        if (sxn <= syn) {
            ix += cp.stepx;
            if ((unsigned)ix >= (unsigned)G.nx) break;
            colbase += dcx;
            sxn = xy_exit(ix, cp.stepx, cp.ex, cp.inv_dx);
        } else {
            iy += cp.stepy;
            if ((unsigned)iy >= (unsigned)G.ny) break;
            colbase += dcy;
            syn = xy_exit(iy, cp.stepy, cp.ey, cp.inv_dy);
        }
        s = se;
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
                           const float *vol, float *out, int mode, const float *b,
                           double *partials, int *nonfinite, cudaStream_t st)
{
    const int nb = project_blocks(g);
    if (nb <= 0) return cudaSuccess;
    if (mode == FWD_RESID) {
        if (partials)
            fwd_kernel<FWD_RESID, true><<<nb, 256, 0, st>>>(g, cols, vrow, vol, out, b, partials,
                                                            nonfinite);
        else
            fwd_kernel<FWD_RESID, false><<<nb, 256, 0, st>>>(g, cols, vrow, vol, out, b, partials,
                                                             nonfinite);
    } else {
        if (partials)
            fwd_kernel<FWD_PLAIN, true><<<nb, 256, 0, st>>>(g, cols, vrow, vol, out, b, partials,
                                                            nonfinite);
        else
            fwd_kernel<FWD_PLAIN, false><<<nb, 256, 0, st>>>(g, cols, vrow, vol, out, b, partials,
                                                             nonfinite);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const ProjGeom &g, const ColParams *cols, const float *vrow,
                           const float *proj, float *vol, cudaStream_t st)
{
    const int nb = project_blocks(g);
    if (nb <= 0) return cudaSuccess;
    const bool vec = (g.nz % 4 == 0) && ((reinterpret_cast<uintptr_t>(vol) & 15u) == 0);
    if (vec)
        adj_kernel<true><<<nb, 256, 0, st>>>(g, cols, vrow, proj, vol);
    else
        adj_kernel<false><<<nb, 256, 0, st>>>(g, cols, vrow, proj, vol);
    return cudaGetLastError();
}

}  // namespace piccs
