// Cone-beam projector A and its matched adjoint A^T for sm_103a.
//
// A_ij is the length (mm) of ray i inside voxel j (the linear model of
// Sec. 2.1, Eq. 1, with exact ray/voxel intersection lengths).  Krylov
// methods need one product with A and one with A^T per iteration (Sec. 2.3,
// the text after the augmented system), so these two kernels carry nearly all
// of the bytes of a reconstruction.
//
// Layout of the work: one thread = one pair of mirror rows (below), one warp =
// 32 consecutive pairs of one detector column of one view, one CTA = 8 such
// warps of the same column (512 rows), so the column's cell list is fetched
// from DRAM once per CTA.  Because the detector v
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
// The adjoint is a gather over the transpose of the same tables: one CTA per
// xy voxel column, one thread per two pairs of mirror layers, visits every
// detector column that crosses its voxel column and, for the two or three rows
// whose rays cross each of its z layers there, adds piece length x ray value
// -- no atomics, one store per voxel, deterministic.  Both kernels evaluate the same piece lengths
//   len = min(s_exit_xy, s_z(exit plane)) - max(s_enter_xy, s_z(entry plane))
// from the same FP32 cell boundaries and the same plane-crossing formula
// fma(kc, KD / v, -s0), with the exact plane coordinate kc (never an
// accumulated distance), so A^T applies bit-identical weights to A; only the
// order of the FP32 sums differs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "internal.h"

namespace piccs {

namespace {

// Gather shape: threads per CTA, layer pairs per thread, and the CTAs per SM
// the register allocation must allow (compile-time, for tuning sweeps).
#ifndef PICCS_GATHER_THREADS
#define PICCS_GATHER_THREADS 64
#endif
#ifndef PICCS_GATHER_LAYERS
#define PICCS_GATHER_LAYERS 2
#endif
#ifndef PICCS_GATHER_MIN_CTAS
#define PICCS_GATHER_MIN_CTAS 32
#endif

constexpr int kRowGroups = 8;    // warps per forward CTA: 8 x 32 row pairs of one column
constexpr int kGatherThreads = PICCS_GATHER_THREADS;
constexpr int kLayersPerThread = PICCS_GATHER_LAYERS;  // layer pairs per gather thread
constexpr unsigned kFull = 0xffffffffu;

// forward walks (walk_pair): one crossing step per cell, repeated steps, and
// one step with the cell table read one entry ahead
constexpr int kWalkOne = 0, kWalkMulti = 1, kWalkAhead = 2;
inline int walk_of(const ProjGeom &g) { return g.multi ? kWalkMulti : g.ahead ? kWalkAhead : kWalkOne; }

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

// The geometry is symmetric about the plane z = 0 (source in it, detector and
// volume centred on it): detector rows iv and nv-1-iv have heights v and -v
// exactly (also in FP32), and their rays are mirror images.  With
// s(kc) = fma(kc, KD/v, -s0), the ray at -v crosses plane -kc at the same s
// as the ray at v crosses plane kc, bit for bit, and it is in layer nz-1-k
// whenever the ray at v is in layer k.  Both kernels therefore work on
// mirror pairs: the forward walks the pair with one shared z state, the
// gather evaluates each piece length once for a layer and its mirror.

// Rows of pair p: the upper row nv-1-p (v >= 0, walked upwards) and the lower
// row p (its mirror; absent when both are the middle row of an odd nv).
__device__ __forceinline__ int npairs_rows(int nv) { return (nv + 1) >> 1; }

// CTA b = one detector column (j, iu) and kRowGroups x 32 row pairs
__device__ __forceinline__ void decode_block(const ProjGeom &G, int b, int &col, int &p)
{
    const int np = npairs_rows(G.nv);
    const int nrgb = (np + 32 * kRowGroups - 1) / (32 * kRowGroups);
    col = b / nrgb;
    p = ((b - col * nrgb) * kRowGroups + (threadIdx.x >> 5)) * 32 + (threadIdx.x & 31);
}

// Walk of one mirror pair of rows (heights v >= 0 and -v) along the
// column's cell list; acca / accb get the upper / lower ray's sum of
// piece length (xy mm) x voxel value.  Every lane takes one piece per cell,
// [s, min(next crossing, se)] in its current layer, with its length clamped
// at 0 so that a ray that has left the volume (or never entered it) adds
// exactly nothing; the z crossings inside a cell are then taken as one
// warp-uniform step, predicated per lane, and only when some lane crosses.
// When the host has shown that a cell holds at most one crossing of any row
// (the xy distance between consecutive z planes of the steepest ray, vz D /
// v_max, exceeds the longest cell), one such step per cell suffices;
// kWalkMulti repeats it until no lane crosses any more.  kWalkAhead is the
// one-step walk with the next cell-table entry loaded one iteration early, for
// volumes larger than the L2, where that load misses (512^3 forward 35.1 ->
// 32.8 ms; 3.84 -> 4.05 ms at 256^3, where it hits).  The piece lengths are the
// expressions the adjoint's gather evaluates, bit for bit, in every walk.
template <int WALK>
__device__ __forceinline__ void walk_pair(const ProjGeom &G, const ColParams &cp,
                                          const int4 *__restrict__ cells,
                                          const float *__restrict__ vol, float2 w, bool pair_ok,
                                          float &acca, float &accb)
{
    const float inv = cp.KD * w.y;  // xy distance per voxel of z (> 0)
    const int nzm1 = G.nz - 1;
    int iz = __float2int_rd(w.x * (cp.s0 * cp.rKD) + G.halfnz);
    const bool act = pair_ok && iz >= 0 && iz < G.nz;
    // centred coordinate of the plane the upper ray leaves layer iz through,
    // and the xy distance at which it does; the FP32 layer index can disagree
    // with the sign of a tiny z offset: a first crossing "behind" the entry
    // is taken at the entry
    float kce = (float)(iz + 1) - G.halfnz;
    float szn = fmaxf(fmaf(kce, inv, -cp.s0), 0.f);
    if (!act) {  // in the top layer with its "exit" behind it: adds 0, never crosses
        iz = nzm1;
        szn = -1.f;
    }
    if (!__any_sync(kFull, act)) return;
    const int4 *t = cells + cp.start2;
    const int n2 = (cp.ncells + 1) >> 1;
    // the lower ray's layer, kept beside iz rather than formed as nzm1 - iz
    // at every load (256^3 forward 4.67 -> 3.84 ms, the same code otherwise)
    int izm = nzm1 - iz;
    float s = 0.f;
    auto cell = [&](int colbase, float se) {
        const float *cpv = vol + colbase;
        const float len = fmaxf(fminf(szn, se) - s, 0.f);
        acca = fmaf(len, __ldg(cpv + iz), acca);
        accb = fmaf(len, __ldg(cpv + izm), accb);
        do {
            const bool up = szn < se && iz < nzm1;
            if (!__any_sync(kFull, up)) break;
            const float kn = kce + 1.f;
            const float sn = fmaf(kn, inv, -cp.s0);
            const float l2 = up ? fminf(sn, se) - szn : 0.f;
            if (up) {
                ++iz;
                --izm;
                kce = kn;
                szn = sn;
            }
            acca = fmaf(l2, __ldg(cpv + iz), acca);
            accb = fmaf(l2, __ldg(cpv + izm), accb);
        } while (WALK == kWalkMulti);
        s = se;
    };
    int4 en = WALK == kWalkAhead ? __ldg(t) : make_int4(0, 0, 0, 0);  // n2 >= 1
    for (int c = 0; c < n2; ++c) {
        int4 e;
        if (WALK == kWalkAhead) {
            e = en;
            if (c + 1 < n2) en = __ldg(t + c + 1);
        } else {
            e = __ldg(t + c);
        }
        cell(e.x, __int_as_float(e.y));
        cell(e.z, __int_as_float(e.w));
        // every lane has left the volume through a z face
        if ((c & 1) && !__any_sync(kFull, iz < nzm1 || szn >= s)) break;
    }
}

// 8 CTAs of 256 threads per SM (32 registers): the walk's gathers need the
// full occupancy to hide their latency once the volume no longer fits in L2
// One CTA (block blk of one scan) of the forward; the buffers are the scan's.
template <int MODE, bool NORM, int WALK>
__device__ __forceinline__ void fwd_block(const ProjGeom &G, const ColParams *__restrict__ cols,
                                          const float2 *__restrict__ vr,
                                          const int4 *__restrict__ cells,
                                          const float *__restrict__ vol, float *__restrict__ out,
                                          const float *__restrict__ aux,
                                          double *__restrict__ partials,
                                          int *__restrict__ nonfinite, float *__restrict__ ra,
                                          float *__restrict__ aw, int blk)
{
    if (MODE == FWD_LSQR && aux[2] != 0.f) return;  // the Krylov cycle has stopped
    __shared__ double red[kRowGroups];  // NORM: the warps' partial sums
    __shared__ unsigned warps_done;
    if (NORM) {
        if (threadIdx.x == 0) warps_done = 0;
        __syncthreads();  // before any warp can finish
    }
    int col, p;
    decode_block(G, blk, col, p);
    const bool pair_ok = p < npairs_rows(G.nv);
    const int iva = G.nv - 1 - p;               // upper row (v >= 0)
    const bool has_b = pair_ok && p != iva;     // lower mirror row p
    float acca = 0.f, accb = 0.f, sec = 1.f;
    const ColParams cp = cols[col];
    if (cp.ncells > 0) {
        const float2 w = pair_ok ? __ldg(vr + iva) : make_float2(0.f, 1e30f);
        sec = ray_sec(w.x, cp.invD);
        walk_pair<WALK>(G, cp, cells, vol, w, pair_ok, acca, accb);
    }

    float sq = 0.f;
    if (pair_ok) {
        const int j = col / G.nu, iu = col - j * G.nu;
        const long long base = (long long)j * G.sj + (long long)iu * G.su;
        const long long ia = base + (long long)iva * G.sv, ib = base + (long long)p * G.sv;
        float qa = sec * acca, qb = sec * accb;
        if (MODE == FWD_RESID || MODE == FWD_RESID16) {
            float ba, bb;
            if (MODE == FWD_RESID) {
                ba = aux[ia];
                bb = has_b ? aux[ib] : 0.f;
            } else {
                const __nv_bfloat16 *b16 = reinterpret_cast<const __nv_bfloat16 *>(aux);
                ba = __bfloat162float(b16[ia]);
                bb = has_b ? __bfloat162float(b16[ib]) : 0.f;
            }
            if (!isfinite(ba) || !isfinite(bb)) atomicOr(nonfinite, 1);
            qa = ba - qa;
            qb = bb - qb;
        } else if (MODE == FWD_LSQR) {
            // u-step, and A w = A v - (theta/rho) A w kept beside it so that the
            // deferred x step can be applied to the data residual rA
            const float ka = aux[0], kb = aux[1], tw = aux[3], pend = aux[4];
            const bool first = aux[5] != 0.f;
            const float sa = ka * qa, sb = ka * qb;
            qa = fmaf(-kb, out[ia], sa);
            if (first) {
                aw[ia] = sa;
            } else {
                const float wa = aw[ia];
                ra[ia] = fmaf(-pend, wa, ra[ia]);
                aw[ia] = fmaf(-tw, wa, sa);
            }
            qb = 0.f;
            if (has_b) {
                qb = fmaf(-kb, out[ib], sb);
                if (first) {
                    aw[ib] = sb;
                } else {
                    const float wb = aw[ib];
                    ra[ib] = fmaf(-pend, wb, ra[ib]);
                    aw[ib] = fmaf(-tw, wb, sb);
                }
            }
        }
        out[ia] = qa;
        if (has_b) out[ib] = qb;
        sq = qa * qa + (has_b ? qb * qb : 0.f);
    }
    if (NORM) {
        // The warps of a CTA finish their walks at different times (steep rows
        // leave through a z face early).  Instead of a barrier, each warp leaves
        // its partial in shared memory and the last one to finish sums the
        // eight in warp order: the same sum, and no warp waits for the slowest
        // (a barrier here cost 22 % at 512^3, where the gathers miss L2).
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = (double)sq;
            __threadfence_block();
            if (atomicAdd(&warps_done, 1u) == kRowGroups - 1) {
                __threadfence_block();
                const volatile double *rv = red;
                double t = 0.0;
#pragma unroll
                for (int w = 0; w < kRowGroups; ++w) t += rv[w];
                partials[blk] = t;
            }
        }
    }
}

// One scan, or the scans of a batch (slot blockIdx.y, buffers sstride bytes apart)
template <int MODE, bool NORM, int WALK>
__global__ void __launch_bounds__(256, 8)
fwd_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
           const int4 *__restrict__ cells, const float *__restrict__ vol,
           float *__restrict__ out, const float *__restrict__ aux, double *__restrict__ partials,
           int *__restrict__ nonfinite, float *__restrict__ ra, float *__restrict__ aw,
           long long sstride)
{
    const long long so = blockIdx.y * sstride;
    fwd_block<MODE, NORM, WALK>(G, cols, vr, cells, slot_ptr(vol, so), slot_ptr(out, so),
                                 slot_ptr(aux, so), slot_ptr(partials, so),
                                 slot_ptr(nonfinite, so), slot_ptr(ra, so), slot_ptr(aw, so),
                                 blockIdx.x);
}

// Scans of different geometries in one grid: the jobs' blocks one after
// another (job m: slots x blocks per slot from block b0); each CTA finds its
// job and runs the same block as the single-scan kernel, so every scan's
// result is bit for bit its standalone result.
__device__ __forceinline__ int find_job(int b, const int *b0, int n)
{
    int m = 0;
    while (m + 1 < n && b >= b0[m + 1]) ++m;
    return m;
}

template <int MODE, bool NORM, int WALK>
__global__ void __launch_bounds__(256, 8) fwd_group_kernel(const FwdGroup grp)
{
    const int m = find_job(blockIdx.x, grp.b0, grp.n);
    const FwdJob &J = grp.job[m];
    const int local = blockIdx.x - grp.b0[m];
    const int slot = local / J.nb;
    const long long so = slot * J.sstride;
    fwd_block<MODE, NORM, WALK>(J.g, J.cols, J.vr, J.cells, slot_ptr(J.vol, so),
                                 slot_ptr(J.out, so), slot_ptr(J.aux, so), slot_ptr(J.partials, so),
                                 slot_ptr(J.nonfinite, so), slot_ptr(J.ra, so), slot_ptr(J.aw, so),
                                 local - slot * J.nb);
}

// rs = proj * sec, per ray (the adjoint's gather then needs no square root).
// PAIRS (even nv): stored per detector column as mirror-row pairs,
// rs2[col h + m] = {rs of row h + m, rs of row h - 1 - m} (h = nv / 2), so that
// the gather fetches a row and its mirror with one 8-byte load; else in the
// projection layout.
template <bool PAIRS>
__global__ void __launch_bounds__(256)
scale_rays_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
                  const float *__restrict__ proj, float *__restrict__ rs, long long sstride)
{
    proj = slot_ptr(proj, blockIdx.y * sstride);
    rs = slot_ptr(rs, blockIdx.y * sstride);
    int col, p;
    decode_block(G, blockIdx.x, col, p);
    if (p >= npairs_rows(G.nv)) return;
    const int j = col / G.nu, iu = col - j * G.nu;
    const long long base = (long long)j * G.sj + (long long)iu * G.su;
    const int iva = G.nv - 1 - p;
    const float sec = ray_sec(__ldg(vr + iva).x, cols[col].invD);  // same for the mirror row
    const long long ia = base + (long long)iva * G.sv, ib = base + (long long)p * G.sv;
    if (PAIRS) {
        const int h = G.nv >> 1;
        reinterpret_cast<float2 *>(rs)[(long long)col * h + (h - 1 - p)] =
            make_float2(proj[ia] * sec, proj[ib] * sec);
    } else {
        rs[ia] = proj[ia] * sec;
        if (p != iva) rs[ib] = proj[ib] * sec;
    }
}

// Adjoint gather: CTA = one xy voxel column (ix, iy), thread = kLayersPerThread
// mirror pairs of z layers (upper layer ku = nz-1-p, lower layer p).  For every
// crossing (view j, detector column iu, xy interval [sa, sb]) of the voxel
// column, the rows whose rays pass through layer ku inside [sa, sb] form a
// short interval of heights v (ray z = v * (s0 + s) * rKD, so
// v in [zl, zh] / ((s0 + s) rKD)); each candidate row r is checked with the
// exact piece length -- the expression the forward walk evaluates -- which is
// also the length of row nv-1-r in layer p.
// EVEN (even nv and nz): no row has v = 0 and no layer straddles z = 0, so
// every upper layer is crossed by the upper rows only (iv >= nv / 2), upwards;
// the ray values are read as mirror-row pairs (scale_rays_kernel<true>).
// One CTA: xy voxel column `cell`, layer-pair chunk `chunk`, of one scan.
template <bool EVEN>
__device__ __forceinline__ void adj_gather_block(const ProjGeom &G, const ColParams *__restrict__ cols,
                                                 const float2 *__restrict__ vr,
                                                 const int *__restrict__ hit_ptr,
                                                 const CellHit *__restrict__ hits,
                                                 const float *__restrict__ rs,
                                                 float *__restrict__ vol, int cell, int chunk)
{
    constexpr int L = kLayersPerThread;
    const int pb = chunk * kGatherThreads * L + threadIdx.x;
    const int nlp = (G.nz + 1) >> 1;  // layer pairs (the middle layer of an odd nz pairs with itself)
    float zlo[L], accu[L], accd[L];
    bool pok[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        const int p = pb + q * kGatherThreads;
        pok[q] = p < nlp;
        // lower plane of the upper layer (>= -0.5); a thread beyond the last
        // pair gets a plane far above every ray, which puts its lower candidate
        // bound above every row (its sums are not written in any case)
        zlo[q] = pok[q] ? (float)(G.nz - 1 - p) - G.halfnz : 1e20f;
        accu[q] = 0.f;
        accd[q] = 0.f;
    }
    const int nvm1 = G.nv - 1;
    const int h0 = __ldg(hit_ptr + cell), h1 = __ldg(hit_ptr + cell + 1);
    // The crossing constants are the same for every thread of the CTA: each
    // chunk of kGatherThreads crossings is prepared once, one per thread, in
    // shared memory ({sa, sb, s0, KD} and {1/G(sa), 1/G(sb), ray offset}).
    __shared__ float4 hc_a[kGatherThreads], hc_b[kGatherThreads];
    for (int hb = h0; hb < h1; hb += kGatherThreads) {
        const int nh = min(kGatherThreads, h1 - hb);
        __syncthreads();  // the previous chunk has been read
        if ((int)threadIdx.x < nh) {
            const CellHit e = __ldg(hits + hb + threadIdx.x);
            const int j = e.x >> 16, iu = e.x & 0xffff;
            const float sa = __int_as_float(e.y), sb = __int_as_float(e.z);
            const float4 cz = __ldg(reinterpret_cast<const float4 *>(cols + (long long)j * G.nu + iu) + 1);
            const float s0 = cz.x, KD = cz.y, rKD = cz.w;
            // detector rows per unit of plane coordinate at sa and at sb,
            // 1 / (G(s) dv): candidate bounds only (rounded as often as
            // zl / G(s) / dv would be, well inside the 1e-3-row margin up to
            // thousands of rows), the rows are then checked exactly
            const float rGa = rcp_approx((s0 + sa) * rKD) * G.rdv;
            const float rGb = rcp_approx((s0 + sb) * rKD) * G.rdv;
            const int roff = EVEN ? (j * G.nu + iu) * (G.nv >> 1)  // pair index of row nv / 2
                                  : (int)((long long)j * G.sj + (long long)iu * G.su);  // N < 2^31
            hc_a[threadIdx.x] = make_float4(sa, sb, s0, KD);
            hc_b[threadIdx.x] = make_float4(rGa, rGb, __int_as_float(roff), 0.f);
        }
        __syncthreads();
        for (int k = 0; k < nh; ++k) {
            const float4 ca = hc_a[k], cb = hc_b[k];
            const float sa = ca.x, sb = ca.y, s0 = ca.z, KD = ca.w;
            const float rGa = cb.x, rGb = cb.y;
            const float *rsc = rs + __float_as_int(cb.z);
            const float *rsm = rsc + nvm1 * G.sv32;  // row nv-1-iv at rsm - iv * sv
            // EVEN: pair of rows iv and nv-1-iv at rp[iv]
            const float2 *rp = reinterpret_cast<const float2 *>(rs) + __float_as_int(cb.z) - (G.nv >> 1);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                const float zl = zlo[q], zh = zl + 1.f;
                // G grows with s, so 1/G(sa) >= 1/G(sb); upper layers have zl >= 0
                // except the middle layer of an odd nz (zl = -0.5)
                // Candidate rows ilo .. ihi, held in 0 (EVEN: nv / 2) .. nv - 1
                // whatever the bounds' values: the conversions saturate, and ilo
                // is clamped to nv at most, so that ilo + 3 cannot overflow.
                const int ilo = min(max(__float2int_ru(fmaf(zl, EVEN || zl >= 0.f ? rGb : rGa,
                                                            G.cv - 1e-3f)),
                                        EVEN ? (G.nv >> 1) : 0),
                                    G.nv);
                const int ihi = min(__float2int_rd(fmaf(zh, rGa, G.cv + 1e-3f)), nvm1);
                // only a layer touching z = 0 can hold the middle row of an odd nv
                // (v = 0), which is its own mirror and belongs to the upper layer
                const bool mid = zl < 1.f && (nvm1 & 1) == 0;
                // ORDERED: the layer lies above z = 0 (zl >= 0), so every
                // candidate row has v >= 0, 1/v > 0 and enters the layer's lower
                // plane before its upper one (xl <= xh, FP32 rounding is monotone)
                auto rows = [&](auto ordered) {
                    auto cand = [&](int iv) {
                        const float inv = KD * __ldg(vr + iv).y;
                        const float xl = fmaf(zl, inv, -s0), xh = fmaf(zh, inv, -s0);
                        // the ray is inside the layer between its two plane crossings
                        const float len = decltype(ordered)::value
                                              ? fminf(sb, xh) - fmaxf(sa, xl)
                                              : fminf(sb, fmaxf(xl, xh)) - fmaxf(sa, fminf(xl, xh));
                        if (len > 0.f) {
                            if (EVEN) {
                                const float2 r2 = __ldg(rp + iv);
                                accu[q] = fmaf(len, r2.x, accu[q]);
                                accd[q] = fmaf(len, r2.y, accd[q]);
                            } else {
                                accu[q] = fmaf(len, __ldg(rsc + iv * G.sv32), accu[q]);
                                if (!mid || 2 * iv != nvm1)
                                    accd[q] = fmaf(len, __ldg(rsm - iv * G.sv32), accd[q]);
                            }
                        }
                    };
                    if (ilo <= ihi) cand(ilo);
                    if (ilo + 1 <= ihi) cand(ilo + 1);
                    if (ilo + 2 <= ihi) cand(ilo + 2);
                    for (int iv = ilo + 3; iv <= ihi; ++iv) cand(iv);
                };
                if (EVEN || zl >= 0.f)
                    rows(std::true_type{});
                else
                    rows(std::false_type{});
            }
        }
    }
    float *colv = vol + (long long)cell * G.nz;
#pragma unroll
    for (int q = 0; q < L; ++q) {
        if (!pok[q]) continue;
        const int p = pb + q * kGatherThreads, ku = G.nz - 1 - p;
        colv[ku] += accu[q];
        if (p != ku) colv[p] += accd[q];
    }
}

// grid: voxel columns x layer-pair chunks x slots
template <bool EVEN>
__global__ void __launch_bounds__(kGatherThreads, PICCS_GATHER_MIN_CTAS)
adj_gather_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
                  const int *__restrict__ hit_ptr, const CellHit *__restrict__ hits,
                  const float *__restrict__ rs, float *__restrict__ vol, long long sstride)
{
    const long long so = blockIdx.z * sstride;
    adj_gather_block<EVEN>(G, cols, vr, hit_ptr, hits, slot_ptr(rs, so), slot_ptr(vol, so),
                           blockIdx.x, blockIdx.y);
}

// scans of different geometries in one grid (see fwd_group_kernel); job m's
// blocks are slots x chunks x voxel columns, voxel columns fastest
template <bool EVEN>
__global__ void __launch_bounds__(kGatherThreads, PICCS_GATHER_MIN_CTAS)
adj_gather_group_kernel(const AdjGroup grp)
{
    const int m = find_job(blockIdx.x, grp.b0, grp.n);
    const AdjJob &J = grp.job[m];
    const int local = blockIdx.x - grp.b0[m];
    const int ncell = J.g.nx * J.g.ny, per_slot = J.nb;
    const int slot = local / per_slot, rem = local - slot * per_slot;
    const int chunk = rem / ncell;
    const long long so = slot * J.sstride;
    adj_gather_block<EVEN>(J.g, J.cols, J.vr, J.hit_ptr, J.hits, slot_ptr(J.rs, so),
                           slot_ptr(J.vol, so), rem - chunk * ncell, chunk);
}

// ---------------------------------------------------------------------------
// Adjoint for geometries with an even number of detector rows and of z
// layers and at most one z crossing of any row per xy cell (the usual case;
// the gather above serves the rest).
//
// For one crossing [sa, sb] of a voxel column and one upper layer k (planes
// p = k and p + 1, centred coordinates >= 0), the rows of the detector
// column split into three contiguous sets, because a row's crossing
// distance x_i(p) = fma(p, KD / v_i, -s0) falls as its height v_i grows:
//   * interior rows, inside the layer over the whole of [sa, sb]: piece
//     length sb - sa, the same for all of them;
//   * rows entering through plane p inside the interval: length sb - x_i(p);
//   * rows leaving through plane p + 1 inside the interval: x_i(p + 1) - sa.
// With the thresholds Ta(p) = first row with x_i(p) <= sa and Tb(p) = first
// row with x_i(p) < sb, the interior rows of layer k are [Ta(k), Tb(k + 1))
// and the boundary rows of plane p are [Tb(p), Ta(p)) -- usually none or one.
// The interior sum is one difference of per-column prefix sums of the scaled
// ray values; only the boundary rows are evaluated one by one.  The lengths
// are the FP32 expressions the forward walk evaluates (a crossing exactly at
// sb belongs to the next cell, as in the walk); only the grouping of the FP32
// sums differs.
//
// Prefix sums: per detector column, over the upper rows h .. nv-1 (h = nv/2,
// heights v > 0) counted outwards from the middle, with the mirror row
// nv-1-i beside row i: pq[c (h + 1) + m] = {sum_{i<h+m} rs_i, sum of the
// mirror rows}, rs = r sec gamma.  Starting at the middle keeps the sums as
// small as half a column.

// one warp per detector column, 32 rows per step
__global__ void __launch_bounds__(256)
ray_prefix_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
                  const float *__restrict__ proj, float2 *__restrict__ pq, long long sstride)
{
    proj = slot_ptr(proj, blockIdx.y * sstride);
    pq = slot_ptr(pq, blockIdx.y * sstride);
    const int col = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (col >= G.n_views * G.nu) return;  // whole warps
    const int h = G.nv >> 1;
    const int j = col / G.nu, iu = col - j * G.nu;
    const long long base = (long long)j * G.sj + (long long)iu * G.su;
    const float invD = cols[col].invD;
    float2 *out = pq + (long long)col * (h + 1);
    float cu = 0.f, cd = 0.f;  // sums of the rows before this step
    for (int m0 = 0; m0 < h; m0 += 32) {
        const int m = m0 + lane;
        float ru = 0.f, rd = 0.f;
        if (m < h) {
            const int iv = h + m;
            const float sec = ray_sec(__ldg(vr + iv).x, invD);
            ru = proj[base + (long long)iv * G.sv] * sec;
            rd = proj[base + (long long)(G.nv - 1 - iv) * G.sv] * sec;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {  // inclusive scan over the lanes
            const float tu = __shfl_up_sync(kFull, ru, o), td = __shfl_up_sync(kFull, rd, o);
            if (lane >= o) {
                ru += tu;
                rd += td;
            }
        }
        if (m < h) out[m + 1] = make_float2(cu + ru, cd + rd);
        cu += __shfl_sync(kFull, ru, 31);
        cd += __shfl_sync(kFull, rd, 31);
    }
    if (lane == 0) out[0] = make_float2(0.f, 0.f);
}

// Row threshold of plane kc at xy distance s: the first row i >= h whose
// crossing x_i = fma(kc, KD / v_i, -s0) is <= s (LE) or < s (!LE), or nv.
// The estimate e = kc KD / ((s0 + s) dv) + cv places the exact crossing in
// row units to a few 1e-4 rows (FP32 rounding of the table values and the
// approximate reciprocal), so ceil(e - d) and ceil(e + d) with d = 1e-2
// bracket the threshold: equal, it is known; one apart, the row ceil(e - d)
// decides.  ceil(y) is taken as y + 0.5 rounded to the nearest integer on the
// FMA pipe (adding 1.5 * 2^23); y is clamped to nv first.  At an exact
// integer y this may give ceil(y) + 1, which still brackets the threshold,
// and the upper bound is held to the lower one + 1.
constexpr int kPrefixWarps = 4;  // voxel columns (one warp each) per CTA
constexpr int kPrefixMaxR = 8;   // layers per lane: nz <= 2 * 32 * 8
constexpr float kRowSlack = 1e-2f;
constexpr float kRoundMagic = 12582912.f;  // 1.5 * 2^23
constexpr int kRoundMagicBits = 0x4B400000;

template <bool LE>
__device__ __forceinline__ int row_threshold(float kc, float rgr, float s, float s0, float KD,
                                             const float2 *__restrict__ vr, float cvlo, float cvhi,
                                             float fnv, int nv)
{
    const float ylo = fminf(fmaf(kc, rgr, cvlo), fnv), yhi = fminf(fmaf(kc, rgr, cvhi), fnv);
    int m = __float_as_int(ylo + kRoundMagic) - kRoundMagicBits;
    const int m2 = min(__float_as_int(yhi + kRoundMagic) - kRoundMagicBits, m + 1);
    if (__any_sync(kFull, m != m2)) {
        if (m != m2) {  // m < m2 <= nv: row m is a real row
            const float x = fmaf(kc, KD * __ldg(vr + m).y, -s0);
            if (!(LE ? x <= s : x < s)) m = m2;
        }
    }
    return m;
}

// Per crossing: the constants of the crossing and the running state of one
// lane (its accumulators and the prefix at Ta of the plane below).
struct PrefixCrossing {
    float sa, sb, s0, KD, rga, rgb, len0, kc0;
    const float2 *P;  // P[i]: prefix sums up to row i (rows h .. nv)
};

// Plane PL (kc = kc0 + PL) of a lane's R layers: its thresholds, the
// interior rows of the layer below it and its boundary rows.
template <int R, int PL>
__device__ __forceinline__ void prefix_plane(const PrefixCrossing &c, const float2 *__restrict__ vr,
                                             float cvlo, float cvhi, float fnv, int nv,
                                             float (&au)[R], float (&ad)[R], float2 &pa)
{
    const float kc = c.kc0 + (float)PL;
    const int ta = row_threshold<true>(kc, c.rga, c.sa, c.s0, c.KD, vr, cvlo, cvhi, fnv, nv);
    const int tb = row_threshold<false>(kc, c.rgb, c.sb, c.s0, c.KD, vr, cvlo, cvhi, fnv, nv);
    const float2 pb = __ldg(c.P + tb);
    if (PL > 0) {  // interior rows of layer PL-1: [Ta(PL-1), Tb(PL))
        au[PL > 0 ? PL - 1 : 0] = fmaf(c.len0, pb.x - pa.x, au[PL > 0 ? PL - 1 : 0]);
        ad[PL > 0 ? PL - 1 : 0] = fmaf(c.len0, pb.y - pa.y, ad[PL > 0 ? PL - 1 : 0]);
    }
    // boundary rows [Tb, Ta): in the layer below from sa to the crossing x,
    // in the layer above from x to sb; p0 = P[i] on entry, P[i + 1] returned
    auto edge = [&](int i, bool ok, float2 p0) {
        const int r = min(i, nv - 1);
        const float x = fmaf(kc, c.KD * __ldg(vr + r).y, -c.s0);
        const float2 p1 = __ldg(c.P + r + 1);
        const float ru = p1.x - p0.x, rd = p1.y - p0.y;
        const float lb = ok ? x - c.sa : 0.f, la = ok ? c.sb - x : 0.f;
        if (PL > 0) {
            au[PL > 0 ? PL - 1 : 0] = fmaf(lb, ru, au[PL > 0 ? PL - 1 : 0]);
            ad[PL > 0 ? PL - 1 : 0] = fmaf(lb, rd, ad[PL > 0 ? PL - 1 : 0]);
        }
        if (PL < R) {
            au[PL < R ? PL : 0] = fmaf(la, ru, au[PL < R ? PL : 0]);
            ad[PL < R ? PL : 0] = fmaf(la, rd, ad[PL < R ? PL : 0]);
        }
        return p1;
    };
    float2 pe = edge(tb, tb < ta, pb);
    if (__any_sync(kFull, ta > tb + 1))
        for (int i = tb + 1; i < ta; ++i) pe = edge(i, true, pe);
    pa = ta == tb ? pb : pe;  // P[Ta]: the last boundary row's end
}

template <int R, int... PL>
__device__ __forceinline__ void prefix_planes(std::integer_sequence<int, PL...>,
                                              const PrefixCrossing &c, const float2 *__restrict__ vr,
                                              float cvlo, float cvhi, float fnv, int nv,
                                              float (&au)[R], float (&ad)[R])
{
    float2 pa = make_float2(0.f, 0.f);
    (prefix_plane<R, PL>(c, vr, cvlo, cvhi, fnv, nv, au, ad, pa), ...);
}

// One warp per xy voxel column (kPrefixWarps per CTA); lane l owns the R
// upper layers hz + l R + q (q < R) and their mirrors nz-1-(hz + l R + q),
// hz = nz/2, i.e. the planes kc = l R .. l R + R.  The crossings of the
// column are prepared 32 at a time, one per lane, in shared memory.
template <int R>
__device__ __forceinline__ void adj_prefix_block(const ProjGeom &G, const ColParams *__restrict__ cols,
                                                 const float2 *__restrict__ vr,
                                                 const int *__restrict__ hit_ptr,
                                                 const CellHit *__restrict__ hits,
                                                 const float2 *__restrict__ pq,
                                                 float *__restrict__ vol, int blk)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cell = blk * kPrefixWarps + w;
    if (cell >= G.nx * G.ny) return;  // whole warps; only __syncwarp below
    const int h = G.nv >> 1, hz = G.nz >> 1, nv = G.nv;
    const float fnv = (float)nv;
    const float cvlo = G.cv + 0.5f - kRowSlack, cvhi = G.cv + 0.5f + kRowSlack;
    float au[R], ad[R];
#pragma unroll
    for (int q = 0; q < R; ++q) au[q] = ad[q] = 0.f;
    __shared__ float4 hc[kPrefixWarps][32][2];
    const int h0 = __ldg(hit_ptr + cell), h1 = __ldg(hit_ptr + cell + 1);
    for (int hb = h0; hb < h1; hb += 32) {
        const int nh = min(32, h1 - hb);
        __syncwarp();
        if (lane < nh) {
            const CellHit e = __ldg(hits + hb + lane);
            const int j = e.x >> 16, iu = e.x & 0xffff;
            const float sa = __int_as_float(e.y), sb = __int_as_float(e.z);
            const int c = j * G.nu + iu;
            const float4 cz = __ldg(reinterpret_cast<const float4 *>(cols + c) + 1);
            const float s0 = cz.x, KD = cz.y, rKD = cz.w;
            // row position per unit plane coordinate at sa and at sb
            const float rga = rcp_approx((s0 + sa) * rKD) * G.rdv;
            const float rgb = rcp_approx((s0 + sb) * rKD) * G.rdv;
            hc[w][lane][0] = make_float4(sa, sb, s0, KD);
            hc[w][lane][1] = make_float4(rga, rgb, __int_as_float(c * (h + 1)), sb - sa);
        }
        __syncwarp();
        for (int k = 0; k < nh; ++k) {
            const float4 ca = hc[w][k][0], cb = hc[w][k][1];
            PrefixCrossing c;
            c.sa = ca.x; c.sb = ca.y; c.s0 = ca.z; c.KD = ca.w;
            c.rga = cb.x; c.rgb = cb.y; c.len0 = cb.w;
            c.kc0 = (float)(lane * R);
            c.P = pq + __float_as_int(cb.z) - h;
            prefix_planes<R>(std::make_integer_sequence<int, R + 1>{}, c, vr, cvlo, cvhi, fnv, nv,
                             au, ad);
        }
    }
    float *colv = vol + (long long)cell * G.nz;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int ku = hz + lane * R + q;
        if (ku < G.nz) {
            colv[ku] += au[q];
            colv[G.nz - 1 - ku] += ad[q];
        }
    }
}

// grid: blocks of kPrefixWarps voxel columns x slots
template <int R>
__global__ void __launch_bounds__(32 * kPrefixWarps)
adj_prefix_kernel(ProjGeom G, const ColParams *__restrict__ cols, const float2 *__restrict__ vr,
                  const int *__restrict__ hit_ptr, const CellHit *__restrict__ hits,
                  const float2 *__restrict__ pq, float *__restrict__ vol, long long sstride)
{
    const long long so = blockIdx.y * sstride;
    adj_prefix_block<R>(G, cols, vr, hit_ptr, hits, slot_ptr(pq, so), slot_ptr(vol, so),
                        blockIdx.x);
}

// scans of different geometries (and the same R) in one grid
template <int R>
__global__ void __launch_bounds__(32 * kPrefixWarps) adj_prefix_group_kernel(const AdjGroup grp)
{
    const int m = find_job(blockIdx.x, grp.b0, grp.n);
    const AdjJob &J = grp.job[m];
    const int local = blockIdx.x - grp.b0[m];
    const int slot = local / J.nb;
    const long long so = slot * J.sstride;
    adj_prefix_block<R>(J.g, J.cols, J.vr, J.hit_ptr, J.hits,
                        reinterpret_cast<const float2 *>(slot_ptr(J.rs, so)), slot_ptr(J.vol, so),
                        local - slot * J.nb);
}

}  // namespace

int project_blocks(const ProjGeom &g)
{
    const int np = (g.nv + 1) >> 1;
    const int nrgb = (np + 32 * kRowGroups - 1) / (32 * kRowGroups);
    return g.n_views * g.nu * nrgb;
}

cudaError_t launch_forward(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                           const int4 *cells, const float *vol, float *out, int mode,
                           const float *aux, double *partials, int *nonfinite, cudaStream_t st,
                           Slots sl)
{
    const int nb = project_blocks(g);
    if (nb <= 0 || sl.n <= 0) return cudaSuccess;
    const dim3 grid((unsigned)nb, (unsigned)sl.n);
    const int walk = walk_of(g);
#define PICCS_FWD_W(M, NORM, W)                                                               \
    fwd_kernel<M, NORM, W><<<grid, 256, 0, st>>>(g, cols, vr, cells, vol, out, aux, partials, \
                                                 nonfinite, nullptr, nullptr, sl.stride)
#define PICCS_FWD(M, NORM)                                                                    \
    do {                                                                                      \
        if (walk == kWalkMulti) PICCS_FWD_W(M, NORM, kWalkMulti);                             \
        else if (walk == kWalkAhead) PICCS_FWD_W(M, NORM, kWalkAhead);                        \
        else PICCS_FWD_W(M, NORM, kWalkOne);                                                  \
    } while (0)
    if (mode == FWD_RESID) {
        if (partials) PICCS_FWD(FWD_RESID, true); else PICCS_FWD(FWD_RESID, false);
    } else if (mode == FWD_RESID16) {
        if (partials) PICCS_FWD(FWD_RESID16, true); else PICCS_FWD(FWD_RESID16, false);
    } else {
        if (partials) PICCS_FWD(FWD_PLAIN, true); else PICCS_FWD(FWD_PLAIN, false);
    }
#undef PICCS_FWD
#undef PICCS_FWD_W
    return cudaGetLastError();
}

cudaError_t launch_forward_lsqr(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                                const int4 *cells, const float *vol, float *U, const float *aux,
                                float *rA, float *Aw, double *partials, cudaStream_t st, Slots sl)
{
    const int nb = project_blocks(g);
    if (nb <= 0 || sl.n <= 0) return cudaSuccess;
    const dim3 grid((unsigned)nb, (unsigned)sl.n);
#define PICCS_FWDL(W)                                                                          \
    fwd_kernel<FWD_LSQR, true, W><<<grid, 256, 0, st>>>(g, cols, vr, cells, vol, U, aux, partials, \
                                                        nullptr, rA, Aw, sl.stride)
    switch (walk_of(g)) {
    case kWalkMulti: PICCS_FWDL(kWalkMulti); break;
    case kWalkAhead: PICCS_FWDL(kWalkAhead); break;
    default: PICCS_FWDL(kWalkOne);
    }
#undef PICCS_FWDL
    return cudaGetLastError();
}

// The prefix-sum gather spends a fixed amount of work per layer and plane;
// the candidate gather one evaluation per candidate row, about
// rows_per_layer + 0.5 of them per layer.  Measured on GB300: at 1.9 rows per
// layer (1 mm voxels, 0.8 mm pitch, magnification 1.5) the candidate gather
// takes 5.5 ms against 6.3 ms; at 3.2 (0.6 mm voxels, 0.3 mm pitch,
// magnification 1.6) 238 ms against 175 ms.
constexpr float kPrefixMinRowsPerLayer = 2.5f;

bool adjoint_uses_prefix(const ProjGeom &g)
{
    return (g.nv & 1) == 0 && (g.nz & 1) == 0 && !g.multi && g.nz <= 2 * 32 * kPrefixMaxR &&
           g.rows_per_layer >= kPrefixMinRowsPerLayer;
}

cudaError_t launch_adjoint(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                           const int *hit_ptr, const CellHit *hits, const float *proj, float *rs,
                           float *vol, cudaStream_t st, Slots sl)
{
    const int nb = project_blocks(g);
    if (nb <= 0 || sl.n <= 0) return cudaSuccess;
    if (adjoint_uses_prefix(g)) {
        const long long ncol = (long long)g.n_views * g.nu;
        const dim3 pgrid((unsigned)((ncol * 32 + 255) / 256), (unsigned)sl.n);
        float2 *pq = reinterpret_cast<float2 *>(rs);
        ray_prefix_kernel<<<pgrid, 256, 0, st>>>(g, cols, vr, proj, pq, sl.stride);
        const int hz = g.nz >> 1;
        const int R = (hz + 31) / 32;  // layers per lane: 1 .. kPrefixMaxR
        const dim3 grid((unsigned)((g.nx * g.ny + kPrefixWarps - 1) / kPrefixWarps), (unsigned)sl.n);
        switch (R) {
#define PICCS_ADJ_R(RR)                                                                        \
    case RR:                                                                                   \
        adj_prefix_kernel<RR><<<grid, 32 * kPrefixWarps, 0, st>>>(g, cols, vr, hit_ptr, hits, pq, \
                                                                   vol, sl.stride);            \
        break;
            PICCS_ADJ_R(1) PICCS_ADJ_R(2) PICCS_ADJ_R(3) PICCS_ADJ_R(4)
            PICCS_ADJ_R(5) PICCS_ADJ_R(6) PICCS_ADJ_R(7) PICCS_ADJ_R(8)
#undef PICCS_ADJ_R
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const int per_cta = kGatherThreads * kLayersPerThread;  // layer pairs per CTA
    const int nlp = (g.nz + 1) >> 1;
    const dim3 grid((unsigned)(g.nx * g.ny), (unsigned)((nlp + per_cta - 1) / per_cta),
                    (unsigned)sl.n);
    const dim3 sgrid((unsigned)nb, (unsigned)sl.n);
    if ((g.nv & 1) == 0 && (g.nz & 1) == 0) {
        scale_rays_kernel<true><<<sgrid, 256, 0, st>>>(g, cols, vr, proj, rs, sl.stride);
        adj_gather_kernel<true><<<grid, kGatherThreads, 0, st>>>(g, cols, vr, hit_ptr, hits, rs, vol,
                                                                 sl.stride);
    } else {
        scale_rays_kernel<false><<<sgrid, 256, 0, st>>>(g, cols, vr, proj, rs, sl.stride);
        adj_gather_kernel<false><<<grid, kGatherThreads, 0, st>>>(g, cols, vr, hit_ptr, hits, rs,
                                                                  vol, sl.stride);
    }
    return cudaGetLastError();
}

cudaError_t launch_forward_group(const FwdJob *jobs, int n, int mode, cudaStream_t st)
{
    if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
    FwdGroup grp{};
    long long total = 0;
    bool multi = false, ahead = true;
    const bool norm = jobs[0].partials != nullptr;
    for (int i = 0; i < n; ++i) {
        grp.job[i] = jobs[i];
        grp.job[i].nb = project_blocks(jobs[i].g);
        grp.b0[i] = (int)total;
        total += (long long)grp.job[i].nb * jobs[i].nslot;
        multi |= jobs[i].g.multi != 0;
        ahead &= jobs[i].g.ahead != 0;
        if ((jobs[i].partials != nullptr) != norm) return cudaErrorInvalidValue;
    }
    grp.n = n;
    if (total <= 0) return cudaSuccess;
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned nb = (unsigned)total;
#define PICCS_FWDG(M, NORM)                                                         \
    do {                                                                            \
        if (multi) fwd_group_kernel<M, NORM, kWalkMulti><<<nb, 256, 0, st>>>(grp);  \
        else if (ahead) fwd_group_kernel<M, NORM, kWalkAhead><<<nb, 256, 0, st>>>(grp); \
        else fwd_group_kernel<M, NORM, kWalkOne><<<nb, 256, 0, st>>>(grp);          \
    } while (0)
    switch (mode) {
    case FWD_RESID:
        if (norm) PICCS_FWDG(FWD_RESID, true); else PICCS_FWDG(FWD_RESID, false);
        break;
    case FWD_RESID16:
        if (norm) PICCS_FWDG(FWD_RESID16, true); else PICCS_FWDG(FWD_RESID16, false);
        break;
    case FWD_LSQR:
        if (!norm) return cudaErrorInvalidValue;
        PICCS_FWDG(FWD_LSQR, true);
        break;
    default:
        if (norm) PICCS_FWDG(FWD_PLAIN, true); else PICCS_FWDG(FWD_PLAIN, false);
    }
#undef PICCS_FWDG
    return cudaGetLastError();
}

cudaError_t launch_adjoint_group(const AdjJob *jobs, int n, cudaStream_t st)
{
    if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
    // the ray scaling (or prefix sums) of each job, then one gather launch per
    // gather kind present: candidate (even sizes / general) or prefix sums (R)
    int kind[kMaxGroup];
    for (int i = 0; i < n; ++i) {
        const ProjGeom &g = jobs[i].g;
        const long long ncol = (long long)g.n_views * g.nu;
        if (project_blocks(g) <= 0) {
            kind[i] = -1;
            continue;
        }
        if (adjoint_uses_prefix(g)) {
            const dim3 pgrid((unsigned)((ncol * 32 + 255) / 256), (unsigned)jobs[i].nslot);
            ray_prefix_kernel<<<pgrid, 256, 0, st>>>(g, jobs[i].cols, jobs[i].vr, jobs[i].proj,
                                                     reinterpret_cast<float2 *>(jobs[i].rs),
                                                     jobs[i].sstride);
            kind[i] = 10 + ((g.nz >> 1) + 31) / 32;  // prefix, R layers per lane
        } else {
            const bool even = (g.nv & 1) == 0 && (g.nz & 1) == 0;
            const dim3 sgrid((unsigned)project_blocks(g), (unsigned)jobs[i].nslot);
            if (even)
                scale_rays_kernel<true><<<sgrid, 256, 0, st>>>(g, jobs[i].cols, jobs[i].vr,
                                                               jobs[i].proj, jobs[i].rs, jobs[i].sstride);
            else
                scale_rays_kernel<false><<<sgrid, 256, 0, st>>>(g, jobs[i].cols, jobs[i].vr,
                                                                jobs[i].proj, jobs[i].rs, jobs[i].sstride);
            kind[i] = even ? 1 : 0;
        }
    }
    bool done[kMaxGroup] = {};
    for (int i = 0; i < n; ++i) {
        if (done[i] || kind[i] < 0) continue;
        AdjGroup grp{};
        long long total = 0;
        for (int k = i; k < n; ++k) {
            if (done[k] || kind[k] != kind[i]) continue;
            done[k] = true;
            AdjJob J = jobs[k];
            const int ncell = J.g.nx * J.g.ny;
            if (kind[i] >= 10) {
                J.nb = (ncell + kPrefixWarps - 1) / kPrefixWarps;
            } else {
                const int per_cta = kGatherThreads * kLayersPerThread;
                J.nb = ncell * (((J.g.nz + 1) / 2 + per_cta - 1) / per_cta);
            }
            grp.job[grp.n] = J;
            grp.b0[grp.n] = (int)total;
            total += (long long)J.nb * J.nslot;
            grp.n += 1;
        }
        if (total <= 0) continue;
        if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
        const unsigned nb = (unsigned)total;
        switch (kind[i]) {
        case 0: adj_gather_group_kernel<false><<<nb, kGatherThreads, 0, st>>>(grp); break;
        case 1: adj_gather_group_kernel<true><<<nb, kGatherThreads, 0, st>>>(grp); break;
#define PICCS_ADJG(RR) \
        case 10 + RR: adj_prefix_group_kernel<RR><<<nb, 32 * kPrefixWarps, 0, st>>>(grp); break;
        PICCS_ADJG(1) PICCS_ADJG(2) PICCS_ADJG(3) PICCS_ADJG(4)
        PICCS_ADJG(5) PICCS_ADJG(6) PICCS_ADJG(7) PICCS_ADJG(8)
#undef PICCS_ADJG
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

// Slots' FP32 projections (src_stride bytes apart) rounded to BF16 (to nearest
// even) into dst (dst_stride bytes apart).
__global__ void __launch_bounds__(256)
to_bf16_kernel(long long n, const float *__restrict__ src, long long src_stride,
               __nv_bfloat16 *__restrict__ dst, long long dst_stride)
{
    src = slot_ptr(src, blockIdx.y * src_stride);
    dst = slot_ptr(dst, blockIdx.y * dst_stride);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

cudaError_t launch_to_bf16(long long n, const float *src, long long src_stride, void *dst,
                           long long dst_stride, int nslot, cudaStream_t st)
{
    to_bf16_kernel<<<dim3(152 * 8, nslot), 256, 0, st>>>(
        n, src, src_stride, reinterpret_cast<__nv_bfloat16 *>(dst), dst_stride);
    return cudaGetLastError();
}

}  // namespace piccs
