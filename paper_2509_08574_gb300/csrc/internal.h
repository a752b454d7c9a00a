// Internal declarations shared by the CUDA translation units of libpiccs.
// Nothing here is part of the public C ABI (include/piccs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace piccs {

// Per (view, detector column) ray-walk constants, computed in FP64 on the host
// and rounded once.  All rays of one detector column share their projection
// onto the xy plane (the detector v axis is parallel to the rotation axis and
// the source lies in z = 0), so the xy part of the Siddon walk is the same for
// the whole column and is stored once as a cell table (see ray_tables.h):
// cells[start2 .. start2 + ceil(ncells/2)) hold, two per 16 bytes, for every
// xy cell the column's rays cross: the flat index of the cell's first voxel
// ((ix*ny + iy)*nz) and the bits of the FP32 xy distance (mm, from the
// column's entry into the volume's xy square) at which the rays leave it.  An
// odd list is padded with a zero-length copy of its last cell.
// Row v (detector height, mm, with rv = 1/v, or 1e30 for v = 0) has z (voxel
// units, centred) = v * (s0 + s) * rKD, so it crosses the z plane with
// centred coordinate kc at s = kc * (KD * rv) - s0, evaluated as
// fma(kc, KD * rv, -s0); s0 is the xy distance from the source to the
// column's entry point.  Its 3D length per unit s is sqrt(1 + (v * invD)^2).
struct __align__(16) ColParams {
    long long start2;        // int4 index of the column's first pair of cells
    int ncells;              // 0: the column misses the volume
    int pad0;
    float s0, KD, invD, rKD; // one 16-byte load for the adjoint's gather
};

// One crossing of an xy voxel column by a detector column (the transpose of
// the column cell tables): x = view << 16 | detector column, y/z = the bits of
// the FP32 xy distances at which the column's rays enter and leave the voxel
// column (the same values the forward walk uses), w unused.
typedef int4 CellHit;

struct ProjGeom {
    int nx, ny, nz;
    int nu, nv, n_views;
    long long sj, su, sv;   // projection strides of view, column, row
    float halfnz;           // nz / 2
    float rdv, cv;          // 1 / dv and (nv - 1) / 2: row index of height v = v * rdv + cv
    int sv32;               // sv as a 32-bit stride (1 or nu)
    int multi;              // a cell can hold more than one z crossing of a row
    int ahead;              // the forward walk loads the cell table one entry early
    float rows_per_layer;   // detector rows one voxel layer spans at the isocentre
};

// Scans of one geometry processed together ("slots", Sec. 3's repeated scans
// batched into one launch per step): every workspace pointer of slot s is the
// slot-0 pointer shifted by s * stride bytes; the ray tables are shared.  A
// kernel takes its slot from blockIdx.y (the adjoint gather: blockIdx.z; the
// one-CTA finalize kernels: blockIdx.x).  Slots{1, 0} is a single scan.
struct Slots {
    int n;
    long long stride;  // bytes
};

#ifdef __CUDACC__
template <class T>
__device__ __forceinline__ T *slot_ptr(T *p, long long off)
{
    return p ? reinterpret_cast<T *>(reinterpret_cast<char *>(const_cast<void *>(
                                         static_cast<const void *>(p))) + off)
             : p;
}
#endif

// Device-side Krylov scalars (FP64), read by every vector kernel so that no
// value has to come back to the host between kernels.
struct KrylovScalars {
    double gamma;     // ||s||^2 of the current normal-equations residual s = A~^T r~
    double gamma0;    // gamma at the start of the current cycle
    double delta;     // ||A~ p||^2
    double a;         // step length gamma / delta (0 when stopped or broken down)
    double beta;      // gamma_new / gamma_old (0 right after a restart)
    int status;       // 0, or a negative PICCS_E* code
    int iters_run;    // inner iterations with a != 0
    int n_hist;
    int stopped;      // the cycle converged (gamma <= 1e-26 gamma0)
    int nonfinite;    // a NaN/Inf was seen in an input
    int pad;
    double hist[512];
};

constexpr int kMaxBasis = 256;  // LSQR re-orthogonalisation: basis vectors per cycle

// Device-side state of LSQR (Golub-Kahan bidiagonalisation of the augmented
// operator with the Givens QR update).  The augmented vector u is held as
// beta * u = [uA; R z + sigma b_R] (R the regularisation rows, b_R their
// right-hand side), so its 3M or 6M regularisation rows are never stored:
// R^T (R z + sigma b_R) = K z + sigma c with K = D^T Omega D (+ lambda^2 I for
// PIPLE), c = R^T b_R, and |R z + sigma b_R|^2 = z.K z + 2 sigma <z, c> +
// sigma^2 |b_R|^2, |b_R|^2 = <x_p, c>.  v is stored unnormalised (vhat =
// alpha v).  The float blocks are the coefficients the vector and projector
// kernels read; the finalize kernels write them.
struct LsqrScalars {
    double alpha, beta;   // alpha_i (= |vhat|) and beta_i (uA and z are beta_i u_i)
    double rhobar, phibar, c, s, rho;
    double sigma;         // coefficient of b_R in beta_i u_i
    double sigma_next;    // coefficient of b_R after the next z-step
    double bR2;           // |b_R|^2 = <x_p, c>
    double normar0;       // |A~^T r~| at the start of the cycle
    int stopped;          // the cycle has converged or a bidiagonal entry vanished
    int nbasis;           // vectors held in the re-orthogonalisation basis
    float fwd[8];         // forward u-step: {1/alpha_i, alpha_i/beta_i, stopped,
                          //  theta_i/rho_{i-1}, x step not yet applied to rA,
                          //  first step of the cycle, 0, 0}
    float ureg[4];        // z-step: {1/alpha_i, alpha_i/beta_i, new sigma, stopped}
    float vx[8];          // {1/alpha_i, theta_i/rho_{i-1}, phi_i/rho_i, 1/beta_{i+1},
                          //  beta_{i+1}, stopped, first step of the cycle, 0}
    double h[kMaxBasis];  // Gram-Schmidt coefficients
};

enum FwdMode { FWD_PLAIN = 0, FWD_RESID = 1, FWD_LSQR = 2, FWD_RESID16 = 3 };

// Scans of different geometries projected in one launch ("groups"): each job
// is one context's part -- its geometry, ray tables and buffers (slot 0's;
// the context's slots sstride bytes apart), nslot slots of nb blocks each.
// The table goes to the kernel by value (kernel parameters), so a captured
// CUDA graph keeps its own copy.
constexpr int kMaxGroup = 8;
struct FwdJob {
    ProjGeom g;
    const ColParams *cols;
    const float2 *vr;
    const int4 *cells;
    const float *vol;
    float *out;
    const float *aux;
    double *partials;
    int *nonfinite;
    float *ra, *aw;
    long long sstride;
    int nslot, nb;
};
struct FwdGroup {
    FwdJob job[kMaxGroup];
    int b0[kMaxGroup];  // the job's first block in the grid
    int n;
};
struct AdjJob {
    ProjGeom g;
    const ColParams *cols;
    const float2 *vr;
    const int *hit_ptr;
    const CellHit *hits;
    const float *proj;
    float *rs;
    float *vol;
    long long sstride;
    int nslot, nb;
};
struct AdjGroup {
    AdjJob job[kMaxGroup];
    int b0[kMaxGroup];
    int n;
};

// ---- projector (kernels_project.cu) ----
int project_blocks(const ProjGeom &g);
// vr[iv] = {v, 1/v} per detector row (1e30 for v = 0)
// mode FWD_PLAIN: out = A vol; FWD_RESID: out = aux - A vol (aux = the data b,
// NaN/Inf in it set *nonfinite); FWD_RESID16: the same with b in BF16.
// partials (may be null) get |out|^2 per block.
cudaError_t launch_forward(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                           const int4 *cells, const float *vol, float *out, int mode,
                           const float *aux, double *partials, int *nonfinite, cudaStream_t st,
                           Slots sl = Slots{1, 0});
// vol += A^T proj (vol holds the starting values, e.g. zeros); rs is a
// scratch of adjoint_rs_floats(N, views x columns) floats: per detector
// column the prefix sums of proj scaled by each ray's sec
// (adjoint_uses_prefix), else those N scaled values themselves.
bool adjoint_uses_prefix(const ProjGeom &g);
inline long long adjoint_rs_floats(long long N, long long ncol) { return N + 2 * ncol; }
cudaError_t launch_adjoint(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                           const int *hit_ptr, const CellHit *hits, const float *proj, float *rs,
                           float *vol, cudaStream_t st, Slots sl = Slots{1, 0});
// The same for 1 <= n <= kMaxGroup jobs in one launch per kernel (the ray
// scaling stays one launch per job): each job's result is bit for bit the
// one launch_forward / launch_forward_lsqr / launch_adjoint gives it.  Every
// job's mode is `mode`; partials (per job) may be null only for all jobs.
cudaError_t launch_forward_group(const FwdJob *jobs, int n, int mode, cudaStream_t st);
cudaError_t launch_adjoint_group(const AdjJob *jobs, int n, cudaStream_t st);
// n FP32 values per slot -> BF16 (round to nearest even)
cudaError_t launch_to_bf16(long long n, const float *src, long long src_stride, void *dst,
                           long long dst_stride, int nslot, cudaStream_t st);

// LSQR u-step with the data residual kept current (aux = LsqrScalars::fwd):
// q = aux[0] A vol; U = q - aux[1] U; first step of a cycle (aux[5]): Aw = q;
// else rA -= aux[4] Aw, Aw = q - aux[3] Aw.  Skipped when aux[2] != 0.
cudaError_t launch_forward_lsqr(const ProjGeom &g, const ColParams *cols, const float2 *vr,
                                const int4 *cells, const float *vol, float *U, const float *aux,
                                float *rA, float *Aw, double *partials, cudaStream_t st,
                                Slots sl = Slots{1, 0});

// ---- regulariser (kernels_reg.cu) ----
struct VolDims { int nx, ny, nz; };
// stencil grids: at most 152 SMs x 8 resident CTAs of 256 threads
constexpr int kStencilMaxBlocks = 152 * 8;
int stencil_blocks(long long M);
cudaError_t launch_weights(VolDims d, const float *x, const float *xp, float alpha2,
                           float lambda2, float tau2, int rule, int variant, float *omega,
                           float *w2sq, cudaStream_t st, Slots sl = Slots{1, 0});
cudaError_t launch_prior_rhs(VolDims d, const float *xp, const float *w2sq, float lambda2,
                             int variant, float *c, cudaStream_t st, Slots sl = Slots{1, 0});
// out = D^T diag(omega) D z (+ lam2_piple z); partials (may be null) get
// sum omega |Dz|^2 (+ lam2_piple z^2) per block.
cudaError_t launch_reg_normal(VolDims d, const float *z, const float *omega, float lam2_piple,
                              float *out, double *partials, cudaStream_t st,
                              Slots sl = Slots{1, 0});
// Restart of a Krylov cycle: gn = c - D^T Omega D x (- lam2_piple x);
// first: g = gn, s = gn; else s += gn - g, g = gn, partials get s^2.
cudaError_t launch_reg_restart(VolDims d, const float *x, const float *omega, float lam2_piple,
                               const float *c, float *g, float *s, int first, double *partials,
                               cudaStream_t st, Slots sl = Slots{1, 0});

// LSQR z-step (see LsqrScalars): init: z' = -src; else z' = co[0] src -
// co[1] zold (co = LsqrScalars::ureg); skipped when co[3] != 0 (not in init).
cudaError_t launch_lsqr_zstep(VolDims d, int init, const float *src, const float *zold, float *znew,
                              const float *co, cudaStream_t st, Slots sl = Slots{1, 0});
// The regularisation part of A~^T u: s = K z + sigma c (sigma = 1 in init,
// else co[2]); partials: 2 (init: 3) arrays of stencil_blocks(M) doubles,
// [z.K z | <z, c> | <x_p, c>].  Skipped when co[3] != 0 (not in init).
cudaError_t launch_lsqr_ureg(VolDims d, int init, const float *z, const float *omega,
                             float lam2_piple, const float *c, const float *xp, float *s,
                             const float *co, double *partials, cudaStream_t st,
                             Slots sl = Slots{1, 0});

// ---- Krylov vector work (kernels_krylov.cu) ----
// (Slots: see above; bstride = the per-slot stride of the LSQR basis region,
// which also holds that slot's Gram-Schmidt partial sums after the vectors)
int vector_blocks();
cudaError_t launch_p_update(long long M, const float *s, float *p, const KrylovScalars *k,
                            cudaStream_t st, Slots sl = Slots{1, 0});
cudaError_t launch_x_update(long long M, long long N, float *x, const float *p, float *g,
                            const float *t, float *s, float *r, const float *q,
                            const KrylovScalars *k, cudaStream_t st, Slots sl = Slots{1, 0});
cudaError_t launch_norm2(long long n, const float *v, double *partials, cudaStream_t st,
                         Slots sl = Slots{1, 0});
cudaError_t launch_finalize_delta(KrylovScalars *k, const double *pa, int na, const double *pb,
                                  int nb, cudaStream_t st, Slots sl = Slots{1, 0});
cudaError_t launch_finalize_gamma(KrylovScalars *k, const double *p, int n, int restart,
                                  cudaStream_t st, Slots sl = Slots{1, 0});
cudaError_t launch_reset_scalars(KrylovScalars *k, cudaStream_t st, Slots sl = Slots{1, 0});
cudaError_t launch_count_nonfinite(long long n, const float *v, int *flag, cudaStream_t st,
                                   Slots sl = Slots{1, 0});
// the same for n BF16 values
cudaError_t launch_count_nonfinite16(long long n, const void *v, int *flag, cudaStream_t st,
                                     Slots sl = Slots{1, 0});
cudaError_t launch_sum_partials(const double *p, int n, double *out, cudaStream_t st);
// LSQR
cudaError_t launch_lsqr_reset(KrylovScalars *k, LsqrScalars *l, cudaStream_t st,
                              Slots sl = Slots{1, 0});
// Start of an LSQR cycle: update (rA -= pending x step * Aw; else rA is
// b - A x already), then U = rA; partials get |U|^2.
cudaError_t launch_lsqr_rinit(long long N, int update, float *rA, const float *Aw, float *U,
                              const LsqrScalars *l, double *partials, cudaStream_t st,
                              Slots sl = Slots{1, 0});
// first: vhat = s / beta_1; else v = vhat / alpha_i, w = v - tw w, x += tx w and,
// unless last, vhat = s / beta_{i+1} - beta_{i+1} v; basis (may be null) gets v.
// partials get |vhat|^2 (unless last).
cudaError_t launch_lsqr_vx(long long M, int first, int last, float *x, float *w, float *vhat,
                           const float *s, void *basis, const LsqrScalars *l, double *partials,
                           cudaStream_t st, Slots sl = Slots{1, 0}, long long bstride = 0,
                           bool basis_bf16 = false);
// beta = sqrt(|uA|^2 + z.Kz + 2 sigma <z,c> + sigma^2 |b_R|^2) and the Givens step
cudaError_t launch_lsqr_finalize_beta(KrylovScalars *k, LsqrScalars *l, int init,
                                      const double *pu, int nu, const double *pr, int nr,
                                      cudaStream_t st, Slots sl = Slots{1, 0});
// alpha = |vhat|, the rest of the Givens step, the stop test
cudaError_t launch_lsqr_finalize_alpha(KrylovScalars *k, LsqrScalars *l, int init,
                                       const double *p, int n, cudaStream_t st,
                                       Slots sl = Slots{1, 0});
// Basis vector j starts at basis + j * ldb, ldb = lsqr_basis_stride(M) (a
// multiple of 64 floats, so every vector is 256-byte aligned for float4 access).
inline long long lsqr_basis_stride(long long M) { return (M + 63) / 64 * 64; }
// one Gram-Schmidt pass of vhat against basis[0..nb) (nb <= kMaxBasis):
// dots: partials[j * lsqr_dot_blocks() + block] = <basis_j, vhat>;
// fin_dots: l->h[j] = their fixed-order sums; sub: vhat -= sum_j h_j basis_j,
// norm_partials (may be null) get |vhat|^2.  All skip once l->stopped.
cudaError_t launch_lsqr_dots(long long M, long long ldb, int nb, const void *basis,
                             const float *vhat, const LsqrScalars *l, double *partials,
                             cudaStream_t st, Slots sl = Slots{1, 0}, long long bstride = 0,
                             bool basis_bf16 = false);
cudaError_t launch_lsqr_fin_dots(int nb, LsqrScalars *l, const double *partials, cudaStream_t st,
                                 Slots sl = Slots{1, 0}, long long bstride = 0);
cudaError_t launch_lsqr_sub(long long M, long long ldb, int nb, const void *basis, float *vhat,
                            const LsqrScalars *l, double *norm_partials, cudaStream_t st,
                            Slots sl = Slots{1, 0}, long long bstride = 0, bool basis_bf16 = false);
int lsqr_dot_blocks();

// ---- host helpers (piccs_api.cpp) ----
// Sets the per-thread message that piccs_last_error(NULL) returns.
void set_thread_error(const char *msg);

}  // namespace piccs
