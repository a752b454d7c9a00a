/*
 * piccs.h -- C ABI of the GB300 (sm_103a) IRN-PICCS cone-beam reconstruction
 * library (libpiccs.so).
 *
 * Method (Hastings, Islam, Sabate Landman et al., "Real-time CBCT
 * reconstructions using Krylov solvers in repeated scanning procedures"):
 *   CT is the linear model A x + e = b (Sec. 2.1, Eq. 1).  Given a prior
 *   reconstruction x_p, PICCS minimises ||Ax-b||^2 + alpha^2 TV(x)
 *   + lambda^2 TV(x - x_p) (Eq. 3).  The IRN scheme (Sec. 2.2-2.3, Eqs. 6-11)
 *   replaces each TV term by a weighted 2-norm whose weights
 *   W(Dz)_ii = (sqrt(sum_d [D_d z]_i^2) + tau^2)^(-1/2) are frozen at the
 *   previous outer iterate, and solves each reweighted problem approximately
 *   with a few CGLS (or LSQR) iterations on the augmented least-squares system
 *   [A; alpha W1 D; lambda W2 D] x ~ [b; 0; lambda W2 D x_p] (the display after
 *   Eq. 11), warm-started at the previous iterate.
 *
 * Conventions shared by every call:
 *   - Geometry: circular cone beam, rotation axis z, volume centred at the
 *     origin; source S_j = DSO (cos t_j, sin t_j, 0); detector centre
 *     -(DSD - DSO)(cos t_j, sin t_j, 0); detector axes u = (-sin t_j, cos t_j, 0),
 *     v = (0, 0, 1); pixel (iu, iv) centre at (iu - (nu-1)/2) du + u_offset
 *     along u and (iv - (nv-1)/2) dv along v; one ray per pixel from the
 *     source through the pixel centre.  The paper names only DSO, DSD and the
 *     pitch (Sec. 3.2); the rest is this library's convention.  The detector
 *     may be shifted along u, not along v: the kernels pair every row with
 *     its mirror about the plane z = 0 of the source.
 *   - A_ij = length in mm of ray i inside voxel j (exact ray/voxel-box
 *     intersection, i.e. Siddon weights).  A^T uses the same weights.
 *   - Volume layout: float32, index (ix*ny + iy)*nz + iz (z fastest).
 *   - Projection layout: PICCS_LAYOUT_UV: (j*nu + iu)*nv + iv (v fastest, the
 *     native and fastest one); PICCS_LAYOUT_VU: (j*nv + iv)*nu + iu.
 *   - Pointers named d_* are CUDA device pointers in the current device's
 *     address space, h_* are host pointers.  The caller owns them; the library
 *     never frees or keeps them after the call returns (except d_* buffers
 *     read asynchronously, which must stay valid until the stream work ends).
 *     Caller buffers need only the alignment of their element type: the
 *     kernels read and write them element by element, and whole-vector moves
 *     go through cudaMemcpy into the context's own (256-byte aligned)
 *     workspace, where the vectorised kernels work.
 *   - Every call that launches work enqueues it on the context's stream and
 *     returns without waiting, unless its comment says it synchronises.
 *   - Return value: PICCS_OK (0) or a negative PICCS_E* code; nothing is
 *     thrown across the ABI.  piccs_last_error() gives a message.
 *   - Sizes: M = nx*ny*nz and N = n_views*nu*nv must each be below 2^31.
 */
#ifndef PICCS_H
#define PICCS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PICCS_OK 0
#define PICCS_EINVAL (-1)      /* invalid argument or geometry */
#define PICCS_ENOMEM (-2)      /* not enough device memory (checked first) */
#define PICCS_ENONFINITE (-3)  /* NaN or Inf found in an input */
#define PICCS_EBREAKDOWN (-4)  /* Krylov breakdown (non-positive or NaN scalar) */
#define PICCS_ETIMEOUT (-5)    /* a bounded device wait gave up */
#define PICCS_ECUDA (-6)       /* a CUDA runtime call failed */
#define PICCS_ENOTIMPL (-7)    /* not available in this build */

enum { PICCS_LAYOUT_UV = 0, PICCS_LAYOUT_VU = 1 };

/* Regulariser variants: PICCS (Eq. 3), PIPLE (Eq. 4: lambda^2 ||x - x_p||^2
 * instead of the prior TV term), TV (lambda ignored), CGLS (alpha and lambda
 * ignored: plain CGLS on A x ~ b, the paper's unregularised comparison). */
enum { PICCS_VARIANT_PICCS = 0, PICCS_VARIANT_PIPLE = 1, PICCS_VARIANT_TV = 2,
       PICCS_VARIANT_CGLS = 3 };

/* Weight rule: R1 is the paper's (|g| + tau^2)^(-1/2); R2 is the common
 * (|g|^2 + tau^2)^(-1/4). */
enum { PICCS_WEIGHT_R1 = 0, PICCS_WEIGHT_R2 = 1 };

/* Initial guess: the prior x_p (default), zero, or a caller volume. */
enum { PICCS_X0_PRIOR = 0, PICCS_X0_ZERO = 1, PICCS_X0_USER = 2 };

/* Inner Krylov solver (Sec. 2.3: LSQR, or the mathematically equivalent
 * CGLS).  CGLS: Hestenes-Stiefel recurrences.  LSQR: Golub-Kahan
 * bidiagonalisation of the augmented operator with a Givens QR update; the
 * data residual is kept current through A w, so it takes as many projections
 * as CGLS.  LSQR_REORTH: LSQR with each new v re-orthogonalised against the
 * cycle's earlier ones (classical Gram-Schmidt, twice); the first such
 * reconstruction on a context allocates the basis, (n_inner - 1) * M values
 * per scan (FP32, or BF16 with PICCS_STORAGE_BF16; PICCS_ENOMEM if the device
 * lacks them), keeps it and grows it when a later one needs more; n_inner - 1
 * must not exceed 256. */
enum { PICCS_SOLVER_CGLS = 0, PICCS_SOLVER_LSQR = 1, PICCS_SOLVER_LSQR_REORTH = 2 };

/* Storage precision.  F32: every vector in FP32.  BF16: the measured
 * projections b and the LSQR re-orthogonalisation basis are held in BF16
 * (rounded to nearest even once, when stored); rays still accumulate in FP32,
 * the recurrence vectors (residuals, search directions, iterates) stay FP32
 * and every inner product and Krylov scalar is FP64.  FP32 input is rounded
 * on the device; piccs_stage_bf16 takes BF16 data directly. */
enum { PICCS_STORAGE_F32 = 0, PICCS_STORAGE_BF16 = 1 };

typedef struct {
    int nx, ny, nz;            /* voxels */
    double vx, vy, vz;         /* voxel size, mm (> 0) */
    int nu, nv;                /* detector pixels */
    double du, dv;             /* detector pitch, mm (> 0) */
    double dso, dsd;           /* source-axis and source-detector distance, mm;
                                  the source and the detector must lie outside
                                  the cylinder circumscribing the volume */
    int n_views;               /* >= 1 */
    const double *angles_rad;  /* host array of n_views angles; copied */
    int proj_layout;           /* PICCS_LAYOUT_UV or PICCS_LAYOUT_VU */
    double u_offset;           /* detector shift along u, mm (finite; 0 = centred):
                                  an offset detector, as on C-arms that widen the
                                  field of view with a half-fan scan */
} piccs_geometry;

typedef struct {
    float alpha, lambda;       /* regularisation parameters (>= 0), Eq. 3 */
    float tau;                 /* smoothing parameter (> 0), the weight equation */
    int n_outer;               /* IRN reweighting cycles (>= 1) */
    int n_inner;               /* Krylov iterations per cycle (>= 0);
                                  total iterations = n_outer * n_inner */
    int x0_mode;               /* PICCS_X0_* */
    int variant;               /* PICCS_VARIANT_* */
    int weight_rule;           /* PICCS_WEIGHT_* */
    int solver;                /* PICCS_SOLVER_* */
    int storage;               /* PICCS_STORAGE_* */
} piccs_params;

/* What the last reconstruction did (filled by piccs_report, which waits). */
typedef struct {
    int status;                /* PICCS_OK, PICCS_EBREAKDOWN or PICCS_ENONFINITE */
    int iterations_run;        /* inner iterations that changed x */
    int n_history;             /* entries written to gamma_history */
    double gamma_history[512]; /* ||A~^T r~||^2 at the start of each cycle and
                                  after every inner iteration, in order, except
                                  where it would cost a backprojection nothing
                                  else needs: after the reconstruction's last
                                  iteration (CGLS), after each cycle's last
                                  iteration (LSQR) */
} piccs_stats;

/* Kernel accounting of a context (see piccs_profile_enable). */
enum { PICCS_KERNEL_FORWARD = 0, PICCS_KERNEL_ADJOINT = 1, PICCS_KERNEL_REG = 2,
       PICCS_KERNEL_VECTOR = 3, PICCS_KERNEL_SCALAR = 4, PICCS_KERNEL_CLASSES = 5 };

typedef struct {
    long long launches[PICCS_KERNEL_CLASSES]; /* kernels launched per class */
    double total_ms[PICCS_KERNEL_CLASSES];    /* summed device time per class (only
                                                 while timing is enabled, else 0) */
    long long total_launches;                 /* all kernels of this library */
    long long calls[PICCS_KERNEL_CLASSES];    /* operator applications per class: one
                                                 per timed interval of total_ms (a
                                                 backprojection A^T is one call of two
                                                 kernels, ray scaling and gather) */
} piccs_profile;

typedef struct piccs_ctx piccs_ctx;

/* Create a context for one scanner geometry: validates it, copies it,
 * checks device memory for the reconstruction workspace (PICCS_ENOMEM before
 * any allocation), allocates the workspace on the current device and
 * uploads the per-view ray tables.  cuda_stream is a cudaStream_t (NULL =
 * legacy default stream).  Synchronises.  The forward projector's walk is
 * chosen here: for a volume larger than the device's L2 it loads the ray's
 * cell table one entry ahead (the same sums); the environment variable
 * PICCS_FORWARD_AHEAD=0 or 1, read at creation, overrides that choice.
 * Paper: Sec. 3 (one geometry per scanning procedure, repeated scans of the
 * same patient). */
int piccs_create(piccs_ctx **out, const piccs_geometry *geometry, void *cuda_stream);

/* Create a context that reconstructs `batch` scans of the same geometry
 * together (1 <= batch <= 64): every kernel of a reconstruction step runs
 * once for all of them, each scan in its own slot of the workspace with its
 * own prior, Krylov scalars and stopping.  All buffers the batched calls
 * take are the batch's arrays back to back: priors, initial and output
 * volumes batch x M floats, projections batch x N floats.  piccs_create is
 * batch 1.  Paper: Sec. 3 (a patient is scanned repeatedly with one geometry;
 * scans from several procedures on one scanner share it too). */
int piccs_create_batched(piccs_ctx **out, const piccs_geometry *geometry, int batch,
                         void *cuda_stream);

/* Free the context and its device memory (synchronises its stream). */
void piccs_destroy(piccs_ctx *ctx);

/* Message for the last failing call on ctx (or of piccs_create when ctx is
 * NULL, per thread).  Valid until the next call on the same context. */
const char *piccs_last_error(const piccs_ctx *ctx);

/* Change the stream later calls enqueue on. */
int piccs_set_stream(piccs_ctx *ctx, void *cuda_stream);

/* Device bytes piccs_create allocates for this geometry (params may be NULL),
 * plus, when params->solver is PICCS_SOLVER_LSQR_REORTH, the basis the first
 * such reconstruction allocates.  Pure host computation; needs no GPU. */
int piccs_query_workspace(const piccs_geometry *geometry, const piccs_params *params,
                          size_t *bytes);

/* The same for a context of `batch` slots (piccs_create_batched). */
int piccs_query_workspace_batched(const piccs_geometry *geometry, const piccs_params *params,
                                  int batch, size_t *bytes);

/* Check a geometry and parameters without creating anything (params may be
 * NULL).  Pure host computation; needs no GPU. */
int piccs_validate(const piccs_geometry *geometry, const piccs_params *params);

/* Copy the prior reconstruction x_p (M floats, device; batch x M in a
 * batched context) into context-owned memory and check it for NaN/Inf
 * (PICCS_ENONFINITE).  Synchronises.
 * Paper: x_p, the "good initial reconstruction" of Sec. 2.1 and Sec. 3. */
int piccs_set_prior(piccs_ctx *ctx, const float *d_xprior);

/* IRN-PICCS reconstruction (Sec. 2.3): writes M floats to d_vol_out.
 * d_proj: N measured log projections b in the context layout.  d_x0: initial
 * volume when params->x0_mode == PICCS_X0_USER, else ignored (may be NULL).
 * The prior must have been set unless variant is TV or CGLS with x0 != PRIOR.
 * Asynchronous: the Krylov scalars stay on the device; breakdown or a NaN/Inf
 * in d_proj is reported by piccs_report. */
int piccs_reconstruct(piccs_ctx *ctx, const float *d_proj, const piccs_params *params,
                      const float *d_x0, float *d_vol_out);

/* Same with host buffers: copies h_proj (and h_x0) to the device, runs
 * piccs_reconstruct and copies the volume back to h_vol_out.  Synchronises;
 * returns the device status (PICCS_EBREAKDOWN, PICCS_ENONFINITE) too. */
int piccs_reconstruct_host(piccs_ctx *ctx, const float *h_proj, const piccs_params *params,
                           const float *h_x0, float *h_vol_out);

/* Wait for the context's stream and describe the last reconstruction (of
 * slot 0 in a batched context). */
int piccs_report(piccs_ctx *ctx, piccs_stats *out);

/* The same for slot `slot` (0 <= slot < batch) of a batched context. */
int piccs_report_slot(piccs_ctx *ctx, int slot, piccs_stats *out);

/* Staged reconstructions: the building blocks of a request loop that keeps a
 * context per patient resident and feeds it scans as they arrive.
 * piccs_set_prior_broadcast copies one prior volume (host or device, M
 * floats) into every slot and checks it (synchronises).  piccs_stage copies
 * one scan's projections (N floats, host or device) into slot `slot`'s
 * staging buffer; piccs_run_staged reconstructs slots 0 .. nactive-1 from
 * their staged projections (x0_mode PRIOR or ZERO); piccs_unstage copies slot
 * `slot`'s volume out.  All three are asynchronous on the context's stream
 * (host buffers should be pinned).  use_graph != 0: the launch sequence of a
 * (params, nactive) pair is captured once as a CUDA graph (on a private
 * stream; the legacy default stream cannot be captured) and replayed on the
 * context's stream -- the per-step scalars stay on the device, so a replay is
 * a full reconstruction; growing the LSQR basis drops the captured graphs.
 * Not with profiling timing on (piccs_profile_enable), which launches
 * kernel by kernel. */
int piccs_set_prior_broadcast(piccs_ctx *ctx, const float *xprior, int from_host);
int piccs_stage(piccs_ctx *ctx, int slot, const float *proj, int from_host);
/* The same with projections already in BF16 (N values, bfloat16 bit
 * patterns); the run must then use PICCS_STORAGE_BF16. */
int piccs_stage_bf16(piccs_ctx *ctx, int slot, const void *proj, int from_host);
int piccs_run_staged(piccs_ctx *ctx, int nactive, const piccs_params *params, int use_graph);

/* The staged reconstructions of several contexts -- scans of different
 * geometries, e.g. of different patients -- run together (Sec. 3's repeated
 * scans of several patients served at once): the same steps in lockstep, every
 * product with A and with A^T one kernel launch for all of them (their CTA
 * index spaces concatenated, each CTA finding its scan in a by-value table of
 * geometries and buffers), every other kernel per context.  ctxs[i] runs its
 * first nactive[i] staged slots, all with `params`; 1 <= n <= 8, distinct
 * contexts on one device.  Each result is bit for bit the one
 * piccs_run_staged gives that context alone.  The work is enqueued on
 * ctxs[0]'s stream, after everything already enqueued on the others'
 * streams (their staging copies); their streams then wait for it (their
 * unstaging copies).  use_graph: one CUDA graph per (contexts, nactive,
 * params), kept by ctxs[0] (captured as in piccs_run_staged); a group's
 * kernels are counted in ctxs[0]'s profile.  Errors: PICCS_EINVAL (bad
 * arguments, a member's staged data or prior), PICCS_ENOMEM (a member's
 * basis), PICCS_ECUDA; the message is on ctxs[0]. */
int piccs_run_staged_group(piccs_ctx *const *ctxs, const int *nactive, int n,
                           const piccs_params *params, int use_graph);
int piccs_unstage(piccs_ctx *ctx, int slot, float *vol, int to_host);

/* Forward projection d_proj = A d_vol (Eq. 1): N floats from M floats (each
 * of the batch's volumes in a batched context, one launch per volume). */
int piccs_forward(piccs_ctx *ctx, const float *d_vol, float *d_proj);

/* Matched backprojection d_vol = A^T d_proj (same ray/voxel weights as
 * piccs_forward): M floats from N floats (per volume of a batched context).
 * Needed by every Krylov step
 * (Sec. 2.3, the text after the augmented system). */
int piccs_adjoint(piccs_ctx *ctx, const float *d_proj, float *d_vol);

/* The reweighting step of one IRN cycle (Eqs. 10-11): from the current
 * iterate d_x and the prior (slot 0's in a batched context), writes per voxel
 *   d_omega = alpha^2 w1^2 + lambda^2 w2^2      (PICCS; alpha^2 w1^2 otherwise)
 *   d_c     = lambda^2 D^T W2^2 D x_p           (PICCS; lambda^2 x_p for PIPLE;
 *                                                0 for TV and CGLS)
 * with w1 = W(D x), w2 = W(D x - D x_p).  M floats each. */
int piccs_reg_weights(piccs_ctx *ctx, const float *d_x, const piccs_params *params,
                      float *d_omega, float *d_c);

/* Regularisation block of the normal operator of the augmented system:
 *   d_out = D^T diag(omega) D d_z   (+ lambda^2 d_z for PIPLE)
 * and *h_rho = sum_i omega_i |(D z)_i|^2 (+ lambda^2 |z|^2 for PIPLE), i.e.
 * ||[alpha W1 D; lambda W2 D] z||^2.  M floats.  Synchronises (h_rho may be
 * NULL, then it does not). */
int piccs_reg_normal(piccs_ctx *ctx, const float *d_omega, const piccs_params *params,
                     const float *d_z, float *d_out, double *h_rho);

/* Reset the context's kernel accounting and switch per-launch device timing
 * on (timing != 0) or off.  With timing on, every kernel launch is bracketed
 * by two CUDA events on the context's stream; launches are always counted. */
int piccs_profile_enable(piccs_ctx *ctx, int timing);

/* Wait for the context's stream and read the accounting since the last
 * piccs_profile_enable.  Synchronises. */
int piccs_profile_read(piccs_ctx *ctx, piccs_profile *out);

/* Allocation-free form of piccs_reg_normal for callers that cannot allocate
 * device memory -- code living inside a host application whose memory pool
 * owns the whole GPU under a hard cap, or a latency-critical loop where a
 * cudaMalloc/cudaFree would synchronise the device.  It needs no context:
 * it computes d_out = D^T diag(d_omega) D d_z + lambda2_piple * d_z and
 * *d_rho = sum_i omega_i |(D z)_i|^2 + lambda2_piple |z|^2 for an nx*ny*nz
 * z-fastest FP32 volume (lambda2_piple = lambda^2 for PIPLE, else 0), on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream).  d_omega, d_z,
 * d_out (M floats) and d_rho (one double) are caller-owned device buffers.
 * The paper has no counterpart to this entry point.
 *   Scratch: the per-CTA FP64 partial sums live in a 32 KiB (4096 doubles)
 *   array inside libpiccs that every GPU loading the library holds until
 *   exit; volumes of any size up to 2^31-1 voxels use at most 1216 entries,
 *   larger ones are rejected with PICCS_EINVAL.  Nothing is allocated or
 *   freed (no cudaMalloc, cudaFree or allocating library routine).
 *   The first call on a device looks up the array's device address on that
 *   device (cudaGetSymbolAddress) and keeps it for the life of the process;
 *   make that first call before any stream capture.  A cudaDeviceReset of
 *   that device invalidates the kept address: do not call this entry point
 *   on a device after resetting it.  All calls share the array and it keeps the last call's
 *   contents (every call overwrites what it reads, so nothing needs
 *   clearing); calls whose kernels overlap on the GPU, e.g. from two
 *   streams, race on it and must be serialised by the caller.
 *   Errors: PICCS_EINVAL / PICCS_ECUDA, message via piccs_last_error(NULL).
 *   Asynchronous with respect to the host. */
int piccs_reg_normal_noalloc(int nx, int ny, int nz, const float *d_omega,
                             float lambda2_piple, const float *d_z, float *d_out,
                             double *d_rho, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PICCS_H */
