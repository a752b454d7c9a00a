// Host side of libpiccs: the C ABI of include/piccs.h.
//
// It validates arguments, builds the per-view ray tables in FP64, owns the
// device workspace and enqueues the IRN-PICCS iteration (Sec. 2.3) on the
// context's stream.  Every step of the arithmetic runs in the CUDA kernels of
// this library; the host only orders launches.  The Krylov scalars stay on
// the device, so a whole reconstruction is enqueued without a round trip.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <string>
#include <vector>

#include "../../include/piccs.h"
#include "internal.h"
#include "ray_tables.h"

using namespace piccs;

struct piccs_ctx {
    piccs_geometry geo;           // angles_rad points into `angles`
    std::vector<double> angles;
    ProjGeom pg;
    VolDims vd;
    long long M = 0, N = 0;
    int nslot = 1;              // scans per batch (same geometry)
    int nactive = 1;            // slots the current call works on (a prefix)
    size_t slot_bytes = 0;      // stride between the slots' workspaces
    cudaStream_t stream = nullptr;
    int device = 0;
    bool has_prior = false;
    std::string err;

    // device workspace (one allocation, carved up)
    void *base = nullptr;
    size_t bytes = 0;
    ColParams *cols = nullptr;
    float2 *vr = nullptr;
    int4 *cells = nullptr;
    int *hit_ptr = nullptr;
    CellHit *hits = nullptr;
    float *xprior = nullptr, *x = nullptr, *p = nullptr, *s = nullptr, *g = nullptr,
          *t = nullptr, *omega = nullptr, *c = nullptr, *w2sq = nullptr;
    float *r = nullptr, *q = nullptr, *bstage = nullptr, *rs = nullptr, *aw = nullptr;
    double *part_fwd = nullptr, *part_vol = nullptr, *part_vec = nullptr;
    int n_part_fwd = 0, n_part_vol = 0, n_part_vec = 0;
    KrylovScalars *ks = nullptr;
    LsqrScalars *ls = nullptr;
    // LSQR re-orthogonalisation basis, allocated on first use: per slot the
    // vectors, then the Gram-Schmidt partial sums, basis_bytes apart
    void *basis = nullptr;  // FP32 or BF16 vectors, by the run's storage
    double *part_dots = nullptr;
    size_t basis_stride = 0;
    std::vector<char> staged16;  // slot's staged projections are BF16
    int *flag = nullptr;
    double *dsum = nullptr;

    // CUDA graphs of staged reconstructions, by (params, active slots)
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        long long launches[PICCS_KERNEL_CLASSES] = {};
        long long calls[PICCS_KERNEL_CLASSES] = {};
    };
    std::map<std::string, GraphEntry> graphs;
    long long graph_launches = 0;
    cudaStream_t cap_stream = nullptr;  // captures run here (the legacy stream cannot capture)
    long long uid = 0;        // unique per context of the process (keys of group graphs)
    long long basis_gen = 0;  // incremented whenever the basis is reallocated
    // kernel accounting
    bool timing = false;
    long long launches[PICCS_KERNEL_CLASSES] = {};
    long long calls[PICCS_KERNEL_CLASSES] = {};
    double total_ms[PICCS_KERNEL_CLASSES] = {};
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

thread_local std::string g_create_err;

int set_err(piccs_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_err = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                               \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_err((ctx), PICCS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

cudaEvent_t take_event(piccs_ctx *ctx)
{
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Counts one operator call of class `kind` (its kernel launches and the call
// itself) and, with timing on, brackets it with two events on the context's
// stream.
struct Launch {
    piccs_ctx *ctx;
    int kind;
    cudaEvent_t a = nullptr;
    Launch(piccs_ctx *c, int k) : ctx(c), kind(k)
    {
        // the backprojection is two kernels (ray scaling, gather)
        ctx->launches[kind] += kind == PICCS_KERNEL_ADJOINT ? 2 : 1;
        ctx->calls[kind] += 1;
        if (ctx->timing) {
            a = take_event(ctx);
            if (a) cudaEventRecord(a, ctx->stream);
        }
    }
    ~Launch()
    {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            if (b) {
                cudaEventRecord(b, ctx->stream);
                ctx->pending.push_back({kind, a, b});
            } else {
                ctx->event_pool.push_back(a);
            }
        }
    }
};

// all slots of the context in one launch
#define SL(ctx) Slots{(ctx)->nactive, (long long)(ctx)->slot_bytes}

#define LAUNCH(ctx, kind, call)                          \
    do {                                                 \
        Launch l_((ctx), (kind));                        \
        CUDA_TRY((ctx), (call));                         \
    } while (0)

int check_geometry(const piccs_geometry *g, char *why, size_t n)
{
    if (!g) { snprintf(why, n, "geometry is NULL"); return PICCS_EINVAL; }
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0) { snprintf(why, n, "volume size must be positive"); return PICCS_EINVAL; }
    if (g->nu <= 0 || g->nv <= 0) { snprintf(why, n, "detector size must be positive"); return PICCS_EINVAL; }
    if (g->n_views <= 0) { snprintf(why, n, "n_views must be positive"); return PICCS_EINVAL; }
    // sizes below 1e-4 mm would push the FP32 crossing parameters out of range
    if (!finite_pos(g->vx) || !finite_pos(g->vy) || !finite_pos(g->vz) || g->vx < 1e-4 || g->vy < 1e-4 || g->vz < 1e-4) { snprintf(why, n, "voxel size must be finite and >= 1e-4 mm"); return PICCS_EINVAL; }
    if (!finite_pos(g->du) || !finite_pos(g->dv) || g->du < 1e-4 || g->dv < 1e-4) { snprintf(why, n, "detector pitch must be finite and >= 1e-4 mm"); return PICCS_EINVAL; }
    if (!std::isfinite(g->u_offset)) { snprintf(why, n, "u_offset must be finite"); return PICCS_EINVAL; }
    if (!(g->dsd < 1e7)) { snprintf(why, n, "dsd must be below 1e7 mm"); return PICCS_EINVAL; }
    const double M = (double)g->nx * g->ny * g->nz;
    const double N = (double)g->n_views * g->nu * g->nv;
    if (M >= 2147483648.0) { snprintf(why, n, "nx*ny*nz = %.0f exceeds 2^31-1", M); return PICCS_EINVAL; }
    if (N >= 2147483648.0) { snprintf(why, n, "n_views*nu*nv = %.0f exceeds 2^31-1", N); return PICCS_EINVAL; }
    if (!g->angles_rad) { snprintf(why, n, "angles_rad is NULL"); return PICCS_EINVAL; }
    for (int j = 0; j < g->n_views; ++j)
        if (!std::isfinite(g->angles_rad[j])) { snprintf(why, n, "angle %d is not finite", j); return PICCS_EINVAL; }
    if (g->n_views > 32767 || g->nu > 65535) { snprintf(why, n, "n_views must be <= 32767 and nu <= 65535"); return PICCS_EINVAL; }
    if ((double)g->n_views * g->nu * (g->nx + g->ny - 1) >= 2147483648.0) { snprintf(why, n, "ray tables would exceed 2^31 entries"); return PICCS_EINVAL; }
    if (g->proj_layout != PICCS_LAYOUT_UV && g->proj_layout != PICCS_LAYOUT_VU) { snprintf(why, n, "unknown proj_layout %d", g->proj_layout); return PICCS_EINVAL; }
    const double R = 0.5 * std::sqrt((g->nx * g->vx) * (g->nx * g->vx) + (g->ny * g->vy) * (g->ny * g->vy));
    if (!std::isfinite(g->dso) || !(g->dso > R)) { snprintf(why, n, "dso=%g must exceed the volume's circumscribed radius %g", g->dso, R); return PICCS_EINVAL; }
    if (!std::isfinite(g->dsd) || !(g->dsd - g->dso > R)) { snprintf(why, n, "dsd-dso=%g must exceed the volume's circumscribed radius %g", g->dsd - g->dso, R); return PICCS_EINVAL; }
    return PICCS_OK;
}

int check_params(const piccs_params *p, char *why, size_t n)
{
    if (!p) { snprintf(why, n, "params is NULL"); return PICCS_EINVAL; }
    if (!std::isfinite(p->alpha) || p->alpha < 0.f) { snprintf(why, n, "alpha must be finite and >= 0"); return PICCS_EINVAL; }
    if (!std::isfinite(p->lambda) || p->lambda < 0.f) { snprintf(why, n, "lambda must be finite and >= 0"); return PICCS_EINVAL; }
    if (!std::isfinite(p->tau) || !(p->tau > 0.f)) { snprintf(why, n, "tau must be finite and > 0"); return PICCS_EINVAL; }
    if (p->n_outer < 1 || p->n_inner < 0) { snprintf(why, n, "need n_outer >= 1 and n_inner >= 0"); return PICCS_EINVAL; }
    if ((long long)p->n_outer * (p->n_inner + 1) > 512) { snprintf(why, n, "n_outer*(n_inner+1) must be <= 512"); return PICCS_EINVAL; }
    if (p->variant < 0 || p->variant > 3) { snprintf(why, n, "unknown variant %d", p->variant); return PICCS_EINVAL; }
    if (p->weight_rule < 0 || p->weight_rule > 1) { snprintf(why, n, "unknown weight_rule %d", p->weight_rule); return PICCS_EINVAL; }
    if (p->x0_mode < 0 || p->x0_mode > 2) { snprintf(why, n, "unknown x0_mode %d", p->x0_mode); return PICCS_EINVAL; }
    if (p->solver < 0 || p->solver > 2) { snprintf(why, n, "unknown solver %d", p->solver); return PICCS_EINVAL; }
    if (p->solver == PICCS_SOLVER_LSQR_REORTH && p->n_inner - 1 > kMaxBasis) { snprintf(why, n, "LSQR_REORTH needs n_inner - 1 <= %d", kMaxBasis); return PICCS_EINVAL; }
    if (p->storage != PICCS_STORAGE_F32 && p->storage != PICCS_STORAGE_BF16) { snprintf(why, n, "unknown storage %d", p->storage); return PICCS_EINVAL; }
    return PICCS_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Workspace: the ray tables (shared by all slots), then one equal-sized
// region per slot holding that scan's vectors, partial sums and scalars.
struct Layout {
    size_t off_cols, off_vr, off_cells, off_hitptr, off_hits, off_slot0;
    // within a slot
    size_t off_img[9], off_r, off_q, off_b, off_rs, off_aw, off_pf, off_pv, off_pvec, off_ks,
        off_ls, off_flag, off_dsum, slot_bytes;
    size_t total;
    int n_pf, n_pv, n_pvec;
};

Layout plan(const piccs_geometry *g, int nslot = 1)
{
    Layout L{};
    const size_t M = (size_t)g->nx * g->ny * g->nz;
    const size_t N = (size_t)g->n_views * g->nu * g->nv;
    ProjGeom pg{};
    pg.nx = g->nx; pg.ny = g->ny; pg.nz = g->nz; pg.nu = g->nu; pg.nv = g->nv; pg.n_views = g->n_views;
    L.n_pf = project_blocks(pg);
    L.n_pv = stencil_blocks((long long)M);
    L.n_pvec = vector_blocks();
    size_t o = 0;
    L.off_cols = o; o += align256((size_t)g->n_views * g->nu * sizeof(ColParams));
    L.off_vr = o; o += align256((size_t)g->nv * sizeof(float2));
    L.off_cells = o; o += align256((size_t)g->n_views * g->nu * cell_stride(g) * 2 * sizeof(int));
    L.off_hitptr = o; o += align256(((size_t)g->nx * g->ny + 1) * sizeof(int));
    L.off_hits = o; o += align256(hit_bound(g) * sizeof(CellHit));
    L.off_slot0 = o;
    size_t q = 0;
    for (int i = 0; i < 9; ++i) { L.off_img[i] = q; q += align256(M * sizeof(float)); }
    L.off_r = q; q += align256(N * sizeof(float));
    L.off_q = q; q += align256(N * sizeof(float));
    L.off_b = q; q += align256(N * sizeof(float));
    L.off_rs = q; q += align256((size_t)adjoint_rs_floats((long long)N, (long long)g->n_views * g->nu) * sizeof(float));
    L.off_aw = q; q += align256(N * sizeof(float));
    L.off_pf = q; q += align256((size_t)L.n_pf * sizeof(double));
    L.off_pv = q; q += align256(3 * (size_t)L.n_pv * sizeof(double));  // up to 3 sums per pass
    L.off_pvec = q; q += align256((size_t)L.n_pvec * sizeof(double));
    L.off_ks = q; q += align256(sizeof(KrylovScalars));
    L.off_ls = q; q += align256(sizeof(LsqrScalars));
    L.off_flag = q; q += align256(sizeof(int));
    L.off_dsum = q; q += align256(sizeof(double));
    L.slot_bytes = q;
    L.total = o + (size_t)nslot * q;
    return L;
}

constexpr int kMaxSlots = 64;

template <class T>
T *slot_at(T *p, const piccs_ctx *ctx, int s)
{
    return reinterpret_cast<T *>(reinterpret_cast<char *>(p) + (size_t)s * ctx->slot_bytes);
}

// LSQR re-orthogonalisation: n_inner - 1 basis vectors (the last step of a
// cycle needs none) and the Gram-Schmidt partial sums
size_t basis_vectors(int n_inner) { return n_inner > 1 ? (size_t)(n_inner - 1) : 0; }

size_t basis_vec_bytes(const piccs_geometry *g, int n_inner, int storage)
{
    const size_t M = (size_t)g->nx * g->ny * g->nz;
    const size_t nv = basis_vectors(n_inner) > 0 ? basis_vectors(n_inner) : 1;
    const size_t es = storage == PICCS_STORAGE_BF16 ? 2 : sizeof(float);
    return align256(nv * (size_t)lsqr_basis_stride((long long)M) * es);
}

// Gram-Schmidt partial sums of one slot (a fixed size)
size_t basis_dots_bytes() { return align256((size_t)kMaxBasis * lsqr_dot_blocks() * sizeof(double)); }

// per slot: the Gram-Schmidt partial sums, then the vectors (FP32 or BF16), so
// that a region sized for one (n_inner, storage) serves every smaller one
size_t basis_bytes(const piccs_geometry *g, int n_inner, int storage)
{
    return basis_dots_bytes() + basis_vec_bytes(g, n_inner, storage);
}

}  // namespace

void piccs::set_thread_error(const char *msg) { g_create_err = msg ? msg : ""; }

extern "C" {

const char *piccs_last_error(const piccs_ctx *ctx)
{
    if (ctx) return ctx->err.c_str();
    return g_create_err.c_str();
}

int piccs_validate(const piccs_geometry *geometry, const piccs_params *params)
{
    char why[256];
    int rc = check_geometry(geometry, why, sizeof why);
    if (rc == PICCS_OK && params) rc = check_params(params, why, sizeof why);
    if (rc != PICCS_OK) return set_err(nullptr, rc, "%s", why);
    return PICCS_OK;
}

int piccs_query_workspace_batched(const piccs_geometry *geometry, const piccs_params *params,
                                  int batch, size_t *bytes)
{
    int rc = piccs_validate(geometry, params);
    if (rc != PICCS_OK) return rc;
    if (!bytes) return set_err(nullptr, PICCS_EINVAL, "bytes is NULL");
    if (batch < 1 || batch > kMaxSlots) return set_err(nullptr, PICCS_EINVAL, "batch must be in [1, %d]", kMaxSlots);
    *bytes = plan(geometry, batch).total;
    if (params && params->solver == PICCS_SOLVER_LSQR_REORTH)
        *bytes += (size_t)batch * basis_bytes(geometry, params->n_inner, params->storage);
    return PICCS_OK;
}

int piccs_query_workspace(const piccs_geometry *geometry, const piccs_params *params,
                          size_t *bytes)
{
    return piccs_query_workspace_batched(geometry, params, 1, bytes);
}

int piccs_create(piccs_ctx **out, const piccs_geometry *geometry, void *cuda_stream)
{
    return piccs_create_batched(out, geometry, 1, cuda_stream);
}

int piccs_create_batched(piccs_ctx **out, const piccs_geometry *geometry, int batch,
                         void *cuda_stream)
{
    if (!out) return set_err(nullptr, PICCS_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = piccs_validate(geometry, nullptr);
    if (rc != PICCS_OK) return rc;
    if (batch < 1 || batch > kMaxSlots) return set_err(nullptr, PICCS_EINVAL, "batch must be in [1, %d]", kMaxSlots);
    const Layout L = plan(geometry, batch);

    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess)
        return set_err(nullptr, PICCS_ECUDA, "cudaMemGetInfo failed: %s", cudaGetErrorString(e));
    if (L.total + (64u << 20) > free_b)
        return set_err(nullptr, PICCS_ENOMEM, "workspace needs %zu bytes, %zu free", L.total, free_b);

    piccs_ctx *ctx = new (std::nothrow) piccs_ctx();
    if (!ctx) return set_err(nullptr, PICCS_ENOMEM, "host allocation failed");
    static std::atomic<long long> next_uid{1};
    ctx->uid = next_uid.fetch_add(1);
    ctx->geo = *geometry;
    ctx->angles.assign(geometry->angles_rad, geometry->angles_rad + geometry->n_views);
    ctx->geo.angles_rad = ctx->angles.data();
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&ctx->device);
    const piccs_geometry &g = ctx->geo;
    ctx->M = (long long)g.nx * g.ny * g.nz;
    ctx->N = (long long)g.n_views * g.nu * g.nv;
    ctx->pg.nx = g.nx; ctx->pg.ny = g.ny; ctx->pg.nz = g.nz;
    ctx->pg.nu = g.nu; ctx->pg.nv = g.nv; ctx->pg.n_views = g.n_views;
    if (g.proj_layout == PICCS_LAYOUT_UV) {
        ctx->pg.sv = 1; ctx->pg.su = g.nv;
    } else {
        ctx->pg.su = 1; ctx->pg.sv = g.nu;
    }
    ctx->pg.sj = (long long)g.nu * g.nv;
    ctx->pg.halfnz = 0.5f * (float)g.nz;
    ctx->pg.rdv = (float)(1.0 / g.dv);
    ctx->pg.cv = 0.5f * (float)(g.nv - 1);
    ctx->pg.sv32 = (int)ctx->pg.sv;
    {
        // Consecutive z planes lie vz D / |v| apart in xy distance along a row
        // of height v (D >= DSD the source-to-pixel xy distance); if that
        // exceeds the longest xy cell (the voxel's diagonal) for the steepest
        // row, with a margin far above FP32 rounding, no cell holds two
        // crossings of a row and the forward walk takes one crossing step per
        // cell.
        const double vmax = 0.5 * (g.nv - 1) * g.dv;
        const double diag = std::sqrt(g.vx * g.vx + g.vy * g.vy);
        ctx->pg.multi = vmax > 0.0 && g.vz * g.dsd <= 1.01 * diag * vmax ? 1 : 0;
        ctx->pg.rows_per_layer = (float)(g.vz * g.dsd / (g.dso * g.dv));
        // A volume larger than the L2 makes the walk's cell-table loads miss:
        // the forward then loads the table one entry ahead (the same sums).
        // PICCS_FORWARD_AHEAD=0/1 overrides the choice (tuning and tests).
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            l2 = 0;
        }
        ctx->pg.ahead = l2 > 0 && (double)ctx->M * sizeof(float) > (double)l2 ? 1 : 0;
        if (const char *ov = std::getenv("PICCS_FORWARD_AHEAD"))
            if (ov[0] == '0' || ov[0] == '1') ctx->pg.ahead = ov[0] - '0';
    }
    ctx->vd = VolDims{g.nx, g.ny, g.nz};

    e = cudaMalloc(&ctx->base, L.total);
    if (e != cudaSuccess) {
        delete ctx;
        return set_err(nullptr, PICCS_ENOMEM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
    }
    ctx->bytes = L.total;
    char *b = static_cast<char *>(ctx->base);
    ctx->cols = reinterpret_cast<ColParams *>(b + L.off_cols);
    ctx->vr = reinterpret_cast<float2 *>(b + L.off_vr);
    ctx->cells = reinterpret_cast<int4 *>(b + L.off_cells);
    ctx->hit_ptr = reinterpret_cast<int *>(b + L.off_hitptr);
    ctx->hits = reinterpret_cast<CellHit *>(b + L.off_hits);
    ctx->nslot = batch;
    ctx->nactive = batch;
    ctx->staged16.assign(batch, 0);
    ctx->slot_bytes = L.slot_bytes;
    b += L.off_slot0;  // slot 0; slot s is s * slot_bytes further
    float **img[9] = {&ctx->xprior, &ctx->x, &ctx->p, &ctx->s, &ctx->g,
                      &ctx->t, &ctx->omega, &ctx->c, &ctx->w2sq};
    for (int i = 0; i < 9; ++i) *img[i] = reinterpret_cast<float *>(b + L.off_img[i]);
    ctx->r = reinterpret_cast<float *>(b + L.off_r);
    ctx->q = reinterpret_cast<float *>(b + L.off_q);
    ctx->bstage = reinterpret_cast<float *>(b + L.off_b);
    ctx->rs = reinterpret_cast<float *>(b + L.off_rs);
    ctx->aw = reinterpret_cast<float *>(b + L.off_aw);
    ctx->part_fwd = reinterpret_cast<double *>(b + L.off_pf);
    ctx->part_vol = reinterpret_cast<double *>(b + L.off_pv);
    ctx->part_vec = reinterpret_cast<double *>(b + L.off_pvec);
    ctx->n_part_fwd = L.n_pf;
    ctx->n_part_vol = L.n_pv;
    ctx->n_part_vec = L.n_pvec;
    ctx->ks = reinterpret_cast<KrylovScalars *>(b + L.off_ks);
    ctx->ls = reinterpret_cast<LsqrScalars *>(b + L.off_ls);
    ctx->flag = reinterpret_cast<int *>(b + L.off_flag);
    ctx->dsum = reinterpret_cast<double *>(b + L.off_dsum);

    std::vector<ColParams> cols;
    std::vector<float2> vr;
    std::vector<int> cells, hit_ptr;
    std::vector<CellHit> hits;
    build_tables(&g, cols, vr, cells, hit_ptr, hits);
    e = cudaMemcpy(ctx->cols, cols.data(), cols.size() * sizeof(ColParams), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->vr, vr.data(), vr.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->cells, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->hit_ptr, hit_ptr.data(), hit_ptr.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hits.empty())
        e = cudaMemcpy(ctx->hits, hits.data(), hits.size() * sizeof(CellHit), cudaMemcpyHostToDevice);
    for (int sl = 0; sl < batch && e == cudaSuccess; ++sl) {
        e = cudaMemset(reinterpret_cast<char *>(ctx->ks) + sl * L.slot_bytes, 0, sizeof(KrylovScalars));
        if (e == cudaSuccess)
            e = cudaMemset(reinterpret_cast<char *>(ctx->ls) + sl * L.slot_bytes, 0, sizeof(LsqrScalars));
    }
    if (e != cudaSuccess) {
        cudaFree(ctx->base);
        delete ctx;
        return set_err(nullptr, PICCS_ECUDA, "table upload failed: %s", cudaGetErrorString(e));
    }
    *out = ctx;
    return PICCS_OK;
}

void piccs_destroy(piccs_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second.exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaFree(ctx->part_dots);  // the basis region starts with the partial sums
    cudaFree(ctx->base);
    delete ctx;
}

int piccs_profile_enable(piccs_ctx *ctx, int timing)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto &p : ctx->pending) {
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < PICCS_KERNEL_CLASSES; ++k) {
        ctx->launches[k] = 0;
        ctx->calls[k] = 0;
        ctx->total_ms[k] = 0.0;
    }
    ctx->timing = timing != 0;
    return PICCS_OK;
}

int piccs_profile_read(piccs_ctx *ctx, piccs_profile *out)
{
    if (!ctx || !out) return set_err(ctx, PICCS_EINVAL, "NULL argument");
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto &p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) ctx->total_ms[p.kind] += ms;
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
    std::memset(out, 0, sizeof *out);
    for (int k = 0; k < PICCS_KERNEL_CLASSES; ++k) {
        out->launches[k] = ctx->launches[k];
        out->calls[k] = ctx->calls[k];
        out->total_ms[k] = ctx->total_ms[k];
        out->total_launches += ctx->launches[k];
    }
    return PICCS_OK;
}

int piccs_set_stream(piccs_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return PICCS_OK;
}

int piccs_set_prior(piccs_ctx *ctx, const float *d_xprior)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    if (!d_xprior) return set_err(ctx, PICCS_EINVAL, "d_xprior is NULL");
    const int B = ctx->nactive = ctx->nslot;
    const size_t vb = ctx->M * sizeof(float);
    CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->xprior, ctx->slot_bytes, d_xprior, vb, vb, B,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaMemset2DAsync(ctx->flag, ctx->slot_bytes, 0, sizeof(int), B, ctx->stream));
    LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_count_nonfinite(ctx->M, ctx->xprior, ctx->flag, ctx->stream, SL(ctx)));
    std::vector<int> bad(B, 0);
    CUDA_TRY(ctx, cudaMemcpy2DAsync(bad.data(), sizeof(int), ctx->flag, ctx->slot_bytes, sizeof(int), B,
                                    cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < B; ++i)
        if (bad[i]) {
            ctx->has_prior = false;
            return set_err(ctx, PICCS_ENONFINITE, "prior volume %d holds NaN or Inf", i);
        }
    ctx->has_prior = true;
    return PICCS_OK;
}

int piccs_forward(piccs_ctx *ctx, const float *d_vol, float *d_proj)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    if (!d_vol || !d_proj) return set_err(ctx, PICCS_EINVAL, "NULL buffer");
    for (int b = 0; b < ctx->nslot; ++b)
        LAUNCH(ctx, PICCS_KERNEL_FORWARD, launch_forward(ctx->pg, ctx->cols, ctx->vr, ctx->cells, d_vol + b * ctx->M,
                                                         d_proj + b * ctx->N, FWD_PLAIN, nullptr, nullptr, nullptr,
                                                         ctx->stream));
    return PICCS_OK;
}

int piccs_adjoint(piccs_ctx *ctx, const float *d_proj, float *d_vol)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    if (!d_vol || !d_proj) return set_err(ctx, PICCS_EINVAL, "NULL buffer");
    CUDA_TRY(ctx, cudaMemsetAsync(d_vol, 0, ctx->nslot * ctx->M * sizeof(float), ctx->stream));
    for (int b = 0; b < ctx->nslot; ++b)
        LAUNCH(ctx, PICCS_KERNEL_ADJOINT, launch_adjoint(ctx->pg, ctx->cols, ctx->vr, ctx->hit_ptr, ctx->hits,
                                                         d_proj + b * ctx->N, ctx->rs, d_vol + b * ctx->M,
                                                         ctx->stream));
    return PICCS_OK;
}

static float lam2_piple(const piccs_params *p)
{
    return p->variant == PICCS_VARIANT_PIPLE ? p->lambda * p->lambda : 0.f;
}

static int enqueue_weights(piccs_ctx *ctx, const float *d_x, const piccs_params *p, float *omega,
                           float *c, Slots sl)
{
    const float a2 = p->alpha * p->alpha, l2 = p->lambda * p->lambda;
    const float tau2 = p->tau * p->tau;
    LAUNCH(ctx, PICCS_KERNEL_REG, launch_weights(ctx->vd, d_x, ctx->xprior, a2, l2, tau2, p->weight_rule,
                                 p->variant, omega, ctx->w2sq, ctx->stream, sl));
    LAUNCH(ctx, PICCS_KERNEL_REG, launch_prior_rhs(ctx->vd, ctx->xprior, ctx->w2sq, l2, p->variant, c, ctx->stream, sl));
    return PICCS_OK;
}

static bool needs_prior(const piccs_params *p)
{
    return p->variant == PICCS_VARIANT_PICCS || p->variant == PICCS_VARIANT_PIPLE ||
           p->x0_mode == PICCS_X0_PRIOR;
}

int piccs_reg_weights(piccs_ctx *ctx, const float *d_x, const piccs_params *params,
                      float *d_omega, float *d_c)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    char why[256];
    if (check_params(params, why, sizeof why) != PICCS_OK) return set_err(ctx, PICCS_EINVAL, "%s", why);
    if (!d_x || !d_omega || !d_c) return set_err(ctx, PICCS_EINVAL, "NULL buffer");
    if ((params->variant == PICCS_VARIANT_PICCS || params->variant == PICCS_VARIANT_PIPLE) &&
        !ctx->has_prior)
        return set_err(ctx, PICCS_EINVAL, "prior not set");
    return enqueue_weights(ctx, d_x, params, d_omega, d_c, Slots{1, 0});
}

int piccs_reg_normal(piccs_ctx *ctx, const float *d_omega, const piccs_params *params,
                     const float *d_z, float *d_out, double *h_rho)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    char why[256];
    if (check_params(params, why, sizeof why) != PICCS_OK) return set_err(ctx, PICCS_EINVAL, "%s", why);
    if (!d_omega || !d_z || !d_out) return set_err(ctx, PICCS_EINVAL, "NULL buffer");
    LAUNCH(ctx, PICCS_KERNEL_REG, launch_reg_normal(ctx->vd, d_z, d_omega, lam2_piple(params), d_out,
                                    h_rho ? ctx->part_vol : nullptr, ctx->stream));
    if (h_rho) {
        LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_sum_partials(ctx->part_vol, ctx->n_part_vol, ctx->dsum, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(h_rho, ctx->dsum, sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return PICCS_OK;
}

// One IRN-PICCS reconstruction from device-resident data d_b into ctx->x.
// Allocates the LSQR re-orthogonalisation basis on first use (synchronises).
static int ensure_basis(piccs_ctx *ctx, int n_inner, int storage)
{
    const size_t per_slot = basis_bytes(&ctx->geo, n_inner, storage);
    if (ctx->basis && per_slot <= ctx->basis_stride) return PICCS_OK;  // large enough
    const size_t bytes = per_slot * ctx->nslot;
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(ctx, cudaMemGetInfo(&free_b, &total_b));
    const size_t held = ctx->basis ? ctx->basis_stride * ctx->nslot : 0;
    if (bytes > free_b + held)
        return set_err(ctx, PICCS_ENOMEM, "LSQR basis needs %zu bytes, %zu free", bytes, free_b + held);
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    // captured graphs hold the old basis pointers and stride
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second.exec);
    ctx->graphs.clear();
    if (ctx->part_dots) cudaFree(ctx->part_dots);
    ctx->basis = nullptr;
    ctx->part_dots = nullptr;
    ctx->basis_stride = 0;
    void *mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, PICCS_ENOMEM, "cudaMalloc of the LSQR basis (%zu bytes) failed", bytes);
    }
    ctx->part_dots = static_cast<double *>(mem);
    ctx->basis = static_cast<char *>(mem) + basis_dots_bytes();
    ctx->basis_stride = per_slot;
    ctx->basis_gen += 1;
    return PICCS_OK;
}

extern "C++" {  // the enqueue helpers are templates

// The contexts one enqueue advances in lockstep, every kernel on its
// context's stream (for a group: the same stream for all).  One context, or
// up to kMaxGroup contexts of different geometries whose projector products
// share one launch per kernel while every other kernel runs per context.
struct Run {
    piccs_ctx *m[kMaxGroup];
    int n;
};

#define EACH(R) for (int i_ = 0; i_ < (R).n; ++i_) if (piccs_ctx *ctx = (R).m[i_])

static FwdJob fwd_job(piccs_ctx *c, const float *vol, float *out, const float *aux, double *partials,
                      int *nonfinite, float *ra = nullptr, float *aw = nullptr)
{
    FwdJob j{};
    j.g = c->pg;
    j.cols = c->cols;
    j.vr = c->vr;
    j.cells = c->cells;
    j.vol = vol;
    j.out = out;
    j.aux = aux;
    j.partials = partials;
    j.nonfinite = nonfinite;
    j.ra = ra;
    j.aw = aw;
    j.sstride = (long long)c->slot_bytes;
    j.nslot = c->nactive;
    return j;
}

static AdjJob adj_job(piccs_ctx *c, const float *proj, float *vol)
{
    AdjJob j{};
    j.g = c->pg;
    j.cols = c->cols;
    j.vr = c->vr;
    j.hit_ptr = c->hit_ptr;
    j.hits = c->hits;
    j.proj = proj;
    j.rs = c->rs;
    j.vol = vol;
    j.sstride = (long long)c->slot_bytes;
    j.nslot = c->nactive;
    return j;
}

// A = the forward in `mode` of every member (job(ctx) gives its buffers).
template <class F>
static int run_forward(const Run &R, int mode, F job)
{
    piccs_ctx *lead = R.m[0];
    if (R.n == 1) {
        const FwdJob j = job(lead);
        if (mode == FWD_LSQR)
            LAUNCH(lead, PICCS_KERNEL_FORWARD,
                   launch_forward_lsqr(j.g, j.cols, j.vr, j.cells, j.vol, j.out, j.aux, j.ra, j.aw,
                                       j.partials, lead->stream, SL(lead)));
        else
            LAUNCH(lead, PICCS_KERNEL_FORWARD,
                   launch_forward(j.g, j.cols, j.vr, j.cells, j.vol, j.out, mode, j.aux, j.partials,
                                  j.nonfinite, lead->stream, SL(lead)));
        return PICCS_OK;
    }
    FwdJob jobs[kMaxGroup];
    for (int i = 0; i < R.n; ++i) jobs[i] = job(R.m[i]);
    LAUNCH(lead, PICCS_KERNEL_FORWARD, launch_forward_group(jobs, R.n, mode, lead->stream));
    return PICCS_OK;
}

// s = A^T r of every member (the data residual r into the image vector s)
static int run_adjoint(const Run &R)
{
    piccs_ctx *lead = R.m[0];
    if (R.n == 1) {
        LAUNCH(lead, PICCS_KERNEL_ADJOINT, launch_adjoint(lead->pg, lead->cols, lead->vr, lead->hit_ptr,
                                                          lead->hits, lead->r, lead->rs, lead->s,
                                                          lead->stream, SL(lead)));
        return PICCS_OK;
    }
    AdjJob jobs[kMaxGroup];
    for (int i = 0; i < R.n; ++i) jobs[i] = adj_job(R.m[i], R.m[i]->r, R.m[i]->s);
    LAUNCH(lead, PICCS_KERNEL_ADJOINT, launch_adjoint_group(jobs, R.n, lead->stream));
    return PICCS_OK;
}

#define RUN_TRY(call)                 \
    do {                              \
        int rc_ = (call);             \
        if (rc_ != PICCS_OK) return rc_; \
    } while (0)

// One IRN cycle with LSQR as the inner solver (weights already frozen in
// omega, c).  Buffers: uA in r, the data residual b - A x in q (kept current
// through A w in aw, so only the first cycle projects x), vhat in p, w in g,
// z alternating between t and w2sq (free once c is formed), s = the
// regularisation part of A~^T u plus, after the adjoint, A^T uA.  d_b(ctx):
// the member's projections.
template <class B>
static int enqueue_lsqr_cycle(const Run &R, B d_b, const piccs_params *p, int cycle)
{
    const float l2p = lam2_piple(p);
    const bool reorth = p->solver == PICCS_SOLVER_LSQR_REORTH;
    const bool bf16 = p->storage == PICCS_STORAGE_BF16;
    const bool prior_rhs = p->variant == PICCS_VARIANT_PICCS || p->variant == PICCS_VARIANT_PIPLE;
    int cur = 0;
    auto zbuf = [](piccs_ctx *c, int k) { return k == 0 ? c->t : c->w2sq; };
    // beta_1 u_1 = b~ - A~ x: uA = b - A x, z = -x, sigma = 1
    if (cycle == 0)
        RUN_TRY(run_forward(R, bf16 ? FWD_RESID16 : FWD_RESID, [&](piccs_ctx *c) {
            return fwd_job(c, c->x, c->q, d_b(c), nullptr, &c->ks->nonfinite);
        }));
    EACH(R) {
        cudaStream_t st = ctx->stream;
        LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_lsqr_rinit(ctx->N, cycle > 0, ctx->q, ctx->aw, ctx->r, ctx->ls,
                                                           ctx->part_vec, st, SL(ctx)));
        LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_lsqr_reset(ctx->ks, ctx->ls, st, SL(ctx)));
        LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_lsqr_zstep(ctx->vd, 1, ctx->x, nullptr, zbuf(ctx, cur), nullptr,
                                                           st, SL(ctx)));
        LAUNCH(ctx, PICCS_KERNEL_REG, launch_lsqr_ureg(ctx->vd, 1, zbuf(ctx, cur), ctx->omega, l2p, ctx->c,
                                                       prior_rhs ? ctx->xprior : nullptr, ctx->s, nullptr,
                                                       ctx->part_vol, st, SL(ctx)));
        LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_lsqr_finalize_beta(ctx->ks, ctx->ls, 1, ctx->part_vec,
                                                                   ctx->n_part_vec, ctx->part_vol,
                                                                   ctx->n_part_vol, st, SL(ctx)));
    }
    // alpha_1 v_1 = A~^T u_1
    RUN_TRY(run_adjoint(R));
    EACH(R) {
        cudaStream_t st = ctx->stream;
        LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_lsqr_vx(ctx->M, 1, 0, ctx->x, ctx->g, ctx->p, ctx->s, nullptr,
                                                        ctx->ls, ctx->part_vec, st, SL(ctx)));
        LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_lsqr_finalize_alpha(ctx->ks, ctx->ls, 1, ctx->part_vec,
                                                                    ctx->n_part_vec, st, SL(ctx)));
    }
    for (int i = 1; i <= p->n_inner; ++i) {
        const bool last = i == p->n_inner;
        // beta_{i+1} u_{i+1} = A~ v_i - alpha_i u_i
        RUN_TRY(run_forward(R, FWD_LSQR, [&](piccs_ctx *c) {
            return fwd_job(c, c->p, c->r, c->ls->fwd, c->part_fwd, nullptr, c->q, c->aw);
        }));
        EACH(R) {
            cudaStream_t st = ctx->stream;
            LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_lsqr_zstep(ctx->vd, 0, ctx->p, zbuf(ctx, cur),
                                                               zbuf(ctx, cur ^ 1), ctx->ls->ureg, st, SL(ctx)));
            LAUNCH(ctx, PICCS_KERNEL_REG, launch_lsqr_ureg(ctx->vd, 0, zbuf(ctx, cur ^ 1), ctx->omega, l2p, ctx->c,
                                                           nullptr, ctx->s, ctx->ls->ureg, ctx->part_vol, st,
                                                           SL(ctx)));
            LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_lsqr_finalize_beta(ctx->ks, ctx->ls, 0, ctx->part_fwd,
                                                                       ctx->n_part_fwd, ctx->part_vol,
                                                                       ctx->n_part_vol, st, SL(ctx)));
        }
        cur ^= 1;
        // alpha_{i+1} v_{i+1} = A~^T u_{i+1} - beta_{i+1} v_i (not needed after the last step)
        if (!last) RUN_TRY(run_adjoint(R));
        EACH(R) {
            cudaStream_t st = ctx->stream;
            const long long M = ctx->M;
            const long long ldb = lsqr_basis_stride(M);
            void *bv = (reorth && !last)
                           ? static_cast<char *>(ctx->basis) + (size_t)(i - 1) * ldb * (bf16 ? 2 : sizeof(float))
                           : nullptr;
            const long long bst = (long long)ctx->basis_stride;
            LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_lsqr_vx(M, 0, last, ctx->x, ctx->g, ctx->p, ctx->s, bv,
                                                            ctx->ls, ctx->part_vec, st, SL(ctx), bst, bf16));
            if (last) continue;
            if (reorth) {
                for (int pass = 0; pass < 2; ++pass) {
                    LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_lsqr_dots(M, ldb, i, ctx->basis, ctx->p, ctx->ls,
                                                                      ctx->part_dots, st, SL(ctx), bst, bf16));
                    LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_lsqr_fin_dots(i, ctx->ls, ctx->part_dots, st,
                                                                          SL(ctx), bst));
                    LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_lsqr_sub(M, ldb, i, ctx->basis, ctx->p, ctx->ls,
                                                                     pass == 1 ? ctx->part_vec : nullptr, st,
                                                                     SL(ctx), bst, bf16));
                }
            }
            LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_lsqr_finalize_alpha(ctx->ks, ctx->ls, 0, ctx->part_vec,
                                                                        ctx->n_part_vec, st, SL(ctx)));
        }
        if (last) break;
    }
    return PICCS_OK;
}

// One IRN-PICCS reconstruction of every member from its device-resident data
// d_b(ctx) into its x; d_x0: the slots' initial volumes, x0_pitch bytes apart
// (one context only).  A context's projections are FP32, or BF16 when
// p->storage is BF16.
template <class B>
static int enqueue_reconstruct(const Run &R, B d_b, const piccs_params *p, const float *d_x0,
                               size_t x0_pitch)
{
    const bool bf16 = p->storage == PICCS_STORAGE_BF16;
    const float l2p = lam2_piple(p);
    EACH(R) {
        cudaStream_t st = ctx->stream;
        const size_t vb = ctx->M * sizeof(float), S = ctx->slot_bytes;
        LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_reset_scalars(ctx->ks, st, SL(ctx)));
        if (p->x0_mode == PICCS_X0_PRIOR) {
            CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->x, S, ctx->xprior, S, vb, ctx->nactive, cudaMemcpyDeviceToDevice, st));
        } else if (p->x0_mode == PICCS_X0_ZERO) {
            CUDA_TRY(ctx, cudaMemset2DAsync(ctx->x, S, 0, vb, ctx->nactive, st));
        } else {
            CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->x, S, d_x0, x0_pitch, vb, ctx->nactive, cudaMemcpyDeviceToDevice, st));
        }
    }
    if (p->solver != PICCS_SOLVER_CGLS) {
        if (p->n_inner == 0) {  // no inner step: x stays x0; still flag NaN/Inf in b
            EACH(R) {
                if (bf16)
                    LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_count_nonfinite16(ctx->N, d_b(ctx), &ctx->ks->nonfinite,
                                                                              ctx->stream, SL(ctx)));
                else
                    LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_count_nonfinite(ctx->N, d_b(ctx), &ctx->ks->nonfinite,
                                                                            ctx->stream, SL(ctx)));
            }
            return PICCS_OK;
        }
        for (int k = 0; k < p->n_outer; ++k) {
            EACH(R) RUN_TRY(enqueue_weights(ctx, ctx->x, p, ctx->omega, ctx->c, SL(ctx)));
            RUN_TRY(enqueue_lsqr_cycle(R, d_b, p, k));
        }
        return PICCS_OK;
    }
    // data residual r = b - A x0 (also flags NaN/Inf in b)
    RUN_TRY(run_forward(R, bf16 ? FWD_RESID16 : FWD_RESID, [&](piccs_ctx *c) {
        return fwd_job(c, c->x, c->r, d_b(c), nullptr, &c->ks->nonfinite);
    }));
    for (int k = 0; k < p->n_outer; ++k) {
        // reweighting at the previous iterate (Eqs. 10-11)
        EACH(R) RUN_TRY(enqueue_weights(ctx, ctx->x, p, ctx->omega, ctx->c, SL(ctx)));
        // restart: g = c - D^T Omega D x, s = A^T r + g
        if (k == 0) {
            EACH(R) LAUNCH(ctx, PICCS_KERNEL_REG, launch_reg_restart(ctx->vd, ctx->x, ctx->omega, l2p, ctx->c, ctx->g,
                                                                     ctx->s, 1, nullptr, ctx->stream, SL(ctx)));
            RUN_TRY(run_adjoint(R));
            EACH(R) {
                LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_norm2(ctx->M, ctx->s, ctx->part_vec, ctx->stream, SL(ctx)));
                LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_finalize_gamma(ctx->ks, ctx->part_vec, ctx->n_part_vec, 1,
                                                                       ctx->stream, SL(ctx)));
            }
        } else {
            EACH(R) {
                LAUNCH(ctx, PICCS_KERNEL_REG, launch_reg_restart(ctx->vd, ctx->x, ctx->omega, l2p, ctx->c, ctx->g,
                                                                 ctx->s, 0, ctx->part_vol, ctx->stream, SL(ctx)));
                LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_finalize_gamma(ctx->ks, ctx->part_vol, ctx->n_part_vol, 1,
                                                                       ctx->stream, SL(ctx)));
            }
        }
        for (int it = 0; it < p->n_inner; ++it) {
            EACH(R) {
                LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_p_update(ctx->M, ctx->s, ctx->p, ctx->ks, ctx->stream, SL(ctx)));
                LAUNCH(ctx, PICCS_KERNEL_REG, launch_reg_normal(ctx->vd, ctx->p, ctx->omega, l2p, ctx->t,
                                                                ctx->part_vol, ctx->stream, SL(ctx)));
            }
            RUN_TRY(run_forward(R, FWD_PLAIN, [&](piccs_ctx *c) {
                return fwd_job(c, c->p, c->q, nullptr, c->part_fwd, nullptr);
            }));
            EACH(R) {
                LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_finalize_delta(ctx->ks, ctx->part_fwd, ctx->n_part_fwd,
                                                                       ctx->part_vol, ctx->n_part_vol, ctx->stream,
                                                                       SL(ctx)));
                LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_x_update(ctx->M, ctx->N, ctx->x, ctx->p, ctx->g, ctx->t,
                                                                 ctx->s, ctx->r, ctx->q, ctx->ks, ctx->stream,
                                                                 SL(ctx)));
            }
            // after the reconstruction's last step s = A^T r + g only feeds the
            // history, so its backprojection is skipped
            if (k == p->n_outer - 1 && it == p->n_inner - 1) break;
            RUN_TRY(run_adjoint(R));
            EACH(R) {
                LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_norm2(ctx->M, ctx->s, ctx->part_vec, ctx->stream, SL(ctx)));
                LAUNCH(ctx, PICCS_KERNEL_SCALAR, launch_finalize_gamma(ctx->ks, ctx->part_vec, ctx->n_part_vec, 0,
                                                                       ctx->stream, SL(ctx)));
            }
        }
    }
    return PICCS_OK;
}

}  // extern "C++"

// one context, its data at d_b (allocates the re-orthogonalisation basis on
// first use, which synchronises)
static int enqueue_reconstruct(piccs_ctx *ctx, const float *d_b, const piccs_params *p,
                               const float *d_x0, size_t x0_pitch)
{
    if (p->solver == PICCS_SOLVER_LSQR_REORTH) RUN_TRY(ensure_basis(ctx, p->n_inner, p->storage));
    Run R{};
    R.m[0] = ctx;
    R.n = 1;
    return enqueue_reconstruct(R, [d_b](piccs_ctx *) { return d_b; }, p, d_x0, x0_pitch);
}

static int check_reconstruct_args(piccs_ctx *ctx, const void *proj, const piccs_params *params,
                                  const void *x0, const void *out)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    char why[256];
    if (check_params(params, why, sizeof why) != PICCS_OK) return set_err(ctx, PICCS_EINVAL, "%s", why);
    if (!proj || !out) return set_err(ctx, PICCS_EINVAL, "NULL buffer");
    if (params->x0_mode == PICCS_X0_USER && !x0) return set_err(ctx, PICCS_EINVAL, "x0_mode USER needs x0");
    if (needs_prior(params) && !ctx->has_prior) return set_err(ctx, PICCS_EINVAL, "prior not set");
    return PICCS_OK;
}

int piccs_reconstruct(piccs_ctx *ctx, const float *d_proj, const piccs_params *params,
                      const float *d_x0, float *d_vol_out)
{
    int rc = check_reconstruct_args(ctx, d_proj, params, d_x0, d_vol_out);
    if (rc != PICCS_OK) return rc;
    ctx->nactive = ctx->nslot;
    const size_t vb = ctx->M * sizeof(float), pb = ctx->N * sizeof(float);
    const float *d_b = d_proj;
    if (params->storage == PICCS_STORAGE_BF16) {  // the slots' projections, rounded once
        LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_to_bf16(ctx->N, d_proj, (long long)pb, ctx->bstage,
                                                        (long long)ctx->slot_bytes, ctx->nslot, ctx->stream));
        d_b = ctx->bstage;
    } else if (ctx->nslot > 1) {  // the kernels read each slot's projections at its workspace stride
        CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->bstage, ctx->slot_bytes, d_proj, pb, pb, ctx->nslot,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
        d_b = ctx->bstage;
    }
    rc = enqueue_reconstruct(ctx, d_b, params, d_x0, vb);
    if (rc != PICCS_OK) return rc;
    CUDA_TRY(ctx, cudaMemcpy2DAsync(d_vol_out, vb, ctx->x, ctx->slot_bytes, vb, ctx->nslot,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
    return PICCS_OK;
}

int piccs_report_slot(piccs_ctx *ctx, int slot, piccs_stats *out)
{
    if (!ctx || !out) return set_err(ctx, PICCS_EINVAL, "NULL argument");
    if (slot < 0 || slot >= ctx->nslot) return set_err(ctx, PICCS_EINVAL, "slot %d out of range", slot);
    KrylovScalars ks;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    CUDA_TRY(ctx, cudaMemcpy(&ks, slot_at(ctx->ks, ctx, slot), sizeof ks, cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof *out);
    out->status = ks.nonfinite ? PICCS_ENONFINITE : ks.status;
    out->iterations_run = ks.iters_run;
    out->n_history = ks.n_hist < 512 ? ks.n_hist : 512;
    std::memcpy(out->gamma_history, ks.hist, sizeof(double) * out->n_history);
    return PICCS_OK;
}

int piccs_report(piccs_ctx *ctx, piccs_stats *out)
{
    return piccs_report_slot(ctx, 0, out);
}

int piccs_reconstruct_host(piccs_ctx *ctx, const float *h_proj, const piccs_params *params,
                           const float *h_x0, float *h_vol_out)
{
    int rc = check_reconstruct_args(ctx, h_proj, params, h_x0, h_vol_out);
    if (rc != PICCS_OK) return rc;
    ctx->nactive = ctx->nslot;
    cudaStream_t st = ctx->stream;
    const size_t vb = ctx->M * sizeof(float), pb = ctx->N * sizeof(float), S = ctx->slot_bytes;
    if (params->storage == PICCS_STORAGE_BF16) {  // through the ray scratch, rounded once
        CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->rs, S, h_proj, pb, pb, ctx->nslot, cudaMemcpyHostToDevice, st));
        LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_to_bf16(ctx->N, ctx->rs, (long long)S, ctx->bstage,
                                                        (long long)S, ctx->nslot, st));
    } else {
        CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->bstage, S, h_proj, pb, pb, ctx->nslot, cudaMemcpyHostToDevice, st));
    }
    const float *dx0 = nullptr;
    if (params->x0_mode == PICCS_X0_USER) {
        // the initial guesses go through the p buffers, which are free until the first step
        CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->p, S, h_x0, vb, vb, ctx->nslot, cudaMemcpyHostToDevice, st));
        dx0 = ctx->p;
    }
    rc = enqueue_reconstruct(ctx, ctx->bstage, params, dx0, S);
    if (rc != PICCS_OK) return rc;
    CUDA_TRY(ctx, cudaMemcpy2DAsync(h_vol_out, vb, ctx->x, S, vb, ctx->nslot, cudaMemcpyDeviceToHost, st));
    for (int sl = 0; sl < ctx->nslot; ++sl) {
        piccs_stats rep;
        rc = piccs_report_slot(ctx, sl, &rep);
        if (rc != PICCS_OK) return rc;
        if (rep.status != PICCS_OK)
            return set_err(ctx, rep.status, rep.status == PICCS_ENONFINITE ? "projections %d hold NaN or Inf"
                                                                           : "Krylov breakdown in scan %d", sl);
    }
    return PICCS_OK;
}

// ---- staged reconstructions (the building blocks of the request server) ----

int piccs_set_prior_broadcast(piccs_ctx *ctx, const float *xprior, int from_host)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    if (!xprior) return set_err(ctx, PICCS_EINVAL, "xprior is NULL");
    const size_t vb = ctx->M * sizeof(float);
    for (int b = 0; b < ctx->nslot; ++b)
        CUDA_TRY(ctx, cudaMemcpyAsync(slot_at(ctx->xprior, ctx, b), b == 0 ? xprior : ctx->xprior, vb,
                                      b == 0 && from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    ctx->nactive = 1;
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->stream));
    LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_count_nonfinite(ctx->M, ctx->xprior, ctx->flag, ctx->stream));
    int bad = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&bad, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->has_prior = !bad;
    if (bad) return set_err(ctx, PICCS_ENONFINITE, "prior volume holds NaN or Inf");
    return PICCS_OK;
}

int piccs_stage(piccs_ctx *ctx, int slot, const float *proj, int from_host)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    if (slot < 0 || slot >= ctx->nslot || !proj) return set_err(ctx, PICCS_EINVAL, "bad slot or NULL buffer");
    CUDA_TRY(ctx, cudaMemcpyAsync(slot_at(ctx->bstage, ctx, slot), proj, ctx->N * sizeof(float),
                                  from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->staged16[slot] = 0;
    return PICCS_OK;
}

int piccs_stage_bf16(piccs_ctx *ctx, int slot, const void *proj, int from_host)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    if (slot < 0 || slot >= ctx->nslot || !proj) return set_err(ctx, PICCS_EINVAL, "bad slot or NULL buffer");
    CUDA_TRY(ctx, cudaMemcpyAsync(slot_at(ctx->bstage, ctx, slot), proj, ctx->N * 2,
                                  from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->staged16[slot] = 1;
    return PICCS_OK;
}

int piccs_unstage(piccs_ctx *ctx, int slot, float *vol, int to_host)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    if (slot < 0 || slot >= ctx->nslot || !vol) return set_err(ctx, PICCS_EINVAL, "bad slot or NULL buffer");
    CUDA_TRY(ctx, cudaMemcpyAsync(vol, slot_at(ctx->x, ctx, slot), ctx->M * sizeof(float),
                                  to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream));
    return PICCS_OK;
}

// Validates and prepares one member of a staged run (BF16 rounding of FP32
// staged data on its own stream, the re-orthogonalisation basis).
static int prepare_staged(piccs_ctx *ctx, int nactive, const piccs_params *params)
{
    if (nactive < 1 || nactive > ctx->nslot) return set_err(ctx, PICCS_EINVAL, "nactive %d out of range", nactive);
    if (params->x0_mode == PICCS_X0_USER) return set_err(ctx, PICCS_EINVAL, "staged runs start from the prior or zero");
    if (needs_prior(params) && !ctx->has_prior) return set_err(ctx, PICCS_EINVAL, "prior not set");
    ctx->nactive = nactive;
    const bool bf16 = params->storage == PICCS_STORAGE_BF16;
    for (int b = 0; b < nactive; ++b) {
        if (ctx->staged16[b] && !bf16)
            return set_err(ctx, PICCS_EINVAL, "slot %d holds BF16 projections; the run needs storage BF16", b);
        if (bf16 && !ctx->staged16[b]) {  // round the staged FP32 projections, through the ray scratch
            LAUNCH(ctx, PICCS_KERNEL_VECTOR, launch_to_bf16(ctx->N, slot_at(ctx->bstage, ctx, b), 0,
                                                            slot_at(ctx->rs, ctx, b), 0, 1, ctx->stream));
            CUDA_TRY(ctx, cudaMemcpyAsync(slot_at(ctx->bstage, ctx, b), slot_at(ctx->rs, ctx, b), ctx->N * 2,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
            ctx->staged16[b] = 1;
        }
    }
    if (params->solver == PICCS_SOLVER_LSQR_REORTH)  // allocate before any capture
        RUN_TRY(ensure_basis(ctx, params->n_inner, params->storage));
    return PICCS_OK;
}

// `after` waits for what has been enqueued on `before` so far
static int stream_after(piccs_ctx *ctx, cudaStream_t before, cudaStream_t after)
{
    if (before == after) return PICCS_OK;
    cudaEvent_t e = take_event(ctx);
    if (!e) return set_err(ctx, PICCS_ECUDA, "cudaEventCreate failed");
    cudaError_t err = cudaEventRecord(e, before);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(after, e, 0);
    ctx->event_pool.push_back(e);  // reusable once the wait is enqueued
    if (err != cudaSuccess) return set_err(ctx, PICCS_ECUDA, "stream ordering failed: %s", cudaGetErrorString(err));
    return PICCS_OK;
}

int piccs_run_staged_group(piccs_ctx *const *ctxs, const int *nactive, int n, const piccs_params *params,
                           int use_graph)
{
    if (!ctxs || !nactive || n < 1 || n > kMaxGroup)
        return set_err(nullptr, PICCS_EINVAL, "group of %d contexts (1 .. %d)", n, kMaxGroup);
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return set_err(nullptr, PICCS_EINVAL, "ctxs[%d] is NULL", i);
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return set_err(ctxs[0], PICCS_EINVAL, "context %d appears twice", i);
        if (ctxs[i]->device != ctxs[0]->device)
            return set_err(ctxs[0], PICCS_EINVAL, "context %d is on another device", i);
    }
    piccs_ctx *lead = ctxs[0];
    char why[256];
    if (check_params(params, why, sizeof why) != PICCS_OK) return set_err(lead, PICCS_EINVAL, "%s", why);
    for (int i = 0; i < n; ++i) {
        int rc = prepare_staged(ctxs[i], nactive[i], params);
        if (rc != PICCS_OK) {
            if (i > 0) set_err(lead, rc, "context %d: %s", i, ctxs[i]->err.c_str());
            return rc;
        }
    }
    Run R{};
    R.n = n;
    for (int i = 0; i < n; ++i) R.m[i] = ctxs[i];
    auto staged = [](piccs_ctx *c) { return static_cast<const float *>(c->bstage); };
    // every member's work on the lead's stream, after each member's staging
    cudaStream_t saved[kMaxGroup];
    for (int i = 0; i < n; ++i) saved[i] = ctxs[i]->stream;
    for (int i = 1; i < n; ++i) RUN_TRY(stream_after(lead, saved[i], saved[0]));
    auto on = [&](cudaStream_t st) {
        for (int i = 0; i < n; ++i) ctxs[i]->stream = st;
    };
    auto restore = [&]() {
        for (int i = 0; i < n; ++i) ctxs[i]->stream = saved[i];
    };
    auto finish = [&](int rc) {
        restore();
        // each member's unstaging copies follow the run
        for (int i = 1; i < n && rc == PICCS_OK; ++i) rc = stream_after(lead, saved[0], saved[i]);
        return rc;
    };
    bool timing = false;
    for (int i = 0; i < n; ++i) timing |= ctxs[i]->timing;
    if (!use_graph || timing) {
        on(saved[0]);
        return finish(enqueue_reconstruct(R, staged, params, nullptr, 0));
    }
    // one CUDA graph per (parameters, members, active slots, basis
    // allocations): the launch sequence is fixed, every per-step scalar lives
    // on the device; kept by the lead
    std::string key(reinterpret_cast<const char *>(params), sizeof *params);
    for (int i = 0; i < n; ++i) {
        const long long id[3] = {ctxs[i]->uid, nactive[i], ctxs[i]->basis_gen};
        key.append(reinterpret_cast<const char *>(id), sizeof id);
    }
    auto it = lead->graphs.find(key);
    if (it == lead->graphs.end()) {
        long long before[kMaxGroup][PICCS_KERNEL_CLASSES], before_calls[kMaxGroup][PICCS_KERNEL_CLASSES];
        for (int i = 0; i < n; ++i) {
            std::memcpy(before[i], ctxs[i]->launches, sizeof before[i]);
            std::memcpy(before_calls[i], ctxs[i]->calls, sizeof before_calls[i]);
        }
        if (!lead->cap_stream)
            CUDA_TRY(lead, cudaStreamCreateWithFlags(&lead->cap_stream, cudaStreamNonBlocking));
        // capture on the private stream (nothing runs during a capture), then
        // launch the graph on the lead's stream
        CUDA_TRY(lead, cudaStreamBeginCapture(lead->cap_stream, cudaStreamCaptureModeThreadLocal));
        on(lead->cap_stream);
        int rc = enqueue_reconstruct(R, staged, params, nullptr, 0);
        restore();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(lead->cap_stream, &graph);
        if (rc != PICCS_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return finish(rc != PICCS_OK ? rc
                                         : set_err(lead, PICCS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e)));
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return finish(set_err(lead, PICCS_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e)));
        piccs_ctx::GraphEntry ge;
        ge.exec = exec;
        for (int k = 0; k < PICCS_KERNEL_CLASSES; ++k) {
            // counted on the lead when the graph runs
            for (int i = 0; i < n; ++i) {
                ge.launches[k] += ctxs[i]->launches[k] - before[i][k];
                ge.calls[k] += ctxs[i]->calls[k] - before_calls[i][k];
                ctxs[i]->launches[k] = before[i][k];
                ctxs[i]->calls[k] = before_calls[i][k];
            }
        }
        it = lead->graphs.emplace(key, ge).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second.exec, saved[0]);
    if (e != cudaSuccess) return finish(set_err(lead, PICCS_ECUDA, "cudaGraphLaunch failed: %s", cudaGetErrorString(e)));
    for (int k = 0; k < PICCS_KERNEL_CLASSES; ++k) {
        lead->launches[k] += it->second.launches[k];
        lead->calls[k] += it->second.calls[k];
    }
    lead->graph_launches += 1;
    return finish(PICCS_OK);
}

int piccs_run_staged(piccs_ctx *ctx, int nactive, const piccs_params *params, int use_graph)
{
    if (!ctx) return set_err(nullptr, PICCS_EINVAL, "ctx is NULL");
    return piccs_run_staged_group(&ctx, &nactive, 1, params, use_graph);
}

}  // extern "C"
