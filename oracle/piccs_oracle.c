/*
 * FP64 CPU oracle for IRN-PICCS cone-beam reconstruction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library; it is plain, slow
 * and written to be checked against the paper by eye.
 *
 * What it computes (paper: Hastings, Islam, Sabate Landman et al.,
 * "Real-time CBCT reconstructions using Krylov solvers in repeated scanning
 * procedures"):
 *   - the linear model A x + e = b (Sec. 2.1, Eq. 1): A_ij is the length (mm)
 *     of ray i inside voxel j, computed with an incremental Siddon walk that
 *     merges the x, y and z plane crossings and assigns each piece to the voxel
 *     holding its midpoint;  A^T is the same walk scattering into the volume;
 *   - D = [D1 (x) I (x) I; I (x) D1 (x) I; I (x) I (x) D1] with D1 rows [1, -1]
 *     (Sec. 2.2), each block zero-padded to M rows (Neumann boundary);
 *   - the IRN weights [W*]_ii = (sqrt(sum_d [D_d z]_i^2) + tau^2)^(-1/2)
 *     (Sec. 2.2, the equation after Eq. 5), rule R1; rule R2 is the common
 *     (|g|^2 + tau^2)^(-1/4) alternative, kept behind a flag;
 *   - IRN-PICCS (Sec. 2.3, Eqs. 9-11): for k = 1..n_outer, W1 = W(D x_{k-1}),
 *     W2 = W(D x_{k-1} - D x_p), then a few CGLS iterations on the augmented
 *     least-squares problem [A; alpha W1 D; lambda W2 D] x ~ [b; 0; lambda W2 D x_p]
 *     warm-started at x_{k-1}, with the augmented residual kept explicitly;
 *     LSQR (Golub-Kahan bidiagonalisation, optionally with the new v
 *     re-orthogonalised against all earlier ones) may replace CGLS, as the
 *     paper allows (Sec. 2.3);
 *   - variants: IRN-PIPLE (Eq. 8: the prior block becomes lambda I, right-hand
 *     side lambda x_p), IRN-TV (Eq. 6: no prior block) and plain CGLS.
 *
 * Parity pins live in tests/test_oracle_*.py; no function here is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double vx, vy, vz;
    int nu, nv;
    double du, dv;
    double dso, dsd;
    int n_views;
    const double *angles;
    int layout; /* 0: (j, iu, iv) v fastest; 1: (j, iv, iu) u fastest */
    double u_offset; /* detector shift along u (mm): pixel centres at
                        (iu - (nu-1)/2) du + u_offset */
} og_geom;

enum { OG_PICCS = 0, OG_PIPLE = 1, OG_TV = 2, OG_CGLS = 3 };

static long long og_M(const og_geom *g) { return (long long)g->nx * g->ny * g->nz; }
static long long og_N(const og_geom *g) { return (long long)g->n_views * g->nu * g->nv; }

static long long og_pidx(const og_geom *g, int j, int iu, int iv)
{
    if (g->layout == 0) return ((long long)j * g->nu + iu) * g->nv + iv;
    return ((long long)j * g->nv + iv) * g->nu + iu;
}

static void og_unpidx(const og_geom *g, long long r, int *j, int *iu, int *iv)
{
    if (g->layout == 0) {
        *iv = (int)(r % g->nv); r /= g->nv;
        *iu = (int)(r % g->nu); *j = (int)(r / g->nu);
    } else {
        *iu = (int)(r % g->nu); r /= g->nu;
        *iv = (int)(r % g->nv); *j = (int)(r / g->nv);
    }
}

/* Source point and pixel centre of ray (j, iu, iv). */
static void og_ray(const og_geom *g, int j, int iu, int iv, double S[3], double P[3])
{
    double c = cos(g->angles[j]), s = sin(g->angles[j]);
    double u = (iu - (g->nu - 1) / 2.0) * g->du + g->u_offset;
    double v = (iv - (g->nv - 1) / 2.0) * g->dv;
    double back = g->dsd - g->dso;
    S[0] = g->dso * c; S[1] = g->dso * s; S[2] = 0.0;
    P[0] = -back * c - u * s;
    P[1] = -back * s + u * c;
    P[2] = v;
}

/* 0 when the geometry is usable: positive sizes and the source and detector
 * outside the cylinder circumscribing the volume. */
int og_check(const og_geom *g)
{
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->nu <= 0 || g->nv <= 0 || g->n_views <= 0)
        return -1;
    if (!(g->vx > 0 && g->vy > 0 && g->vz > 0 && g->du > 0 && g->dv > 0)) return -1;
    double R = 0.5 * sqrt(g->nx * g->vx * g->nx * g->vx + g->ny * g->vy * g->ny * g->vy);
    if (!(g->dso > R) || !(g->dsd - g->dso > R)) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Siddon walk                                                               */
/* ------------------------------------------------------------------------ */
typedef void (*og_seg_fn)(void *ctx, long long vox, double len);

/* Calls fn(ctx, voxel, length_mm) for every piece of the segment S->P inside
 * the volume, walking the merged x/y/z plane crossings in order. */
static void og_siddon(const og_geom *g, const double S[3], const double P[3],
                      og_seg_fn fn, void *ctx)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    const double vs[3] = {g->vx, g->vy, g->vz};
    double lo[3], d[3];
    double amin = 0.0, amax = 1.0; /* only the part between source and pixel */
    for (int a = 0; a < 3; ++a) {
        lo[a] = -0.5 * n[a] * vs[a];
        d[a] = P[a] - S[a];
        double hi = lo[a] + n[a] * vs[a];
        if (d[a] == 0.0) {
            if (S[a] < lo[a] || S[a] > hi) return;
            continue;
        }
        double t0 = (lo[a] - S[a]) / d[a], t1 = (hi - S[a]) / d[a];
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        if (t0 > amin) amin = t0;
        if (t1 < amax) amax = t1;
    }
    if (!(amax > amin)) return;
    const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);

    /* next plane index and its crossing parameter, per axis */
    int k[3], step[3];
    double anext[3];
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) { anext[a] = INFINITY; step[a] = 0; k[a] = 0; continue; }
        double pos = (S[a] + amin * d[a] - lo[a]) / vs[a];
        if (d[a] > 0) { k[a] = (int)floor(pos) + 1; step[a] = 1; }
        else          { k[a] = (int)ceil(pos) - 1;  step[a] = -1; }
        if (k[a] < 0 || k[a] > n[a]) anext[a] = INFINITY;
        else anext[a] = (lo[a] + k[a] * vs[a] - S[a]) / d[a];
    }
    double acur = amin;
    for (;;) {
        double an = amax;
        for (int a = 0; a < 3; ++a) if (anext[a] < an) an = anext[a];
        if (an > acur) {
            double am = 0.5 * (acur + an);
            long long idx[3];
            int ok = 1;
            for (int a = 0; a < 3; ++a) {
                double q = floor((S[a] + am * d[a] - lo[a]) / vs[a]);
                if (q < 0 || q >= n[a]) { ok = 0; break; }
                idx[a] = (long long)q;
            }
            if (ok) fn(ctx, (idx[0] * g->ny + idx[1]) * g->nz + idx[2], (an - acur) * len);
        }
        if (an >= amax) break;
        for (int a = 0; a < 3; ++a) {
            if (anext[a] == an) {
                k[a] += step[a];
                if (k[a] < 0 || k[a] > n[a]) anext[a] = INFINITY;
                else anext[a] = (lo[a] + k[a] * vs[a] - S[a]) / d[a];
            }
        }
        acur = an;
    }
}

typedef struct { const double *x; double acc; long long cnt; } og_fwd_ctx;
static void og_fwd_cb(void *c, long long vox, double len)
{
    og_fwd_ctx *f = (og_fwd_ctx *)c;
    f->acc += len * f->x[vox];
    f->cnt += 1;
}

static int og_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* y = A x, every ray. */
void og_forward(const og_geom *g, const double *x, double *y, int nthreads)
{
    const long long N = og_N(g);
    int nt = og_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
    for (long long r = 0; r < N; ++r) {
        int j, iu, iv;
        double S[3], P[3];
        og_unpidx(g, r, &j, &iu, &iv);
        og_ray(g, j, iu, iv, S, P);
        og_fwd_ctx c = {x, 0.0, 0};
        og_siddon(g, S, P, og_fwd_cb, &c);
        y[r] = c.acc;
    }
}

/* (A x) for the listed rays only. */
void og_forward_rays(const og_geom *g, const double *x, const long long *rays, long long n,
                     double *out, int nthreads)
{
    int nt = og_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (long long q = 0; q < n; ++q) {
        int j, iu, iv;
        double S[3], P[3];
        og_unpidx(g, rays[q], &j, &iu, &iv);
        og_ray(g, j, iu, iv, S, P);
        og_fwd_ctx c = {x, 0.0, 0};
        og_siddon(g, S, P, og_fwd_cb, &c);
        out[q] = c.acc;
    }
}

/* Number of nonzero A_ij (pieces of positive length inside the volume). */
static void og_cnt_cb(void *c, long long vox, double len)
{
    (void)vox;
    if (len > 0.0) *(long long *)c += 1;
}

long long og_count_nnz(const og_geom *g, int nthreads)
{
    const long long N = og_N(g);
    long long total = 0;
    int nt = og_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total) num_threads(nt)
    for (long long r = 0; r < N; ++r) {
        int j, iu, iv;
        double S[3], P[3];
        og_unpidx(g, r, &j, &iu, &iv);
        og_ray(g, j, iu, iv, S, P);
        long long c = 0;
        og_siddon(g, S, P, og_cnt_cb, &c);
        total += c;
    }
    return total;
}

typedef struct { double *x; double w; } og_adj_ctx;
static void og_adj_cb(void *c, long long vox, double len)
{
    og_adj_ctx *a = (og_adj_ctx *)c;
    a->x[vox] += len * a->w;
}

/* x = A^T y.  Each thread scatters into its own FP64 volume over a fixed
 * (static) share of the rays; the volumes are then added in thread order, so
 * the result does not depend on timing. */
void og_adjoint(const og_geom *g, const double *y, double *x, int nthreads)
{
    const long long N = og_N(g), M = og_M(g);
    int nt = og_threads(nthreads);
    double *priv = (double *)calloc((size_t)nt * (size_t)M, sizeof(double));
    if (!priv) { for (long long i = 0; i < M; ++i) x[i] = NAN; return; }
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        og_adj_ctx c = {priv + (size_t)t * (size_t)M, 0.0};
#pragma omp for schedule(static)
        for (long long r = 0; r < N; ++r) {
            if (y[r] == 0.0) continue;
            int j, iu, iv;
            double S[3], P[3];
            og_unpidx(g, r, &j, &iu, &iv);
            og_ray(g, j, iu, iv, S, P);
            c.w = y[r];
            og_siddon(g, S, P, og_adj_cb, &c);
        }
    }
    for (long long i = 0; i < M; ++i) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += priv[(size_t)t * (size_t)M + i];
        x[i] = s;
    }
    free(priv);
}

/* ------------------------------------------------------------------------ */
/* Brute force: each ray clipped against one voxel box (slab method).        */
/* ------------------------------------------------------------------------ */
static double og_clip_len(const double S[3], const double P[3], const double lo[3],
                          const double hi[3])
{
    double amin = 0.0, amax = 1.0;
    for (int a = 0; a < 3; ++a) {
        double d = P[a] - S[a];
        if (d == 0.0) {
            if (S[a] < lo[a] || S[a] > hi[a]) return 0.0;
            continue;
        }
        double t0 = (lo[a] - S[a]) / d, t1 = (hi[a] - S[a]) / d;
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        if (t0 > amin) amin = t0;
        if (t1 < amax) amax = t1;
    }
    if (!(amax > amin)) return 0.0;
    double dx = P[0] - S[0], dy = P[1] - S[1], dz = P[2] - S[2];
    return (amax - amin) * sqrt(dx * dx + dy * dy + dz * dz);
}

/* Length of ray r inside voxel v, by clipping the ray against that voxel. */
double og_clip_ray_voxel(const og_geom *g, long long r, long long v)
{
    int j, iu, iv;
    double S[3], P[3], lo[3], hi[3];
    og_unpidx(g, r, &j, &iu, &iv);
    og_ray(g, j, iu, iv, S, P);
    long long iz = v % g->nz, iy = (v / g->nz) % g->ny, ix = v / ((long long)g->nz * g->ny);
    const long long id[3] = {ix, iy, iz};
    const int n[3] = {g->nx, g->ny, g->nz};
    const double vs[3] = {g->vx, g->vy, g->vz};
    for (int a = 0; a < 3; ++a) {
        lo[a] = (id[a] - 0.5 * n[a]) * vs[a];
        hi[a] = lo[a] + vs[a];
    }
    return og_clip_len(S, P, lo, hi);
}

/* (A^T y) at the listed voxels only: for each voxel and view, the rays whose
 * pixel lies in the detector footprint of the voxel's eight corners (plus a
 * one-pixel margin) are clipped against the voxel box. */
void og_adjoint_voxels(const og_geom *g, const double *y, const long long *vox, long long n,
                       double *out, int nthreads)
{
    int nt = og_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (long long q = 0; q < n; ++q) {
        long long v = vox[q];
        long long iz = v % g->nz, iy = (v / g->nz) % g->ny, ix = v / ((long long)g->nz * g->ny);
        const long long id[3] = {ix, iy, iz};
        const int nn[3] = {g->nx, g->ny, g->nz};
        const double vs[3] = {g->vx, g->vy, g->vz};
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (id[a] - 0.5 * nn[a]) * vs[a];
            hi[a] = lo[a] + vs[a];
        }
        double acc = 0.0;
        for (int j = 0; j < g->n_views; ++j) {
            double c = cos(g->angles[j]), s = sin(g->angles[j]);
            double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
            for (int corner = 0; corner < 8; ++corner) {
                double X[3] = {(corner & 1) ? hi[0] : lo[0], (corner & 2) ? hi[1] : lo[1],
                               (corner & 4) ? hi[2] : lo[2]};
                /* depth along the central ray from the source */
                double depth = g->dso - (X[0] * c + X[1] * s);
                double mag = g->dsd / depth;
                double u = (-X[0] * s + X[1] * c) * mag;
                double vv = X[2] * mag;
                if (u < umin) umin = u;
                if (u > umax) umax = u;
                if (vv < vmin) vmin = vv;
                if (vv > vmax) vmax = vv;
            }
            int iu0 = (int)floor((umin - g->u_offset) / g->du + (g->nu - 1) / 2.0) - 1;
            int iu1 = (int)ceil((umax - g->u_offset) / g->du + (g->nu - 1) / 2.0) + 1;
            int iv0 = (int)floor(vmin / g->dv + (g->nv - 1) / 2.0) - 1;
            int iv1 = (int)ceil(vmax / g->dv + (g->nv - 1) / 2.0) + 1;
            if (iu0 < 0) iu0 = 0;
            if (iv0 < 0) iv0 = 0;
            if (iu1 > g->nu - 1) iu1 = g->nu - 1;
            if (iv1 > g->nv - 1) iv1 = g->nv - 1;
            for (int iu = iu0; iu <= iu1; ++iu)
                for (int iv = iv0; iv <= iv1; ++iv) {
                    double Sr[3], P[3];
                    og_ray(g, j, iu, iv, Sr, P);
                    double L = og_clip_len(Sr, P, lo, hi);
                    if (L > 0) acc += L * y[og_pidx(g, j, iu, iv)];
                }
        }
        out[q] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Finite differences D (Sec. 2.2), zero-padded to M rows per direction       */
/* ------------------------------------------------------------------------ */

/* g[d*M + i] = (D_d z)_i = z_i - z_{i+e_d}, or 0 when i+e_d leaves the grid. */
void og_grad(int nx, int ny, int nz, const double *z, double *g)
{
    const long long M = (long long)nx * ny * nz;
    for (int ix = 0; ix < nx; ++ix)
        for (int iy = 0; iy < ny; ++iy)
            for (int iz = 0; iz < nz; ++iz) {
                long long i = ((long long)ix * ny + iy) * nz + iz;
                g[i] = (ix + 1 < nx) ? z[i] - z[i + (long long)ny * nz] : 0.0;
                g[M + i] = (iy + 1 < ny) ? z[i] - z[i + nz] : 0.0;
                g[2 * M + i] = (iz + 1 < nz) ? z[i] - z[i + 1] : 0.0;
            }
}

/* out = D^T f for f = (f_x, f_y, f_z) stacked as f[d*M + i]. */
void og_grad_adj(int nx, int ny, int nz, const double *f, double *out)
{
    const long long M = (long long)nx * ny * nz;
    const long long sx = (long long)ny * nz, sy = nz;
    for (int ix = 0; ix < nx; ++ix)
        for (int iy = 0; iy < ny; ++iy)
            for (int iz = 0; iz < nz; ++iz) {
                long long i = ((long long)ix * ny + iy) * nz + iz;
                double acc = 0.0;
                if (ix + 1 < nx) acc += f[i];
                if (ix >= 1) acc -= f[i - sx];
                if (iy + 1 < ny) acc += f[M + i];
                if (iy >= 1) acc -= f[M + i - sy];
                if (iz + 1 < nz) acc += f[2 * M + i];
                if (iz >= 1) acc -= f[2 * M + i - 1];
                out[i] = acc;
            }
}

/* IRN weight per voxel from a stacked gradient field g (3M values).
 * rule 0 (R1, the paper's formula): w = (|g| + tau^2)^(-1/2)
 * rule 1 (R2): w = (|g|^2 + tau^2)^(-1/4)                                    */
void og_weights(long long M, const double *g, double tau, int rule, double *w)
{
    for (long long i = 0; i < M; ++i) {
        double n2 = g[i] * g[i] + g[M + i] * g[M + i] + g[2 * M + i] * g[2 * M + i];
        if (rule == 0) w[i] = 1.0 / sqrt(sqrt(n2) + tau * tau);
        else w[i] = 1.0 / sqrt(sqrt(n2 + tau * tau));
    }
}

/* ------------------------------------------------------------------------ */
/* Augmented operator  A~ = [A; alpha W1 D; lambda W2 D]  (Sec. 2.3)          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const og_geom *g;
    int variant;
    double alpha, lambda;
    const double *w1, *w2; /* M each (w2 unused unless PICCS) */
    long long M, N, R;     /* R = total rows */
    double *tmp3;          /* 3M scratch */
    double *tmpM;          /* M scratch */
    int nthreads;
} og_aug;

static long long og_aug_rows(int variant, long long N, long long M)
{
    switch (variant) {
    case OG_PICCS: return N + 6 * M;
    case OG_PIPLE: return N + 4 * M;
    case OG_TV: return N + 3 * M;
    default: return N;
    }
}

/* out (R) = A~ x */
static void og_aug_apply(og_aug *a, const double *x, double *out)
{
    const long long M = a->M, N = a->N;
    og_forward(a->g, x, out, a->nthreads);
    if (a->variant == OG_CGLS) return;
    og_grad(a->g->nx, a->g->ny, a->g->nz, x, a->tmp3);
    for (int d = 0; d < 3; ++d)
        for (long long i = 0; i < M; ++i)
            out[N + d * M + i] = a->alpha * a->w1[i] * a->tmp3[d * M + i];
    if (a->variant == OG_PICCS) {
        for (int d = 0; d < 3; ++d)
            for (long long i = 0; i < M; ++i)
                out[N + 3 * M + d * M + i] = a->lambda * a->w2[i] * a->tmp3[d * M + i];
    } else if (a->variant == OG_PIPLE) {
        for (long long i = 0; i < M; ++i) out[N + 3 * M + i] = a->lambda * x[i];
    }
}

/* out (M) = A~^T r */
static void og_aug_adjoint(og_aug *a, const double *r, double *out)
{
    const long long M = a->M, N = a->N;
    og_adjoint(a->g, r, out, a->nthreads);
    if (a->variant == OG_CGLS) return;
    for (int d = 0; d < 3; ++d)
        for (long long i = 0; i < M; ++i)
            a->tmp3[d * M + i] = a->alpha * a->w1[i] * r[N + d * M + i];
    og_grad_adj(a->g->nx, a->g->ny, a->g->nz, a->tmp3, a->tmpM);
    for (long long i = 0; i < M; ++i) out[i] += a->tmpM[i];
    if (a->variant == OG_PICCS) {
        for (int d = 0; d < 3; ++d)
            for (long long i = 0; i < M; ++i)
                a->tmp3[d * M + i] = a->lambda * a->w2[i] * r[N + 3 * M + d * M + i];
        og_grad_adj(a->g->nx, a->g->ny, a->g->nz, a->tmp3, a->tmpM);
        for (long long i = 0; i < M; ++i) out[i] += a->tmpM[i];
    } else if (a->variant == OG_PIPLE) {
        for (long long i = 0; i < M; ++i) out[i] += a->lambda * r[N + 3 * M + i];
    }
}

/* b~ = [b; 0; lambda W2 D x_p] (PICCS), [b; 0; lambda x_p] (PIPLE), [b; 0] (TV), b */
static void og_aug_rhs(og_aug *a, const double *b, const double *xp, double *bt)
{
    const long long M = a->M, N = a->N;
    memcpy(bt, b, (size_t)N * sizeof(double));
    if (a->variant == OG_CGLS) return;
    for (long long i = 0; i < 3 * M; ++i) bt[N + i] = 0.0;
    if (a->variant == OG_PICCS) {
        og_grad(a->g->nx, a->g->ny, a->g->nz, xp, a->tmp3);
        for (int d = 0; d < 3; ++d)
            for (long long i = 0; i < M; ++i)
                bt[N + 3 * M + d * M + i] = a->lambda * a->w2[i] * a->tmp3[d * M + i];
    } else if (a->variant == OG_PIPLE) {
        for (long long i = 0; i < M; ++i) bt[N + 3 * M + i] = a->lambda * xp[i];
    }
}

static double og_dot(const double *a, const double *b, long long n)
{
    double s = 0.0;
    for (long long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Textbook CGLS (Hestenes-Stiefel form) on A~ x ~ b~ with FIXED weights,
 * started at x (overwritten with the iterate after `iters` steps, or earlier
 * if ||A~^T r|| falls below 1e-13 of its initial value).
 * resid[k] (if given, iters+1 values) = ||b~ - A~ x_k||^2.
 * Returns the number of steps taken (fewer if the gradient vanished). */
static int og_cgls_core(og_aug *a, const double *bt, double *x, int iters, double *resid)
{
    const long long M = a->M, R = a->R;
    double *r = (double *)malloc((size_t)R * sizeof(double));
    double *q = (double *)malloc((size_t)R * sizeof(double));
    double *s = (double *)malloc((size_t)M * sizeof(double));
    double *p = (double *)malloc((size_t)M * sizeof(double));
    int done = 0;
    og_aug_apply(a, x, q);
    for (long long i = 0; i < R; ++i) r[i] = bt[i] - q[i];
    if (resid) resid[0] = og_dot(r, r, R);
    og_aug_adjoint(a, r, s);
    memcpy(p, s, (size_t)M * sizeof(double));
    double gamma = og_dot(s, s, M);
    const double gamma0 = gamma;
    for (int k = 0; k < iters; ++k) {
        /* stop once the normal-equations residual ||s|| has dropped to 1e-13
         * of its start: past that point the recurrences only amplify rounding */
        if (!(gamma > 1e-26 * gamma0)) break;
        og_aug_apply(a, p, q);
        double delta = og_dot(q, q, R);
        if (!(delta > 0.0)) break;
        double step = gamma / delta;
        for (long long i = 0; i < M; ++i) x[i] += step * p[i];
        for (long long i = 0; i < R; ++i) r[i] -= step * q[i];
        og_aug_adjoint(a, r, s);
        double gnew = og_dot(s, s, M);
        double beta = gnew / gamma;
        for (long long i = 0; i < M; ++i) p[i] = s[i] + beta * p[i];
        gamma = gnew;
        ++done;
        if (resid) resid[done] = og_dot(r, r, R);
    }
    free(r); free(q); free(s); free(p);
    return done;
}

/* LSQR (Paige and Saunders' Golub-Kahan form, the Krylov method Sec. 2.3
 * names as mathematically equivalent to CGLS) on A~ x ~ b~ with FIXED
 * weights, started at x.  Steps, with u, v, w the bidiagonalisation and
 * search vectors:
 *   beta1 u1 = b~ - A~ x0,  alpha1 v1 = A~^T u1,  w1 = v1,
 *   phibar1 = beta1,  rhobar1 = alpha1;  then for each step i
 *   beta_{i+1} u_{i+1} = A~ v_i - alpha_i u_i
 *   alpha_{i+1} v_{i+1} = A~^T u_{i+1} - beta_{i+1} v_i
 *   rho_i = |(rhobar_i, beta_{i+1})|,  c_i = rhobar_i / rho_i,  s_i = beta_{i+1} / rho_i
 *   theta_{i+1} = s_i alpha_{i+1},  rhobar_{i+1} = -c_i alpha_{i+1}
 *   phi_i = c_i phibar_i,  phibar_{i+1} = s_i phibar_i
 *   x_i = x_{i-1} + (phi_i / rho_i) w_i,  w_{i+1} = v_{i+1} - (theta_{i+1} / rho_i) w_i.
 * reorth != 0: every new v is re-orthogonalised against all earlier v by
 * classical Gram-Schmidt applied twice, before its norm is taken.
 * Stops like og_cgls_core: once ||A~^T r_i|| = phibar_{i+1} alpha_{i+1} |c_i|
 * falls to 1e-13 of ||A~^T r_0|| = alpha1 beta1, or when a bidiagonal entry
 * vanishes (the least-squares solution has been reached).
 * resid[i] (if given) = ||b~ - A~ x_i||^2 computed explicitly.
 * basis_out (if given, (iters + 1) x M) receives v_1, v_2, ... in order.
 * Returns the number of steps taken. */
static int og_lsqr_core(og_aug *a, const double *bt, double *x, int iters, int reorth,
                        double *resid, double *basis_out)
{
    const long long M = a->M, R = a->R;
    double *u = (double *)malloc((size_t)R * sizeof(double));
    double *q = (double *)malloc((size_t)R * sizeof(double));
    double *v = (double *)malloc((size_t)M * sizeof(double));
    double *t = (double *)malloc((size_t)M * sizeof(double));
    double *w = (double *)malloc((size_t)M * sizeof(double));
    double *V = reorth ? (double *)malloc((size_t)(iters + 1) * (size_t)M * sizeof(double)) : 0;
    double *h = (double *)malloc((size_t)(iters + 1) * sizeof(double));
    int done = 0;
    og_aug_apply(a, x, q);
    for (long long i = 0; i < R; ++i) u[i] = bt[i] - q[i];
    double beta = sqrt(og_dot(u, u, R));
    if (resid) resid[0] = beta * beta;
    double alpha = 0.0;
    if (beta > 0.0) {
        for (long long i = 0; i < R; ++i) u[i] /= beta;
        og_aug_adjoint(a, u, v);
        alpha = sqrt(og_dot(v, v, M));
    }
    if (alpha > 0.0) {
        for (long long i = 0; i < M; ++i) v[i] /= alpha;
        if (V) memcpy(V, v, (size_t)M * sizeof(double));
        if (basis_out) memcpy(basis_out, v, (size_t)M * sizeof(double));
        memcpy(w, v, (size_t)M * sizeof(double));
        double phibar = beta, rhobar = alpha, normar = alpha * beta;
        const double normar0 = normar;
        for (int k = 0; k < iters; ++k) {
            if (!(normar > 1e-13 * normar0)) break;
            /* beta u <- A~ v - alpha u */
            og_aug_apply(a, v, q);
            for (long long i = 0; i < R; ++i) u[i] = q[i] - alpha * u[i];
            beta = sqrt(og_dot(u, u, R));
            if (beta > 0.0)
                for (long long i = 0; i < R; ++i) u[i] /= beta;
            /* alpha v <- A~^T u - beta v */
            og_aug_adjoint(a, u, t);
            for (long long i = 0; i < M; ++i) t[i] -= beta * v[i];
            if (V) {
                for (int pass = 0; pass < 2; ++pass) {
                    for (int j = 0; j <= k; ++j) h[j] = og_dot(V + (size_t)j * M, t, M);
                    for (int j = 0; j <= k; ++j)
                        for (long long i = 0; i < M; ++i) t[i] -= h[j] * V[(size_t)j * M + i];
                }
            }
            const double alpha_new = sqrt(og_dot(t, t, M));
            /* one Givens rotation of the lower bidiagonal */
            const double rho = hypot(rhobar, beta);
            const double c = rhobar / rho, s = beta / rho;
            const double theta = s * alpha_new;
            rhobar = -c * alpha_new;
            const double phi = c * phibar;
            phibar = s * phibar;
            for (long long i = 0; i < M; ++i) x[i] += (phi / rho) * w[i];
            if (alpha_new > 0.0)
                for (long long i = 0; i < M; ++i) v[i] = t[i] / alpha_new;
            for (long long i = 0; i < M; ++i) w[i] = v[i] - (theta / rho) * w[i];
            if (V && alpha_new > 0.0) memcpy(V + (size_t)(k + 1) * M, v, (size_t)M * sizeof(double));
            if (basis_out && alpha_new > 0.0)
                memcpy(basis_out + (size_t)(k + 1) * M, v, (size_t)M * sizeof(double));
            alpha = alpha_new;
            normar = phibar * alpha_new * fabs(c);
            ++done;
            if (resid) {
                og_aug_apply(a, x, q);
                double r2 = 0.0;
                for (long long i = 0; i < R; ++i) r2 += (bt[i] - q[i]) * (bt[i] - q[i]);
                resid[done] = r2;
            }
            if (!(beta > 0.0) || !(alpha_new > 0.0)) break;
        }
    }
    free(u); free(q); free(v); free(t); free(w); free(h);
    if (V) free(V);
    return done;
}

static void og_aug_init(og_aug *a, const og_geom *g, const double *w1, const double *w2,
                        double alpha, double lambda, int variant, int nthreads)
{
    a->g = g; a->variant = variant; a->alpha = alpha; a->lambda = lambda;
    a->w1 = w1; a->w2 = w2; a->M = og_M(g); a->N = og_N(g);
    a->R = og_aug_rows(variant, a->N, a->M); a->nthreads = nthreads;
    a->tmp3 = (double *)malloc((size_t)(3 * a->M) * sizeof(double));
    a->tmpM = (double *)malloc((size_t)a->M * sizeof(double));
}

/* LSQR with given weights (solver 1: plain, 2: with re-orthogonalisation). */
int og_lsqr_fixed(const og_geom *g, const double *b, const double *xp, const double *w1,
                  const double *w2, double alpha, double lambda, int variant, double *x,
                  int iters, int reorth, double *resid, double *basis_out, int nthreads)
{
    if (og_check(g) != 0) return -1;
    og_aug a;
    og_aug_init(&a, g, w1, w2, alpha, lambda, variant, nthreads);
    double *bt = (double *)malloc((size_t)a.R * sizeof(double));
    og_aug_rhs(&a, b, xp, bt);
    int n = og_lsqr_core(&a, bt, x, iters, reorth, resid, basis_out);
    free(bt); free(a.tmp3); free(a.tmpM);
    return n;
}

/* CGLS with given weights w1, w2 (M each; w2 only used by PICCS). */
int og_cgls_fixed(const og_geom *g, const double *b, const double *xp, const double *w1,
                  const double *w2, double alpha, double lambda, int variant, double *x,
                  int iters, double *resid, int nthreads)
{
    if (og_check(g) != 0) return -1;
    og_aug a;
    a.g = g; a.variant = variant; a.alpha = alpha; a.lambda = lambda;
    a.w1 = w1; a.w2 = w2; a.M = og_M(g); a.N = og_N(g);
    a.R = og_aug_rows(variant, a.N, a.M); a.nthreads = nthreads;
    a.tmp3 = (double *)malloc((size_t)(3 * a.M) * sizeof(double));
    a.tmpM = (double *)malloc((size_t)a.M * sizeof(double));
    double *bt = (double *)malloc((size_t)a.R * sizeof(double));
    og_aug_rhs(&a, b, xp, bt);
    int n = og_cgls_core(&a, bt, x, iters, resid);
    free(bt); free(a.tmp3); free(a.tmpM);
    return n;
}

/* IRN outer loop (Sec. 2.3, Eqs. 10-11).  x holds x_0 on entry and the final
 * iterate on exit.  For each outer k the weights are frozen at the previous
 * iterate, then n_inner steps of the inner solver (solver 0: CGLS, 1: LSQR,
 * 2: LSQR with re-orthogonalisation) are taken on the augmented problem,
 * warm-started at x_{k-1}.  resid (if given) gets n_outer*(n_inner+1) values:
 * the augmented residual before and after every inner step of every cycle.
 * w_out (if given) gets the last cycle's w1 and w2 (2M values). */
int og_irn(const og_geom *g, const double *b, const double *xp, double *x, double alpha,
           double lambda, double tau, int rule, int variant, int n_outer, int n_inner,
           int solver, double *resid, double *w_out, int nthreads)
{
    if (og_check(g) != 0) return -1;
    const long long M = og_M(g);
    double *g3 = (double *)malloc((size_t)(3 * M) * sizeof(double));
    double *w1 = (double *)malloc((size_t)M * sizeof(double));
    double *w2 = (double *)malloc((size_t)M * sizeof(double));
    double *dif = (double *)malloc((size_t)M * sizeof(double));
    for (long long i = 0; i < M; ++i) w1[i] = w2[i] = 0.0;
    for (int k = 0; k < n_outer; ++k) {
        if (variant != OG_CGLS) {
            og_grad(g->nx, g->ny, g->nz, x, g3);
            og_weights(M, g3, tau, rule, w1);
        }
        if (variant == OG_PICCS) {
            for (long long i = 0; i < M; ++i) dif[i] = x[i] - xp[i];
            og_grad(g->nx, g->ny, g->nz, dif, g3);
            og_weights(M, g3, tau, rule, w2);
        }
        double *rk = resid ? resid + (size_t)k * (n_inner + 1) : 0;
        if (solver == 0)
            og_cgls_fixed(g, b, xp, w1, w2, alpha, lambda, variant, x, n_inner, rk, nthreads);
        else
            og_lsqr_fixed(g, b, xp, w1, w2, alpha, lambda, variant, x, n_inner, solver == 2, rk,
                          0, nthreads);
    }
    if (w_out) {
        memcpy(w_out, w1, (size_t)M * sizeof(double));
        memcpy(w_out + M, w2, (size_t)M * sizeof(double));
    }
    free(g3); free(w1); free(w2); free(dif);
    return 0;
}
