// FP64 construction of the per-view ray tables used by the projector
// kernels (host code, shared by the library and its host-side checks).
//
// For every (view, detector column) the xy part of the Siddon walk is the same
// for all rows of the column, so it is walked once here, in FP64, and stored as
// the list of xy cells the column's rays cross: per cell the flat index of its
// first voxel and the xy distance (mm, measured from the entry into the
// volume's xy square) at which the rays leave it, rounded once to FP32.  The
// kernels then only add the z crossings, per row, in FP32.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/piccs.h"
#include "internal.h"

namespace piccs {

// Cells reserved per column: a column crosses at most nx + ny - 1 cells;
// rounded up to an even count (two cells per 16-byte load).
inline int cell_stride(const piccs_geometry *g) { return ((g->nx + g->ny + 1) / 2) * 2; }

// Walks one column in FP64; fills cp (z constants, cell count) and the
// column's cell list (two ints per cell: first voxel index, exit distance
// bits), padded to an even count; returns the number of cells.
inline int walk_column(const piccs_geometry *g, int j, int iu, ColParams &cp, int *cells)
{
    const double Wx = g->nx * g->vx, Wy = g->ny * g->vy;
    const double cth = std::cos(g->angles_rad[j]), sth = std::sin(g->angles_rad[j]);
    const double Sx = g->dso * cth, Sy = g->dso * sth;
    const double back = g->dsd - g->dso;
    const double u = (iu - 0.5 * (g->nu - 1)) * g->du + g->u_offset;
    const double Px = -back * cth - u * sth, Py = -back * sth + u * cth;
    const double dx = Px - Sx, dy = Py - Sy;
    const double D = std::sqrt(dx * dx + dy * dy);
    const double cx = dx / D, cy = dy / D;
    cp = ColParams{};
    // xy slab clip of the source->pixel segment against the volume square
    double s0 = 0.0, s1 = D;
    const double c2[2] = {cx, cy}, S2[2] = {Sx, Sy}, W2[2] = {Wx, Wy};
    for (int a = 0; a < 2; ++a) {
        const double lo = -0.5 * W2[a], hi = 0.5 * W2[a];
        if (c2[a] == 0.0) {
            if (S2[a] < lo || S2[a] > hi) return 0;
            continue;
        }
        double ta = (lo - S2[a]) / c2[a], tb = (hi - S2[a]) / c2[a];
        if (ta > tb) std::swap(ta, tb);
        s0 = std::max(s0, ta);
        s1 = std::min(s1, tb);
    }
    if (!(s1 > s0)) return 0;
    const double L = s1 - s0;
    const double ex = (Sx + s0 * cx + 0.5 * Wx) / g->vx;  // entry point, voxel units
    const double ey = (Sy + s0 * cy + 0.5 * Wy) / g->vy;
    int ix = std::min(std::max((int)std::floor(ex), 0), g->nx - 1);
    int iy = std::min(std::max((int)std::floor(ey), 0), g->ny - 1);
    const int stx = cx >= 0.0 ? 1 : -1, sty = cy >= 0.0 ? 1 : -1;
    const double invx = cx != 0.0 ? g->vx / cx : 0.0;  // xy distance per voxel step
    const double invy = cy != 0.0 ? g->vy / cy : 0.0;
    auto next_x = [&](int i) {
        return cx != 0.0 ? std::max(((i + (stx > 0)) - ex) * invx, 0.0) : INFINITY;
    };
    auto next_y = [&](int i) {
        return cy != 0.0 ? std::max(((i + (sty > 0)) - ey) * invy, 0.0) : INFINITY;
    };
    cp.s0 = (float)s0;
    cp.KD = (float)(g->vz * D);
    cp.invD = (float)(1.0 / D);
    cp.rKD = (float)(1.0 / (g->vz * D));
    double sxn = next_x(ix), syn = next_y(iy);
    int n = 0;
    for (;;) {
        const double se = std::min(std::min(sxn, syn), L);
        bool last = se >= L;
        const bool xstep = sxn <= syn;
        if (!last) last = xstep ? (unsigned)(ix + stx) >= (unsigned)g->nx
                                : (unsigned)(iy + sty) >= (unsigned)g->ny;
        const float e = (float)se;
        cells[2 * n] = (ix * g->ny + iy) * g->nz;
        std::memcpy(&cells[2 * n + 1], &e, 4);
        ++n;
        if (last) break;
        if (xstep) {
            ix += stx;
            sxn = next_x(ix);
        } else {
            iy += sty;
            syn = next_y(iy);
        }
    }
    cp.ncells = n;
    if (n & 1) {  // pad: a zero-length copy of the last cell
        cells[2 * n] = cells[2 * n - 2];
        cells[2 * n + 1] = cells[2 * n - 1];
    }
    return n;
}

// Per (view, column) constants, per-row {v, 1/v} (1e30 for v = 0), the cell
// table (cell_stride cells per column, column (j, iu) at cell offset
// (j*nu + iu)*stride) and its transpose: for every xy voxel column
// (ix*ny + iy) the crossings hits[hit_ptr[c] .. hit_ptr[c+1]) by detector
// columns, in view-then-column order.
inline void build_tables(const piccs_geometry *g, std::vector<ColParams> &cols,
                         std::vector<float2> &vr, std::vector<int> &cells,
                         std::vector<int> &hit_ptr, std::vector<CellHit> &hits)
{
    const size_t ncol = (size_t)g->n_views * g->nu;
    const int stride = cell_stride(g);
    cols.assign(ncol, ColParams{});
    cells.assign(ncol * (size_t)stride * 2, 0);
    vr.resize(g->nv);
    for (int iv = 0; iv < g->nv; ++iv) {
        const double v = (iv - 0.5 * (g->nv - 1)) * g->dv;
        vr[iv].x = (float)v;
        vr[iv].y = v != 0.0 ? (float)(1.0 / v) : 1e30f;
    }
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    nt = (unsigned)std::min<size_t>(nt, (size_t)g->n_views);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t) {
        pool.emplace_back([&, t]() {
            for (int j = (int)t; j < g->n_views; j += (int)nt)
                for (int iu = 0; iu < g->nu; ++iu) {
                    const size_t c = (size_t)j * g->nu + iu;
                    walk_column(g, j, iu, cols[c], cells.data() + c * stride * 2);
                    cols[c].start2 = (long long)(c * stride / 2);
                }
        });
    }
    for (auto &th : pool) th.join();

    // transpose: count crossings per voxel column, then fill in column order
    const size_t nxy = (size_t)g->nx * g->ny;
    hit_ptr.assign(nxy + 1, 0);
    auto for_each_cell = [&](auto &&fn) {
        for (size_t c = 0; c < ncol; ++c) {
            const int *e = cells.data() + c * stride * 2;
            float sa = 0.f;
            for (int k = 0; k < cols[c].ncells; ++k) {
                float sb;
                std::memcpy(&sb, &e[2 * k + 1], 4);
                fn(c, (size_t)(e[2 * k] / g->nz), sa, sb);
                sa = sb;
            }
        }
    };
    for_each_cell([&](size_t, size_t cell, float, float) { hit_ptr[cell + 1] += 1; });
    for (size_t i = 0; i < nxy; ++i) hit_ptr[i + 1] += hit_ptr[i];
    hits.assign((size_t)hit_ptr[nxy], CellHit{});
    std::vector<int> fill(hit_ptr.begin(), hit_ptr.end() - 1);
    for_each_cell([&](size_t c, size_t cell, float sa, float sb) {
        const int j = (int)(c / g->nu), iu = (int)(c % g->nu);
        CellHit h;
        h.x = (j << 16) | iu;
        std::memcpy(&h.y, &sa, 4);
        std::memcpy(&h.z, &sb, 4);
        h.w = 0;
        hits[(size_t)fill[cell]++] = h;
    });
}

// Upper bound of the number of crossings (for sizing the workspace before the
// tables are built): every column crosses at most nx + ny - 1 voxel columns.
inline size_t hit_bound(const piccs_geometry *g)
{
    return (size_t)g->n_views * g->nu * (size_t)(g->nx + g->ny - 1);
}

}  // namespace piccs
