// FP64 construction of the per-view ray tables used by the projector
// kernels (host code, shared by the library and its host-side checks).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/piccs.h"
#include "internal.h"

namespace piccs {

// FP64 ray tables: per (view, column) xy-walk constants and per-row heights.
inline void build_tables(const piccs_geometry *g, std::vector<ColParams> &cols, std::vector<float> &vrow)
{
    const double Wx = g->nx * g->vx, Wy = g->ny * g->vy;
    cols.assign((size_t)g->n_views * g->nu, ColParams{});
    vrow.resize(g->nv);
    for (int iv = 0; iv < g->nv; ++iv) vrow[iv] = (float)((iv - 0.5 * (g->nv - 1)) * g->dv);
    for (int j = 0; j < g->n_views; ++j) {
        const double cth = std::cos(g->angles_rad[j]), sth = std::sin(g->angles_rad[j]);
        const double Sx = g->dso * cth, Sy = g->dso * sth;
        const double back = g->dsd - g->dso;
        for (int iu = 0; iu < g->nu; ++iu) {
            ColParams &cp = cols[(size_t)j * g->nu + iu];
            const double u = (iu - 0.5 * (g->nu - 1)) * g->du;
            const double Px = -back * cth - u * sth, Py = -back * sth + u * cth;
            const double dx = Px - Sx, dy = Py - Sy;
            const double D = std::sqrt(dx * dx + dy * dy);
            const double cx = dx / D, cy = dy / D;
            // xy slab clip of the source->pixel segment against the volume square
            double s0 = 0.0, s1 = D;
            bool hit = true;
            const double c2[2] = {cx, cy}, S2[2] = {Sx, Sy}, W2[2] = {Wx, Wy};
            for (int a = 0; a < 2; ++a) {
                const double lo = -0.5 * W2[a], hi = 0.5 * W2[a];
                if (c2[a] == 0.0) {
                    if (S2[a] < lo || S2[a] > hi) hit = false;
                    continue;
                }
                double ta = (lo - S2[a]) / c2[a], tb = (hi - S2[a]) / c2[a];
                if (ta > tb) std::swap(ta, tb);
                s0 = std::max(s0, ta);
                s1 = std::min(s1, tb);
            }
            if (!hit || !(s1 > s0)) {
                cp.L = 0.f;
                continue;
            }
            // entry point in voxel units, rounded once to FP32; the start cell is
            // taken from the rounded value so that the first plane ahead of it
            // is never crossed at s < 0
            const double exd = (Sx + s0 * cx + 0.5 * Wx) / g->vx;
            const double eyd = (Sy + s0 * cy + 0.5 * Wy) / g->vy;
            const double span = s1 - s0;
            auto axis = [&](double e, double c, double vox, int n, float &inv, float &ef, int &i0,
                            int &step) {
                if (std::fabs(c) * span / vox < 1e-7) {
                    // parallel to this axis' planes over the whole chord
                    inv = INFINITY;
                    ef = -1e30f;
                    step = 1;
                    i0 = std::min(std::max((int)std::floor(e), 0), n - 1);
                    return;
                }
                ef = (float)e;
                inv = (float)(vox / c);  // xy distance per voxel step
                step = c > 0.0 ? 1 : -1;
                i0 = std::min(std::max((int)std::floor(ef), 0), n - 1);
            };
            axis(exd, cx, g->vx, g->nx, cp.inv_dx, cp.ex, cp.ix0, cp.stepx);
            axis(eyd, cy, g->vy, g->ny, cp.inv_dy, cp.ey, cp.iy0, cp.stepy);
            cp.L = (float)(s1 - s0);
            cp.kE = (float)(s0 / (D * g->vz));
            cp.KD = (float)(g->vz * D);
            cp.invD = (float)(1.0 / D);
        }
    }
}

}  // namespace piccs
