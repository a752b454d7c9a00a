"""Seeded synthetic inputs for the cone-beam PICCS reconstruction path.

This module is the one place both the FP64 oracle (``oracle/``) and the CUDA
path get their inputs from.  It holds the scanner geometry *parameters*, the
seeded phantoms, their exact (analytic) line integrals and the Poisson noise
model of the measured data.  It holds none of the reconstruction method's
arithmetic: no voxel projector, no finite differences, no Krylov solver.

Geometry convention (the paper names only DSO, DSD and the detector pitch of
a circular cone-beam scanner, Sec. 3.2; every other choice below is ours and
is shared by the oracle and the CUDA path, each implementing it on its own):

* rotation axis z, volume centred at the origin; voxel ``(ix, iy, iz)``
  occupies ``[(ix - nx/2) vx, (ix + 1 - nx/2) vx] x ...`` and is stored at
  flat index ``(ix*ny + iy)*nz + iz`` (z fastest);
* view ``j`` at angle ``theta_j``: source ``S = DSO (cos, sin, 0)``, detector
  centre ``-(DSD - DSO)(cos, sin, 0)``, detector axes
  ``u = (-sin, cos, 0)`` and ``v = (0, 0, 1)``;
* pixel ``(iu, iv)`` centre ``C + ((iu - (nu-1)/2) du + u_offset) u + (iv - (nv-1)/2) dv v``;
  one ray per pixel, from the source through the pixel centre;
* projection layout ``LAYOUT_UV``: ``(j*nu + iu)*nv + iv`` (v fastest, the
  native one) or ``LAYOUT_VU``: ``(j*nv + iv)*nu + iu`` (u fastest).
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import List, Optional, Sequence

import numpy as np

LAYOUT_UV = 0  # v fastest: (j, iu, iv)
LAYOUT_VU = 1  # u fastest: (j, iv, iu)


# --------------------------------------------------------------------------
# geometry parameters
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Geometry:
    nx: int
    ny: int
    nz: int
    vx: float
    vy: float
    vz: float
    nu: int
    nv: int
    du: float
    dv: float
    dso: float
    dsd: float
    angles: np.ndarray  # radians, float64, shape (n_views,)
    layout: int = LAYOUT_UV
    u_offset: float = 0.0  # detector shift along u (mm)

    @property
    def n_views(self) -> int:
        return int(self.angles.shape[0])

    @property
    def M(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def N(self) -> int:
        return self.n_views * self.nu * self.nv

    def vol_shape(self):
        return (self.nx, self.ny, self.nz)

    def proj_shape(self):
        if self.layout == LAYOUT_UV:
            return (self.n_views, self.nu, self.nv)
        return (self.n_views, self.nv, self.nu)

    def replace(self, **kw) -> "Geometry":
        return dataclasses.replace(self, **kw)


def scan_angles(n_views: int, arc_deg: float, start_deg: float = 0.0) -> np.ndarray:
    """theta_j = start + j * arc / n_views (end point excluded)."""
    j = np.arange(n_views, dtype=np.float64)
    return np.deg2rad(start_deg + j * (arc_deg / n_views))


def ray_endpoints(g: Geometry, views: Optional[Sequence[int]] = None):
    """Source points (V, 3) and pixel centres (V, A, B, 3) in the layout order.

    ``A, B`` are ``(nu, nv)`` for LAYOUT_UV and ``(nv, nu)`` for LAYOUT_VU.
    """
    ang = g.angles if views is None else g.angles[np.asarray(views)]
    c, s = np.cos(ang), np.sin(ang)
    src = np.stack([g.dso * c, g.dso * s, np.zeros_like(c)], axis=-1)
    det_c = np.stack([-(g.dsd - g.dso) * c, -(g.dsd - g.dso) * s, np.zeros_like(c)], axis=-1)
    uhat = np.stack([-s, c, np.zeros_like(c)], axis=-1)
    u = (np.arange(g.nu) - (g.nu - 1) / 2.0) * g.du + g.u_offset
    v = (np.arange(g.nv) - (g.nv - 1) / 2.0) * g.dv
    if g.layout == LAYOUT_UV:
        uu, vv = np.meshgrid(u, v, indexing="ij")
    else:
        vv, uu = np.meshgrid(v, u, indexing="ij")
    pix = (det_c[:, None, None, :]
           + uu[None, :, :, None] * uhat[:, None, None, :])
    pix[..., 2] += vv[None, :, :]
    return src, pix


# --------------------------------------------------------------------------
# analytic primitives (additive attenuation increments, 1/mm)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Ellipsoid:
    center: np.ndarray      # (3,) mm
    semi: np.ndarray        # (3,) mm
    rot: np.ndarray         # (3, 3) columns = ellipsoid axes in world frame
    mu: float


@dataclasses.dataclass
class Box:
    lo: np.ndarray          # (3,) mm, axis aligned
    hi: np.ndarray
    mu: float


@dataclasses.dataclass
class Cylinder:
    p0: np.ndarray          # (3,) axis end points, mm
    p1: np.ndarray
    radius: float
    mu: float


Primitive = object


def _interval_ellipsoid(e: Ellipsoid, S, d):
    """Parameter interval [t0, t1] of x = S + t d inside the ellipsoid."""
    q = (S - e.center) @ e.rot / e.semi
    w = (d @ e.rot) / e.semi
    a = np.einsum("...k,...k->...", w, w)
    b = np.einsum("...k,...k->...", q, w)
    c = np.einsum("...k,...k->...", q, q) - 1.0
    disc = b * b - a * c
    ok = disc > 0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    t0 = np.where(ok, (-b - sq) / a, 0.0)
    t1 = np.where(ok, (-b + sq) / a, 0.0)
    return t0, t1


def _interval_box(lo, hi, S, d):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta = (lo - S) * inv
        tb = (hi - S) * inv
    tmin = np.where(np.isnan(ta), -np.inf, np.minimum(ta, tb))
    tmax = np.where(np.isnan(ta), np.inf, np.maximum(ta, tb))
    # rays parallel to a slab: inside iff the origin coordinate is inside
    par = d == 0
    inside = (S >= lo) & (S <= hi)
    tmin = np.where(par, np.where(inside, -np.inf, np.inf), tmin)
    tmax = np.where(par, np.where(inside, np.inf, -np.inf), tmax)
    t0 = tmin.max(axis=-1)
    t1 = tmax.min(axis=-1)
    return t0, np.maximum(t1, t0)


def _interval_cylinder(cy: Cylinder, S, d):
    ax = cy.p1 - cy.p0
    h = np.linalg.norm(ax)
    a_hat = ax / h
    rel = S - cy.p0
    ra = rel @ a_hat
    da = d @ a_hat
    rp = rel - ra[..., None] * a_hat
    dp = d - da[..., None] * a_hat
    A = np.einsum("...k,...k->...", dp, dp)
    B = np.einsum("...k,...k->...", rp, dp)
    C = np.einsum("...k,...k->...", rp, rp) - cy.radius ** 2
    disc = B * B - A * C
    okc = (disc > 0) & (A > 0)
    sq = np.sqrt(np.where(okc, disc, 0.0))
    Asafe = np.where(A > 0, A, 1.0)
    t0 = np.where(okc, (-B - sq) / Asafe, 0.0)
    t1 = np.where(okc, (-B + sq) / Asafe, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (0.0 - ra) / da
        tb = (h - ra) / da
    s0 = np.where(da != 0, np.minimum(ta, tb), -np.inf)
    s1 = np.where(da != 0, np.maximum(ta, tb), np.inf)
    inside_par = (ra >= 0) & (ra <= h)
    s0 = np.where((da == 0) & ~inside_par, np.inf, s0)
    lo = np.maximum(t0, s0)
    hi = np.minimum(t1, s1)
    hi = np.where(okc, np.maximum(hi, lo), lo)
    return lo, hi


def chord_lengths(prim, S, d) -> np.ndarray:
    """Length (mm) of the segment of the line S + t d (|d| = 1) inside prim."""
    if isinstance(prim, Ellipsoid):
        t0, t1 = _interval_ellipsoid(prim, S, d)
    elif isinstance(prim, Box):
        t0, t1 = _interval_box(prim.lo, prim.hi, S, d)
    elif isinstance(prim, Cylinder):
        t0, t1 = _interval_cylinder(prim, S, d)
    else:
        raise TypeError(prim)
    return np.maximum(t1 - t0, 0.0)


def project_analytic(phantom: List[Primitive], g: Geometry, views=None,
                     chunk_views: int = 8) -> np.ndarray:
    """Exact line integrals of the additive phantom along every ray, float64,
    shaped like ``g.proj_shape()`` (or restricted to ``views``)."""
    vidx = np.arange(g.n_views) if views is None else np.asarray(views)
    out = np.zeros((len(vidx),) + g.proj_shape()[1:], dtype=np.float64)
    for c0 in range(0, len(vidx), chunk_views):
        sel = vidx[c0:c0 + chunk_views]
        src, pix = ray_endpoints(g, sel)
        S = np.broadcast_to(src[:, None, None, :], pix.shape)
        d = pix - S
        d = d / np.linalg.norm(d, axis=-1, keepdims=True)
        acc = np.zeros(pix.shape[:-1])
        for p in phantom:
            acc += p.mu * chord_lengths(p, S, d)
        out[c0:c0 + len(sel)] = acc
    return out


def volume_box_chords(g: Geometry) -> np.ndarray:
    """Length of every ray inside the whole volume box (mm)."""
    half = np.array([g.nx * g.vx, g.ny * g.vy, g.nz * g.vz]) / 2.0
    return project_analytic([Box(-half, half, 1.0)], g)


def _inside(prim, P) -> np.ndarray:
    if isinstance(prim, Ellipsoid):
        q = (P - prim.center) @ prim.rot / prim.semi
        return np.einsum("...k,...k->...", q, q) <= 1.0
    if isinstance(prim, Box):
        return np.all((P >= prim.lo) & (P <= prim.hi), axis=-1)
    if isinstance(prim, Cylinder):
        ax = prim.p1 - prim.p0
        h = np.linalg.norm(ax)
        a_hat = ax / h
        rel = P - prim.p0
        ra = rel @ a_hat
        rp = rel - ra[..., None] * a_hat
        return (ra >= 0) & (ra <= h) & (np.einsum("...k,...k->...", rp, rp) <= prim.radius ** 2)
    raise TypeError(prim)


def voxelize(phantom: List[Primitive], g: Geometry, ss: int = 2) -> np.ndarray:
    """Mean attenuation over each voxel estimated on an ss^3 sub-grid, float64,
    shape (nx, ny, nz).  Each primitive is evaluated only on its bounding box."""
    vol = np.zeros((g.nx, g.ny, g.nz), dtype=np.float64)
    vs = np.array([g.vx, g.vy, g.vz])
    n = np.array([g.nx, g.ny, g.nz])
    sub = (np.arange(ss) + 0.5) / ss
    for p in phantom:
        lo, hi = _bbox(p)
        i0 = np.clip(np.floor(lo / vs + n / 2).astype(int), 0, n)
        i1 = np.clip(np.ceil(hi / vs + n / 2).astype(int), 0, n)
        if np.any(i1 <= i0):
            continue
        axes = []
        for a in range(3):
            idx = np.arange(i0[a], i1[a])
            pts = ((idx[:, None] + sub[None, :]) - n[a] / 2.0) * vs[a]
            axes.append(pts.reshape(-1))
        X, Y, Z = np.meshgrid(*axes, indexing="ij")
        P = np.stack([X, Y, Z], axis=-1)
        ins = _inside(p, P).astype(np.float64)
        shp = tuple(int(i1[a] - i0[a]) for a in range(3))
        frac = ins.reshape(shp[0], ss, shp[1], ss, shp[2], ss).mean(axis=(1, 3, 5))
        vol[i0[0]:i1[0], i0[1]:i1[1], i0[2]:i1[2]] += p.mu * frac
    return vol


def _bbox(p):
    if isinstance(p, Ellipsoid):
        ext = np.sqrt(((p.rot * p.semi[None, :]) ** 2).sum(axis=1))
        return p.center - ext, p.center + ext
    if isinstance(p, Box):
        return p.lo, p.hi
    if isinstance(p, Cylinder):
        lo = np.minimum(p.p0, p.p1) - p.radius
        hi = np.maximum(p.p0, p.p1) + p.radius
        return lo, hi
    raise TypeError(p)


# --------------------------------------------------------------------------
# noise model
# --------------------------------------------------------------------------
def poisson_log_data(line_integrals: np.ndarray, I0: float, seed: int) -> np.ndarray:
    """b = -ln(max(n, 1) / I0),  n ~ Poisson(I0 exp(-integral)), PCG64(seed).
    Zero counts are clamped to one."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = I0 * np.exp(-line_integrals)
    n = rng.poisson(lam).astype(np.float64)
    return -np.log(np.maximum(n, 1.0) / I0)


# --------------------------------------------------------------------------
# seeded phantoms
# --------------------------------------------------------------------------
def random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def ellipsoid_phantom(g: Geometry, n_ell: int, seed: int, mu_lo: float = 0.01,
                      mu_hi: float = 0.04, semi_lo: float = 0.05,
                      semi_hi: float = 0.35, body_mu: float = 0.0) -> List[Primitive]:
    """Additive random ellipsoids inside the inscribed cylinder of the volume.

    Semi-axes are U[semi_lo, semi_hi] times the half width; each ellipsoid is
    shrunk if needed so that its bounding sphere stays inside the cylinder.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    R = 0.5 * min(g.nx * g.vx, g.ny * g.vy)
    H = 0.5 * g.nz * g.vz
    prims: List[Primitive] = []
    if body_mu > 0:
        prims.append(Ellipsoid(np.zeros(3), np.array([0.9 * R, 0.8 * R, 0.9 * H]),
                               np.eye(3), body_mu))
    for _ in range(n_ell):
        semi = rng.uniform(semi_lo, semi_hi, size=3) * R
        rot = random_rotation(rng)
        rr = rng.uniform(0, 0.6) * R
        ang = rng.uniform(0, 2 * np.pi)
        zc = rng.uniform(-0.6, 0.6) * H
        c = np.array([rr * np.cos(ang), rr * np.sin(ang), zc])
        # keep the bounding sphere inside the cylinder
        room = min(0.95 * R - rr, 0.95 * H - abs(zc))
        m = semi.max()
        if m > room:
            semi = semi * (max(room, 0.05 * R) / m)
        mu = float(rng.uniform(mu_lo, mu_hi))
        prims.append(Ellipsoid(c, semi, rot, mu))
    return prims


def random_chord_cylinder(g: Geometry, seed: int, radius: float, mu: float,
                          length: Optional[float] = None) -> Cylinder:
    """A cylinder (needle / screw) along a seeded random line through the
    inner part of the volume; ``length`` None means a chord of the inscribed
    cylinder."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = 0.5 * min(g.nx * g.vx, g.ny * g.vy)
    H = 0.5 * g.nz * g.vz
    c = np.array([rng.uniform(-0.3, 0.3) * R, rng.uniform(-0.3, 0.3) * R,
                  rng.uniform(-0.3, 0.3) * H])
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    half = 0.5 * length if length is not None else 0.7 * min(R, H)
    return Cylinder(c - half * d, c + half * d, radius, mu)


# --------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Scan:
    name: str
    geometry: Geometry
    prior_phantom: List[Primitive]
    scan_phantom: List[Primitive]
    I0: float
    noise_seed: int
    alpha: float
    lam: float
    tau: float
    n_outer: int
    n_inner: int
    prior_file: Optional[str] = None  # stored prior volume (float32 .npy), if any

    @property
    def iterations(self) -> int:
        return self.n_outer * self.n_inner

    def prior_volume(self, ss: int = 2) -> np.ndarray:
        """Prior x_p (float32): the stored fixture when the workload has one
        (a reconstruction from a dense scan of the change-free phantom), else
        the change-free phantom voxelised on an ss^3 sub-grid."""
        if self.prior_file is not None:
            x = np.load(self.prior_file)
            assert x.shape == self.geometry.vol_shape() and x.dtype == np.float32
            return x
        return voxelize(self.prior_phantom, self.geometry, ss).astype(np.float32)

    def truth_volume(self, ss: int = 2) -> np.ndarray:
        return voxelize(self.scan_phantom, self.geometry, ss).astype(np.float32)

    def measured(self) -> np.ndarray:
        """Noisy log-transformed projections b (float32)."""
        li = project_analytic(self.scan_phantom, self.geometry)
        return poisson_log_data(li, self.I0, self.noise_seed).astype(np.float32)


_GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests",
                       "golden")


def c1_small(layout: int = LAYOUT_UV) -> Scan:
    """64^3 x 1 mm, 40 views / 360 deg, 96x96 x 1.2 mm, DSO 1000, DSD 1500,
    additive seeded ellipsoid head (water-like 0.02/mm body) plus a sphere
    of radius 4 voxels (0.025/mm), I0 = 1e5, alpha 0.5, 15 iterations.  The
    prior is the change-free head reconstructed from 360 views (20 plain CGLS
    iterations in the FP64 oracle; tests/golden/make_c1_prior.py)."""
    g = Geometry(64, 64, 64, 1.0, 1.0, 1.0, 96, 96, 1.2, 1.2, 1000.0, 1500.0,
                 scan_angles(40, 360.0), layout)
    prior = ellipsoid_phantom(g, 10, seed=1, mu_lo=-0.004, mu_hi=0.006,
                              semi_lo=0.08, semi_hi=0.3, body_mu=0.02)
    rng = np.random.Generator(np.random.PCG64(101))
    c = np.array([rng.uniform(-10, 10), rng.uniform(-10, 10), rng.uniform(-8, 8)])
    sphere = Ellipsoid(c, np.full(3, 4.0), np.eye(3), 0.005)
    return Scan("c1_64cubed_40views", g, prior, prior + [sphere], 1e5, 11,
                0.5, 0.5, 1e-2, 3, 5, os.path.join(_GOLDEN, "c1_prior_360views.npy"))


def c2_needle(layout: int = LAYOUT_UV) -> Scan:
    """256^3 x 1 mm, 20 ellipsoids mu U[0.01,0.04]/mm, needle r 1 mm mu 0.2/mm
    along a seeded random line, 90 views over a 200 deg short scan,
    512x512 x 0.8 mm, DSO 1000, DSD 1500, I0 5e4, 30 iterations."""
    g = Geometry(256, 256, 256, 1.0, 1.0, 1.0, 512, 512, 0.8, 0.8, 1000.0, 1500.0,
                 scan_angles(90, 200.0), layout)
    prior = ellipsoid_phantom(g, 20, seed=2)
    needle = random_chord_cylinder(g, seed=12, radius=1.0, mu=0.2)
    return Scan("c2_256cubed_90views", g, prior, prior + [needle], 5e4, 12,
                0.5, 0.5, 1e-2, 3, 10)


def c3_sphere_growth(layout: int = LAYOUT_UV) -> Scan:
    """512^3 x 0.5 mm ellipsoids, a 6 mm sphere growing to 8 mm, 100 views /
    360 deg, 1024x768 x 0.4 mm, I0 1e5, 40 iterations."""
    g = Geometry(512, 512, 512, 0.5, 0.5, 0.5, 1024, 768, 0.4, 0.4, 1000.0, 1500.0,
                 scan_angles(100, 360.0), layout)
    base = ellipsoid_phantom(g, 20, seed=3)
    c = np.array([20.0, -15.0, 10.0])
    s6 = Ellipsoid(c, np.full(3, 6.0), np.eye(3), 0.01)
    s8 = Ellipsoid(c, np.full(3, 8.0), np.eye(3), 0.01)
    return Scan("c3_512cubed_100views", g, base + [s6], base + [s8], 1e5, 13,
                0.5, 0.5, 1e-2, 4, 10)


def c5_carm(layout: int = LAYOUT_UV) -> Scan:
    """512x512x400 x 0.6 mm, DSO 750, DSD 1200, 200 views / 200 deg,
    1536x1280 x 0.3 mm, I0 2e4, screw r 3 mm, 40 mm, mu 0.5/mm, 60 its."""
    g = Geometry(512, 512, 400, 0.6, 0.6, 0.6, 1536, 1280, 0.3, 0.3, 750.0, 1200.0,
                 scan_angles(200, 200.0), layout)
    base = ellipsoid_phantom(g, 20, seed=5)
    screw = random_chord_cylinder(g, seed=15, radius=3.0, mu=0.5, length=40.0)
    return Scan("c5_512x512x400_200views", g, base, base + [screw], 2e4, 15,
                0.5, 0.5, 1e-2, 1, 60)


def tiny_geometry(n=(8, 8, 8), vox=(1.0, 1.0, 1.0), det=(12, 10), pitch=(1.5, 1.5),
                  n_views=6, arc=360.0, dso=40.0, dsd=60.0, start=7.0,
                  layout=LAYOUT_UV) -> Geometry:
    """Small geometry for brute-force checks (large cone angle on purpose)."""
    return Geometry(n[0], n[1], n[2], vox[0], vox[1], vox[2], det[0], det[1],
                    pitch[0], pitch[1], dso, dsd, scan_angles(n_views, arc, start), layout)


def random_volume(g: Geometry, seed: int, smooth: bool = False) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(0.0, 1.0, size=g.vol_shape())
    return x


def random_projections(g: Geometry, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, size=g.proj_shape())


def bf16_bits(x) -> np.ndarray:
    """Round float32 values to bfloat16 (to nearest, ties to even) and return
    the 16-bit patterns (uint16): keep the upper half of the float32 bits after
    adding 0x7FFF plus the lowest kept bit.  Finite inputs only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return (u >> 16).astype(np.uint16)


def bf16_values(bits) -> np.ndarray:
    """float32 values of bfloat16 bit patterns."""
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32)
