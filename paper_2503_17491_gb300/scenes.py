"""Seeded synthetic LiDAR scenes shaped like the workloads of Splat-LOAM (arXiv 2503.17491, Sec. 4).

This module only generates inputs: analytic surfaces (planes, vertical cylinders, boxes,
ellipsoids), 2D-Gaussian parameters sampled on them, sensor poses and ray-cast target range and
normal images.  It holds none of the rasterizer's arithmetic, and both the CUDA path and the CPU
oracle consume what it produces.

Parameter distributions (shared by every workload):
  * means: surface samples (area-proportional) plus N(0, 0.02 m) along the surface normal;
  * log-scales: U(-3, -1) per axis (s in [0.05, 0.37] m);
  * rotation: t_n aligned with the surface normal, random in-plane angle, then N(0, 0.05) added to
    every quaternion component (w, x, y, z) and the result normalised;
  * opacity: U(0.3, 0.99), stored as its logit.
Targets: the analytic scene is ray-cast per pixel; range gets N(0, 0.01 m) noise; the target
normal is the exact surface normal turned towards the sensor; rays that miss (or go beyond
``max_range``) get range 0 (invalid pixel).

Image grid (the reading used across the project): column c looks along azimuth
pi - 2 pi (c + 1/2) / W, row r along elevation elev_max - r (elev_max - elev_min) / (H - 1);
x forward, y left, z up (Sec. 3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["View", "Scene", "Rect", "Cylinder", "Ellipsoid", "workload", "tiny_scene",
           "render_targets", "pixel_dirs", "WORKLOADS"]


# --------------------------------------------------------------------------------------------
# analytic surfaces
# --------------------------------------------------------------------------------------------

@dataclass
class Rect:
    c: np.ndarray          # centre
    n: np.ndarray          # unit normal
    u: np.ndarray          # unit in-plane axis
    v: np.ndarray          # unit in-plane axis
    hu: float
    hv: float

    def area(self):
        return 4.0 * self.hu * self.hv

    def bound(self):
        """Centre and radius of a sphere holding the surface."""
        return self.c, math.hypot(self.hu, self.hv)

    def sample(self, k, rng):
        a = rng.uniform(-self.hu, self.hu, k)[:, None]
        b = rng.uniform(-self.hv, self.hv, k)[:, None]
        p = self.c[None] + a * self.u[None] + b * self.v[None]
        return p, np.repeat(self.n[None], k, 0)

    def intersect(self, o, d):
        """o: (3,) origin, d: (R,3) unit dirs -> t (R,), normal (R,3)."""
        dn = d @ self.n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = ((self.c - o) @ self.n) / dn
        p = o[None] + t[:, None] * d
        q = p - self.c[None]
        ok = (np.abs(dn) > 1e-12) & (t > 1e-6) & (np.abs(q @ self.u) <= self.hu) & \
             (np.abs(q @ self.v) <= self.hv)
        t = np.where(ok, t, np.inf)
        return t, np.repeat(self.n[None], len(d), 0)


@dataclass
class Cylinder:
    """Vertical cylinder (pole / trunk)."""
    cx: float
    cy: float
    r: float
    z0: float
    z1: float

    def area(self):
        return 2.0 * math.pi * self.r * (self.z1 - self.z0)

    def bound(self):
        return (np.array([self.cx, self.cy, 0.5 * (self.z0 + self.z1)]),
                math.hypot(self.r, 0.5 * (self.z1 - self.z0)))

    def sample(self, k, rng):
        a = rng.uniform(0, 2 * math.pi, k)
        z = rng.uniform(self.z0, self.z1, k)
        n = np.stack([np.cos(a), np.sin(a), np.zeros(k)], 1)
        p = np.stack([self.cx + self.r * np.cos(a), self.cy + self.r * np.sin(a), z], 1)
        return p, n

    def intersect(self, o, d):
        ox, oy = o[0] - self.cx, o[1] - self.cy
        a = d[:, 0] ** 2 + d[:, 1] ** 2
        b = 2 * (ox * d[:, 0] + oy * d[:, 1])
        c = ox * ox + oy * oy - self.r ** 2
        disc = b * b - 4 * a * c
        with np.errstate(divide="ignore", invalid="ignore"):
            sq = np.sqrt(np.maximum(disc, 0))
            t1 = (-b - sq) / (2 * a)
            t2 = (-b + sq) / (2 * a)
        t = np.where(t1 > 1e-6, t1, t2)
        z = o[2] + t * d[:, 2]
        ok = (disc > 0) & (a > 1e-12) & (t > 1e-6) & (z >= self.z0) & (z <= self.z1)
        t = np.where(ok, t, np.inf)
        p = o[None] + np.where(ok, t, 0)[:, None] * d
        n = np.stack([p[:, 0] - self.cx, p[:, 1] - self.cy, np.zeros(len(d))], 1) / self.r
        return t, n


@dataclass
class Ellipsoid:
    c: np.ndarray
    radii: np.ndarray

    def area(self):
        a, b, c = self.radii
        p = 1.6075
        return 4 * math.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)

    def bound(self):
        return self.c, float(np.max(self.radii))

    def sample(self, k, rng):
        x = rng.normal(size=(k, 3))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        p = self.c[None] + x * self.radii[None]
        n = x / self.radii[None]
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        return p, n

    def intersect(self, o, d):
        oo = (o - self.c) / self.radii
        dd = d / self.radii[None]
        a = np.sum(dd * dd, 1)
        b = 2 * dd @ oo
        c = oo @ oo - 1
        disc = b * b - 4 * a * c
        sq = np.sqrt(np.maximum(disc, 0))
        t1 = (-b - sq) / (2 * a)
        t2 = (-b + sq) / (2 * a)
        t = np.where(t1 > 1e-6, t1, t2)
        ok = (disc > 0) & (t > 1e-6)
        t = np.where(ok, t, np.inf)
        p = o[None] + np.where(ok, t, 0)[:, None] * d
        n = (p - self.c[None]) / self.radii[None] ** 2
        n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-30)
        return t, n


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def box(center, half, yaw=0.0, with_bottom=False):
    """Axis-aligned (up to yaw) box as rectangles."""
    c = np.asarray(center, np.float64)
    hx, hy, hz = half
    cy, sy = math.cos(yaw), math.sin(yaw)
    ex = np.array([cy, sy, 0.0])
    ey = np.array([-sy, cy, 0.0])
    ez = np.array([0.0, 0.0, 1.0])
    faces = [
        Rect(c + hx * ex, ex, ey, ez, hy, hz), Rect(c - hx * ex, -ex, ey, ez, hy, hz),
        Rect(c + hy * ey, ey, ex, ez, hx, hz), Rect(c - hy * ey, -ey, ex, ez, hx, hz),
        Rect(c + hz * ez, ez, ex, ey, hx, hy),
    ]
    if with_bottom:
        faces.append(Rect(c - hz * ez, -ez, ex, ey, hx, hy))
    return faces


def plane_xy(z, cx, cy, hx, hy):
    return Rect(np.array([cx, cy, z], np.float64), np.array([0, 0, 1.0]),
                np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), hx, hy)


# --------------------------------------------------------------------------------------------
# Gaussians on surfaces
# --------------------------------------------------------------------------------------------

def _quat_from_R(R):
    """Rotation matrices (k,3,3) -> unit quaternions (k,4) as (w,x,y,z)."""
    k = R.shape[0]
    q = np.zeros((k, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    cases = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1).argmax(1)
    for case in range(4):
        m = cases == case
        if not m.any():
            continue
        Rm = R[m]
        if case == 0:
            s = np.sqrt(1.0 + tr[m]) * 2
            q[m] = np.stack([0.25 * s, (Rm[:, 2, 1] - Rm[:, 1, 2]) / s,
                             (Rm[:, 0, 2] - Rm[:, 2, 0]) / s, (Rm[:, 1, 0] - Rm[:, 0, 1]) / s], 1)
        elif case == 1:
            s = np.sqrt(1.0 + Rm[:, 0, 0] - Rm[:, 1, 1] - Rm[:, 2, 2]) * 2
            q[m] = np.stack([(Rm[:, 2, 1] - Rm[:, 1, 2]) / s, 0.25 * s,
                             (Rm[:, 0, 1] + Rm[:, 1, 0]) / s, (Rm[:, 0, 2] + Rm[:, 2, 0]) / s], 1)
        elif case == 2:
            s = np.sqrt(1.0 + Rm[:, 1, 1] - Rm[:, 0, 0] - Rm[:, 2, 2]) * 2
            q[m] = np.stack([(Rm[:, 0, 2] - Rm[:, 2, 0]) / s, (Rm[:, 0, 1] + Rm[:, 1, 0]) / s,
                             0.25 * s, (Rm[:, 1, 2] + Rm[:, 2, 1]) / s], 1)
        else:
            s = np.sqrt(1.0 + Rm[:, 2, 2] - Rm[:, 0, 0] - Rm[:, 1, 1]) * 2
            q[m] = np.stack([(Rm[:, 1, 0] - Rm[:, 0, 1]) / s, (Rm[:, 0, 2] + Rm[:, 2, 0]) / s,
                             (Rm[:, 1, 2] + Rm[:, 2, 1]) / s, 0.25 * s], 1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def gaussians_on(points, normals, rng, *, jitter=0.02, log_scale=(-3.0, -1.0),
                 quat_noise=0.05, opacity=(0.3, 0.99)):
    """2D-Gaussian parameters (pos_logit (k,4), quat (k,4), log_scale (k,2)) as float32."""
    k = len(points)
    n = normals / np.linalg.norm(normals, axis=1, keepdims=True)
    mu = points + rng.normal(0.0, jitter, (k, 1)) * n
    # tangent frame: t_a = any unit vector orthogonal to n, rotated by a random angle
    ref = np.where(np.abs(n[:, 2:3]) < 0.9, np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]]))
    t1 = np.cross(ref, n)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(n, t1)
    ang = rng.uniform(0, 2 * math.pi, (k, 1))
    ta = np.cos(ang) * t1 + np.sin(ang) * t2
    tb = np.cross(n, ta)
    R = np.stack([ta, tb, n], 2)   # columns t_a, t_b, t_n (t_n = t_a x t_b)
    q = _quat_from_R(R) + rng.normal(0.0, quat_noise, (k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ls = rng.uniform(log_scale[0], log_scale[1], (k, 2))
    o = rng.uniform(opacity[0], opacity[1], k)
    logit = np.log(o / (1.0 - o))
    pos_logit = np.concatenate([mu, logit[:, None]], 1).astype(np.float32)
    return pos_logit, q.astype(np.float32), ls.astype(np.float32)


def sample_surfaces(surfaces, n_total, rng, **kw):
    areas = np.array([s.area() for s in surfaces])
    counts = rng.multinomial(n_total, areas / areas.sum())
    pts, nrm = [], []
    for s, k in zip(surfaces, counts):
        if k:
            p, nn = s.sample(int(k), rng)
            pts.append(p)
            nrm.append(nn)
    p = np.concatenate(pts)
    nn = np.concatenate(nrm)
    perm = rng.permutation(len(p))
    return gaussians_on(p[perm], nn[perm], rng, **kw)


# --------------------------------------------------------------------------------------------
# views and targets
# --------------------------------------------------------------------------------------------

@dataclass
class View:
    T_ws: np.ndarray      # (4,4) float64, sensor -> world, row-major
    rows: int
    cols: int
    elev_min: float       # radians (float32-representable)
    elev_max: float

    @property
    def n_pixels(self):
        return self.rows * self.cols


@dataclass
class Scene:
    name: str
    pos_logit: np.ndarray
    quat: np.ndarray
    log_scale: np.ndarray
    views: list
    surfaces: list = field(default_factory=list)
    seed: int = 0

    @property
    def n(self):
        return self.pos_logit.shape[0]


def deg(x):
    return float(np.float32(math.radians(x)))


def pixel_dirs(view: View):
    """Unit ray directions (H, W, 3) in the sensor frame."""
    c = np.arange(view.cols)
    r = np.arange(view.rows)
    g = math.pi - 2 * math.pi * (c + 0.5) / view.cols
    th = view.elev_max - r * (view.elev_max - view.elev_min) / (view.rows - 1)
    cg, sg = np.cos(g)[None, :], np.sin(g)[None, :]
    ct, st = np.cos(th)[:, None], np.sin(th)[:, None]
    return np.stack([ct * cg, ct * sg, np.broadcast_to(st, (view.rows, view.cols))], 2)


def render_targets(scene: Scene, view: View, rng=None, noise=0.01, max_range=100.0,
                   chunk=1 << 16):
    """Ray-cast the analytic scene: target range (H,W) f32 with N(0, noise) added, and the exact
    surface normal (3,H,W) f32 in the sensor frame, turned towards the sensor; 0 where invalid."""
    rng = rng if rng is not None else np.random.default_rng(scene.seed + 7)
    d_s = pixel_dirs(view).reshape(-1, 3)
    R = view.T_ws[:3, :3]
    o = view.T_ws[:3, 3]
    d_w = d_s @ R.T
    best = np.full(len(d_w), np.inf)
    nrm = np.zeros((len(d_w), 3))
    # surfaces wholly beyond max_range cannot give a valid hit: left out
    near = []
    for surf in scene.surfaces:
        c, r = surf.bound()
        if np.linalg.norm(np.asarray(c, np.float64) - o) - r <= max_range:
            near.append(surf)
    for s0 in range(0, len(d_w), chunk):
        dw = d_w[s0:s0 + chunk]
        bt = best[s0:s0 + chunk]
        bn = nrm[s0:s0 + chunk]
        for surf in near:
            t, n = surf.intersect(o, dw)
            m = t < bt
            bt[m] = t[m]
            bn[m] = n[m]
    valid = np.isfinite(best) & (best <= max_range)
    n_s = nrm @ R                      # world -> sensor (R^T n as row vectors)
    flipn = np.sum(n_s * d_s, 1) > 0
    n_s[flipn] *= -1
    depth = np.where(valid, best + rng.normal(0.0, noise, len(best)), 0.0)
    depth = np.where(depth > 0, depth, 0.0)
    n_s[~valid] = 0
    return (depth.reshape(view.rows, view.cols).astype(np.float32),
            np.ascontiguousarray(n_s.T.reshape(3, view.rows, view.cols)).astype(np.float32))


def _pose(t=(0, 0, 0), rotvec=(0, 0, 0)):
    T = np.eye(4)
    rv = np.asarray(rotvec, np.float64)
    th = np.linalg.norm(rv)
    if th > 0:
        k = rv / th
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        T[:3, :3] = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    T[:3, 3] = t
    return T


def random_pose(rng, max_t=1.0, max_deg=5.0, base=(0, 0, 0), yaw=0.0):
    """Pose within max_t metres / max_deg degrees of base (and base yaw)."""
    while True:
        t = rng.uniform(-max_t, max_t, 3)
        if np.linalg.norm(t) <= max_t:
            break
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = math.radians(rng.uniform(0, max_deg))
    T = _pose(np.asarray(base) + t, axis * ang)
    Y = _pose(rotvec=(0, 0, yaw))
    T[:3, :3] = Y[:3, :3] @ T[:3, :3]
    return T


# --------------------------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------------------------

GROUND_Z = -1.7


def _street(rng, x0, x1, n_poles):
    yl = rng.uniform(8, 30)
    yr = rng.uniform(8, 30)
    cx, hx = (x0 + x1) / 2, (x1 - x0) / 2
    surf = [plane_xy(GROUND_Z, cx, (yl - yr) / 2, hx, (yl + yr) / 2)]
    top = 12.0
    hz = (top - GROUND_Z) / 2
    zc = GROUND_Z + hz
    surf.append(Rect(np.array([cx, yl, zc]), np.array([0, -1.0, 0]), np.array([1.0, 0, 0]),
                     np.array([0, 0, 1.0]), hx, hz))
    surf.append(Rect(np.array([cx, -yr, zc]), np.array([0, 1.0, 0]), np.array([1.0, 0, 0]),
                     np.array([0, 0, 1.0]), hx, hz))
    for _ in range(n_poles):
        side = rng.choice([-1, 1])
        y = (yl - 2.0) if side > 0 else -(yr - 2.0)
        surf.append(Cylinder(rng.uniform(x0, x1), y + rng.uniform(-0.5, 0.5), 0.3, GROUND_Z, 4.0))
    return surf


def _block(rng, half=50.0):
    """100 x 100 m urban block: ground, buildings on a grid off two crossing streets, poles and a
    few near objects."""
    surf = [plane_xy(GROUND_Z, 0, 0, half, half)]
    for gx in np.arange(-40, 41, 16.0):
        for gy in np.arange(-40, 41, 16.0):
            if abs(gx) < 10 or abs(gy) < 10:
                continue
            hx, hy = rng.uniform(3, 6.5), rng.uniform(3, 6.5)
            h = rng.uniform(5, 25)
            surf += box((gx + rng.uniform(-1, 1), gy + rng.uniform(-1, 1), GROUND_Z + h / 2),
                        (hx, hy, h / 2), yaw=rng.uniform(-0.2, 0.2))
    for _ in range(60):
        x, y = rng.uniform(-45, 45, 2)
        if abs(x) < 8 or abs(y) < 8:
            surf.append(Cylinder(x, y, 0.3, GROUND_Z, 4.0))
    # near objects: ranges down to ~0.5 m
    surf.append(Cylinder(1.2, 0.8, 0.3, GROUND_Z, 1.5))
    surf += box((-2.5, -1.5, GROUND_Z + 0.75), (0.8, 0.4, 0.75))
    return surf


def _city(rng, length=600.0):
    """Long street through buildings, trees (ellipsoid clusters) and vehicles (boxes)."""
    surf = [plane_xy(GROUND_Z, length / 2, 0, length / 2 + 60, 60)]
    x = -40.0
    while x < length + 40:
        for side in (-1, 1):
            w = rng.uniform(8, 25)
            d = rng.uniform(8, 15)
            h = rng.uniform(6, 30)
            y = side * (rng.uniform(10, 18) + d / 2)
            surf += box((x + w / 2, y, GROUND_Z + h / 2), (w / 2, d / 2, h / 2),
                        yaw=rng.uniform(-0.05, 0.05))
        x += rng.uniform(15, 35)
    for _ in range(int(length / 12)):
        tx = rng.uniform(-20, length + 20)
        ty = rng.choice([-1, 1]) * rng.uniform(6, 8)
        surf.append(Cylinder(tx, ty, 0.25, GROUND_Z, 2.5))
        for _k in range(3):
            c = np.array([tx + rng.uniform(-1, 1), ty + rng.uniform(-1, 1), rng.uniform(2.5, 4.5)])
            surf.append(Ellipsoid(c, rng.uniform(1.0, 2.2, 3)))
    for _ in range(int(length / 15)):
        vx = rng.uniform(-20, length + 20)
        vy = rng.choice([-1, 1]) * rng.uniform(2.5, 5)
        surf += box((vx, vy, GROUND_Z + 0.8), (2.2, 0.9, 0.8), yaw=rng.uniform(-0.1, 0.1))
    return surf


def _c1(rng):
    surf = [plane_xy(GROUND_Z, 0, 0, 25, 25)]
    for nrm in ([-1.0, 0, 0], [0, -1.0, 0], [0, 1.0, 0]):
        nrm = np.array(nrm)
        d = rng.uniform(5, 20)
        c = -nrm * d
        u = np.cross(nrm, [0, 0, 1.0])
        hz = (4.0 - GROUND_Z) / 2
        c[2] = GROUND_Z + hz
        surf.append(Rect(c, nrm, _unit(u), np.array([0, 0, 1.0]), 20.0, hz))
    return surf


WORKLOADS = {
    0: "plain forward, 32x512 (elev +-15 deg), 2,000 primitives on 4 planes, identity pose",
    1: "forward + backward, 64x1024 (elev +-22.5 deg), 100,000 primitives on a street with 200 "
       "poles, pose within 1 m / 5 deg",
    2: "single-keyframe refinement step, 128x2048 (elev +-22.5 deg), 1,000,000 primitives over a "
       "100x100 m urban block",
    3: "batched refinement, 12 keyframes (4x 64x1024, 4x 128x1024, 4x 32x1800) along a 50 m "
       "trajectory, one map of 500,000 primitives",
    4: "long incremental mapping run, 300 scans of 128x1024 along a 600 m trajectory, map up to "
       "3,000,000 primitives",
}


def workload(index: int, seed: int | None = None, n: int | None = None) -> Scene:
    """The synthetic scene of one workload (seed defaults to 1000 + index)."""
    seed = 1000 + index if seed is None else seed
    rng = np.random.default_rng(seed)
    if index == 0:
        surf = _c1(rng)
        n = n or 2000
        views = [View(np.eye(4), 32, 512, deg(-15), deg(15))]
    elif index == 1:
        surf = _street(rng, -60, 60, 200)
        n = n or 100_000
        views = [View(random_pose(rng, 1.0, 5.0), 64, 1024, deg(-22.5), deg(22.5))]
    elif index == 2:
        surf = _block(rng)
        n = n or 1_000_000
        views = [View(np.eye(4), 128, 2048, deg(-22.5), deg(22.5))]
    elif index == 3:
        surf = _street(rng, -40, 90, 200)
        n = n or 500_000
        shapes = [(64, 1024, 22.5), (128, 1024, 22.5), (32, 1800, 15.0)] * 4
        views = []
        for k, (h, w, e) in enumerate(shapes):
            x = 50.0 * k / 11 + rng.uniform(-1, 1)
            T = random_pose(rng, 0.5, 3.0, base=(x, rng.uniform(-1.5, 1.5), 0.0),
                            yaw=rng.uniform(-0.15, 0.15))
            views.append(View(T, h, w, deg(-e), deg(e)))
    elif index == 4:
        surf = _city(rng)
        n = n or 3_000_000
        views = []
        for k in range(300):
            x = 600.0 * k / 299
            T = random_pose(rng, 0.2, 1.0, base=(x, 0.5 * math.sin(x / 40.0), 0.0))
            views.append(View(T, 128, 1024, deg(-22.5), deg(22.5)))
    else:
        raise ValueError(index)
    pl, q, ls = sample_surfaces(surf, n, rng)
    return Scene(f"workload{index}", pl, q, ls, views, surf, seed)


def tiny_scene(n: int, seed: int = 0, rows: int = 16, cols: int = 64, fov_deg: float = 20.0,
               spread: float = 1.0, dist=(2.0, 8.0), log_scale=(-2.2, -0.8)) -> Scene:
    """A few primitives in random directions around the sensor (for gradient checks and edge
    cases); one view at identity pose."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(-math.pi, math.pi, n)
    th = rng.uniform(-math.radians(fov_deg) * 0.8, math.radians(fov_deg) * 0.8, n)
    r = rng.uniform(*dist, n)
    p = np.stack([r * np.cos(th) * np.cos(g), r * np.cos(th) * np.sin(g), r * np.sin(th)], 1)
    nrm = -p / np.linalg.norm(p, axis=1, keepdims=True) + rng.normal(0, 0.4 * spread, (n, 3))
    pl, q, ls = gaussians_on(p, nrm, rng, log_scale=log_scale)
    view = View(np.eye(4), rows, cols, deg(-fov_deg), deg(fov_deg))
    return Scene(f"tiny{n}_{seed}", pl, q, ls, [view], [], seed)
