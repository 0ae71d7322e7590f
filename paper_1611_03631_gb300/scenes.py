"""Seeded synthetic scenes and posed scans (sensor simulation only).

This module is the single source of input bytes for both the CUDA path and the
CPU oracle. It simulates sensors against analytic scenes in float64 and emits
float32 sensor-frame points plus float32 row-major 4x4 poses T_world_sensor.
It contains none of the mapping method's arithmetic (no transform into the map,
no binning, no raycasting into voxels, no TSDF or ESDF math).

Scenes (the paper's datasets, EuRoC V1_01_easy and the cow dataset of Sec. VI,
are not available; these stand in for them):

* ``plane_sphere``: ground plane z=0 and a sphere of radius 1 m at (0,0,1),
  ten 64x48 pinhole frames (fx=fy=50, cx=32, cy=24) on a 3 m circle at 1.5 m
  height looking at the origin; range noise N(0, 5 mm) along each ray.
* ``room``: 10 x 10 x 3 m room with 20 seeded boxes, spheres and vertical
  cylinders (0.2-1.5 m); 640x480 RGB-D frames (fx=fy=525, cx=319.5,
  cy=239.5) along a Catmull-Rom random walk at 1.2-1.8 m height with yaw along
  the path; depth noise sigma = 0.0012 z^2; depth beyond 5 m is invalid.
* ``lidar_terrain``: 200 x 200 m heightfield (sum of 8 sinusoids, 3 m total
  amplitude), 300 box buildings (4-20 m), 500 cylinder trees; 64 x 2048 beam
  spinning LiDAR (elevation -25..+15 deg, 60 m max range, sigma 2 cm) along a
  400 m path; no-returns are invalid.

Invalid measurements are emitted as NaN rows so that the map's input filter
(non-finite points are dropped) sees them.

For the mesh, ``synthetic_tsdf`` stands in for a fused map: per-voxel (D, W) values sampled
from the ESDF benchmark scene's analytic distance with noise, clipped to the truncation band,
with unobserved voxels, missing blocks and exact zeros (it is not the fusion of Eq. (1)-(3)).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

__all__ = [
    "ScanSet",
    "plane_sphere",
    "room",
    "lidar_terrain",
    "random_queries",
    "esdf_benchmark",
    "esdf_benchmark_sdf",
    "synthetic_tsdf",
    "make_scene",
]


@dataclasses.dataclass
class ScanSet:
    """A sequence of posed scans plus the map parameters the scene is run with."""

    name: str
    points: List[np.ndarray]  # per scan: (N, 3) float32, sensor frame, NaN = invalid
    poses: List[np.ndarray]  # per scan: (4, 4) float32 row-major T_world_sensor
    params: Dict[str, float]
    meta: Dict[str, object] = dataclasses.field(default_factory=dict)

    def __len__(self) -> int:
        return len(self.points)


# --------------------------------------------------------------------------------------
# camera / pose helpers


def _look_at(pos: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Optical-frame rotation (x right, y down, z forward) looking from pos to target."""
    f = target - pos
    f = f / np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    x = np.cross(f, up)
    x = x / np.linalg.norm(x)
    y = np.cross(f, x)
    return np.stack([x, y, f], axis=1)


def _yaw_camera(yaw: float) -> np.ndarray:
    """Optical-frame rotation of a level camera whose forward axis has heading yaw."""
    f = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    return _look_at(np.zeros(3), f)


def _yaw_lidar(yaw: float) -> np.ndarray:
    """LiDAR frame (x forward, y left, z up) rotated by yaw about world z."""
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _pose(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T.astype(np.float32)


def _pinhole_dirs(w: int, h: int, fx: float, fy: float, cx: float, cy: float) -> np.ndarray:
    """Per-pixel ray directions with unit z, row-major over (v, u)."""
    u, v = np.meshgrid(np.arange(w, dtype=np.float64), np.arange(h, dtype=np.float64))
    d = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1)
    return d.reshape(-1, 3)


def _catmull_rom(pts: np.ndarray, samples: int) -> np.ndarray:
    """Uniform Catmull-Rom spline through pts (K, D), sampled at `samples` points."""
    P = np.concatenate([pts[:1], pts, pts[-1:]], axis=0)
    nseg = len(pts) - 1
    out = []
    for i in range(samples):
        s = i / max(samples - 1, 1) * nseg
        k = min(int(s), nseg - 1)
        t = s - k
        p0, p1, p2, p3 = P[k], P[k + 1], P[k + 2], P[k + 3]
        t2, t3 = t * t, t * t * t
        out.append(
            0.5
            * (
                2 * p1
                + (-p0 + p2) * t
                + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                + (-p0 + 3 * p1 - 3 * p2 + p3) * t3
            )
        )
    return np.asarray(out)


# --------------------------------------------------------------------------------------
# analytic ray intersections (float64, vectorised over rays)


def _hit_plane_z(o, u, z0=0.0):
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (z0 - o[..., 2]) / u[..., 2]
    return np.where((t > 1e-9) & np.isfinite(t), t, np.inf)


def _hit_sphere(o, u, c, r):
    oc = o - c
    b = np.sum(oc * u, axis=-1)
    cc = np.sum(oc * oc, axis=-1) - r * r
    disc = b * b - cc
    sq = np.sqrt(np.maximum(disc, 0.0))
    t0 = -b - sq
    t1 = -b + sq
    t = np.where(t0 > 1e-9, t0, np.where(t1 > 1e-9, t1, np.inf))
    return np.where(disc >= 0.0, t, np.inf)


def _hit_box_outside(o, u, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / u
        t1 = (lo - o) * inv
        t2 = (hi - o) * inv
    tmin = np.nanmax(np.minimum(t1, t2), axis=-1)
    tmax = np.nanmin(np.maximum(t1, t2), axis=-1)
    hit = (tmax >= tmin) & (tmin > 1e-9)
    return np.where(hit, tmin, np.inf)


def _hit_box_inside(o, u, lo, hi):
    """Exit distance of rays starting inside an axis-aligned box (room walls)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(u > 0, (hi - o) / u, np.where(u < 0, (lo - o) / u, np.inf))
    return np.min(t, axis=-1)


def _hit_cylinder_z(o, u, cxy, r, z0, z1):
    """Vertical capped cylinder: side wall plus top cap."""
    dx = o[..., 0] - cxy[0]
    dy = o[..., 1] - cxy[1]
    a = u[..., 0] ** 2 + u[..., 1] ** 2
    b = dx * u[..., 0] + dy * u[..., 1]
    c = dx * dx + dy * dy - r * r
    with np.errstate(divide="ignore", invalid="ignore"):
        disc = b * b - a * c
        sq = np.sqrt(np.maximum(disc, 0.0))
        ts = (-b - sq) / a
    zs = o[..., 2] + ts * u[..., 2]
    side = np.where((disc >= 0) & (a > 1e-12) & (ts > 1e-9) & (zs >= z0) & (zs <= z1), ts, np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        tt = (z1 - o[..., 2]) / u[..., 2]
    px = dx + tt * u[..., 0]
    py = dy + tt * u[..., 1]
    top = np.where((tt > 1e-9) & (px * px + py * py <= r * r), tt, np.inf)
    return np.minimum(side, top)


# --------------------------------------------------------------------------------------
# scene 1: plane + sphere


def plane_sphere(
    frames: int = 10,
    width: int = 64,
    height: int = 48,
    fx: float = 50.0,
    fy: float = 50.0,
    cx: float = 32.0,
    cy: float = 24.0,
    noise: float = 0.005,
    seed: int = 1,
) -> ScanSet:
    """Ground plane z=0 plus a sphere r=1 m at (0,0,1), cameras on a 3 m circle."""
    rng = np.random.default_rng(seed)
    dirs = _pinhole_dirs(width, height, fx, fy, cx, cy)
    dn = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    pts, poses = [], []
    for k in range(frames):
        a = 2.0 * math.pi * k / frames
        pos = np.array([3.0 * math.cos(a), 3.0 * math.sin(a), 1.5])
        R = _look_at(pos, np.zeros(3))
        uw = dn @ R.T
        o = np.broadcast_to(pos, uw.shape)
        t = np.minimum(_hit_plane_z(o, uw), _hit_sphere(o, uw, np.array([0.0, 0.0, 1.0]), 1.0))
        t = t + rng.normal(0.0, noise, size=t.shape)
        p = dn * t[:, None]
        p[~np.isfinite(t)] = np.nan
        pts.append(p.astype(np.float32))
        poses.append(_pose(R, pos))
    params = dict(
        voxel_size=0.1,
        voxels_per_block=8,
        truncation=0.3,
        max_esdf_dist=2.0,
        weighting=0,
        eps=0.1,
        fixed_band=0.1,
        max_range=math.inf,
    )
    return ScanSet("plane_sphere", pts, poses, params)


def plane_sphere_sdf(x: np.ndarray) -> np.ndarray:
    """True signed distance of the plane_sphere scene (positive in free space)."""
    ds = np.linalg.norm(x - np.array([0.0, 0.0, 1.0]), axis=-1) - 1.0
    return np.minimum(x[..., 2], ds)


# --------------------------------------------------------------------------------------
# scene 2: room


def _room_objects(rng: np.random.Generator, path: np.ndarray, n: int, size: float):
    objs = []
    tries = 0
    while len(objs) < n and tries < 10000:
        tries += 1
        kind = int(rng.integers(0, 3))
        s = float(rng.uniform(0.2, 1.5))
        c = np.array([rng.uniform(0.3, size - 0.3), rng.uniform(0.3, size - 0.3)])
        dmin = np.min(np.linalg.norm(path[:, :2] - c, axis=1))
        if dmin < s * 0.75 + 0.4:
            continue
        if kind == 0:  # box standing on the floor
            h = float(rng.uniform(0.2, 1.5))
            lo = np.array([c[0] - s / 2, c[1] - s / 2, 0.0])
            hi = np.array([c[0] + s / 2, c[1] + s / 2, h])
            objs.append(("box", lo, hi))
        elif kind == 1:  # sphere floating or resting
            r = s / 2
            z = float(rng.uniform(r, 3.0 - r))
            objs.append(("sphere", np.array([c[0], c[1], z]), r))
        else:  # vertical cylinder on the floor
            r = s / 2
            h = float(rng.uniform(0.2, 1.5))
            objs.append(("cyl", c, r, 0.0, h))
    return objs


def room(
    frames: int = 30,
    width: int = 640,
    height: int = 480,
    fx: float = 525.0,
    fy: float = 525.0,
    cx: Optional[float] = None,
    cy: Optional[float] = None,
    n_objects: int = 20,
    max_depth: float = 5.0,
    seed: int = 2,
    size: float = 10.0,
    voxel_size: float = 0.05,
    block: int = 16,
) -> ScanSet:
    """10 x 10 x 3 m room with seeded objects and an RGB-D camera random walk."""
    if cx is None:
        cx = (width - 1) / 2.0
    if cy is None:
        cy = (height - 1) / 2.0
    rng = np.random.default_rng(seed)
    way = np.stack(
        [
            rng.uniform(1.5, size - 1.5, 6),
            rng.uniform(1.5, size - 1.5, 6),
            rng.uniform(1.2, 1.8, 6),
        ],
        axis=1,
    )
    path = _catmull_rom(way, max(frames, 2) + 1)
    objs = _room_objects(rng, path, n_objects, size)
    dirs = _pinhole_dirs(width, height, fx, fy, cx, cy)
    dlen = np.linalg.norm(dirs, axis=1)
    dn = dirs / dlen[:, None]
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([size, size, 3.0])
    pts, poses = [], []
    for k in range(frames):
        pos = path[k]
        tang = path[k + 1] - path[k]
        yaw = math.atan2(tang[1], tang[0])
        R = _yaw_camera(yaw)
        uw = dn @ R.T
        o = np.broadcast_to(pos, uw.shape)
        t = _hit_box_inside(o, uw, lo, hi)
        for ob in objs:
            if ob[0] == "box":
                t = np.minimum(t, _hit_box_outside(o, uw, ob[1], ob[2]))
            elif ob[0] == "sphere":
                t = np.minimum(t, _hit_sphere(o, uw, ob[1], ob[2]))
            else:
                t = np.minimum(t, _hit_cylinder_z(o, uw, ob[1], ob[2], ob[3], ob[4]))
        z = t / dlen  # depth along the optical axis
        z = z + rng.normal(0.0, 1.0, size=z.shape) * 0.0012 * z * z
        p = dirs * z[:, None]
        p[~(np.isfinite(z) & (z > 0.0) & (z <= max_depth))] = np.nan
        pts.append(p.astype(np.float32))
        poses.append(_pose(R, pos))
    params = dict(
        voxel_size=voxel_size,
        voxels_per_block=block,
        truncation=2.0 * voxel_size,
        max_esdf_dist=2.0,
        weighting=1,
        eps=voxel_size,
        fixed_band=voxel_size,
        max_range=math.inf,
    )
    return ScanSet("room", pts, poses, params, meta=dict(objects=len(objs)))


# --------------------------------------------------------------------------------------
# scene 3: LiDAR over terrain


class _Terrain:
    def __init__(self, rng: np.random.Generator, amplitude: float = 3.0):
        self.k = rng.uniform(2 * math.pi / 120.0, 2 * math.pi / 15.0, size=8)
        ang = rng.uniform(0, 2 * math.pi, size=8)
        self.fx = self.k * np.cos(ang)
        self.fy = self.k * np.sin(ang)
        self.ph = rng.uniform(0, 2 * math.pi, size=8)
        a = rng.uniform(0.5, 1.0, size=8)
        self.a = a / a.sum() * amplitude
        self.hmax = float(self.a.sum())
        self.slope = float(np.sum(self.a * self.k))

    def h(self, x, y):
        out = np.zeros(np.broadcast(x, y).shape)
        for i in range(8):
            out += self.a[i] * np.sin(self.fx[i] * x + self.fy[i] * y + self.ph[i])
        return out

    def hit(self, o: np.ndarray, u: np.ndarray, tmax: float) -> np.ndarray:
        """First crossing of rays with the heightfield: fixed-step march plus bisection."""
        n = o.shape[0]
        t_hit = np.full(n, np.inf)
        # Rays that start above every terrain point and do not descend never hit.
        active = np.nonzero(~((o[:, 2] > self.hmax) & (u[:, 2] >= 0.0)))[0]
        step = 0.5
        t_prev = 0.0
        while active.size and t_prev < tmax:
            t = t_prev + step
            oo = o[active]
            uu = u[active]
            p = oo + uu * t
            f = p[:, 2] - self.h(p[:, 0], p[:, 1])
            crossed = f <= 0.0
            if np.any(crossed):
                idx = np.nonzero(crossed)[0]
                lo = np.full(idx.size, t_prev)
                hi = np.full(idx.size, t)
                oi, ui = oo[idx], uu[idx]
                for _ in range(30):
                    mid = 0.5 * (lo + hi)
                    pm = oi + ui * mid[:, None]
                    fm = pm[:, 2] - self.h(pm[:, 0], pm[:, 1])
                    below = fm <= 0.0
                    hi = np.where(below, mid, hi)
                    lo = np.where(below, lo, mid)
                t_hit[active[idx]] = 0.5 * (lo + hi)
            # drop rays that crossed or climbed above every terrain point
            keep = ~crossed & ~((p[:, 2] > self.hmax) & (uu[:, 2] >= 0.0))
            active = active[keep]
            t_prev = t
        return t_hit


def _lidar_scan(args):
    """Scan k of a LiDAR world (run in a worker process when scans are generated in parallel).
    The range noise of scan k comes from its own generator, seeded by (seed, k), so the scans
    do not depend on how many workers generate them or in which order."""
    w, k = args
    ter, pxy, dirs = w["terrain"], w["pxy"], w["dirs"]
    beams, columns, max_range = w["beams"], w["columns"], w["max_range"]
    buildings, trees, b_center, t_center = w["buildings"], w["trees"], w["b_center"], w["t_center"]
    azim = np.arange(columns) * (2 * math.pi / columns)
    xy = pxy[k]
    pos = np.array([xy[0], xy[1], float(ter.h(xy[0], xy[1])) + w["sensor_height"]])
    tang = pxy[k + 1] - pxy[k]
    yaw = math.atan2(tang[1], tang[0])
    R = _yaw_lidar(yaw)
    uw = dirs @ R.T
    o = np.broadcast_to(pos, uw.shape).copy()
    t = ter.hit(o, uw, max_range)
    col_az = yaw + azim  # world azimuth of each column

    def _cols(center, rb):
        dvec = center - xy
        D = float(np.hypot(dvec[0], dvec[1]))
        if D <= rb:
            return np.arange(columns)
        phi = math.atan2(dvec[1], dvec[0])
        hw = math.asin(min(1.0, rb / D)) + 2.0 * (2 * math.pi / columns)
        diff = np.angle(np.exp(1j * (col_az - phi)))
        return np.nonzero(np.abs(diff) <= hw)[0]

    def _rays(cols):
        return (np.arange(beams)[:, None] * columns + cols[None, :]).reshape(-1)

    for i in np.nonzero(np.linalg.norm(b_center - xy, axis=1) < max_range + 15.0)[0] if len(b_center) else []:
        lo, hi = buildings[i]
        rb = 0.5 * float(np.hypot(hi[0] - lo[0], hi[1] - lo[1]))
        ri = _rays(_cols(b_center[i], rb))
        if ri.size:
            t[ri] = np.minimum(t[ri], _hit_box_outside(o[ri], uw[ri], lo, hi))
    for i in np.nonzero(np.linalg.norm(t_center - xy, axis=1) < max_range + 1.0)[0] if len(t_center) else []:
        c, r, z0, z1 = trees[i]
        ri = _rays(_cols(c, r))
        if ri.size:
            t[ri] = np.minimum(t[ri], _hit_cylinder_z(o[ri], uw[ri], c, r, z0, z1))
    t = np.where(t <= max_range, t, np.inf)
    t = t + np.random.default_rng([w["seed"], 7, k]).normal(0.0, w["noise"], size=t.shape)
    with np.errstate(invalid="ignore"):
        p = dirs * t[:, None]
    p[~np.isfinite(t)] = np.nan
    return p.astype(np.float32), _pose(R, pos)


def lidar_terrain(
    scans: int = 100,
    beams: int = 64,
    columns: int = 2048,
    path_length: float = 400.0,
    n_buildings: int = 300,
    n_trees: int = 500,
    extent: float = 200.0,
    max_range: float = 60.0,
    noise: float = 0.02,
    seed: int = 3,
    voxel_size: float = 0.2,
    sensor_height: float = 2.0,
    workers: int = 0,
    generate: Optional[int] = None,
) -> ScanSet:
    """Spinning LiDAR over a heightfield with box buildings and cylinder trees. The scans are
    generated in `workers` spawned processes when workers > 1 (same result as one process).
    `generate` limits the output to the first scans of the `scans`-scan path (the same scans
    the full sequence starts with)."""
    rng = np.random.default_rng(seed)
    ter = _Terrain(rng)
    half = extent / 2.0
    # a smooth 2-D path of the requested length through random waypoints
    way = rng.uniform(-0.6 * half, 0.6 * half, size=(8, 2))
    dense = _catmull_rom(way, 4000)
    seg = np.linalg.norm(np.diff(dense, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    L = min(path_length, float(cum[-1]))
    s_samples = np.linspace(0.0, L, scans + 1)
    pxy = np.stack([np.interp(s_samples, cum, dense[:, 0]), np.interp(s_samples, cum, dense[:, 1])], 1)
    # buildings and trees, kept clear of the path
    buildings, trees = [], []
    tries = 0
    while len(buildings) < n_buildings and tries < 20000:
        tries += 1
        c = rng.uniform(-half, half, 2)
        sx, sy, sh = rng.uniform(4.0, 20.0, 3)
        if np.min(np.linalg.norm(dense - c, axis=1)) < 0.75 * max(sx, sy) + 4.0:
            continue
        base = float(ter.h(c[0], c[1])) - 1.0
        buildings.append((np.array([c[0] - sx / 2, c[1] - sy / 2, base]), np.array([c[0] + sx / 2, c[1] + sy / 2, base + 1.0 + sh])))
    tries = 0
    while len(trees) < n_trees and tries < 20000:
        tries += 1
        c = rng.uniform(-half, half, 2)
        r = float(rng.uniform(0.2, 0.6))
        h = float(rng.uniform(3.0, 10.0))
        if np.min(np.linalg.norm(dense - c, axis=1)) < r + 3.0:
            continue
        base = float(ter.h(c[0], c[1])) - 0.5
        trees.append((c, r, base, base + 0.5 + h))
    elev = np.deg2rad(np.linspace(-25.0, 15.0, beams))
    azim = np.arange(columns) * (2 * math.pi / columns)
    E, A = np.meshgrid(elev, azim, indexing="ij")
    world = dict(
        terrain=ter,
        pxy=pxy,
        dirs=np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3),
        beams=beams,
        columns=columns,
        max_range=max_range,
        noise=noise,
        seed=seed,
        sensor_height=sensor_height,
        buildings=buildings,
        trees=trees,
        b_center=np.array([0.5 * (b[0][:2] + b[1][:2]) for b in buildings]) if buildings else np.zeros((0, 2)),
        t_center=np.array([t[0] for t in trees]) if trees else np.zeros((0, 2)),
    )
    jobs = [(world, k) for k in range(scans if generate is None else min(scans, generate))]
    if workers and workers > 1 and len(jobs) > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            out = pool.map(_lidar_scan, jobs, chunksize=1)
    else:
        out = [_lidar_scan(j) for j in jobs]
    pts = [o[0] for o in out]
    poses = [o[1] for o in out]
    params = dict(
        voxel_size=voxel_size,
        voxels_per_block=8,
        truncation=3.0 * voxel_size,
        max_esdf_dist=5.0,
        weighting=0,
        eps=voxel_size,
        fixed_band=voxel_size,
        max_range=math.inf,
    )
    return ScanSet("lidar_terrain", pts, poses, params, meta=dict(buildings=len(buildings), trees=len(trees)))


# --------------------------------------------------------------------------------------
# query points


def random_queries(scans: ScanSet, n: int, radius: float = 2.0, seed: int = 5, scan_index: Optional[int] = None) -> np.ndarray:
    """Uniform points within `radius` of the sensor trajectory (float32, world frame)."""
    rng = np.random.default_rng(seed)
    centers = np.stack([p[:3, 3] for p in scans.poses]).astype(np.float64)
    if scan_index is not None:
        centers = centers[scan_index : scan_index + 1]
    k = rng.integers(0, len(centers), n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    return (centers[k] + d * r[:, None]).astype(np.float32)


def _mix_one(args):
    kind, kw = args
    return make_scene(kind, **kw)


def batch_mix_specs(n_maps: int = 64, frames: int = 4, seed: int = 4, kinds=("room", "lidar_terrain")):
    """Seeded specifications of independent map workloads of uneven sizes: rooms of 5-40 m with
    v in {0.05, 0.1} m and 160x120 .. 640x480 RGB-D frames, and LiDAR terrains of 40-80 m with
    v = 0.2 m and 16x1024 .. 64x2048 beams."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_maps):
        kind = kinds[int(rng.integers(0, len(kinds)))] if len(kinds) > 1 else kinds[0]
        if kind == "room":
            w, h = [(160, 120), (320, 240), (640, 480)][int(rng.integers(0, 3))]
            v = [0.05, 0.1][int(rng.integers(0, 2))]
            size = float(rng.uniform(5.0, 40.0))
            kw = dict(
                frames=frames,
                width=w,
                height=h,
                fx=525.0 * w / 640.0,
                fy=525.0 * w / 640.0,
                n_objects=int(max(5, min(60, size * size / 5.0))),
                seed=1000 + i,
                size=size,
                voxel_size=v,
                block=16 if v < 0.075 else 8,
            )
        else:
            beams, cols = [(16, 1024), (32, 1024), (64, 2048)][int(rng.integers(0, 3))]
            ext = float(rng.uniform(40.0, 80.0))
            kw = dict(
                scans=frames,
                beams=beams,
                columns=cols,
                path_length=ext,
                n_buildings=int(ext * ext / 130.0),
                n_trees=int(ext * ext / 80.0),
                extent=ext,
                seed=2000 + i,
            )
        specs.append((kind, kw))
    return specs


def batch_mix(n_maps: int = 64, frames: int = 4, seed: int = 4, kinds=("room", "lidar_terrain"), workers: int = 0):
    """The scan sets of batch_mix_specs, generated in parallel worker processes when workers > 1."""
    specs = batch_mix_specs(n_maps, frames, seed, kinds)
    if workers and workers > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.map(_mix_one, specs)
    return [_mix_one(x) for x in specs]


# --------------------------------------------------------------------------------------
# scene 4: the simulated ESDF benchmark of Sec. VI-B (three planes, a sphere and a cube in a
# 10 x 10 x 10 m space; noiseless RGB-D from random free-space poses)

_EB_SPHERE = (np.array([6.5, 4.0, 2.0]), 1.5)
_EB_CUBE = (np.array([2.0, 5.5, 0.0]), np.array([4.0, 7.5, 2.0]))  # lo, hi (resting on the ground)


def esdf_benchmark_sdf(x: np.ndarray) -> np.ndarray:
    """True signed distance of the ESDF benchmark scene (positive in free space): the union of
    the ground z = 0, the walls x = 0 and y = 10, the sphere and the cube."""
    x = np.asarray(x, np.float64)
    d = np.minimum(np.minimum(x[..., 2], x[..., 0]), 10.0 - x[..., 1])
    c, r = _EB_SPHERE
    d = np.minimum(d, np.linalg.norm(x - c, axis=-1) - r)
    lo, hi = _EB_CUBE
    ctr, half = (lo + hi) / 2.0, (hi - lo) / 2.0
    q = np.abs(x - ctr) - half
    box = np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(np.max(q, axis=-1), 0.0)
    return np.minimum(d, box)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
        ]
    )


def esdf_benchmark(
    poses: int = 50,
    width: int = 320,
    height: int = 240,
    fx: float = 262.5,
    voxel_size: float = 0.10,
    max_depth: float = 5.0,
    min_clearance: float = 1.0,
    seed: int = 4,
) -> ScanSet:
    """Noiseless 320x240 depth images from `poses` random 6-DoF poses at least
    `min_clearance` from every obstacle, depth beyond `max_depth` invalid. Map: B = 8,
    delta = 4 v, constant weight, d_max = 2 m, gamma = v (the one-voxel band)."""
    rng = np.random.default_rng(seed)
    dirs = _pinhole_dirs(width, height, fx, fx, (width - 1) / 2.0, (height - 1) / 2.0)
    dn = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    pts, Ts = [], []
    while len(pts) < poses:
        pos = rng.uniform(0.0, 10.0, 3)
        if esdf_benchmark_sdf(pos[None])[0] < min_clearance:
            continue
        R = _random_rotation(rng)
        uw = dn @ R.T
        o = np.broadcast_to(pos, uw.shape)
        with np.errstate(divide="ignore", invalid="ignore"):
            tx = np.where(uw[:, 0] < 0, -o[:, 0] / uw[:, 0], np.inf)  # wall x = 0
            ty = np.where(uw[:, 1] > 0, (10.0 - o[:, 1]) / uw[:, 1], np.inf)  # wall y = 10
        t = np.minimum(_hit_plane_z(o, uw), np.minimum(tx, ty))
        t = np.minimum(t, _hit_sphere(o, uw, *_EB_SPHERE))
        t = np.minimum(t, _hit_box_outside(o, uw, *_EB_CUBE))
        depth = t * dn[:, 2]
        p = dn * t[:, None]
        p[~(np.isfinite(t) & (depth <= max_depth))] = np.nan
        pts.append(p.astype(np.float32))
        Ts.append(_pose(R, pos))
    v = float(voxel_size)
    params = dict(
        voxel_size=v,
        voxels_per_block=8,
        truncation=4.0 * v,
        max_esdf_dist=2.0,
        weighting=0,
        eps=v,
        fixed_band=v,
        max_range=math.inf,
    )
    return ScanSet("esdf_benchmark", pts, Ts, params)


def synthetic_tsdf(
    lo=(-8, 30, -4),
    shape=(70, 60, 44),
    voxel_size: float = 0.1,
    voxels_per_block: int = 8,
    truncation: float = 0.4,
    noise: float = 0.01,
    p_unobserved: float = 0.05,
    p_missing_block: float = 0.04,
    p_zero: float = 0.02,
    seed: int = 7,
):
    """Seeded (vox, D, W) voxels of a truncated distance field over the voxel box
    [lo, lo + shape): the ESDF benchmark scene's distance at the voxel centres
    ((i + 1/2) voxel_size) plus N(0, noise) noise, kept where it lies within 1.5 truncation
    distances and clipped to [-truncation, truncation]; W ~ U(0.5, 4), zero for a fraction
    p_unobserved of the voxels; whole blocks dropped with probability p_missing_block; a
    fraction p_zero of the D values set to +0 or -0. Returns int32 (n, 3), float32 (n,),
    float32 (n,)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, np.int64)
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), -1).reshape(-1, 3) + lo
    d = esdf_benchmark_sdf((idx + 0.5) * float(np.float32(voxel_size))) + rng.normal(0.0, noise, idx.shape[0])
    keep = np.abs(d) < 1.5 * truncation
    idx, d = idx[keep], d[keep]
    blocks = np.floor_divide(idx, voxels_per_block)
    ub, inv = np.unique(blocks, axis=0, return_inverse=True)
    dropped = rng.random(ub.shape[0]) < p_missing_block
    keep = ~dropped[inv.reshape(-1)]
    idx, d = idx[keep], d[keep]
    D = np.clip(d, -truncation, truncation).astype(np.float32)
    W = rng.uniform(0.5, 4.0, D.shape[0]).astype(np.float32)
    W[rng.random(D.shape[0]) < p_unobserved] = 0.0
    z = rng.random(D.shape[0]) < p_zero
    D[z] = np.where(rng.random(D.shape[0]) < 0.5, np.float32(0.0), np.float32(-0.0))[z]
    return idx.astype(np.int32), D, W


def make_scene(name: str, **kw) -> ScanSet:
    return {"plane_sphere": plane_sphere, "room": room, "lidar_terrain": lidar_terrain, "esdf_benchmark": esdf_benchmark}[name](**kw)
