"""Seeded synthetic scenes, sensor specs and sensor-pose sequences.

This module only *generates inputs*: object-frame base meshes, per-object
poses (position + unit quaternion x,y,z,w) and sensor poses. It holds none of
the renderer's arithmetic (no object-to-world transform, no rays, no
intersection); both the CUDA renderer and the FP64 oracle consume what it
makes.

The paper's own benchmark scenes (twenty cubes in front of each robot, Table I;
a static room with fifteen floating obstacles, Table II) are built from the
simulator's assets, which are not available here. The
workloads below stand in for them with the same structure: a 10 x 10 x 4 m
room per environment with 20-40 obstacles of several mesh types, or a forest of
procedural trees on a 40 x 40 m ground plane for the 3-D LiDAR. All randomness
comes from numpy PCG64 seeded with ``20250303 + 1000 * workload + env``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20250303

ROOM_HALF_XY = 5.0
ROOM_HEIGHT = 4.0
WALL_MARGIN = 0.3


# ---------------------------------------------------------------- containers
@dataclass
class SceneBatch:
    """Environments as a CSR of sub-meshes (one sub-mesh per object).

    vertices   float32 [sum V, 3]   object-frame vertices, sub-mesh after sub-mesh
    indices    int32   [sum F, 3]   triangle corners, local to their sub-mesh
    sub_vert   int64   [J + 1]      vertex offsets of each sub-mesh
    sub_tri    int64   [J + 1]      triangle offsets of each sub-mesh
    sub_seg    int32   [J]          segment ID reported for each sub-mesh
    env_sub    int64   [E + 1]      sub-mesh offsets of each environment
    poses      float32 [J, 7]       object pose (px, py, pz, qx, qy, qz, qw)
    """
    vertices: np.ndarray
    indices: np.ndarray
    sub_vert: np.ndarray
    sub_tri: np.ndarray
    sub_seg: np.ndarray
    env_sub: np.ndarray
    poses: np.ndarray

    @property
    def n_envs(self) -> int:
        return int(self.env_sub.shape[0] - 1)

    def env_tri_counts(self) -> np.ndarray:
        return self.sub_tri[self.env_sub[1:]] - self.sub_tri[self.env_sub[:-1]]

    def env_submeshes(self, e: int):
        """Lists (vertices, indices, poses, segs) of environment e."""
        j0, j1 = int(self.env_sub[e]), int(self.env_sub[e + 1])
        vs, ix = [], []
        for j in range(j0, j1):
            vs.append(self.vertices[self.sub_vert[j]:self.sub_vert[j + 1]])
            ix.append(self.indices[self.sub_tri[j]:self.sub_tri[j + 1]])
        return vs, ix, self.poses[j0:j1], self.sub_seg[j0:j1]

    def subset(self, envs) -> "SceneBatch":
        lists = []
        for e in envs:
            vs, ix, ps, sg = self.env_submeshes(int(e))
            lists.append(list(zip(vs, ix, ps, (int(x) for x in sg))))
        return scene_from_lists(lists)

    def translated(self, offset) -> "SceneBatch":
        """Same scene with every object moved by ``offset`` (poses only)."""
        p = self.poses.copy()
        p[:, :3] += np.asarray(offset, np.float32)
        return SceneBatch(self.vertices, self.indices, self.sub_vert, self.sub_tri,
                          self.sub_seg, self.env_sub, p)


class _Builder:
    def __init__(self):
        self.v, self.i, self.p, self.s = [], [], [], []
        self.sub_v, self.sub_t, self.env = [0], [0], [0]

    def add(self, verts, idx, pose, seg):
        verts = np.asarray(verts, np.float32).reshape(-1, 3)
        idx = np.asarray(idx, np.int32).reshape(-1, 3)
        self.v.append(verts)
        self.i.append(idx)
        self.p.append(np.asarray(pose, np.float32).reshape(7))
        self.s.append(int(seg))
        self.sub_v.append(self.sub_v[-1] + verts.shape[0])
        self.sub_t.append(self.sub_t[-1] + idx.shape[0])


def scene_from_lists(envs) -> SceneBatch:
    """Build a SceneBatch from ``[[(verts, idx, pose, seg), ...], ...]`` (one list per env)."""
    b = _Builder()
    for env in envs:
        for verts, idx, pose, seg in env:
            b.add(verts, idx, pose, seg)
        b.env.append(len(b.p))
    v = np.concatenate(b.v) if b.v else np.zeros((0, 3), np.float32)
    i = np.concatenate(b.i) if b.i else np.zeros((0, 3), np.int32)
    p = np.stack(b.p) if b.p else np.zeros((0, 7), np.float32)
    return SceneBatch(np.ascontiguousarray(v, np.float32), np.ascontiguousarray(i, np.int32),
                      np.asarray(b.sub_v, np.int64), np.asarray(b.sub_t, np.int64),
                      np.asarray(b.s, np.int32), np.asarray(b.env, np.int64),
                      np.ascontiguousarray(p, np.float32))


@dataclass
class SensorSpec:
    """Sensor model (mirrors ags_sensor_spec). Angles in radians, ranges in metres."""
    type: int            # 0 pinhole camera, 1 LiDAR
    width: int           # camera columns / LiDAR azimuth bins
    height: int          # camera rows / LiDAR channels
    hfov: float
    min_range: float
    max_range: float
    vfov_min: float = 0.0
    vfov_max: float = 0.0
    near_mode: int = 0   # 0 clamp to min_range, 1 report as invalid (max_range, -1)
    flags: int = 0


def pinhole(width, height, hfov_deg=87.0, min_range=0.2, max_range=10.0, near_mode=0):
    return SensorSpec(0, width, height, math.radians(hfov_deg), min_range, max_range,
                      near_mode=near_mode)


def lidar(azimuth_bins=512, channels=64, vfov_deg=(-22.5, 22.5), min_range=0.3,
          max_range=50.0, hfov_deg=360.0, near_mode=0):
    return SensorSpec(1, azimuth_bins, channels, math.radians(hfov_deg), min_range, max_range,
                      math.radians(vfov_deg[0]), math.radians(vfov_deg[1]), near_mode)


def dome_lidar(azimuth_bins=512, channels=64, min_range=0.3, max_range=50.0):
    """Hemispherical dome LiDAR: channels from the horizon (0 deg) to the zenith (90 deg) all around."""
    return lidar(azimuth_bins, channels, (0.0, 90.0), min_range, max_range)


def ray_table_spec(width, height, min_range=0.2, max_range=10.0, near_mode=0):
    """Sensor spec of a user projection model; its directions come from a separate table."""
    return SensorSpec(2, width, height, 0.0, min_range, max_range, near_mode=near_mode)


def fisheye_table(width, height, fov_deg=180.0):
    """Equidistant fisheye (image radius proportional to the angle off the +x optical axis), unit
    sensor-frame rows [height, width, 3]; pixels beyond the image circle look along its rim."""
    half = math.radians(fov_deg) / 2
    cx, cy = width / 2.0, height / 2.0
    rad = min(cx, cy)
    cols, rows = np.meshgrid(np.arange(width) + 0.5, np.arange(height) + 0.5)
    u, v = (cx - cols) / rad, (cy - rows) / rad  # +u left (+y), +v up (+z)
    r = np.hypot(u, v)
    theta = np.minimum(r, 1.0) * half
    phi = np.arctan2(v, u)
    out = np.stack([np.cos(theta), np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi)], -1)
    return np.ascontiguousarray(out, np.float32)


# ---------------------------------------------------------------- primitives
IDENTITY_POSE = np.array([0, 0, 0, 0, 0, 0, 1], np.float32)


def box(ex, ey, ez):
    hx, hy, hz = ex / 2, ey / 2, ez / 2
    v = np.array([[x, y, z] for x in (-hx, hx) for y in (-hy, hy) for z in (-hz, hz)], np.float32)
    # corner index = 4*ix + 2*iy + iz
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    f = []
    for a, b, c, d in quads:
        f += [(a, b, c), (a, c, d)]
    return v, np.array(f, np.int32)


def room(half_xy=ROOM_HALF_XY, height=ROOM_HEIGHT):
    """Six wall quads (12 triangles) of an axis-aligned room, world frame."""
    v, f = box(2 * half_xy, 2 * half_xy, height)
    v = v + np.array([0, 0, height / 2], np.float32)
    return v.astype(np.float32), f


_ICO_CACHE: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def icosphere_unit(level: int):
    if level in _ICO_CACHE:
        return _ICO_CACHE[level]
    g = (1 + 5 ** 0.5) / 2
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0), (0, -1, g), (0, 1, g), (0, -1, -g),
         (0, 1, -g), (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    v = [np.array(p, float) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                mid[key] = len(v) - 1
            return mid[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    out = (np.array(v, np.float64), np.array(f, np.int32))
    _ICO_CACHE[level] = out
    return out


def icosphere(radius, level=2):
    v, f = icosphere_unit(level)
    return (v * radius).astype(np.float32), f.copy()


def cylinder(radius, height, segments=32):
    """Closed cylinder along z centred at the origin: 2*segments side + 2*segments cap triangles."""
    k = np.arange(segments)
    th = 2 * np.pi * k / segments
    ring = np.stack([np.cos(th), np.sin(th)], 1) * radius
    bot = np.concatenate([ring, np.full((segments, 1), -height / 2)], 1)
    top = np.concatenate([ring, np.full((segments, 1), height / 2)], 1)
    v = np.concatenate([bot, top, [[0, 0, -height / 2], [0, 0, height / 2]]]).astype(np.float32)
    n = segments
    k1 = (k + 1) % n
    side = np.concatenate([np.stack([k, k1, n + k1], 1), np.stack([k, n + k1, n + k], 1)])
    cb = np.stack([np.full(n, 2 * n), k1, k], 1)
    ct = np.stack([np.full(n, 2 * n + 1), n + k, n + k1], 1)
    return v, np.concatenate([side, cb, ct]).astype(np.int32)


def cone(radius, height, segments=32):
    """Cone along +z, base disc at z=0, apex at z=height: 2*segments triangles."""
    k = np.arange(segments)
    th = 2 * np.pi * k / segments
    ring = np.stack([np.cos(th) * radius, np.sin(th) * radius, np.zeros(segments)], 1)
    v = np.concatenate([ring, [[0, 0, height], [0, 0, 0]]]).astype(np.float32)
    k1 = (k + 1) % segments
    side = np.stack([k, k1, np.full(segments, segments)], 1)
    base = np.stack([np.full(segments, segments + 1), k1, k], 1)
    return v, np.concatenate([side, base]).astype(np.int32)


def panel(size, rng, n=32, displacement=0.1):
    """n x n quad grid in the y-z plane (2 n^2 triangles), random x displacement per vertex."""
    s = np.linspace(-size / 2, size / 2, n + 1)
    yy, zz = np.meshgrid(s, s, indexing="ij")
    xx = rng.uniform(-displacement, displacement, size=yy.shape)
    v = np.stack([xx, yy, zz], -1).reshape(-1, 3).astype(np.float32)
    i = np.arange(n)[:, None] * (n + 1) + np.arange(n)[None, :]
    a, b, c, d = i, i + 1, i + n + 1, i + n + 2
    f = np.concatenate([np.stack([a, c, d], -1).reshape(-1, 3), np.stack([a, d, b], -1).reshape(-1, 3)])
    return v, f.astype(np.int32)


# ---------------------------------------------------------------- poses
def quat_from_euler_zyx(yaw, pitch, roll):
    """Unit quaternion (x, y, z, w) of the intrinsic Z-Y-X (yaw, pitch, roll) rotation."""
    cy, sy = np.cos(yaw / 2), np.sin(yaw / 2)
    cp, sp = np.cos(pitch / 2), np.sin(pitch / 2)
    cr, sr = np.cos(roll / 2), np.sin(roll / 2)
    w = cr * cp * cy + sr * sp * sy
    x = sr * cp * cy - cr * sp * sy
    y = cr * sp * cy + sr * cp * sy
    z = cr * cp * sy - sr * sp * cy
    return np.stack([x, y, z, w], -1)


def random_unit_quat(rng, n=None):
    q = rng.normal(size=(4,) if n is None else (n, 4))
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


def rng_for(workload: int, env: int):
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * workload + env))


def room_camera_pose(rng, margin=WALL_MARGIN):
    p = np.array([rng.uniform(-ROOM_HALF_XY + margin, ROOM_HALF_XY - margin),
                  rng.uniform(-ROOM_HALF_XY + margin, ROOM_HALF_XY - margin),
                  rng.uniform(margin, ROOM_HEIGHT - margin)])
    yaw = rng.uniform(-np.pi, np.pi)
    pitch = rng.uniform(-0.2, 0.2)
    roll = rng.uniform(-0.2, 0.2)
    return np.concatenate([p, quat_from_euler_zyx(yaw, pitch, roll)]).astype(np.float32), (yaw, pitch, roll)


def random_walk(init_pos, init_euler, steps, rng, lo, hi, sigma_p=0.05, sigma_yaw=0.05):
    """Sensor poses [steps, 7]: position and yaw random walk, clamped to [lo, hi]."""
    p = np.array(init_pos, np.float64)
    yaw, pitch, roll = init_euler
    out = np.zeros((steps, 7), np.float32)
    for s in range(steps):
        if s > 0:
            p = np.clip(p + rng.normal(0, sigma_p, 3), lo, hi)
            yaw = yaw + rng.normal(0, sigma_yaw)
        out[s, :3] = p
        out[s, 3:] = quat_from_euler_zyx(yaw, pitch, roll)
    return out


# ---------------------------------------------------------------- workloads
def tiny_room(seed_env: int = 0):
    """1 env: room (seg 0) + 8 axis-aligned boxes (seg 1..8); 16 camera poses; 64x48 at 87 deg."""
    rng = rng_for(1, seed_env)
    rv, rf = room()
    objs = [(rv, rf, IDENTITY_POSE, 0)]
    for k in range(8):
        e = rng.uniform(0.5, 2.0, 3)
        c = np.array([rng.uniform(-ROOM_HALF_XY, ROOM_HALF_XY), rng.uniform(-ROOM_HALF_XY, ROOM_HALF_XY),
                      rng.uniform(0, ROOM_HEIGHT)])
        v, f = box(*e)
        objs.append((v, f, np.concatenate([c, [0, 0, 0, 1]]).astype(np.float32), k + 1))
    scene = scene_from_lists([objs])
    poses = np.stack([room_camera_pose(rng)[0] for _ in range(16)])
    return scene, pinhole(64, 48), poses


OBSTACLE_TYPES = ("box", "icosphere", "cylinder", "panel")


def _obstacle(kind, rng):
    if kind == "box":
        return box(*rng.uniform(0.5, 2.0, 3))
    if kind == "icosphere":
        return icosphere(rng.uniform(0.2, 1.0), 2)
    if kind == "cylinder":
        return cylinder(rng.uniform(0.2, 0.6), rng.uniform(0.5, 3.0), 32)
    return panel(rng.uniform(1.0, 3.0), rng, 32, 0.1)


def obstacle_room_env(rng, n_lo=20, n_hi=40):
    rv, rf = room()
    objs = [(rv, rf, IDENTITY_POSE, 0)]
    n = int(rng.integers(n_lo, n_hi + 1))
    for k in range(n):
        kind = OBSTACLE_TYPES[int(rng.integers(0, 4))]
        v, f = _obstacle(kind, rng)
        p = np.array([rng.uniform(-ROOM_HALF_XY, ROOM_HALF_XY), rng.uniform(-ROOM_HALF_XY, ROOM_HALF_XY),
                      rng.uniform(0, ROOM_HEIGHT)])
        objs.append((v, f, np.concatenate([p, random_unit_quat(rng)]).astype(np.float32), k + 1))
    return objs


def obstacle_rooms(n_envs=1024, steps=100, width=480, height=270, workload=2, envs=None):
    """Rooms with 20-40 random obstacles each, one camera per env walking for ``steps`` steps.

    Returns (scene, spec, sensor_poses [steps, E, 7]). ``envs`` selects a subset
    of environment indices (same content as in the full batch).
    """
    env_ids = range(n_envs) if envs is None else envs
    lists, walks = [], []
    lo = np.array([-ROOM_HALF_XY + WALL_MARGIN, -ROOM_HALF_XY + WALL_MARGIN, WALL_MARGIN])
    hi = np.array([ROOM_HALF_XY - WALL_MARGIN, ROOM_HALF_XY - WALL_MARGIN, ROOM_HEIGHT - WALL_MARGIN])
    for e in env_ids:
        rng = rng_for(workload, int(e))
        lists.append(obstacle_room_env(rng))
        p0, eul = room_camera_pose(rng)
        walks.append(random_walk(p0[:3], eul, steps, rng, lo, hi))
    scene = scene_from_lists(lists)
    poses = np.ascontiguousarray(np.stack(walks, 1), np.float32)
    return scene, pinhole(width, height), poses


def _tree(rng, target_tris):
    """Trunk cylinder plus a cluster of cones; about ``target_tris`` triangles, object frame."""
    h = rng.uniform(3.0, 8.0)
    tv, tf = cylinder(rng.uniform(0.1, 0.3), h, 32)
    tv = tv + np.array([0, 0, h / 2], np.float32)
    n_cones = max(1, int(round((target_tris - tf.shape[0]) / 64)))
    cv, cf = cone(1.0, 1.0, 32)
    r = rng.uniform(0.3, 1.5, n_cones)
    hh = rng.uniform(0.5, 2.0, n_cones)
    z0 = rng.uniform(0.3 * h, h, n_cones)
    az = rng.uniform(0, 2 * np.pi, n_cones)
    off = rng.uniform(0, 1.5, n_cones)
    tilt = rng.uniform(0, 0.6, n_cones)
    # cone k: scale (r, r, hh), tilt about a horizontal axis at azimuth az, then move out
    ca, sa = np.cos(az), np.sin(az)
    ct, st = np.cos(tilt), np.sin(tilt)
    local = cv[None].astype(np.float64) * np.stack([r, r, hh], 1)[:, None, :]
    # tilt about the axis (-sin az, cos az, 0): rotate the cone's +z towards (cos az, sin az)
    x, y, z = local[..., 0], local[..., 1], local[..., 2]
    # decompose in the (radial, tangential, z) frame of azimuth az
    rad = x * ca[:, None] + y * sa[:, None]
    tan = -x * sa[:, None] + y * ca[:, None]
    rad2 = rad * ct[:, None] + z * st[:, None]
    z2 = -rad * st[:, None] + z * ct[:, None]
    x2 = rad2 * ca[:, None] - tan * sa[:, None]
    y2 = rad2 * sa[:, None] + tan * ca[:, None]
    pos = np.stack([off * ca, off * sa, z0], 1)
    cones = np.stack([x2, y2, z2], -1) + pos[:, None, :]
    nv = cv.shape[0]
    faces = cf[None] + (tv.shape[0] + nv * np.arange(n_cones))[:, None, None]
    v = np.concatenate([tv, cones.reshape(-1, 3)]).astype(np.float32)
    f = np.concatenate([tf, faces.reshape(-1, 3)]).astype(np.int32)
    return v, f


def forest_env(rng, n_lo=50, n_hi=200, tri_lo=2000, tri_hi=10000, half=20.0):
    gv = np.array([[-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]], np.float32)
    gf = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    objs = [(gv, gf, IDENTITY_POSE, 0)]
    n = int(rng.integers(n_lo, n_hi + 1))
    for k in range(n):
        v, f = _tree(rng, int(rng.integers(tri_lo, tri_hi + 1)))
        p = np.array([rng.uniform(-half, half), rng.uniform(-half, half), 0.0])
        q = quat_from_euler_zyx(rng.uniform(-np.pi, np.pi), 0.0, 0.0)
        objs.append((v, f, np.concatenate([p, q]).astype(np.float32), k + 1))
    return objs


def lidar_forests(n_envs=256, steps=10, workload=3, envs=None, trees=(50, 200), tris=(2000, 10000)):
    """Forests of uneven size with one 64 x 512 LiDAR per env at 1.5 m height."""
    env_ids = range(n_envs) if envs is None else envs
    lists, walks = [], []
    half = 20.0
    lo = np.array([-half + 2, -half + 2, 1.5])
    hi = np.array([half - 2, half - 2, 1.5])
    for e in env_ids:
        rng = rng_for(workload, int(e))
        lists.append(forest_env(rng, trees[0], trees[1], tris[0], tris[1], half))
        p0 = np.array([rng.uniform(lo[0], hi[0]), rng.uniform(lo[1], hi[1]), 1.5])
        walks.append(random_walk(p0, (rng.uniform(-np.pi, np.pi), 0.0, 0.0), steps, rng, lo, hi))
    scene = scene_from_lists(lists)
    poses = np.ascontiguousarray(np.stack(walks, 1), np.float32)
    return scene, lidar(), poses


def _primitive_pool(rng, n_each=16):
    """Object-frame meshes reused across serving environments (each env still gets its own copy)."""
    pool = []
    for _ in range(n_each):
        pool.append(box(*rng.uniform(0.5, 2.0, 3)))
        pool.append(icosphere(rng.uniform(0.2, 1.0), 2))
        pool.append(cylinder(rng.uniform(0.2, 0.6), rng.uniform(0.5, 3.0), 32))
        pool.append(panel(rng.uniform(1.0, 3.0), rng, 32, 0.1))
    return pool


def serving_rooms(n_envs=8192, tri_lo=1000, tri_hi=200000, workload=5, steps=1):
    """Rooms whose triangle counts are log-uniform in [tri_lo, tri_hi]: obstacles drawn from a pool of
    primitive meshes until the count is reached, uniform poses. Returns (scene, sensor poses [steps, E, 7])."""
    pool_rng = rng_for(workload, 10**6)
    pool = _primitive_pool(pool_rng)
    rv, rf = room()
    lists, walks = [], []
    lo = np.array([-ROOM_HALF_XY + WALL_MARGIN, -ROOM_HALF_XY + WALL_MARGIN, WALL_MARGIN])
    hi = np.array([ROOM_HALF_XY - WALL_MARGIN, ROOM_HALF_XY - WALL_MARGIN, ROOM_HEIGHT - WALL_MARGIN])
    for e in range(n_envs):
        rng = rng_for(workload, e)
        target = int(np.exp(rng.uniform(np.log(tri_lo), np.log(tri_hi))))
        objs = [(rv, rf, IDENTITY_POSE, 0)]
        total, k = rf.shape[0], 0
        while total < target:
            v, f = pool[int(rng.integers(0, len(pool)))]
            p = np.array([rng.uniform(-ROOM_HALF_XY, ROOM_HALF_XY), rng.uniform(-ROOM_HALF_XY, ROOM_HALF_XY),
                          rng.uniform(0, ROOM_HEIGHT)])
            objs.append((v, f, np.concatenate([p, random_unit_quat(rng)]).astype(np.float32), k + 1))
            total += f.shape[0]
            k += 1
        lists.append(objs)
        p0, eul = room_camera_pose(rng)
        walks.append(random_walk(p0[:3], eul, steps, rng, lo, hi))
    return scene_from_lists(lists), np.ascontiguousarray(np.stack(walks, 1), np.float32)
