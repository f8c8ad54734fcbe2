"""FP64 brute-force ray-cast oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. The product renderer (``paper_2503_01471_gb300``)
never imports it, and the two share no code.

The C library ``oracle.c`` implements the method of the Aerial Gym Simulator
paper, Sec. III-D.1 (per-object rigid transform of the base meshes, one ray
per pixel or beam, nearest hit against every triangle, depth vs range, segment
IDs) in double precision. This module compiles it with gcc on first use and
wraps it with ctypes. The only non-C step here is gathering a sub-mesh's
transformed vertices by its triangle indices (numpy fancy indexing).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

MAX_CAND = 4
MAX_TRI = 8
F_COUNTED = 1
F_SILHOUETTE = 2
F_NEAR_TIE = 4
F_RANGE_EDGE = 8
F_GRAZING = 16
F_OVERFLOW = 32
F_MISS_OK = 64
F_WIDE = 128
F_TRI_OVERFLOW = 256
F_COARSE = 512
# the reasons a ray may be counted (judged against its listed outcomes rather than the tolerance)
F_REASONS = F_SILHOUETTE | F_NEAR_TIE | F_RANGE_EDGE | F_GRAZING | F_COARSE

PINHOLE = 0
LIDAR = 1
RAY_TABLE = 2
NEAR_CLAMP = 0
NEAR_INVALID = 1

# Error bands of the float32 renderer being judged: world vertex coordinates
# within VERT_REL * max(|x|, 1) of exact (one unit in the last place, the bound
# the transform test holds the renderer to), ray directions within DIR_REL
# (relative; a float32 rotation of the pixel direction is good to ~4e-7), and
# intersection arithmetic that moves the ray sideways by at most ARITH_REL
# times the distance to the vertices.
VERT_REL = 2.0 ** -23
DIR_REL = 6e-7
ARITH_REL = 4.0 * 2.0 ** -24


def build(force: bool = False, extra_flags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile oracle.c into a shared library (gcc, OpenMP, no FP contraction)."""
    out = out or _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", *extra_flags, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Sensor(ctypes.Structure):
    _fields_ = [
        ("type", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("near_mode", ctypes.c_int32), ("hfov", ctypes.c_double), ("vfov_min", ctypes.c_double),
        ("vfov_max", ctypes.c_double), ("min_range", ctypes.c_double),
        ("max_range", ctypes.c_double), ("vert_rel", ctypes.c_double),
        ("dir_rel", ctypes.c_double), ("arith_rel", ctypes.c_double), ("dirs", ctypes.c_void_p),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("v", ctypes.c_double), ("seg", ctypes.c_int32), ("tri", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("n_cand", ctypes.c_int32),
        ("cand_seg", ctypes.c_int32 * MAX_CAND), ("cand_lo", ctypes.c_double * MAX_CAND),
        ("cand_hi", ctypes.c_double * MAX_CAND), ("n_tri", ctypes.c_int32),
        ("cand_tri", ctypes.c_int32 * MAX_TRI), ("t_hit", ctypes.c_double), ("cos_hit", ctypes.c_double),
        ("hit_dev", ctypes.c_double),
    ]


RESULT_DTYPE = np.dtype({
    "names": ["v", "seg", "tri", "flags", "n_cand", "cand_seg", "cand_lo", "cand_hi", "n_tri", "cand_tri",
              "t_hit", "cos_hit", "hit_dev"],
    "formats": ["<f8", "<i4", "<i4", "<i4", "<i4", ("<i4", MAX_CAND), ("<f8", MAX_CAND),
                ("<f8", MAX_CAND), "<i4", ("<i4", MAX_TRI), "<f8", "<f8", "<f8"],
    "offsets": [_Result.v.offset, _Result.seg.offset, _Result.tri.offset, _Result.flags.offset,
                _Result.n_cand.offset, _Result.cand_seg.offset, _Result.cand_lo.offset,
                _Result.cand_hi.offset, _Result.n_tri.offset, _Result.cand_tri.offset, _Result.t_hit.offset,
                _Result.cos_hit.offset, _Result.hit_dev.offset],
    "itemsize": ctypes.sizeof(_Result),
})

_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building if needed) the oracle library; ``path`` selects a variant build."""
    with _lock:
        key = path or _LIB
        if key in _libs:
            return _libs[key]
        if path is None:
            build()
        lib = ctypes.CDLL(key)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_rotation.argtypes = [dp, dp]
        lib.orc_rotation.restype = None
        lib.orc_transform.argtypes = [dp, ctypes.c_int64, dp, dp]
        lib.orc_transform.restype = None
        lib.orc_ray.argtypes = [ctypes.POINTER(_Sensor), dp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp]
        lib.orc_ray.restype = ctypes.c_int
        lib.orc_render.argtypes = [dp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                   ctypes.POINTER(_Sensor), dp, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.c_int64, ctypes.c_void_p]
        lib.orc_render.restype = ctypes.c_int
        lib.orc_hit_channels.argtypes = [dp, ctypes.c_int64, ctypes.POINTER(_Sensor), dp,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), dp,
                                         ctypes.c_int64, dp, dp, dp]
        lib.orc_hit_channels.restype = ctypes.c_int
        lib.orc_shadow.argtypes = [dp, ctypes.c_int64, ctypes.POINTER(_Sensor), dp, dp, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_int32)]
        lib.orc_shadow.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = ctypes.c_int
        _libs[key] = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Sensor:
    """Sensor model of the oracle (angles in radians, ranges in metres)."""
    type: int
    width: int
    height: int
    hfov: float
    min_range: float
    max_range: float
    vfov_min: float = 0.0
    vfov_max: float = 0.0
    near_mode: int = NEAR_CLAMP
    vert_rel: float = VERT_REL
    dir_rel: float = DIR_REL
    arith_rel: float = ARITH_REL
    dirs: np.ndarray | None = None  # RAY_TABLE: [height, width, 3] sensor-frame directions

    def _c(self) -> _Sensor:
        ptr = None
        if self.dirs is not None:
            self._dirs64 = np.ascontiguousarray(self.dirs, np.float64).reshape(self.height, self.width, 3)
            ptr = self._dirs64.ctypes.data
        return _Sensor(self.type, self.width, self.height, self.near_mode, self.hfov,
                       self.vfov_min, self.vfov_max, self.min_range, self.max_range,
                       self.vert_rel, self.dir_rel, self.arith_rel, ptr)


def rotation(q, lib=None) -> np.ndarray:
    lib = lib or load()
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros(9, np.float64)
    lib.orc_rotation(_dp(q), _dp(R))
    return R.reshape(3, 3)


def transform(v, pose, lib=None) -> np.ndarray:
    """World coordinates v' = R(q) v + p of object-frame points v [n,3]."""
    lib = lib or load()
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(7)
    out = np.empty_like(v)
    lib.orc_transform(_dp(v), v.shape[0], _dp(pose), _dp(out))
    return out


def ray(sensor: Sensor, pose, row: int, col: int, lib=None):
    """(origin, unit direction, value scale) of one pixel/beam."""
    lib = lib or load()
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(7)
    o = np.zeros(3)
    d = np.zeros(3)
    sc = np.zeros(1)
    s = sensor._c()
    rc = lib.orc_ray(ctypes.byref(s), _dp(pose), row, col, _dp(o), _dp(d), _dp(sc))
    if rc != 0:
        raise ValueError("orc_ray: bad sensor or pixel")
    return o, d, float(sc[0])


def world_triangles(vertices_list, indices_list, poses, segs):
    """FP64 world-space triangles [F,9] and segment IDs [F] of one environment.

    ``vertices_list[j]`` [n_j,3] and ``indices_list[j]`` [m_j,3] are sub-mesh j
    in its object frame, ``poses[j]`` its (p, q) pose and ``segs[j]`` its ID.
    """
    lib = load()
    tris, seg = [], []
    for v, idx, pose, s in zip(vertices_list, indices_list, poses, segs):
        w = transform(np.asarray(v, np.float64), np.asarray(pose, np.float64), lib)
        idx = np.asarray(idx, np.int64)
        tris.append(w[idx].reshape(-1, 9))
        seg.append(np.full(idx.shape[0], int(s), np.int32))
    if not tris:
        return np.zeros((0, 9)), np.zeros(0, np.int32)
    return np.ascontiguousarray(np.concatenate(tris)), np.ascontiguousarray(np.concatenate(seg))


def render(tris, seg, sensor: Sensor, pose, rays=None, lib=None) -> np.ndarray:
    """Oracle result for each listed ray (flat index row*width+col; all if None)."""
    lib = lib or load()
    tris = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
    seg = np.ascontiguousarray(seg, dtype=np.int32).reshape(-1)
    if seg.shape[0] != tris.shape[0]:
        raise ValueError("seg and tris disagree")
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(7)
    if rays is None:
        rays = np.arange(sensor.width * sensor.height, dtype=np.int64)
    rays = np.ascontiguousarray(rays, dtype=np.int64).reshape(-1)
    out = np.zeros(rays.shape[0], RESULT_DTYPE)
    s = sensor._c()
    rc = lib.orc_render(_dp(tris), seg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        tris.shape[0], ctypes.byref(s), _dp(pose),
                        rays.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rays.shape[0],
                        out.ctypes.data)
    if rc != 0:
        raise ValueError("orc_render: bad input")
    return out


def hit_channels(tris, sensor: Sensor, pose, rays, face, v, lib=None):
    """Barycentrics [n,2], world normals [n,3] and sensor-frame points [n,3] of rays (flat indices) that
    hit triangle ``face`` (env-local; < 0 for a miss) and report value ``v``."""
    lib = lib or load()
    tris = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(7)
    rays = np.ascontiguousarray(rays, dtype=np.int64).reshape(-1)
    face = np.ascontiguousarray(face, dtype=np.int32).reshape(-1)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    n = rays.shape[0]
    if face.shape[0] != n or v.shape[0] != n:
        raise ValueError("rays, face and v disagree")
    bary, normal, point = np.zeros((n, 2)), np.zeros((n, 3)), np.zeros((n, 3))
    s = sensor._c()
    rc = lib.orc_hit_channels(_dp(tris), tris.shape[0], ctypes.byref(s), _dp(pose),
                              rays.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              face.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(v), n, _dp(bary),
                              _dp(normal), _dp(point))
    if rc != 0:
        raise ValueError("orc_hit_channels: bad input or degenerate face")
    return bary, normal, point


def shadow(tris, sensor: Sensor, pose, baseline, eps, rays, res, lib=None) -> np.ndarray:
    """Stereo shadow verdicts (0 free, 1 shadowed, 2 either) of rays whose oracle results are ``res``."""
    lib = lib or load()
    tris = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(7)
    baseline = np.ascontiguousarray(baseline, dtype=np.float64).reshape(3)
    rays = np.ascontiguousarray(rays, dtype=np.int64).reshape(-1)
    res = np.ascontiguousarray(res)
    if res.dtype != RESULT_DTYPE or res.shape[0] != rays.shape[0]:
        raise ValueError("res must be the oracle results of the listed rays")
    out = np.zeros(rays.shape[0], np.int32)
    s = sensor._c()
    rc = lib.orc_shadow(_dp(tris), tris.shape[0], ctypes.byref(s), _dp(pose), _dp(baseline), float(eps),
                        rays.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), res.ctypes.data, rays.shape[0],
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError("orc_shadow: bad input")
    return out


def num_threads(lib=None) -> int:
    return int((lib or load()).orc_num_threads())


def tol(v):
    """Depth/range tolerance |dv| <= 1e-5 v + 1e-6 m."""
    return 1e-5 * np.abs(v) + 1e-6


def check(res: np.ndarray, v_gpu, seg_gpu, max_range: float, with_strict: bool = False):
    """Element-wise acceptance of renderer outputs against oracle results.

    Returns (ok, counted) -- or (ok, counted, strict) with ``with_strict``.

    An uncounted ray must give the exact answer: a miss bit-exact (float32
    max_range, segment -1); a hit with the exact segment and a value within
    tol(v) = 1e-5 v + 1e-6 of the exact FP64 value. A counted ray (the oracle
    states its reason: silhouette, near tie, range edge, grazing incidence or
    coarse coordinates) may give any outcome the oracle lists: a miss where
    that is allowed, or a hit whose segment is a candidate group's and whose
    value lies in that group's range widened by the tolerance. A ray whose
    outcome list overflowed always fails. strict: uncounted and ok.
    """
    v = np.asarray(v_gpu, np.float64).reshape(-1)
    s = np.asarray(seg_gpu, np.int64).reshape(-1)
    flags = res["flags"]
    miss_val = float(np.float32(max_range))
    is_miss = (s == -1) & (v == miss_val)
    counted = (flags & F_COUNTED) != 0
    exact = np.where(res["seg"] == -1, is_miss,
                     (s == res["seg"]) & (np.abs(v - res["v"]) <= tol(res["v"])))
    hit_ok = np.zeros(v.shape[0], bool)
    for k in range(MAX_CAND):
        valid = res["n_cand"] > k
        lo = res["cand_lo"][:, k]
        hi = res["cand_hi"][:, k]
        hit_ok |= valid & (res["cand_seg"][:, k] == s) & (v >= lo - tol(lo)) & (v <= hi + tol(hi))
    listed = (is_miss & ((flags & F_MISS_OK) != 0)) | ((s != -1) & hit_ok)
    ok = np.where(counted, listed, exact) & ((flags & F_OVERFLOW) == 0)
    if not with_strict:
        return ok, counted
    return ok, counted, ok & ~counted
