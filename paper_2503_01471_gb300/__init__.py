"""GB300-native batched ray-cast sensor renderer (Aerial Gym Simulator, Sec. III-D.1).

Thin ctypes binding of the C ABI in ``include/ags.h``: the functions below
carry the same names and only marshal arguments (numpy arrays on the host,
torch CUDA tensors or raw device pointers on the device). Every step of the
method runs in the CUDA library ``_build/libags.so``; there is no CPU or
PyTorch fallback: if the library is missing or fails to load, the import of
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import scenes  # noqa: F401  (input generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libags.so")

AGS_OK = 0
AGS_ERR_INVALID_ARG = 1
AGS_ERR_OUT_OF_MEMORY = 2
AGS_ERR_CUDA = 3
AGS_ERR_TRAVERSAL_LIMIT = 4
AGS_ERR_NOT_READY = 5
AGS_ERR_BUSY = 6
AGS_ERR_CANCELLED = 7
STATUS_NAMES = {0: "AGS_OK", 1: "AGS_ERR_INVALID_ARG", 2: "AGS_ERR_OUT_OF_MEMORY", 3: "AGS_ERR_CUDA",
                4: "AGS_ERR_TRAVERSAL_LIMIT", 5: "AGS_ERR_NOT_READY", 6: "AGS_ERR_BUSY", 7: "AGS_ERR_CANCELLED"}

AGS_PINHOLE = 0
AGS_LIDAR = 1
AGS_RAY_TABLE = 2
AGS_NEAR_CLAMP = 0
AGS_NEAR_INVALID = 1
AGS_BVH_FP32 = 0
AGS_BVH_FP16 = 1
AGS_BVH_Q8 = 2
AGS_BUILD_LBVH = 1 << 20
AGS_BUILD_INSTANCED = 1 << 21
AGS_BUILD_GREEDY_COLLAPSE = 1 << 22


def AGS_LEAF_SIZE(n: int) -> int:
    return (int(n) & 0xF) << 8


def AGS_SPLIT_CELLS(n: int) -> int:
    return (int(n) & 0xFF) << 12


def AGS_CLUSTER_RADIUS(r: int) -> int:
    r = int(r)
    return (3 if r >= 128 else 2 if r >= 64 else 1 if r >= 32 else 0) << 23

# every symbol declared in include/ags.h
EXPORTS = [
    "ags_context_create", "ags_context_destroy", "ags_scene_build", "ags_scene_destroy", "ags_render",
    "ags_render_envs", "ags_render_host", "ags_render_count", "ags_stream_status", "ags_last_error",
    "ags_scene_n_envs", "ags_scene_get_world_triangles", "ags_scene_stats", "ags_scene_node_bytes",
    "ags_context_set_traversal_cap", "ags_transform_vertices_noalloc", "ags_autotune",
    "ags_set_launch_config", "ags_get_launch_config", "ags_memcpy_d2h", "ags_server_create", "ags_server_destroy",
    "ags_server_submit", "ags_server_poll", "ags_server_release", "ags_server_stats", "ags_server_replay",
    "ags_replay_sequential", "ags_scene_update_poses", "ags_render_graph_create", "ags_render_graph_launch",
    "ags_render_graph_destroy", "ags_render_channels", "ags_render_ex", "ags_autotune_build", "ags_scene_validate",
    "ags_server_cancel", "ags_test_sort_pairs", "ags_test_exclusive_scan", "ags_context_device",
    "ags_render_bruteforce", "ags_scene_tree_cost", "ags_scene_set_rebuild_ratio", "ags_context_set_retry_capacity",
    "ags_autotune_build_flags",
]


class AgsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ags_submesh(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("n_vertices", ctypes.c_int32), ("indices", ctypes.c_void_p),
                ("n_triangles", ctypes.c_int32), ("segment_id", ctypes.c_int32)]


class ags_env_mesh(ctypes.Structure):
    _fields_ = [("submeshes", ctypes.c_void_p), ("n_submeshes", ctypes.c_int32)]


class ags_hit_channels(ctypes.Structure):
    _fields_ = [("face", ctypes.c_void_p), ("bary", ctypes.c_void_p), ("normal", ctypes.c_void_p),
                ("point", ctypes.c_void_p)]


class ags_stereo(ctypes.Structure):
    _fields_ = [("baseline", ctypes.c_float * 3), ("eps", ctypes.c_float)]


class ags_render_options(ctypes.Structure):
    _fields_ = [("channels", ctypes.POINTER(ags_hit_channels)), ("stereo", ctypes.POINTER(ags_stereo)),
                ("ray_table", ctypes.c_void_p)]


class ags_launch_config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("rays_per_lane", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("ms", ctypes.c_float), ("stack_depth", ctypes.c_int32)]

    def as_dict(self):
        return {"tile_w": self.tile_w, "tile_h": 32 * self.rays_per_lane // self.tile_w,
                "rays_per_lane": self.rays_per_lane, "blocks_per_sm": self.blocks_per_sm, "ms": self.ms,
                "stack_depth": self.stack_depth}


class ags_server_config(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("arena_bytes", ctypes.c_int64),
                ("specs", ctypes.c_void_p), ("n_specs", ctypes.c_int32), ("auto_release", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("pad0", ctypes.c_int32)]


class ags_request(ctypes.Structure):
    _fields_ = [("env", ctypes.c_int32), ("spec", ctypes.c_int32), ("pose", ctypes.c_float * 7),
                ("tag", ctypes.c_uint64)]


class ags_completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("depth_dev", ctypes.c_void_p), ("seg_dev", ctypes.c_void_p), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


REQUEST_DTYPE = np.dtype({"names": ["env", "spec", "pose", "tag"], "formats": ["<i4", "<i4", ("<f4", 7), "<u8"],
                          "offsets": [ags_request.env.offset, ags_request.spec.offset, ags_request.pose.offset,
                                      ags_request.tag.offset], "itemsize": ctypes.sizeof(ags_request)})
COMPLETION_DTYPE = np.dtype({"names": ["request_id", "tag", "status", "depth_dev", "seg_dev", "t_submit", "t_start",
                                       "t_done"],
                             "formats": ["<u8", "<u8", "<i4", "<u8", "<u8", "<f8", "<f8", "<f8"],
                             "offsets": [getattr(ags_completion, f).offset for f in
                                         ("request_id", "tag", "status", "depth_dev", "seg_dev", "t_submit",
                                          "t_start", "t_done")],
                             "itemsize": ctypes.sizeof(ags_completion)})


class ags_sensor_spec(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("hfov_rad", ctypes.c_float), ("vfov_min_rad", ctypes.c_float), ("vfov_max_rad", ctypes.c_float),
                ("min_range", ctypes.c_float), ("max_range", ctypes.c_float), ("near_mode", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


_SUB_DTYPE = np.dtype({"names": ["vertices", "n_vertices", "indices", "n_triangles", "segment_id"],
                       "formats": ["<u8", "<i4", "<u8", "<i4", "<i4"],
                       "offsets": [ags_submesh.vertices.offset, ags_submesh.n_vertices.offset,
                                   ags_submesh.indices.offset, ags_submesh.n_triangles.offset,
                                   ags_submesh.segment_id.offset],
                       "itemsize": ctypes.sizeof(ags_submesh)})
_ENV_DTYPE = np.dtype({"names": ["submeshes", "n_submeshes"], "formats": ["<u8", "<i4"],
                       "offsets": [ags_env_mesh.submeshes.offset, ags_env_mesh.n_submeshes.offset],
                       "itemsize": ctypes.sizeof(ags_env_mesh)})

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA renderer library not built: {LIB_PATH} (run paper_2503_01471_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64
    sig = {
        "ags_context_create": (i32, [ctypes.c_int, ctypes.POINTER(vp)]),
        "ags_context_destroy": (None, [vp]),
        "ags_scene_build": (i32, [vp, vp, i32, vp, u32, ctypes.POINTER(vp)]),
        "ags_scene_destroy": (None, [vp]),
        "ags_render": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp, vp]),
        "ags_render_envs": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, i32, vp, vp, vp, vp]),
        "ags_render_host": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp]),
        "ags_render_count": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, ctypes.POINTER(ctypes.c_uint64)]),
        "ags_stream_status": (i32, [vp, vp]),
        "ags_last_error": (ctypes.c_char_p, []),
        "ags_scene_n_envs": (i32, [vp]),
        "ags_scene_get_world_triangles": (i32, [vp, i32, vp, vp, i64]),
        "ags_scene_stats": (i32, [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "ags_scene_node_bytes": (i32, [vp]),
        "ags_context_set_traversal_cap": (i32, [vp, i32]),
        "ags_context_set_retry_capacity": (i32, [vp, i32]),
        "ags_transform_vertices_noalloc": (i32, [vp, vp, i32, vp, i32, vp, vp, vp]),
        "ags_autotune": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp, i32,
                               ctypes.POINTER(ags_launch_config)]),
        "ags_set_launch_config": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), ctypes.POINTER(ags_launch_config)]),
        "ags_get_launch_config": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), ctypes.POINTER(ags_launch_config)]),
        "ags_memcpy_d2h": (i32, [vp, vp, i64]),
        "ags_server_create": (i32, [vp, vp, ctypes.POINTER(ags_server_config), ctypes.POINTER(vp)]),
        "ags_server_destroy": (None, [vp]),
        "ags_server_submit": (i32, [vp, ctypes.POINTER(ags_request), ctypes.POINTER(ctypes.c_uint64)]),
        "ags_server_poll": (i32, [vp, vp, i32, ctypes.POINTER(i32)]),
        "ags_server_release": (i32, [vp, ctypes.c_uint64]),
        "ags_server_stats": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64)]),
        "ags_server_replay": (i32, [vp, vp, vp, i32, vp]),
        "ags_replay_sequential": (i32, [vp, vp, vp, i32, vp, vp, i32, vp]),
        "ags_scene_update_poses": (i32, [vp, vp, vp, i32]),
        "ags_render_graph_create": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp, ctypes.POINTER(vp)]),
        "ags_render_graph_launch": (i32, [vp, vp]),
        "ags_render_graph_destroy": (None, [vp]),
        "ags_render_channels": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp,
                                      ctypes.POINTER(ags_hit_channels), vp]),
        "ags_render_ex": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp,
                                ctypes.POINTER(ags_render_options), vp]),
        "ags_scene_validate": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ags_server_cancel": (i32, [vp, ctypes.c_uint64]),
        "ags_render_bruteforce": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp, vp]),
        "ags_scene_tree_cost": (i32, [vp, vp, ctypes.POINTER(ctypes.c_double)]),
        "ags_scene_set_rebuild_ratio": (i32, [vp, ctypes.c_double]),
        "ags_context_device": (i32, [vp, ctypes.c_char_p, i32, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32)]),
        "ags_test_sort_pairs": (i32, [vp, vp, vp, ctypes.c_int64, i32]),
        "ags_test_exclusive_scan": (i32, [vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]),
        "ags_autotune_build": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp,
                                     ctypes.POINTER(ctypes.c_uint32), i32, i32, ctypes.POINTER(ctypes.c_uint32)]),
        "ags_autotune_build_flags": (i32, [vp, vp, ctypes.POINTER(ags_sensor_spec), vp, vp, vp,
                                           ctypes.POINTER(ctypes.c_uint32), i32, i32, ctypes.POINTER(ctypes.c_uint32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != AGS_OK:
        msg = lib().ags_last_error()
        raise AgsError(status, where, msg.decode() if msg else "")


def _ptr(x) -> int:
    """Device or host address of a torch tensor, a numpy array or an int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_spec(spec) -> ags_sensor_spec:
    """ags_sensor_spec from a ``scenes.SensorSpec`` (or anything with those fields)."""
    return ags_sensor_spec(int(spec.type), int(spec.width), int(spec.height), float(spec.hfov),
                           float(getattr(spec, "vfov_min", 0.0)), float(getattr(spec, "vfov_max", 0.0)),
                           float(spec.min_range), float(spec.max_range), int(getattr(spec, "near_mode", 0)),
                           int(getattr(spec, "flags", 0)))


# ---------------------------------------------------------------- context
def ags_context_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().ags_context_create(int(device), ctypes.byref(h)), "ags_context_create")
    return h.value


def ags_context_destroy(ctx: int) -> None:
    lib().ags_context_destroy(ctx)


def ags_context_set_traversal_cap(ctx: int, max_node_visits: int) -> None:
    _check(lib().ags_context_set_traversal_cap(ctx, int(max_node_visits)), "ags_context_set_traversal_cap")


# ---------------------------------------------------------------- scene

def ags_context_set_retry_capacity(ctx: int, rays: int) -> None:
    """Rays a short-stack render may hand to its full-stack retry pass (0..1048576)."""
    _check(lib().ags_context_set_retry_capacity(ctx, int(rays)), "ags_context_set_retry_capacity")

def ags_scene_build(ctx: int, batch, build_flags: int = AGS_BVH_FP32) -> int:
    """Build per-environment BVHs from a ``scenes.SceneBatch`` (host arrays)."""
    verts = np.ascontiguousarray(batch.vertices, np.float32)
    idx = np.ascontiguousarray(batch.indices, np.int32)
    poses = np.ascontiguousarray(batch.poses, np.float32)
    J = int(batch.sub_seg.shape[0])
    subs = np.zeros(max(J, 1), _SUB_DTYPE)
    vbase, ibase = verts.ctypes.data, idx.ctypes.data
    sv, st = np.asarray(batch.sub_vert, np.int64), np.asarray(batch.sub_tri, np.int64)
    subs["vertices"][:J] = vbase + sv[:J] * 12
    subs["n_vertices"][:J] = sv[1:] - sv[:-1]
    subs["indices"][:J] = ibase + st[:J] * 12
    subs["n_triangles"][:J] = st[1:] - st[:-1]
    subs["segment_id"][:J] = batch.sub_seg
    E = batch.n_envs
    env_sub = np.asarray(batch.env_sub, np.int64)
    envs = np.zeros(E, _ENV_DTYPE)
    envs["submeshes"] = subs.ctypes.data + env_sub[:E] * _SUB_DTYPE.itemsize
    envs["n_submeshes"] = env_sub[1:] - env_sub[:-1]
    h = ctypes.c_void_p()
    _check(lib().ags_scene_build(ctx, envs.ctypes.data, E, poses.ctypes.data if J else None, int(build_flags),
                                 ctypes.byref(h)), "ags_scene_build")
    return h.value


AGS_UPDATE_REFIT = 0
AGS_UPDATE_REBUILD = 1
AGS_UPDATE_AUTO = 2


def ags_scene_update_poses(ctx: int, scene: int, obstacle_poses, mode: int = AGS_UPDATE_REFIT) -> None:
    """Move every object to new poses ([J,7] float32, build order): refit or rebuild the BVHs."""
    p = np.ascontiguousarray(obstacle_poses, np.float32).reshape(-1, 7)
    _check(lib().ags_scene_update_poses(ctx, scene, p.ctypes.data if p.size else None, int(mode)),
           "ags_scene_update_poses")


def ags_scene_destroy(scene: int) -> None:
    lib().ags_scene_destroy(scene)


def ags_scene_n_envs(scene: int) -> int:
    return int(lib().ags_scene_n_envs(scene))


def ags_scene_node_bytes(scene: int) -> int:
    return int(lib().ags_scene_node_bytes(scene))


def ags_scene_stats(scene: int, env: int = -1):
    t, n, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ags_scene_stats(scene, int(env), ctypes.byref(t), ctypes.byref(n), ctypes.byref(b)),
           "ags_scene_stats")
    return t.value, n.value, b.value


def ags_scene_get_world_triangles(scene: int, env: int):
    n, _, _ = ags_scene_stats(scene, env)
    out = np.zeros((n, 9), np.float32)
    seg = np.zeros(n, np.int32)
    _check(lib().ags_scene_get_world_triangles(scene, int(env), out.ctypes.data, seg.ctypes.data, n),
           "ags_scene_get_world_triangles")
    return out, seg


def ags_transform_vertices_noalloc(ctx: int, base_vertices, submesh_vertex_offsets, poses, world_vertices,
                                   stream=None) -> None:
    """Object-to-world transform into caller-owned device buffers, allocating nothing.

    base_vertices float32 [V,3], submesh_vertex_offsets int32 [J+1], poses
    float32 [J,7], world_vertices float32 [>=V,4]: CUDA tensors, whose shapes
    give the sizes. Dtypes and shapes are checked here on the host (a short
    offsets array or a small output would make the kernels read or write out
    of bounds); a mismatch raises ValueError before anything is launched.
    """
    def _need(t, name, dtype, ndim, cols=None):
        if not (hasattr(t, "dtype") and hasattr(t, "shape") and hasattr(t, "is_cuda")):
            raise ValueError(f"{name} must be a CUDA tensor")
        if not t.is_cuda or t.dtype != dtype or t.dim() != ndim or (cols is not None and t.shape[1] != cols):
            raise ValueError(f"{name} must be a CUDA {dtype} tensor of {ndim} dims"
                             + (f" with {cols} columns" if cols is not None else "") + f", got {t.dtype} "
                             f"{tuple(t.shape)} on {t.device}")

    import torch
    _need(base_vertices, "base_vertices", torch.float32, 2, 3)
    _need(submesh_vertex_offsets, "submesh_vertex_offsets", torch.int32, 1)
    _need(poses, "poses", torch.float32, 2, 7)
    _need(world_vertices, "world_vertices", torch.float32, 2, 4)
    V = int(base_vertices.shape[0])
    J = int(poses.shape[0])
    if int(submesh_vertex_offsets.shape[0]) != J + 1:
        raise ValueError(f"submesh_vertex_offsets must hold J+1 = {J + 1} entries, got "
                         f"{int(submesh_vertex_offsets.shape[0])}")
    if int(world_vertices.shape[0]) < V:
        raise ValueError(f"world_vertices must have at least V = {V} rows, got {int(world_vertices.shape[0])}")
    _check(lib().ags_transform_vertices_noalloc(ctx, _ptr(base_vertices), V, _ptr(submesh_vertex_offsets), J,
                                                _ptr(poses), _ptr(world_vertices), _stream(stream)),
           "ags_transform_vertices_noalloc")


# ---------------------------------------------------------------- render
def _device_buffer(x, name: str, dtype: str, numel: int) -> None:
    """Host-side check of one device-buffer argument before any launch: a CUDA tensor of ``dtype`` ("float32"
    or "int32") holding at least ``numel`` elements. A raw device address (an int) or None passes unchecked
    (the caller vouches for it); a host array is refused, since a kernel would write through its address."""
    if x is None or isinstance(x, int):
        return
    if isinstance(x, np.ndarray):
        raise ValueError(f"{name} must be a device buffer (a CUDA tensor or a device address), not a host array")
    if hasattr(x, "is_cuda") and hasattr(x, "numel"):
        if not x.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor, not one on {x.device}")
        if str(x.dtype) != "torch." + dtype:
            raise ValueError(f"{name} must hold {dtype}, not {x.dtype}")
        if int(x.numel()) < numel:
            raise ValueError(f"{name} holds {int(x.numel())} elements, fewer than the {numel} the render writes or reads")


def _render_buffers(spec, n: int, sensor_poses, out_depth, out_seg, face=None, bary=None, normal=None, point=None,
                    ray_table=None) -> None:
    """The buffers of a render of n environments with ``spec`` (validated spec fields only: an invalid spec is
    left to the library, which rejects it)."""
    w, h = int(spec.width), int(spec.height)
    pix = n * w * h if w > 0 and h > 0 else 0
    _device_buffer(sensor_poses, "sensor_poses", "float32", 7 * n)
    _device_buffer(out_depth, "out_depth", "float32", pix)
    _device_buffer(out_seg, "out_seg", "int32", pix)
    _device_buffer(face, "face", "int32", pix)
    _device_buffer(bary, "bary", "float32", 2 * pix)
    _device_buffer(normal, "normal", "float32", 3 * pix)
    _device_buffer(point, "point", "float32", 3 * pix)
    _device_buffer(ray_table, "ray_table", "float32", 3 * w * h if w > 0 and h > 0 else 0)


def ags_render(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, stream=None) -> None:
    """Enqueue a render of every environment; tensors are CUDA tensors (or device pointers)."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg)
    _check(lib().ags_render(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth), _ptr(out_seg),
                            _stream(stream)), "ags_render")


def ags_render_envs(ctx: int, scene: int, spec, env_ids, sensor_poses, out_depth, out_seg, stream=None) -> None:
    s = make_spec(spec)
    n = int(env_ids.numel() if hasattr(env_ids, "numel") else len(env_ids))
    _device_buffer(env_ids, "env_ids", "int32", n)
    _render_buffers(s, n, sensor_poses, out_depth, out_seg)
    _check(lib().ags_render_envs(ctx, scene, ctypes.byref(s), _ptr(env_ids), n, _ptr(sensor_poses), _ptr(out_depth),
                                 _ptr(out_seg), _stream(stream)), "ags_render_envs")


def ags_render_host(ctx: int, scene: int, spec, sensor_poses_host, out_depth_host=None, out_seg_host=None):
    """Render with host buffers (numpy or pinned torch CPU tensors); returns (depth, seg)."""
    s = make_spec(spec)
    E = ags_scene_n_envs(scene)
    if out_depth_host is None:
        out_depth_host = np.zeros((E, spec.height, spec.width), np.float32)
    if out_seg_host is None:
        out_seg_host = np.zeros((E, spec.height, spec.width), np.int32)
    _check(lib().ags_render_host(ctx, scene, ctypes.byref(s), _ptr(sensor_poses_host), _ptr(out_depth_host),
                                 _ptr(out_seg_host)), "ags_render_host")
    return out_depth_host, out_seg_host


def ags_render_count(ctx: int, scene: int, spec, sensor_poses):
    """(rays, wide nodes visited, triangles tested) of one render."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, None, None)
    c = (ctypes.c_uint64 * 3)()
    _check(lib().ags_render_count(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), c), "ags_render_count")
    return int(c[0]), int(c[1]), int(c[2])


def ags_autotune(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, repeats: int = 3):
    """Pick (and remember for this scene and sensor shape) the fastest launch shape; returns it."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg)
    best = ags_launch_config()
    _check(lib().ags_autotune(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth), _ptr(out_seg),
                              int(repeats), ctypes.byref(best)), "ags_autotune")
    return best


def ags_set_launch_config(ctx: int, scene: int, spec, tile_w=None, rays_per_lane=1, blocks_per_sm=0,
                          stack_depth=0) -> None:
    """Set the launch shape for this scene and sensor shape (tile_w None clears it)."""
    s = make_spec(spec)
    cfg = None if tile_w is None else ctypes.byref(ags_launch_config(int(tile_w), int(rays_per_lane),
                                                                     int(blocks_per_sm), 0.0, int(stack_depth)))
    _check(lib().ags_set_launch_config(ctx, scene, ctypes.byref(s), cfg), "ags_set_launch_config")


def ags_get_launch_config(ctx: int, scene: int, spec) -> dict:
    s = make_spec(spec)
    c = ags_launch_config()
    _check(lib().ags_get_launch_config(ctx, scene, ctypes.byref(s), ctypes.byref(c)), "ags_get_launch_config")
    return c.as_dict()


def ags_stream_status(ctx: int, stream=None) -> int:
    """Synchronise the stream and return the device status (raises on errors)."""
    st = lib().ags_stream_status(ctx, _stream(stream))
    _check(st, "ags_stream_status")
    return st


def ags_last_error() -> str:
    m = lib().ags_last_error()
    return m.decode() if m else ""


# ---------------------------------------------------------------- serving
def ags_memcpy_d2h(dst_host: np.ndarray, src_dev: int) -> None:
    _check(lib().ags_memcpy_d2h(dst_host.ctypes.data, int(src_dev), dst_host.nbytes), "ags_memcpy_d2h")


def _spec_array(specs):
    arr = (ags_sensor_spec * len(specs))(*[make_spec(x) for x in specs])
    return arr


def ags_server_create(ctx: int, scene: int, specs, max_slots: int = 256, max_inflight: int = 2,
                      arena_bytes: int = 0, auto_release: bool = False, use_graph: bool = False) -> int:
    arr = _spec_array(specs)
    cfg = ags_server_config(int(max_slots), int(max_inflight), int(arena_bytes), ctypes.cast(arr, ctypes.c_void_p),
                            len(specs), 1 if auto_release else 0, 1 if use_graph else 0, 0)
    h = ctypes.c_void_p()
    _check(lib().ags_server_create(ctx, scene, ctypes.byref(cfg), ctypes.byref(h)), "ags_server_create")
    return h.value


def ags_server_destroy(server: int) -> None:
    lib().ags_server_destroy(server)


def ags_server_submit(server: int, env: int, spec: int, pose, tag: int = 0) -> int:
    r = ags_request(int(env), int(spec), (ctypes.c_float * 7)(*[float(x) for x in pose]), int(tag))
    rid = ctypes.c_uint64()
    _check(lib().ags_server_submit(server, ctypes.byref(r), ctypes.byref(rid)), "ags_server_submit")
    return rid.value


def ags_server_poll(server: int, max_n: int = 1024) -> np.ndarray:
    out = np.zeros(max_n, COMPLETION_DTYPE)
    n = ctypes.c_int32()
    _check(lib().ags_server_poll(server, out.ctypes.data, int(max_n), ctypes.byref(n)), "ags_server_poll")
    return out[: n.value]


def ags_server_release(server: int, request_id: int) -> None:
    _check(lib().ags_server_release(server, int(request_id)), "ags_server_release")


def ags_server_stats(server: int) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().ags_server_stats(server, *[ctypes.byref(x) for x in v]), "ags_server_stats")
    return dict(zip(("submitted", "completed", "batches", "arena_free_bytes"), (x.value for x in v)))


def make_requests(env, spec, poses, tags=None) -> np.ndarray:
    n = len(env)
    r = np.zeros(n, REQUEST_DTYPE)
    r["env"] = env
    r["spec"] = spec
    r["pose"] = np.asarray(poses, np.float32).reshape(n, 7)
    r["tag"] = np.arange(n) if tags is None else tags
    return r


def ags_server_replay(server: int, requests: np.ndarray, arrival_s) -> np.ndarray:
    arr = np.ascontiguousarray(arrival_s, np.float64)
    out = np.zeros(len(requests), COMPLETION_DTYPE)
    req = np.ascontiguousarray(requests)
    _check(lib().ags_server_replay(server, req.ctypes.data, arr.ctypes.data, len(req), out.ctypes.data),
           "ags_server_replay")
    return out


def ags_replay_sequential(ctx: int, scene: int, specs, requests: np.ndarray, arrival_s) -> np.ndarray:
    arr = np.ascontiguousarray(arrival_s, np.float64)
    out = np.zeros(len(requests), COMPLETION_DTYPE)
    req = np.ascontiguousarray(requests)
    sa = _spec_array(specs)
    _check(lib().ags_replay_sequential(ctx, scene, ctypes.cast(sa, ctypes.c_void_p), len(specs), req.ctypes.data,
                                       arr.ctypes.data, len(req), out.ctypes.data), "ags_replay_sequential")
    return out


# ---------------------------------------------------------------- step graph
def ags_render_graph_create(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg) -> int:
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg)
    h = ctypes.c_void_p()
    _check(lib().ags_render_graph_create(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth),
                                         _ptr(out_seg), ctypes.byref(h)), "ags_render_graph_create")
    return h.value


def ags_render_graph_launch(graph: int, stream=None) -> None:
    _check(lib().ags_render_graph_launch(graph, _stream(stream)), "ags_render_graph_launch")


def ags_render_graph_destroy(graph: int) -> None:
    lib().ags_render_graph_destroy(graph)


# ---------------------------------------------------------------- extra hit channels
def ags_render_channels(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, face=None, bary=None,
                        normal=None, point=None, stream=None) -> None:
    """ags_render plus the extra hit channels given (device tensors; None = not written)."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg, face, bary, normal, point)
    ch = ags_hit_channels(_ptr(face) or None, _ptr(bary) or None, _ptr(normal) or None, _ptr(point) or None)
    _check(lib().ags_render_channels(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth),
                                     _ptr(out_seg), ctypes.byref(ch), _stream(stream)), "ags_render_channels")


def ags_render_ex(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, face=None, bary=None, normal=None,
                  point=None, baseline=None, eps=0.0, ray_table=None, stream=None) -> None:
    """ags_render with optional hit channels (device tensors), stereo shadow invalidation towards a second
    sensor at ``baseline`` (3 floats, sensor frame), and, for an AGS_RAY_TABLE spec, its device direction
    table ``ray_table`` [height, width, 3]."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg, face, bary, normal, point,
                    ray_table)
    chans = (face, bary, normal, point)
    ch = None
    if any(c is not None for c in chans):
        ch = ctypes.pointer(ags_hit_channels(*(_ptr(c) or None for c in chans)))
    st = None
    if baseline is not None:
        b = [float(x) for x in baseline]
        if len(b) != 3:
            raise ValueError("baseline needs 3 values")
        st = ctypes.pointer(ags_stereo((ctypes.c_float * 3)(*b), float(eps)))
    opt = ags_render_options(ch, st, _ptr(ray_table) or None)
    _check(lib().ags_render_ex(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth), _ptr(out_seg),
                               ctypes.byref(opt), _stream(stream)), "ags_render_ex")


def ags_autotune_build(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, split_cells=(16, 32, 48, 64),
                       repeats: int = 2) -> int:
    """Rebuild the scene with each reference-splitting setting, keep the fastest; returns its cell count."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg)
    c = (ctypes.c_uint32 * len(split_cells))(*[int(x) for x in split_cells])
    best = ctypes.c_uint32()
    _check(lib().ags_autotune_build(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth), _ptr(out_seg),
                                    c, len(split_cells), int(repeats), ctypes.byref(best)), "ags_autotune_build")
    return int(best.value)


def ags_autotune_build_flags(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, flags,
                             repeats: int = 2) -> int:
    """Rebuild the scene with each candidate build_flags word, keep the fastest BVH; returns its flags."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg)
    c = (ctypes.c_uint32 * max(len(flags), 1))(*[int(x) for x in flags])
    best = ctypes.c_uint32()
    _check(lib().ags_autotune_build_flags(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth),
                                          _ptr(out_seg), c, len(flags), int(repeats), ctypes.byref(best)),
           "ags_autotune_build_flags")
    return int(best.value)


def ags_scene_validate(scene: int) -> dict:
    """Structural BVH checks; returns nodes, points, violations, depth (and the first problems if any)."""
    c = (ctypes.c_int64 * 4)()
    _check(lib().ags_scene_validate(scene, c), "ags_scene_validate")
    out = {"nodes": c[0], "points": c[1], "violations": c[2], "depth": c[3]}
    if c[2]:
        msg = lib().ags_last_error()
        out["problems"] = msg.decode() if msg else ""
    return out


def ags_server_cancel(server: int, request_id: int) -> bool:
    """Cancel a queued request; False if it is already batched, done or unknown."""
    rc = lib().ags_server_cancel(server, int(request_id))
    if rc == 0:
        return True
    if rc == AGS_ERR_BUSY:
        return False
    _check(rc, "ags_server_cancel")
    return False


def ags_test_sort_pairs(ctx: int, keys, vals, end_bit: int = 64) -> None:
    """Stable radix sort of device (uint64 key, uint32 value) pairs in place (test hook)."""
    _check(lib().ags_test_sort_pairs(ctx, _ptr(keys), _ptr(vals), int(keys.numel()), int(end_bit)),
           "ags_test_sort_pairs")


def ags_test_exclusive_scan(ctx: int, data) -> int:
    """Exclusive scan of a device int32 buffer in place; returns the total (test hook)."""
    t = ctypes.c_int32()
    _check(lib().ags_test_exclusive_scan(ctx, _ptr(data), int(data.numel()), ctypes.byref(t)),
           "ags_test_exclusive_scan")
    return int(t.value)


def ags_context_device(ctx: int) -> dict:
    """Name, SM count and compute capability of the context's device."""
    buf = ctypes.create_string_buffer(256)
    sm, cc = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().ags_context_device(ctx, buf, 256, ctypes.byref(sm), ctypes.byref(cc)), "ags_context_device")
    return {"name": buf.value.decode(), "sm_count": sm.value, "compute_capability": cc.value}


def ags_render_bruteforce(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, stream=None) -> None:
    """Every ray against every reference of its environment, no tree (a test aid; synchronous)."""
    s = make_spec(spec)
    _render_buffers(s, ags_scene_n_envs(scene), sensor_poses, out_depth, out_seg)
    _check(lib().ags_render_bruteforce(ctx, scene, ctypes.byref(s), _ptr(sensor_poses), _ptr(out_depth),
                                       _ptr(out_seg), _stream(stream)), "ags_render_bruteforce")


def ags_scene_tree_cost(ctx: int, scene: int):
    """(surface-area cost of the BVH now, as built or last rebuilt; -1 when not measured)."""
    c = (ctypes.c_double * 2)()
    _check(lib().ags_scene_tree_cost(ctx, scene, c), "ags_scene_tree_cost")
    return float(c[0]), float(c[1])


def ags_scene_set_rebuild_ratio(scene: int, ratio: float) -> None:
    _check(lib().ags_scene_set_rebuild_ratio(scene, float(ratio)), "ags_scene_set_rebuild_ratio")
