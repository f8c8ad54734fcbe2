"""Persistent cache of tuned launch shapes (a JSON file), so a later process on the same kind of GPU skips
``ags_autotune``. Entries are keyed by the device name, the sensor shape (type, width, height) and a bucket of
the scene's size (environments, and triangles rounded to a power of two); a hit is applied with
``ags_set_launch_config``. The launch shape never changes an output bit, only the speed."""
from __future__ import annotations

import json
import math
import os

from . import ags_autotune, ags_context_device, ags_scene_n_envs, ags_scene_stats, ags_set_launch_config


def cache_key(ctx: int, scene: int, spec) -> str:
    dev = ags_context_device(ctx)
    tris = ags_scene_stats(scene)[0]
    bucket = 0 if tris <= 0 else int(round(math.log2(tris)))
    return f"{dev['name']}|sm{dev['compute_capability']}|{int(spec.type)}x{int(spec.width)}x{int(spec.height)}|" \
           f"envs{ags_scene_n_envs(scene)}|tris2^{bucket}"


def autotune_cached(ctx: int, scene: int, spec, sensor_poses, out_depth, out_seg, path: str,
                    repeats: int = 2) -> dict:
    """The cached launch shape for this device, sensor shape and scene size, or a fresh ``ags_autotune``
    whose result is added to the cache file. Returns the shape (with ``"cached": True/False``)."""
    key = cache_key(ctx, scene, spec)
    cache = {}
    if os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
    if key in cache:
        c = cache[key]
        ags_set_launch_config(ctx, scene, spec, int(c["tile_w"]), int(c["rays_per_lane"]), int(c["blocks_per_sm"]),
                              int(c.get("stack_depth", 0)))
        return dict(c, cached=True)
    c = ags_autotune(ctx, scene, spec, sensor_poses, out_depth, out_seg, repeats).as_dict()
    cache[key] = c
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return dict(c, cached=False)
