"""Shared test helpers: spec conversion and oracle comparison of renderer outputs."""
from __future__ import annotations

import numpy as np

import oracle as O


def oracle_sensor(spec) -> O.Sensor:
    """The oracle's sensor for a renderer spec (same float32 values, widened)."""
    f = lambda x: float(np.float32(x))  # noqa: E731
    return O.Sensor(type=int(spec.type), width=int(spec.width), height=int(spec.height), hfov=f(spec.hfov),
                    min_range=f(spec.min_range), max_range=f(spec.max_range), vfov_min=f(spec.vfov_min),
                    vfov_max=f(spec.vfov_max), near_mode=int(spec.near_mode))


def oracle_env(batch, e):
    vs, ix, ps, sg = batch.env_submeshes(e)
    return O.world_triangles(vs, ix, ps, sg)


def compare_env(batch, e, spec, pose, depth, seg, rays=None):
    """Check renderer outputs of env e (flat [H*W] arrays) on the listed rays. Returns (ok, counted)."""
    tris, tseg = oracle_env(batch, e)
    s = oracle_sensor(spec)
    if rays is None:
        rays = np.arange(spec.width * spec.height, dtype=np.int64)
    res = O.render(tris, tseg, s, np.asarray(pose, np.float32).astype(np.float64), rays)
    d = np.asarray(depth, np.float32).reshape(-1)[rays]
    g = np.asarray(seg, np.int32).reshape(-1)[rays]
    ok, counted, strict = O.check(res, d, g, s.max_range, with_strict=True)
    compare_env.last_strict = strict
    compare_env.last_wide = (res["flags"] & O.F_WIDE) != 0
    return ok, counted, res


def describe_failures(ok, res, depth, seg, rays, limit=5):
    bad = np.nonzero(~ok)[0][:limit]
    lines = []
    for i in bad:
        r = res[i]
        lines.append(f"ray {int(rays[i])}: gpu=({float(depth[i])!r}, {int(seg[i])}) oracle v={r['v']!r} seg={r['seg']} "
                     f"flags={r['flags']} cand={list(zip(r['cand_seg'][:r['n_cand']], r['cand_lo'][:r['n_cand']], r['cand_hi'][:r['n_cand']]))}")
    return "\n".join(lines)
