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
    ok, counted = O.check(res, d, g, s.max_range)
    return ok, counted, res


def describe_failures(ok, res, depth, seg, rays, limit=5):
    """The first failing rays: renderer vs exact value and segment, the error in tolerances, the hit surface's
    incidence |n.d|, how far the float32 bands move its hit (in tolerances), the flags and the listed outcomes."""
    bad = np.nonzero(~ok)[0][:limit]
    lines = []
    for i in bad:
        r = res[i]
        t = O.tol(r["v"])
        lines.append(f"ray {int(rays[i])}: gpu=({float(depth[i])!r}, {int(seg[i])}) oracle v={r['v']!r} seg={r['seg']} "
                     f"err={abs(float(depth[i]) - r['v']) / t:.2f} tol |n.d|={r['cos_hit']:.4f} "
                     f"band={r['hit_dev'] / t:.2f} tol flags={r['flags']} "
                     f"cand={list(zip(r['cand_seg'][:r['n_cand']], r['cand_lo'][:r['n_cand']], r['cand_hi'][:r['n_cand']]))}")
    return "\n".join(lines)


U32 = 2.0 ** -24  # unit roundoff of float32


def check_channels_sensor(tris, s, pose64, res, seg, depth, ch, e, rays, detail=None):
    """check_channels for an explicit oracle scene and sensor (channel arrays ``ch`` [E, ...], env e)."""
    return _check_channels(tris, s, pose64, res, seg, depth, ch["face"][e], ch["bary"][e], ch["normal"][e],
                           ch["point"][e], rays, detail)


def check_channels(batch, e, spec, pose, res, seg, depth, face, bary, normal, point, rays, detail=None):
    """Element-wise acceptance of the extra hit channels of env e on the listed rays (flat [H*W] inputs);
    ``res`` is the oracle's result for the same rays. Returns a bool array.

    - face: -1 exactly where the segment is -1; otherwise one of the triangles the oracle's error bands
      allow for this ray (any, if that list overflowed).
    - misses: zero barycentrics and normal.
    - point: within 16 u |p| (+1e-7 m) of the FP64 reported-value-times-direction for the renderer's own
      value (the value itself is checked against the oracle separately).
    - barycentrics, through the point they name on the face: within 8 (dir_rel t + arith_rel r + 2u c) /
      |cos(n, d)| of the FP64 hit, i.e. the float32 ray's and the intersection arithmetic's displacement
      of the hit across the face, stretched by the incidence angle.
    - normal: within 16 u / sin(angle at v0) + 8 sqrt(3) u c / h + 1e-6 of the FP64 unit normal (the
      rounding of the two edge vectors and their cross product, and the float32 world vertices' rounding
      against the shortest altitude h); the sign is free where |cos(n, d)| < 1e-4.
    ``detail`` (a dict) receives each check's pass mask and the errors, for failure reports.
    """
    tris, _ = oracle_env(batch, e)
    return _check_channels(tris, oracle_sensor(spec), np.asarray(pose, np.float32).astype(np.float64), res, seg,
                           depth, face, bary, normal, point, rays, detail)


def _check_channels(tris, s, pose64, res, seg, depth, face, bary, normal, point, rays, detail):
    g = np.asarray(seg).reshape(-1)[rays]
    v = np.asarray(depth, np.float32).reshape(-1)[rays].astype(np.float64)
    f = np.asarray(face).reshape(-1)[rays]
    b = np.asarray(bary, np.float32).reshape(-1, 2)[rays].astype(np.float64)
    nm = np.asarray(normal, np.float32).reshape(-1, 3)[rays].astype(np.float64)
    pt = np.asarray(point, np.float32).reshape(-1, 3)[rays].astype(np.float64)
    miss = g == -1
    d = detail if detail is not None else {}
    d["face_vs_seg"] = (f == -1) == miss
    d["miss_zero"] = ~miss | ((b == 0).all(1) & (nm == 0).all(1))
    overflow = (res["flags"] & O.F_TRI_OVERFLOW) != 0
    in_cand = np.array([bool(overflow[i]) or int(f[i]) in res["cand_tri"][i][:res["n_tri"][i]]
                        for i in range(len(rays))])
    d["face_candidate"] = miss | in_cand
    fb, fn, fp = O.hit_channels(tris, s, pose64, rays, np.where(miss | (f < 0), -1, f), v)
    lp = np.linalg.norm(fp, axis=1)
    d["point_err"] = np.linalg.norm(pt - fp, axis=1)
    d["point"] = d["point_err"] <= 16 * U32 * lp + 1e-7
    ok = d["face_vs_seg"] & d["miss_zero"] & d["face_candidate"] & d["point"]
    hit = np.nonzero(~miss & (f >= 0))[0]
    if hit.size:
        tri = tris[f[hit]].reshape(-1, 3, 3)
        v0, e1, e2 = tri[:, 0], tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]
        p_gpu = v0 + b[hit, :1] * e1 + b[hit, 1:] * e2
        p_orc = v0 + fb[hit, :1] * e1 + fb[hit, 1:] * e2
        R = O.rotation(pose64[3:])
        dw = fp[hit] @ R.T
        dw /= np.linalg.norm(dw, axis=1, keepdims=True)
        o = pose64[:3]
        cosn = np.abs(np.sum(fn[hit] * dw, 1))
        rmax = np.max(np.linalg.norm(tri - o, axis=2), axis=1)
        cmax = np.maximum(np.max(np.abs(tri), axis=(1, 2)), 1.0)
        t = lp[hit]
        tol_p = 8 * (s.dir_rel * t + s.arith_rel * rmax + 2 * U32 * cmax) / np.maximum(cosn, 1e-6)
        bary_err = np.linalg.norm(p_gpu - p_orc, axis=1)
        cr = np.linalg.norm(np.cross(e1, e2), axis=1)
        sin0 = cr / (np.linalg.norm(e1, axis=1) * np.linalg.norm(e2, axis=1))
        lmax = np.max(np.linalg.norm(np.stack([e1, e2, e2 - e1], 1), axis=2), axis=1)
        # the float32 world vertices differ from the oracle's FP64 ones by up to 2 u c per coordinate:
        # that turns the plane by up to 4 sqrt(3) (2 u c) / (shortest altitude)
        tol_n = 16 * U32 / sin0 + 4 * np.sqrt(3) * 2 * U32 * cmax / (cr / lmax) + 1e-6
        dn = np.linalg.norm(nm[hit] - fn[hit], axis=1)
        dn_flip = np.linalg.norm(nm[hit] + fn[hit], axis=1)
        d["bary"] = np.ones(len(rays), bool)
        d["bary"][hit] = bary_err <= tol_p
        d["normal"] = np.ones(len(rays), bool)
        d["normal"][hit] = (dn <= tol_n) | ((cosn < 1e-4) & (dn_flip <= tol_n))
        d["bary_err"], d["bary_tol"], d["normal_err"], d["normal_tol"], d["hit"] = bary_err, tol_p, dn, tol_n, hit
        d["oracle_bary"], d["oracle_normal"] = fb, fn
        ok &= d["bary"] & d["normal"]
    return ok


def describe_channel_failures(ok, detail, res, face, bary, normal, limit=5):
    lines = []
    hit_pos = {int(h): k for k, h in enumerate(detail.get("hit", []))}
    for i in np.nonzero(~ok)[0][:limit]:
        failed = [k for k in ("face_vs_seg", "miss_zero", "face_candidate", "point", "bary", "normal")
                  if k in detail and not detail[k][i]]
        line = (f"ray {int(i)}: failed {failed}; gpu face {int(face[i])} bary {bary[i]} normal {normal[i]}; oracle tri "
                f"{int(res[i]['tri'])} cands {list(res[i]['cand_tri'][:res[i]['n_tri']])} bary {detail['oracle_bary'][i]} "
                f"normal {detail['oracle_normal'][i]}; point err {detail['point_err'][i]:.3g}")
        if i in hit_pos:
            k = hit_pos[int(i)]
            line += (f"; bary err {detail['bary_err'][k]:.3g} tol {detail['bary_tol'][k]:.3g}; normal err "
                     f"{detail['normal_err'][k]:.3g} tol {detail['normal_tol'][k]:.3g}")
        lines.append(line)
    return "\n".join(lines)
