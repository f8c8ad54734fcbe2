"""Checks that pin the FP64 oracle to facts outside itself.

Each ``pin_*`` function takes a loaded oracle library (so the same checks can
run against deliberately broken builds in test_oracle_mutants.py) and raises
AssertionError when the oracle disagrees with:
  - scipy's quaternion rotation (a library routine, for the transform);
  - closed forms of the camera / LiDAR ray geometry;
  - closed-form depths and ranges (wall, cylinder facets, icosphere bounds);
  - hand-worked cases stored in tests/golden/hand_worked.json;
  - a numpy.linalg.solve brute force on tiny random scenes;
  - invariants (exact misses, translation/rotation of the whole scene).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_worked.json")


def _sensor_from(d):
    return O.Sensor(
        type=d["type"], width=d["width"], height=d["height"], hfov=math.radians(d["hfov_deg"]),
        min_range=d["min_range"], max_range=d["max_range"],
        vfov_min=math.radians(d.get("vfov_min_deg", 0.0)),
        vfov_max=math.radians(d.get("vfov_max_deg", 0.0)), near_mode=d.get("near_mode", 0))


def _rot_scipy(q):
    from scipy.spatial.transform import Rotation
    return Rotation.from_quat(np.asarray(q, np.float64)).as_matrix()


def _quat_from_matrix_scipy(R):
    from scipy.spatial.transform import Rotation
    return Rotation.from_matrix(R).as_quat()


IDENT = np.array([0, 0, 0, 0, 0, 0, 1.0])


# ---------------------------------------------------------------- a1 transform
def pin_rotation_vs_scipy(lib):
    rng = np.random.default_rng(11)
    for _ in range(200):
        q = rng.normal(size=4) * rng.uniform(0.1, 5.0)  # not normalised on purpose
        R = O.rotation(q, lib)
        assert np.allclose(R, _rot_scipy(q), atol=1e-13, rtol=0), (q, R)


def pin_transform_vs_scipy(lib):
    rng = np.random.default_rng(12)
    for _ in range(50):
        q = rng.normal(size=4)
        p = rng.uniform(-10, 10, 3)
        v = rng.uniform(-3, 3, (40, 3))
        out = O.transform(v, np.concatenate([p, q]), lib)
        ref = v @ _rot_scipy(q).T + p
        assert np.allclose(out, ref, atol=1e-12, rtol=0)


def pin_transform_identity_exact(lib):
    rng = np.random.default_rng(13)
    v = rng.uniform(-100, 100, (1000, 3))
    out = O.transform(v, IDENT, lib)
    assert np.array_equal(out, v)


# ---------------------------------------------------------------- a3 rays
def pin_camera_centre_and_corner(lib):
    rng = np.random.default_rng(14)
    for _ in range(20):
        W, H = 2 * int(rng.integers(1, 40)) + 1, 2 * int(rng.integers(1, 30)) + 1
        hfov = rng.uniform(0.3, 2.5)
        s = O.Sensor(O.PINHOLE, W, H, hfov, 0.1, 10.0)
        q = rng.normal(size=4)
        pose = np.concatenate([rng.uniform(-5, 5, 3), q])
        R = _rot_scipy(q)
        fwd = R[:, 0]
        o, d, sc = O.ray(s, pose, H // 2, W // 2, lib)
        assert np.allclose(o, pose[:3], atol=0)
        assert np.allclose(d, fwd, atol=1e-14), "centre pixel looks along the optical axis"
        assert abs(sc - 1.0) < 1e-14
        f = (W / 2) / math.tan(hfov / 2)
        a, b = (W / 2 - 0.5) / f, (H / 2 - 0.5) / f
        o, d, sc = O.ray(s, pose, 0, 0, lib)
        ang = math.acos(min(1.0, float(d @ fwd)))
        assert abs(ang - math.atan(math.hypot(a, b))) < 1e-12
        # top-left pixel looks left (+y body) and up (+z body)
        local = R.T @ d
        assert local[1] > 0 and local[2] > 0
        assert abs(sc - 1.0 / math.sqrt(1 + a * a + b * b)) < 1e-13
        assert abs(np.linalg.norm(d) - 1) < 1e-14


def pin_camera_column_angles(lib):
    W, H, hfov = 16, 4, math.radians(87)
    s = O.Sensor(O.PINHOLE, W, H, hfov, 0.1, 10.0)
    f = (W / 2) / math.tan(hfov / 2)
    for c in range(W):
        o, d, _ = O.ray(s, IDENT, 1, c, lib)
        az = math.atan2(d[1], d[0])
        assert abs(az - math.atan((W / 2 - c - 0.5) / f)) < 1e-13
    # mirrored columns mirror the direction in y
    for c in range(W):
        _, d1, _ = O.ray(s, IDENT, 0, c, lib)
        _, d2, _ = O.ray(s, IDENT, 0, W - 1 - c, lib)
        assert np.allclose(d1 * [1, -1, 1], d2, atol=1e-15)


def pin_lidar_angles(lib):
    C, A = 7, 12
    vmin, vmax = math.radians(-22.5), math.radians(22.5)
    s = O.Sensor(O.LIDAR, A, C, 2 * math.pi, 0.3, 50.0, vmin, vmax)
    for k in range(C):
        for j in range(A):
            o, d, sc = O.ray(s, IDENT, k, j, lib)
            assert abs(np.linalg.norm(d) - 1) < 1e-14 and sc == 1.0
            el = math.asin(d[2])
            assert abs(el - (vmax - k * (vmax - vmin) / (C - 1))) < 1e-13
            az = math.atan2(d[1], d[0]) % (2 * math.pi)
            want = (2 * math.pi * j / A) % (2 * math.pi)
            assert min(abs(az - want), 2 * math.pi - abs(az - want)) < 1e-13
    # yaw by +90 deg turns azimuth 0 into +y
    q = np.array([0, 0, math.sin(math.pi / 4), math.cos(math.pi / 4)])
    _, d, _ = O.ray(s, np.concatenate([[1, 2, 3], q]), (C - 1) // 2, 0, lib)
    assert np.allclose(d, [0, 1, 0], atol=1e-15)


# ---------------------------------------------------------------- a4-a6 closed forms
def _quad(x, half, seg, tris, segs):
    tris += [[x, -half, -half, x, half, -half, x, half, half], [x, -half, -half, x, half, half, x, -half, half]]
    segs += [seg, seg]


def pin_wall_depth_constant(lib):
    """Camera facing a huge wall at distance D: depth = D everywhere, range = D / cos."""
    rng = np.random.default_rng(15)
    for _ in range(6):
        D = rng.uniform(0.5, 9.0)
        q = rng.normal(size=4)
        R = _rot_scipy(q)
        p = rng.uniform(-3, 3, 3)
        # wall in the camera frame at x = D, moved to the world by the same pose
        local = np.array([[D, -60, -60], [D, 60, -60], [D, 60, 60], [D, -60, 60]])
        wv = local @ R.T + p
        tris = np.array([np.concatenate([wv[0], wv[1], wv[2]]), np.concatenate([wv[0], wv[2], wv[3]])])
        seg = np.array([3, 3], np.int32)
        s = O.Sensor(O.PINHOLE, 24, 18, math.radians(87), 0.1, 10.0)
        pose = np.concatenate([p, q])
        r = O.render(tris, seg, s, pose, lib=lib)
        assert np.all(np.abs(r["v"] - D) <= 1e-9 * D)
        assert np.all(r["seg"] == 3)
        sl = O.Sensor(O.LIDAR, 16, 5, 2 * math.pi, 0.1, 1e5, -0.4, 0.4)
        rl = O.render(tris, seg, sl, pose, lib=lib)
        for idx in range(16 * 5):
            k, j = divmod(idx, 16)
            _, d, _ = O.ray(sl, pose, k, j, lib)
            cos = float(d @ R[:, 0])
            if cos > 1e-3:
                assert abs(rl["v"][idx] - D / cos) <= 1e-9 * D / cos
                assert rl["seg"][idx] == 3
            elif cos < 0:
                assert rl["seg"][idx] == -1 and rl["v"][idx] == 1e5


def pin_lidar_cylinder_facets(lib):
    """LiDAR on the axis of a closed 32-gon prism: range = r cos(pi/n) / cos(psi - facet normal) / cos(phi)."""
    n, r, h = 32, 2.0, 40.0
    th = 2 * np.pi * np.arange(n) / n
    ring = np.stack([np.cos(th), np.sin(th)], 1) * r
    tris, segs = [], []
    for k in range(n):
        k1 = (k + 1) % n
        a0, a1 = ring[k], ring[k1]
        v0, v1 = [a0[0], a0[1], -h / 2], [a1[0], a1[1], -h / 2]
        v2, v3 = [a1[0], a1[1], h / 2], [a0[0], a0[1], h / 2]
        tris += [v0 + v1 + v2, v0 + v2 + v3]
        segs += [k, k]
    tris = np.array(tris, float)
    seg = np.array(segs, np.int32)
    C, A = 9, 100
    s = O.Sensor(O.LIDAR, A, C, 2 * math.pi, 0.1, 50.0, math.radians(-22.5), math.radians(22.5))
    pose = np.array([0, 0, 0.0, 0, 0, 0, 1])
    res = O.render(tris, seg, s, pose, lib=lib)
    for idx in range(C * A):
        k, j = divmod(idx, A)
        phi = math.radians(22.5) - k * math.radians(45) / (C - 1)
        psi = 2 * math.pi * j / A
        f = int(psi // (2 * math.pi / n)) % n
        normal = (th[f] + math.pi / n)
        want = r * math.cos(math.pi / n) / math.cos(psi - normal) / math.cos(phi)
        if res["flags"][idx] & O.F_SILHOUETTE:
            continue  # beam along a facet edge: either facet is right
        assert abs(res["v"][idx] - want) < 1e-10 * want, (idx, res["v"][idx], want)
        assert res["seg"][idx] == f


def pin_icosphere_bounds(lib):
    """Rays at an icosphere: the hit lies between the analytic spheres of radius r and r_in."""
    from paper_2503_01471_gb300.scenes import icosphere_unit
    v, f = icosphere_unit(2)
    r, L = 0.8, 4.0
    c = np.array([L, 0.3, -0.2])
    verts = v * r + c
    tris = verts[f].reshape(-1, 9)
    # inscribed radius: smallest distance from the centre to a face plane
    a, b, cc = verts[f[:, 0]], verts[f[:, 1]], verts[f[:, 2]]
    nrm = np.cross(b - a, cc - a)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = float(np.min(np.abs(np.sum((a - c) * nrm, 1))))
    assert r_in < r
    seg = np.full(len(tris), 6, np.int32)
    s = O.Sensor(O.LIDAR, 64, 16, 0.6, 0.1, 50.0, -0.25, 0.25)
    q = _quat_from_matrix_scipy(np.eye(3))
    pose = np.concatenate([[0, 0, 0.0], q])
    # aim the azimuth fan at the sphere: rotate by -0.3 rad about z
    from scipy.spatial.transform import Rotation
    pose[3:] = Rotation.from_euler("z", math.atan2(c[1], c[0]) - 0.3).as_quat()
    res = O.render(tris, seg, s, pose, lib=lib)
    n_hit = 0
    for idx in range(64 * 16):
        k, j = divmod(idx, 64)
        o, d, _ = O.ray(s, pose, k, j, lib)
        m = float(d @ (c - o))
        b2 = float((c - o) @ (c - o)) - m * m
        if b2 < r_in * r_in * 0.999:
            lo, hi = m - math.sqrt(r * r - b2), m - math.sqrt(r_in * r_in - b2)
            assert res["seg"][idx] == 6
            assert lo - 1e-12 <= res["v"][idx] <= hi + 1e-12, (idx, lo, res["v"][idx], hi)
            n_hit += 1
        elif b2 > r * r * 1.001:
            assert res["seg"][idx] == -1 and res["v"][idx] == 50.0
    assert n_hit > 50
    # the centre ray: t in [L' - r, L' - r_in]
    s1 = O.Sensor(O.PINHOLE, 1, 1, 0.5, 0.1, 50.0)
    d0 = c / np.linalg.norm(c)
    from scipy.spatial.transform import Rotation as Rot
    rot, _ = Rot.align_vectors([d0], [[1, 0, 0]])
    res = O.render(tris, seg, s1, np.concatenate([[0, 0, 0], rot.as_quat()]), lib=lib)
    Lc = float(np.linalg.norm(c))
    assert Lc - r - 1e-12 <= res["v"][0] <= Lc - r_in + 1e-12


def pin_hand_worked(lib):
    with open(GOLDEN) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        s = _sensor_from(case["sensor"])
        tris = np.array(case["triangles"], float)
        seg = np.array(case["segs"], np.int32)
        res = O.render(tris, seg, s, IDENT, lib=lib)
        depth = np.array(case["depth"], float).reshape(-1)
        want_seg = np.array(case["seg"]).reshape(-1)
        counted = np.zeros(depth.shape, bool)
        if "counted" in case:
            counted = np.array(case["counted"]).reshape(-1).astype(bool)
            assert np.array_equal((res["flags"] & O.F_COUNTED) != 0, counted), case["name"]
        for i in range(depth.shape[0]):
            if not counted[i]:
                assert abs(res["v"][i] - depth[i]) <= 1e-12, (case["name"], i, res["v"][i], depth[i])
                assert res["seg"][i] == want_seg[i], (case["name"], i, res["seg"][i], want_seg[i])
                continue
            # several outcomes are right (an exact edge or range tie): the
            # hand-worked one must be among the accepted outcomes
            ok, _ = O.check(res[i:i + 1], [depth[i]], [want_seg[i]], s.max_range)
            assert ok[0], (case["name"], i, res[i])


def _brute_solve(tris, seg, o, d, t_far):
    """Nearest hit by solving o + t d = v0 + u e1 + w e2 with numpy.linalg.solve."""
    best_t, best_i = math.inf, -1
    for i, tri in enumerate(tris):
        v0, v1, v2 = tri[:3], tri[3:6], tri[6:]
        M = np.stack([d, v0 - v1, v0 - v2], 1)
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        t, u, w = np.linalg.solve(M, v0 - o)
        if u >= 0 and w >= 0 and u + w <= 1 and 0 <= t <= t_far and t < best_t:
            best_t, best_i = t, i
    return best_t, best_i


def pin_brute_force_linear_solve(lib):
    rng = np.random.default_rng(16)
    checked = 0
    for trial in range(12):
        F = int(rng.integers(1, 9))
        tris = rng.uniform(-4, 4, (F, 9))
        seg = rng.integers(0, 5, F).astype(np.int32)
        s = O.Sensor(O.PINHOLE, 12, 9, math.radians(100), 0.05, 20.0)
        q = rng.normal(size=4)
        pose = np.concatenate([rng.uniform(-1, 1, 3), q])
        res = O.render(tris, seg, s, pose, lib=lib)
        for idx in range(12 * 9):
            if res["flags"][idx] & (O.F_SILHOUETTE | O.F_NEAR_TIE | O.F_RANGE_EDGE):
                continue
            k, j = divmod(idx, 12)
            o, d, sc = O.ray(s, pose, k, j, lib)
            t, i = _brute_solve(tris, seg, o, d, 20.0 / sc)
            if i < 0:
                assert res["seg"][idx] == -1 and res["v"][idx] == 20.0
            else:
                v = max(t * sc, 0.05)
                assert abs(res["v"][idx] - v) < 1e-9, (trial, idx, res["v"][idx], v)
                assert res["seg"][idx] == seg[i] and res["tri"][idx] == i
            checked += 1
    assert checked > 800


# ---------------------------------------------------------------- invariants
def _room_scene():
    from paper_2503_01471_gb300 import scenes as S
    sc, spec, poses = S.tiny_room()
    vs, ix, ps, sg = sc.env_submeshes(0)
    return vs, ix, ps, sg, spec, poses


def pin_miss_exact(lib):
    """Rays leaving an open scene report exactly max_range and segment -1."""
    tris = np.array([[3, -1, -1, 3, 1, -1, 3, 0, 1.0]])
    seg = np.array([2], np.int32)
    s = O.Sensor(O.LIDAR, 36, 9, 2 * math.pi, 0.3, 37.5, -0.3, 0.3)
    res = O.render(tris, seg, s, IDENT, lib=lib)
    miss = res["seg"] == -1
    assert miss.sum() > 300
    assert np.all(res["v"][miss] == 37.5)
    assert np.all(res["flags"][miss] & O.F_MISS_OK)
    assert np.all(res["n_cand"][miss] == 0)


def pin_translation_rotation_invariance(lib):
    vs, ix, ps, sg, spec, poses = _room_scene()
    s = O.Sensor(O.PINHOLE, spec.width, spec.height, spec.hfov, spec.min_range, spec.max_range)
    tris, seg = O.world_triangles(vs, ix, ps, sg)
    rng = np.random.default_rng(17)
    for p in poses[:4].astype(np.float64):
        base = O.render(tris, seg, s, p, lib=lib)
        off = rng.uniform(-50, 50, 3)
        t2 = tris + np.tile(off, 3)
        p2 = p.copy()
        p2[:3] += off
        moved = O.render(t2, seg, s, p2, lib=lib)
        amb = O.F_SILHOUETTE | O.F_NEAR_TIE
        ok = ((base["flags"] | moved["flags"]) & amb) == 0
        assert ok.mean() > 0.9
        assert np.array_equal(base["seg"][ok], moved["seg"][ok])
        assert np.all(np.abs(base["v"][ok] - moved["v"][ok]) <= O.tol(base["v"][ok]))
        # common rotation about the sensor
        from scipy.spatial.transform import Rotation
        rot = Rotation.from_quat(rng.normal(size=4))
        t3 = (rot.apply((tris.reshape(-1, 3) - p[:3])) + p[:3]).reshape(-1, 9)
        p3 = p.copy()
        p3[3:] = (rot * Rotation.from_quat(p[3:])).as_quat()
        rotd = O.render(t3, seg, s, p3, lib=lib)
        ok = ((base["flags"] | rotd["flags"]) & amb) == 0
        assert np.array_equal(base["seg"][ok], rotd["seg"][ok])
        assert np.all(np.abs(base["v"][ok] - rotd["v"][ok]) <= O.tol(base["v"][ok]))


def pin_degenerate_never_hits(lib):
    tris = np.array([[3, -1, -1, 3, 1, 1, 3, 0, 0.0], [3, 0, 0, 3, 0, 0, 3, 0, 0.0]])  # collinear, point
    seg = np.array([1, 2], np.int32)
    s = O.Sensor(O.PINHOLE, 1, 1, 1.0, 0.1, 10.0)
    res = O.render(tris, seg, s, IDENT, lib=lib)
    assert res["seg"][0] == -1 and res["v"][0] == 10.0
    # the ray runs exactly through both: still no acceptable hit outcome
    assert res["n_cand"][0] == 0 and (res["flags"][0] & O.F_COUNTED) == 0


def pin_tie_break(lib):
    """Coincident triangles: equal distance goes to the smaller index; both are acceptable."""
    t = [4, -2, -2, 4, 2, -2, 4, 0, 2.0]
    s = O.Sensor(O.PINHOLE, 1, 1, 1.0, 0.1, 10.0)
    for segs, want in (([5, 8], 5), ([8, 5], 8)):
        res = O.render(np.array([t, t]), np.array(segs, np.int32), s, IDENT, lib=lib)
        assert res["seg"][0] == want and res["tri"][0] == 0 and res["v"][0] == 4.0
        assert res["flags"][0] & O.F_NEAR_TIE and res["flags"][0] & O.F_COUNTED
        assert sorted(res["cand_seg"][0][:res["n_cand"][0]]) == [5, 8]


# ---------------------------------------------------------------- extra hit channels
def pin_channels_wall(lib):
    """Wall at x = D in the sensor frame (either winding): the normal is minus the camera axis, and the
    sensor-frame point, moved to the world, lies on the wall and on the pixel's ray."""
    rng = np.random.default_rng(17)
    for trial in range(6):
        D = rng.uniform(0.5, 9.0)
        q = rng.normal(size=4)
        R = _rot_scipy(q)
        p = rng.uniform(-3, 3, 3)
        local = np.array([[D, -60, -60], [D, 60, -60], [D, 60, 60], [D, -60, 60]])
        wv = local @ R.T + p
        order = (0, 1, 2, 0, 2, 3) if trial % 2 == 0 else (0, 2, 1, 0, 3, 2)
        tris = np.array([np.concatenate([wv[i] for i in order[:3]]), np.concatenate([wv[i] for i in order[3:]])])
        seg = np.array([3, 3], np.int32)
        pose = np.concatenate([p, q])
        for s in (O.Sensor(O.PINHOLE, 24, 18, math.radians(87), 0.1, 10.0),
                  O.Sensor(O.LIDAR, 16, 5, math.radians(80), 0.1, 1e5, -0.4, 0.4)):
            n = s.width * s.height
            rays = np.arange(n)
            r = O.render(tris, seg, s, pose, lib=lib)
            assert (r["seg"] == 3).all()
            bary, normal, point = O.hit_channels(tris, s, pose, rays, r["tri"], r["v"], lib=lib)
            assert np.allclose(normal, -R[:, 0], atol=1e-12)
            Pw = point @ R.T + p
            assert np.allclose((Pw - p) @ R[:, 0], D, rtol=0, atol=1e-9 * D)
            for idx in range(n):
                o, d, _ = O.ray(s, pose, idx // s.width, idx % s.width, lib)
                assert np.linalg.norm(np.cross(Pw[idx] - o, d)) <= 1e-9 * np.linalg.norm(Pw[idx] - o)
                assert (Pw[idx] - o) @ d > 0
                w = tris[r["tri"][idx]].reshape(3, 3)
                assert np.allclose(w[0] + bary[idx, 0] * (w[1] - w[0]) + bary[idx, 1] * (w[2] - w[0]), Pw[idx],
                                   atol=1e-9)


def pin_channels_linear_solve(lib):
    """Barycentrics against numpy.linalg.solve of o + t d = v0 + u (v1 - v0) + w (v2 - v0), and the
    normal against the null space of the edge vectors (SVD), on random triangles."""
    rng = np.random.default_rng(18)
    checked = 0
    for trial in range(12):
        F = int(rng.integers(1, 9))
        tris = rng.uniform(-4, 4, (F, 9))
        seg = rng.integers(0, 5, F).astype(np.int32)
        s = O.Sensor(O.PINHOLE, 12, 9, math.radians(100), 0.05, 20.0)
        pose = np.concatenate([rng.uniform(-1, 1, 3), rng.normal(size=4)])
        res = O.render(tris, seg, s, pose, lib=lib)
        hit = np.nonzero(res["tri"] >= 0)[0]
        bary, normal, _ = O.hit_channels(tris, s, pose, hit, res["tri"][hit], res["v"][hit], lib=lib)
        for k, idx in enumerate(hit):
            if res["flags"][idx] & (O.F_SILHOUETTE | O.F_NEAR_TIE | O.F_RANGE_EDGE):
                continue
            o, d, _ = O.ray(s, pose, idx // 12, idx % 12, lib)
            v0, v1, v2 = tris[res["tri"][idx]].reshape(3, 3)
            t, u, w = np.linalg.solve(np.stack([d, v0 - v1, v0 - v2], 1), v0 - o)
            assert abs(bary[k, 0] - u) < 1e-9 and abs(bary[k, 1] - w) < 1e-9, (trial, idx, bary[k], u, w)
            nul = np.linalg.svd(np.stack([v1 - v0, v2 - v0]))[2][2]
            assert abs(abs(float(normal[k] @ nul)) - 1.0) < 1e-12
            assert float(normal[k] @ d) <= 0.0
            checked += 1
    assert checked > 300


def pin_channels_icosphere(lib):
    """Rays at an icosphere from outside: the face normal points out (within the facet angle), and the
    reported face holds the hit point."""
    from paper_2503_01471_gb300.scenes import icosphere_unit
    v, f = icosphere_unit(2)
    c = np.array([3.0, 0.2, -0.1])
    tris = (v * 0.7 + c)[f].reshape(-1, 9)
    seg = np.full(len(tris), 2, np.int32)
    s = O.Sensor(O.PINHOLE, 32, 24, 0.6, 0.1, 20.0)
    res = O.render(tris, seg, s, IDENT, lib=lib)
    hit = np.nonzero(res["tri"] >= 0)[0]
    assert hit.shape[0] > 100
    bary, normal, point = O.hit_channels(tris, s, IDENT, hit, res["tri"][hit], res["v"][hit], lib=lib)
    radial = point - c
    radial /= np.linalg.norm(radial, axis=1, keepdims=True)
    assert (np.sum(normal * radial, 1) > 0.95).all()
    assert (bary >= -1e-12).all() and (bary.sum(1) <= 1 + 1e-12).all()


def pin_channels_miss_and_lidar_norm(lib):
    """A miss gives zero barycentrics and normal and the point at the reported value along the ray; a LiDAR
    point's length is the range."""
    s = O.Sensor(O.LIDAR, 32, 4, 2 * math.pi, 0.1, 30.0, -0.3, 0.3)
    rays = np.arange(128)
    v = np.linspace(1.0, 30.0, 128)
    bary, normal, point = O.hit_channels(np.zeros((0, 9)), s, IDENT, rays, np.full(128, -1), v, lib=lib)
    assert not bary.any() and not normal.any()
    assert np.allclose(np.linalg.norm(point, axis=1), v, rtol=1e-14)
    for idx in (0, 37, 127):
        o, d, _ = O.ray(s, IDENT, idx // 32, idx % 32, lib)
        assert np.allclose(point[idx], v[idx] * d, atol=1e-12)


def pin_candidate_triangles(lib):
    """A ray through the interior of one triangle lists only it; a ray along the shared edge of two
    lists both."""
    quad = [[3, -1, -1, 3, 1, -1, 3, 1, 1], [3, -1, -1, 3, 1, 1, 3, -1, 1]]  # diagonal through (3, 0, 0)
    s = O.Sensor(O.PINHOLE, 1, 1, 1.0, 0.1, 10.0)
    res = O.render(np.array(quad, float), np.array([4, 4], np.int32), s, IDENT, lib=lib)
    assert sorted(res["cand_tri"][0][:res["n_tri"][0]]) == [0, 1]
    off = np.array(quad, float) + np.array([0, 0.5, -0.3] * 3)
    res = O.render(off, np.array([4, 4], np.int32), s, IDENT, lib=lib)
    assert res["n_tri"][0] == 1 and res["cand_tri"][0][0] == res["tri"][0] == 1  # (y, z) = (-0.5, 0.3): y < z


# ---------------------------------------------------------------- stereo shadows
def _rect(x, y0, y1, z0, z1):
    return [[x, y0, z0, x, y1, z0, x, y1, z1], [x, y0, z0, x, y1, z1, x, y0, z1]]


def pin_shadow_plate_closed_form(lib):
    """Wall at x = D behind a plate at x = D/2, second sensor at baseline (0, b, 0): a wall pixel is
    shadowed iff the segment from its wall point to the second sensor crosses the plate, which happens
    where it meets x = D/2, at the midpoint; plate pixels are never shadowed."""
    rng = np.random.default_rng(19)
    n_sh = 0
    for _ in range(5):
        D = rng.uniform(2.0, 8.0)
        y0, z0 = rng.uniform(-1.5, 0.5), rng.uniform(-1.0, 0.3)
        y1, z1 = y0 + rng.uniform(0.3, 1.2), z0 + rng.uniform(0.3, 1.0)
        b = rng.uniform(0.4, 1.0) * rng.choice([-1.0, 1.0])
        tris = np.array(_rect(D, -80, 80, -80, 80) + _rect(D / 2, y0, y1, z0, z1), float)
        seg = np.array([0, 0, 1, 1], np.int32)
        s = O.Sensor(O.PINHOLE, 48, 36, math.radians(90), 0.1, 50.0)
        r = O.render(tris, seg, s, IDENT, lib=lib)
        rays = np.arange(48 * 36)
        sh = O.shadow(tris, s, IDENT, [0, b, 0], 1e-4, rays, r, lib=lib)
        for i in rays:
            _, d, _ = O.ray(s, IDENT, i // 48, i % 48, lib)
            P = d * (D / d[0])
            cy, cz = (P[1] + b) / 2, P[2] / 2  # midpoint of P and (0, b, 0)
            m = 1e-6 + 1e-4 * D
            inside = y0 + m < cy < y1 - m and z0 + m < cz < z1 - m
            outside = cy < y0 - m or cy > y1 + m or cz < z0 - m or cz > z1 + m
            if r["seg"][i] == 1:
                assert sh[i] == 0
            elif inside:
                assert sh[i] in (1, 2)
                n_sh += sh[i] == 1
            elif outside:
                assert sh[i] == 0, (i, cy, cz)
    assert n_sh > 20


def pin_shadow_zero_baseline_and_open_scene(lib):
    """A second sensor at the first one's position sees every hit (the segment is the primary ray
    reversed, and the hit is the nearest); with no geometry between, nothing is shadowed."""
    vs, ix, ps, sg, _, _ = _room_scene()
    sc_tris, sc_seg = O.world_triangles(vs, ix, ps, sg)
    s = O.Sensor(O.PINHOLE, 24, 18, math.radians(87), 0.2, 10.0)
    rng = np.random.default_rng(20)
    for _ in range(3):
        pose = np.concatenate([rng.uniform(-3, 3, 2), [rng.uniform(0.5, 3.5)], rng.normal(size=4)])
        r = O.render(sc_tris, sc_seg, s, pose, lib=lib)
        rays = np.arange(24 * 18)
        sh = O.shadow(sc_tris, s, pose, [0, 0, 0], 1e-4, rays, r, lib=lib)
        assert (sh != 1).all() and (sh == 2).mean() < 0.05
    wall = np.array(_rect(5.0, -50, 50, -50, 50), float)
    r = O.render(wall, np.array([0, 0], np.int32), s, IDENT, lib=lib)
    sh = O.shadow(wall, s, IDENT, [0, -0.3, 0.1], 1e-4, np.arange(24 * 18), r, lib=lib)
    assert (sh == 0).all()


def pin_shadow_linear_solve(lib):
    """Shadow verdicts against numpy.linalg.solve of P + s (o2 - P) = v0 + u e1 + w e2 on random scenes."""
    rng = np.random.default_rng(21)
    checked = 0
    for trial in range(10):
        F = int(rng.integers(2, 10))
        tris = rng.uniform(-4, 4, (F, 9))
        seg = np.arange(F, dtype=np.int32)
        s = O.Sensor(O.PINHOLE, 12, 9, math.radians(100), 0.05, 20.0)
        pose = np.concatenate([rng.uniform(-1, 1, 3), rng.normal(size=4)])
        base = rng.uniform(-2, 2, 3)
        r = O.render(tris, seg, s, pose, lib=lib)
        rays = np.arange(12 * 9)
        sh = O.shadow(tris, s, pose, base, 1e-4, rays, r, lib=lib)
        R = _rot_scipy(pose[3:])
        o2 = pose[:3] + R @ base
        for i in rays:
            if r["seg"][i] < 0 or sh[i] == 2:
                continue
            o, d, _ = O.ray(s, pose, i // 12, i % 12, lib)
            P = o + r["t_hit"][i] * d
            hit = False
            for tri in tris:
                v0, v1, v2 = tri[:3], tri[3:6], tri[6:]
                M = np.stack([o2 - P, v0 - v1, v0 - v2], 1)
                if abs(np.linalg.det(M)) < 1e-12:
                    continue
                t, u, w = np.linalg.solve(M, v0 - P)
                hit |= bool(u >= 0 and w >= 0 and u + w <= 1 and 1e-4 <= t <= 1)
            assert sh[i] == int(hit), (trial, i)
            checked += 1
    assert checked > 200


# ---------------------------------------------------------------- user projection model (ray table)
def pin_ray_table_reproduces_builtin_models(lib):
    """A table holding the camera's (1, a, b) rows renders exactly like the camera (depth), and one
    holding the LiDAR's unit beams exactly like the LiDAR (range)."""
    vs, ix, ps, sg, _, _ = _room_scene()
    tris, seg = O.world_triangles(vs, ix, ps, sg)
    rng = np.random.default_rng(22)
    pose = np.concatenate([[0.5, -0.3, 1.7], rng.normal(size=4)])
    cam = O.Sensor(O.PINHOLE, 20, 14, math.radians(87), 0.2, 10.0)
    f = 10.0 / math.tan(math.radians(87) / 2)
    cols, rows = np.meshgrid(np.arange(20) + 0.5, np.arange(14) + 0.5)
    table = np.stack([np.ones_like(cols), (10.0 - cols) / f, (7.0 - rows) / f], -1)
    tab = O.Sensor(O.RAY_TABLE, 20, 14, 0.0, 0.2, 10.0, dirs=table)
    a, b = O.render(tris, seg, cam, pose, lib=lib), O.render(tris, seg, tab, pose, lib=lib)
    assert np.allclose(a["v"], b["v"], rtol=1e-12, atol=1e-12) and np.array_equal(a["seg"], b["seg"])
    lid = O.Sensor(O.LIDAR, 32, 8, 2 * math.pi, 0.2, 10.0, -0.4, 0.4)
    R = _rot_scipy(pose[3:])
    beams = np.array([R.T @ O.ray(lid, pose, k, j, lib)[1] for k in range(8) for j in range(32)]).reshape(8, 32, 3)
    tab = O.Sensor(O.RAY_TABLE, 32, 8, 0.0, 0.2, 10.0, dirs=beams)
    a, b = O.render(tris, seg, lid, pose, lib=lib), O.render(tris, seg, tab, pose, lib=lib)
    assert np.allclose(a["v"], b["v"], rtol=1e-12, atol=1e-12) and np.array_equal(a["seg"], b["seg"])


def pin_ray_table_wall_units(lib):
    """Wall at x = D: a row g with g_x > 0 reports D / g_x (distance in units of |g|), whatever |g|."""
    rng = np.random.default_rng(23)
    D = 3.5
    wall = np.array(_rect(D, -80, 80, -80, 80), float)
    g = rng.normal(size=(6, 9, 3))
    g[..., 0] = np.abs(g[..., 0]) + 0.3
    g *= rng.uniform(0.2, 5.0, (6, 9, 1))
    tab = O.Sensor(O.RAY_TABLE, 9, 6, 0.0, 0.01, 1e4, dirs=g)
    r = O.render(wall, np.array([0, 0], np.int32), tab, IDENT, lib=lib)
    assert np.allclose(r["v"], (D / g[..., 0]).reshape(-1), rtol=1e-12)
    _, _, point = O.hit_channels(wall, tab, IDENT, np.arange(54), r["tri"], r["v"], lib=lib)
    assert np.allclose(point[:, 0], D, rtol=1e-12)


ALL_PINS = [
    pin_rotation_vs_scipy, pin_transform_vs_scipy, pin_transform_identity_exact,
    pin_camera_centre_and_corner, pin_camera_column_angles, pin_lidar_angles,
    pin_wall_depth_constant, pin_lidar_cylinder_facets, pin_icosphere_bounds, pin_hand_worked,
    pin_brute_force_linear_solve, pin_miss_exact, pin_translation_rotation_invariance,
    pin_degenerate_never_hits, pin_tie_break, pin_channels_wall, pin_channels_linear_solve,
    pin_channels_icosphere, pin_channels_miss_and_lidar_norm, pin_candidate_triangles,
    pin_shadow_plate_closed_form, pin_shadow_zero_baseline_and_open_scene, pin_shadow_linear_solve,
    pin_ray_table_reproduces_builtin_models, pin_ray_table_wall_units,
]


# ---------------------------------------------------------------- error bands (counting and acceptance)
# The oracle judges a float32 renderer with three stated error bands: each world vertex coordinate off by up
# to VERT_REL * cmax (cmax: the largest |coordinate| of the ray origin and the triangle, at least 1), the ray
# direction tilted by up to DIR_REL, and the intersection arithmetic moving the ray sideways by up to
# ARITH_REL * rmax (rmax: the farthest vertex) and its distance along the ray by as much. The pins below
# apply those perturbations to the exact geometry, intersect in FP64, and hold the oracle's bands, edge
# flags and counting reasons to what the perturbed rays actually do: every perturbed hit must fall inside
# the band (sound) and the band may be at most twice as wide as the largest perturbed deviation (tight).

def _one_ray(d):
    """A 1x1 ray-table sensor casting unit direction d (reported value = distance along the ray)."""
    d = np.asarray(d, float) / np.linalg.norm(d)
    return O.Sensor(O.RAY_TABLE, 1, 1, 0.0, 1e-9, 1e6, dirs=d.reshape(1, 1, 3))


def _frame(d):
    """Unit d and two unit vectors spanning the plane orthogonal to it."""
    d = np.asarray(d, float) / np.linalg.norm(d)
    a = np.array([1.0, 0, 0]) if abs(d[0]) < 0.9 else np.array([0, 1.0, 0])
    u = np.cross(d, a)
    u /= np.linalg.norm(u)
    return d, u, np.cross(d, u)


def _perturbed(tri, o, d, rng, n_random=400):
    """(t, barycentrics) of the ray's meet with the triangle's plane under the band perturbations: every
    combination of extreme signs along the plane normal's in-ray-plane direction, plus random extremes."""
    tri = np.asarray(tri, float).reshape(3, 3)
    cmax = max(1.0, np.abs(tri).max(), np.abs(o).max())
    vert = O.VERT_REL * cmax
    rmax = np.linalg.norm(tri - o, axis=1).max()
    ar = O.ARITH_REL * rmax
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    n /= np.linalg.norm(n)
    e = n - (n @ d) * d  # the sideways direction that moves the hit most
    e = e / np.linalg.norm(e) if np.linalg.norm(e) > 1e-12 else _frame(d)[1]
    cases = []
    for sv in (-1, 1):
        for st in (-1, 1):
            for ss in (-1, 1):
                for sa in (-1, 1):
                    cases.append((np.tile(sv * np.sign(n), (3, 1)), st * e, ss * e, sa))
    for _ in range(n_random):
        dv = rng.choice([-1.0, 1.0], size=(3, 3))
        r1, r2 = rng.normal(size=3), rng.normal(size=3)
        r1 -= (r1 @ d) * d
        r2 -= (r2 @ d) * d
        cases.append((dv, r1 / np.linalg.norm(r1), r2 / np.linalg.norm(r2), rng.choice([-1, 1])))
    out = []
    for dv, tilt, side, along in cases:
        T = tri + vert * dv
        dd = np.cos(O.DIR_REL) * d + np.sin(O.DIR_REL) * tilt
        oo = o + ar * side
        # o + t dd = T0 + b1 (T1 - T0) + b2 (T2 - T0)
        A = np.column_stack([dd, T[0] - T[1], T[0] - T[2]])
        t, b1, b2 = np.linalg.solve(A, T[0] - oo)
        out.append((t + along * ar, 1 - b1 - b2, b1, b2))
    return np.array(out)


def _tilted_triangle(o, d, D, theta, rng, size=2.0):
    """A large triangle whose plane meets the ray at distance D with incidence angle theta (|n.d| = cos)."""
    d, u, w = _frame(d)
    phi = rng.uniform(0, 2 * np.pi)
    a = np.cos(phi) * u + np.sin(phi) * w  # the tilt axis, orthogonal to the ray
    n = np.cos(theta) * d + np.sin(theta) * np.cross(a, d)
    b1 = a
    b2 = np.cross(n, b1)
    c = o + D * d
    return np.array([c + size * b1 - size * b2, c - size * b1 - size * b2, c + 1.3 * size * b2])


def pin_band_width_against_perturbations(lib):
    """Sound and tight t bands across incidences, near the origin (direction and arithmetic bands dominate)
    and 200 m from it (the vertex band dominates)."""
    rng = np.random.default_rng(31)
    for o in (np.array([0.3, -0.2, 0.1]), np.array([180.0, -140.0, 95.0])):
        for theta_deg in (0.0, 40.0, 70.0, 82.0, 87.0):
            d = _frame(rng.normal(size=3))[0]
            D = rng.uniform(2.0, 6.0)
            tri = _tilted_triangle(o, d, D, math.radians(theta_deg), rng)
            res = O.render(tri.reshape(1, 9), np.array([1], np.int32), _one_ray(d),
                           np.concatenate([o, [0, 0, 0, 1]]), lib=lib)[0]
            assert res["seg"] == 1 and res["n_cand"] == 1, (theta_deg, res)
            t0 = res["v"]
            pert = _perturbed(tri, o, d, rng)
            assert np.all(pert[:, 1:] > 0)  # every perturbed ray still meets the triangle inside
            lo, hi = res["cand_lo"][0], res["cand_hi"][0]
            dev = np.abs(pert[:, 0] - t0).max()
            assert lo <= pert[:, 0].min() + 1e-12 * t0 and pert[:, 0].max() <= hi + 1e-12 * t0, \
                (theta_deg, lo, hi, pert[:, 0].min(), pert[:, 0].max())
            assert (hi - lo) / 2 <= 2.0 * dev, (theta_deg, (hi - lo) / 2, dev)
            assert abs(res["hit_dev"] - max(t0 - lo, hi - t0)) <= 1e-12 * t0


def pin_silhouette_band_against_perturbations(lib):
    """A ray passing an edge at sideways distance s is flagged (and counted) when a band perturbation can
    carry it across the edge, and not once s is 1.6 times the largest such displacement."""
    rng = np.random.default_rng(32)
    o = np.array([0.2, 0.1, -0.3])
    d, u, w = _frame([1.0, 0.3, 0.2])
    D, a, h = 5.0, 0.03, 0.04
    # the edge v0-v1 runs along u at sideways offset s0 (along w) from the ray; v2 lies at s0 + h
    def tri_at(s0):
        c = o + D * d + (rng.uniform(-1, 1) * 0.002) * d
        return np.array([c + a * u + s0 * w, c - a * u + s0 * w, c + (s0 + h) * w])
    base = tri_at(0.0)
    pert = _perturbed(base, o, d, rng)
    s_flip = np.abs(pert[:, 3] * h).max()  # how far the perturbations move the ray across the edge
    assert s_flip > 0
    pose = np.concatenate([o, [0, 0, 0, 1]])
    for frac, inside in ((0.8, True), (0.8, False), (1.6, True), (1.6, False)):
        s0 = -frac * s_flip if inside else frac * s_flip
        res = O.render(tri_at(s0).reshape(1, 9), np.array([2], np.int32), _one_ray(d), pose, lib=lib)[0]
        sil = bool(res["flags"] & O.F_SILHOUETTE)
        counted = bool(res["flags"] & O.F_COUNTED)
        if frac < 1:
            assert sil and counted and (res["flags"] & O.F_MISS_OK), (frac, inside, res["flags"])
        else:
            assert not sil and not counted, (frac, inside, res["flags"], s_flip)
            assert res["seg"] == (2 if inside else -1)


def pin_grazing_and_coarse_reasons(lib):
    """Counted for incidence: when the direction band alone can move the hit by more than the relative
    tolerance (grazing), and when the vertex band alone exceeds the tolerance at normal incidence (coarse
    coordinates, far from the origin). Not counted when every band perturbation stays within the tolerance."""
    rng = np.random.default_rng(33)
    o = np.array([0.4, 0.7, -0.2])
    for theta_deg in (30.0, 60.0, 80.0, 86.0, 87.5, 88.5):
        d = _frame(rng.normal(size=3))[0]
        D = 3.0
        tri = _tilted_triangle(o, d, D, math.radians(theta_deg), rng)
        res = O.render(tri.reshape(1, 9), np.array([5], np.int32), _one_ray(d),
                       np.concatenate([o, [0, 0, 0, 1]]), lib=lib)[0]
        # deviation from the direction tilt alone, in the plane of the ray and the normal
        n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        n /= np.linalg.norm(n)
        e = n - (n @ d) * d
        e /= np.linalg.norm(e)
        tilt = [np.linalg.solve(np.column_stack([np.cos(O.DIR_REL) * d + s * np.sin(O.DIR_REL) * e,
                                                 tri[0] - tri[1], tri[0] - tri[2]]), tri[0] - o)[0]
                for s in (-1, 1)]
        dev_tilt = max(abs(t - res["v"]) for t in tilt)
        dev_all = np.abs(_perturbed(tri, o, d, rng)[:, 0] - res["v"]).max()
        graze = bool(res["flags"] & O.F_GRAZING)
        if dev_tilt > 1e-5 * res["v"] * 1.02:
            assert graze and (res["flags"] & O.F_COUNTED), (theta_deg, dev_tilt, res["flags"])
        if dev_all < O.tol(res["v"]):
            assert not (res["flags"] & O.F_COUNTED), (theta_deg, dev_all, res["flags"])
    # a wall 5 km from the origin seen head on from 3 m: its coordinates' float32 spacing alone exceeds the
    # tolerance; the same wall near the origin is judged by the tolerance
    for centre, coarse in ((np.array([5000.0, -3000.0, 2000.0]), True), (np.array([2.0, 1.0, 0.5]), False)):
        d = np.array([1.0, 0.0, 0.0])
        oc = centre - 3.0 * d + np.array([0.0, 1.1, -0.7])  # off the diagonal shared by the two triangles
        wall = np.array(_rect(centre[0], centre[1] - 5, centre[1] + 5, centre[2] - 5, centre[2] + 5), float)
        res = O.render(wall, np.array([0, 0], np.int32), _one_ray(d), np.concatenate([oc, [0, 0, 0, 1]]),
                       lib=lib)[0]
        dev_vert = O.VERT_REL * max(1.0, np.abs(wall).max(), np.abs(oc).max())  # a wall coordinate moved
        assert (dev_vert > O.tol(res["v"])) == coarse
        assert bool(res["flags"] & O.F_COARSE) == coarse and bool(res["flags"] & O.F_COUNTED) == coarse


ALL_PINS += [pin_band_width_against_perturbations, pin_silhouette_band_against_perturbations,
             pin_grazing_and_coarse_reasons]
