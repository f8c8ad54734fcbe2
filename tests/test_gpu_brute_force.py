"""The BVH render against a brute-force render on every ray of large scenes, bit for bit.

The brute-force kernel tests every BVH reference of a ray's environment with the render kernel's own ray
set-up and watertight triangle test, no tree. Box culling in the BVH walk is conservative and the nearest
hit is the minimum of (t, triangle id), which does not depend on the order of the tests, so every tree
(builder, node format, leaf size, reference splitting, refit) must give exactly the brute-force images.
This checks the trees on millions of rays at the workloads' own scales, where the FP64 oracle checks
samples (the oracle itself checks the brute-force images on a sample here too).
"""
import numpy as np
import pytest
import torch

import paper_2503_01471_gb300 as ags
from paper_2503_01471_gb300 import build as B
from paper_2503_01471_gb300 import scenes as S

from helpers import compare_env, describe_failures

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = ags.ags_context_create(0)
    yield c
    ags.ags_context_destroy(c)


def both(ctx, scene, spec, poses):
    E = poses.shape[0]
    p = torch.as_tensor(np.ascontiguousarray(poses, np.float32)).cuda()
    out = []
    for fn in (ags.ags_render, ags.ags_render_bruteforce):
        d = torch.full((E, spec.height, spec.width), -7.0, device="cuda")
        s = torch.full((E, spec.height, spec.width), -7, dtype=torch.int32, device="cuda")
        fn(ctx, scene, spec, p, d, s)
        ags.ags_stream_status(ctx)
        out.append((d.cpu().numpy(), s.cpu().numpy()))
    return out


def assert_same(out, tag):
    (d, s), (bd, bs) = out
    bad = (d.view(np.uint32) != bd.view(np.uint32)) | (s != bs)
    if bad.any():
        i = np.argwhere(bad)[:5]
        raise AssertionError(f"{tag}: {int(bad.sum())} of {bad.size} rays differ from brute force, e.g. "
                             + "; ".join(f"{tuple(j)} bvh ({d[tuple(j)]!r}, {s[tuple(j)]}) brute "
                                         f"({bd[tuple(j)]!r}, {bs[tuple(j)]})" for j in i))
    hits = float((s >= 0).mean())
    print(f"[brute] {tag}: {d.size} rays bit-identical, {hits:.1%} hits")
    return hits


def test_rooms_1024_envs_every_variant(ctx):
    """The 1024-room workload (every environment, 96x54 camera) under the builders, node formats, leaf
    sizes and splitting settings the benchmark and the tuner use."""
    batch, _, poses = S.obstacle_rooms(1024, steps=1)
    spec = S.pinhole(96, 54)
    for flags, tag in [(0, "default"), (ags.AGS_BVH_Q8, "8-bit nodes"), (ags.AGS_BVH_FP16, "16-bit nodes"),
                       (ags.AGS_BUILD_LBVH | ags.AGS_LEAF_SIZE(4), "Morton tree, leaves of 4"),
                       (ags.AGS_SPLIT_CELLS(64) | ags.AGS_LEAF_SIZE(1), "64 split cells, leaves of 1"),
                       (ags.AGS_BUILD_GREEDY_COLLAPSE, "greedy collapse"), (ags.AGS_LEAF_SIZE(4), "leaves of 4")]:
        scene = ags.ags_scene_build(ctx, batch, flags)
        try:
            assert assert_same(both(ctx, scene, spec, poses[0]), f"1024 rooms 96x54, {tag}") > 0.5
        finally:
            ags.ags_scene_destroy(scene)


def test_rooms_full_resolution_and_lidar(ctx):
    """The benchmark's 480x270 camera on 24 of the rooms, and a 512x64 LiDAR, with the oracle checking a
    sample of the brute-force images."""
    batch, spec, poses = S.obstacle_rooms(24, steps=1)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        out = both(ctx, scene, spec, poses[0])
        assert_same(out, "24 rooms 480x270")
        lid = S.lidar(512, 64)
        assert_same(both(ctx, scene, lid, poses[0]), "24 rooms, 512x64 LiDAR")
        d, s = out[1]
        rng = np.random.default_rng(40)
        for e in (0, 11, 23):
            rays = np.sort(rng.choice(spec.width * spec.height, 64, replace=False)).astype(np.int64)
            ok, _, res = compare_env(batch, e, spec, poses[0][e], d[e], s[e], rays)
            assert ok.all(), describe_failures(ok, res, d[e].reshape(-1)[rays], s[e].reshape(-1)[rays], rays)
    finally:
        ags.ags_scene_destroy(scene)


def test_refit_scene_after_motion(ctx):
    """After refits that move every object (rooms included), the refitted tree still finds every nearest
    hit."""
    batch, _, poses = S.obstacle_rooms(256, steps=1)
    spec = S.pinhole(96, 54)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        rng = np.random.default_rng(41)
        cur = batch.poses.copy()
        for step in range(2):
            cur[:, :3] += rng.normal(0, 0.3, (cur.shape[0], 3)).astype(np.float32)
            q = cur[:, 3:] + rng.normal(0, 0.2, (cur.shape[0], 4)).astype(np.float32)
            cur[:, 3:] = q / np.linalg.norm(q, axis=1, keepdims=True)
            ags.ags_scene_update_poses(ctx, scene, cur, ags.AGS_UPDATE_REFIT)
            assert_same(both(ctx, scene, spec, poses[0]), f"256 rooms 96x54 after refit {step + 1}")
    finally:
        ags.ags_scene_destroy(scene)


def test_lidar_forests(ctx):
    """Four full-size forests (about 650k triangles each) under the 64x512 LiDAR, with the splitting the
    tuner picks on this workload and without splitting."""
    batch, spec, poses = S.lidar_forests(4, steps=1)
    for flags, tag in [(ags.AGS_SPLIT_CELLS(64), "64 split cells"), (ags.AGS_SPLIT_CELLS(1), "no splitting"),
                       (ags.AGS_BVH_Q8 | ags.AGS_SPLIT_CELLS(48), "8-bit nodes, 48 cells")]:
        scene = ags.ags_scene_build(ctx, batch, flags)
        try:
            assert assert_same(both(ctx, scene, spec, poses[0]), f"4 forests 64x512, {tag}") > 0.2
        finally:
            ags.ags_scene_destroy(scene)


def test_empty_and_invalid(ctx):
    """Environments without triangles miss everywhere; a pose the method cannot use gives NaN, segment -1
    and the invalid-argument status in both renders; two-level scenes are refused."""
    tri = (np.array([[3, -3, -3], [3, 3, -3], [3, 0, 3]], np.float32), np.array([[0, 1, 2]], np.int32),
           S.IDENTITY_POSE, 7)
    batch = S.scene_from_lists([[], [tri], [tri, tri]])
    spec = S.pinhole(16, 12, 90.0, 0.1, 10.0)
    poses = np.tile(S.IDENTITY_POSE, (3, 1))
    scene = ags.ags_scene_build(ctx, batch)
    try:
        out = both(ctx, scene, spec, poses)
        assert_same(out, "empty and single-triangle envs")
        d, s = out[0]
        assert (s[0] == -1).all() and (s[1] >= 0).any()
        p = torch.as_tensor(poses).cuda()
        p[2, 3:] = 0.0
        for fn in (ags.ags_render, ags.ags_render_bruteforce):
            d = torch.zeros((3, 12, 16), device="cuda")
            s = torch.zeros((3, 12, 16), dtype=torch.int32, device="cuda")
            fn(ctx, scene, spec, p, d, s)
            with pytest.raises(ags.AgsError) as ei:
                ags.ags_stream_status(ctx)
            assert ei.value.status == ags.AGS_ERR_INVALID_ARG
            assert torch.isnan(d[2]).all() and (s[2] == -1).all() and not torch.isnan(d[:2]).any()
    finally:
        ags.ags_scene_destroy(scene)
    inst = ags.ags_scene_build(ctx, S.obstacle_rooms(2, steps=1)[0], ags.AGS_BUILD_INSTANCED)
    try:
        p = torch.as_tensor(np.tile(S.IDENTITY_POSE, (2, 1))).cuda()
        d = torch.empty((2, 12, 16), device="cuda")
        s = torch.empty((2, 12, 16), dtype=torch.int32, device="cuda")
        with pytest.raises(ags.AgsError):
            ags.ags_render_bruteforce(ctx, inst, spec, p, d, s)
    finally:
        ags.ags_scene_destroy(inst)


def same_or_oracle(out, batch, spec, poses, tag, max_frac=1e-4):
    """Bit-identical, except on at most max_frac of the rays, where the BVH render must then agree with the
    FP64 oracle. A float32 triangle test on a ray within ~1e-7 rad of a sliver's plane can accept the sliver
    at a t outside the sliver's box along the ray (its barycentric weights are rounding noise, so t is any
    depth of its vertices); whether such a hit is found then depends on the order of the tests, and the
    FP64 oracle places it elsewhere or nowhere."""
    (d, s), (bd, bs) = out
    bad = (d.view(np.uint32) != bd.view(np.uint32)) | (s != bs)
    n_bad = int(bad.sum())
    assert n_bad <= max(1, max_frac * bad.size), f"{tag}: {n_bad} of {bad.size} rays differ"
    W = spec.width
    for e, r, c in np.argwhere(bad):
        ray = np.array([r * W + c], np.int64)
        ok, _, res = compare_env(batch, int(e), spec, poses[e], d[e], s[e], ray)
        assert ok.all(), f"{tag}: env {e}: " + describe_failures(ok, res, d[e].reshape(-1)[ray], s[e].reshape(-1)[ray], ray)
    print(f"[brute] {tag}: {bad.size - n_bad} of {bad.size} rays bit-identical, {n_bad} differing "
          f"(the BVH render's value checked against the oracle)")


def _soup(rng, n, scale, offset):
    """n random triangles: mixed sizes, some degenerate (repeated or collinear vertices), some duplicated
    exactly (equal t: the smaller triangle id must win) and some axis-aligned (flat boxes)."""
    c = offset + rng.uniform(-scale, scale, (n, 1, 3))
    size = scale * 10.0 ** rng.uniform(-3, -0.3, (n, 1, 1))
    v = (c + size * rng.normal(size=(n, 3, 3))).astype(np.float32)
    k = rng.random(n)
    v[k < 0.05, 2] = v[k < 0.05, 1]                                     # repeated vertex
    col = (k >= 0.05) & (k < 0.1)
    v[col, 2] = (2.0 * v[col, 1] - v[col, 0]).astype(np.float32)       # (nearly) collinear
    flat = (k >= 0.1) & (k < 0.3)
    axis = rng.integers(0, 3, int(flat.sum()))
    v[np.where(flat)[0], :, axis] = v[np.where(flat)[0], 0:1, axis]    # axis-aligned plane
    dup = rng.random(n) < 0.05
    v[dup] = v[np.roll(np.arange(n), 1)][dup]                          # exact copies of a neighbour
    return v.reshape(-1, 3), np.arange(3 * n, dtype=np.int32).reshape(-1, 3)


@pytest.mark.parametrize("offset", [0.0, 1000.0, -5000.0])
def test_random_soups_far_from_the_origin(ctx, offset):
    """Random triangle soups (degenerate, duplicated and axis-aligned triangles) at growing distances from
    the origin, seen by cameras with axis-aligned and random poses and by a LiDAR: every ray bit-identical
    to brute force under three builds (but for rare grazing slivers, see same_or_oracle), and every ray
    within the tolerance of the FP64 oracle."""
    rng = np.random.default_rng(int(abs(offset)) + 50)
    o = np.array([offset, -0.5 * offset, 0.25 * offset])
    envs = []
    for e in range(48):
        objs = []
        for j in range(int(rng.integers(1, 5))):
            v, f = _soup(rng, int(rng.integers(50, 800)), 8.0, o)
            objs.append((v, f, S.IDENTITY_POSE, int(rng.integers(0, 5))))
        envs.append(objs)
    batch = S.scene_from_lists(envs)
    poses = np.zeros((48, 7), np.float32)
    poses[:, :3] = o + rng.uniform(-6, 6, (48, 3))
    poses[:, 3:] = S.random_unit_quat(rng, 48)
    poses[::4, 3:] = S.IDENTITY_POSE[3:]                                # exact axis directions
    poses[1::8, 3:] = np.array([0.0, 0.0, np.sqrt(0.5), np.sqrt(0.5)], np.float32)  # 90 degrees about z
    for spec in (S.pinhole(64, 48, max_range=30.0), S.lidar(128, 16, max_range=40.0)):
        outs = []
        for flags in (0, ags.AGS_BUILD_LBVH | ags.AGS_LEAF_SIZE(4), ags.AGS_BVH_Q8 | ags.AGS_SPLIT_CELLS(32)):
            scene = ags.ags_scene_build(ctx, batch, flags)
            try:
                out = both(ctx, scene, spec, poses)
                tag = f"soups at {offset:g} m, {'camera' if spec.type == 0 else 'LiDAR'}, flags {flags}"
                same_or_oracle(out, batch, spec, poses, tag)
                outs.append(out[0])
            finally:
                ags.ags_scene_destroy(scene)
        for d, s in outs[1:]:
            same_or_oracle([(d, s), outs[0]], batch, spec, poses, f"soups at {offset:g} m, builds")
        d, s = outs[0]
        n = counted = 0
        for e in range(batch.n_envs):  # every ray against the oracle
            ok, cnt, res = compare_env(batch, e, spec, poses[e], d[e], s[e])
            rays = np.arange(spec.width * spec.height)
            assert ok.all(), f"env {e}: " + describe_failures(ok, res, d[e].reshape(-1), s[e].reshape(-1), rays)
            n += ok.size
            counted += int(cnt.sum())
        print(f"[parity] soups at {offset:g} m, {'camera' if spec.type == 0 else 'LiDAR'}: {n} rays, {counted} counted")
