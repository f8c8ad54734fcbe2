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
