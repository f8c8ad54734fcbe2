"""CUDA renderer vs the FP64 oracle, element by element, through the C ABI.

Tolerance (from the benchmark spec of the method's accuracy): |depth - oracle|
<= 1e-5 * depth + 1e-6 m on every ray whose outcome is unique; misses exactly
max_range with segment -1; segment IDs exact. Rays where several outcomes are
correct within the float32 error bands (edges, near ties, range limits) must
match one of the outcomes the oracle lists for them, and are counted.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2503_01471_gb300 as ags
from paper_2503_01471_gb300 import build as B
from paper_2503_01471_gb300 import scenes as S

from helpers import (check_channels, check_channels_sensor, compare_env, describe_channel_failures, describe_failures,
                     oracle_env, oracle_sensor)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = ags.ags_context_create(0)
    yield c
    ags.ags_context_destroy(c)


def render(ctx, scene, spec, poses):
    E = poses.shape[0]
    p = torch.as_tensor(np.ascontiguousarray(poses, np.float32)).cuda()
    depth = torch.empty((E, spec.height, spec.width), dtype=torch.float32, device="cuda")
    seg = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device="cuda")
    ags.ags_render(ctx, scene, spec, p, depth, seg)
    ags.ags_stream_status(ctx)
    return depth.cpu().numpy(), seg.cpu().numpy()


STATS = {}


def check_all(batch, spec, poses, depth, seg, envs=None, rays=None, tag=None, report=True):
    """Every listed ray acceptable (oracle.check: uncounted rays within 1e-5*d+1e-6 of the exact FP64 value
    with the exact segment; counted rays one of their listed outcomes); returns (rays, counted). Records, per
    tag, the counted rays by reason."""
    envs = range(batch.n_envs) if envs is None else envs
    n_cnt = n = 0
    by_reason = np.zeros(4, np.int64)  # several outcomes, grazing, coarse, rays with a band wider than tol
    for e in envs:
        ok, counted, res = compare_env(batch, e, spec, poses[e], depth[e], seg[e], rays)
        rr = np.arange(spec.width * spec.height) if rays is None else rays
        assert ok.all(), f"env {e}: {int((~ok).sum())} rays off\n" + describe_failures(
            ok, res, depth[e].reshape(-1)[rr], seg[e].reshape(-1)[rr], rr)
        f = res["flags"]
        assert np.all((f[counted] & O.F_REASONS) != 0)  # every counted ray has a stated reason
        n += ok.size
        n_cnt += int(counted.sum())
        several = (f & (O.F_SILHOUETTE | O.F_NEAR_TIE | O.F_RANGE_EDGE)) != 0
        by_reason += [int((counted & several).sum()), int(((f & O.F_GRAZING) != 0).sum()),
                      int(((f & O.F_COARSE) != 0).sum()), int((((f & O.F_WIDE) != 0) & ~counted).sum())]
    if tag:
        st = STATS.setdefault(tag, np.zeros(6, np.int64))
        st += [n, n_cnt, *by_reason]
        if report:
            print(f"[parity] {tag}: {st[0]} rays, {st[1]} counted ({st[2]} with several outcomes, {st[3]} grazing, "
                  f"{st[4]} coarse); every other ray within 1e-5*d+1e-6 of the FP64 value with the exact segment "
                  f"({st[5]} of them with float32 bands wider than that)")
    return n, n_cnt


# ---------------------------------------------------------------- a1
def test_transform_within_one_ulp(ctx):
    rng = np.random.default_rng(5)
    envs = []
    for e in range(3):
        objs = []
        for k in range(20):
            v = rng.uniform(-3, 3, (30, 3)).astype(np.float32)
            f = rng.integers(0, 30, (10, 3)).astype(np.int32)
            q = rng.normal(size=4) * rng.uniform(0.2, 3.0)  # non-unit on purpose
            p = rng.uniform(-20, 20, 3)
            objs.append((v, f, np.concatenate([p, q]).astype(np.float32), k))
        objs.append((rng.uniform(-9, 9, (5, 3)).astype(np.float32), np.array([[0, 1, 2], [2, 3, 4]], np.int32),
                     S.IDENTITY_POSE, 99))
        envs.append(objs)
    batch = S.scene_from_lists(envs)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        for e in range(batch.n_envs):
            gpu, gseg = ags.ags_scene_get_world_triangles(scene, e)
            ref, rseg = oracle_env(batch, e)
            assert np.array_equal(gseg, rseg)
            ulp = np.spacing(np.maximum(np.abs(ref), 1.0).astype(np.float32)).astype(np.float64)
            err = np.abs(gpu.astype(np.float64) - ref) / ulp
            assert err.max() <= 1.0, err.max()
            # identity pose: bit-exact
            assert np.array_equal(gpu[-2:], ref[-2:].astype(np.float32))
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- tiny room: every ray
def test_tiny_room_all_rays(ctx):
    batch, spec, poses = S.tiny_room()
    scene = ags.ags_scene_build(ctx, batch)
    try:
        n = cnt = 0
        for k in range(poses.shape[0]):
            d, s = render(ctx, scene, spec, poses[k:k + 1])
            a, b = check_all(batch, spec, poses[k:k + 1], d, s, tag="tiny room 64x48")
            n += a
            cnt += b
        assert n == 16 * 64 * 48
        print(f"tiny room: {n} rays, {cnt} counted")
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- obstacle rooms: every ray, ragged tiles
@pytest.mark.parametrize("W,H", [(96, 72), (13, 7), (1, 1)])
def test_obstacle_rooms_all_rays(ctx, W, H):
    batch, spec, poses = S.obstacle_rooms(4, steps=2, width=W, height=H)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        for step in range(2):
            d, s = render(ctx, scene, spec, poses[step])
            check_all(batch, spec, poses[step], d, s, tag=f"obstacle rooms {W}x{H}")
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- LiDAR forest
def test_lidar_forest_all_rays(ctx):
    batch, spec, poses = S.lidar_forests(2, steps=1, trees=(6, 10), tris=(2000, 3000))
    spec.width = 256
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d, s = render(ctx, scene, spec, poses[0])
        check_all(batch, spec, poses[0], d, s, tag="LiDAR forest 64x256")
        hit = (s >= 0).mean()
        assert hit > 0.3
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- full size, sampled
def test_full_size_1024_envs_sampled(ctx):
    """1024 rooms x 270x480 in the launch configuration the benchmark times; oracle on samples."""
    batch, spec, poses = S.obstacle_rooms(1024, steps=1)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d, s = render(ctx, scene, spec, poses[0])
        assert np.isfinite(d).all()
        rng = np.random.default_rng(99)
        n_pix = spec.width * spec.height
        total = cnt = 0
        for e in range(batch.n_envs):
            k = 256 if e in (0, 511, 1023) else 8
            rays = np.sort(rng.choice(n_pix, k, replace=False)).astype(np.int64)
            a, b = check_all(batch, spec, poses[0], d, s, envs=[e], rays=rays,
                             tag="1024 rooms 270x480 (sampled)", report=e == batch.n_envs - 1)
            total += a
            cnt += b
        # properties that hold for every ray
        assert (d[s == -1] == np.float32(spec.max_range)).all()
        assert ((d >= np.float32(spec.min_range)) & (d <= np.float32(spec.max_range))).all()
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- edge cases
def test_empty_and_single_triangle_envs(ctx):
    tri = (np.array([[3, -3, -3], [3, 3, -3], [3, 0, 3]], np.float32), np.array([[0, 1, 2]], np.int32),
           S.IDENTITY_POSE, 7)
    batch = S.scene_from_lists([[], [tri], [tri, tri]])
    spec = S.pinhole(3, 3, 90.0, 0.1, 10.0)
    poses = np.tile(S.IDENTITY_POSE, (3, 1))
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d, s = render(ctx, scene, spec, poses)
        assert (s[0] == -1).all() and (d[0] == np.float32(10.0)).all()
        want = np.array([[-1, 7, -1], [-1, 7, -1], [7, 7, 7]])
        assert np.array_equal(s[1], want) and np.array_equal(s[2], want)
        assert np.allclose(d[1][want == 7], 3.0, rtol=1e-6)
        check_all(batch, spec, poses, d, s, envs=[1, 2])
        t, n, b = ags.ags_scene_stats(scene, 0)
        assert (t, n, b) == (0, 0, 0)
    finally:
        ags.ags_scene_destroy(scene)


def test_near_modes_and_host_path(ctx):
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=40, height=30)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        for mode, mn in ((ags.AGS_NEAR_CLAMP, 1.5), (ags.AGS_NEAR_INVALID, 1.5)):
            spec.near_mode, spec.min_range = mode, mn
            d, s = render(ctx, scene, spec, poses[0])
            check_all(batch, spec, poses[0], d, s)
            hd, hs = ags.ags_render_host(ctx, scene, spec, np.ascontiguousarray(poses[0]))
            assert np.array_equal(hd, d) and np.array_equal(hs, s)
    finally:
        ags.ags_scene_destroy(scene)


def test_subset_render_matches_full(ctx):
    batch, spec, poses = S.obstacle_rooms(6, steps=1, width=32, height=24)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d, s = render(ctx, scene, spec, poses[0])
        ids = torch.tensor([4, 1, 1, 5], dtype=torch.int32, device="cuda")
        p = torch.as_tensor(poses[0][[4, 1, 1, 5]]).cuda()
        dd = torch.empty((4, 24, 32), device="cuda")
        ss = torch.empty((4, 24, 32), dtype=torch.int32, device="cuda")
        ags.ags_render_envs(ctx, scene, spec, ids, p, dd, ss)
        ags.ags_stream_status(ctx)
        assert np.array_equal(dd.cpu().numpy(), d[[4, 1, 1, 5]])
        assert np.array_equal(ss.cpu().numpy(), s[[4, 1, 1, 5]])
        rays, nodes, tris = ags.ags_render_count(ctx, scene, spec, torch.as_tensor(poses[0]).cuda())
        assert rays == 6 * 24 * 32 and nodes >= rays and tris > 0
    finally:
        ags.ags_scene_destroy(scene)


def test_deterministic_repeat(ctx):
    batch, spec, poses = S.obstacle_rooms(8, steps=1, width=64, height=48)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        a = render(ctx, scene, spec, poses[0])
        b = render(ctx, scene, spec, poses[0])
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        scene2 = ags.ags_scene_build(ctx, batch)
        c = render(ctx, scene2, spec, poses[0])
        ags.ags_scene_destroy(scene2)
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
    finally:
        ags.ags_scene_destroy(scene)


def test_host_validation_errors(ctx):
    v = np.zeros((3, 3), np.float32)
    bad_idx = S.scene_from_lists([[(v, np.array([[0, 1, 3]], np.int32), S.IDENTITY_POSE, 0)]])
    with pytest.raises(ags.AgsError, match="out of range"):
        ags.ags_scene_build(ctx, bad_idx)
    nan_pose = S.IDENTITY_POSE.copy()
    nan_pose[0] = np.nan
    with pytest.raises(ags.AgsError, match="non-finite pose"):
        ags.ags_scene_build(ctx, S.scene_from_lists([[(v, np.array([[0, 1, 2]], np.int32), nan_pose, 0)]]))
    zq = np.zeros(7, np.float32)
    with pytest.raises(ags.AgsError, match="zero length"):
        ags.ags_scene_build(ctx, S.scene_from_lists([[(v, np.array([[0, 1, 2]], np.int32), zq, 0)]]))
    with pytest.raises(ags.AgsError, match="segment_id"):
        ags.ags_scene_build(ctx, S.scene_from_lists([[(v, np.array([[0, 1, 2]], np.int32), S.IDENTITY_POSE, -3)]]))
    batch, spec, poses = S.obstacle_rooms(1, steps=1, width=8, height=8)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        p = torch.as_tensor(poses[0]).cuda()
        out = torch.empty((1, 8, 8), device="cuda")
        seg = torch.empty((1, 8, 8), dtype=torch.int32, device="cuda")
        for field, val in (("width", 0), ("max_range", 0.1), ("hfov", 4.0), ("type", 7)):
            bad = S.pinhole(8, 8)
            setattr(bad, field, val)
            with pytest.raises(ags.AgsError) as ei:
                ags.ags_render(ctx, scene, bad, p, out, seg)
            assert ei.value.status == ags.AGS_ERR_INVALID_ARG
        # buffers too small, of the wrong type or on the host are refused before anything is launched
        spec8 = S.pinhole(8, 8)
        for args in ((p[:, :6].contiguous(), out, seg), (p, out[:, :7].contiguous(), seg),
                     (p, out, seg.float()), (p, out.cpu(), seg)):
            with pytest.raises(ValueError):
                ags.ags_render(ctx, scene, spec8, *args)
        with pytest.raises(ValueError):
            ags.ags_render_ex(ctx, scene, spec8, p, out, seg, normal=torch.empty((1, 8, 8, 2), device="cuda"))
        assert ags.ags_stream_status(ctx) == ags.AGS_OK
    finally:
        ags.ags_scene_destroy(scene)


def test_device_limits_report_status_without_faulting(ctx):
    """A tiny traversal cap and an unusable device pose end in an error status, not a fault."""
    batch, spec, poses = S.obstacle_rooms(2, steps=1, width=16, height=12)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        ags.ags_context_set_traversal_cap(ctx, 1)
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((2, 12, 16), device="cuda")
        s = torch.empty((2, 12, 16), dtype=torch.int32, device="cuda")
        ags.ags_render(ctx, scene, spec, p, d, s)
        with pytest.raises(ags.AgsError) as ei:
            ags.ags_stream_status(ctx)
        assert ei.value.status == ags.AGS_ERR_TRAVERSAL_LIMIT
        assert torch.isnan(d).any()
        ags.ags_context_set_traversal_cap(ctx, 1 << 20)
        # context still usable; a zero quaternion is reported as invalid input
        bad = p.clone()
        bad[1, 3:] = 0.0
        ags.ags_render(ctx, scene, spec, bad, d, s)
        with pytest.raises(ags.AgsError) as ei:
            ags.ags_stream_status(ctx)
        assert ei.value.status == ags.AGS_ERR_INVALID_ARG
        assert torch.isnan(d[1]).all() and (s[1] == -1).all() and not torch.isnan(d[0]).any()
        ags.ags_render(ctx, scene, spec, p, d, s)
        assert ags.ags_stream_status(ctx) == ags.AGS_OK
        check_all(batch, spec, poses[0], d.cpu().numpy(), s.cpu().numpy())
    finally:
        ags.ags_context_set_traversal_cap(ctx, 1 << 20)
        ags.ags_scene_destroy(scene)


def test_bit_exact_across_bvh_variants(ctx):
    """Culling is conservative and the triangle test and tie-break do not depend on the tree, so every
    BVH variant gives bit-identical depth and segments."""
    batch, spec, poses = S.obstacle_rooms(6, steps=1, width=120, height=90)
    outs = []
    variants = [ags.AGS_LEAF_SIZE(n) for n in (1, 2, 3, 4)]
    variants += [ags.AGS_SPLIT_CELLS(1), ags.AGS_SPLIT_CELLS(64) | ags.AGS_LEAF_SIZE(2), ags.AGS_SPLIT_CELLS(4)]
    variants += [ags.AGS_BVH_FP16, ags.AGS_BVH_Q8, ags.AGS_BVH_Q8 | ags.AGS_LEAF_SIZE(4) | ags.AGS_SPLIT_CELLS(1),
                 ags.AGS_BVH_FP16 | ags.AGS_LEAF_SIZE(1)]
    # the Morton radix tree instead of clustering, alone and with the other options
    variants += [ags.AGS_BUILD_LBVH, ags.AGS_BUILD_LBVH | ags.AGS_LEAF_SIZE(4) | ags.AGS_SPLIT_CELLS(1),
                 ags.AGS_BUILD_LBVH | ags.AGS_BVH_Q8]
    # the greedy collapse instead of the least-cost slots
    variants += [ags.AGS_BUILD_GREEDY_COLLAPSE, ags.AGS_BUILD_GREEDY_COLLAPSE | ags.AGS_LEAF_SIZE(4),
                 ags.AGS_LEAF_SIZE(4) | ags.AGS_BVH_FP16]
    # wider clustering searches
    variants += [ags.AGS_CLUSTER_RADIUS(32), ags.AGS_CLUSTER_RADIUS(64) | ags.AGS_SPLIT_CELLS(64),
                 ags.AGS_CLUSTER_RADIUS(128) | ags.AGS_BVH_Q8]
    for flags in variants:
        scene = ags.ags_scene_build(ctx, batch, flags)
        try:
            outs.append(render(ctx, scene, spec, poses[0]))
        finally:
            ags.ags_scene_destroy(scene)
    for d, s in outs[1:]:
        assert np.array_equal(d, outs[0][0]) and np.array_equal(s, outs[0][1])
    check_all(batch, spec, poses[0], outs[0][0], outs[0][1], tag="BVH variants 120x90")


def test_reference_splitting_keeps_results_and_adds_references(ctx):
    """Large triangles (the room's walls, a forest's ground) get several BVH references; the scene's
    triangles and every ray's result stay the same."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=64, height=48)
    off = ags.ags_scene_build(ctx, batch, ags.AGS_SPLIT_CELLS(1))
    on = ags.ags_scene_build(ctx, batch)
    try:
        t0, n0, b0 = ags.ags_scene_stats(off)
        t1, n1, b1 = ags.ags_scene_stats(on)
        assert t0 == t1 == int(batch.env_tri_counts().sum())
        assert b1 > b0  # more references, each a 48-byte triangle copy
        a = render(ctx, off, spec, poses[0])
        b = render(ctx, on, spec, poses[0])
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        for e in range(3):
            assert np.array_equal(ags.ags_scene_get_world_triangles(off, e)[0],
                                  ags.ags_scene_get_world_triangles(on, e)[0])
    finally:
        ags.ags_scene_destroy(off)
        ags.ags_scene_destroy(on)


def test_launch_shapes_and_autotune_keep_results(ctx):
    """Every launch shape (tile, rays per lane, grid) renders the same bits; the autotuner's pick is
    remembered for the scene and sensor shape."""
    batch, spec, poses = S.obstacle_rooms(5, steps=1, width=70, height=45)  # ragged for every tile shape
    scene = ags.ags_scene_build(ctx, batch)
    try:
        ref = render(ctx, scene, spec, poses[0])
        for w, rpl, b in [(8, 1, 0), (4, 1, 0), (8, 2, 1), (16, 2, 0), (16, 4, 2), (16, 1, 0), (32, 1, 3)]:
            ags.ags_set_launch_config(ctx, scene, spec, w, rpl, b)
            cfg = ags.ags_get_launch_config(ctx, scene, spec)
            assert cfg["tile_w"] == w and cfg["rays_per_lane"] == rpl and cfg["blocks_per_sm"] == b
            out = render(ctx, scene, spec, poses[0])
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), (w, rpl, b)
            # a subset of the environments, in another order, through the same launch shape
            ids = torch.tensor([3, 0, 4], dtype=torch.int32, device="cuda")
            p = torch.as_tensor(poses[0][[3, 0, 4]]).cuda()
            d = torch.empty((3, 45, 70), device="cuda")
            sg = torch.empty((3, 45, 70), dtype=torch.int32, device="cuda")
            ags.ags_render_envs(ctx, scene, spec, ids, p, d, sg)
            ags.ags_stream_status(ctx)
            assert np.array_equal(d.cpu().numpy(), ref[0][[3, 0, 4]]) and np.array_equal(sg.cpu().numpy(),
                                                                                        ref[1][[3, 0, 4]])
        for bad in [(3, 1, 0), (8, 3, 0), (64, 1, 0), (32, 2, 0), (8, 1, 10_000), (8, 1, -1)]:
            with pytest.raises(ags.AgsError):
                ags.ags_set_launch_config(ctx, scene, spec, *bad)
        ags.ags_set_launch_config(ctx, scene, spec, None)
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((5, 45, 70), device="cuda")
        s = torch.empty((5, 45, 70), dtype=torch.int32, device="cuda")
        best = ags.ags_autotune(ctx, scene, spec, p, d, s, 1)
        assert best.ms > 0
        assert ags.ags_get_launch_config(ctx, scene, spec) == best.as_dict()
        out = render(ctx, scene, spec, poses[0])
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        check_all(batch, spec, poses[0], out[0], out[1], tag="launch shapes 70x45")
    finally:
        ags.ags_scene_destroy(scene)


@pytest.mark.parametrize("fmt", ["fp16", "q8"])
def test_compressed_nodes_bit_exact_on_lidar_forest_and_launch_shapes(ctx, fmt):
    """Compressed child bounds are rounded outward: the LiDAR forest (large ground triangles, long rays)
    renders the same bits as with float32 nodes, under every launch shape, and matches the oracle."""
    flag = ags.AGS_BVH_FP16 if fmt == "fp16" else ags.AGS_BVH_Q8
    batch, spec, poses = S.lidar_forests(2, steps=1, trees=(6, 10), tris=(2000, 3000))
    spec.width = 128
    ref_scene = ags.ags_scene_build(ctx, batch)
    scene = ags.ags_scene_build(ctx, batch, flag)
    try:
        assert ags.ags_scene_node_bytes(scene) == (128 if fmt == "fp16" else 80)
        ref = render(ctx, ref_scene, spec, poses[0])
        for w, rpl in [(8, 1), (4, 1), (8, 2), (16, 2), (16, 4), (16, 1), (32, 1)]:
            ags.ags_set_launch_config(ctx, scene, spec, w, rpl, 0)
            out = render(ctx, scene, spec, poses[0])
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), (w, rpl)
        check_all(batch, spec, poses[0], ref[0], ref[1], tag=f"LiDAR forest 64x128 ({fmt} nodes)")
    finally:
        ags.ags_scene_destroy(scene)
        ags.ags_scene_destroy(ref_scene)


@pytest.mark.parametrize("fmt", ["fp32", "fp16", "q8"])
def test_short_stack_retries_give_the_full_stack_results(ctx, fmt):
    """A 16- or 32-entry stack hands every ray that outgrows it to the full-stack retry pass: images equal the
    full stack's bit for bit (LiDAR forests, whose long beams do outgrow 16 entries, and rooms), also for an
    env subset and a captured step graph. With no room in the retry list the outgrown rays report NaN and the
    status says so, which shows the retry pass is what renders them."""
    flag = {"fp32": 0, "fp16": ags.AGS_BVH_FP16, "q8": ags.AGS_BVH_Q8}[fmt]
    batch, spec, poses = S.lidar_forests(2, steps=1, trees=(180, 200))  # dense: some beams need > 16 entries
    spec.width = 256
    scene = ags.ags_scene_build(ctx, batch, flag | ags.AGS_SPLIT_CELLS(64))
    try:
        ref = render(ctx, scene, spec, poses[0])
        for depth in (16, 32, 64):
            ags.ags_set_launch_config(ctx, scene, spec, 8, 1, 0, depth)
            assert ags.ags_get_launch_config(ctx, scene, spec)["stack_depth"] == depth
            out = render(ctx, scene, spec, poses[0])
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), depth
        ags.ags_set_launch_config(ctx, scene, spec, 8, 1, 0, 16)
        ids = torch.tensor([1], dtype=torch.int32, device="cuda")
        p = torch.as_tensor(poses[0][[1]]).cuda()
        d = torch.empty((1, spec.height, spec.width), device="cuda")
        sg = torch.empty((1, spec.height, spec.width), dtype=torch.int32, device="cuda")
        ags.ags_render_envs(ctx, scene, spec, ids, p, d, sg)
        ags.ags_stream_status(ctx)
        assert np.array_equal(d.cpu().numpy(), ref[0][[1]]) and np.array_equal(sg.cpu().numpy(), ref[1][[1]])
        gp = torch.as_tensor(poses[0]).cuda()
        gd = torch.empty((2, spec.height, spec.width), device="cuda")
        gs = torch.empty((2, spec.height, spec.width), dtype=torch.int32, device="cuda")
        g = ags.ags_render_graph_create(ctx, scene, spec, gp, gd, gs)
        try:
            gd.fill_(-1.0)
            ags.ags_render_graph_launch(g)
            ags.ags_stream_status(ctx)
            assert np.array_equal(gd.cpu().numpy(), ref[0]) and np.array_equal(gs.cpu().numpy(), ref[1])
        finally:
            ags.ags_render_graph_destroy(g)
        ags.ags_context_set_retry_capacity(ctx, 0)
        try:
            p2 = torch.as_tensor(poses[0]).cuda()
            d2 = torch.empty((2, spec.height, spec.width), device="cuda")
            s2 = torch.empty((2, spec.height, spec.width), dtype=torch.int32, device="cuda")
            ags.ags_render(ctx, scene, spec, p2, d2, s2)
            with pytest.raises(ags.AgsError) as ei:
                ags.ags_stream_status(ctx)
            assert ei.value.status == ags.AGS_ERR_TRAVERSAL_LIMIT
            lost = torch.isnan(d2).cpu().numpy()
            assert lost.any() and not lost.all()
            keep = ~lost
            assert np.array_equal(d2.cpu().numpy()[keep], ref[0][keep])
        finally:
            ags.ags_context_set_retry_capacity(ctx, 1 << 20)
        for bad in ((4, 1, 0, 16), (8, 1, 0, 8), (8, 1, 0, 48)):
            with pytest.raises(ags.AgsError):
                ags.ags_set_launch_config(ctx, scene, spec, *bad)
    finally:
        ags.ags_scene_destroy(scene)
    # rooms: the short stacks rarely run out; same images
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=70, height=45)
    scene = ags.ags_scene_build(ctx, batch, flag)
    try:
        ref = render(ctx, scene, spec, poses[0])
        for depth in (16, 32):
            ags.ags_set_launch_config(ctx, scene, spec, 8, 1, 0, depth)
            out = render(ctx, scene, spec, poses[0])
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), depth
    finally:
        ags.ags_scene_destroy(scene)


def test_update_poses_refit_and_rebuild_match_a_fresh_build(ctx):
    """Moving the obstacles by refit or by rebuild gives exactly the images of a scene built with the new
    poses (the traversal is exact, so the tree shape cannot change a result), and they match the oracle."""
    batch, spec, poses = S.obstacle_rooms(4, steps=1, width=64, height=48)
    rng = np.random.default_rng(21)
    new = batch.poses.copy()
    movable = np.ones(new.shape[0], bool)
    movable[batch.env_sub[:-1]] = False  # the rooms stay put
    new[movable, :3] += rng.normal(0, 0.5, (movable.sum(), 3)).astype(np.float32)
    q = rng.normal(size=(movable.sum(), 4))
    new[movable, 3:] = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                         batch.env_sub, new)
    fresh = ags.ags_scene_build(ctx, moved)
    refit = ags.ags_scene_build(ctx, batch)
    rebuilt = ags.ags_scene_build(ctx, batch, ags.AGS_BVH_Q8)
    try:
        ref = render(ctx, fresh, spec, poses[0])
        before = render(ctx, refit, spec, poses[0])
        assert not np.array_equal(before[0], ref[0])
        ags.ags_scene_update_poses(ctx, refit, new, ags.AGS_UPDATE_REFIT)
        out = render(ctx, refit, spec, poses[0])
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        with pytest.raises(ags.AgsError):
            ags.ags_scene_update_poses(ctx, rebuilt, new, ags.AGS_UPDATE_REFIT)  # compressed nodes: rebuild only
        ags.ags_scene_update_poses(ctx, rebuilt, new, ags.AGS_UPDATE_REBUILD)
        out = render(ctx, rebuilt, spec, poses[0])
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        for e in range(4):
            a, _ = ags.ags_scene_get_world_triangles(refit, e)
            b, _ = ags.ags_scene_get_world_triangles(fresh, e)
            assert np.array_equal(a, b)
        check_all(moved, spec, poses[0], ref[0], ref[1], tag="moved obstacles 64x48")
        bad = new.copy()
        bad[5, 3:] = 0.0
        with pytest.raises(ags.AgsError):
            ags.ags_scene_update_poses(ctx, refit, bad, ags.AGS_UPDATE_REFIT)
    finally:
        for sc in (fresh, refit, rebuilt):
            ags.ags_scene_destroy(sc)


def test_refit_after_moving_every_object_including_split_walls(ctx):
    """The rooms themselves (large split wall triangles) turn and move too: refit boxes built from each
    reference's barycentric range still cover every triangle, so the images equal a fresh build's."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=48, height=36)
    rng = np.random.default_rng(22)
    refit = ags.ags_scene_build(ctx, batch)
    try:
        cur = batch.poses.copy()
        for step in range(3):
            cur[:, :3] += rng.normal(0, 0.3, (cur.shape[0], 3)).astype(np.float32)
            q = cur[:, 3:] + rng.normal(0, 0.2, (cur.shape[0], 4)).astype(np.float32)
            cur[:, 3:] = q / np.linalg.norm(q, axis=1, keepdims=True)
            ags.ags_scene_update_poses(ctx, refit, cur, ags.AGS_UPDATE_REFIT)
            moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                                 batch.env_sub, cur.copy())
            fresh = ags.ags_scene_build(ctx, moved)
            try:
                a = render(ctx, refit, spec, poses[0])
                b = render(ctx, fresh, spec, poses[0])
                assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), step
            finally:
                ags.ags_scene_destroy(fresh)
        check_all(moved, spec, poses[0], a[0], a[1], tag="refit, every object moved 48x36")
    finally:
        ags.ags_scene_destroy(refit)


def test_auto_update_refits_then_rebuilds_when_the_tree_degrades(ctx):
    """AGS_UPDATE_AUTO keeps a refitted tree while its surface-area cost stays within the rebuild ratio of the
    built tree's, and rebuilds past it; either way the images equal a fresh build's."""
    batch, spec, poses = S.obstacle_rooms(6, steps=1, width=48, height=36)
    scene = ags.ags_scene_build(ctx, batch)
    q8 = ags.ags_scene_build(ctx, batch, ags.AGS_BVH_Q8)
    try:
        now, built = ags.ags_scene_tree_cost(ctx, scene)
        assert built > 0 and abs(now - built) <= 1e-9 * built
        rng = np.random.default_rng(23)
        movable = np.ones(batch.poses.shape[0], bool)
        movable[batch.env_sub[:-1]] = False
        cur = batch.poses.copy()

        def fresh_images(p):
            moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                                 batch.env_sub, p.copy())
            f = ags.ags_scene_build(ctx, moved)
            try:
                return render(ctx, f, spec, poses[0])
            finally:
                ags.ags_scene_destroy(f)

        # a small move: refitted, kept (the built cost stays that of the build)
        cur[movable, :3] += rng.normal(0, 0.01, (movable.sum(), 3)).astype(np.float32)
        ags.ags_scene_update_poses(ctx, scene, cur, ags.AGS_UPDATE_AUTO)
        now1, built1 = ags.ags_scene_tree_cost(ctx, scene)
        assert built1 == built and now1 != built and now1 <= 1.25 * built
        ref = fresh_images(cur)
        out = render(ctx, scene, spec, poses[0])
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        # a large move past a tight ratio: rebuilt (a new built cost, equal to the tree's own)
        ags.ags_scene_set_rebuild_ratio(scene, 1.0)
        cur[movable, :3] += rng.normal(0, 1.0, (movable.sum(), 3)).astype(np.float32)
        ags.ags_scene_update_poses(ctx, scene, cur, ags.AGS_UPDATE_AUTO)
        now2, built2 = ags.ags_scene_tree_cost(ctx, scene)
        assert built2 != built and abs(now2 - built2) <= 1e-9 * built2
        ref = fresh_images(cur)
        out = render(ctx, scene, spec, poses[0])
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                             batch.env_sub, cur.copy())
        check_all(moved, spec, poses[0], out[0], out[1], envs=[0, 5], tag="automatic refit or rebuild 48x36")
        # compressed nodes cannot refit: AUTO rebuilds them; their cost is not defined
        ags.ags_scene_update_poses(ctx, q8, cur, ags.AGS_UPDATE_AUTO)
        out = render(ctx, q8, spec, poses[0])
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        with pytest.raises(ags.AgsError):
            ags.ags_scene_tree_cost(ctx, q8)
        for bad in (0.5, float("nan"), float("inf")):
            with pytest.raises(ags.AgsError):
                ags.ags_scene_set_rebuild_ratio(scene, bad)
        with pytest.raises(ags.AgsError):
            ags.ags_scene_update_poses(ctx, scene, cur, 3)
    finally:
        ags.ags_scene_destroy(scene)
        ags.ags_scene_destroy(q8)


def test_step_graph_replays_the_render(ctx):
    batch, spec, poses = S.obstacle_rooms(3, steps=3, width=48, height=36)
    scene = ags.ags_scene_build(ctx, batch)
    p = torch.as_tensor(poses[0]).cuda()
    d = torch.empty((3, 36, 48), device="cuda")
    s = torch.empty((3, 36, 48), dtype=torch.int32, device="cuda")
    g = ags.ags_render_graph_create(ctx, scene, spec, p, d, s)
    try:
        for step in range(3):
            p.copy_(torch.as_tensor(poses[step]).cuda())
            ags.ags_render_graph_launch(g)
            ags.ags_stream_status(ctx)
            ref = render(ctx, scene, spec, poses[step])
            assert np.array_equal(d.cpu().numpy(), ref[0]) and np.array_equal(s.cpu().numpy(), ref[1])
    finally:
        ags.ags_render_graph_destroy(g)
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- extra hit channels
def render_channels(ctx, scene, spec, poses, which=("face", "bary", "normal", "point")):
    E = poses.shape[0]
    H, W = spec.height, spec.width
    p = torch.as_tensor(np.ascontiguousarray(poses, np.float32)).cuda()
    depth = torch.empty((E, H, W), device="cuda")
    seg = torch.empty((E, H, W), dtype=torch.int32, device="cuda")
    shapes = {"face": ((E, H, W), torch.int32), "bary": ((E, H, W, 2), torch.float32),
              "normal": ((E, H, W, 3), torch.float32), "point": ((E, H, W, 3), torch.float32)}
    ch = {k: torch.full(shapes[k][0], 7, dtype=shapes[k][1], device="cuda") for k in which}
    ags.ags_render_channels(ctx, scene, spec, p, depth, seg, **ch)
    ags.ags_stream_status(ctx)
    return depth.cpu().numpy(), seg.cpu().numpy(), {k: v.cpu().numpy() for k, v in ch.items()}


@pytest.mark.parametrize("sensor", ["camera", "lidar", "camera_near_invalid"])
def test_hit_channels_match_oracle(ctx, sensor):
    """Face index, barycentrics, normal and sensor-frame point against the FP64 oracle on every ray;
    depth and segment IDs bit-identical to the plain render."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=40, height=30)
    if sensor == "lidar":
        spec = S.lidar(128, 24, (-30.0, 30.0), 0.2, 12.0)
    elif sensor == "camera_near_invalid":
        spec.near_mode, spec.min_range = ags.AGS_NEAR_INVALID, 1.2
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d0, s0 = render(ctx, scene, spec, poses[0])
        d, s, ch = render_channels(ctx, scene, spec, poses[0])
        assert np.array_equal(d, d0) and np.array_equal(s, s0)
        n = spec.width * spec.height
        rays = np.arange(n, dtype=np.int64)
        total = 0
        for e in range(3):
            ok, counted, res = compare_env(batch, e, spec, poses[0][e], d[e], s[e])
            assert ok.all(), describe_failures(ok, res, d[e].reshape(-1), s[e].reshape(-1), rays)
            det = {}
            okc = check_channels(batch, e, spec, poses[0][e], res, s[e], d[e], ch["face"][e], ch["bary"][e],
                                 ch["normal"][e], ch["point"][e], rays, det)
            assert okc.all(), f"env {e}: {int((~okc).sum())} rays\n" + describe_channel_failures(
                okc, det, res, ch["face"][e].reshape(-1), ch["bary"][e].reshape(-1, 2), ch["normal"][e].reshape(-1, 3))
            total += int((s[e] >= 0).sum())
        print(f"[parity] hit channels {sensor} {spec.height}x{spec.width}: {3 * n} rays, {total} hits, all within "
              f"the channel tolerances")
    finally:
        ags.ags_scene_destroy(scene)


def test_hit_channels_subsets_and_formats_are_bit_identical(ctx):
    """Any subset of channels gives the same bits, and so do compressed nodes and another leaf size."""
    batch, spec, poses = S.obstacle_rooms(2, steps=1, width=33, height=17)
    scenes = [ags.ags_scene_build(ctx, batch, f) for f in (ags.AGS_BVH_FP32, ags.AGS_BVH_FP16, ags.AGS_BVH_Q8)]
    try:
        _, _, ref = render_channels(ctx, scenes[0], spec, poses[0])
        for sc in scenes[1:]:
            _, _, got = render_channels(ctx, sc, spec, poses[0])
            for k in ref:
                assert np.array_equal(ref[k], got[k]), k
        for which in (("point",), ("face", "normal"), ("bary",)):
            _, _, got = render_channels(ctx, scenes[0], spec, poses[0], which)
            for k in which:
                assert np.array_equal(ref[k], got[k]), k
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((2, 17, 33), device="cuda")
        sg = torch.empty((2, 17, 33), dtype=torch.int32, device="cuda")
        buf = torch.empty(2 * 17 * 33 * 3 + 1, device="cuda")
        with pytest.raises(ags.AgsError):  # misaligned channel pointer
            ags.ags_render_channels(ctx, scenes[0], spec, p, d, sg, point=buf.data_ptr() + 2)
    finally:
        for sc in scenes:
            ags.ags_scene_destroy(sc)


# ---------------------------------------------------------------- stereo shadows
@pytest.mark.parametrize("baseline", [(0.0, -0.095, 0.0), (0.0, -0.6, 0.2)])
def test_stereo_shadows_match_oracle(ctx, baseline):
    """A pixel is invalidated exactly when the oracle's segment from the hit to the second sensor surely
    meets a triangle, kept (bit-identical) when it surely does not; either where the oracle's bands allow."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=40, height=30)
    scene = ags.ags_scene_build(ctx, batch)
    E, H, W = 3, 30, 40
    try:
        d0, s0 = render(ctx, scene, spec, poses[0])
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((E, H, W), device="cuda")
        sg = torch.empty((E, H, W), dtype=torch.int32, device="cuda")
        face = torch.empty((E, H, W), dtype=torch.int32, device="cuda")
        ags.ags_render_ex(ctx, scene, spec, p, d, sg, face=face, baseline=baseline)
        ags.ags_stream_status(ctx)
        d, sg, face = d.cpu().numpy(), sg.cpu().numpy(), face.cpu().numpy()
        _, _, ch = render_channels(ctx, scene, spec, poses[0], ("face",))
        miss_v = np.float32(spec.max_range)
        n_sh = n_either = 0
        rays = np.arange(H * W, dtype=np.int64)
        for e in range(E):
            tris, tseg = oracle_env(batch, e)
            s = oracle_sensor(spec)
            pose64 = np.asarray(poses[0][e], np.float32).astype(np.float64)
            res = O.render(tris, tseg, s, pose64, rays)
            verdict = O.shadow(tris, s, pose64, np.asarray(baseline, np.float32).astype(np.float64),
                               np.float32(1e-4), rays, res)
            a0, b0 = d0[e].reshape(-1), s0[e].reshape(-1)
            a, b = d[e].reshape(-1), sg[e].reshape(-1)
            kept = (a == a0) & (b == b0)
            invalid = (a == miss_v) & (b == -1)
            loose = (res["flags"] & (O.F_COUNTED | O.F_WIDE)) != 0
            free = b0 == -1
            ok = np.where(free, kept, np.where(loose | (verdict == 2), kept | invalid,
                                               np.where(verdict == 1, invalid, kept)))
            bad = np.nonzero(~ok)[0][:5]
            assert ok.all(), [(int(i), float(a0[i]), int(b0[i]), float(a[i]), int(b[i]), int(verdict[i]),
                               int(res["flags"][i])) for i in bad]
            # the face channel follows the verdict: -1 where invalidated, as without stereo elsewhere
            f, f0 = face[e].reshape(-1), ch["face"][e].reshape(-1)
            assert np.array_equal(f[b == -1], np.full(int((b == -1).sum()), -1))
            assert np.array_equal(f[b >= 0], f0[b >= 0])
            n_sh += int(((b == -1) & (b0 >= 0)).sum())
            n_either += int((verdict == 2).sum())
        print(f"[parity] stereo baseline {baseline}: {E * H * W} rays, {n_sh} shadowed, {n_either} either")
        assert n_sh > 0
    finally:
        ags.ags_scene_destroy(scene)


def test_stereo_zero_baseline_shadows_nothing_and_bad_args(ctx):
    batch, spec, poses = S.obstacle_rooms(2, steps=1, width=24, height=16)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d0, s0 = render(ctx, scene, spec, poses[0])
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((2, 16, 24), device="cuda")
        sg = torch.empty((2, 16, 24), dtype=torch.int32, device="cuda")
        ags.ags_render_ex(ctx, scene, spec, p, d, sg, baseline=(0.0, 0.0, 0.0))
        ags.ags_stream_status(ctx)
        assert np.array_equal(d.cpu().numpy(), d0) and np.array_equal(sg.cpu().numpy(), s0)
        for bad in (dict(baseline=(float("nan"), 0, 0)), dict(baseline=(0, 0.1, 0), eps=1.5)):
            with pytest.raises(ags.AgsError):
                ags.ags_render_ex(ctx, scene, spec, p, d, sg, **bad)
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- user projection models
def test_ray_table_of_camera_rows_is_bit_identical_to_the_camera(ctx):
    """A table holding the camera's own float32 (1, a, b) rows renders bit-identically to the camera."""
    batch, spec, poses = S.obstacle_rooms(2, steps=1, width=37, height=23)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d0, s0 = render(ctx, scene, spec, poses[0])
        W, H = spec.width, spec.height
        inv_f = np.float32(math.tan(0.5 * float(np.float32(spec.hfov))) / (0.5 * W))
        col = np.arange(W, dtype=np.float32)[None, :]
        row = np.arange(H, dtype=np.float32)[:, None]
        ly = (np.float32(0.5) * np.float32(W) - (col + np.float32(0.5))) * inv_f
        lz = (np.float32(0.5) * np.float32(H) - (row + np.float32(0.5))) * inv_f
        table = np.stack(np.broadcast_arrays(np.ones((H, W), np.float32), ly, lz), -1).astype(np.float32)
        tspec = S.ray_table_spec(W, H, spec.min_range, spec.max_range)
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((2, H, W), device="cuda")
        sg = torch.empty((2, H, W), dtype=torch.int32, device="cuda")
        ags.ags_render_ex(ctx, scene, tspec, p, d, sg, ray_table=torch.as_tensor(table).cuda())
        ags.ags_stream_status(ctx)
        assert np.array_equal(d.cpu().numpy(), d0) and np.array_equal(sg.cpu().numpy(), s0)
        with pytest.raises(ags.AgsError):  # a ray-table spec without its table
            ags.ags_render(ctx, scene, tspec, p, d, sg)
        with pytest.raises(ags.AgsError):  # a table for a camera spec
            ags.ags_render_ex(ctx, scene, spec, p, d, sg, ray_table=torch.as_tensor(table).cuda())
    finally:
        ags.ags_scene_destroy(scene)


@pytest.mark.parametrize("model", ["fisheye", "dome", "random"])
def test_user_projection_models_match_oracle(ctx, model):
    """A 180-degree equidistant fisheye, a dome LiDAR and random scaled rows against the FP64 oracle on
    every ray (with extra channels)."""
    batch, _, poses = S.obstacle_rooms(2, steps=1, width=8, height=8)
    W, H = 48, 32
    if model == "fisheye":
        table = S.fisheye_table(W, H, 180.0)
        spec = S.ray_table_spec(W, H, 0.2, 10.0)
    elif model == "random":
        rng = np.random.default_rng(24)
        table = (rng.normal(size=(H, W, 3)) * rng.uniform(0.3, 3.0, (H, W, 1))).astype(np.float32)
        spec = S.ray_table_spec(W, H, 0.05, 8.0)
    else:
        table = None
        spec = S.dome_lidar(W, H, 0.2, 12.0)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((2, H, W), device="cuda")
        sg = torch.empty((2, H, W), dtype=torch.int32, device="cuda")
        ch = {"face": torch.empty((2, H, W), dtype=torch.int32, device="cuda"),
              "bary": torch.empty((2, H, W, 2), device="cuda"), "normal": torch.empty((2, H, W, 3), device="cuda"),
              "point": torch.empty((2, H, W, 3), device="cuda")}
        ags.ags_render_ex(ctx, scene, spec, p, d, sg, ray_table=None if table is None else torch.as_tensor(table).cuda(),
                          **ch)
        ags.ags_stream_status(ctx)
        d, sg = d.cpu().numpy(), sg.cpu().numpy()
        ch = {k: v.cpu().numpy() for k, v in ch.items()}
        rays = np.arange(W * H, dtype=np.int64)
        for e in range(2):
            tris, tseg = oracle_env(batch, e)
            s = oracle_sensor(spec)
            if table is not None:
                s.dirs = table.astype(np.float64)
            pose64 = np.asarray(poses[0][e], np.float32).astype(np.float64)
            res = O.render(tris, tseg, s, pose64, rays)
            ok, counted = O.check(res, d[e].reshape(-1), sg[e].reshape(-1), s.max_range)
            assert ok.all(), describe_failures(ok, res, d[e].reshape(-1), sg[e].reshape(-1), rays)
            det = {}
            okc = check_channels_sensor(tris, s, pose64, res, sg[e], d[e], ch, e, rays, det)
            assert okc.all(), describe_channel_failures(okc, det, res, ch["face"][e].reshape(-1),
                                                        ch["bary"][e].reshape(-1, 2), ch["normal"][e].reshape(-1, 3))
            print(f"[parity] {model} {H}x{W}: {W * H} rays, {int(counted.sum())} counted; every other ray within "
                  f"1e-5*d+1e-6 of the FP64 value")
    finally:
        ags.ags_scene_destroy(scene)


def test_host_path_with_page_locked_outputs_writes_in_place(ctx):
    """ags_render_host into page-locked buffers (written by the kernel over the host link) equals the device
    render and the pageable-buffer path bit for bit."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=40, height=30)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d0, s0 = render(ctx, scene, spec, poses[0])
        pd = torch.full((3, 30, 40), 7.0).pin_memory()
        ps = torch.full((3, 30, 40), 7, dtype=torch.int32).pin_memory()
        pp = torch.as_tensor(np.ascontiguousarray(poses[0])).pin_memory()
        for _ in range(2):
            ags.ags_render_host(ctx, scene, spec, pp.numpy(), pd.numpy(), ps.numpy())
            assert np.array_equal(pd.numpy(), d0) and np.array_equal(ps.numpy(), s0)
        hd, hs = ags.ags_render_host(ctx, scene, spec, np.ascontiguousarray(poses[0]))
        assert np.array_equal(hd, d0) and np.array_equal(hs, s0)
    finally:
        ags.ags_scene_destroy(scene)


def test_build_tuning_keeps_results_and_updates(ctx):
    """Rebuilding with each splitting setting and keeping the fastest changes no output bit; the tuned
    scene still refits to exactly a fresh build's images."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=40, height=30)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        d0, s0 = render(ctx, scene, spec, poses[0])
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((3, 30, 40), device="cuda")
        sg = torch.empty((3, 30, 40), dtype=torch.int32, device="cuda")
        best = ags.ags_autotune_build(ctx, scene, spec, p, d, sg, (1, 16, 48), 1)
        assert best in (0, 1, 16, 48)
        d1, s1 = render(ctx, scene, spec, poses[0])
        assert np.array_equal(d1, d0) and np.array_equal(s1, s0)
        with pytest.raises(ags.AgsError):
            ags.ags_autotune_build(ctx, scene, spec, p, d, sg, (300,), 1)
        # whole build settings: splitting, clustering radius, node format and leaf size at once
        cands = [ags.AGS_CLUSTER_RADIUS(64), ags.AGS_CLUSTER_RADIUS(32) | ags.AGS_SPLIT_CELLS(32),
                 ags.AGS_BVH_FP16 | ags.AGS_LEAF_SIZE(3), ags.AGS_BUILD_LBVH]
        flags = ags.ags_autotune_build_flags(ctx, scene, spec, p, d, sg, cands, 1)
        assert flags in cands or (flags >> 12) & 0xFF in (0, 1, 16, 48)
        d2, s2 = render(ctx, scene, spec, poses[0])
        assert np.array_equal(d2, d0) and np.array_equal(s2, s0)
        for bad in ([1 << 25], [ags.AGS_BUILD_INSTANCED], [7]):
            with pytest.raises(ags.AgsError):
                ags.ags_autotune_build_flags(ctx, scene, spec, p, d, sg, bad, 1)
        rng = np.random.default_rng(23)
        new = batch.poses.copy()
        new[:, :3] += rng.normal(0, 0.2, (new.shape[0], 3)).astype(np.float32)
        ags.ags_scene_update_poses(ctx, scene, new, ags.AGS_UPDATE_REFIT)
        moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                             batch.env_sub, new)
        fresh = ags.ags_scene_build(ctx, moved)
        try:
            a, b = render(ctx, scene, spec, poses[0]), render(ctx, fresh, spec, poses[0])
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        finally:
            ags.ags_scene_destroy(fresh)
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- two-level scenes
@pytest.mark.parametrize("sensor", ["camera", "lidar"])
def test_two_level_scene_matches_oracle(ctx, sensor):
    """Objects with their own BVHs under a per-environment BVH over their boxes: every ray against the
    oracle, and against a single-level scene of the same objects within the tolerance."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=64, height=48)
    if sensor == "lidar":
        spec = S.lidar(128, 24, (-30.0, 30.0), 0.2, 12.0)
    two = ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED)
    one = ags.ags_scene_build(ctx, batch)
    try:
        d2, s2 = render(ctx, two, spec, poses[0])
        d1, s1 = render(ctx, one, spec, poses[0])
        check_all(batch, spec, poses[0], d2, s2, tag=f"two-level {sensor} {spec.height}x{spec.width}")
        same_seg = (s1 == s2).mean()
        assert same_seg > 0.99
        both = (s1 >= 0) & (s2 >= 0) & (s1 == s2)
        assert np.all(np.abs(d1[both] - d2[both]) <= 1e-5 * d1[both] + 1e-6)
        for e in range(3):
            a, sa = ags.ags_scene_get_world_triangles(two, e)
            b, sb = ags.ags_scene_get_world_triangles(one, e)
            assert np.array_equal(a, b) and np.array_equal(sa, sb)
    finally:
        ags.ags_scene_destroy(two)
        ags.ags_scene_destroy(one)


def test_two_level_scene_updates_and_limits(ctx):
    """Moving every object rewrites the object table and rebuilds only the top level; the images then
    match the oracle of the moved scene. Unsupported options are refused."""
    batch, spec, poses = S.obstacle_rooms(3, steps=1, width=48, height=36)
    two = ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED)
    try:
        rng = np.random.default_rng(25)
        cur = batch.poses.copy()
        for step in range(2):
            cur[:, :3] += rng.normal(0, 0.3, (cur.shape[0], 3)).astype(np.float32)
            q = cur[:, 3:] + rng.normal(0, 0.2, (cur.shape[0], 4)).astype(np.float32)
            cur[:, 3:] = q / np.linalg.norm(q, axis=1, keepdims=True)
            ags.ags_scene_update_poses(ctx, two, cur, ags.AGS_UPDATE_REFIT)
            moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                                 batch.env_sub, cur.copy())
            d, s = render(ctx, two, spec, poses[0])
            check_all(moved, spec, poses[0], d, s, tag="two-level after moves 48x36")
        p = torch.as_tensor(poses[0]).cuda()
        dd = torch.empty((3, 36, 48), device="cuda")
        ss = torch.empty((3, 36, 48), dtype=torch.int32, device="cuda")
        with pytest.raises(ags.AgsError):
            ags.ags_render_ex(ctx, two, spec, p, dd, ss, face=torch.empty((3, 36, 48), dtype=torch.int32,
                                                                          device="cuda"))
        with pytest.raises(ags.AgsError):
            ags.ags_render_count(ctx, two, spec, p)
        with pytest.raises(ags.AgsError):
            ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED | ags.AGS_BVH_Q8)
        cfg = ags.ags_autotune(ctx, two, spec, p, dd, ss, 1).as_dict()
        assert cfg["tile_w"] == 8 and cfg["rays_per_lane"] == 1
        hd, hs = ags.ags_render_host(ctx, two, spec, np.ascontiguousarray(poses[0]))
        d, s = render(ctx, two, spec, poses[0])
        assert np.array_equal(hd, d) and np.array_equal(hs, s)
    finally:
        ags.ags_scene_destroy(two)


def test_two_level_opened_roots(ctx):
    """Objects whose box spans their environment have their roots opened into the top level: a sphere of
    1280 triangles around the sensor (its root's children are inner nodes) and a room (its root's children
    are leaves), each with smaller objects inside, turned and moved; every ray against the oracle."""
    rng = np.random.default_rng(41)
    sv, sf = S.icosphere(4.0, 3)
    rv, rf = S.room()
    inner = [(*S.box(0.6, 0.8, 1.0), np.array([1.5, 0.2, 0.3, *S.random_unit_quat(rng)], np.float32), 2),
             (*S.icosphere(0.5, 2), np.array([-1.0, 1.2, -0.4, 0, 0, 0, 1], np.float32), 3)]
    turned = np.array([0.1, -0.2, 0.05, *S.random_unit_quat(rng)], np.float32)
    room_inner = [(*S.box(1.0, 0.5, 0.7), np.array([2.0, 1.0, 1.5, *S.random_unit_quat(rng)], np.float32), 2)]
    batch = S.scene_from_lists([[(sv, sf, S.IDENTITY_POSE, 1)] + inner, [(sv, sf, turned, 1)] + inner,
                                [(rv, rf, S.IDENTITY_POSE, 0)] + room_inner])
    spec = S.pinhole(64, 48, 100.0, 0.1, 12.0)
    poses = np.array([[0, 0, 0, 0, 0, 0, 1], [0.3, 0.1, -0.2, *S.random_unit_quat(rng)],
                      [-1.0, -2.0, 2.0, *S.quat_from_euler_zyx(0.4, 0.1, 0.0)]], np.float32)
    two = ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED)
    try:
        d, s = render(ctx, two, spec, poses)
        assert (s >= 0).all()  # closed sphere and room: every ray hits
        check_all(batch, spec, poses, d, s, tag="two-level opened roots 64x48")
        cur = batch.poses.copy()
        cur[:, :3] += rng.normal(0, 0.05, (cur.shape[0], 3)).astype(np.float32)
        ags.ags_scene_update_poses(ctx, two, cur, ags.AGS_UPDATE_REBUILD)
        moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                             batch.env_sub, cur.copy())
        d, s = render(ctx, two, spec, poses)
        check_all(moved, spec, poses, d, s, tag="two-level opened roots after a move")
    finally:
        ags.ags_scene_destroy(two)


def test_two_level_empty_and_tiny(ctx):
    tri = (np.array([[3, -3, -3], [3, 3, -3], [3, 0, 3]], np.float32), np.array([[0, 1, 2]], np.int32),
           S.IDENTITY_POSE, 7)
    empty_obj = (np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), S.IDENTITY_POSE, 3)
    batch = S.scene_from_lists([[], [tri], [tri, empty_obj, tri]])
    spec = S.pinhole(5, 3, 90.0, 0.1, 10.0)
    poses = np.tile(S.IDENTITY_POSE, (3, 1))
    two = ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED)
    try:
        d, s = render(ctx, two, spec, poses)
        assert (s[0] == -1).all() and (d[0] == np.float32(10.0)).all()
        check_all(batch, spec, poses, d, s)
    finally:
        ags.ags_scene_destroy(two)
    batch, spec, poses = S.tiny_room()
    two = ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED)
    try:
        for k in range(0, 16, 5):
            d, s = render(ctx, two, spec, poses[k:k + 1])
            check_all(batch, spec, poses[k:k + 1], d, s, tag="two-level tiny room 64x48")
    finally:
        ags.ags_scene_destroy(two)


# ---------------------------------------------------------------- watertightness
@pytest.mark.parametrize("mesh", ["icosphere", "cylinder", "box", "cone"])
def test_no_ray_slips_through_closed_meshes(ctx, mesh):
    """From inside a closed mesh every ray must hit, including rays aimed exactly at its vertices and at the
    midpoints of its edges (where a test that is not watertight lets rays through cracks); the hits also
    match the oracle. Ray tables carry the aimed directions."""
    if mesh == "icosphere":
        v, f = S.icosphere(1.7, level=3)
        centre = np.array([0.11, -0.07, 0.05])
    elif mesh == "cylinder":
        v, f = S.cylinder(0.9, 2.5, 48)
        centre = np.array([0.05, 0.1, -0.3])
    elif mesh == "box":
        v, f = S.box(2.0, 1.4, 3.1)
        centre = np.array([0.2, -0.1, 0.3])
    else:
        v, f = S.cone(1.2, 2.0, 40)
        centre = np.array([0.05, -0.02, 0.4])
    batch = S.scene_from_lists([[(v, f, S.IDENTITY_POSE, 4)]])
    scene = ags.ags_scene_build(ctx, batch)
    try:
        v64 = v.astype(np.float64)
        edges = set()
        for a, b, c in f:
            for x, y in ((a, b), (b, c), (c, a)):
                edges.add((min(x, y), max(x, y)))
        targets = [v64] + [np.array([(v64[x] + v64[y]) / 2 for x, y in sorted(edges)])]
        rng = np.random.default_rng(26)
        targets.append(rng.normal(size=(512, 3)) + centre)
        dirs = np.concatenate(targets) - centre
        n = dirs.shape[0]
        W = 64
        H = (n + W - 1) // W
        table = np.zeros((H * W, 3), np.float32)
        table[:n] = dirs
        table[n:] = dirs[0]
        table = table.reshape(H, W, 3)
        spec = S.ray_table_spec(W, H, 0.01, 100.0)
        pose = np.concatenate([centre, [0, 0, 0, 1]]).astype(np.float32)[None]
        p = torch.as_tensor(pose).cuda()
        d = torch.empty((1, H, W), device="cuda")
        sg = torch.empty((1, H, W), dtype=torch.int32, device="cuda")
        ags.ags_render_ex(ctx, scene, spec, p, d, sg, ray_table=torch.as_tensor(table).cuda())
        ags.ags_stream_status(ctx)
        d, sg = d.cpu().numpy().reshape(-1), sg.cpu().numpy().reshape(-1)
        assert (sg == 4).all(), f"{int((sg != 4).sum())} of {sg.size} rays slipped through"
        tris, tseg = oracle_env(batch, 0)
        s = oracle_sensor(spec)
        s.dirs = table.astype(np.float64)
        rays = np.arange(H * W, dtype=np.int64)
        res = O.render(tris, tseg, s, pose[0].astype(np.float64), rays)
        ok, counted = O.check(res, d, sg, s.max_range)
        assert ok.all(), describe_failures(ok, res, d, sg, rays)
        print(f"[parity] watertight {mesh}: {n} aimed rays ({v.shape[0]} vertices, {len(edges)} edge midpoints), "
              f"all hit, {int(counted.sum())} counted")
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- BVH structure
def test_bvh_structure_of_every_variant(ctx):
    """Every node and reference reached once, copies equal to their triangles, and every point of every
    triangle inside the boxes of a path to one of its references: all builders, formats, leaf sizes and
    splitting settings, a two-level scene, a refitted scene and a LiDAR forest."""
    batch, spec, poses = S.obstacle_rooms(4, steps=1, width=8, height=8)
    variants = [0, ags.AGS_BVH_FP16, ags.AGS_BVH_Q8, ags.AGS_LEAF_SIZE(1), ags.AGS_LEAF_SIZE(4),
                ags.AGS_SPLIT_CELLS(1), ags.AGS_SPLIT_CELLS(64), ags.AGS_BUILD_LBVH,
                ags.AGS_BUILD_LBVH | ags.AGS_BVH_Q8 | ags.AGS_LEAF_SIZE(3), ags.AGS_BUILD_INSTANCED,
                ags.AGS_BUILD_GREEDY_COLLAPSE, ags.AGS_LEAF_SIZE(3) | ags.AGS_SPLIT_CELLS(64),
                ags.AGS_CLUSTER_RADIUS(32), ags.AGS_CLUSTER_RADIUS(128) | ags.AGS_LEAF_SIZE(1)]
    for flags in variants:
        scene = ags.ags_scene_build(ctx, batch, flags)
        try:
            r = ags.ags_scene_validate(scene)
            assert r["violations"] == 0 and r["points"] > 0, (flags, r.get("problems"), r)
            assert r["depth"] * 7 <= 64 or flags & ags.AGS_BUILD_INSTANCED, (flags, r)
        finally:
            ags.ags_scene_destroy(scene)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        rng = np.random.default_rng(27)
        new = batch.poses.copy()
        new[:, :3] += rng.normal(0, 0.4, (new.shape[0], 3)).astype(np.float32)
        q = new[:, 3:] + rng.normal(0, 0.3, (new.shape[0], 4)).astype(np.float32)
        new[:, 3:] = q / np.linalg.norm(q, axis=1, keepdims=True)
        ags.ags_scene_update_poses(ctx, scene, new, ags.AGS_UPDATE_REFIT)
        r = ags.ags_scene_validate(scene)
        assert r["violations"] == 0, r
    finally:
        ags.ags_scene_destroy(scene)
    fb, _, _ = S.lidar_forests(1, steps=1, trees=(5, 8), tris=(2000, 3000))
    scene = ags.ags_scene_build(ctx, fb, ags.AGS_SPLIT_CELLS(48))
    try:
        r = ags.ags_scene_validate(scene)
        assert r["violations"] == 0, r
        print(f"[structure] forest: {r}")
    finally:
        ags.ags_scene_destroy(scene)


# ---------------------------------------------------------------- building blocks
@pytest.mark.parametrize("n,end_bit", [(0, 64), (1, 64), (1000, 12), (257 * 1024 + 3, 40), (3_000_001, 64)])
def test_radix_sort_is_a_stable_sort(ctx, n, end_bit):
    """The device radix sort against numpy's stable argsort on keys with many ties, on the low end_bit bits."""
    rng = np.random.default_rng(28 + n)
    keys = rng.integers(0, 1 << 62, n, dtype=np.int64).astype(np.uint64)
    keys[: n // 2] = keys[: n // 2] % 97  # plenty of equal keys
    keys = rng.permutation(keys) if n else keys
    mask = np.uint64((1 << end_bit) - 1) if end_bit < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    keys &= mask
    vals = np.arange(n, dtype=np.uint32)
    kd = torch.as_tensor(keys.view(np.int64)).cuda()
    vd = torch.as_tensor(vals.view(np.int32)).cuda()
    ags.ags_test_sort_pairs(ctx, kd, vd, end_bit)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vd.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("n", [0, 1, 2, 1023, 1024, 1025, 1_000_003])
def test_exclusive_scan(ctx, n):
    rng = np.random.default_rng(29 + n)
    x = rng.integers(0, 50, n).astype(np.int32)
    d = torch.as_tensor(x).cuda()
    total = ags.ags_test_exclusive_scan(ctx, d)
    ref = np.concatenate([[0], np.cumsum(x)[:-1]]).astype(np.int64) if n else np.zeros(0, np.int64)
    assert np.array_equal(d.cpu().numpy().astype(np.int64), ref)
    assert total == int(x.sum())


def test_launch_shape_cache(ctx, tmp_path):
    """A tuned shape is stored under the device, sensor shape and scene size, and a later lookup applies it
    without tuning; outputs do not depend on it."""
    from paper_2503_01471_gb300 import tuning
    batch, spec, poses = S.obstacle_rooms(2, steps=1, width=40, height=30)
    dev = ags.ags_context_device(ctx)
    assert dev["sm_count"] > 0 and dev["compute_capability"] >= 100 and dev["name"]
    path = str(tmp_path / "shapes.json")
    scene = ags.ags_scene_build(ctx, batch)
    try:
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((2, 30, 40), device="cuda")
        s = torch.empty((2, 30, 40), dtype=torch.int32, device="cuda")
        a = tuning.autotune_cached(ctx, scene, spec, p, d, s, path, 1)
        assert a["cached"] is False
        ags.ags_set_launch_config(ctx, scene, spec, None)
        b = tuning.autotune_cached(ctx, scene, spec, p, d, s, path, 1)
        assert b["cached"] is True and b["tile_w"] == a["tile_w"] and b["rays_per_lane"] == a["rays_per_lane"]
        got = ags.ags_get_launch_config(ctx, scene, spec)
        assert got["tile_w"] == a["tile_w"] and got["rays_per_lane"] == a["rays_per_lane"]
    finally:
        ags.ags_scene_destroy(scene)
