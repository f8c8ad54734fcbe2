"""Parity at the full sizes of the LiDAR-forest, precision and serving workloads, in the launch configuration
the benchmark uses: the GPU renders everything, the FP64 oracle checks sampled rays one by one, and
properties that hold at any size are checked on every ray. (The 1024-room camera workload has its own
full-size test in test_gpu_parity.py.)"""
import numpy as np
import pytest
import torch

import oracle as O
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


def sampled_parity(batch, spec, poses, depth, seg, envs, k, rng, tag):
    n_pix = spec.width * spec.height
    n = counted = 0
    for e in envs:
        rays = np.sort(rng.choice(n_pix, k, replace=False)).astype(np.int64)
        ok, cnt, res = compare_env(batch, e, spec, poses[e], depth[e], seg[e], rays)
        d, s = depth[e].reshape(-1)[rays], seg[e].reshape(-1)[rays]
        assert ok.all(), f"{tag} env {e}:\n" + describe_failures(ok, res, d, s, rays)
        n += rays.size
        counted += int(cnt.sum())
    print(f"[parity] {tag}: {n} sampled rays of {len(envs)} envs, {counted} counted")


def every_ray(depth, seg, spec):
    """Properties of every output: misses exactly max range, values within [min, max] range, finite."""
    assert np.isfinite(depth).all()
    assert (depth[seg == -1] == np.float32(spec.max_range)).all()
    assert ((depth >= np.float32(spec.min_range)) & (depth <= np.float32(spec.max_range))).all()
    assert (seg >= -1).all()


def test_lidar_forests_full_size(ctx):
    """256 forests x 64x512 LiDAR (~193 M triangles), reference splitting tuned and launch shape autotuned
    as the benchmark does."""
    batch, spec, poses = S.lidar_forests(256, steps=1)
    scene = ags.ags_scene_build(ctx, batch)
    try:
        E = batch.n_envs
        p = torch.as_tensor(poses[0]).cuda()
        d = torch.empty((E, spec.height, spec.width), device="cuda")
        s = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device="cuda")
        cells = ags.ags_autotune_build(ctx, scene, spec, p, d, s, (16, 32, 48, 64), 1)
        ags.ags_autotune(ctx, scene, spec, p, d, s, 1)
        ags.ags_render(ctx, scene, spec, p, d, s)
        ags.ags_stream_status(ctx)
        depth, seg = d.cpu().numpy(), s.cpu().numpy()
        every_ray(depth, seg, spec)
        assert (seg >= 0).mean() > 0.2
        rng = np.random.default_rng(30)
        envs = sorted(set([0, E - 1] + list(rng.choice(E, 6, replace=False))))
        sampled_parity(batch, spec, poses[0], depth, seg, envs, 48, rng, f"256 forests 64x512 ({cells} cells)")
    finally:
        ags.ags_scene_destroy(scene)


def test_two_level_rooms_full_size(ctx):
    """The dynamic workload's two-level scene at full size: 1024 rooms x 270x480 (31k objects, the rooms'
    roots opened into the top level), before and after every obstacle moves; sampled rays against the oracle
    of the moved scene, and every ray against the single-level scene of the same poses (same segment where
    both hit; depths within the tolerance)."""
    batch, spec, poses = S.obstacle_rooms(1024, steps=1)
    E = batch.n_envs
    p = torch.as_tensor(poses[0]).cuda()
    rng = np.random.default_rng(35)
    cur = batch.poses.copy()
    movable = np.ones(cur.shape[0], bool)
    movable[batch.env_sub[:-1]] = False
    two = ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED)
    try:
        for step in range(2):
            if step:
                cur[movable, :3] += rng.normal(0, 0.05, (int(movable.sum()), 3)).astype(np.float32)
                q = cur[movable, 3:] + rng.normal(0, 0.025, (int(movable.sum()), 4)).astype(np.float32)
                cur[movable, 3:] = q / np.linalg.norm(q, axis=1, keepdims=True)
                ags.ags_scene_update_poses(ctx, two, cur, ags.AGS_UPDATE_REBUILD)
            moved = S.SceneBatch(batch.vertices, batch.indices, batch.sub_vert, batch.sub_tri, batch.sub_seg,
                                 batch.env_sub, cur.copy())
            d = torch.empty((E, spec.height, spec.width), device="cuda")
            s = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device="cuda")
            ags.ags_render(ctx, two, spec, p, d, s)
            ags.ags_stream_status(ctx)
            depth, seg = d.cpu().numpy(), s.cpu().numpy()
            every_ray(depth, seg, spec)
            one = ags.ags_scene_build(ctx, moved)
            try:
                ags.ags_render(ctx, one, spec, p, d, s)
                ags.ags_stream_status(ctx)
                d1, s1 = d.cpu().numpy(), s.cpu().numpy()
            finally:
                ags.ags_scene_destroy(one)
            assert (s1 == seg).mean() > 0.9999
            both = (s1 >= 0) & (s1 == seg)
            assert (np.abs(d1[both] - depth[both]) <= 2 * (1e-5 * d1[both] + 1e-6)).mean() > 0.9999
            envs = sorted(set([0, E - 1] + list(rng.choice(E, 6, replace=False))))
            sampled_parity(moved, spec, poses[0], depth, seg, envs, 64, rng, f"two-level 1024 rooms, step {step}")
    finally:
        ags.ags_scene_destroy(two)


def test_precision_full_size(ctx):
    """4096 rooms x 135x240 with float32, float16 and 8-bit child bounds: outputs bit-identical, sampled rays
    within the tolerance of the oracle."""
    batch, spec, poses = S.obstacle_rooms(4096, steps=1, width=240, height=135)
    E = batch.n_envs
    p = torch.as_tensor(poses[0]).cuda()
    outs = []
    for fmt in (ags.AGS_BVH_FP32, ags.AGS_BVH_FP16, ags.AGS_BVH_Q8):
        scene = ags.ags_scene_build(ctx, batch, fmt)
        try:
            d = torch.empty((E, spec.height, spec.width), device="cuda")
            s = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device="cuda")
            ags.ags_autotune(ctx, scene, spec, p, d, s, 1)
            ags.ags_render(ctx, scene, spec, p, d, s)
            ags.ags_stream_status(ctx)
            outs.append((d.cpu().numpy(), s.cpu().numpy()))
        finally:
            ags.ags_scene_destroy(scene)
    for d, s in outs[1:]:
        assert np.array_equal(d, outs[0][0]) and np.array_equal(s, outs[0][1])
    every_ray(outs[0][0], outs[0][1], spec)
    rng = np.random.default_rng(31)
    envs = sorted(set([0, E - 1] + list(rng.choice(E, 30, replace=False))))
    sampled_parity(batch, spec, poses[0], outs[0][0], outs[0][1], envs, 32, rng, "4096 rooms 135x240 (3 formats)")


def test_serving_full_size(ctx):
    """8192 rooms of 1k-200k triangles served with mixed cameras and LiDARs: a burst's results equal direct
    renders of the same requests, and sampled requests match the oracle."""
    batch, poses = S.serving_rooms(8192)
    specs = [S.pinhole(240, 135), S.pinhole(480, 270), S.lidar(512, 64)]
    scene = ags.ags_scene_build(ctx, batch)
    rng = np.random.default_rng(32)
    n = 3000
    env = rng.integers(0, batch.n_envs, n)
    sp = rng.integers(0, 3, n)
    server = ags.ags_server_create(ctx, scene, specs, max_slots=512, max_inflight=3, arena_bytes=1 << 31)
    try:
        ids = [ags.ags_server_submit(server, int(env[i]), int(sp[i]), poses[0][env[i]]) for i in range(n)]
        got = {}
        import time
        t0 = time.time()
        while len(got) < n and time.time() - t0 < 120:
            for c in ags.ags_server_poll(server, 4096):
                got[int(c["request_id"])] = c
        assert len(got) == n
        check = rng.choice(n, 24, replace=False)
        for i in check:
            c = got[ids[i]]
            assert int(c["status"]) == 0
            spec = specs[sp[i]]
            npx = spec.width * spec.height
            d = np.zeros(npx, np.float32)
            s = np.zeros(npx, np.int32)
            ags.ags_memcpy_d2h(d, int(c["depth_dev"]))
            ags.ags_memcpy_d2h(s, int(c["seg_dev"]))
            # the same request rendered directly
            ids_d = torch.tensor([int(env[i])], dtype=torch.int32, device="cuda")
            pd = torch.as_tensor(poses[0][env[i]][None]).cuda()
            dd = torch.empty((1, spec.height, spec.width), device="cuda")
            ss = torch.empty((1, spec.height, spec.width), dtype=torch.int32, device="cuda")
            ags.ags_render_envs(ctx, scene, spec, ids_d, pd, dd, ss)
            ags.ags_stream_status(ctx)
            assert np.array_equal(dd.cpu().numpy().reshape(-1), d) and np.array_equal(ss.cpu().numpy().reshape(-1), s)
            rays = np.sort(rng.choice(npx, 16, replace=False)).astype(np.int64)
            ok, _, res = compare_env(batch, int(env[i]), spec, poses[0][env[i]], d, s, rays)
            assert ok.all(), describe_failures(ok, res, d[rays], s[rays], rays)
        for rid in ids:
            ags.ags_server_release(server, rid)
        print(f"[parity] serving 8192 rooms: {n} requests served, 24 checked against direct renders and the oracle")
    finally:
        ags.ags_server_destroy(server)
        ags.ags_scene_destroy(scene)
