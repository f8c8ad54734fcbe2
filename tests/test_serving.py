"""Continuous-batching server: every result is the same alone and in a mix of other requests, admission
waits for free arena space, and the load generator and the sequential baseline complete every request."""
import numpy as np
import pytest
import torch

import paper_2503_01471_gb300 as ags
from paper_2503_01471_gb300 import build as B
from paper_2503_01471_gb300 import scenes as S

from helpers import compare_env

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    B.build()
    ctx = ags.ags_context_create(0)
    batch, _, poses = S.obstacle_rooms(6, steps=1, width=8, height=8)
    scene = ags.ags_scene_build(ctx, batch)
    specs = [S.pinhole(64, 48), S.pinhole(32, 24, 70.0, 0.1, 8.0), S.lidar(64, 16, (-20.0, 20.0), 0.2, 12.0)]
    yield ctx, batch, scene, specs, poses[0]
    ags.ags_scene_destroy(scene)
    ags.ags_context_destroy(ctx)


def _result(c, spec):
    n = spec.width * spec.height
    d = np.zeros(n, np.float32)
    s = np.zeros(n, np.int32)
    ags.ags_memcpy_d2h(d, int(c["depth_dev"]))
    ags.ags_memcpy_d2h(s, int(c["seg_dev"]))
    return d, s


def _reference(ctx, scene, spec, env, pose):
    ids = torch.tensor([env], dtype=torch.int32, device="cuda")
    p = torch.as_tensor(np.asarray(pose, np.float32)[None]).cuda()
    d = torch.empty((1, spec.height, spec.width), device="cuda")
    s = torch.empty((1, spec.height, spec.width), dtype=torch.int32, device="cuda")
    ags.ags_render_envs(ctx, scene, spec, ids, p, d, s)
    ags.ags_stream_status(ctx)
    return d.cpu().numpy().reshape(-1), s.cpu().numpy().reshape(-1)


def _wait(server, ids, timeout=20.0):
    import time
    got = {}
    t0 = time.time()
    while len(got) < len(ids) and time.time() - t0 < timeout:
        for c in ags.ags_server_poll(server, 4096):
            got[int(c["request_id"])] = c
    assert len(got) >= len(ids), f"{len(got)} of {len(ids)} completed"
    return got


@pytest.mark.parametrize("use_graph", [False, True])
def test_alone_equals_in_the_mix(setup, use_graph):
    """Each result is the same served alone and inside a burst of other requests, with the batch step
    launched call by call or replayed from each stream's captured graph."""
    ctx, batch, scene, specs, poses = setup
    rng = np.random.default_rng(3)
    server = ags.ags_server_create(ctx, scene, specs, max_slots=64, max_inflight=2, arena_bytes=64 << 20,
                                   use_graph=use_graph)
    try:
        probe = [(2, 0), (5, 2), (0, 1)]
        alone = {}
        for env, sp in probe:
            rid = ags.ags_server_submit(server, env, sp, poses[env])
            c = _wait(server, [rid])[rid]
            alone[(env, sp)] = _result(c, specs[sp])
            ags.ags_server_release(server, rid)
            ref = _reference(ctx, scene, specs[sp], env, poses[env])
            assert np.array_equal(alone[(env, sp)][0], ref[0]) and np.array_equal(alone[(env, sp)][1], ref[1])
            ok, _, _ = compare_env(batch, env, specs[sp], poses[env], ref[0], ref[1])
            assert ok.all()
        # the same requests inside a burst of 300 others (mixed environments and sensors)
        ids, keys = [], []
        for k in range(300):
            env, sp = int(rng.integers(0, 6)), int(rng.integers(0, 3))
            p = poses[env].copy()
            p[:3] += rng.normal(0, 0.2, 3).astype(np.float32)
            ids.append(ags.ags_server_submit(server, env, sp, p))
            keys.append(None)
            if k in (10, 150, 299):
                env, sp = probe[(10, 150, 299).index(k)]
                ids.append(ags.ags_server_submit(server, env, sp, poses[env]))
                keys.append((env, sp))
        got = _wait(server, ids)
        for rid, key in zip(ids, keys):
            if key is not None:
                d, s = _result(got[rid], specs[key[1]])
                assert np.array_equal(d, alone[key][0]) and np.array_equal(s, alone[key][1]), key
            ags.ags_server_release(server, rid)
        st = ags.ags_server_stats(server)
        assert st["completed"] == st["submitted"] == 306 and st["batches"] >= 4
    finally:
        ags.ags_server_destroy(server)


def test_admission_waits_for_arena_space(setup):
    ctx, batch, scene, specs, poses = setup
    req_bytes = 64 * 48 * 8
    server = ags.ags_server_create(ctx, scene, specs[:1], max_slots=16, max_inflight=1,
                                   arena_bytes=2 * req_bytes + 100)
    try:
        ids = [ags.ags_server_submit(server, e % 6, 0, poses[e % 6]) for e in range(5)]
        first = _wait(server, ids[:2])
        import time
        time.sleep(0.2)
        assert len(ags.ags_server_poll(server)) == 0  # no room until released
        assert ags.ags_server_stats(server)["arena_free_bytes"] < req_bytes
        for rid in ids[:2]:
            ags.ags_server_release(server, rid)
        rest = _wait(server, ids[2:4])
        for rid in ids[2:4]:
            ags.ags_server_release(server, rid)
        _wait(server, ids[4:])
        with pytest.raises(ags.AgsError):
            ags.ags_server_submit(server, 99, 0, poses[0])
        with pytest.raises(ags.AgsError):
            ags.ags_server_submit(server, 0, 5, poses[0])
        assert first and rest
    finally:
        ags.ags_server_destroy(server)


def test_replay_and_sequential_baseline(setup):
    ctx, batch, scene, specs, poses = setup
    rng = np.random.default_rng(4)
    n = 400
    env = rng.integers(0, 6, n)
    sp = rng.integers(0, 3, n)
    reqs = ags.make_requests(env, sp, poses[env])
    arrival = np.cumsum(rng.exponential(1 / 4000.0, n))
    server = ags.ags_server_create(ctx, scene, specs, max_slots=128, max_inflight=2, arena_bytes=64 << 20)
    try:
        out = ags.ags_server_replay(server, reqs, arrival)
    finally:
        ags.ags_server_destroy(server)
    assert (out["status"] == 0).all() and (out["tag"] == np.arange(n)).all()
    lat = out["t_done"] - out["t_submit"]
    assert (lat > 0).all() and (out["t_start"] >= out["t_submit"] - 1e-6).all()
    seq = ags.ags_replay_sequential(ctx, scene, specs, reqs[:100], arrival[:100])
    assert (seq["status"] == 0).all()
    assert ((seq["t_done"] - seq["t_submit"]) > 0).all()


def test_cancel_queued_requests(setup):
    """A queued request can be cancelled (it completes at once, cancelled, with no outputs); a request
    already served cannot."""
    ctx, batch, scene, specs, poses = setup
    # an arena that holds one request at a time keeps the rest queued
    req_bytes = 64 * 48 * 8
    server = ags.ags_server_create(ctx, scene, specs[:1], max_slots=4, max_inflight=1, arena_bytes=req_bytes + 64)
    try:
        ids = [ags.ags_server_submit(server, e % 6, 0, poses[e % 6]) for e in range(6)]
        first = _wait(server, ids[:1])
        cancelled = [rid for rid in ids[2:] if ags.ags_server_cancel(server, rid)]
        assert len(cancelled) >= 3
        assert not ags.ags_server_cancel(server, ids[0])  # already done
        got = _wait(server, cancelled)
        for rid in cancelled:
            c = got[rid]
            assert int(c["status"]) == ags.AGS_ERR_CANCELLED and int(c["depth_dev"]) == 0
        ags.ags_server_release(server, ids[0])
        rest = [rid for rid in ids[1:] if rid not in cancelled]
        done = _wait(server, rest)
        for rid in rest:
            assert int(done[rid]["status"]) == 0
            ags.ags_server_release(server, rid)
        assert first
    finally:
        ags.ags_server_destroy(server)
