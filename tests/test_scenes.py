"""The seeded input generators follow the stated recipe: seeds, object counts, triangle counts, segment
IDs, pose ranges and sensor shapes (CPU only; nothing here renders)."""
import math

import numpy as np

from paper_2503_01471_gb300 import scenes as S


def _env_objects(batch, e):
    return int(batch.env_sub[e + 1] - batch.env_sub[e])


def test_obstacle_rooms_recipe_and_seeds():
    b, spec, poses = S.obstacle_rooms(12, steps=20)
    again, _, poses2 = S.obstacle_rooms(12, steps=20)
    for name in ("vertices", "indices", "sub_vert", "sub_tri", "sub_seg", "env_sub", "poses"):
        assert np.array_equal(getattr(b, name), getattr(again, name)), name
    assert np.array_equal(poses, poses2)
    # one environment alone has exactly its content in the full batch
    one, _, p_one = S.obstacle_rooms(12, steps=20, envs=[7])
    vs, ix, ps, sg = b.env_submeshes(7)
    vs1, ix1, ps1, sg1 = one.env_submeshes(0)
    assert all(np.array_equal(x, y) for x, y in zip(vs, vs1)) and np.array_equal(ps, ps1)
    assert np.array_equal(sg, sg1) and np.array_equal(poses[:, 7], p_one[:, 0])
    for e in range(b.n_envs):
        n = _env_objects(b, e) - 1
        assert 20 <= n <= 40
        _, ix, ps, sg = b.env_submeshes(e)
        assert ix[0].shape[0] == 12 and sg[0] == 0                 # the room: 6 walls, segment 0
        assert list(sg[1:]) == list(range(1, n + 1))               # obstacles 1..n
        assert {x.shape[0] for x in ix[1:]} <= {12, 320, 128, 2048}  # box, icosphere, cylinder, panel
        assert np.allclose(np.linalg.norm(ps[:, 3:], axis=1), 1.0, atol=1e-6)
        assert (np.abs(ps[1:, :2]) <= S.ROOM_HALF_XY).all() and (ps[1:, 2] >= 0).all()
        assert (ps[1:, 2] <= S.ROOM_HEIGHT).all()
    # sensor: 480x270 pinhole, 87 degrees, 0.2-10 m; the walk stays 0.3 m inside the walls
    assert (spec.width, spec.height, spec.type) == (480, 270, 0)
    assert math.isclose(spec.hfov, math.radians(87.0), rel_tol=1e-9)
    assert (spec.min_range, spec.max_range) == (0.2, 10.0)
    assert poses.shape == (20, 12, 7)
    m = S.WALL_MARGIN - 1e-6
    assert (np.abs(poses[..., :2]) <= S.ROOM_HALF_XY - m).all()
    assert (poses[..., 2] >= m).all() and (poses[..., 2] <= S.ROOM_HEIGHT - m).all()
    assert np.allclose(np.linalg.norm(poses[..., 3:], axis=-1), 1.0, atol=1e-6)
    # mean triangles per environment near the stated ~18.8k (20-40 obstacles of mean ~627 triangles)
    assert 10_000 < b.env_tri_counts().mean() < 30_000


def test_tiny_room_recipe():
    b, spec, poses = S.tiny_room()
    assert b.n_envs == 1 and int(b.env_tri_counts()[0]) == 12 + 8 * 12
    assert list(b.sub_seg) == list(range(9))
    assert (spec.width, spec.height) == (64, 48) and poses.shape == (16, 7)


def test_lidar_forest_recipe():
    b, spec, poses = S.lidar_forests(3, steps=4)
    for e in range(b.n_envs):
        n = _env_objects(b, e) - 1
        assert 50 <= n <= 200
        _, ix, ps, sg = b.env_submeshes(e)
        assert ix[0].shape[0] == 2 and sg[0] == 0                  # the ground
        counts = np.array([x.shape[0] for x in ix[1:]])
        assert (counts >= 1900).all() and (counts <= 10100).all()  # trunk + cones near the drawn target
        assert (np.abs(ps[1:, :2]) <= 20.0).all() and (ps[1:, 2] == 0).all()
    assert (spec.type, spec.width, spec.height) == (1, 512, 64)
    assert math.isclose(spec.vfov_min, math.radians(-22.5)) and math.isclose(spec.vfov_max, math.radians(22.5))
    assert (poses[..., 2] == np.float32(1.5)).all() and (np.abs(poses[..., :2]) <= 18.0 + 1e-6).all()


def test_serving_rooms_triangle_range():
    b, poses = S.serving_rooms(24)
    t = b.env_tri_counts()
    assert (t >= 1000).all() and (t <= 200_000 + 2048).all()   # the last object may overshoot its target
    assert poses.shape == (1, 24, 7)


def test_sensor_helpers():
    d = S.dome_lidar(128, 32)
    assert math.isclose(d.vfov_min, 0.0) and math.isclose(d.vfov_max, math.radians(90.0))
    table = S.fisheye_table(64, 48)
    assert table.shape == (48, 64, 3) and np.isfinite(table).all()
    assert np.allclose(np.linalg.norm(table, axis=-1), 1.0, atol=1e-5)
