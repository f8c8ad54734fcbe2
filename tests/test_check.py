"""The element-wise acceptance rule used by the parity tests (oracle.check)."""
import numpy as np

import oracle as O
from paper_2503_01471_gb300 import scenes as S


def _room_result():
    sc, spec, poses = S.tiny_room()
    vs, ix, ps, sg = sc.env_submeshes(0)
    tris, seg = O.world_triangles(vs, ix, ps, sg)
    s = O.Sensor(O.PINHOLE, spec.width, spec.height, spec.hfov, spec.min_range, spec.max_range)
    return O.render(tris, seg, s, poses[3].astype(np.float64)), spec


def test_exact_answers_accepted():
    res, spec = _room_result()
    v = res["v"].astype(np.float32)
    ok, counted = O.check(res, v, res["seg"], spec.max_range)
    assert ok.all()
    assert counted.mean() < 0.5


def test_planted_errors_rejected():
    res, spec = _room_result()
    v = res["v"].astype(np.float32).astype(np.float64)
    seg = res["seg"].copy()
    hit = np.nonzero((res["seg"] >= 0) & ((res["flags"] & (O.F_COUNTED | O.F_WIDE)) == 0))[0]
    miss = np.nonzero((res["seg"] == -1) & ((res["flags"] & O.F_COUNTED) == 0))[0]
    assert len(hit) > 100
    i, j, k = hit[0], hit[1], hit[2]
    v[i] += 3 * O.tol(v[i])                  # value off by 3 tolerances
    seg[j] = seg[j] + 100                    # wrong segment
    seg[k] = -1                              # a hit reported as a miss
    v[k] = spec.max_range
    if len(miss):
        m = miss[0]
        v[m] = spec.max_range - 1e-3         # a miss with a wrong value
    ok, _ = O.check(res, v, seg, spec.max_range)
    bad = set(np.nonzero(~ok)[0])
    assert {i, j, k} <= bad
    if len(miss):
        assert miss[0] in bad
    assert len(bad) == 3 + (1 if len(miss) else 0)
