"""The element-wise acceptance rule used by the parity tests (oracle.check).

Each ``_rule_*`` check takes an acceptance function with oracle.check's
signature, so the same checks run against the real rule and against planted
mistakes in its source (the last test): a rule that is too loose or too
strict fails at least one of them.
"""
import inspect
import types

import numpy as np
import pytest

import oracle as O
from paper_2503_01471_gb300 import scenes as S


def _room_result():
    sc, spec, poses = S.tiny_room()
    vs, ix, ps, sg = sc.env_submeshes(0)
    tris, seg = O.world_triangles(vs, ix, ps, sg)
    s = O.Sensor(O.PINHOLE, spec.width, spec.height, spec.hfov, spec.min_range, spec.max_range)
    return O.render(tris, seg, s, poses[3].astype(np.float64)), spec


def _obstacle_results():
    """Oracle results of two obstacle rooms (every ray), with more counted rays than the tiny room."""
    batch, spec, poses = S.obstacle_rooms(2, steps=1, width=64, height=48)
    out = []
    for e in range(2):
        vs, ix, ps, sg = batch.env_submeshes(e)
        tris, seg = O.world_triangles(vs, ix, ps, sg)
        s = O.Sensor(O.PINHOLE, spec.width, spec.height, spec.hfov, spec.min_range, spec.max_range)
        out.append(O.render(tris, seg, s, np.asarray(poses[0][e], np.float32).astype(np.float64)))
    return np.concatenate(out), spec


def _rule_exact_answers_accepted(check):
    res, spec = _room_result()
    ok, counted = check(res, res["v"].astype(np.float32), res["seg"], spec.max_range)
    assert ok.all()
    # every counted ray names its reason, and they are rare
    assert np.all((res["flags"][counted] & O.F_REASONS) != 0)
    assert counted.sum() <= 0.01 * counted.size
    res, spec = _obstacle_results()
    ok, counted = check(res, res["v"].astype(np.float32), res["seg"], spec.max_range)
    assert ok.all()
    assert np.all((res["flags"][counted] & O.F_REASONS) != 0)
    assert counted.sum() <= 0.01 * counted.size


def _rule_planted_errors_rejected(check):
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
    ok, _ = check(res, v, seg, spec.max_range)
    bad = set(np.nonzero(~ok)[0])
    assert {i, j, k} <= bad
    if len(miss):
        assert miss[0] in bad
    assert len(bad) == 3 + (1 if len(miss) else 0)


def _rule_uncounted_held_to_tolerance_not_band(check):
    """An uncounted ray whose float32 band is wider than the tolerance is still held to the tolerance: a
    value inside the band but 1.3 tolerances from the exact one fails; 0.9 tolerances passes."""
    res, spec = _obstacle_results()
    wide = np.nonzero(((res["flags"] & O.F_WIDE) != 0) & ((res["flags"] & O.F_COUNTED) == 0)
                      & (res["seg"] >= 0) & (res["n_cand"] == 1))[0]
    up = res["cand_hi"][wide, 0] - res["v"][wide] > 1.35 * O.tol(res["v"][wide])
    down = res["v"][wide] - res["cand_lo"][wide, 0] > 1.35 * O.tol(res["v"][wide])
    keep = up | down
    assert keep.sum() >= 5
    sub = res[wide[keep]]
    sign = np.where(up[keep], 1.0, -1.0)
    far = sub["v"] + sign * 1.3 * O.tol(sub["v"])
    assert np.all((far <= sub["cand_hi"][:, 0]) & (far >= sub["cand_lo"][:, 0]))  # inside the band
    ok, counted = check(sub, far, sub["seg"], spec.max_range)
    assert not counted.any() and not ok.any()
    near = sub["v"] + sign * 0.9 * O.tol(sub["v"])
    ok, _ = check(sub, near, sub["seg"], spec.max_range)
    assert ok.all()


def _rule_counted_held_to_listed_outcomes(check):
    """A counted ray may give any listed outcome, but not a value beyond its group's band (either side), a
    segment no group has, or a miss where none is allowed."""
    res, spec = _obstacle_results()
    cnt = np.nonzero(((res["flags"] & O.F_COUNTED) != 0) & (res["n_cand"] >= 1))[0]
    assert len(cnt) >= 3
    sub = res[cnt]
    lo, hi, sg = sub["cand_lo"][:, 0], sub["cand_hi"][:, 0], sub["cand_seg"][:, 0]
    ok, counted = check(sub, hi, sg, spec.max_range)
    assert ok.all() and counted.all()
    ok, _ = check(sub, lo, sg, spec.max_range)
    assert ok.all()
    ok, _ = check(sub, hi + 3 * O.tol(hi), sg, spec.max_range)
    assert not ok.any()
    ok, _ = check(sub, lo - 3 * O.tol(lo), sg, spec.max_range)
    assert not ok.any()
    ok, _ = check(sub, lo, sg + 1000, spec.max_range)
    assert not ok.any()
    no_miss = (sub["flags"] & O.F_MISS_OK) == 0
    if no_miss.any():
        ok, _ = check(sub[no_miss], np.full(int(no_miss.sum()), spec.max_range),
                      np.full(int(no_miss.sum()), -1), spec.max_range)
        assert not ok.any()


RULES = [_rule_exact_answers_accepted, _rule_planted_errors_rejected, _rule_uncounted_held_to_tolerance_not_band,
         _rule_counted_held_to_listed_outcomes]


@pytest.mark.parametrize("rule", RULES, ids=[r.__name__ for r in RULES])
def test_acceptance_rule(rule):
    rule(O.check)


# planted mistakes in oracle.check's own source
CHECK_MUTANTS = {
    "ignores_band_top": ("(v <= hi + tol(hi))", "(v <= np.inf)"),
    "ignores_band_bottom": ("(v >= lo - tol(lo))", "(v >= -np.inf)"),
    "band_for_uncounted_rays": ("ok = np.where(counted, listed, exact)", "ok = np.where(counted, listed, listed)"),
    "segment_free_for_uncounted_rays": ("(s == res[\"seg\"]) & (np.abs", "(np.abs"),
    "tolerance_tenfold": ("(np.abs(v - res[\"v\"]) <= tol(res[\"v\"]))", "(np.abs(v - res[\"v\"]) <= 10 * tol(res[\"v\"]))"),
    "miss_always_allowed": ("(is_miss & ((flags & F_MISS_OK) != 0))", "(is_miss)"),
    "any_segment_for_counted": ("(res[\"cand_seg\"][:, k] == s) & ", ""),
}


@pytest.mark.parametrize("name", sorted(CHECK_MUTANTS))
def test_check_mutant_is_caught(name):
    old, new = CHECK_MUTANTS[name]
    src = inspect.getsource(O.check)
    assert src.count(old) == 1, f"mutation site of {name} not found"
    mod = types.ModuleType("check_mutant")
    mod.__dict__.update({k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
    exec(compile(src.replace(old, new), "check_mutant", "exec"), mod.__dict__)
    for rule in RULES:
        try:
            rule(mod.check)
        except AssertionError:
            return
    pytest.fail(f"no acceptance rule catches {name}")
