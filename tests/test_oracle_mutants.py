"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Every mutant is a one-line textual change of oracle/oracle.c compiled into a
temporary library; the pins of oracle_pins.py must reject all of them. This
shows the pins constrain every step the oracle takes (transform, ray
generation, intersection, nearest-hit resolution, reported value).
"""
import os
import subprocess

import pytest

import oracle as O
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

MUTANTS = {
    "rotation_sign": ("R[1] = 2.0 * (x * y - z * w);", "R[1] = 2.0 * (x * y + z * w);"),
    "rotation_transposed": ("b[r] = R[3 * r + 0] * a[0] + R[3 * r + 1] * a[1] + R[3 * r + 2] * a[2] + pose[r];",
                            "b[r] = R[r] * a[0] + R[3 + r] * a[1] + R[6 + r] * a[2] + pose[r];"),
    "no_translation": ("R[3 * r + 2] * a[2] + pose[r];", "R[3 * r + 2] * a[2];"),
    "no_normalise": ("double x = q[0] / n, y = q[1] / n, z = q[2] / n, w = q[3] / n;",
                     "double x = q[0], y = q[1], z = q[2], w = q[3]; (void)n;"),
    "pixel_corner_not_centre": ("local[1] = -(((double)col + 0.5) - W / 2.0) / f;",
                                "local[1] = -(((double)col) - W / 2.0) / f;"),
    "row_flipped": ("local[2] = -(((double)row + 0.5) - H / 2.0) / f;",
                    "local[2] = (((double)row + 0.5) - H / 2.0) / f;"),
    "depth_reported_as_range": ("*scale = dot3(d, fwd);", "*scale = 1.0;"),
    "lidar_rows_upside_down": ("s->vfov_max - (double)row * (s->vfov_max - s->vfov_min) / (C - 1.0)",
                               "s->vfov_min + (double)row * (s->vfov_max - s->vfov_min) / (C - 1.0)"),
    "lidar_azimuth_clockwise": ("local[1] = cos(phi) * sin(psi);", "local[1] = -cos(phi) * sin(psi);"),
    "backface_culling": ("if (area2 != 0.0 && ((e0 >= 0 && e1 >= 0 && e2 >= 0) || (e0 <= 0 && e1 <= 0 && e2 <= 0))) {",
                         "if (area2 != 0.0 && ((e0 >= 0 && e1 >= 0 && e2 >= 0))) {"),
    "open_edges": ("if (area2 != 0.0 && ((e0 >= 0 && e1 >= 0 && e2 >= 0) || (e0 <= 0 && e1 <= 0 && e2 <= 0))) {",
                   "if (area2 != 0.0 && ((e0 > 0 && e1 > 0 && e2 > 0) || (e0 < 0 && e1 < 0 && e2 < 0))) {"),
    "t_wrong_vertex": ("    double t = (e0 * za + e1 * zb + e2 * zc) / area2;",
                       "    double t = (e0 * za + e1 * zc + e2 * zb) / area2;"),
    "farthest_not_nearest": ("if (ev.exact_hit && (ev.t_exact < best_t ||", "if (ev.exact_hit && (ev.t_exact > -best_t ||"),
    "tie_to_larger_index": ("(ev.t_exact == best_t && i < best_i)", "(ev.t_exact == best_t && (i > best_i || best_i < 0))"),
    "no_near_clamp": ("        res->v = s->min_range;\n", "        res->v = v;\n"),
    "miss_value_zero": ("  } else {\n    res->v = s->max_range;", "  } else {\n    res->v = 0.0;"),
    "max_applies_to_range": ("double t_far = s->max_range / scale;", "double t_far = s->max_range;"),
    "hits_behind_sensor": ("    if (t >= 0.0 && t <= t_far) {", "    if (t <= t_far) {"),
    "degenerate_hits": ("  if (nn == 0.0) return; /* zero-area triangle: never hit */", "  if (nn < 0.0) return;"),
    "bary_swapped": ("bary[2 * i] = dot3(c1, nrm) / (nn * nn);", "bary[2 * i] = dot3(c2, nrm) / (nn * nn);"),
    "normal_not_turned": ("double sgn = nd > 0.0 ? -1.0 : 1.0;", "double sgn = 1.0;"),
    "point_scaled_as_range": ("point[3 * i + k] = v[i] * local[k];",
                              "point[3 * i + k] = v[i] * local[k] / sqrt(dot3(local, local));"),
    "point_pixel_corner": ("local[1] = (W / 2.0 - ((double)col + 0.5)) / f;", "local[1] = (W / 2.0 - (double)col) / f;"),
    "candidate_triangle_dropped": ("res->cand_tri[res->n_tri++] = c->tri;", "res->cand_tri[res->n_tri] = c->tri;"),
    "baseline_in_world_frame": ("  matvec(R, baseline, o2);\n", "  for (int k = 0; k < 3; ++k) o2[k] = baseline[k];\n"),
    "shadow_from_sensor_origin": ("      P[k] = o[k] + res[i].t_hit * d[k];", "      P[k] = o[k];"),
    "shadow_without_eps": ("      start[k] = P[k] + eps * L * dir[k];", "      start[k] = P[k];"),
    "shadow_segment_too_long": ("    double t_far = (1.0 - eps) * L;", "    double t_far = 2.0 * L;"),
    "ray_table_scale_inverted": ("    *scale = 1.0 / n;", "    *scale = n;"),
    "ray_table_not_normalised": ("    for (int k = 0; k < 3; ++k) local[k] = g[k] / n;", "    for (int k = 0; k < 3; ++k) local[k] = g[k];"),
    # the error bands and the counting reasons
    "band_delta_inflated": ("double delta = (bands->dir_rel * fabs(tc) + ar) * fmin(tan_n, bary) + ar + vert / cosn;",
                            "double delta = 10.0 * ((bands->dir_rel * fabs(tc) + ar) * fmin(tan_n, bary) + ar + vert / cosn);"),
    "band_vertex_term_without_cos": ("* fmin(tan_n, bary) + ar + vert / cosn;", "* fmin(tan_n, bary) + ar + vert;"),
    "band_without_sideways_slope": ("* fmin(tan_n, bary) + ar + vert / cosn;", "* 0.0 + ar + vert / cosn;"),
    "band_without_direction_term": ("double delta = (bands->dir_rel * fabs(tc) + ar)", "double delta = (ar)"),
    "band_depth_clamp_without_eps": ("double zmin = fmin(za, fmin(zb, zc)) - eps, zmax = fmax(za, fmax(zb, zc)) + eps;",
                                     "double zmin = fmin(za, fmin(zb, zc)) - vert, zmax = fmax(za, fmax(zb, zc)) + vert;"),
    "eps_doubled": ("double eps = vert + (bands->dir_rel + bands->arith_rel) * rmax;",
                    "double eps = 2.0 * (vert + (bands->dir_rel + bands->arith_rel) * rmax);"),
    "eps_halved": ("double eps = vert + (bands->dir_rel + bands->arith_rel) * rmax;",
                   "double eps = 0.5 * (vert + (bands->dir_rel + bands->arith_rel) * rmax);"),
    "grazing_reason_dropped": ("if (best_cos < cos_graze) flags |=", "if (best_cos < 0.0) flags |="),
    "grazing_bound_tenfold": ("if (best_cos < cos_graze) flags |=", "if (best_cos < 10.0 * cos_graze) flags |="),
    "coarse_reason_dropped": ("if (best_vert * scale > tolv(res->v)) flags |=", "if (best_vert * scale > 1e9) flags |="),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / "oracle.c"
    cpath.write_text(mutated)
    hdr = os.path.join(os.path.dirname(SRC), "oracle.h")
    (tmp_path / "oracle.h").write_text(open(hdr).read())
    lib_path = str(tmp_path / "libmut.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                    str(cpath), "-o", lib_path, "-lm"], check=True)
    lib = O.load(lib_path)
    for pin in ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError, FloatingPointError, IndexError):
            return  # caught
    pytest.fail(f"no pin catches mutant {name}")
