/*
 * FP64 brute-force ray-cast oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load
 * this file's library; the product path never does. It shares no code with
 * the CUDA renderer. Everything is double precision and deliberately plain:
 * every ray is tested against every triangle of its environment.
 *
 * Paper: Aerial Gym Simulator (Kulkarni, Rehberg, Alexis; IEEE RA-L 2025),
 * Sec. III-D.1 "Exteroceptive Sensors". Readings of points the paper leaves
 * open are marked "reading:" below.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- a1: per-object transform (Sec. III-D.1, the T o M^base composition) ----
 * reading: each T_{j,t} is a rigid motion given as position p and quaternion q
 * (x, y, z, w); the vertex map is v' = R(q) v + p with q normalised first. */
void orc_rotation(const double q[4], double R[9]) {
  double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double x = q[0] / n, y = q[1] / n, z = q[2] / n, w = q[3] / n;
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - z * w);
  R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w);
  R[7] = 2.0 * (y * z + x * w);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

void orc_transform(const double* v, int64_t n, const double pose[7], double* out) {
  double R[9];
  orc_rotation(pose + 3, R);
  for (int64_t i = 0; i < n; ++i) {
    const double* a = v + 3 * i;
    double* b = out + 3 * i;
    for (int r = 0; r < 3; ++r)
      b[r] = R[3 * r + 0] * a[0] + R[3 * r + 1] * a[1] + R[3 * r + 2] * a[2] + pose[r];
  }
}

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static void matvec(const double R[9], const double a[3], double b[3]) {
  for (int r = 0; r < 3; ++r) b[r] = R[3 * r] * a[0] + R[3 * r + 1] * a[1] + R[3 * r + 2] * a[2];
}

/* ---- a3: one ray per pixel / beam (Sec. III-D.1: a ray leaves the sensor through each pixel) ----
 * reading (camera): body axes +x forward, +y left, +z up; row 0 is the top
 *   image row, column 0 the left column; the ray passes through the pixel
 *   centre; square pixels with focal length f = (W/2)/tan(hfov/2).
 * reading (LiDAR): channel k (row) at elevation vfov_max - k (vfov_max -
 *   vfov_min)/(C-1), both end points included; azimuth bin j (column) at
 *   hfov * j / A counter-clockwise from +x, end point excluded. */
int orc_ray(const orc_sensor* s, const double pose[7], int64_t row, int64_t col,
            double o[3], double d[3], double* scale) {
  if (!s || s->width <= 0 || s->height <= 0 || row < 0 || col < 0 || row >= s->height ||
      col >= s->width)
    return -1;
  double R[9];
  orc_rotation(pose + 3, R);
  o[0] = pose[0];
  o[1] = pose[1];
  o[2] = pose[2];
  double local[3];
  if (s->type == ORC_PINHOLE) {
    double W = (double)s->width, H = (double)s->height;
    double f = (W / 2.0) / tan(s->hfov / 2.0);
    local[0] = 1.0;
    local[1] = -(((double)col + 0.5) - W / 2.0) / f;
    local[2] = -(((double)row + 0.5) - H / 2.0) / f;
    double n = sqrt(dot3(local, local));
    for (int k = 0; k < 3; ++k) local[k] /= n;
    matvec(R, local, d);
    /* optical axis f = R (1,0,0); depth = distance from the image plane = t (d.f) */
    double fwd[3] = {R[0], R[3], R[6]};
    *scale = dot3(d, fwd);
  } else if (s->type == ORC_LIDAR) {
    double C = (double)s->height;
    double phi = (s->height > 1) ? s->vfov_max - (double)row * (s->vfov_max - s->vfov_min) / (C - 1.0)
                                 : s->vfov_max;
    double psi = s->hfov * (double)col / (double)s->width;
    local[0] = cos(phi) * cos(psi);
    local[1] = cos(phi) * sin(psi);
    local[2] = sin(phi);
    matvec(R, local, d);
    *scale = 1.0; /* range = distance between sensor and hit */
  } else if (s->type == ORC_RAY_TABLE && s->dirs) {
    /* Sec. III-D.1 (user-defined sensors with their own projection model):
     * the pixel's direction is given; the value is the distance along it in
     * units of its length, so (1, a, b) rows give depth and unit rows range */
    const double* g = s->dirs + 3 * (row * (int64_t)s->width + col);
    double n = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(n > 0.0) || !isfinite(n)) return -1;
    for (int k = 0; k < 3; ++k) local[k] = g[k] / n;
    matvec(R, local, d);
    *scale = 1.0 / n;
  } else {
    return -1;
  }
  return 0;
}

/* ---- a4-a6: nearest hit over every triangle, then the reported value ----
 * The plain definition: the ray o + t d (t >= 0) hits triangle (v0, v1, v2)
 * iff o + t d = sum_k lambda_k v_k with every lambda_k >= 0 and sum 1.
 * Projecting onto a plane orthogonal to d turns this into a 2-D point-in-
 * triangle test of the origin; the lambdas are the 2-D barycentrics and
 * t = sum_k lambda_k (v_k - o).d. reading: two-sided (no culling), closed
 * edges, zero-area triangles never hit, nearest t wins and equal t goes to
 * the smaller triangle index. */

typedef struct {
  double t_lo, t_hi; /* range of t a perturbed ray could report */
  int32_t seg;
  int32_t tri;
  int32_t sure;      /* every ray within eps hits it inside the valid t range */
  int32_t edge;      /* possible but not geometrically sure */
  int32_t grazing;
} orc_cand;

typedef struct {
  int exact_hit;     /* plain closed test result */
  double t_exact;
  int possible, sure, edge, grazing;
  double t_lo, t_hi;
  double cosn;       /* |n.d| (0 for a zero-area triangle) */
  double vert;       /* the vertex band: how far rounding may move the triangle's plane */
} orc_tri_eval;

static void eval_triangle(const double* tri, const double o[3], const double d[3],
                          const double u[3], const double w[3], double t_far, double et0,
                          double et_far, const orc_sensor* bands, double vert_extra, orc_tri_eval* r) {
  memset(r, 0, sizeof(*r));
  double a[3], b[3], c[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = tri[k] - o[k];
    b[k] = tri[3 + k] - o[k];
    c[k] = tri[6 + k] - o[k];
  }
  double ab[3], ac[3], n[3];
  for (int k = 0; k < 3; ++k) {
    ab[k] = b[k] - a[k];
    ac[k] = c[k] - a[k];
  }
  cross3(ab, ac, n);
  double nn = sqrt(dot3(n, n));
  if (nn == 0.0) return; /* zero-area triangle: never hit */

  /* 2-D coordinates of the vertices in the plane orthogonal to d, and depth along d */
  double pa[2] = {dot3(a, u), dot3(a, w)}, pb[2] = {dot3(b, u), dot3(b, w)},
         pc[2] = {dot3(c, u), dot3(c, w)};
  double za = dot3(a, d), zb = dot3(b, d), zc = dot3(c, d);
  /* e_k: twice the signed area of (origin, edge opposite vertex k) */
  double e0 = pb[0] * pc[1] - pb[1] * pc[0];
  double e1 = pc[0] * pa[1] - pc[1] * pa[0];
  double e2 = pa[0] * pb[1] - pa[1] * pb[0];
  double area2 = e0 + e1 + e2;

  if (area2 != 0.0 && ((e0 >= 0 && e1 >= 0 && e2 >= 0) || (e0 <= 0 && e1 <= 0 && e2 <= 0))) {
    double t = (e0 * za + e1 * zb + e2 * zc) / area2;
    if (t >= 0.0 && t <= t_far) {
      r->exact_hit = 1;
      r->t_exact = t;
    }
  }

  /* Tolerance bands. A single-precision renderer sees each vertex displaced by
   * up to vert (per coordinate: its transform's rounding), its ray direction
   * off by up to dir_rel (relative), and its own intersection arithmetic
   * displacing the ray sideways by up to arith_rel times the distance to the
   * vertices. eps is the sideways band used to decide which triangles such a
   * renderer surely / possibly hits. */
  double cmax = 1.0, rmax = 0.0;
  for (int k = 0; k < 3; ++k) {
    if (fabs(o[k]) > cmax) cmax = fabs(o[k]);
    if (fabs(tri[k]) > cmax) cmax = fabs(tri[k]);
    if (fabs(tri[3 + k]) > cmax) cmax = fabs(tri[3 + k]);
    if (fabs(tri[6 + k]) > cmax) cmax = fabs(tri[6 + k]);
  }
  rmax = fmax(sqrt(dot3(a, a)), fmax(sqrt(dot3(b, b)), sqrt(dot3(c, c))));
  double vert = sqrt(3.0) * bands->vert_rel * cmax + vert_extra;
  r->vert = vert;
  double eps = vert + (bands->dir_rel + bands->arith_rel) * rmax;
  double len0 = hypot(pc[0] - pb[0], pc[1] - pb[1]);
  double len1 = hypot(pa[0] - pc[0], pa[1] - pc[1]);
  double len2 = hypot(pb[0] - pa[0], pb[1] - pa[1]);
  int pos_orient = (e0 >= -eps * len0 && e1 >= -eps * len1 && e2 >= -eps * len2);
  int neg_orient = (e0 <= eps * len0 && e1 <= eps * len1 && e2 <= eps * len2);
  if (!pos_orient && !neg_orient) return;
  double sg = (area2 >= 0.0) ? 1.0 : -1.0;
  int geo_sure = area2 != 0.0 && sg * e0 >= eps * len0 && sg * e1 >= eps * len1 &&
                 sg * e2 >= eps * len2;

  /* Range of t over the perturbations. A ray displaced sideways by e meets
   * the triangle's plane at a t that differs by at most e tan(n, d); the
   * renderer's arithmetic error displaces the ray that way (arith_rel * rmax)
   * and also shifts t along the ray directly (the same amount); moving the
   * plane by vert along its normal moves t by vert / cos(n, d). */
  double cosn = fabs(dot3(n, d)) / nn;
  r->cosn = cosn;
  /* the hit lies in the triangle, so its t is within the vertices' depths,
   * widened by what the bands do to those depths: the vertex band, the
   * direction band over the vertex distance, and the arithmetic band's shift
   * along the ray (together: eps) */
  double zmin = fmin(za, fmin(zb, zc)) - eps, zmax = fmax(za, fmax(zb, zc)) + eps;
  double t_lo = zmin, t_hi = zmax;
  if (area2 != 0.0 && cosn > 0.0) {
    double tc = (e0 * za + e1 * zb + e2 * zc) / area2;
    double ar = bands->arith_rel * rmax;
    /* the sideways effect is bounded two ways; both hold, take the smaller:
     * the plane's slope tan(n, d), and the barycentric bound (a shift moves
     * each barycentric by at most e len_k / |area2| and they sum to one) */
    double tan_n = sqrt(fmax(0.0, 1.0 - cosn * cosn)) / cosn;
    double bary = (len0 * fabs(za - tc) + len1 * fabs(zb - tc) + len2 * fabs(zc - tc)) / fabs(area2);
    double delta = (bands->dir_rel * fabs(tc) + ar) * fmin(tan_n, bary) + ar + vert / cosn;
    double lo = fmax(zmin, tc - delta), hi = fmin(zmax, tc + delta);
    if (lo > hi) {
      double tcc = fmin(fmax(tc, zmin), zmax);
      lo = hi = tcc;
    }
    t_lo = lo;
    t_hi = hi;
  }
  if (t_hi < -et0 || t_lo > t_far + et_far) return;
  r->possible = 1;
  r->sure = geo_sure && t_lo >= et0 && t_hi <= t_far - et_far;
  r->edge = !geo_sure;
  r->grazing = cosn < 1e-3;
  r->t_lo = t_lo;
  r->t_hi = t_hi;
}

static double tolv(double v) { return 1e-5 * fabs(v) + 1e-6; }

#define ORC_LIST_CAP 512

static void render_one(const double* tris, const int32_t* seg, int64_t F, const orc_sensor* s,
                       const double pose[7], int64_t ray, orc_result* res, orc_cand* list) {
  memset(res, 0, sizeof(*res));
  int64_t row = ray / s->width, col = ray % s->width;
  double o[3], d[3], scale;
  orc_ray(s, pose, row, col, o, d, &scale);

  /* orthonormal basis (u, w) of the plane orthogonal to d */
  double h[3] = {0, 0, 0};
  int kmin = 0;
  for (int k = 1; k < 3; ++k)
    if (fabs(d[k]) < fabs(d[kmin])) kmin = k;
  h[kmin] = 1.0;
  double u[3], w[3];
  cross3(d, h, u);
  double un = sqrt(dot3(u, u));
  for (int k = 0; k < 3; ++k) u[k] /= un;
  cross3(d, u, w);

  /* reading: the max applies to the reported value (depth for a camera) */
  double t_far = s->max_range / scale;
  double et0 = 1e-6 / scale, et_far = tolv(s->max_range) / scale;

  double best_t = INFINITY;
  int64_t best_i = -1;
  double best_cos = 0.0, best_lo = 0.0, best_hi = 0.0, best_vert = 0.0;
  double sure_thi = INFINITY;
  int n_list = 0, list_overflow = 0;

  orc_tri_eval ev;
  for (int64_t i = 0; i < F; ++i) {
    eval_triangle(tris + 9 * i, o, d, u, w, t_far, et0, et_far, s, 0.0, &ev);
    if (ev.exact_hit && (ev.t_exact < best_t || (ev.t_exact == best_t && i < best_i))) {
      best_t = ev.t_exact;
      best_i = i;
      best_cos = ev.cosn;
      best_vert = ev.vert;
      best_lo = ev.t_lo;
      best_hi = ev.t_hi;
    }
    if (!ev.possible) continue;
    if (ev.sure && ev.t_hi < sure_thi) sure_thi = ev.t_hi;
    double bound = sure_thi + tolv(sure_thi * scale) / scale;
    if (ev.t_lo > bound) continue;
    if (n_list == ORC_LIST_CAP) {
      /* drop entries that can no longer qualify (the bound only shrinks) */
      int m = 0;
      for (int k = 0; k < n_list; ++k)
        if (list[k].t_lo <= bound) list[m++] = list[k];
      n_list = m;
      if (n_list == ORC_LIST_CAP) {
        list_overflow = 1;
        continue;
      }
    }
    orc_cand* c = &list[n_list++];
    c->t_lo = ev.t_lo;
    c->t_hi = ev.t_hi;
    c->seg = seg[i];
    c->tri = (int32_t)i;
    c->sure = ev.sure;
    c->edge = ev.edge;
    c->grazing = ev.grazing;
  }

  /* exact answer (a6): value, clamp, miss */
  res->t_hit = best_i >= 0 ? best_t : INFINITY;
  if (best_i >= 0) {
    res->cos_hit = best_cos;
    res->hit_dev = fmax(best_t - best_lo, best_hi - best_t) * scale;
  }
  if (best_i >= 0) {
    double v = best_t * scale;
    if (v > s->max_range) v = s->max_range;
    res->v = v;
    res->seg = seg[best_i];
    res->tri = (int32_t)best_i;
    if (v < s->min_range) {
      if (s->near_mode == ORC_NEAR_CLAMP) {
        res->v = s->min_range;
      } else {
        res->v = s->max_range;
        res->seg = -1;
        res->tri = -1;
      }
    }
  } else {
    res->v = s->max_range;
    res->seg = -1;
    res->tri = -1;
  }

  /* acceptable outcomes, grouped by segment */
  int flags = 0;
  int miss_ok = (sure_thi == INFINITY);
  double bound = sure_thi + tolv(sure_thi * scale) / scale;
  int32_t sure_seg0 = -1;
  int n_sure_segs = 0;
  for (int k = 0; k < n_list; ++k) {
    orc_cand* c = &list[k];
    if (c->t_lo > bound) continue;
    if (c->edge) flags |= ORC_F_SILHOUETTE;
    /* geometrically sure but its t band crosses the sensor's origin or the
     * far limit: hit vs miss is open there */
    if (!c->sure && !c->edge) flags |= ORC_F_RANGE_EDGE;
    if (c->sure) {
      if (n_sure_segs == 0) {
        sure_seg0 = c->seg;
        n_sure_segs = 1;
      } else if (c->seg != sure_seg0) {
        n_sure_segs = 2;
      }
    }
    double vlo = fmax(c->t_lo, 0.0) * scale, vhi = c->t_hi * scale;
    if (vhi >= s->max_range - tolv(s->max_range)) flags |= ORC_F_RANGE_EDGE;
    if (vhi > s->max_range) vhi = s->max_range;
    if (vlo > vhi) vlo = vhi;
    if (vlo < s->min_range + tolv(s->min_range)) {
      if (s->near_mode == ORC_NEAR_CLAMP) {
        vlo = fmax(vlo, s->min_range);
        vhi = fmax(vhi, s->min_range);
      } else {
        flags |= ORC_F_RANGE_EDGE;
        miss_ok = 1;
        if (vhi < s->min_range) continue;
        vlo = fmax(vlo, s->min_range);
      }
    }
    if (res->n_tri < ORC_MAX_TRI)
      res->cand_tri[res->n_tri++] = c->tri;
    else
      flags |= ORC_F_TRI_OVERFLOW;
    int g;
    for (g = 0; g < res->n_cand; ++g)
      if (res->cand_seg[g] == c->seg) break;
    if (g < res->n_cand) {
      res->cand_lo[g] = fmin(res->cand_lo[g], vlo);
      res->cand_hi[g] = fmax(res->cand_hi[g], vhi);
    } else if (res->n_cand < ORC_MAX_CAND) {
      res->cand_seg[g] = c->seg;
      res->cand_lo[g] = vlo;
      res->cand_hi[g] = vhi;
      res->n_cand++;
    } else {
      flags |= ORC_F_OVERFLOW;
    }
  }
  if (list_overflow) flags |= ORC_F_OVERFLOW;
  if (n_sure_segs > 1) flags |= ORC_F_NEAR_TIE;
  if (miss_ok) flags |= ORC_F_MISS_OK;
  int outcomes = res->n_cand + (miss_ok ? 1 : 0);
  for (int g = 0; g < res->n_cand; ++g)
    if (res->cand_hi[g] - res->cand_lo[g] > 2.0 * tolv(res->cand_hi[g])) flags |= ORC_F_WIDE;

  /* Counting. A ray is held to the tolerance around the exact answer unless
   * one of these reasons applies; then any outcome the bands allow is
   * accepted and the ray is counted:
   *  - several outcomes (a silhouette, a near tie or a range edge above);
   *  - grazing: the exact hit surface meets the ray so obliquely that the
   *    direction band alone moves the hit by more than the relative
   *    tolerance: a tilt of dir_rel moves it by t dir_rel tan(theta), above
   *    1e-5 t once tan(theta) > 1e-5 / dir_rel (|n.d| < 0.06 for 6e-7);
   *  - coarse: the vertex band of the hit triangle (the float32 spacing of
   *    its coordinates) is above the tolerance at the hit's value, so no
   *    float32 scene can place that surface within it, at any incidence. */
  if (outcomes > 1) flags |= ORC_F_COUNTED;
  if (best_i >= 0 && res->seg >= 0) {
    const double cos_graze = s->dir_rel / sqrt(s->dir_rel * s->dir_rel + 1e-10);
    if (best_cos < cos_graze) flags |= ORC_F_GRAZING | ORC_F_COUNTED;
    if (best_vert * scale > tolv(res->v)) flags |= ORC_F_COARSE | ORC_F_COUNTED;
  }
  res->flags = flags;
}

/* a sensor the oracle can cast every listed ray of */
static int sensor_ok(const orc_sensor* s, const int64_t* rays, int64_t n_rays) {
  if (s->width <= 0 || s->height <= 0) return 0;
  if (s->type != ORC_PINHOLE && s->type != ORC_LIDAR && !(s->type == ORC_RAY_TABLE && s->dirs)) return 0;
  int64_t n_pix = (int64_t)s->width * s->height;
  double o[3], d[3], scale, pose[7] = {0, 0, 0, 0, 0, 0, 1};
  for (int64_t i = 0; i < n_rays; ++i) {
    if (rays[i] < 0 || rays[i] >= n_pix) return 0;
    if (s->type == ORC_RAY_TABLE && orc_ray(s, pose, rays[i] / s->width, rays[i] % s->width, o, d, &scale) != 0)
      return 0;
  }
  return 1;
}

int orc_render(const double* tris, const int32_t* seg, int64_t F, const orc_sensor* s,
               const double pose[7], const int64_t* rays, int64_t n_rays, orc_result* out) {
  if (!s || !pose || !out || (F > 0 && (!tris || !seg)) || F < 0 || n_rays < 0) return -1;
  if (n_rays > 0 && !rays) return -1;
  if (!sensor_ok(s, rays, n_rays)) return -1;
#pragma omp parallel
  {
    orc_cand list[ORC_LIST_CAP];
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < n_rays; ++i) render_one(tris, seg, F, s, pose, rays[i], &out[i], list);
  }
  return 0;
}

/* ---- extra hit channels (Sec. III-D.1: the index of the face hit with the
 * barycentric coordinates of the hit, point clouds, surface normals) ----
 * reading: the face index is the env-local triangle index; the barycentrics
 * are those of the point where the ray meets the face's plane, weights of its
 * second and third vertex; the normal is the face's geometric normal turned
 * towards the sensor (meshes are two-sided); the point is the hit in the
 * sensor frame, consistent with the reported value. */
static void sensor_local(const orc_sensor* s, int64_t row, int64_t col, double local[3]) {
  if (s->type == ORC_RAY_TABLE) {
    /* the given direction: distance along it is the reported value */
    for (int k = 0; k < 3; ++k) local[k] = s->dirs[3 * (row * (int64_t)s->width + col) + k];
  } else if (s->type == ORC_PINHOLE) {
    /* the camera ray through the pixel centre, scaled to unit forward component */
    double W = (double)s->width, H = (double)s->height;
    double f = (W / 2.0) / tan(s->hfov / 2.0);
    local[0] = 1.0;
    local[1] = (W / 2.0 - ((double)col + 0.5)) / f;
    local[2] = (H / 2.0 - ((double)row + 0.5)) / f;
  } else {
    double C = (double)s->height;
    double phi = (s->height > 1) ? s->vfov_max - (double)row * (s->vfov_max - s->vfov_min) / (C - 1.0)
                                 : s->vfov_max;
    double psi = s->hfov * (double)col / (double)s->width;
    local[0] = cos(phi) * cos(psi);
    local[1] = cos(phi) * sin(psi);
    local[2] = sin(phi);
  }
}

int orc_hit_channels(const double* tris, int64_t F, const orc_sensor* s, const double pose[7],
                     const int64_t* rays, const int32_t* face, const double* v, int64_t n,
                     double* bary, double* normal, double* point) {
  if (!s || !pose || n < 0 || (n > 0 && (!rays || !face || !v || !bary || !normal || !point))) return -1;
  if (!sensor_ok(s, rays, n)) return -1;
  for (int64_t i = 0; i < n; ++i) {
    if (face[i] >= F) return -1;
    int64_t row = rays[i] / s->width, col = rays[i] % s->width;
    double local[3];
    sensor_local(s, row, col, local);
    for (int k = 0; k < 3; ++k) point[3 * i + k] = v[i] * local[k];
    for (int k = 0; k < 2; ++k) bary[2 * i + k] = 0.0;
    for (int k = 0; k < 3; ++k) normal[3 * i + k] = 0.0;
    if (face[i] < 0) continue;
    double o[3], d[3], scale;
    if (orc_ray(s, pose, row, col, o, d, &scale) != 0) return -1;
    const double* tri = tris + 9 * (int64_t)face[i];
    double e1[3], e2[3], nrm[3], q[3];
    for (int k = 0; k < 3; ++k) {
      e1[k] = tri[3 + k] - tri[k];
      e2[k] = tri[6 + k] - tri[k];
      q[k] = o[k] - tri[k];
    }
    cross3(e1, e2, nrm);
    double nn = sqrt(dot3(nrm, nrm));
    double nd = dot3(nrm, d);
    if (nn == 0.0 || nd == 0.0) return -1;
    /* the plane point o + t d with t = -(q.n)/(d.n), then its barycentrics
     * from the areas of the sub-triangles it spans with the edges */
    double t = -dot3(q, nrm) / nd;
    double x[3], c1[3], c2[3];
    for (int k = 0; k < 3; ++k) x[k] = q[k] + t * d[k]; /* hit point relative to v0 */
    cross3(x, e2, c1);
    cross3(e1, x, c2);
    bary[2 * i] = dot3(c1, nrm) / (nn * nn);
    bary[2 * i + 1] = dot3(c2, nrm) / (nn * nn);
    double sgn = nd > 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < 3; ++k) normal[3 * i + k] = sgn * nrm[k] / nn;
  }
  return 0;
}

/* ---- stereo shadows (Sec. III-D.1: rays projected back from the points of
 * intersection towards the second sensor; pixels whose ray meets the
 * environment are invalid) ----
 * reading: the second sensor sits at o2 = p + R(q) b (b in the sensor frame);
 * the pixel is shadowed when a triangle meets the segment P + s (o2 - P) at
 * some s in [eps, 1], where P is the exact hit; eps keeps the surface at P
 * itself out. The verdict is banded like a render: the renderer's P may sit
 * up to e_P from the exact one, so every triangle is judged with that much
 * extra vertex displacement; a triangle possibly but not surely on the
 * segment makes the verdict "either". */
static void orthobasis(const double d[3], double u[3], double w[3]) {
  double h[3] = {0, 0, 0};
  int kmin = 0;
  for (int k = 1; k < 3; ++k)
    if (fabs(d[k]) < fabs(d[kmin])) kmin = k;
  h[kmin] = 1.0;
  cross3(d, h, u);
  double un = sqrt(dot3(u, u));
  for (int k = 0; k < 3; ++k) u[k] /= un;
  cross3(d, u, w);
}

int orc_shadow(const double* tris, int64_t F, const orc_sensor* s, const double pose[7],
               const double baseline[3], double eps, const int64_t* rays, const orc_result* res,
               int64_t n, int32_t* out) {
  if (!s || !pose || !baseline || n < 0 || (n > 0 && (!rays || !res || !out)) || (F > 0 && !tris)) return -1;
  if (!sensor_ok(s, rays, n)) return -1;
  if (!(eps >= 0.0 && eps < 1.0)) return -1;
  double R[9];
  orc_rotation(pose + 3, R);
  double o2[3];
  matvec(R, baseline, o2);
  for (int k = 0; k < 3; ++k) o2[k] += pose[k];
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    out[i] = 0;
    if (res[i].seg < 0 || !(res[i].t_hit < INFINITY)) continue;
    int64_t row = rays[i] / s->width, col = rays[i] % s->width;
    double o[3], d[3], scale;
    orc_ray(s, pose, row, col, o, d, &scale);
    double P[3], seg[3];
    for (int k = 0; k < 3; ++k) {
      P[k] = o[k] + res[i].t_hit * d[k];
      seg[k] = o2[k] - P[k];
    }
    double L = sqrt(dot3(seg, seg));
    if (L == 0.0) continue;
    double dir[3], start[3], u[3], w[3];
    for (int k = 0; k < 3; ++k) {
      dir[k] = seg[k] / L;
      start[k] = P[k] + eps * L * dir[k];
    }
    orthobasis(dir, u, w);
    /* how far the renderer's P may sit from the exact one: the value
     * tolerance along the ray, the direction and arithmetic bands across it,
     * and float32 rounding of the segment's ends */
    double pmax = 1.0;
    for (int k = 0; k < 3; ++k) pmax = fmax(pmax, fmax(fabs(P[k]), fabs(o2[k])));
    double e_p = tolv(res[i].t_hit * scale) / scale + 4.0 * (s->dir_rel + s->arith_rel) * res[i].t_hit +
                 8.0 * 5.9604644775390625e-8 * pmax;
    double t_far = (1.0 - eps) * L;
    int verdict = 0;
    orc_tri_eval ev;
    for (int64_t f = 0; f < F && verdict != 1; ++f) {
      eval_triangle(tris + 9 * f, start, dir, u, w, t_far, e_p, e_p, s, e_p, &ev);
      if (ev.possible) verdict = (ev.sure && !ev.grazing) ? 1 : 2;
    }
    out[i] = verdict;
  }
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
