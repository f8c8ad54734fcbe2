/*
 * FP64 brute-force ray-cast oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library. The product (the CUDA renderer behind include/ags.h) never
 * calls it and shares no code, header or constant with it.
 *
 * What it computes (Aerial Gym Simulator, Sec. III-D.1 "Exteroceptive Sensors"):
 *   - the per-object rigid transform of each base sub-mesh into the world
 *     (the "T o M^base" composition, read as v' = R(q) v + p);
 *   - one ray per pixel (pinhole camera) or per channel/azimuth bin (3-D LiDAR);
 *   - the nearest intersection of that ray with every triangle of the
 *     environment (no acceleration structure: the plain definition);
 *   - the reported value: range (distance sensor -> hit) for LiDAR, depth
 *     (distance of the hit from the image plane) for the camera, and the
 *     segment ID of the object hit; misses report max_range and -1.
 * On top of the exact answer it classifies each ray's tolerance-ambiguous
 * outcomes (edge/silhouette, near-tie, range boundary, grazing incidence,
 * coarse coordinates) so that a single-precision implementation can be judged
 * element by element: a ray none of these applies to must match the exact
 * answer within the tolerance.
 */
#ifndef AGS_ORACLE_H
#define AGS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_PINHOLE 0
#define ORC_LIDAR 1
#define ORC_RAY_TABLE 2 /* user projection model: one sensor-frame direction per pixel */
#define ORC_NEAR_CLAMP 0
#define ORC_NEAR_INVALID 1

/* maximum number of distinct-segment outcome groups reported per ray */
#define ORC_MAX_CAND 4
/* maximum number of candidate triangles listed per ray */
#define ORC_MAX_TRI 8

/* flag bits of orc_result.flags */
#define ORC_F_COUNTED 1      /* judged against the listed outcomes, not the tolerance (a reason below holds) */
#define ORC_F_SILHOUETTE 2   /* a candidate lies within eps of a triangle edge */
#define ORC_F_NEAR_TIE 4     /* two surely-hit triangles of different segments within tol */
#define ORC_F_RANGE_EDGE 8   /* a candidate lies within tol of a range limit or of the sensor's origin */
#define ORC_F_GRAZING 16     /* the exact hit surface has |n.d| below the grazing bound (counted) */
#define ORC_F_OVERFLOW 32    /* more than ORC_MAX_CAND segment groups (test must fail) */
#define ORC_F_MISS_OK 64     /* "miss" (max_range, -1) is an acceptable outcome */
#define ORC_F_WIDE 128       /* the error bands widen an outcome's value range beyond +-tol (information only) */
#define ORC_F_TRI_OVERFLOW 256 /* more than ORC_MAX_TRI candidate triangles */
#define ORC_F_COARSE 512     /* the hit triangle's vertex band exceeds the tolerance (counted) */

typedef struct {
  int32_t type;        /* ORC_PINHOLE or ORC_LIDAR */
  int32_t width;       /* camera columns, or LiDAR azimuth bins */
  int32_t height;      /* camera rows, or LiDAR channels */
  int32_t near_mode;   /* ORC_NEAR_CLAMP or ORC_NEAR_INVALID */
  double hfov;         /* camera: horizontal field of view; LiDAR: azimuth span (rad) */
  double vfov_min;     /* LiDAR: lowest channel elevation (rad); unused by the camera */
  double vfov_max;     /* LiDAR: highest channel elevation (rad) */
  double min_range;    /* metres; applies to depth (camera) or range (LiDAR) */
  double max_range;
  /* error bands of the single-precision renderer being judged (see orc_render) */
  double vert_rel;     /* world vertex coordinate error, relative to max(|coord|, 1) */
  double dir_rel;      /* ray direction error, relative */
  double arith_rel;    /* intersection arithmetic error, relative to the vertex distance */
  const double* dirs;  /* ORC_RAY_TABLE: [height][width][3] sensor-frame directions; the reported
                          value is the distance along each in units of its length */
} orc_sensor;

typedef struct {
  double v;            /* exact reported value (depth or range), metres */
  int32_t seg;         /* exact segment ID, -1 on miss */
  int32_t tri;         /* env-local triangle index of the exact nearest hit, -1 on miss */
  int32_t flags;       /* ORC_F_* */
  int32_t n_cand;      /* number of valid candidate groups */
  int32_t cand_seg[ORC_MAX_CAND];
  double cand_lo[ORC_MAX_CAND];   /* acceptable reported-value interval per segment */
  double cand_hi[ORC_MAX_CAND];
  int32_t n_tri;       /* triangles a single-precision renderer may report (within the bands) */
  int32_t cand_tri[ORC_MAX_TRI];
  double t_hit;        /* exact distance to the nearest hit along the unit ray (INFINITY: none) */
  double cos_hit;      /* |n.d| of the exact nearest triangle (0 on a miss) */
  double hit_dev;      /* how far the error bands move that triangle's own hit, in reported units
                          (the larger side of its band around the exact value; 0 on a miss) */
} orc_result;

/* Rotation matrix of the unit quaternion q/|q| (x, y, z, w order), row-major. */
void orc_rotation(const double q[4], double R[9]);

/* v' = R(q) v + p for n points; pose = (px, py, pz, qx, qy, qz, qw). */
void orc_transform(const double* v, int64_t n, const double pose[7], double* out);

/* The ray of pixel/beam (row, col): origin o, unit direction d, and the factor
 * that turns distance along d into the reported value (d.f for a camera whose
 * optical axis is f = R(q) (1,0,0); 1 for LiDAR). Returns 0, or -1 on bad input. */
int orc_ray(const orc_sensor* s, const double pose[7], int64_t row, int64_t col,
            double o[3], double d[3], double* scale);

/* Nearest hit for each listed ray (flat index row*width+col) against all F
 * triangles tris[F][9] (x0 y0 z0 x1 y1 z1 x2 y2 z2), segment IDs seg[F].
 * Parallel over rays with OpenMP. Returns 0, or -1 on bad input. */
int orc_render(const double* tris, const int32_t* seg, int64_t F,
               const orc_sensor* s, const double pose[7],
               const int64_t* rays, int64_t n_rays, orc_result* out);

/* Extra hit channels of a ray (Sec. III-D.1: face indices with barycentric
 * coordinates, surface normals, point clouds), for n rays (flat index
 * row*width+col) that hit triangle face[i] of tris (or miss: face[i] < 0) and
 * report value v[i]:
 *   bary[2i..]   (u, v): weights of the triangle's second and third vertex at
 *                the point where the ray meets the triangle's plane; 0 on a miss;
 *   normal[3i..] unit geometric normal (v1 - v0) x (v2 - v0) in the world frame,
 *                turned to face the sensor (n.d <= 0); 0 on a miss;
 *   point[3i..]  the hit in the sensor frame, v[i] times the sensor-frame ray
 *                direction scaled to unit reported value (camera: (1, a, b),
 *                LiDAR: the unit direction).
 * Returns 0, or -1 on bad input or a zero-area / parallel face. */
int orc_hit_channels(const double* tris, int64_t F, const orc_sensor* s, const double pose[7],
                     const int64_t* rays, const int32_t* face, const double* v, int64_t n,
                     double* bary, double* normal, double* point);

/* Stereo shadow verdict of each listed ray (Sec. III-D.1): with the second
 * sensor at o2 = p + R(q) baseline and P the exact hit of ray i (from
 * res[i], an orc_render result for the same ray), out[i] = 1 if a triangle
 * surely meets the segment P + s (o2 - P) for s in [eps, 1], 0 if none can,
 * 2 if one lies within the error bands (either verdict is acceptable);
 * rays without a reported hit get 0. Returns 0, or -1 on bad input. */
int orc_shadow(const double* tris, int64_t F, const orc_sensor* s, const double pose[7],
               const double baseline[3], double eps, const int64_t* rays, const orc_result* res,
               int64_t n, int32_t* out);

/* Number of OpenMP threads the oracle uses. */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
