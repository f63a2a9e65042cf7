/*
 * prrtc_oracle.h -- plain, slow FP64 CPU oracle of the pRRTC hot path.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or table with the CUDA path (paper_2503_06757_gb300/csrc), and the product
 * path never calls it.
 *
 * What it computes (pRRTC, Huang et al. 2025):
 *   - Alg. 1 (pRRTC top level) executed serially: balanced tree choice,
 *     sampling, nearest neighbour, pEXTEND, insertion, greedy connect, PATH;
 *     or by B workers in lockstep rounds, a deterministic schedule of the
 *     concurrent iterations of Sec. III.
 *   - Alg. 2 (pEXTEND): steer by at most delta, then check the interpolated
 *     states of the edge at the fixed collision-checking resolution.
 *   - Sec. III-A: collision checking of a sphere model against cuboids,
 *     capped cylinders and spheres, plus self-collision between sphere pairs.
 *   - Philox4x32-10 (Salmon et al., SC'11) for the sampler, or the
 *     multi-dimensional Halton sequence the paper samples with (Sec. IV-A).
 *   - Dynamic-domain sampling (Yershova et al. 2005, with the adaptive
 *     radius of Jaillet et al. 2005), which the paper adds to Alg. 1 (Sec. III).
 * Every floating-point step is in IEEE binary64.
 *
 * Parity-pinned functions (see tests/test_oracle_pins.py):
 *   orc_philox4x32_10  - published known-answer vectors of Random123.
 *   orc_fk             - closed-form tip positions of 1-, 2- and 3-link chains.
 *   orc_sd_box/cyl/sph - brute-force surface/volume sampling on tiny inputs.
 *   orc_plan           - tree invariants, obstacle-free and walled-off special
 *                        cases, grid-BFS reachability of a point robot; the
 *                        lockstep form: one worker reproduces the serial
 *                        trees, the obstacle-free round in closed form, the
 *                        round structure of every tree it builds.
 *   orc_occupancy      - closed-form voxel sets of a sphere and a box.
 *   orc_voxelize / orc_esdf / orc_esdf_query - closed-form fields of one
 *                        occupied voxel, of a half-space and of empty / full
 *                        grids; exact reproduction of linear fields; the true
 *                        signed distance of a sphere obstacle within the
 *                        discretisation bound.
 *   orc_sample_learned - the mixture statistics of its draws (component
 *                        frequencies, per-component mean and spread).
 *   orc_halton         - the printed van der Corput fractions of bases 2 and 3,
 *                        exact stratification of the first b^m points.
 *   dynamic domain     - an unbounded radius and an obstacle-free scene both
 *                        reduce to the plain planner; a 1-DoF slider against a
 *                        wall advances by at most the radius after its first
 *                        failed extension.
 */
#ifndef PRRTC_ORACLE_H
#define PRRTC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_REV_Z = 0, ORC_REV_Y = 1, ORC_PRISM_Z = 2, ORC_PRISM_X = 3, ORC_PRISM_Y = 4, ORC_REV_X = 5 };

enum {
  ORC_SOLVED = 0,
  ORC_START_IN_COLLISION = 1,
  ORC_GOAL_IN_COLLISION = 2,
  ORC_NO_SOLUTION = 3,
  ORC_PATH_OVERFLOW = 4,
  ORC_BAD_INPUT = -1
};

/* Ambiguity kinds recorded by the planner: decisions whose outcome could flip
 * under FP32 rounding (the device path) and so end an exact comparison. */
enum {
  ORC_AMB_NONE = 0,
  ORC_AMB_CLEARANCE = 1, /* a checked state had |clearance| <= band       */
  ORC_AMB_NN_TIE = 2,    /* best and second-best squared distances close  */
  ORC_AMB_CEIL = 3,      /* a ceil() argument lay next to an integer      */
  ORC_AMB_STEER = 4,     /* sample distance next to the range delta        */
  ORC_AMB_COMPONENT = 5, /* mixture component draw next to a boundary      */
  ORC_AMB_DOMAIN = 6     /* sample distance next to a dynamic-domain radius */
};

enum { ORC_SAMPLER_PHILOX = 0, ORC_SAMPLER_HALTON = 1 };

typedef struct orc_robot {
  int32_t dof;
  const int32_t* joint_type;   /* [dof]  ORC_REV_* / ORC_PRISM_* (local axis)  */
  const int32_t* joint_parent; /* [dof]  parent joint, -1 = world             */
  const double* joint_base;    /* [dof*3] world offset of world-parented joints */
  const double* link_length;   /* [dof]  translation along local z after J_i  */
  const double* lower;         /* [dof]  joint limits                          */
  const double* upper;         /* [dof]                                        */
  int32_t n_spheres;
  const int32_t* sphere_frame; /* [S]    frame (joint) carrying the sphere     */
  const double* sphere_offset; /* [S*3]  centre in frame coordinates           */
  const double* sphere_radius; /* [S]                                          */
  int32_t n_pairs;
  const int32_t* pairs;        /* [P*2]  sphere pairs tested for self-collision */
} orc_robot;

typedef struct orc_env {
  int32_t n_box;
  const double* box;   /* [n_box*15]: centre(3) half(3) R(9, row-major, world = R*local + c) */
  int32_t n_cyl;
  const double* cyl;   /* [n_cyl*8]: centre(3) unit axis(3) radius half_length */
  int32_t n_sph;
  const double* sph;   /* [n_sph*4]: centre(3) radius */
  /* optional Euclidean signed distance field (nullable): values at voxel
   * centres origin + (index + 0.5) * voxel, index i + nx*(j + ny*k); spheres
   * are tested against it (trilinear read) in addition to the primitives */
  const double* esdf;
  double esdf_origin[3];
  double esdf_voxel;
  int32_t esdf_dims[3];
} orc_env;

typedef struct orc_params {
  double range;          /* delta: extension range (configuration-space L2)  */
  double resolution;     /* collision-checking resolution along an edge      */
  double goal_bias;      /* probability of sampling the opposite tree's root */
  double amb_band;       /* clearance band treated as ambiguous (1e-5 m)     */
  double amb_rel;        /* relative gap that makes an NN / ceil decision ambiguous */
  uint64_t seed;         /* Philox key                                       */
  uint32_t problem;      /* Philox counter word 0                            */
  int32_t max_iters;     /* global budget of Alg. 1 bodies                    */
  int32_t tree_capacity; /* nodes per tree; an insertion into a full tree fails */
  int32_t path_capacity; /* rows of the caller's path buffer                 */
  /* learned proposal (nullable): mixture of 8 diagonal Gaussians over joint
   * values normalised to [-1, 1]; layout logits[8], mean[8*dof],
   * log_sigma[8*dof] (clamped to [-5, 2] when used) */
  const double* gmm;
  double learned_ratio;  /* probability of drawing from the mixture (after goal bias) */
  /* uniform branch of RANDOM_CONFIG: ORC_SAMPLER_PHILOX (words 1..dof of the
   * iteration's Philox stream) or ORC_SAMPLER_HALTON (point it + 1 +
   * halton_offset of the Halton sequence in the first dof prime bases) */
  int32_t sampler;
  uint32_t halton_offset;
  /* dynamic-domain sampling: every node carries a radius, unbounded when the
   * node is added.  A random (not goal-bias) sample farther than the radius
   * from its nearest node is rejected: the iteration ends there.  After the
   * check of the edge from nearest node n: on success a bounded radius grows,
   * r <- r (1 + alpha); on a collision an unbounded radius becomes dd_radius,
   * a bounded one shrinks to max(r (1 - alpha), dd_min_radius).  Greedy
   * connect steps leave radii alone.  dd_radius <= 0 turns it off. */
  double dd_radius;
  double dd_alpha;
  double dd_min_radius;
  /* concurrent workers (Sec. III: iterations of Alg. 1 run in parallel
   * against two shared trees).  0: serial Alg. 1.  B >= 1: lockstep
   * rounds (B = 1 gives the serial trees by a separate route) -- in round r, worker b runs iteration r B + b (sampling, nearest
   * neighbour, pEXTEND and the greedy connect) against the trees as they
   * stood when the round began, holding its new rows back; at the end of the
   * round the held rows are appended in worker order.  Of the workers whose
   * connect reached its target (with every row they added in the tree), the
   * one a concurrent run would finish first -- fewest edges checked in its
   * iteration, ties to the lowest worker -- ends the search with PATH. */
  int32_t workers;
} orc_params;

typedef struct orc_result {
  int32_t status;
  int32_t iterations;          /* Alg. 1 bodies executed (it + 1 at success)    */
  int32_t n_a, n_b;            /* tree sizes                                   */
  int32_t join_a, join_b;      /* joined nodes (indices into T_a, T_b)         */
  int32_t path_n;              /* waypoints written to path                    */
  int32_t first_amb_iter;      /* first iteration with an ambiguous decision, -1 none */
  int32_t first_amb_kind;
  int32_t pad_;
  double cost;                 /* sum of L2 segment lengths                    */
  int64_t edges_checked;       /* edges whose states were examined            */
  int64_t states_checked;      /* states examined (stop at the first collision) */
  int64_t edge_states;         /* sum over checked edges of their state count   */
  int64_t dd_rejected;         /* iterations ended by the dynamic-domain test    */
  /* caller-owned buffers (nullable): trees and path */
  double* nodes_a;             /* [tree_capacity*dof] */
  int32_t* parent_a;           /* [tree_capacity]     */
  double* nodes_b;
  int32_t* parent_b;
  double* path;                /* [path_capacity*dof] */
  double* radius_a;            /* [tree_capacity] dynamic-domain radii (INFINITY = unbounded) */
  double* radius_b;
} orc_result;

/* Philox4x32-10 block: out = Philox(ctr, key).  Salmon et al. SC'11. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The same for n counters (ctr, out: [4n] words). */
void orc_philox_blocks(const uint32_t* ctr, int32_t n, const uint32_t key[2], uint32_t* out);

/* Sample of Alg. 1 (RANDOM_CONFIG) for iteration `it`: returns 1 when the
 * goal-bias branch fires (the caller substitutes the opposite root), else 0
 * and writes a uniform configuration inside the joint limits to q. */
int orc_sample(const orc_robot* r, uint64_t seed, uint32_t problem, uint32_t it,
               double goal_bias, double* q);

/* Sample with the learned proposal enabled: goal bias first (returns 1),
 * then with probability learned_ratio a draw from the mixture (returns 2),
 * else uniform (returns 0).  *amb is set when the component choice fell next
 * to a cumulative-probability boundary. */
int orc_sample_learned(const orc_robot* r, uint64_t seed, uint32_t problem, uint32_t it, double goal_bias,
                       const double* gmm, double learned_ratio, double amb_rel, double* q, int* amb);

/* Point `index` of the Halton sequence in `dim` dimensions: coordinate j is
 * the radical inverse of index in the j-th prime base (2, 3, 5, ...), i.e.
 * its base-p digits mirrored about the radix point.  dim <= 16. */
void orc_halton(uint32_t index, int32_t dim, double* u);

/* Occupancy grid of an environment: voxel (i, j, k), index i + n*j + n*n*k,
 * centre origin + (index + 0.5) * cell per axis, is occupied iff its centre
 * lies closer than `radius` to some obstacle (signed distance < radius). */
void orc_occupancy(const orc_env* e, const double origin[3], double cell, int32_t n, double radius,
                   uint8_t* out);

/* ESDF collision checking (Sec. III-A, ESDF maps of the real-world setup):
 * occupancy of a voxel grid (voxel centre strictly inside some primitive),
 * the signed Euclidean distance transform of an occupancy grid, and its
 * trilinear read.  dims = {nx, ny, nz}, index i + nx*(j + ny*k).
 *   orc_voxelize:   occ = 1 iff the centre's signed distance to some primitive is < 0.
 *   orc_esdf:       free voxel: +voxel * (distance in voxel units to the nearest
 *                   occupied voxel centre); occupied voxel: -voxel * (distance to
 *                   the nearest free voxel centre); written by brute force over all
 *                   voxel pairs.  A grid without occupied (free) voxels gives every
 *                   voxel +(-) the grid diagonal voxel * sqrt(nx^2 + ny^2 + nz^2).
 *   orc_esdf_query: continuous index u = (p - origin) / voxel - 1/2 per axis,
 *                   clamped to [0, n - 1]; base i0 = min(floor(u), n - 2),
 *                   t = u - i0; linear blends along x, then y, then z.  n >= 2. */
void orc_voxelize(const orc_env* e, const double origin[3], double voxel, const int32_t dims[3], uint8_t* occ);
void orc_esdf(const uint8_t* occ, const int32_t dims[3], double voxel, double* out);
/* The same field at one voxel (i, j, k), for spot checks of large grids. */
double orc_esdf_at(const uint8_t* occ, const int32_t dims[3], double voxel, int32_t i, int32_t j, int32_t k);
double orc_esdf_query(const double* esdf, const double origin[3], double voxel, const int32_t dims[3],
                      const double p[3]);

/* Forward kinematics by 4x4 homogeneous products.  centres: [S*3];
 * frames (nullable): [dof*16] row-major world transforms. */
void orc_fk(const orc_robot* r, const double* q, double* centres, double* frames);

/* Signed distances from a point to one obstacle (negative inside). */
double orc_sd_box(const double* box15, const double p[3]);
double orc_sd_cyl(const double* cyl8, const double p[3]);
double orc_sd_sph(const double* sph4, const double p[3]);

/* Clearance of one configuration: min over (sphere, obstacle) of sd - r and
 * over self pairs of |ci - cj| - ri - rj.  The state is in collision iff the
 * clearance is negative.  env_c / self_c (nullable) receive the two parts. */
double orc_clearance(const orc_robot* r, const orc_env* e, const double* q,
                     double* env_c, double* self_c);

/* Verdicts for n states (row-major [n*dof]); free[i] = clearance >= 0. */
void orc_check_states(const orc_robot* r, const orc_env* e, const double* Q, int32_t n,
                      uint8_t* free_out, double* clearance_out);

/* pRRTC (Alg. 1 with Alg. 2): serial, or B workers in lockstep rounds
 * (p->workers).  Returns res->status. */
int32_t orc_plan(const orc_robot* r, const orc_env* e, const double* q_start,
                 const double* q_goal, const orc_params* p, orc_result* res);

/* Re-check every segment of a path at resolution `res`: each segment of
 * length l is split into ceil(l/res) steps and all states after the first
 * waypoint are tested.  Returns the number of segments with a colliding state;
 * *min_clearance receives the smallest clearance seen. */
int32_t orc_revalidate(const orc_robot* r, const orc_env* e, const double* path,
                       int32_t n, double res, double* min_clearance);

/* Batch of independent plans on `threads` POSIX threads (one problem at a
 * time per thread).  Arrays are indexed by problem. */
typedef struct orc_problem {
  const orc_robot* robot;
  const orc_env* env;
  const double* q_start;
  const double* q_goal;
  orc_params params;
  orc_result* result;
  double seconds;              /* wall time of this plan (output) */
} orc_problem;

void orc_plan_batch(orc_problem* problems, int32_t n, int32_t threads);

#ifdef __cplusplus
}
#endif
#endif
