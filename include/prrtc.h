/*
 * prrtc.h -- C ABI of the GB300-native pRRTC planner (libprrtc.so).
 *
 * pRRTC (Huang, Jadhav, Plancher, Kingston, "pRRTC: GPU-Parallel RRT-Connect
 * for Fast, Consistent, and Low-Cost Motion Planning", arXiv 2503.06757):
 * RRT-Connect whose iterations run concurrently against two shared trees on
 * the GPU (Sec. III, Alg. 1), with every interpolated state of a candidate
 * edge collision-checked in parallel (Alg. 2, Sec. III-A) and a parallel
 * nearest-neighbour scan (Sec. III-C).
 *
 * Conventions for every entry point:
 *   - Return value: PRRTC_OK (0) on success, a negative PRRTC_ERR_* code on
 *     failure.  Planning outcomes (no solution, start in collision, ...) are
 *     positive status codes reported per problem, never as errors.  No C++
 *     exception crosses this boundary.
 *   - Handles (prrtc_env, prrtc_robot) are opaque, owned by the library and
 *     released by the matching *_destroy call.  Their geometry lives in device
 *     memory of the CUDA device that was current when they were created.
 *   - Pointers without a "_device" suffix are host pointers; the library
 *     copies what it needs before returning and keeps no reference.
 *   - Floating-point inputs are IEEE binary32; configurations are row-major
 *     [n x dof] arrays of joint values (radians / metres).
 *   - Thread safety: calls on different handles may run from different host
 *     threads; each planning call serialises on the library's stream for the
 *     current device, so an env update issued between two calls applies
 *     exactly between them.
 *   - There is no CPU fallback: without a usable CUDA device every call
 *     returns PRRTC_ERR_NO_DEVICE.
 */
#ifndef PRRTC_H
#define PRRTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define PRRTC_OK 0
#define PRRTC_ERR_INVALID_ARG (-1)   /* a pointer, size or descriptor is invalid      */
#define PRRTC_ERR_OOM (-2)           /* device or host allocation failed              */
#define PRRTC_ERR_CUDA (-3)          /* a CUDA runtime call failed                    */
#define PRRTC_ERR_TIMEOUT (-4)       /* a bounded device-side wait gave up            */
#define PRRTC_ERR_DEVICE_INDEX (-5)  /* a device-side bounds check fired              */
#define PRRTC_ERR_NO_DEVICE (-6)     /* no CUDA device is available                   */
#define PRRTC_ERR_UNSUPPORTED (-7)   /* a feature outside the compiled limits         */

/* per-problem planning outcomes (prrtc_path.status, out_status[]) */
#define PRRTC_SOLVED 0
#define PRRTC_START_IN_COLLISION 1
#define PRRTC_GOAL_IN_COLLISION 2
#define PRRTC_NO_SOLUTION 3          /* iteration budget spent (Alg. 1 "return Failed") */
#define PRRTC_PATH_OVERFLOW 4        /* solved, but the path exceeded path_capacity    */
#define PRRTC_TIME_LIMIT 5           /* wall-clock budget spent on the device          */

/* compiled limits */
#define PRRTC_MAX_DOF 16
#define PRRTC_MAX_SPHERES 128        /* spheres per robot as given (before merging)    */
#define PRRTC_MAX_PAIRS 4096         /* self-collision sphere pairs as given           */
#define PRRTC_MAX_OBSTACLES 1024
#define PRRTC_ESDF_MAX_DIM 1024   /* voxels per axis of a distance field */

/* ------------------------------------------------------------ geometry */
#define PRRTC_OBS_BOX 0       /* cuboid: centre, half extents, rotation                 */
#define PRRTC_OBS_CYLINDER 1  /* solid cylinder with flat caps: centre, axis, radius, half length */
#define PRRTC_OBS_SPHERE 2    /* centre, radius                                          */

/* One obstacle primitive (Sec. III-A: environments of primitive geometry).
 *   box:      centre, half[0..2] = half extents, rot = row-major rotation
 *             (world = rot * local + centre); identity rot = axis-aligned.
 *   cylinder: centre, axis = unit axis direction, half[0] = radius,
 *             half[1] = half length.
 *   sphere:   centre, half[0] = radius.
 * A robot sphere of radius r collides with a primitive iff the squared
 * distance from its centre to the primitive is < r^2 (touching is free). */
typedef struct prrtc_obstacle {
  int32_t type;
  float center[3];
  float half[3];
  float axis[3];
  float rot[9];
} prrtc_obstacle;

#define PRRTC_JOINT_REV_Z 0
#define PRRTC_JOINT_REV_Y 1
#define PRRTC_JOINT_PRISM_Z 2
#define PRRTC_JOINT_PRISM_X 3
#define PRRTC_JOINT_PRISM_Y 4
#define PRRTC_JOINT_REV_X 5

/* Sphere model of a robot (Sec. III-A, bounding spheres per link).
 * Frame i = T_parent(i) * J_i(q_i) * Trans(0, 0, link_length[i]), where J_i
 * rotates about / translates along a local axis (PRRTC_JOINT_*), and
 * T_parent = Trans(joint_base[3i..3i+2]) when joint_parent[i] == -1.
 * joint_parent[i] must be -1 or i-1 (one or more serial chains).
 * Sphere s has centre T_{sphere_frame[s]} * [sphere_offset[3s..3s+2], 1] and
 * radius sphere_radius[s].  self_pairs lists sphere index pairs checked for
 * self-collision (collide iff |ci - cj|^2 < (ri + rj)^2).  Joint values are
 * sampled uniformly in [lower, upper]. */
typedef struct prrtc_robot_desc {
  int32_t dof;
  const int32_t* joint_type;    /* [dof] */
  const int32_t* joint_parent;  /* [dof] */
  const float* joint_base;      /* [dof*3] */
  const float* link_length;     /* [dof] */
  const float* lower;           /* [dof] */
  const float* upper;           /* [dof] */
  int32_t n_spheres;
  const int32_t* sphere_frame;  /* [n_spheres] */
  const float* sphere_offset;   /* [n_spheres*3] */
  const float* sphere_radius;   /* [n_spheres] */
  int32_t n_pairs;
  const int32_t* self_pairs;    /* [n_pairs*2] */
} prrtc_robot_desc;

typedef struct prrtc_env prrtc_env;
typedef struct prrtc_robot prrtc_robot;

/* ------------------------------------------------------------ parameters */
#define PRRTC_MODE_ASYNC 0   /* blocks x warps run Alg. 1 iterations concurrently (Sec. III) */
#define PRRTC_MODE_SERIAL 1  /* one warp runs the iterations in order: the serial Alg. 1   */
/* B = params.workers concurrent iterations per round on a fixed schedule (the
 * concurrency of Sec. III made deterministic): in round r, worker b runs
 * iteration r B + b -- sampling, nearest neighbour, pEXTEND and the greedy
 * connect -- against both trees as they stood when the round began and holds
 * its new rows back; at the end of the round every worker's rows are appended
 * in worker order.  Of the workers whose connect reached its target with all
 * their rows in the tree, the one that checked the fewest edges in its
 * iteration (ties: lowest b) wins, as the first connection to finish would in
 * a concurrent run.  B = 1 is the serial Alg. 1.  The trees equal those of the
 * FP64 oracle's lockstep form outside the 1e-5 m clearance band. */
#define PRRTC_MODE_LOCKSTEP 2

typedef struct prrtc_params {
  float range;            /* delta: extension range in configuration space (L2)        */
  float resolution;       /* collision-checking resolution: an edge of length l is
                             checked at ceil(l / resolution) states (Alg. 2, N_cc)    */
  float goal_bias;        /* probability of sampling the opposite tree's root          */
  int32_t max_iters;      /* budget of Alg. 1 iterations per problem, shared by all workers */
  int32_t tree_capacity;  /* nodes per tree per problem                                */
  int32_t path_capacity;  /* waypoints per returned path                               */
  int32_t mode;           /* PRRTC_MODE_*                                              */
  int32_t blocks;         /* grid size of the planner launch; 0 = one wave of resident blocks */
  int32_t warps_per_block;/* worker warps per block; 0 = 4                             */
  float learned_ratio;    /* probability of drawing from a problem's learned mixture
                             (after the goal bias); 0 = uniform sampling only         */
  uint64_t seed;          /* Philox key used by prrtc_plan                             */
  double time_limit_s;    /* device-side wall-clock budget per launch; 0 = none        */
  int32_t sampler;        /* uniform branch of RANDOM_CONFIG (Alg. 1): PRRTC_SAMPLER_PHILOX
                             (words of the iteration's Philox stream) or
                             PRRTC_SAMPLER_HALTON (the paper's Halton sequence, Sec. IV-A:
                             iteration `it` takes point it + 1 + halton_offset)          */
  uint32_t halton_offset;
  float dd_radius;        /* dynamic-domain sampling (Sec. III; Yershova et al. 2005): a
                             random sample farther than its nearest node's radius is
                             rejected and the iteration ends.  Radii start unbounded; the
                             first collision of an extension from a node bounds its radius
                             to dd_radius.  0 = off                                    */
  float dd_alpha;         /* adaptive radius (Jaillet et al. 2005): a bounded radius grows
                             by (1 + dd_alpha) after a free extension and shrinks by
                             (1 - dd_alpha), not below dd_min_radius, after a collision */
  float dd_min_radius;
  int32_t workers;        /* PRRTC_MODE_LOCKSTEP: concurrent iterations per round, 1..1024
                             (other modes ignore it); warps_per_block 0 = min(workers, 8)
                             warps per problem, each running workers / warps iterations
                             of a round in turn                                       */
  int32_t debug_wait_polls;  /* test hook for the bounded device waits; 0 = off.  When > 0, the
                             path extraction of a solved problem first spins, for at most
                             this many polls, on a device flag that nothing sets; the wait
                             gives up like a parent walk that found an unwritten row: the
                             problem reports PRRTC_ERR_TIMEOUT, the call returns
                             PRRTC_ERR_TIMEOUT, and later calls on the same handles work */
  int32_t expansions;     /* async mode: Alg. 1 iterations (expansions) a worker takes per claim
                             of its problem's shared iteration counter, 1..64; 0 = 1.  Fewer
                             claims mean less contention on the counter when many workers share
                             a problem.  Every iteration id below max_iters is claimed once; when
                             the budget runs out, ids claimed but not yet started are dropped */
  int32_t obstacle_tile;  /* primitives of each type tested per round of the warp-wide first
                             stage of the collision check (one or two per lane): 32 or 64;
                             0 = 32.  The verdicts do not depend on it */
  int32_t reserved[2];
} prrtc_params;

#define PRRTC_SAMPLER_PHILOX 0
#define PRRTC_SAMPLER_HALTON 1

/* Fills the defaults: range 1.0, resolution 1/32, goal bias 0.05, 50000
 * iterations, 65536 nodes per tree, 16384 waypoints, async mode, seed 1. */
void prrtc_params_default(prrtc_params* p);

/* ------------------------------------------------------------ results */
typedef struct prrtc_path {
  int32_t status;          /* PRRTC_SOLVED or another planning outcome                    */
  int32_t n;               /* waypoints in q                                              */
  int32_t dof;
  int32_t iterations;      /* Alg. 1 iterations started for this problem                  */
  float* q;                /* [n*dof] host memory owned by the library; prrtc_path_free   */
  double cost;             /* sum of L2 segment lengths (Table I "arclength")             */
  int32_t nodes_a;         /* start-tree size                                             */
  int32_t nodes_b;         /* goal-tree size                                              */
  int64_t edges_checked;   /* edges whose states were tested                              */
  int64_t edge_states;     /* sum over tested edges of their state count                  */
  double solve_time_us;    /* device time from launch start to this problem's solution    */
  int64_t sphere_tests;    /* lane-level sphere passes over the obstacle set              */
  int64_t pair_tests;      /* lane-level self-collision pair tests                        */
  int64_t fk_states;       /* lane-level forward-kinematics evaluations                   */
  int64_t nn_nodes;        /* tree rows scanned by nearest-neighbour queries              */
  int64_t dd_rejected;     /* iterations ended by the dynamic-domain test                 */
  int64_t prim_tests[4];   /* lane-level tests of one fine sphere against one primitive in
                              the second stage of the two-stage check, per primitive type
                              (AABB, oriented box, capped cylinder, sphere)               */
  int64_t verdict_states;  /* states whose collision verdict was established: every state
                              of a free edge, and for an edge found in collision the states
                              of its earlier passes plus the colliding one (states stopped by
                              the early exit are not counted)                              */
} prrtc_path;

void prrtc_path_free(prrtc_path* path);
/* prrtc_path_free on paths[0 .. n-1] (the results of one batch call) in one
 * call.  A null paths or n <= 0 does nothing. */
void prrtc_paths_free(prrtc_path* paths, int32_t n);

/* Work counters and timing of the most recent planning launch on the current
 * device (for throughput and roofline accounting). */
typedef struct prrtc_launch_stats {
  double kernel_ms;          /* planner kernel, CUDA events on the library stream    */
  double setup_ms;           /* arena reset + root insertion kernel                   */
  int64_t edges_checked;
  int64_t edge_states;       /* states of all tested edges                            */
  int64_t sphere_tests;      /* lane-level sphere passes over the whole environment
                                (fine spheres of one-stage frames, bounding spheres of
                                two-stage frames)                                       */
  int64_t env_tests;         /* lane-level second-stage sphere-primitive tests (sum of
                                prim_tests)                                              */
  int64_t pair_tests;        /* lane-level self-collision pair tests                  */
  int64_t fk_states;         /* lane-level forward-kinematics evaluations              */
  int64_t nn_nodes;          /* tree nodes scanned by nearest-neighbour queries        */
  int64_t iterations;        /* Alg. 1 iterations across all problems                  */
  int32_t grid;              /* blocks launched                                        */
  int32_t block_threads;
  int32_t smem_bytes;
  int32_t problems;
  int64_t h2d_bytes;         /* host -> device bytes copied by the call                */
  int64_t d2h_bytes;         /* device -> host bytes copied by the call                */
  int32_t kernels;           /* kernels the call launched                              */
  int32_t lean_kernel;       /* 1: the planner instance without the learned draw, Halton,
                                distance fields, oriented boxes and one-stage links (the
                                batch used none)                                          */
  double prep_ms;            /* from the call's first device work to the setup kernel:
                                learned-mixture inference and descriptor upload         */
  int64_t prim_tests[4];     /* second-stage tests per primitive type (AABB, oriented
                                box, capped cylinder, sphere)                            */
  int64_t dd_rejected;       /* iterations ended by the dynamic-domain test            */
  int64_t verdict_states;    /* see prrtc_path.verdict_states                          */
  double infer_ms;           /* device time of the learned-mixture inference (staging
                                copy and kernel chain; part of prep_ms), 0 without     */
} prrtc_launch_stats;

int prrtc_last_launch_stats(prrtc_launch_stats* out);

/* Copy tree `tree` (0 = start tree T_a, 1 = goal tree T_b) of problem
 * `problem` of the most recent planning launch on the current device:
 * rows [min(size, cap) * dof] into nodes, parent indices into parents (-1 for
 * the root), *out_n = rows available.  Buffers are host memory of `cap` rows;
 * either may be null.  For tests and diagnostics (tree invariants, lockstep
 * comparison with a serial reference). */
int prrtc_debug_tree(int32_t problem, int32_t tree, float* nodes, int32_t* parents, int32_t cap, int32_t* out_n);

/* ------------------------------------------------------------ entry points */
const char* prrtc_status_string(int code);
const char* prrtc_version(void);

/* Message of the last failing call on this host thread ("" if none). */
const char* prrtc_last_error(void);

/* Upload an obstacle set (Sec. III-A; obstacles cached in GPU memory).
 * n may be 0.  Returns PRRTC_ERR_INVALID_ARG for an unknown type, a
 * non-positive size or n > PRRTC_MAX_OBSTACLES. */
int prrtc_env_create(const prrtc_obstacle* obstacles, int32_t n, prrtc_env** out);

/* Replace obstacles ids[k] (indices in creation order) by obstacles[k]; each
 * keeps its type.  Stream-ordered: applies between planning calls. */
int prrtc_env_update(prrtc_env* env, const int32_t* ids, const prrtc_obstacle* obstacles, int32_t n);

void prrtc_env_destroy(prrtc_env* env);

/* ------------------------------------------------------------ distance-field environments */
/* The paper's real-world setting checks spheres against a Euclidean signed
 * distance field (ESDF) built from sensor data instead of primitives
 * (Sec. III-A, Sec. IV).  Grids: dims = {nx, ny, nz} (each 2..PRRTC_ESDF_MAX_DIM,
 * at most 2^28 voxels), voxel (i, j, k) has index i + nx*(j + ny*k) and centre
 * origin + (i + 1/2, j + 1/2, k + 1/2) * voxel.
 *
 * prrtc_env_create_esdf: an environment holding the signed distance field of
 * `occupancy` (host [nx*ny*nz], nonzero = occupied): free voxels get +voxel x
 * the Euclidean distance (in voxels) to the nearest occupied voxel centre,
 * occupied voxels -voxel x the distance to the nearest free one (exact,
 * computed on the device); +/- the grid diagonal when the grid has no voxel
 * of the other kind.  A sphere (c, r) of the robot collides with it iff the
 * field's trilinear read at c is < r; the read clamps c into the grid of voxel
 * centres (the field continues flat beyond it).  Such an environment has no
 * primitives; planning and checking calls take it like any other.
 * prrtc_env_update_esdf: replace the occupancy (same grid) and recompute;
 * ordered with planning calls on the library's stream.
 * prrtc_env_esdf_values: host [nx*ny*nz] copy of the field.
 * prrtc_voxelize: occupancy of a grid from an environment's primitives
 * (voxel centre strictly inside some primitive), host [nx*ny*nz] output --
 * synthetic occupancy for distance-field environments.
 * Errors: PRRTC_ERR_INVALID_ARG (bad grid, null pointers, env without field),
 * PRRTC_ERR_OOM. */
int prrtc_env_create_esdf(const float origin[3], float voxel, const int32_t dims[3], const uint8_t* occupancy,
                          prrtc_env** out);
int prrtc_env_update_esdf(prrtc_env* env, const uint8_t* occupancy);
int prrtc_env_esdf_values(const prrtc_env* env, float* out);
int prrtc_voxelize(const prrtc_env* env, const float origin[3], float voxel, const int32_t dims[3],
                   uint8_t* occupancy);

/* Upload a robot sphere model.  Coincident spheres of equal radius on the same
 * frame are merged (the verdicts do not change); self pairs are re-indexed. */
int prrtc_robot_create(const prrtc_robot_desc* desc, prrtc_robot** out);
void prrtc_robot_destroy(prrtc_robot* robot);

/* Sizes after merging: DoF, distinct spheres, distinct self pairs and the
 * tree row stride in floats (any pointer may be null). */
int prrtc_robot_info(const prrtc_robot* robot, int32_t* dof, int32_t* n_spheres, int32_t* n_pairs, int32_t* dpad);

/* Two-stage collision checking (Sec. III-A: a low-resolution pass flags the
 * links that may collide, only those are re-checked with the fine spheres).
 * Every frame with two or more distinct spheres gets one bounding sphere that
 * contains all of them with a 1e-5 m margin; the first stage tests it against
 * every primitive, the second tests the frame's fine spheres only against the
 * primitives that some state of the warp's edge flagged.  The verdicts equal
 * those of the one-stage check.  On by default; `enabled` = 0 switches to the
 * one-stage check.  Applies to calls issued after it returns (it writes the
 * device copy of the robot synchronously). */
int prrtc_robot_set_two_stage(prrtc_robot* robot, int32_t enabled);

/* Bounding spheres of the first stage: out4[4*f .. 4*f+3] = centre (frame f
 * coordinates) and radius, radius 0 where frame f has fewer than two distinct
 * spheres (checked in one stage).  out4: host [dof*4]. */
int prrtc_robot_bounds(const prrtc_robot* robot, float* out4);

/* counts4 = {axis-aligned boxes, oriented boxes, cylinders, spheres}. */
int prrtc_env_info(const prrtc_env* env, int32_t* counts4);

/* Collision verdicts of n configurations (Sec. III-A): FK of the sphere model,
 * sphere-vs-primitive and self-collision tests.  q: host [n*dof];
 * out_valid: host [n], 1 = collision-free; out_spheres (nullable): host
 * [n*n_spheres*4], world centre xyz and radius of every sphere in the order
 * given to prrtc_robot_create. */
int prrtc_check_states(const prrtc_robot* robot, const prrtc_env* env, const float* q, int32_t n,
                       uint8_t* out_valid, float* out_spheres);

/* As prrtc_check_states with device pointers, enqueued on `stream`
 * (cudaStream_t, 0 = legacy default stream); returns without synchronising. */
int prrtc_check_states_device(const prrtc_robot* robot, const prrtc_env* env, const float* q_device,
                              int32_t n, uint8_t* valid_device, float* spheres_device, void* stream);

/* The sampler's counter-based generator on the device: Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, SC'11), whose words RANDOM_CONFIG (Alg. 1
 * line 4) draws.  out[4i .. 4i+3] = Philox4x32-10(counter ctr[4i .. 4i+3],
 * key {low 32 bits of key, high 32 bits}) for i < n.  ctr and out: host
 * arrays of 4n words owned by the caller; blocks until done.  For tests of
 * the device generator against an independent implementation.  n = 0 does
 * nothing; n < 0, or a null buffer with n > 0: PRRTC_ERR_INVALID_ARG. */
int prrtc_philox(const uint32_t* ctr, int32_t n, uint64_t key, uint32_t* out);

/* The device's FP32 issue rate, for the denominator of the collision check's
 * ALU roofline (lane-ops per second = SMs x 128 lanes x SM clock, one FMA per
 * lane per cycle): times one launch of 8 independent FMA chains per thread,
 * `iters` steps each, on 8 blocks of 256 threads per SM, after one untimed
 * launch.  *lane_ops_per_s receives the FMAs per second; *kernel_ms (nullable)
 * the timed launch.  Blocks until done.  iters < 1 or a null lane_ops_per_s:
 * PRRTC_ERR_INVALID_ARG. */
int prrtc_alu_peak(int32_t iters, double* lane_ops_per_s, double* kernel_ms);

/* Solve one planning problem (Alg. 1) on the device; blocks until done.
 * out_path receives the path (host memory, free with prrtc_path_free). */
int prrtc_plan(const prrtc_robot* robot, const prrtc_env* env, const float* q_start,
               const float* q_goal, const prrtc_params* params, prrtc_path* out_path);

/* One planning problem of a batch. */
typedef struct prrtc_problem {
  const prrtc_robot* robot;
  const prrtc_env* env;
  const float* q_start;   /* host [robot dof] */
  const float* q_goal;    /* host [robot dof] */
  uint64_t seed;          /* Philox key of this problem                  */
  uint32_t problem_id;    /* Philox counter word 0 of this problem        */
  int32_t reserved;
  /* nullable: sampling mixture of this problem, host [8 + 16*dof] floats:
   * logits[8], means[8*dof], log-sigmas[8*dof] over joint values normalised
   * to [-1, 1] (log-sigmas clamped to [-5, 2]); used with params->learned_ratio */
  const float* gmm;
} prrtc_problem;

/* Solve n independent problems in one persistent launch: blocks take
 * problems from a device work queue and move to unsolved ones as problems
 * finish.  out_paths [n] and out_status [n] (nullable) receive per-problem
 * results.  Robots of different DoF and environments of different sizes may
 * be mixed. */
int prrtc_plan_batch(const prrtc_problem* problems, int32_t n, const prrtc_params* params,
                     prrtc_path* out_paths, int32_t* out_status);

/* Autotuner (the number of concurrent workers is the paper's scaling knob,
 * Sec. IV-C): plan the given problems `trials` times (the same varied seeds
 * for every candidate) and score a candidate by the mean of the batch's median
 * and 95th-percentile time to first solution (setup time plus each problem's
 * device time from launch start to its solution; an unsolved problem counts
 * the whole launch), averaged over the trials.  It picks, one after the other: the launch shape
 * (grid size x warps per block; shapes within 2% of the fastest count as
 * equal and the one with the most workers wins), the obstacle tile (32 or
 * 64) and, in async mode, the expansions per claim (1, 2, 4 or 8); a
 * non-default tile or expansions must be 3% faster to be chosen, and fields
 * the caller set (non-zero) are kept.  The choice goes to *best and is remembered for this
 * device: later calls whose params leave blocks and warps_per_block at 0 use
 * it (and its tile and expansions where those are 0) for the same row width,
 * obstacle-count bucket (64 float4) and batch-size bucket (power of two).
 * *best_ms (nullable) receives the chosen candidate's score (ms).  Lockstep
 * mode has nothing to tune: PRRTC_ERR_INVALID_ARG. */
int prrtc_autotune(const prrtc_problem* problems, int32_t n, const prrtc_params* params, int32_t trials,
                   prrtc_params* best, double* best_ms);

/* ------------------------------------------------------------ learned proposal: dense layers */
/* BF16 GEMM on the tensor cores (tcgen05, FP32 accumulation in tensor memory)
 * for the dense layers of the learned sampling proposal:
 *   C[M, N] = A[M, K] * B[N, K]^T (+ bias[N]) (then ReLU if relu != 0).
 * A and B are row-major BF16 device arrays (K contiguous, 16-byte aligned);
 * c32 (FP32, row stride N) and/or c16 (BF16, row stride N) receive C; either
 * may be null but not both.  K and N must be multiples of 8
 * (PRRTC_ERR_UNSUPPORTED otherwise).  Enqueued on `stream`; no
 * synchronisation.  prrtc_gemm_error() returns and clears the error word of
 * the kernels (a bounded device wait that gave up: PRRTC_ERR_TIMEOUT). */
int prrtc_gemm_bf16(const void* a, const void* b, int32_t M, int32_t N, int32_t K, const float* bias,
                    int32_t relu, float* c32, void* c16, void* stream);
/* As prrtc_gemm_bf16 with the K dimension split into `splits` ranges (0 = the
 * library's choice, which splits while the 128 x 256 output tiles fill less
 * than one wave of SMs).  Each range writes an FP32 partial tile to a
 * library-owned workspace (per device and stream, grown on demand); a second
 * kernel sums the partials in range order, so results do not depend on
 * timing, then applies bias, ReLU and the output conversions. */
int prrtc_gemm_bf16_splitk(const void* a, const void* b, int32_t M, int32_t N, int32_t K, const float* bias,
                           int32_t relu, float* c32, void* c16, int32_t splits, void* stream);
int prrtc_gemm_error(void);

/* ------------------------------------------------------------ learned proposal */
/* Not part of the paper (which samples uniformly): an MLP maps [start, goal,
 * 16^3 occupancy grid of the 1.6 m workspace] to an 8-component diagonal
 * Gaussian mixture over joint values normalised to [-1, 1].  Mixed with
 * uniform sampling at params->learned_ratio, so planning stays
 * probabilistically complete; the collision checker remains the judge.
 * Layers 4160 -> 1024 -> 512 -> 512 -> 8(1 + 2 dof) (padded to 128), ReLU,
 * BF16 weights and activations on the tensor cores, FP32 accumulation, FP32
 * master weights and Adam moments.  Flat parameter layout:
 * [W1 (1024 x 4160), b1, W2 (512 x 1024), b2, W3 (512 x 512), b3,
 *  W4 (head x 512), b4], W row-major [out x in].  Input row:
 * [occupancy (voxel i + 16 j + 256 k, centre (-0.8, -0.8, 0) + 0.1 (idx + 0.5),
 *  occupied iff closer than 0.05 m to an obstacle) | 2 (q_start - lo)/(hi - lo) - 1
 *  padded to 32 | same for q_goal].  All calls are synchronous. */
typedef struct prrtc_proposal prrtc_proposal;

/* params: host [n_params] FP32 initial parameters, or null for zeros. */
int prrtc_proposal_create(int32_t dof, const float* lower, const float* upper, const float* params,
                          prrtc_proposal** out);
void prrtc_proposal_destroy(prrtc_proposal* proposal);
int prrtc_proposal_info(const prrtc_proposal* proposal, int32_t* dof, int32_t* head, int64_t* n_params,
                        int32_t* step);
/* Copies the FP32 master parameters and/or the last computed gradients (host [n_params]). */
int prrtc_proposal_get_params(const prrtc_proposal* proposal, float* params, float* grads);
/* Raw head output for B inputs: occ host [B * 4096] (0/1), q_* host [B * dof];
 * out host [B * head]. */
int prrtc_proposal_forward(prrtc_proposal* proposal, const uint8_t* occ, const float* q_start,
                           const float* q_goal, int32_t B, float* out);
/* The same forward with its intermediate values, for element-wise tests of
 * each layer: x host [B * 4160] (the BF16 input features: occupancy, then
 * start and goal normalised to [-1, 1], each zero-padded to 32), h1 / h2 / h3
 * host [B * 1024], [B * 512], [B * 512] (the BF16 activations after bias and
 * ReLU), out host [B * head] (FP32 head), BF16 values widened to FP32.  Any
 * output may be null. */
int prrtc_proposal_forward_layers(prrtc_proposal* proposal, const uint8_t* occ, const float* q_start,
                                  const float* q_goal, int32_t B, float* x, float* h1, float* h2, float* h3,
                                  float* out);
/* The hidden activations (BF16 widened to FP32, host [B * 1024], [B * 512],
 * [B * 512]; any may be null) of the first B problems of the last inference
 * batch of this proposal (prrtc_proposal_mixtures or prrtc_plan_batch_learned),
 * for element-wise tests of the fused inference kernel.  B larger than that
 * batch: PRRTC_ERR_INVALID_ARG. */
int prrtc_proposal_inference_layers(prrtc_proposal* proposal, int32_t B, float* h1, float* h2, float* h3);
/* Mean mixture negative log-likelihood of target [B * dof] and its gradient
 * (stored in the proposal, read with prrtc_proposal_get_params); no update. */
int prrtc_proposal_grads(prrtc_proposal* proposal, const uint8_t* occ, const float* q_start,
                         const float* q_goal, const float* target, int32_t B, float* loss);
/* `steps` Adam steps (learning rate lr) on batches drawn without replacement
 * from n_samples samples (seeded shuffle per epoch); sample i uses occupancy
 * row scene_of[i] of occ [n_scenes * 4096].  losses (nullable) host [steps]. */
int prrtc_proposal_train(prrtc_proposal* proposal, const uint8_t* occ, int32_t n_scenes, const int32_t* scene_of,
                         const float* q_start, const float* q_goal, const float* target, int32_t n_samples,
                         int32_t batch, int32_t steps, float lr, uint64_t seed, float* losses);
/* Checkpoint: header (magic, version, dof, head, n_params, step, limits) then
 * FP32 master parameters and Adam moments. */
int prrtc_proposal_save(const prrtc_proposal* proposal, const char* path);
int prrtc_proposal_load(const char* path, prrtc_proposal** out);
/* Occupancy grid of an environment (host [4096]), computed on the device. */
int prrtc_occupancy(const prrtc_env* env, uint8_t* out);
/* The mixtures prrtc_plan_batch_learned would sample from for B problems
 * (envs[b], q_start / q_goal host [B * dof]), inferred on the device by the
 * same code: out host [B * (8 + 16 dof)] in the layout of prrtc_problem.gmm,
 * log-sigmas clamped to [-5, 2].  The occupancy part of the first layer is
 * computed once per distinct environment of the batch (environments are
 * told apart by their device data); the first layer then differs from
 * prrtc_proposal_forward's single contraction by FP32 summation order only.
 * Errors: PRRTC_ERR_INVALID_ARG (null or non-finite input), PRRTC_ERR_OOM,
 * PRRTC_ERR_CUDA. */
int prrtc_proposal_mixtures(prrtc_proposal* proposal, const prrtc_env* const* envs, const float* q_start,
                            const float* q_goal, int32_t B, float* out);

/* prrtc_plan_batch with the learned proposal: for every problem whose
 * proposals[p] is non-null (its DoF must match the robot's), the mixture is
 * inferred on the device from the problem's environment, start and goal and
 * used with params->learned_ratio.  proposals may be null (plain planning). */
int prrtc_plan_batch_learned(const prrtc_problem* problems, prrtc_proposal* const* proposals, int32_t n,
                             const prrtc_params* params, prrtc_path* out_paths, int32_t* out_status);

/* ------------------------------------------------------------ serving loop */
/* Continuous-batching request loop (not part of the paper).  Queries are
 * submitted from any thread; a server thread admits them into free device
 * slots (their number follows memory_budget_bytes), snapshots each query's
 * environment at admission (later prrtc_env_update calls affect only later
 * admissions), infers learned mixtures on the device, and runs the planner
 * in resumable time slices of slice_us device microseconds over every
 * occupied slot: queries that arrive while others plan join the next slice
 * and their work overlaps on the device.  Finished queries are returned by
 * prrtc_server_poll.  In PRRTC_MODE_SERIAL a query's result does not depend
 * on what else is in flight. */
typedef struct prrtc_server prrtc_server;

typedef struct prrtc_server_config {
  int32_t max_slots;           /* 0 = as many as memory_budget_bytes allows           */
  int32_t slice_us;            /* device time slice between admissions (>= 10)         */
  int64_t memory_budget_bytes; /* device memory for query slots (trees, paths, env)    */
  prrtc_params params;         /* planner parameters for every query                    */
} prrtc_server_config;

typedef struct prrtc_server_stats {
  int32_t slots;
  int32_t active;
  int64_t submitted, admitted, completed, pending, slices;
  double busy_s;               /* host time spent in server rounds                     */
  double uptime_s;
} prrtc_server_stats;

/* Defaults: 2 GiB budget, 500 us slices, prrtc_params_default with 8192 nodes
 * per tree and 4096 waypoints per path. */
void prrtc_server_config_default(prrtc_server_config* config);
int prrtc_server_create(const prrtc_server_config* config, prrtc_server** out);
/* Queue a query (copied; the handles must outlive it).  proposal (nullable,
 * DoF of the robot) turns on learned sampling with params.learned_ratio; a
 * proposal must not be used by another call at the same time. */
int prrtc_server_submit(prrtc_server* server, const prrtc_problem* problem, prrtc_proposal* proposal,
                        uint64_t* ticket);
/* Up to max finished queries, oldest first: paths (free q with
 * prrtc_path_free), tickets, latency from submission to completion and time
 * spent waiting for a slot (host clock, ms); any output array may be null. */
int prrtc_server_poll(prrtc_server* server, int32_t max, prrtc_path* paths, uint64_t* tickets, double* latency_ms,
                      double* queue_ms, int32_t* n_out);
/* Block until at least `completed` queries have finished or timeout_s passes
 * (PRRTC_ERR_TIMEOUT). */
int prrtc_server_wait(prrtc_server* server, int64_t completed, double timeout_s);
int prrtc_server_get_stats(prrtc_server* server, prrtc_server_stats* out);
/* Stops the loop (after the current slice) and frees everything. */
void prrtc_server_destroy(prrtc_server* server);

/* ------------------------------------------------------------ planning without allocation */
/* The paper has no counterpart of this entry point; it exists for callers
 * that must not allocate device memory while they plan -- a real-time control
 * thread that cannot block in an allocator, or an application whose framework
 * owns all device memory through its own pool or budget.  The call waits for
 * its stream and reads results back synchronously, so it is not for use
 * inside another component's stream capture.
 *
 * prrtc_plan_noalloc solves one problem like prrtc_plan but keeps the trees,
 * the planner state and the path in one fixed, file-scope device array of
 * about 0.8 MiB, resident on every GPU that loads the library until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Robot and env handles are created beforehand with the usual
 * calls (those do allocate).
 *   params->tree_capacity and params->path_capacity must be <=
 *   PRRTC_NOALLOC_MAX_ROWS, else PRRTC_ERR_INVALID_ARG (nothing runs).
 *   path_out: host buffer of path_rows * dof floats owned by the caller; a
 *   path longer than path_rows is reported as PRRTC_PATH_OVERFLOW.
 *   info_out: host struct filled like prrtc_plan's path; its q points at
 *   path_out (nothing to free).  prrtc_last_error() is not updated.
 *   stream: cudaStream_t the kernels run on (0 = legacy default stream); the
 *   call returns after the stream has completed them.
 * The first call on a device resolves the array's address and marks every
 * tree row unwritten; make that first call before any stream capture.  Every
 * call shares the one array and leaves its contents for the next; calls that
 * overlap on the GPU (other threads or streams) race on it and must be
 * serialised by the caller.  A device reset (cudaDeviceReset) between calls
 * is not supported: the first-call set-up is not repeated afterwards. */
#define PRRTC_NOALLOC_MAX_ROWS 4096
int prrtc_plan_noalloc(const prrtc_robot* robot, const prrtc_env* env, const float* q_start,
                       const float* q_goal, const prrtc_params* params, float* path_out,
                       int32_t path_rows, prrtc_path* info_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
