// prrtc_launch.h -- descriptors shared by the host runtime and the planner
// kernels, and the kernel launchers each .cu file exports.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "prrtc.h"
#include "prrtc_device.cuh"

namespace prrtc {

constexpr int kRootParent = -2;    // parent of a tree root
constexpr int kMixK = 8;           // learned mixture components
constexpr int kGmmStride = kMixK + 2 * kMixK * kMaxDof;  // logits | means [8][16] | log-sigmas [8][16]
constexpr int kUnsetParent = -1;   // parent slot not written yet (0xFF fill)
constexpr int kHeldMeta = 8;       // ints per lockstep worker record

// Launch-wide parameters and bookkeeping (one per planning launch).
struct PlanGlobals {
  int n_problems;
  int mode;              // PRRTC_MODE_*
  int max_iters;
  int n_full;            // ceil(range / resolution): states of a full-length step
  float range;
  float resolution;
  uint32_t bias_thr;     // goal bias as a threshold on the top 24 bits of a Philox word
  int path_cap;
  unsigned long long t0;             // launch start (min over blocks, %globaltimer ns)
  unsigned long long time_limit_ns;  // 0 = none
  int cursor;            // work-queue ticket counter
  int error;             // device-side error code (PRRTC_ERR_*), 0 = none
  int error_info;
  uint32_t learned_thr;  // learned-vs-uniform draw as a threshold on the top 24 bits of a Philox word
  const int* active;     // problems of this launch as indices into the descriptors (null: 0..n-1)
  unsigned long long slice_ns;  // 0 = run problems to completion; else stop starting iterations
                                // this long after the launch start (problems resume next launch)
  int sampler;           // PRRTC_SAMPLER_*
  uint32_t halton_offset;
  float dd_radius;       // dynamic domain: 0 = off
  float dd_alpha;
  float dd_min_radius;
  int workers;           // lockstep mode: iterations per round (B)
  uint32_t debug_wait_polls;  // test hook: bounded wait on ProblemState::never_set before a path walk
  int expansions;        // async: iterations a worker claims per atomic on the problem's counter
  int obstacle_tile;     // primitives per type per first-stage round (32 or 64): picks the kernel instance
};

// Check of the sampler and dynamic-domain fields of a parameter block; null
// when they are usable, else the reason.
inline const char* sampling_params_problem(const prrtc_params& p) {
  if (p.sampler != PRRTC_SAMPLER_PHILOX && p.sampler != PRRTC_SAMPLER_HALTON) return "unknown sampler";
  if (!(p.dd_radius >= 0.f)) return "dd_radius must be >= 0";
  if (p.dd_radius > 0.f) {
    if (!(p.dd_alpha >= 0.f && p.dd_alpha < 1.f)) return "dd_alpha must be in [0, 1)";
    if (!(p.dd_min_radius >= 0.f) || !std::isfinite(p.dd_min_radius)) return "dd_min_radius must be >= 0";
  }
  return nullptr;
}

// The launch-wide fields that follow from a parameter block alone.
inline void globals_from_params(PlanGlobals& G, const prrtc_params& p) {
  G.mode = p.mode;
  G.max_iters = p.max_iters;
  G.n_full = (int)std::ceil((double)p.range / (double)p.resolution);
  if (G.n_full < 1) G.n_full = 1;
  G.range = p.range;
  G.resolution = p.resolution;
  G.bias_thr = (uint32_t)std::ceil((double)p.goal_bias * 16777216.0);
  G.learned_thr = (uint32_t)std::ceil((double)p.learned_ratio * 16777216.0);
  G.path_cap = p.path_capacity;
  G.sampler = p.sampler;
  G.halton_offset = p.halton_offset;
  G.dd_radius = p.dd_radius;
  G.dd_alpha = p.dd_alpha;
  G.dd_min_radius = p.dd_min_radius;
  G.workers = p.mode == PRRTC_MODE_LOCKSTEP ? p.workers : 1;
  G.debug_wait_polls = p.debug_wait_polls > 0 ? (uint32_t)p.debug_wait_polls : 0u;
  G.expansions = (p.mode == PRRTC_MODE_ASYNC && p.expansions > 1) ? p.expansions : 1;
  G.obstacle_tile = p.obstacle_tile == 64 ? 64 : 32;
}

// Per-problem inputs (uploaded every call).
struct ProblemDesc {
  const RobotDev* robot;
  EnvView env;
  float* nodes[2];       // [cap * dpad] per tree, rows NaN until written
  int* parent[2];        // [cap] per tree
  float* radius[2];      // [cap] per tree: dynamic-domain radius, NaN = unbounded
  float* path;           // [path_cap * dof]
  int* path_idx;         // [path_cap] scratch of (tree << 30 | node)
  int cap;
  int dpad;
  int dof;
  int n_spheres;         // distinct spheres (staging size)
  int n_pairs;
  uint32_t key_lo, key_hi;
  uint32_t pid;
  const float* gmm;      // learned mixture (kGmmStride floats, device) or null
  // lockstep mode: the rows each worker of a round holds back, [workers][held_rows * dpad],
  // and per worker kHeldMeta ints (see LockstepHeld in prrtc_plan.cu); null otherwise
  float* held;
  int* held_meta;
  int held_rows;         // rows one iteration can add: 1 + the most connect steps
  float q_start[kMaxDof];
  float q_goal[kMaxDof];
};

// Per-problem device state.  The setup kernel resets everything but the
// arena bookkeeping (used[]), which tells it which rows to clear next time.
struct ProblemState {
  int iter;              // Alg. 1 iteration tickets handed out
  int count[2];          // tree sizes (may exceed cap after failed insertions)
  int solved;
  int done;
  int timed_out;
  int pre_status;        // start / goal in collision
  int s_tree;            // tree extended by the winning iteration
  int join_s, join_o;
  int path_n;
  int path_status;
  double cost;
  unsigned long long t_solve;
  unsigned long long edges, edge_states, sphere_tests, pair_tests, fk_states, nn_nodes, iterations, insert_fail;
  unsigned long long dd_rejected;
  unsigned long long prim_tests[4];
  unsigned long long verdict_states;
  // arena bookkeeping, preserved across launches
  int used_rows[2];
  int used_dpad;
  int never_set;         // stays 0: the flag the bounded-wait test hook waits on
};

// Alg. 1 iterations a problem ran: the tickets handed out, or with batched
// claims (expansions > 1) the iteration bodies the workers counted.
inline int reported_iterations(const ProblemState& S, const prrtc_params& p) {
  const long long n = (p.mode == PRRTC_MODE_ASYNC && p.expansions > 1) ? (long long)S.iterations : (long long)S.iter;
  return (int)(n < p.max_iters ? n : p.max_iters);
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_check_states(const RobotDev* robot, const RobotHeader& host_header, EnvView env, const float* q,
                                int n, uint8_t* valid, float* spheres, unsigned long long* counters, int* error,
                                cudaStream_t stream);

// Philox4x32-10 of n counters (device arrays of 4n words each).
cudaError_t launch_philox(const uint32_t* ctr, int n, uint64_t key, uint32_t* out, cudaStream_t stream);

// FP32 FMA loop over 8 blocks of 256 threads per SM; *lane_ops receives the
// FMAs it issues (one lane-op each).  sink: one float per block (never written
// in practice).
cudaError_t launch_fma_loop(int sm_count, int iters, float* sink, cudaStream_t stream, long long* lane_ops);

// idx (nullable, device): the problems to set up, as indices into desc/state.
// error (nullable, device): receives PRRTC_ERR_TIMEOUT if a block's staging
// copies did not complete within the bounded wait.
cudaError_t launch_setup(const ProblemDesc* desc, ProblemState* state, int n, int max_spheres, int max_pairs,
                         int max_env_f4, cudaStream_t stream, const int* idx = nullptr, int* error = nullptr);

struct PlanLaunch {
  int grid;
  int warps;
  bool lockstep;         // lockstep_kernel (PRRTC_MODE_LOCKSTEP) instead of plan_kernel
  int smem;
  int robot_bytes;
  int env_bytes;
  int stage_bytes;
};

// workers: the lockstep round size (PRRTC_MODE_LOCKSTEP), else ignored.
PlanLaunch plan_launch_config(int n_problems, int mode, int blocks, int warps, int max_spheres, int max_pairs,
                              int max_env_f4, int sm_count, int workers = 1);

// obstacle_tile: 64 launches the 64-obstacle-tile instance of the async/serial
// kernel, anything else the 32 one (lockstep always uses 32).  lean: the
// instance without the learned mixture draw, the Halton sampler, distance
// fields, oriented boxes and one-stage links; only for batches that use none of
// them
// (problem_is_lean).
cudaError_t launch_plan(const PlanGlobals* g, const ProblemDesc* desc, ProblemState* state, const PlanLaunch& cfg,
                        int obstacle_tile, bool lean, cudaStream_t stream);

// Whether the lean planner instance serves a problem: no mixture, no distance
// field, at least one primitive and no oriented box, a bounding sphere on every
// robot link that has spheres (with the sphere hierarchy on), and revolute
// joints within +-3.2 rad.  The batch also needs Philox sampling and no dynamic
// domain.  The batch is lean when every
// problem is and the sampler is Philox.
inline bool problem_is_lean(const RobotHeader& H, const ProblemDesc& D) {
  if (D.gmm || D.env.esdf.v || D.env.n_float4() == 0 || D.env.n_obb || !H.two_stage) return false;
  for (int f = 0; f < H.dof; ++f) {
    if (H.sph_begin[f + 1] > H.sph_begin[f] && !(H.coarse[f].w > 0.f)) return false;
    // every joint value the planner forms lies between the limits, the start and
    // the goal: within +-3.2 rad the hardware sine/cosine is the one taken
    const bool revolute = H.jtype[f] == kRevZ || H.jtype[f] == kRevY || H.jtype[f] == kRevX;
    const float lo = std::min({H.lo[f], D.q_start[f], D.q_goal[f]});
    const float hi = std::max({H.lo[f] + H.span[f], D.q_start[f], D.q_goal[f]});
    if (revolute && !(lo >= -3.2f && hi <= 3.2f)) return false;
  }
  return true;
}

// Clear-list bookkeeping after a plan: rows each tree used, for the next setup.
cudaError_t launch_record_usage(const ProblemDesc* desc, ProblemState* state, int n, cudaStream_t stream,
                                const int* idx = nullptr);

// Copy every problem's path into one packed buffer; offsets[p]..offsets[p+1]
// is problem p's float range (n + 1 entries, device memory).
cudaError_t launch_gather_paths(const ProblemDesc* desc, const int* offsets, int n, float* out, cudaStream_t stream);

// The first `rows` rows of each solved problem's path (dof floats per row)
// into out + p * stride; stride >= rows * dof.
cudaError_t launch_gather_heads(const ProblemDesc* desc, const ProblemState* state, int n, int rows, int stride,
                                float* out, cudaStream_t stream);

// Distance fields (prrtc_esdf.cu): occupancy of voxel centres inside the
// environment's primitives, and the signed distance transform of an
// occupancy grid (tmp_a, tmp_b: V int2 each).
cudaError_t launch_voxelize(const EnvView& env, const float origin[3], float voxel, const int dims[3], uint8_t* occ,
                            cudaStream_t stream);
cudaError_t launch_esdf(const uint8_t* occ, const int dims[3], float voxel, int2* tmp_a, int2* tmp_b, float* out,
                        cudaStream_t stream);

// Tensor-core GEMM (prrtc_gemm.cu): C[M,N] = A[M,K] B[N,K]^T (+bias, ReLU).
int gemm_bf16(const void* a, const void* b, int M, int N, int K, const float* bias, int relu, float* c32, int ldc32,
              void* c16, int ldc16, cudaStream_t stream);
// The same with row strides lda / ldb (elements, multiples of 8, >= K) of the
// operands, e.g. a column range of a wider weight matrix; splits_hint 0 = auto.
int gemm_bf16_ld(const void* a, int lda, const void* b, int ldb, int M, int N, int K, const float* bias, int relu,
                 float* c32, int ldc32, void* c16, int ldc16, cudaStream_t stream, int splits_hint);
int gemm_take_error();

// Fused inference of the learned proposal after the occupancy part of its
// first layer (prrtc_gemm.cu): first hidden layer from its per-environment
// occupancy part plus the start / goal part, the three tensor-core layers,
// and the mixture parameters written into the planner's rows -- one launch.
// Weights and activations are pre-tiled: [slice or row tile][64-column
// k-block] blocks in the 128-byte-swizzled layout of the MMA operands
// (weights: kIC = 8 slices of out/8 rows, tiled by mlp_tile_weights;
// activations: 128-row tiles, buffers of ceil(rows / 128) * 128 rows).
struct MlpInferArgs {
  int rows, B, dof;            // rows: activation rows (B rounded up to 8)
  int h0, h1, h2, head;        // widths: hidden 1, 2, 3 and the padded head
  int qpad;                    // start / goal input columns per side
  const float* h1o;            // [U x h0] occupancy part of hidden 1, one row per environment
  const int* row_env;          // [rows] environment row of each problem
  const float* qs;             // [B x dof] starts
  const float* qg;             // [B x dof] goals
  const float* lo;             // [dof] joint lower limits
  const float* span;           // [dof] upper - lower
  const void* wq;              // BF16 [2 qpad x h0]: start / goal columns of layer 1, transposed
  const void* w[3];            // tiled BF16 weights of layers 2, 3 and the head
  const float* bias[4];        // biases of layers 1..4
  void* act[3];                // tiled BF16 activations of hidden layers 1, 2, 3
  float* const* gmm_rows;      // [B] planner mixture rows (device pointers)
  int mix_k, gmm_dof;          // planner layout: logits[mix_k] | means[mix_k][gmm_dof] | log-sigmas
                               // (entries of joints >= dof are not written; the planner skips them)
  float logsig_lo, logsig_hi;  // log-sigma clamp
};
// PRRTC_OK when the fused kernel supports these layer widths.
int mlp_check_shapes(int h0, int h1, int h2, int head);
// Weight matrix [N x K] (BF16, row-major) -> the tiled layout above.
int mlp_tile_weights(const void* w, int N, int K, void* out, cudaStream_t stream);
int mlp_infer(const MlpInferArgs& a, cudaStream_t stream);

}  // namespace prrtc
