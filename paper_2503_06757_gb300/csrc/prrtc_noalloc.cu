// prrtc_noalloc.cu -- single-problem planning that allocates nothing.
//
// Some callers cannot allocate device memory when they plan: a real-time
// control thread that must not block in the allocator, or a host application
// whose framework owns every byte of device memory through its own pool or
// budget.  prrtc_plan_noalloc serves them: the trees, the per-problem state
// and the path buffer of the planner kernels live in one file-scope static
// device array of fixed size, and the caller supplies the stream and the host
// buffers for the results.  The call synchronises its stream and copies the
// results back before it returns.
//
// The array is shared by every call on a device and keeps the contents of the
// last call.  The set-up on the first call per device fills the tree rows
// with NaN (the planner's "not yet written" marker); each call's setup kernel
// then clears exactly the rows the previous call wrote and zeroes the state.
// Calls that overlap on the GPU (two host threads, or two streams) race on
// the same array and must be serialised by the caller.  The per-device
// set-up flag lives for the process: a device reset between calls is not
// supported.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "prrtc.h"
#include "prrtc_launch.h"

namespace prrtc {
namespace {

constexpr int kNoAllocRows = PRRTC_NOALLOC_MAX_ROWS;

struct alignas(256) NoAllocScratch {
  PlanGlobals glob;
  ProblemDesc desc;
  ProblemState state;
  alignas(16) int path_idx[kNoAllocRows];
  alignas(16) int parents[2][kNoAllocRows];
  alignas(16) float radius[2][kNoAllocRows];
  alignas(16) float path[kNoAllocRows * kMaxDof];
  alignas(16) float nodes[2][kNoAllocRows * kMaxDof];
};

// The only device memory this entry point uses (about 0.8 MiB per device,
// resident from module load until the process exits).
static __device__ __align__(256) unsigned char prrtc_noalloc_scratch[sizeof(NoAllocScratch)];

struct NoAllocDevice {
  bool ready = false;
  NoAllocScratch* scratch = nullptr;  // device address of prrtc_noalloc_scratch
};

NoAllocDevice g_noalloc[64];
std::mutex g_noalloc_mu;

// First call on a device: resolve the array's device address (host code only
// holds a stand-in symbol) and mark every tree row unwritten.
int noalloc_setup(int dev, cudaStream_t stream, NoAllocScratch** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, prrtc_noalloc_scratch);
    if (e != cudaSuccess) return PRRTC_ERR_CUDA;
    NoAllocScratch* s = static_cast<NoAllocScratch*>(p);
    e = cudaMemsetAsync(s->nodes, 0xFF, sizeof(s->nodes), stream);                       // NaN rows
    if (e == cudaSuccess) e = cudaMemsetAsync(s->parents, 0xFF, sizeof(s->parents), stream);  // unset parents
    if (e == cudaSuccess) e = cudaMemsetAsync(s->radius, 0xFF, sizeof(s->radius), stream);    // NaN radii
    if (e == cudaSuccess) e = cudaMemsetAsync(&s->state, 0, sizeof(s->state), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return PRRTC_ERR_CUDA;
    d.scratch = s;
    d.ready = true;
  }
  *out = d.scratch;
  return PRRTC_OK;
}

}  // namespace
}  // namespace prrtc

using namespace prrtc;

// Handle internals needed to fill a descriptor (defined in prrtc_api.cu).
extern "C" int prrtc_internal_views(const prrtc_robot* robot, const prrtc_env* env, const void** robot_dev,
                                    const void** robot_header, EnvView* env_view, int* device);

extern "C" int prrtc_plan_noalloc(const prrtc_robot* robot, const prrtc_env* env, const float* q_start,
                                  const float* q_goal, const prrtc_params* params, float* path_out,
                                  int32_t path_rows, prrtc_path* info_out, void* stream_ptr) {
  if (!robot || !env || !q_start || !q_goal || !params || !info_out || (path_rows > 0 && !path_out) || path_rows < 0)
    return PRRTC_ERR_INVALID_ARG;
  // Sizes beyond the fixed scratch are refused, never truncated.
  if (params->tree_capacity > kNoAllocRows || params->path_capacity > kNoAllocRows) return PRRTC_ERR_INVALID_ARG;
  if (params->tree_capacity < 2 || params->path_capacity < 2 || params->max_iters < 1 || !(params->range > 0.f) ||
      !(params->resolution > 0.f) || !(params->goal_bias >= 0.f && params->goal_bias <= 1.f) ||
      (params->mode != PRRTC_MODE_ASYNC && params->mode != PRRTC_MODE_SERIAL) || params->blocks < 0 ||
      params->warps_per_block < 0 || params->warps_per_block > 16 || params->time_limit_s < 0.0 ||
      (double)params->range / (double)params->resolution > 4096.0 || sampling_params_problem(*params))
    return PRRTC_ERR_INVALID_ARG;
  const void* robot_dev = nullptr;
  const void* header = nullptr;
  EnvView ev{};
  int handle_dev = -1;
  int rc = prrtc_internal_views(robot, env, &robot_dev, &header, &ev, &handle_dev);
  if (rc) return rc;
  const RobotHeader& H = *static_cast<const RobotHeader*>(header);
  for (int j = 0; j < H.dof; ++j)
    if (!std::isfinite(q_start[j]) || !std::isfinite(q_goal[j]))
      return PRRTC_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return PRRTC_ERR_NO_DEVICE;
  if (dev != handle_dev) return PRRTC_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  NoAllocScratch* S = nullptr;
  rc = noalloc_setup(dev, stream, &S);
  if (rc) return rc;

  // Descriptor and launch parameters, built on the host stack.
  ProblemDesc D;
  std::memset(&D, 0, sizeof(D));
  D.robot = static_cast<const RobotDev*>(robot_dev);
  D.env = ev;
  D.nodes[0] = S->nodes[0];
  D.nodes[1] = S->nodes[1];
  D.parent[0] = S->parents[0];
  D.parent[1] = S->parents[1];
  D.radius[0] = S->radius[0];
  D.radius[1] = S->radius[1];
  D.path = S->path;
  D.path_idx = S->path_idx;
  D.cap = params->tree_capacity;
  D.dpad = H.dpad;
  D.dof = H.dof;
  D.n_spheres = H.n_spheres;
  D.n_pairs = H.n_pairs;
  D.key_lo = (uint32_t)(params->seed & 0xffffffffu);
  D.key_hi = (uint32_t)(params->seed >> 32);
  D.pid = 0;
  for (int j = 0; j < H.dof; ++j) {
    D.q_start[j] = q_start[j];
    D.q_goal[j] = q_goal[j];
  }
  PlanGlobals G;
  std::memset(&G, 0, sizeof(G));
  G.n_problems = 1;
  globals_from_params(G, *params);
  G.learned_thr = 0;  // no mixtures on this path
  G.t0 = ULLONG_MAX;
  G.time_limit_ns = (unsigned long long)(params->time_limit_s * 1e9);

  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PRRTC_ERR_CUDA;
  const PlanLaunch cfg = plan_launch_config(1, params->mode, params->blocks, params->warps_per_block,
                                            H.n_spheres + H.dof, H.n_pairs, ev.n_float4(), sms);
  if (cfg.smem > 227 * 1024) return PRRTC_ERR_UNSUPPORTED;

  cudaError_t e = cudaMemcpyAsync(&S->desc, &D, sizeof(D), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&S->glob, &G, sizeof(G), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = launch_setup(&S->desc, &S->state, 1, H.n_spheres + H.dof, H.n_pairs, ev.n_float4(), stream, nullptr,
                     &S->glob.error);
  if (e == cudaSuccess) e = launch_plan(&S->glob, &S->desc, &S->state, cfg, G.obstacle_tile, false, stream);
  if (e == cudaSuccess) e = launch_record_usage(&S->desc, &S->state, 1, stream);
  ProblemState st;
  PlanGlobals gout;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, &S->state, sizeof(st), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&gout, &S->glob, sizeof(gout), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return PRRTC_ERR_CUDA;

  int status;
  if (st.pre_status) status = st.pre_status;
  else if (st.solved) status = (st.path_status == PRRTC_SOLVED || st.path_status == PRRTC_PATH_OVERFLOW) ? st.path_status : PRRTC_ERR_TIMEOUT;
  else if (st.timed_out) status = PRRTC_TIME_LIMIT;
  else status = PRRTC_NO_SOLUTION;
  if (status == PRRTC_SOLVED && st.path_n > path_rows) status = PRRTC_PATH_OVERFLOW;
  if (status == PRRTC_SOLVED && st.path_n > 0) {
    e = cudaMemcpyAsync(path_out, S->path, (size_t)st.path_n * H.dof * sizeof(float), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return PRRTC_ERR_CUDA;
  }
  std::memset(info_out, 0, sizeof(*info_out));
  info_out->status = status;
  info_out->n = (status == PRRTC_SOLVED || status == PRRTC_PATH_OVERFLOW) ? st.path_n : 0;
  info_out->dof = H.dof;
  info_out->iterations = reported_iterations(st, *params);
  info_out->q = (status == PRRTC_SOLVED) ? path_out : nullptr;
  info_out->cost = st.cost;
  info_out->nodes_a = std::min(st.count[0], params->tree_capacity);
  info_out->nodes_b = std::min(st.count[1], params->tree_capacity);
  info_out->edges_checked = (int64_t)st.edges;
  info_out->edge_states = (int64_t)st.edge_states;
  info_out->solve_time_us = (st.solved && st.t_solve >= gout.t0) ? (double)(st.t_solve - gout.t0) * 1e-3 : -1.0;
  info_out->sphere_tests = (int64_t)st.sphere_tests;
  info_out->pair_tests = (int64_t)st.pair_tests;
  info_out->fk_states = (int64_t)st.fk_states;
  info_out->nn_nodes = (int64_t)st.nn_nodes;
  info_out->dd_rejected = (int64_t)st.dd_rejected;
  info_out->verdict_states = (int64_t)st.verdict_states;
  for (int k = 0; k < 4; ++k) info_out->prim_tests[k] = (int64_t)st.prim_tests[k];
  if (gout.error) return gout.error;
  return PRRTC_OK;
}
