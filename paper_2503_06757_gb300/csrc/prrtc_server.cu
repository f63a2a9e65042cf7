// prrtc_server.cu -- continuous-batching request loop for planning queries.
//
// Clients submit queries from any thread; a server thread owns the device:
//   1. admit pending queries into free arena slots (the slot count follows a
//      device-memory budget); each admitted query gets a private snapshot of
//      its environment, so dynamic-obstacle updates published with
//      prrtc_env_update apply to queries admitted afterwards and never change
//      the obstacles of a query in flight;
//   2. infer learned mixtures for the new queries, set up their trees;
//   3. run one planner launch over every occupied slot for a device time
//      slice -- trees and counters persist, so unfinished queries resume in
//      the next slice and queries that arrived meanwhile join them;
//   4. harvest finished queries (path copied out, slot freed).
// This is the persistent planner of prrtc_plan_batch run as resumable slices
// (not a queue in front of one-shot launches): work of queries admitted at
// different times overlaps on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "prrtc.h"
#include "prrtc_launch.h"

using namespace prrtc;

extern "C" int prrtc_internal_env_snapshot(prrtc_env* env, float4* dst, int max_f4, EnvView* view,
                                           cudaStream_t stream);
extern "C" int prrtc_internal_robot_view(const prrtc_robot* robot, const RobotDev** dev, const RobotHeader** header,
                                         int* device);
extern "C" void prrtc_internal_set_error(const char* msg);
int prrtc_internal_proposal_mixtures(prrtc_proposal* p, const EnvView* envs, const float* qs_host,
                                     const float* qg_host, int B, float* const* gmm_rows, cudaStream_t stream);

namespace {

constexpr int kEnvSnapF4 = 2048;  // per-slot obstacle snapshot (32 KiB): up to ~1000 primitives

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Query {
  uint64_t ticket = 0;
  const prrtc_robot* robot = nullptr;
  prrtc_env* env = nullptr;
  prrtc_proposal* proposal = nullptr;
  std::vector<float> qs, qg, gmm;
  uint64_t seed = 0;
  uint32_t pid = 0;
  double t_submit = 0, t_admit = 0;
  int slot = -1;
  int slices = 0;
};

struct Done {
  uint64_t ticket;
  prrtc_path path;
  double latency_ms, queue_ms;
  int slices;
};

}  // namespace

struct prrtc_server {
  int device = -1;
  int sms = 0;
  cudaStream_t stream = nullptr;
  prrtc_params params{};
  int slots = 0;
  int slice_us = 0;
  // device arenas
  float* nodes = nullptr;
  int* parents = nullptr;
  float* paths = nullptr;
  int* path_idx = nullptr;
  float4* env_snap = nullptr;
  float* d_gmm = nullptr;
  ProblemDesc* d_desc = nullptr;
  ProblemState* d_state = nullptr;
  PlanGlobals* d_glob = nullptr;
  int* d_active = nullptr;
  int* d_new = nullptr;
  ProblemDesc* h_desc = nullptr;
  ProblemState* h_state = nullptr;
  PlanGlobals* h_glob = nullptr;
  int* h_active = nullptr;
  int* h_new = nullptr;
  float* h_gmm = nullptr;
  // host bookkeeping
  std::vector<Query*> slot_query;
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Query*> pending;
  std::deque<Done> done;
  std::thread thread;
  std::atomic<bool> stop{false};
  uint64_t next_ticket = 1;
  int error = 0;
  // statistics
  int64_t submitted = 0, admitted = 0, completed = 0, slices = 0;
  double busy_s = 0, t_start = 0;
};

namespace {

void free_server(prrtc_server* s) {
  cudaFree(s->nodes); cudaFree(s->parents); cudaFree(s->paths); cudaFree(s->path_idx); cudaFree(s->env_snap);
  cudaFree(s->d_gmm); cudaFree(s->d_desc); cudaFree(s->d_state); cudaFree(s->d_glob); cudaFree(s->d_active);
  cudaFree(s->d_new);
  cudaFreeHost(s->h_desc); cudaFreeHost(s->h_state); cudaFreeHost(s->h_glob); cudaFreeHost(s->h_active);
  cudaFreeHost(s->h_new); cudaFreeHost(s->h_gmm);
  if (s->stream) cudaStreamDestroy(s->stream);
}

size_t slot_bytes(const prrtc_params& p) {
  return (size_t)2 * p.tree_capacity * (kMaxDof * 4 + 8) + (size_t)p.path_capacity * (kMaxDof * 4 + 4) +
         (size_t)kEnvSnapF4 * 16 + kGmmStride * 4 + sizeof(ProblemDesc) + sizeof(ProblemState);
}

int status_of(const ProblemState& S) {
  if (S.pre_status) return S.pre_status;
  if (S.solved)
    return (S.path_status == PRRTC_SOLVED || S.path_status == PRRTC_PATH_OVERFLOW) ? S.path_status : PRRTC_ERR_TIMEOUT;
  if (S.timed_out) return PRRTC_TIME_LIMIT;
  return PRRTC_NO_SOLUTION;
}

// One round of the server loop; returns false when idle.
bool server_round(prrtc_server* s) {
  std::vector<Query*> fresh;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    int active = 0;
    for (Query* q : s->slot_query) active += q != nullptr;
    if (active == 0 && s->pending.empty()) {
      s->cv.wait_for(lk, std::chrono::milliseconds(1));
      return false;
    }
    while (!s->pending.empty() && !s->free_slots.empty()) {
      Query* q = s->pending.front();
      s->pending.pop_front();
      q->slot = s->free_slots.back();
      s->free_slots.pop_back();
      q->t_admit = now_s();
      s->slot_query[q->slot] = q;
      fresh.push_back(q);
      s->admitted++;
    }
  }
  const double t0 = now_s();
  const cudaStream_t st = s->stream;
  const prrtc_params& prm = s->params;
  const size_t tree_stride = (size_t)prm.tree_capacity * kMaxDof;
  // --- set up freshly admitted queries
  std::map<prrtc_proposal*, std::vector<Query*>> learned;
  for (size_t k = 0; k < fresh.size(); ++k) {
    Query* q = fresh[k];
    const int p = q->slot;
    const RobotDev* rdev = nullptr;
    const RobotHeader* H = nullptr;
    int dev = -1;
    prrtc_internal_robot_view(q->robot, &rdev, &H, &dev);
    ProblemDesc& D = s->h_desc[p];
    std::memset(&D, 0, sizeof(D));
    EnvView view{};
    if (prrtc_internal_env_snapshot(q->env, s->env_snap + (size_t)p * kEnvSnapF4, kEnvSnapF4, &view, st)) {
      s->error = PRRTC_ERR_UNSUPPORTED;
      return true;
    }
    D.robot = rdev;
    D.env = view;
    D.nodes[0] = s->nodes + ((size_t)p * 2 + 0) * tree_stride;
    D.nodes[1] = s->nodes + ((size_t)p * 2 + 1) * tree_stride;
    D.parent[0] = s->parents + ((size_t)p * 2 + 0) * prm.tree_capacity;
    D.parent[1] = s->parents + ((size_t)p * 2 + 1) * prm.tree_capacity;
    float* radii = reinterpret_cast<float*>(s->parents + (size_t)s->slots * 2 * prm.tree_capacity);
    D.radius[0] = radii + ((size_t)p * 2 + 0) * prm.tree_capacity;
    D.radius[1] = radii + ((size_t)p * 2 + 1) * prm.tree_capacity;
    D.path = s->paths + (size_t)p * prm.path_capacity * kMaxDof;
    D.path_idx = s->path_idx + (size_t)p * prm.path_capacity;
    D.cap = prm.tree_capacity;
    D.dpad = H->dpad;
    D.dof = H->dof;
    D.n_spheres = H->n_spheres;
    D.n_pairs = H->n_pairs;
    D.key_lo = (uint32_t)(q->seed & 0xffffffffu);
    D.key_hi = (uint32_t)(q->seed >> 32);
    D.pid = q->pid;
    for (int j = 0; j < H->dof; ++j) {
      D.q_start[j] = q->qs[j];
      D.q_goal[j] = q->qg[j];
    }
    float* grow = s->d_gmm + (size_t)p * kGmmStride;
    if (q->proposal) {
      learned[q->proposal].push_back(q);
      D.gmm = grow;
    } else if (!q->gmm.empty()) {
      float* g = s->h_gmm + (size_t)p * kGmmStride;
      std::memset(g, 0, kGmmStride * sizeof(float));
      const int d = H->dof;
      for (int c = 0; c < kMixK; ++c) {
        g[c] = q->gmm[c];
        for (int j = 0; j < d; ++j) {
          g[kMixK + c * kMaxDof + j] = q->gmm[kMixK + c * d + j];
          g[kMixK + kMixK * kMaxDof + c * kMaxDof + j] = std::min(std::max(q->gmm[kMixK + kMixK * d + c * d + j], -5.f), 2.f);
        }
      }
      cudaMemcpyAsync(grow, g, kGmmStride * sizeof(float), cudaMemcpyHostToDevice, st);
      D.gmm = grow;
    }
    cudaMemcpyAsync(s->d_desc + p, &D, sizeof(D), cudaMemcpyHostToDevice, st);
    s->h_new[k] = p;
  }
  for (auto& kv : learned) {
    std::vector<EnvView> envs;
    std::vector<float> qs, qg;
    std::vector<float*> rows;
    for (Query* q : kv.second) {
      envs.push_back(s->h_desc[q->slot].env);
      qs.insert(qs.end(), q->qs.begin(), q->qs.end());
      qg.insert(qg.end(), q->qg.begin(), q->qg.end());
      rows.push_back(s->d_gmm + (size_t)q->slot * kGmmStride);
    }
    if (prrtc_internal_proposal_mixtures(kv.first, envs.data(), qs.data(), qg.data(), (int)envs.size(), rows.data(),
                                         st)) {
      s->error = PRRTC_ERR_CUDA;
      return true;
    }
  }
  int max_spheres = 1, max_pairs = 0, max_env = 0;
  int n_active = 0;
  for (int p = 0; p < s->slots; ++p) {
    if (!s->slot_query[p]) continue;
    s->h_active[n_active++] = p;
    const ProblemDesc& D = s->h_desc[p];
    max_spheres = std::max(max_spheres, D.n_spheres + D.dof);  // staging slots: spheres + group centres
    max_pairs = std::max(max_pairs, D.n_pairs);
    max_env = std::max(max_env, D.env.n_float4());
  }
  if (!fresh.empty()) {
    cudaMemcpyAsync(s->d_new, s->h_new, fresh.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    launch_setup(s->d_desc, s->d_state, (int)fresh.size(), max_spheres, max_pairs, max_env, st, s->d_new);
  }
  // --- one time slice over every occupied slot
  PlanGlobals& G = *s->h_glob;
  std::memset(&G, 0, sizeof(G));
  G.n_problems = n_active;
  globals_from_params(G, prm);
  G.t0 = ULLONG_MAX;
  G.active = s->d_active;
  G.slice_ns = (unsigned long long)s->slice_us * 1000ull;
  const PlanLaunch cfg = plan_launch_config(n_active, prm.mode, prm.blocks, prm.warps_per_block, max_spheres,
                                            max_pairs, max_env, s->sms);
  // rotate the work order every slice so that no query starves when more
  // slots are occupied than blocks are resident
  if (n_active > 1) {
    const int r = (int)(((int64_t)s->slices * cfg.grid) % n_active);
    std::rotate(s->h_active, s->h_active + r, s->h_active + n_active);
  }
  cudaMemcpyAsync(s->d_active, s->h_active, n_active * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s->d_glob, s->h_glob, sizeof(PlanGlobals), cudaMemcpyHostToDevice, st);
  launch_plan(s->d_glob, s->d_desc, s->d_state, cfg, G.obstacle_tile, false, st);
  launch_record_usage(s->d_desc, s->d_state, n_active, st, s->d_active);
  cudaMemcpyAsync(s->h_state, s->d_state, (size_t)s->slots * sizeof(ProblemState), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(s->h_glob, s->d_glob, sizeof(PlanGlobals), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || s->h_glob->error) {
    s->error = e != cudaSuccess ? PRRTC_ERR_CUDA : s->h_glob->error;
    return true;
  }
  s->slices++;
  // --- harvest
  std::vector<Done> out;
  std::vector<int> freed;
  for (int k = 0; k < n_active; ++k) {
    const int p = s->h_active[k];
    Query* q = s->slot_query[p];
    q->slices++;
    const ProblemState& S = s->h_state[p];
    const bool finished = S.pre_status || S.solved || S.done || S.iter >= prm.max_iters;
    if (!finished) continue;
    Done d{};
    d.ticket = q->ticket;
    prrtc_path& P = d.path;
    std::memset(&P, 0, sizeof(P));
    const int dof = s->h_desc[p].dof;
    P.status = status_of(S);
    P.dof = dof;
    P.iterations = reported_iterations(S, prm);
    P.nodes_a = std::min(S.count[0], prm.tree_capacity);
    P.nodes_b = std::min(S.count[1], prm.tree_capacity);
    P.edges_checked = (int64_t)S.edges;
    P.edge_states = (int64_t)S.edge_states;
    P.sphere_tests = (int64_t)S.sphere_tests;
    P.pair_tests = (int64_t)S.pair_tests;
    P.fk_states = (int64_t)S.fk_states;
    P.nn_nodes = (int64_t)S.nn_nodes;
    P.dd_rejected = (int64_t)S.dd_rejected;
    P.verdict_states = (int64_t)S.verdict_states;
    for (int k = 0; k < 4; ++k) P.prim_tests[k] = (int64_t)S.prim_tests[k];
    P.cost = S.cost;
    P.solve_time_us = -1.0;
    if (P.status == PRRTC_SOLVED || P.status == PRRTC_PATH_OVERFLOW) P.n = S.path_n;
    if (P.status == PRRTC_SOLVED && S.path_n > 0) {
      P.q = (float*)std::malloc((size_t)S.path_n * dof * sizeof(float));
      if (P.q)
        cudaMemcpy(P.q, s->h_desc[p].path, (size_t)S.path_n * dof * sizeof(float), cudaMemcpyDeviceToHost);
    }
    const double t = now_s();
    d.latency_ms = (t - q->t_submit) * 1e3;
    d.queue_ms = (q->t_admit - q->t_submit) * 1e3;
    d.slices = q->slices;
    out.push_back(d);
    freed.push_back(p);
  }
  s->busy_s += now_s() - t0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int p : freed) {
      delete s->slot_query[p];
      s->slot_query[p] = nullptr;
      s->free_slots.push_back(p);
    }
    for (auto& d : out) s->done.push_back(d);
    s->completed += (int64_t)out.size();
  }
  s->cv.notify_all();
  return true;
}

void server_main(prrtc_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    server_round(s);
    if (s->error) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->cv.notify_all();
      break;
    }
  }
}

}  // namespace

extern "C" {

void prrtc_server_config_default(prrtc_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->max_slots = 0;
  c->memory_budget_bytes = (int64_t)2 << 30;
  c->slice_us = 500;
  prrtc_params_default(&c->params);
  c->params.tree_capacity = 1 << 13;
  c->params.path_capacity = 1 << 12;
}

int prrtc_server_create(const prrtc_server_config* cfg, prrtc_server** out) {
  if (!cfg || !out) return PRRTC_ERR_INVALID_ARG;
  *out = nullptr;
  const prrtc_params& p = cfg->params;
  if (!(p.range > 0.f) || !(p.resolution > 0.f) || p.max_iters < 1 || p.tree_capacity < 2 || p.path_capacity < 2 ||
      cfg->slice_us < 10 || cfg->memory_budget_bytes <= 0 || cfg->max_slots < 0 ||
      !(p.learned_ratio >= 0.f && p.learned_ratio <= 1.f) || !(p.goal_bias >= 0.f && p.goal_bias <= 1.f) ||
      (p.mode != PRRTC_MODE_ASYNC && p.mode != PRRTC_MODE_SERIAL) || (double)p.range / p.resolution > 4096.0 ||
      sampling_params_problem(p)) {
    prrtc_internal_set_error("invalid server configuration");
    return PRRTC_ERR_INVALID_ARG;
  }
  int dev = -1, count = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
    return PRRTC_ERR_NO_DEVICE;
  prrtc_server* s = new prrtc_server();
  s->device = dev;
  s->params = p;
  s->slice_us = cfg->slice_us;
  const size_t per = slot_bytes(p);
  int slots = (int)std::min<int64_t>(cfg->memory_budget_bytes / (int64_t)per, 1 << 16);
  if (cfg->max_slots > 0) slots = std::min(slots, cfg->max_slots);
  if (slots < 1) {
    delete s;
    prrtc_internal_set_error("memory budget below one query slot");
    return PRRTC_ERR_INVALID_ARG;
  }
  s->slots = slots;
  const size_t rows = (size_t)slots * 2 * p.tree_capacity;
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&s->nodes, rows * kMaxDof * 4) == cudaSuccess && cudaMalloc(&s->parents, 2 * rows * 4) == cudaSuccess &&
            cudaMalloc(&s->paths, (size_t)slots * p.path_capacity * kMaxDof * 4) == cudaSuccess &&
            cudaMalloc(&s->path_idx, (size_t)slots * p.path_capacity * 4) == cudaSuccess &&
            cudaMalloc(&s->env_snap, (size_t)slots * kEnvSnapF4 * 16) == cudaSuccess &&
            cudaMalloc(&s->d_gmm, (size_t)slots * kGmmStride * 4) == cudaSuccess &&
            cudaMalloc(&s->d_desc, (size_t)slots * sizeof(ProblemDesc)) == cudaSuccess &&
            cudaMalloc(&s->d_state, (size_t)slots * sizeof(ProblemState)) == cudaSuccess &&
            cudaMalloc(&s->d_glob, sizeof(PlanGlobals)) == cudaSuccess &&
            cudaMalloc(&s->d_active, (size_t)slots * 4) == cudaSuccess &&
            cudaMalloc(&s->d_new, (size_t)slots * 4) == cudaSuccess &&
            cudaMallocHost(&s->h_desc, (size_t)slots * sizeof(ProblemDesc)) == cudaSuccess &&
            cudaMallocHost(&s->h_state, (size_t)slots * sizeof(ProblemState)) == cudaSuccess &&
            cudaMallocHost(&s->h_glob, sizeof(PlanGlobals)) == cudaSuccess &&
            cudaMallocHost(&s->h_active, (size_t)slots * 4) == cudaSuccess &&
            cudaMallocHost(&s->h_new, (size_t)slots * 4) == cudaSuccess &&
            cudaMallocHost(&s->h_gmm, (size_t)slots * kGmmStride * 4) == cudaSuccess;
  if (ok)
    ok = cudaMemsetAsync(s->nodes, 0xFF, rows * kMaxDof * 4, s->stream) == cudaSuccess &&
         cudaMemsetAsync(s->parents, 0xFF, 2 * rows * 4, s->stream) == cudaSuccess &&  // parents, NaN radii
         cudaMemsetAsync(s->d_state, 0, (size_t)slots * sizeof(ProblemState), s->stream) == cudaSuccess &&
         cudaStreamSynchronize(s->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_server(s);
    delete s;
    prrtc_internal_set_error("server allocation failed");
    return PRRTC_ERR_OOM;
  }
  s->slot_query.assign(slots, nullptr);
  for (int k = slots - 1; k >= 0; --k) s->free_slots.push_back(k);
  s->t_start = now_s();
  s->thread = std::thread(server_main, s);
  *out = s;
  return PRRTC_OK;
}

int prrtc_server_submit(prrtc_server* s, const prrtc_problem* pb, prrtc_proposal* proposal, uint64_t* ticket) {
  if (!s || !pb || !pb->robot || !pb->env || !pb->q_start || !pb->q_goal) return PRRTC_ERR_INVALID_ARG;
  if (s->error) return s->error;
  const RobotDev* rdev = nullptr;
  const RobotHeader* H = nullptr;
  int dev = -1;
  prrtc_internal_robot_view(pb->robot, &rdev, &H, &dev);
  if (dev != s->device) return PRRTC_ERR_INVALID_ARG;
  Query* q = new Query();
  q->robot = pb->robot;
  q->env = const_cast<prrtc_env*>(pb->env);
  q->proposal = proposal;
  q->qs.assign(pb->q_start, pb->q_start + H->dof);
  q->qg.assign(pb->q_goal, pb->q_goal + H->dof);
  for (int j = 0; j < H->dof; ++j)
    if (!std::isfinite(q->qs[j]) || !std::isfinite(q->qg[j])) {
      delete q;
      return PRRTC_ERR_INVALID_ARG;
    }
  if (pb->gmm) q->gmm.assign(pb->gmm, pb->gmm + kMixK * (1 + 2 * H->dof));
  q->seed = pb->seed;
  q->pid = pb->problem_id;
  q->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    s->pending.push_back(q);
    s->submitted++;
  }
  s->cv.notify_all();
  if (ticket) *ticket = q->ticket;
  return PRRTC_OK;
}

int prrtc_server_poll(prrtc_server* s, int32_t max, prrtc_path* paths, uint64_t* tickets, double* latency_ms,
                      double* queue_ms, int32_t* n_out) {
  if (!s || !n_out || max < 0) return PRRTC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  while (n < max && !s->done.empty()) {
    Done& d = s->done.front();
    if (paths) paths[n] = d.path;
    else std::free(d.path.q);
    if (tickets) tickets[n] = d.ticket;
    if (latency_ms) latency_ms[n] = d.latency_ms;
    if (queue_ms) queue_ms[n] = d.queue_ms;
    s->done.pop_front();
    ++n;
  }
  *n_out = n;
  return s->error;
}

int prrtc_server_wait(prrtc_server* s, int64_t completed_at_least, double timeout_s) {
  if (!s) return PRRTC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                 [&] { return s->completed >= completed_at_least || s->error; });
  if (s->error) return s->error;
  return ok ? PRRTC_OK : PRRTC_ERR_TIMEOUT;
}

int prrtc_server_get_stats(prrtc_server* s, prrtc_server_stats* out) {
  if (!s || !out) return PRRTC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->slots = s->slots;
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->slices = s->slices;
  out->pending = (int64_t)s->pending.size();
  int active = 0;
  for (Query* q : s->slot_query) active += q != nullptr;
  out->active = active;
  out->busy_s = s->busy_s;
  out->uptime_s = now_s() - s->t_start;
  return s->error;
}

void prrtc_server_destroy(prrtc_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  for (Query* q : s->slot_query) delete q;
  for (Query* q : s->pending) delete q;
  for (auto& d : s->done) std::free(d.path.q);
  free_server(s);
  delete s;
}

}  // extern "C"
