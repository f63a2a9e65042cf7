// prrtc_api.cu -- host runtime of libprrtc: handles, device arenas, launch
// sequencing and the extern "C" entry points declared in include/prrtc.h.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "prrtc.h"
#include "prrtc_launch.h"

using namespace prrtc;

// ------------------------------------------------------------------ errors
static thread_local std::string t_last_error;

static int fail(int code, const std::string& msg) {
  t_last_error = msg;
  return code;
}

static int cuda_fail(const char* what, cudaError_t e) {
  t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return PRRTC_ERR_CUDA;
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(#call, e_); \
  } while (0)

// ------------------------------------------------------------------ handles
struct prrtc_env {
  std::mutex mu;            // guards h_data against concurrent updates and snapshots
  int device = -1;
  float4* d_data = nullptr;
  std::vector<float4> h_data;
  int n_aabb = 0, n_obb = 0, n_cyl = 0, n_sph = 0;
  std::vector<int> kind;    // per obstacle id: 0 aabb, 1 obb, 2 cylinder, 3 sphere
  std::vector<int> offset;  // per obstacle id: first float4 in the blob
  // optional distance field
  float* d_esdf = nullptr;
  uint8_t* d_occ = nullptr;
  int2* d_tmp = nullptr;    // 2 x voxels, scratch of the transform
  int dims[3] = {0, 0, 0};
  float origin[3] = {0.f, 0.f, 0.f};
  float voxel = 0.f;
  size_t voxels() const { return (size_t)dims[0] * dims[1] * dims[2]; }
  EnvView view() const {
    EnvView v;
    v.data = d_data;
    v.n_aabb = n_aabb;
    v.n_obb = n_obb;
    v.n_cyl = n_cyl;
    v.n_sph = n_sph;
    v.esdf = EsdfGrid{d_esdf, origin[0], origin[1], origin[2], d_esdf ? 1.f / voxel : 0.f, dims[0], dims[1], dims[2],
                      0};
    return v;
  }
};

struct prrtc_robot {
  int device = -1;
  RobotDev* d = nullptr;
  RobotDev* h = nullptr;
};

// ------------------------------------------------------------------ per-device context
namespace {

struct DeviceCtx {
  bool ready = false;
  int device = -1;
  int sms = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  // planner arenas
  int slots = 0, cap = 0, path_cap = 0;
  float* nodes = nullptr;
  int* parents = nullptr;
  float* paths = nullptr;
  int* path_idx = nullptr;
  ProblemDesc* d_desc = nullptr;
  ProblemState* d_state = nullptr;
  PlanGlobals* d_glob = nullptr;
  ProblemDesc* h_desc = nullptr;
  ProblemState* h_state = nullptr;
  PlanGlobals* h_glob = nullptr;
  int* d_offsets = nullptr;
  int* h_offsets = nullptr;
  float* d_packed = nullptr;
  float* h_packed = nullptr;
  size_t packed_cap = 0;
  float* d_held = nullptr;  // lockstep mode: rows each worker of a round holds back
  size_t held_cap = 0;
  int* d_held_meta = nullptr;
  size_t held_meta_cap = 0;
  float* d_gmm = nullptr;   // [slots][kGmmStride] learned mixtures
  float* h_gmm = nullptr;
  size_t gmm_cap = 0;
  // CUDA graph of the launch sequence, keyed by everything it bakes in
  struct GraphKey {
    int n, grid, warps, smem, robot_bytes, env_bytes, stage_bytes, max_spheres, max_pairs, max_env, gen, head,
        lockstep, tile, batch_head, lean;
    bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
  };
  GraphKey gkey{};
  cudaGraphExec_t gexec = nullptr;
  int arena_gen = 0;
  float* h_path_head = nullptr;  // first kHeadRows path rows of a single-problem call
  float* d_heads = nullptr;      // first kBatchHeadRows path rows of each problem of a batch
  float* h_heads = nullptr;
  size_t heads_cap = 0;
  // autotuned (blocks, warps) per (row width, obstacle bucket, batch-size bucket, mode)
  struct Tuned {
    int blocks, warps, tile, expansions;
  };
  std::map<uint64_t, Tuned> tuned;
  // check_states scratch
  float* d_q = nullptr;
  uint8_t* d_valid = nullptr;
  float* d_spheres = nullptr;
  size_t q_cap = 0, valid_cap = 0, spheres_cap = 0;
  unsigned long long* d_counters = nullptr;
  int* d_error = nullptr;
  cudaEvent_t ev[4] = {};
  prrtc_launch_stats last{};
};

constexpr int kHeadRows = 512;
constexpr int kBatchHeadRows = 32;

DeviceCtx g_ctx[64];
std::mutex g_init_mu;

int current_ctx(DeviceCtx** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  int count = 0;
  if (e != cudaSuccess || cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
    return fail(PRRTC_ERR_NO_DEVICE, "no CUDA device available");
  if (dev < 0 || dev >= 64) return fail(PRRTC_ERR_NO_DEVICE, "device index out of range");
  DeviceCtx* c = &g_ctx[dev];
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (!c->ready) {
    c->device = dev;
    CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    for (auto& ev : c->ev) CK(cudaEventCreate(&ev));
    CK(cudaMalloc(&c->d_counters, 8 * sizeof(unsigned long long)));
    CK(cudaMalloc(&c->d_error, sizeof(int)));
    CK(cudaMallocHost(&c->h_glob, sizeof(PlanGlobals)));
    CK(cudaMalloc(&c->d_glob, sizeof(PlanGlobals)));
    CK(cudaMallocHost(&c->h_path_head, (size_t)kHeadRows * kMaxDof * sizeof(float)));
    c->ready = true;
  }
  *out = c;
  return PRRTC_OK;
}

template <class T>
int grow_device(T** p, size_t* cap, size_t need) {
  if (*cap >= need && *p) return PRRTC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  size_t n = std::max<size_t>(need, 1);
  if (cudaMalloc(p, n * sizeof(T)) != cudaSuccess) return fail(PRRTC_ERR_OOM, "device allocation failed");
  *cap = n;
  return PRRTC_OK;
}

void free_arenas(DeviceCtx* c) {
  cudaFree(c->nodes);
  cudaFree(c->parents);
  cudaFree(c->paths);
  cudaFree(c->path_idx);
  cudaFree(c->d_desc);
  cudaFree(c->d_state);
  cudaFree(c->d_offsets);
  cudaFreeHost(c->h_desc);
  cudaFreeHost(c->h_state);
  cudaFreeHost(c->h_offsets);
  c->nodes = nullptr;
  c->parents = nullptr;
  c->paths = nullptr;
  c->path_idx = nullptr;
  c->d_desc = nullptr;
  c->d_state = nullptr;
  c->d_offsets = nullptr;
  c->h_desc = nullptr;
  c->h_state = nullptr;
  c->h_offsets = nullptr;
  c->slots = c->cap = c->path_cap = 0;
}

// Tree arenas: slot p, tree t occupies cap rows of kMaxDof floats (the row
// stride used is the problem's dpad, so any DoF fits), cap parent indices and
// cap dynamic-domain radii (the radii follow all parent arrays).
int ensure_arenas(DeviceCtx* c, int slots, int cap, int path_cap) {
  if (c->slots >= slots && c->cap >= cap && c->path_cap >= path_cap) return PRRTC_OK;
  CK(cudaStreamSynchronize(c->stream));
  slots = std::max(slots, c->slots);
  cap = std::max(cap, c->cap);
  path_cap = std::max(path_cap, c->path_cap);
  free_arenas(c);
  const size_t rows = (size_t)slots * 2 * cap;
  bool ok = cudaMalloc(&c->nodes, rows * kMaxDof * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->parents, 2 * rows * sizeof(int)) == cudaSuccess &&   // parents, then radii
            cudaMalloc(&c->paths, (size_t)slots * path_cap * kMaxDof * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->path_idx, (size_t)slots * path_cap * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->d_desc, (size_t)slots * sizeof(ProblemDesc)) == cudaSuccess &&
            cudaMalloc(&c->d_state, (size_t)slots * sizeof(ProblemState)) == cudaSuccess &&
            cudaMalloc(&c->d_offsets, (size_t)(slots + 1) * sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&c->h_desc, (size_t)slots * sizeof(ProblemDesc)) == cudaSuccess &&
            cudaMallocHost(&c->h_state, (size_t)slots * sizeof(ProblemState)) == cudaSuccess &&
            cudaMallocHost(&c->h_offsets, (size_t)(slots + 1) * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_arenas(c);
    return fail(PRRTC_ERR_OOM, "planner arena allocation failed");
  }
  CK(cudaMemsetAsync(c->nodes, 0xFF, rows * kMaxDof * sizeof(float), c->stream));   // NaN rows
  CK(cudaMemsetAsync(c->parents, 0xFF, 2 * rows * sizeof(int), c->stream));         // unset parents, NaN radii
  CK(cudaMemsetAsync(c->d_state, 0, (size_t)slots * sizeof(ProblemState), c->stream));
  c->slots = slots;
  c->cap = cap;
  c->path_cap = path_cap;
  c->arena_gen++;
  return PRRTC_OK;
}

uint64_t tune_key(int dpad, int env_f4, int n, int mode) {
  int nb = 0;
  while ((1 << nb) < n) ++nb;
  return ((uint64_t)dpad << 48) | ((uint64_t)((env_f4 + 63) / 64) << 32) | ((uint64_t)nb << 8) | (uint64_t)mode;
}

bool finite_all(const float* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

int validate_params(const prrtc_params* p) {
  if (!p) return fail(PRRTC_ERR_INVALID_ARG, "params is null");
  if (!(p->range > 0.f) || !std::isfinite(p->range)) return fail(PRRTC_ERR_INVALID_ARG, "range must be > 0");
  if (!(p->resolution > 0.f) || !std::isfinite(p->resolution))
    return fail(PRRTC_ERR_INVALID_ARG, "resolution must be > 0");
  if (!(p->goal_bias >= 0.f && p->goal_bias <= 1.f)) return fail(PRRTC_ERR_INVALID_ARG, "goal_bias must be in [0,1]");
  if (p->max_iters < 1) return fail(PRRTC_ERR_INVALID_ARG, "max_iters must be >= 1");
  if (p->tree_capacity < 2) return fail(PRRTC_ERR_INVALID_ARG, "tree_capacity must be >= 2");
  if (p->tree_capacity > (1 << 26)) return fail(PRRTC_ERR_INVALID_ARG, "tree_capacity too large");
  if (p->path_capacity < 2) return fail(PRRTC_ERR_INVALID_ARG, "path_capacity must be >= 2");
  if (p->mode != PRRTC_MODE_ASYNC && p->mode != PRRTC_MODE_SERIAL && p->mode != PRRTC_MODE_LOCKSTEP)
    return fail(PRRTC_ERR_INVALID_ARG, "unknown mode");
  if (p->mode == PRRTC_MODE_LOCKSTEP && (p->workers < 1 || p->workers > 1024))
    return fail(PRRTC_ERR_INVALID_ARG, "lockstep workers must be in 1..1024");
  if (p->expansions < 0 || p->expansions > 64) return fail(PRRTC_ERR_INVALID_ARG, "expansions must be in 0..64");
  if (p->obstacle_tile != 0 && p->obstacle_tile != 32 && p->obstacle_tile != 64)
    return fail(PRRTC_ERR_INVALID_ARG, "obstacle_tile must be 0, 32 or 64");
  if (p->blocks < 0 || p->warps_per_block < 0 || p->warps_per_block > 16)
    return fail(PRRTC_ERR_INVALID_ARG, "blocks / warps_per_block out of range");
  if (p->time_limit_s < 0.0) return fail(PRRTC_ERR_INVALID_ARG, "time_limit_s must be >= 0");
  if (!(p->learned_ratio >= 0.f && p->learned_ratio <= 1.f))
    return fail(PRRTC_ERR_INVALID_ARG, "learned_ratio must be in [0,1]");
  const double ratio = (double)p->range / (double)p->resolution;
  if (ratio > 4096.0) return fail(PRRTC_ERR_INVALID_ARG, "range / resolution too large");
  if (const char* why = sampling_params_problem(*p)) return fail(PRRTC_ERR_INVALID_ARG, why);
  return PRRTC_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* prrtc_version(void) { return "prrtc-gb300 0.1 (sm_103a)"; }

const char* prrtc_last_error(void) { return t_last_error.c_str(); }

const char* prrtc_status_string(int code) {
  switch (code) {
    case PRRTC_OK: return "ok / solved";
    case PRRTC_ERR_INVALID_ARG: return "invalid argument";
    case PRRTC_ERR_OOM: return "out of memory";
    case PRRTC_ERR_CUDA: return "CUDA error";
    case PRRTC_ERR_TIMEOUT: return "device wait timed out";
    case PRRTC_ERR_DEVICE_INDEX: return "device bounds check failed";
    case PRRTC_ERR_NO_DEVICE: return "no CUDA device";
    case PRRTC_ERR_UNSUPPORTED: return "unsupported (exceeds compiled limits)";
    case PRRTC_START_IN_COLLISION: return "start in collision";
    case PRRTC_GOAL_IN_COLLISION: return "goal in collision";
    case PRRTC_NO_SOLUTION: return "no solution within the iteration budget";
    case PRRTC_PATH_OVERFLOW: return "path longer than path_capacity";
    case PRRTC_TIME_LIMIT: return "time limit reached";
    default: return "unknown status";
  }
}

void prrtc_params_default(prrtc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->range = 1.0f;
  p->resolution = 1.0f / 32.0f;
  p->goal_bias = 0.05f;
  p->max_iters = 50000;
  p->tree_capacity = 1 << 16;
  p->path_capacity = 1 << 14;
  p->mode = PRRTC_MODE_ASYNC;
  p->blocks = 0;
  p->warps_per_block = 0;
  p->seed = 1;
  p->time_limit_s = 0.0;
}

void prrtc_path_free(prrtc_path* path) {
  if (!path) return;
  std::free(path->q);
  path->q = nullptr;
  path->n = 0;
}

void prrtc_paths_free(prrtc_path* paths, int32_t n) {
  if (!paths) return;
  for (int32_t k = 0; k < n; ++k) prrtc_path_free(paths + k);
}

int prrtc_last_launch_stats(prrtc_launch_stats* out) {
  if (!out) return fail(PRRTC_ERR_INVALID_ARG, "out is null");
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->last;
  return PRRTC_OK;
}

// -------------------------------------------------------------- environment
static int pack_obstacle(const prrtc_obstacle& o, int* kind, float4* out) {
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(o.center[k]) || !std::isfinite(o.half[k]) || !std::isfinite(o.axis[k])) return -1;
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(o.rot[k])) return -1;
  const float* c = o.center;
  if (o.type == PRRTC_OBS_BOX) {
    if (!(o.half[0] > 0.f && o.half[1] > 0.f && o.half[2] > 0.f)) return -1;
    bool identity = true;
    for (int i = 0; i < 9; ++i) identity &= (o.rot[i] == ((i % 4 == 0) ? 1.f : 0.f));
    out[0] = make_float4(c[0], c[1], c[2], 0.f);
    out[1] = make_float4(o.half[0], o.half[1], o.half[2], 0.f);
    if (identity) {
      *kind = 0;
      return 2;
    }
    // rows of R^T (columns of R): local_k = <column k of R, p - c>
    for (int k = 0; k < 3; ++k) out[2 + k] = make_float4(o.rot[0 * 3 + k], o.rot[1 * 3 + k], o.rot[2 * 3 + k], 0.f);
    *kind = 1;
    return 5;
  }
  if (o.type == PRRTC_OBS_CYLINDER) {
    const double n = std::sqrt((double)o.axis[0] * o.axis[0] + (double)o.axis[1] * o.axis[1] +
                               (double)o.axis[2] * o.axis[2]);
    if (!(o.half[0] > 0.f && o.half[1] > 0.f) || std::fabs(n - 1.0) > 1e-3) return -1;
    out[0] = make_float4(c[0], c[1], c[2], o.half[0]);
    out[1] = make_float4(o.axis[0], o.axis[1], o.axis[2], o.half[1]);
    *kind = 2;
    return 2;
  }
  if (o.type == PRRTC_OBS_SPHERE) {
    if (!(o.half[0] > 0.f)) return -1;
    out[0] = make_float4(c[0], c[1], c[2], o.half[0]);
    *kind = 3;
    return 1;
  }
  return -1;
}

int prrtc_env_create(const prrtc_obstacle* obstacles, int32_t n, prrtc_env** out) {
  if (!out) return fail(PRRTC_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (n < 0 || n > PRRTC_MAX_OBSTACLES || (n > 0 && !obstacles))
    return fail(PRRTC_ERR_INVALID_ARG, "bad obstacle count or null obstacles");
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  std::vector<int> kinds(n);
  std::vector<std::vector<float4>> packed(n);
  int cnt[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    float4 tmp[5];
    int kind = 0;
    const int m = pack_obstacle(obstacles[i], &kind, tmp);
    if (m < 0) return fail(PRRTC_ERR_INVALID_ARG, "invalid obstacle " + std::to_string(i));
    kinds[i] = kind;
    packed[i].assign(tmp, tmp + m);
    cnt[kind]++;
  }
  prrtc_env* e = new prrtc_env();
  e->device = c->device;
  e->n_aabb = cnt[0];
  e->n_obb = cnt[1];
  e->n_cyl = cnt[2];
  e->n_sph = cnt[3];
  const int width[4] = {2, 5, 2, 1};
  int base[4];
  base[0] = 0;
  for (int k = 1; k < 4; ++k) base[k] = base[k - 1] + cnt[k - 1] * width[k - 1];
  const int total = base[3] + cnt[3] * width[3];
  e->h_data.assign(std::max(total, 1), make_float4(0.f, 0.f, 0.f, 0.f));
  e->kind.resize(n);
  e->offset.resize(n);
  int fill[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const int k = kinds[i];
    const int off = base[k] + fill[k] * width[k];
    fill[k]++;
    e->kind[i] = k;
    e->offset[i] = off;
    std::copy(packed[i].begin(), packed[i].end(), e->h_data.begin() + off);
  }
  if (cudaMalloc(&e->d_data, e->h_data.size() * sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    delete e;
    return fail(PRRTC_ERR_OOM, "env allocation failed");
  }
  cudaError_t ce = cudaMemcpy(e->d_data, e->h_data.data(), e->h_data.size() * sizeof(float4), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaFree(e->d_data);
    delete e;
    return cuda_fail("env upload", ce);
  }
  *out = e;
  return PRRTC_OK;
}

int prrtc_env_update(prrtc_env* env, const int32_t* ids, const prrtc_obstacle* obstacles, int32_t n) {
  if (!env || n < 0 || (n > 0 && (!ids || !obstacles))) return fail(PRRTC_ERR_INVALID_ARG, "bad env update");
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  if (c->device != env->device) return fail(PRRTC_ERR_INVALID_ARG, "env belongs to another device");
  std::lock_guard<std::mutex> lk(c->mu);
  std::lock_guard<std::mutex> lk_env(env->mu);
  int lo = INT_MAX, hi = -1;
  for (int k = 0; k < n; ++k) {
    const int id = ids[k];
    if (id < 0 || id >= (int)env->kind.size()) return fail(PRRTC_ERR_INVALID_ARG, "obstacle id out of range");
    float4 tmp[5];
    int kind = 0;
    const int m = pack_obstacle(obstacles[k], &kind, tmp);
    if (m < 0 || kind != env->kind[id]) return fail(PRRTC_ERR_INVALID_ARG, "update changes an obstacle's kind");
    std::copy(tmp, tmp + m, env->h_data.begin() + env->offset[id]);
    lo = std::min(lo, env->offset[id]);
    hi = std::max(hi, env->offset[id] + m);
  }
  if (hi < 0) return PRRTC_OK;
  // Stream-ordered upload: lands between the planning launches around it.
  CK(cudaMemcpyAsync(env->d_data + lo, env->h_data.data() + lo, (size_t)(hi - lo) * sizeof(float4),
                     cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PRRTC_OK;
}

// Consistent copy of an environment's current obstacle blob into device
// memory `dst` (at most max_f4 float4) on `stream`; *view describes the copy.
// The host mirror is read under the env's lock before this returns.
int prrtc_internal_env_snapshot(prrtc_env* env, float4* dst, int max_f4, EnvView* view, cudaStream_t stream) {
  if (!env || !dst || !view) return PRRTC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(env->mu);
  const int n = env->view().n_float4();
  if (n > max_f4) return PRRTC_ERR_UNSUPPORTED;
  if (n > 0) CK(cudaMemcpyAsync(dst, env->h_data.data(), (size_t)n * sizeof(float4), cudaMemcpyHostToDevice, stream));
  *view = env->view();
  view->data = dst;
  return PRRTC_OK;
}

void prrtc_env_destroy(prrtc_env* env) {
  if (!env) return;
  cudaFree(env->d_data);
  cudaFree(env->d_esdf);
  cudaFree(env->d_occ);
  cudaFree(env->d_tmp);
  delete env;
}

// -------------------------------------------------------------- distance fields
static int check_grid(const float origin[3], float voxel, const int32_t dims[3]) {
  if (!origin || !dims) return fail(PRRTC_ERR_INVALID_ARG, "null grid argument");
  if (!(voxel > 0.f) || !std::isfinite(voxel) || !finite_all(origin, 3))
    return fail(PRRTC_ERR_INVALID_ARG, "voxel must be > 0 and the origin finite");
  size_t V = 1;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 2 || dims[a] > PRRTC_ESDF_MAX_DIM) return fail(PRRTC_ERR_INVALID_ARG, "grid dimension out of range");
    V *= (size_t)dims[a];
  }
  if (V > ((size_t)1 << 28)) return fail(PRRTC_ERR_INVALID_ARG, "grid has too many voxels");
  return PRRTC_OK;
}

int prrtc_env_create_esdf(const float origin[3], float voxel, const int32_t dims[3], const uint8_t* occupancy,
                          prrtc_env** out) {
  if (!out) return fail(PRRTC_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  int rc = check_grid(origin, voxel, dims);
  if (rc) return rc;
  if (!occupancy) return fail(PRRTC_ERR_INVALID_ARG, "occupancy is null");
  prrtc_env* e = nullptr;
  if ((rc = prrtc_env_create(nullptr, 0, &e))) return rc;
  for (int a = 0; a < 3; ++a) {
    e->dims[a] = dims[a];
    e->origin[a] = origin[a];
  }
  e->voxel = voxel;
  const size_t V = e->voxels();
  if (cudaMalloc(&e->d_esdf, V * sizeof(float)) != cudaSuccess || cudaMalloc(&e->d_occ, V) != cudaSuccess ||
      cudaMalloc(&e->d_tmp, 2 * V * sizeof(int2)) != cudaSuccess) {
    cudaGetLastError();
    prrtc_env_destroy(e);
    return fail(PRRTC_ERR_OOM, "distance field allocation failed");
  }
  if ((rc = prrtc_env_update_esdf(e, occupancy))) {
    prrtc_env_destroy(e);
    return rc;
  }
  *out = e;
  return PRRTC_OK;
}

int prrtc_env_update_esdf(prrtc_env* env, const uint8_t* occupancy) {
  if (!env || !occupancy || !env->d_esdf) return fail(PRRTC_ERR_INVALID_ARG, "env has no distance field");
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  if (c->device != env->device) return fail(PRRTC_ERR_INVALID_ARG, "env belongs to another device");
  std::lock_guard<std::mutex> lk(c->mu);
  std::lock_guard<std::mutex> lk_env(env->mu);
  const size_t V = env->voxels();
  // stream-ordered: planning calls issued before see the old field, later ones the new
  CK(cudaMemcpyAsync(env->d_occ, occupancy, V, cudaMemcpyHostToDevice, c->stream));
  cudaError_t e = launch_esdf(env->d_occ, env->dims, env->voxel, env->d_tmp, env->d_tmp + V, env->d_esdf, c->stream);
  if (e != cudaSuccess) return cuda_fail("distance transform launch", e);
  CK(cudaStreamSynchronize(c->stream));
  return PRRTC_OK;
}

int prrtc_env_esdf_values(const prrtc_env* env, float* out) {
  if (!env || !out || !env->d_esdf) return fail(PRRTC_ERR_INVALID_ARG, "env has no distance field");
  CK(cudaMemcpy(out, env->d_esdf, env->voxels() * sizeof(float), cudaMemcpyDeviceToHost));
  return PRRTC_OK;
}

int prrtc_voxelize(const prrtc_env* env, const float origin[3], float voxel, const int32_t dims[3],
                   uint8_t* occupancy) {
  if (!env || !occupancy) return fail(PRRTC_ERR_INVALID_ARG, "null argument");
  int rc = check_grid(origin, voxel, dims);
  if (rc) return rc;
  DeviceCtx* c = nullptr;
  if ((rc = current_ctx(&c))) return rc;
  if (c->device != env->device) return fail(PRRTC_ERR_INVALID_ARG, "env belongs to another device");
  const size_t V = (size_t)dims[0] * dims[1] * dims[2];
  uint8_t* d = nullptr;
  if (cudaMalloc(&d, V) != cudaSuccess) {
    cudaGetLastError();
    return fail(PRRTC_ERR_OOM, "voxel buffer allocation failed");
  }
  std::lock_guard<std::mutex> lk(c->mu);
  const int dd[3] = {dims[0], dims[1], dims[2]};
  cudaError_t e = launch_voxelize(env->view(), origin, voxel, dd, d, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(occupancy, d, V, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail("voxelize", e);
  return PRRTC_OK;
}

// -------------------------------------------------------------- robot
}  // extern "C"

namespace {

// First-stage spheres of the two-stage check: for each frame with two or more
// distinct spheres, the sphere around the centre of their offsets' bounding
// box that contains every one of them, enlarged by 1e-5 m (plus one part in
// 10^6) so that FP32 rounding of the FK cannot make a fine sphere poke out.
void set_bounding_spheres(RobotHeader& H) {
  for (int f = 0; f < kMaxDof; ++f) H.coarse[f] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int f = 0; f < H.dof; ++f) {
    const int s0 = H.sph_begin[f], s1 = H.sph_begin[f + 1];
    if (s1 - s0 < 2) continue;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int s = s0; s < s1; ++s) {
      const double o[3] = {H.sph[s].x, H.sph[s].y, H.sph[s].z};
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], o[a]);
        hi[a] = std::max(hi[a], o[a]);
      }
    }
    const float cx = (float)(0.5 * (lo[0] + hi[0])), cy = (float)(0.5 * (lo[1] + hi[1])),
                cz = (float)(0.5 * (lo[2] + hi[2]));
    double rad = 0.0;
    for (int s = s0; s < s1; ++s) {
      const double dx = (double)H.sph[s].x - cx, dy = (double)H.sph[s].y - cy, dz = (double)H.sph[s].z - cz;
      rad = std::max(rad, std::sqrt(dx * dx + dy * dy + dz * dz) + (double)H.sph[s].w);
    }
    H.coarse[f] = make_float4(cx, cy, cz, (float)(rad * (1.0 + 1e-6) + 1e-5));
  }
}

}  // namespace

extern "C" {

int prrtc_robot_create(const prrtc_robot_desc* d, prrtc_robot** out) {
  if (!out) return fail(PRRTC_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!d) return fail(PRRTC_ERR_INVALID_ARG, "desc is null");
  if (d->dof < 1 || d->dof > PRRTC_MAX_DOF) return fail(PRRTC_ERR_INVALID_ARG, "dof out of range");
  if (!d->joint_type || !d->joint_parent || !d->joint_base || !d->link_length || !d->lower || !d->upper)
    return fail(PRRTC_ERR_INVALID_ARG, "null joint table");
  if (d->n_spheres < 0 || d->n_spheres > PRRTC_MAX_SPHERES || (d->n_spheres > 0 && (!d->sphere_frame ||
      !d->sphere_offset || !d->sphere_radius)))
    return fail(PRRTC_ERR_INVALID_ARG, "bad sphere table");
  if (d->n_pairs < 0 || d->n_pairs > PRRTC_MAX_PAIRS || (d->n_pairs > 0 && !d->self_pairs))
    return fail(PRRTC_ERR_INVALID_ARG, "bad pair table");
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  const int dof = d->dof;
  for (int i = 0; i < dof; ++i) {
    if (d->joint_type[i] < 0 || d->joint_type[i] > 5) return fail(PRRTC_ERR_INVALID_ARG, "unknown joint type");
    if (d->joint_parent[i] != -1 && d->joint_parent[i] != i - 1)
      return fail(PRRTC_ERR_UNSUPPORTED, "joint_parent must be -1 or i-1 (serial chains)");
    if (!std::isfinite(d->lower[i]) || !std::isfinite(d->upper[i]) || d->lower[i] > d->upper[i])
      return fail(PRRTC_ERR_INVALID_ARG, "bad joint limits");
  }
  if (!finite_all(d->joint_base, 3 * dof) || !finite_all(d->link_length, dof))
    return fail(PRRTC_ERR_INVALID_ARG, "non-finite joint table");
  // Home frame of every sphere: a sphere on the rotation axis of a revolute
  // joint whose link has zero length does not move with that joint, so it is
  // carried by the parent frame with the same offset (T_f o = T_{f-1} J_f o
  // = T_{f-1} o).  This puts the joint-housing spheres into the group of the
  // link that ends at the joint, where the two-stage check bounds them; FK
  // places them at bit-identical centres (the offset is on the axis).
  std::vector<int> home(d->n_spheres, 0);
  for (int s = 0; s < d->n_spheres; ++s) {
    int f = d->sphere_frame[s];
    if (f < 0 || f >= dof) return fail(PRRTC_ERR_INVALID_ARG, "sphere frame out of range");
    const float* o = d->sphere_offset + 3 * s;
    while (f > 0 && d->joint_parent[f] == f - 1 && d->link_length[f] == 0.f) {
      const int ty = d->joint_type[f];
      const bool on_axis = (ty == PRRTC_JOINT_REV_Z && o[0] == 0.f && o[1] == 0.f) ||
                           (ty == PRRTC_JOINT_REV_Y && o[0] == 0.f && o[2] == 0.f) ||
                           (ty == PRRTC_JOINT_REV_X && o[1] == 0.f && o[2] == 0.f);
      if (!on_axis) break;
      --f;
    }
    home[s] = f;
  }
  // merge coincident equal-radius spheres of one frame; keep them grouped by frame
  std::vector<int> raw_to(d->n_spheres, -1);
  std::vector<std::tuple<int, float, float, float, float>> distinct;
  for (int f = 0; f < dof; ++f) {
    for (int s = 0; s < d->n_spheres; ++s) {
      const int fr = home[s];
      if (fr != f) continue;
      const float* o = d->sphere_offset + 3 * s;
      const float r = d->sphere_radius[s];
      if (!(r > 0.f) || !finite_all(o, 3) || !std::isfinite(r)) return fail(PRRTC_ERR_INVALID_ARG, "bad sphere");
      auto key = std::make_tuple(f, o[0], o[1], o[2], r);
      int idx = -1;
      for (size_t k = 0; k < distinct.size(); ++k)
        if (distinct[k] == key) idx = (int)k;
      if (idx < 0) {
        idx = (int)distinct.size();
        distinct.push_back(key);
      }
      raw_to[s] = idx;
    }
  }
  if ((int)distinct.size() > kMaxDistinctSpheres) return fail(PRRTC_ERR_UNSUPPORTED, "too many distinct spheres");
  std::vector<std::pair<int, int>> pairs;
  for (int k = 0; k < d->n_pairs; ++k) {
    const int a = d->self_pairs[2 * k], b = d->self_pairs[2 * k + 1];
    if (a < 0 || b < 0 || a >= d->n_spheres || b >= d->n_spheres) return fail(PRRTC_ERR_INVALID_ARG, "pair index");
    int x = raw_to[a], y = raw_to[b];
    if (x > y) std::swap(x, y);
    pairs.emplace_back(x, y);
  }
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  if ((int)pairs.size() > kMaxDistinctPairs) return fail(PRRTC_ERR_UNSUPPORTED, "too many distinct pairs");

  RobotDev* h = (RobotDev*)std::calloc(1, sizeof(RobotDev));
  if (!h) return fail(PRRTC_ERR_OOM, "host allocation failed");
  RobotHeader& H = h->h;
  H.dof = dof;
  H.dpad = std::max(4, (dof + 3) & ~3);
  H.n_spheres = (int)distinct.size();
  H.n_pairs = (int)pairs.size();
  H.n_raw = d->n_spheres;
  for (int i = 0; i < dof; ++i) {
    H.jtype[i] = d->joint_type[i];
    H.jparent[i] = d->joint_parent[i];
    H.jlen[i] = d->link_length[i];
    H.lo[i] = d->lower[i];
    H.span[i] = d->upper[i] - d->lower[i];
    H.jbase[i] = make_float4(d->joint_base[3 * i], d->joint_base[3 * i + 1], d->joint_base[3 * i + 2], 0.f);
  }
  int s = 0;
  for (int f = 0; f <= dof; ++f) {
    while (s < (int)distinct.size() && std::get<0>(distinct[s]) < f) ++s;
    H.sph_begin[f] = s;
  }
  H.sph_begin[dof] = (int)distinct.size();
  for (int f = dof + 1; f <= kMaxDof; ++f) H.sph_begin[f] = (int)distinct.size();
  for (size_t k = 0; k < distinct.size(); ++k)
    H.sph[k] = make_float4(std::get<1>(distinct[k]), std::get<2>(distinct[k]), std::get<3>(distinct[k]),
                           std::get<4>(distinct[k]));
  set_bounding_spheres(H);
  H.two_stage = 1;
  // group sphere per link for the self-collision first stage: its bounding
  // sphere when it has several spheres, else its only sphere
  for (int f = 0; f < kMaxDof; ++f) H.grp[f] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int f = 0; f < dof; ++f) {
    const int n_f = H.sph_begin[f + 1] - H.sph_begin[f];
    if (n_f >= 2) H.grp[f] = H.coarse[f];
    else if (n_f == 1) H.grp[f] = H.sph[H.sph_begin[f]];
  }
  // pairs in blocks of one link pair each, sorted by first sphere inside a block
  auto frame_of = [&](int k) { return std::get<0>(distinct[k]); };
  std::sort(pairs.begin(), pairs.end(), [&](const std::pair<int, int>& a, const std::pair<int, int>& b) {
    const int fa = frame_of(a.first), fb = frame_of(b.first), ga = frame_of(a.second), gb = frame_of(b.second);
    if (fa != fb) return fa < fb;
    if (ga != gb) return ga < gb;
    return a < b;
  });
  int nb = 0;
  for (size_t k = 0; k < pairs.size();) {
    const int fa = frame_of(pairs[k].first), fb = frame_of(pairs[k].second);
    size_t e = k;
    while (e < pairs.size() && frame_of(pairs[e].first) == fa && frame_of(pairs[e].second) == fb) ++e;
    if (nb >= kMaxPairBlocks) {
      std::free(h);
      return fail(PRRTC_ERR_UNSUPPORTED, "too many self-collision link pairs");
    }
    H.blk_frames[nb] = (uint32_t)fa | ((uint32_t)fb << 16);
    H.blk_range[nb] = (uint32_t)k | ((uint32_t)e << 16);
    const float rr = H.grp[fa].w + H.grp[fb].w;
    // one pair, or pairs within one link: no first stage
    H.blk_thr[nb] = (e - k > 1 && fa != fb) ? rr * rr : INFINITY;
    ++nb;
    k = e;
  }
  H.n_blocks = nb;
  for (size_t k = 0; k < pairs.size(); ++k) {
    h->pair[k] = (uint32_t)pairs[k].first | ((uint32_t)pairs[k].second << 16);
    const float rr = H.sph[pairs[k].first].w + H.sph[pairs[k].second].w;
    h->thr[k] = rr * rr;
  }
  for (int r = 0; r < d->n_spheres; ++r) h->raw_to_distinct[r] = (int16_t)raw_to[r];

  prrtc_robot* rb = new prrtc_robot();
  rb->device = c->device;
  rb->h = h;
  if (cudaMalloc(&rb->d, sizeof(RobotDev)) != cudaSuccess) {
    cudaGetLastError();
    std::free(h);
    delete rb;
    return fail(PRRTC_ERR_OOM, "robot allocation failed");
  }
  cudaError_t ce = cudaMemcpy(rb->d, h, sizeof(RobotDev), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaFree(rb->d);
    std::free(h);
    delete rb;
    return cuda_fail("robot upload", ce);
  }
  *out = rb;
  return PRRTC_OK;
}

void prrtc_robot_destroy(prrtc_robot* robot) {
  if (!robot) return;
  cudaFree(robot->d);
  std::free(robot->h);
  delete robot;
}

int prrtc_robot_set_two_stage(prrtc_robot* robot, int32_t enabled) {
  if (!robot || !robot->h) return fail(PRRTC_ERR_INVALID_ARG, "robot is null");
  robot->h->h.two_stage = enabled ? 1 : 0;
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != robot->device) return fail(PRRTC_ERR_INVALID_ARG, "robot belongs to another device");
  // everything queued on the device may still read the old header: wait for it
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&robot->d->h.two_stage, &robot->h->h.two_stage, sizeof(int), cudaMemcpyHostToDevice));
  return PRRTC_OK;
}

int prrtc_robot_bounds(const prrtc_robot* robot, float* out4) {
  if (!robot || !robot->h || !out4) return fail(PRRTC_ERR_INVALID_ARG, "null argument");
  const RobotHeader& H = robot->h->h;
  for (int f = 0; f < H.dof; ++f) {
    out4[4 * f + 0] = H.coarse[f].x;
    out4[4 * f + 1] = H.coarse[f].y;
    out4[4 * f + 2] = H.coarse[f].z;
    out4[4 * f + 3] = H.coarse[f].w;
  }
  return PRRTC_OK;
}

// Extra introspection used by tests and the benchmark.
int prrtc_robot_info(const prrtc_robot* robot, int32_t* dof, int32_t* n_spheres, int32_t* n_pairs, int32_t* dpad) {
  if (!robot) return fail(PRRTC_ERR_INVALID_ARG, "robot is null");
  if (dof) *dof = robot->h->h.dof;
  if (n_spheres) *n_spheres = robot->h->h.n_spheres;
  if (n_pairs) *n_pairs = robot->h->h.n_pairs;
  if (dpad) *dpad = robot->h->h.dpad;
  return PRRTC_OK;
}

// Device-side views of two handles, for entry points compiled in other files
// (not part of the public header).  Allocates nothing.
int prrtc_internal_views(const prrtc_robot* robot, const prrtc_env* env, const void** robot_dev,
                         const void** robot_header, EnvView* env_view, int* device) {
  if (!robot || !env || !robot->h || robot->device != env->device) return PRRTC_ERR_INVALID_ARG;
  *robot_dev = robot->d;
  *robot_header = &robot->h->h;
  *env_view = env->view();
  *device = robot->device;
  return PRRTC_OK;
}

int prrtc_internal_env_view(const prrtc_env* env, EnvView* view, int* device) {
  if (!env) return PRRTC_ERR_INVALID_ARG;
  *view = env->view();
  *device = env->device;
  return PRRTC_OK;
}

void prrtc_internal_set_error(const char* msg) { t_last_error = msg ? msg : ""; }

int prrtc_internal_robot_view(const prrtc_robot* robot, const RobotDev** dev, const RobotHeader** header,
                              int* device) {
  if (!robot) return PRRTC_ERR_INVALID_ARG;
  *dev = robot->d;
  *header = &robot->h->h;
  *device = robot->device;
  return PRRTC_OK;
}

int prrtc_env_info(const prrtc_env* env, int32_t* counts4) {
  if (!env || !counts4) return fail(PRRTC_ERR_INVALID_ARG, "null argument");
  counts4[0] = env->n_aabb;
  counts4[1] = env->n_obb;
  counts4[2] = env->n_cyl;
  counts4[3] = env->n_sph;
  return PRRTC_OK;
}

// -------------------------------------------------------------- collision checking
int prrtc_check_states_device(const prrtc_robot* robot, const prrtc_env* env, const float* q_device, int32_t n,
                              uint8_t* valid_device, float* spheres_device, void* stream) {
  if (!robot || !env || n < 0 || (n > 0 && (!q_device || !valid_device)))
    return fail(PRRTC_ERR_INVALID_ARG, "bad check_states arguments");
  if (n == 0) return PRRTC_OK;
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  if (robot->device != c->device || env->device != c->device)
    return fail(PRRTC_ERR_INVALID_ARG, "handle belongs to another device");
  cudaError_t e = launch_check_states(robot->d, robot->h->h, env->view(), q_device, n, valid_device, spheres_device,
                                      c->d_counters, c->d_error, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail("check_states launch", e);
  return PRRTC_OK;
}

int prrtc_philox(const uint32_t* ctr, int32_t n, uint64_t key, uint32_t* out) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return fail(PRRTC_ERR_INVALID_ARG, "bad philox arguments");
  if (n == 0) return PRRTC_OK;
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  uint32_t* d = nullptr;
  const size_t bytes = (size_t)n * 4 * sizeof(uint32_t);
  if (cudaMalloc(&d, 2 * bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(PRRTC_ERR_OOM, "philox buffer allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(d, ctr, bytes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_philox(d, n, key, d + (size_t)n * 4, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + (size_t)n * 4, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail("philox", e);
  return PRRTC_OK;
}

int prrtc_alu_peak(int32_t iters, double* lane_ops_per_s, double* kernel_ms) {
  if (iters < 1 || !lane_ops_per_s) return fail(PRRTC_ERR_INVALID_ARG, "bad alu_peak arguments");
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  float* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)c->sms * 8 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(PRRTC_ERR_OOM, "alu_peak buffer allocation failed");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  long long ops = 0;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_fma_loop(c->sms, iters, sink, c->stream, &ops);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  if (e == cudaSuccess) e = launch_fma_loop(c->sms, iters, sink, c->stream, &ops);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail("alu_peak", e);
  *lane_ops_per_s = (double)ops / ((double)ms * 1e-3);
  if (kernel_ms) *kernel_ms = ms;
  return PRRTC_OK;
}

int prrtc_check_states(const prrtc_robot* robot, const prrtc_env* env, const float* q, int32_t n, uint8_t* out_valid,
                       float* out_spheres) {
  if (!robot || !env || n < 0 || (n > 0 && (!q || !out_valid)))
    return fail(PRRTC_ERR_INVALID_ARG, "bad check_states arguments");
  if (n == 0) return PRRTC_OK;
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  if (robot->device != c->device || env->device != c->device)
    return fail(PRRTC_ERR_INVALID_ARG, "handle belongs to another device");
  std::lock_guard<std::mutex> lk(c->mu);
  const int dof = robot->h->h.dof, n_raw = robot->h->h.n_raw;
  if ((rc = grow_device(&c->d_q, &c->q_cap, (size_t)n * dof))) return rc;
  if ((rc = grow_device(&c->d_valid, &c->valid_cap, (size_t)n))) return rc;
  if (out_spheres && (rc = grow_device(&c->d_spheres, &c->spheres_cap, (size_t)n * n_raw * 4))) return rc;
  CK(cudaMemcpyAsync(c->d_q, q, (size_t)n * dof * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->d_counters, 0, 8 * sizeof(unsigned long long), c->stream));
  CK(cudaMemsetAsync(c->d_error, 0, sizeof(int), c->stream));
  CK(cudaEventRecord(c->ev[0], c->stream));
  cudaError_t e = launch_check_states(robot->d, robot->h->h, env->view(), c->d_q, n, c->d_valid,
                                      out_spheres ? c->d_spheres : nullptr, c->d_counters, c->d_error, c->stream);
  if (e != cudaSuccess) return cuda_fail("check_states launch", e);
  CK(cudaEventRecord(c->ev[1], c->stream));
  CK(cudaMemcpyAsync(out_valid, c->d_valid, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
  if (out_spheres)
    CK(cudaMemcpyAsync(out_spheres, c->d_spheres, (size_t)n * n_raw * 4 * sizeof(float), cudaMemcpyDeviceToHost,
                       c->stream));
  unsigned long long cnt[7] = {0, 0, 0, 0, 0, 0, 0};
  int err = 0;
  CK(cudaMemcpyAsync(cnt, c->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&err, c->d_error, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
  cudaGetLastError();
  c->last = prrtc_launch_stats{};
  c->last.kernel_ms = ms;
  c->last.sphere_tests = (int64_t)cnt[0];
  c->last.pair_tests = (int64_t)cnt[1];
  c->last.fk_states = (int64_t)cnt[2];
  for (int k = 0; k < 4; ++k) {
    c->last.prim_tests[k] = (int64_t)cnt[3 + k];
    c->last.env_tests += (int64_t)cnt[3 + k];
  }
  c->last.problems = 0;
  c->last.kernels = 1;
  c->last.h2d_bytes = (int64_t)n * dof * (int64_t)sizeof(float);
  c->last.d2h_bytes = (int64_t)n + (out_spheres ? (int64_t)n * n_raw * 4 * (int64_t)sizeof(float) : 0);
  if (err) return fail(err, "device-side wait gave up in check_states");
  return PRRTC_OK;
}

// -------------------------------------------------------------- planning
}  // extern "C"

// Implemented in prrtc_mlp.cu.
int prrtc_internal_proposal_stage(prrtc_proposal* p, const EnvView* envs, const float* qs_host, const float* qg_host,
                                  int B, float* const* gmm_rows);
int prrtc_internal_proposal_submit(prrtc_proposal* p, cudaStream_t stream);
float prrtc_internal_proposal_infer_ms(prrtc_proposal* p);
extern "C" int prrtc_proposal_info(const prrtc_proposal*, int32_t*, int32_t*, int64_t*, int32_t*);

static int plan_batch_impl(const prrtc_problem* problems, int32_t n, const prrtc_params* params,
                           prrtc_proposal* const* proposals, prrtc_path* out_paths, int32_t* out_status) {
  if (!problems || n < 1) return fail(PRRTC_ERR_INVALID_ARG, "no problems");
  int rc = validate_params(params);
  if (rc) return rc;
  DeviceCtx* c = nullptr;
  rc = current_ctx(&c);
  if (rc) return rc;
  for (int p = 0; p < n; ++p) {
    const prrtc_problem& pb = problems[p];
    if (!pb.robot || !pb.env || !pb.q_start || !pb.q_goal)
      return fail(PRRTC_ERR_INVALID_ARG, "problem " + std::to_string(p) + " has a null field");
    if (pb.robot->device != c->device || pb.env->device != c->device)
      return fail(PRRTC_ERR_INVALID_ARG, "handle belongs to another device");
    const int dof = pb.robot->h->h.dof;
    if (!finite_all(pb.q_start, dof) || !finite_all(pb.q_goal, dof))
      return fail(PRRTC_ERR_INVALID_ARG, "non-finite start or goal");
  }
  std::lock_guard<std::mutex> lk(c->mu);
  if ((rc = ensure_arenas(c, n, params->tree_capacity, params->path_capacity))) return rc;

  // learned mixtures: given by the caller (host) or inferred on the device
  bool any_gmm = false;
  for (int p = 0; p < n; ++p) any_gmm |= (problems[p].gmm != nullptr) || (proposals && proposals[p]);
  if (any_gmm && c->gmm_cap < (size_t)n) {
    cudaFree(c->d_gmm);
    cudaFreeHost(c->h_gmm);
    c->d_gmm = nullptr;
    c->h_gmm = nullptr;
    c->gmm_cap = 0;
    if (cudaMalloc(&c->d_gmm, (size_t)n * kGmmStride * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&c->h_gmm, (size_t)n * kGmmStride * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(PRRTC_ERR_OOM, "mixture buffer allocation failed");
    }
    c->gmm_cap = (size_t)n;
  }
  // lockstep mode: each problem's held rows, [workers][held_rows x dpad].  Every
  // node lies in the box spanned by the joint limits, the start and the goal
  // (samples lie in the limits, steps are convex combinations), so a connect
  // takes at most ceil(diagonal / range) steps.
  std::vector<int> held_rows(n, 0);
  std::vector<size_t> held_off(n + 1, 0);
  if (params->mode == PRRTC_MODE_LOCKSTEP) {
    for (int p = 0; p < n; ++p) {
      const prrtc_problem& pb = problems[p];
      const RobotHeader& H = pb.robot->h->h;
      double diag2 = 0.0;
      for (int j = 0; j < H.dof; ++j) {
        const double lo = std::min({(double)H.lo[j], (double)pb.q_start[j], (double)pb.q_goal[j]});
        const double hi = std::max({(double)H.lo[j] + (double)H.span[j], (double)pb.q_start[j], (double)pb.q_goal[j]});
        diag2 += (hi - lo) * (hi - lo);
      }
      held_rows[p] = 3 + (int)std::ceil(std::sqrt(diag2) / (double)params->range * (1.0 + 1e-5));
      held_off[p + 1] = held_off[p] + (size_t)params->workers * held_rows[p] * H.dpad;
    }
    if (held_off[n] > ((size_t)1 << 28)) return fail(PRRTC_ERR_OOM, "lockstep scratch above 1 GiB");
    if ((rc = grow_device(&c->d_held, &c->held_cap, held_off[n]))) return rc;
    if ((rc = grow_device(&c->d_held_meta, &c->held_meta_cap, (size_t)n * params->workers * kHeldMeta))) return rc;
  }
  int max_spheres = 1, max_pairs = 0, max_env = 0, max_dof = 1;
  for (int p = 0; p < n; ++p) {
    const prrtc_problem& pb = problems[p];
    const RobotHeader& H = pb.robot->h->h;
    max_dof = std::max(max_dof, H.dof);
    ProblemDesc& D = c->h_desc[p];
    std::memset(&D, 0, sizeof(D));
    D.robot = pb.robot->d;
    D.env = pb.env->view();
    const size_t tree_stride = (size_t)c->cap * kMaxDof;
    D.nodes[0] = c->nodes + ((size_t)p * 2 + 0) * tree_stride;
    D.nodes[1] = c->nodes + ((size_t)p * 2 + 1) * tree_stride;
    D.parent[0] = c->parents + ((size_t)p * 2 + 0) * c->cap;
    D.parent[1] = c->parents + ((size_t)p * 2 + 1) * c->cap;
    float* radii = reinterpret_cast<float*>(c->parents + (size_t)c->slots * 2 * c->cap);
    D.radius[0] = radii + ((size_t)p * 2 + 0) * c->cap;
    D.radius[1] = radii + ((size_t)p * 2 + 1) * c->cap;
    D.path = c->paths + (size_t)p * c->path_cap * kMaxDof;
    D.path_idx = c->path_idx + (size_t)p * c->path_cap;
    D.cap = params->tree_capacity;
    D.dpad = H.dpad;
    D.dof = H.dof;
    D.n_spheres = H.n_spheres;
    D.n_pairs = H.n_pairs;
    D.key_lo = (uint32_t)(pb.seed & 0xffffffffu);
    D.key_hi = (uint32_t)(pb.seed >> 32);
    D.pid = pb.problem_id;
    D.gmm = (pb.gmm || (proposals && proposals[p])) ? c->d_gmm + (size_t)p * kGmmStride : nullptr;
    if (params->mode == PRRTC_MODE_LOCKSTEP) {
      D.held = c->d_held + held_off[p];
      D.held_meta = c->d_held_meta + (size_t)p * params->workers * kHeldMeta;
      D.held_rows = held_rows[p];
    }
    for (int j = 0; j < H.dof; ++j) {
      D.q_start[j] = pb.q_start[j];
      D.q_goal[j] = pb.q_goal[j];
    }
    max_spheres = std::max(max_spheres, H.n_spheres + H.dof);  // staging slots: spheres + group centres
    max_pairs = std::max(max_pairs, H.n_pairs);
    max_env = std::max(max_env, D.env.n_float4());
  }
  PlanGlobals& G = *c->h_glob;
  std::memset(&G, 0, sizeof(G));
  G.n_problems = n;
  globals_from_params(G, *params);
  G.t0 = ULLONG_MAX;
  G.time_limit_ns = (unsigned long long)(params->time_limit_s * 1e9);
  G.cursor = 0;
  G.error = 0;

  int blocks = params->blocks, warps = params->warps_per_block;
  if (blocks == 0 && warps == 0) {
    // the autotuner's choice for this workload, for the fields the caller left at 0
    auto it = c->tuned.find(tune_key(c->h_desc[0].dpad, max_env, n, params->mode));
    if (it != c->tuned.end()) {
      blocks = it->second.blocks;
      warps = it->second.warps;
      if (params->obstacle_tile == 0) G.obstacle_tile = it->second.tile;
      if (params->expansions == 0 && params->mode == PRRTC_MODE_ASYNC) G.expansions = it->second.expansions;
    }
  }
  const PlanLaunch cfg =
      plan_launch_config(n, params->mode, blocks, warps, max_spheres, max_pairs, max_env, c->sms, params->workers);
  bool lean = params->sampler == PRRTC_SAMPLER_PHILOX && !cfg.lockstep && !(params->dd_radius > 0.f);
  for (int p = 0; p < n && lean; ++p) lean = problem_is_lean(problems[p].robot->h->h, c->h_desc[p]);
  if (cfg.smem > 227 * 1024) return fail(PRRTC_ERR_UNSUPPORTED, "robot + environment exceed shared memory");
  const int head_rows = (n == 1) ? std::min(kHeadRows, params->path_capacity) : 0;
  // A batch copies the first rows of every path back with its results; only a
  // longer path needs the gather after the results are read.
  const int batch_head = (n > 1) ? std::min(kBatchHeadRows, params->path_capacity) : 0;
  const int head_stride = batch_head * max_dof;
  if (batch_head && (size_t)n * head_stride > c->heads_cap) {
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_heads);
    cudaFreeHost(c->h_heads);
    c->d_heads = nullptr;
    c->h_heads = nullptr;
    c->heads_cap = 0;
    const size_t want = (size_t)n * head_stride;
    if (cudaMalloc(&c->d_heads, want * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&c->h_heads, want * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(PRRTC_ERR_OOM, "path head buffer allocation failed");
    }
    c->heads_cap = want;
    c->arena_gen++;  // the captured launch sequence holds the old buffers
  }

  // Host half of the learned inference (grouping, staging), before the timed
  // device work like the descriptors: one batch per distinct proposal.
  std::vector<prrtc_proposal*> staged;
  if (proposals) {
    std::vector<int> done(n, 0);
    for (int p = 0; p < n; ++p) {
      if (!proposals[p] || done[p]) continue;
      prrtc_proposal* prop = proposals[p];
      int pdof = 0;
      prrtc_proposal_info(prop, &pdof, nullptr, nullptr, nullptr);
      std::vector<EnvView> envs;
      std::vector<float> qs, qg;
      std::vector<float*> rows;
      for (int r = p; r < n; ++r) {
        if (proposals[r] != prop) continue;
        const prrtc_problem& pb = problems[r];
        if (pb.robot->h->h.dof != pdof) return fail(PRRTC_ERR_INVALID_ARG, "proposal DoF does not match the robot");
        envs.push_back(pb.env->view());
        qs.insert(qs.end(), pb.q_start, pb.q_start + pdof);
        qg.insert(qg.end(), pb.q_goal, pb.q_goal + pdof);
        rows.push_back(c->d_gmm + (size_t)r * kGmmStride);
        done[r] = 1;
      }
      const int rc2 = prrtc_internal_proposal_stage(prop, envs.data(), qs.data(), qg.data(), (int)envs.size(),
                                                    rows.data());
      if (rc2) return rc2;
      staged.push_back(prop);
    }
  }

  // Prep time runs from the call's first device work -- the mixture upload or
  // inference, else the descriptor upload -- to the setup kernel.  The host
  // work above (descriptors, launch shape, inference staging) comes before it
  // in both cases.
  CK(cudaEventRecord(c->ev[3], c->stream));
  bool host_gmm = false;
  for (int p = 0; p < n; ++p) {
    const prrtc_problem& pb = problems[p];
    if (!pb.gmm || (proposals && proposals[p])) continue;
    const int dof = pb.robot->h->h.dof;
    float* g = c->h_gmm + (size_t)p * kGmmStride;
    std::memset(g, 0, kGmmStride * sizeof(float));
    for (int k = 0; k < kMixK; ++k) {
      g[k] = pb.gmm[k];
      for (int j = 0; j < dof; ++j) {
        g[kMixK + k * kMaxDof + j] = pb.gmm[kMixK + k * dof + j];
        g[kMixK + kMixK * kMaxDof + k * kMaxDof + j] =
            std::min(std::max(pb.gmm[kMixK + kMixK * dof + k * dof + j], -5.f), 2.f);
      }
    }
    if (!finite_all(g, kGmmStride)) return fail(PRRTC_ERR_INVALID_ARG, "non-finite mixture");
    host_gmm = true;
  }
  if (host_gmm)
    CK(cudaMemcpyAsync(c->d_gmm, c->h_gmm, (size_t)n * kGmmStride * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  for (prrtc_proposal* prop : staged) {
    const int rc2 = prrtc_internal_proposal_submit(prop, c->stream);
    if (rc2) return rc2;
  }

  // The launch sequence: descriptors in, setup, planner, bookkeeping, results
  // out (and, for one problem, the head of its path).  Replayed as a CUDA graph
  // while its shape stays the same.
  // Timing events become external event nodes when the sequence is captured.
  auto enqueue = [&](bool capturing) -> int {
    const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    CK(cudaMemcpyAsync(c->d_desc, c->h_desc, (size_t)n * sizeof(ProblemDesc), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_glob, c->h_glob, sizeof(PlanGlobals), cudaMemcpyHostToDevice, c->stream));
    CK(cudaEventRecordWithFlags(c->ev[0], c->stream, ev_flags));
    cudaError_t e =
        launch_setup(c->d_desc, c->d_state, n, max_spheres, max_pairs, max_env, c->stream, nullptr, &c->d_glob->error);
    if (e != cudaSuccess) return cuda_fail("setup launch", e);
    CK(cudaEventRecordWithFlags(c->ev[1], c->stream, ev_flags));
    e = launch_plan(c->d_glob, c->d_desc, c->d_state, cfg, G.obstacle_tile, lean, c->stream);
    if (e != cudaSuccess) return cuda_fail("plan launch", e);
    CK(cudaEventRecordWithFlags(c->ev[2], c->stream, ev_flags));
    e = launch_record_usage(c->d_desc, c->d_state, n, c->stream);
    if (e != cudaSuccess) return cuda_fail("usage launch", e);
    CK(cudaMemcpyAsync(c->h_state, c->d_state, (size_t)n * sizeof(ProblemState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->h_glob, c->d_glob, sizeof(PlanGlobals), cudaMemcpyDeviceToHost, c->stream));
    if (head_rows)
      CK(cudaMemcpyAsync(c->h_path_head, c->paths, (size_t)head_rows * c->h_desc[0].dof * sizeof(float),
                         cudaMemcpyDeviceToHost, c->stream));
    if (batch_head) {
      e = launch_gather_heads(c->d_desc, c->d_state, n, batch_head, head_stride, c->d_heads, c->stream);
      if (e != cudaSuccess) return cuda_fail("path head launch", e);
      CK(cudaMemcpyAsync(c->h_heads, c->d_heads, (size_t)n * head_stride * sizeof(float), cudaMemcpyDeviceToHost,
                         c->stream));
    }
    return PRRTC_OK;
  };
  static const bool no_graph = std::getenv("PRRTC_NO_GRAPH") != nullptr;
  if (no_graph) {
    if ((rc = enqueue(false))) return rc;
  } else {
    const DeviceCtx::GraphKey key{n, cfg.grid, cfg.warps, cfg.smem, cfg.robot_bytes, cfg.env_bytes, cfg.stage_bytes,
                                  max_spheres, max_pairs, max_env, c->arena_gen, head_rows * c->h_desc[0].dof,
                                  cfg.lockstep ? 1 : 0, G.obstacle_tile, head_stride, lean ? 1 : 0};
    if (!c->gexec || !(c->gkey == key)) {
      if (c->gexec) cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
      const int rc2 = enqueue(true);
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
      if (rc2) {
        if (graph) cudaGraphDestroy(graph);
        return rc2;
      }
      if (ec != cudaSuccess) return cuda_fail("graph capture", ec);
      const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail("graph instantiate", ei);
      }
      c->gkey = key;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));

  // per-problem outcome and packed path offsets
  std::vector<int> status(n);
  int total = 0;
  c->h_offsets[0] = 0;
  for (int p = 0; p < n; ++p) {
    const ProblemState& S = c->h_state[p];
    int st;
    if (S.pre_status) st = S.pre_status;
    else if (S.solved) st = (S.path_status == PRRTC_SOLVED || S.path_status == PRRTC_PATH_OVERFLOW) ? S.path_status
                                                                                                     : PRRTC_ERR_TIMEOUT;
    else if (S.timed_out) st = PRRTC_TIME_LIMIT;
    else st = PRRTC_NO_SOLUTION;
    status[p] = st;
    const int rows = (st == PRRTC_SOLVED) ? S.path_n : 0;
    total += rows * c->h_desc[p].dof;
    c->h_offsets[p + 1] = total;
  }
  const bool from_head = head_rows > 0 && status[0] == PRRTC_SOLVED && c->h_state[0].path_n <= head_rows;
  bool from_heads = batch_head > 0;
  for (int p = 0; p < n && from_heads; ++p)
    if (status[p] == PRRTC_SOLVED && c->h_state[p].path_n > batch_head) from_heads = false;
  const bool gathered = !from_head && !from_heads && total > 0;
  if (from_head || (from_heads && total > 0)) {
    if ((size_t)total > c->packed_cap) {
      cudaFreeHost(c->h_packed);
      cudaFree(c->d_packed);
      c->d_packed = nullptr;
      c->h_packed = nullptr;
      c->packed_cap = 0;
      if (cudaMallocHost(&c->h_packed, (size_t)std::max(total, 1) * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&c->d_packed, (size_t)std::max(total, 1) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(PRRTC_ERR_OOM, "path buffer allocation failed");
      }
      c->packed_cap = (size_t)std::max(total, 1);
    }
    if (from_head) {
      std::memcpy(c->h_packed, c->h_path_head, (size_t)total * sizeof(float));
    } else {
      for (int p = 0; p < n; ++p)
        if (status[p] == PRRTC_SOLVED)
          std::memcpy(c->h_packed + c->h_offsets[p], c->h_heads + (size_t)p * head_stride,
                      (size_t)(c->h_offsets[p + 1] - c->h_offsets[p]) * sizeof(float));
    }
  } else if (gathered) {
    if ((size_t)total > c->packed_cap) {
      cudaFree(c->d_packed);
      cudaFreeHost(c->h_packed);
      c->d_packed = nullptr;
      c->h_packed = nullptr;
      c->packed_cap = 0;
      if (cudaMalloc(&c->d_packed, (size_t)total * sizeof(float)) != cudaSuccess ||
          cudaMallocHost(&c->h_packed, (size_t)total * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(PRRTC_ERR_OOM, "path buffer allocation failed");
      }
      c->packed_cap = (size_t)total;
    }
    CK(cudaMemcpyAsync(c->d_offsets, c->h_offsets, (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    const cudaError_t e = launch_gather_paths(c->d_desc, c->d_offsets, n, c->d_packed, c->stream);
    if (e != cudaSuccess) return cuda_fail("gather launch", e);
    CK(cudaMemcpyAsync(c->h_packed, c->d_packed, (size_t)total * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }

  float setup_ms = 0.f, plan_ms = 0.f, prep_ms = 0.f;
  cudaEventElapsedTime(&setup_ms, c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&plan_ms, c->ev[1], c->ev[2]);
  cudaEventElapsedTime(&prep_ms, c->ev[3], c->ev[0]);
  cudaGetLastError();  // timing is best effort: leave no error behind for later calls
  prrtc_launch_stats L{};
  L.prep_ms = prep_ms;
  for (prrtc_proposal* prop : staged) L.infer_ms += prrtc_internal_proposal_infer_ms(prop);
  L.kernel_ms = plan_ms;
  L.setup_ms = setup_ms;
  L.grid = cfg.grid;
  L.block_threads = cfg.warps * 32;
  L.smem_bytes = cfg.smem;
  L.problems = n;
  L.h2d_bytes = (int64_t)n * (int64_t)sizeof(ProblemDesc) + (int64_t)sizeof(PlanGlobals) +
                (gathered ? (int64_t)(n + 1) * (int64_t)sizeof(int) : 0);
  L.d2h_bytes = (int64_t)n * (int64_t)sizeof(ProblemState) + (int64_t)sizeof(PlanGlobals) +
                ((int64_t)head_rows * c->h_desc[0].dof + (int64_t)n * head_stride + (gathered ? total : 0)) *
                    (int64_t)sizeof(float);
  L.kernels = 3 + (batch_head ? 1 : 0) + (gathered ? 1 : 0);
  L.lean_kernel = lean ? 1 : 0;
  const unsigned long long t0 = c->h_glob->t0;
  for (int p = 0; p < n; ++p) {
    const ProblemState& S = c->h_state[p];
    L.edges_checked += (int64_t)S.edges;
    L.edge_states += (int64_t)S.edge_states;
    L.sphere_tests += (int64_t)S.sphere_tests;
    L.pair_tests += (int64_t)S.pair_tests;
    L.fk_states += (int64_t)S.fk_states;
    L.nn_nodes += (int64_t)S.nn_nodes;
    L.iterations += (int64_t)S.iterations;
    L.dd_rejected += (int64_t)S.dd_rejected;
    L.verdict_states += (int64_t)S.verdict_states;
    for (int k = 0; k < 4; ++k) {
      L.prim_tests[k] += (int64_t)S.prim_tests[k];
      L.env_tests += (int64_t)S.prim_tests[k];
    }
    if (out_status) out_status[p] = status[p];
    if (out_paths) {
      prrtc_path& P = out_paths[p];
      std::memset(&P, 0, sizeof(P));
      const int dof = c->h_desc[p].dof;
      P.status = status[p];
      P.dof = dof;
      P.iterations = reported_iterations(S, *params);
      P.nodes_a = std::min(S.count[0], params->tree_capacity);
      P.nodes_b = std::min(S.count[1], params->tree_capacity);
      P.edges_checked = (int64_t)S.edges;
      P.edge_states = (int64_t)S.edge_states;
      P.solve_time_us = (S.solved && S.t_solve >= t0) ? (double)(S.t_solve - t0) * 1e-3 : -1.0;
      P.sphere_tests = (int64_t)S.sphere_tests;
      P.pair_tests = (int64_t)S.pair_tests;
      P.fk_states = (int64_t)S.fk_states;
      P.nn_nodes = (int64_t)S.nn_nodes;
      P.dd_rejected = (int64_t)S.dd_rejected;
      P.verdict_states = (int64_t)S.verdict_states;
      for (int k = 0; k < 4; ++k) P.prim_tests[k] = (int64_t)S.prim_tests[k];
      if (status[p] == PRRTC_SOLVED) {
        P.n = S.path_n;
        P.cost = S.cost;
        P.q = (float*)std::malloc((size_t)S.path_n * dof * sizeof(float));
        if (!P.q) return fail(PRRTC_ERR_OOM, "host path allocation failed");
        std::memcpy(P.q, c->h_packed + c->h_offsets[p], (size_t)S.path_n * dof * sizeof(float));
      } else if (status[p] == PRRTC_PATH_OVERFLOW) {
        P.n = S.path_n;
        P.cost = S.cost;
      }
    }
  }
  c->last = L;
  if (c->h_glob->error) return fail(c->h_glob->error, "device-side wait gave up in the planner");
  return PRRTC_OK;
}

extern "C" {

int prrtc_plan_batch(const prrtc_problem* problems, int32_t n, const prrtc_params* params, prrtc_path* out_paths,
                     int32_t* out_status) {
  return plan_batch_impl(problems, n, params, nullptr, out_paths, out_status);
}

int prrtc_plan_batch_learned(const prrtc_problem* problems, prrtc_proposal* const* proposals, int32_t n,
                             const prrtc_params* params, prrtc_path* out_paths, int32_t* out_status) {
  return plan_batch_impl(problems, n, params, proposals, out_paths, out_status);
}

int prrtc_autotune(const prrtc_problem* problems, int32_t n, const prrtc_params* params, int32_t trials,
                   prrtc_params* best, double* best_ms) {
  if (!problems || n < 1 || !params || trials < 1 || !best) return fail(PRRTC_ERR_INVALID_ARG, "bad autotune arguments");
  int rc = validate_params(params);
  if (rc) return rc;
  if (params->mode == PRRTC_MODE_LOCKSTEP)
    return fail(PRRTC_ERR_INVALID_ARG, "lockstep mode runs a fixed schedule: nothing to tune");
  DeviceCtx* c = nullptr;
  if ((rc = current_ctx(&c))) return rc;
  int resident = 0, max_env = 0;
  {
    // one wave of resident blocks for 4 warps, the default grid of a batch
    const RobotHeader& H = problems[0].robot->h->h;
    for (int p = 0; p < n; ++p) max_env = std::max(max_env, problems[p].env->view().n_float4());
    resident = plan_launch_config(n, params->mode, 0, 4, H.n_spheres + H.dof, H.n_pairs, max_env, c->sms).grid;
    if (n == 1) resident = c->sms * 4;
  }
  std::vector<prrtc_problem> pb(problems, problems + n);
  // The score of a candidate: the mean over `trials` runs (the same trial keys
  // for every candidate) of the mean of the batch's median and 95th-percentile
  // time to first solution -- the two quantiles of the planning-time metric --
  // with setup time plus each problem's device time from launch start to its
  // solution, an unsolved problem counting the whole launch.  The batch's step
  // time (the maximum) and mean are led by the few hardest problems and are
  // noisy; the two quantiles follow the typical and the hard problems.  The
  // choices below keep a default unless a candidate beats it clearly.
  std::vector<double> ttfs(n);
  auto measure = [&](const prrtc_params& q, double* out) -> int {
    double tot = 0.0;
    for (int k = 0; k < trials; ++k) {
      for (int p = 0; p < n; ++p) pb[p].seed = problems[p].seed + 7919ull * (uint64_t)(k + 1);
      const int r = plan_batch_impl(pb.data(), n, &q, nullptr, nullptr, nullptr);
      if (r) return r;
      const unsigned long long t0 = c->h_glob->t0;
      for (int p = 0; p < n; ++p) {
        const ProblemState& S = c->h_state[p];
        const bool solved = S.solved && S.t_solve >= t0;
        ttfs[p] = solved ? (double)(S.t_solve - t0) * 1e-6 : c->last.kernel_ms;
      }
      std::sort(ttfs.begin(), ttfs.end());
      const double p50 = ttfs[n / 2], p95 = ttfs[std::min(n - 1, (int)std::ceil(0.95 * n) - 1)];
      tot += c->last.setup_ms + 0.5 * (p50 + p95);
    }
    *out = tot / trials;
    return PRRTC_OK;
  };
  constexpr double kClearly = 0.97;  // a non-default tile or expansions must be 3% faster
  constexpr double kTie = 1.02;      // launch shapes within 2% count as equal: more workers win
  // 1. launch shape: blocks x warps per block (Sec. IV-C: the number of
  //    concurrent workers), obstacle tile and expansions at their defaults
  std::vector<std::pair<int, int>> cands;
  const int warp_opts[5] = {2, 3, 4, 6, 8};
  for (int w : warp_opts) {
    if (params->mode == PRRTC_MODE_SERIAL && w != 1) continue;
    if (n == 1) {
      for (int workers : {64, 128, 256, 512, 1024}) cands.emplace_back(std::max(1, workers / w), w);
    } else {
      const int full = std::max(1, resident * 4 / w);
      cands.emplace_back(std::max(1, full / 2), w);
      cands.emplace_back(full, w);
    }
  }
  if (params->mode == PRRTC_MODE_SERIAL) cands.emplace_back(0, 1);
  prrtc_params q = *params;
  q.obstacle_tile = params->obstacle_tile ? params->obstacle_tile : 32;
  q.expansions = params->expansions ? params->expansions : 1;
  std::vector<double> times(cands.size());
  double best_t = 1e30;
  for (size_t i = 0; i < cands.size(); ++i) {
    prrtc_params r = q;
    r.blocks = cands[i].first;
    r.warps_per_block = cands[i].second;
    if ((rc = measure(r, &times[i]))) return rc;
    best_t = std::min(best_t, times[i]);
  }
  // among the shapes within kTie of the fastest, the one with the most workers
  // (it checks the most states in the same time)
  long long most = -1;
  for (size_t i = 0; i < cands.size(); ++i) {
    const long long workers = (long long)std::max(cands[i].first, 1) * cands[i].second;
    if (times[i] <= kTie * best_t && workers > most) {
      most = workers;
      q.blocks = cands[i].first;
      q.warps_per_block = cands[i].second;
      best_t = std::min(best_t, times[i]);
    }
  }
  for (size_t i = 0; i < cands.size(); ++i)
    if (cands[i].first == q.blocks && cands[i].second == q.warps_per_block) best_t = times[i];
  // 2. obstacle tile: primitives per first-stage round (one or two per lane)
  if (params->obstacle_tile == 0) {
    prrtc_params r = q;
    r.obstacle_tile = 64;
    double t = 0.0;
    if ((rc = measure(r, &t))) return rc;
    if (t < kClearly * best_t) {
      best_t = t;
      q.obstacle_tile = 64;
    }
  }
  // 3. expansions per claim of a problem's iteration counter (async mode)
  if (params->expansions == 0 && params->mode == PRRTC_MODE_ASYNC) {
    for (int e : {2, 4, 8}) {
      prrtc_params r = q;
      r.expansions = e;
      double t = 0.0;
      if ((rc = measure(r, &t))) return rc;
      if (t < kClearly * best_t) {
        best_t = t;
        q.expansions = e;
      }
    }
  }
  *best = q;
  if (best_ms) *best_ms = best_t;
  std::lock_guard<std::mutex> lk(c->mu);
  c->tuned[tune_key(problems[0].robot->h->h.dpad, max_env, n, params->mode)] =
      DeviceCtx::Tuned{q.blocks, q.warps_per_block, q.obstacle_tile, q.expansions};
  return PRRTC_OK;
}

int prrtc_debug_tree(int32_t problem, int32_t tree, float* nodes, int32_t* parents, int32_t cap, int32_t* out_n) {
  if (tree < 0 || tree > 1 || cap < 0 || !out_n) return fail(PRRTC_ERR_INVALID_ARG, "bad debug_tree arguments");
  DeviceCtx* c = nullptr;
  int rc = current_ctx(&c);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  if (problem < 0 || problem >= c->last.problems || !c->h_desc)
    return fail(PRRTC_ERR_INVALID_ARG, "problem not in the last launch");
  const ProblemDesc& D = c->h_desc[problem];
  const ProblemState& S = c->h_state[problem];
  const int rows = std::min(S.count[tree], D.cap);
  *out_n = rows;
  const int m = std::min(rows, cap);
  if (m <= 0) return PRRTC_OK;
  if (nodes) {
    std::vector<float> buf((size_t)m * D.dpad);
    CK(cudaMemcpy(buf.data(), D.nodes[tree], buf.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (int r = 0; r < m; ++r)
      for (int j = 0; j < D.dof; ++j) nodes[(size_t)r * D.dof + j] = buf[(size_t)r * D.dpad + j];
  }
  if (parents) {
    CK(cudaMemcpy(parents, D.parent[tree], (size_t)m * sizeof(int), cudaMemcpyDeviceToHost));
    for (int r = 0; r < m; ++r)
      if (parents[r] == kRootParent) parents[r] = -1;
  }
  return PRRTC_OK;
}

int prrtc_plan(const prrtc_robot* robot, const prrtc_env* env, const float* q_start, const float* q_goal,
               const prrtc_params* params, prrtc_path* out_path) {
  if (!out_path) return fail(PRRTC_ERR_INVALID_ARG, "out_path is null");
  prrtc_problem pb;
  std::memset(&pb, 0, sizeof(pb));
  pb.robot = robot;
  pb.env = env;
  pb.q_start = q_start;
  pb.q_goal = q_goal;
  pb.seed = params ? params->seed : 1;
  pb.problem_id = 0;
  pb.gmm = nullptr;
  return prrtc_plan_batch(&pb, 1, params, out_path, nullptr);
}

}  // extern "C"
