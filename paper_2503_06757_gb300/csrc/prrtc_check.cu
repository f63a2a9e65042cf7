// prrtc_check.cu -- batched collision verdicts of given configurations
// (Sec. III-A): sphere-model FK, sphere-vs-primitive and self-collision tests.
// One lane per configuration; robot tables and the obstacle set are staged in
// shared memory by TMA bulk copies.  Used for the per-state parity check
// against the oracle and as the FP32-roofline microbenchmark (collision-free
// states: every test must run).
#include <algorithm>

#include "prrtc.h"
#include "prrtc_launch.h"

namespace prrtc {

namespace {

constexpr int kCheckWarps = 4;

constexpr int kQStageFloats = kMaxDof * 32;  // per warp: [joint][lane]

__global__ void __launch_bounds__(kCheckWarps * 32) check_states_kernel(const RobotDev* __restrict__ robot, EnvView env,
                                                                        const float* __restrict__ q, int n,
                                                                        uint8_t* __restrict__ valid,
                                                                        float* __restrict__ spheres,
                                                                        unsigned long long* __restrict__ counters,
                                                                        int* __restrict__ error, int np_pad) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_ok;
  __shared__ WarpCount s_count[kCheckWarps];
  const int robot_bytes = robot_smem_bytes(np_pad);
  RobotHeader* R = reinterpret_cast<RobotHeader*>(smem);
  uint32_t* pair = reinterpret_cast<uint32_t*>(smem + sizeof(RobotHeader));
  float* thr = reinterpret_cast<float*>(pair + np_pad);
  const int env_f4 = env.n_float4();
  float4* senv = reinterpret_cast<float4*>(smem + robot_bytes);
  float* warp_all = reinterpret_cast<float*>(smem + robot_bytes + env_f4 * 16);

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    const uint32_t bytes = (uint32_t)sizeof(RobotHeader) + 8u * (uint32_t)np_pad + 16u * (uint32_t)env_f4;
    mbar_arrive_expect_tx(&bar, bytes);
    bulk_g2s(R, &robot->h, sizeof(RobotHeader), &bar);
    if (np_pad) {
      bulk_g2s(pair, robot->pair, 4u * np_pad, &bar);
      bulk_g2s(thr, robot->thr, 4u * np_pad, &bar);
    }
    if (env_f4) bulk_g2s(senv, env.data, 16u * env_f4, &bar);
    s_ok = mbar_wait(&bar, 0, 1u << 26) ? 1 : 0;
    if (!s_ok) {
      atomicExch(error, PRRTC_ERR_TIMEOUT);
      mbar_wait(&bar, 0, 1u << 26);  // the block leaves: its copies first (bounded)
    }
  }
  __syncthreads();
  if (!s_ok) return;  // block-uniform

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int dof = R->dof;
  const int n_raw = R->n_raw;
  float* qst = warp_all + warp * (kQStageFloats + (R->n_spheres + R->dof) * 96);
  float* stage = qst + kQStageFloats;
  const int gw = blockIdx.x * kCheckWarps + warp;
  const int nw = gridDim.x * kCheckWarps;
  WarpCount* wc = &s_count[warp];
  warp_count_clear(wc, lane);
  const LaneQ qs{qst, lane};
  for (int base = gw * 32; base < n; base += nw * 32) {
    const int idx = base + lane;
    const bool active = idx < n;
    const size_t src = (size_t)(active ? idx : n - 1) * dof;
    for (int j = 0; j < dof; ++j) qst[j * 32 + lane] = q[src + j];
    const bool hit = state_collides<false>(R, pair, thr, senv, env.n_aabb, env.n_obb, env.n_cyl, env.n_sph, env.esdf,
                                           stage, qs, active, lane, wc);
    if (active) {
      valid[idx] = hit ? 0 : 1;
      if (spheres) {
        float4* out = reinterpret_cast<float4*>(spheres) + (size_t)idx * n_raw;
        for (int r = 0; r < n_raw; ++r) {
          const int ds = robot->raw_to_distinct[r];
          const float* st = stage + ds * 96 + lane;
          out[r] = make_float4(st[0], st[32], st[64], R->sph[ds].w);
        }
      }
    }
  }
  // the warp's work counters: sphere passes, pairs, FK states, second-stage tests
  __syncwarp();
  if (lane < 7 && counters) atomicAdd(counters + lane, reinterpret_cast<const unsigned long long*>(wc)[lane]);
}

}  // namespace

// One Philox4x32-10 block per thread (the sampler's generator).
__global__ void philox_kernel(const uint4* __restrict__ ctr, int n, uint2 key, uint4* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = philox4x32_10(ctr[i], key);
}

cudaError_t launch_philox(const uint32_t* ctr, int n, uint64_t key, uint32_t* out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>(((long long)n + 255) / 256, 152LL * 16);
  philox_kernel<<<blocks, 256, 0, stream>>>(reinterpret_cast<const uint4*>(ctr), n,
                                            make_uint2((uint32_t)(key & 0xffffffffu), (uint32_t)(key >> 32)),
                                            reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

// The FP32 pipe at full rate: kChains independent FMA chains per thread, so
// that every warp scheduler always has an FMA ready.  One FMA counts one
// lane-op, the unit of the planner's ALU roofline.  The sum is stored only
// when it equals a value it never takes, which keeps the chains alive.
constexpr int kFmaChains = 8;
__global__ void fma_loop_kernel(int iters, float m, float* __restrict__ sink) {
  float a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], m, 1e-7f);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  if (s == -1.f) sink[blockIdx.x] = s;
}

cudaError_t launch_fma_loop(int sm_count, int iters, float* sink, cudaStream_t stream, long long* lane_ops) {
  const int blocks = sm_count * 8, threads = 256;  // 64 warps per SM
  fma_loop_kernel<<<blocks, threads, 0, stream>>>(iters, 0.9999999f, sink);
  *lane_ops = (long long)blocks * threads * iters * kFmaChains;
  return cudaGetLastError();
}

cudaError_t launch_check_states(const RobotDev* robot, const RobotHeader& h, EnvView env, const float* q, int n,
                                uint8_t* valid, float* spheres, unsigned long long* counters, int* error,
                                cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int np_pad = (h.n_pairs + 3) & ~3;
  const int smem = robot_smem_bytes(np_pad) + env.n_float4() * 16 +
                   kCheckWarps * (kQStageFloats * (int)sizeof(float) + stage_bytes(h.n_spheres + h.dof));
  cudaError_t e = cudaFuncSetAttribute(check_states_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, check_states_kernel, kCheckWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long want = ((long long)n + kCheckWarps * 32 - 1) / (kCheckWarps * 32);
  const int grid = (int)(want < (long long)sms * per_sm ? (want > 0 ? want : 1) : (long long)sms * per_sm);
  check_states_kernel<<<grid, kCheckWarps * 32, smem, stream>>>(robot, env, q, n, valid, spheres, counters, error,
                                                               np_pad);
  return cudaGetLastError();
}

}  // namespace prrtc
