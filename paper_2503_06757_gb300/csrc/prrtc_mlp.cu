// prrtc_mlp.cu -- the learned sampling proposal on the device.
//
// A small MLP maps [occupancy 16^3 | start | goal] to an 8-component diagonal
// Gaussian mixture over joint values normalised to [-1, 1].  Dense layers run
// on the tensor cores (prrtc_gemm.cu: BF16 operands, FP32 accumulation);
// everything else is elementwise or per-sample work:
//   forward   x -> relu(W1 x + b1) -> relu(W2 .) -> relu(W3 .) -> W4 . + b4
//   loss      mean mixture negative log-likelihood of target configurations
//   backward  dW = dZ^T H, dH = dZ W (BF16 operands transposed explicitly),
//             ReLU masks, bias column sums
//   update    Adam on FP32 master weights, then BF16 copies (and transposes)
// The proposal is an addition to pRRTC (the paper samples uniformly).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <random>
#include <string>
#include <vector>

#include "prrtc.h"
#include "prrtc_launch.h"

using bf16 = __nv_bfloat16;

namespace prrtc {
namespace {

constexpr int kGrid = 16, kVox = kGrid * kGrid * kGrid, kQPad = 32, kIn = kVox + 2 * kQPad, kK = 8;
constexpr int kHid0 = 1024, kHid1 = 512, kHid2 = 512;
constexpr float kCell = 0.1f, kOccRadius = 0.05f;
constexpr float kLogSigMin = -5.f, kLogSigMax = 2.f;

int head_pad(int dof) { return ((kK * (1 + 2 * dof) + 127) / 128) * 128; }

// ------------------------------------------------------------------ kernels
// Occupancy grids of B environments, scattered per obstacle: voxel
// (i, j, k) -> index i + 16 j + 256 k is occupied iff its centre is closer
// than 5 cm to an obstacle (a 5 cm sphere there would collide).  One warp per
// obstacle visits only the voxels inside the obstacle's bounding box grown by
// 5 cm and applies the exact primitive test; grids must start zeroed (all
// writers store 1, so overlapping obstacles need no ordering).  blockIdx.y
// selects the environment.
__device__ __forceinline__ float grid_origin(int axis) { return axis < 2 ? -0.8f : 0.0f; }
__device__ __forceinline__ int vox_lo(float x, int axis) {
  return max(0, (int)floorf((x - grid_origin(axis)) / kCell - 0.5f));
}
__device__ __forceinline__ int vox_hi(float x, int axis) {
  return min(kGrid - 1, (int)ceilf((x - grid_origin(axis)) / kCell - 0.5f));
}

__global__ void occupancy_scatter_kernel(const EnvView* __restrict__ envs, uint8_t* __restrict__ out) {
  const EnvView env = envs[blockIdx.y];
  uint8_t* grid = out + (size_t)blockIdx.y * kVox;
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const int n_obs = env.n_aabb + env.n_obb + env.n_cyl + env.n_sph;
  for (int o = (int)(blockIdx.x * warps + (threadIdx.x >> 5)); o < n_obs; o += gridDim.x * warps) {
    // locate obstacle o in the blob and bound it
    EnvView one{};
    float3 c, e;
    const float m = kOccRadius;
    if (o < env.n_aabb) {
      one.data = env.data + 2 * o;
      one.n_aabb = 1;
      const float4 a = one.data[0], h = one.data[1];
      c = make_float3(a.x, a.y, a.z);
      e = make_float3(h.x + m, h.y + m, h.z + m);
    } else if (o < env.n_aabb + env.n_obb) {
      one.data = env.data + 2 * env.n_aabb + 5 * (o - env.n_aabb);
      one.n_obb = 1;
      const float4 a = one.data[0], h = one.data[1], r0 = one.data[2], r1 = one.data[3], r2 = one.data[4];
      c = make_float3(a.x, a.y, a.z);
      // world half extents of the rotated box: sum_j |R[k][j]| h_j (r_j = column j of R)
      e = make_float3(fabsf(r0.x) * h.x + fabsf(r1.x) * h.y + fabsf(r2.x) * h.z + m,
                      fabsf(r0.y) * h.x + fabsf(r1.y) * h.y + fabsf(r2.y) * h.z + m,
                      fabsf(r0.z) * h.x + fabsf(r1.z) * h.y + fabsf(r2.z) * h.z + m);
    } else if (o < env.n_aabb + env.n_obb + env.n_cyl) {
      one.data = env.data + 2 * env.n_aabb + 5 * env.n_obb + 2 * (o - env.n_aabb - env.n_obb);
      one.n_cyl = 1;
      const float4 a = one.data[0], ax = one.data[1];
      c = make_float3(a.x, a.y, a.z);
      const float rb = sqrtf(a.w * a.w + ax.w * ax.w) + m;
      e = make_float3(rb, rb, rb);
    } else {
      one.data = env.data + 2 * env.n_aabb + 5 * env.n_obb + 2 * env.n_cyl + (o - env.n_aabb - env.n_obb - env.n_cyl);
      one.n_sph = 1;
      const float4 a = one.data[0];
      c = make_float3(a.x, a.y, a.z);
      e = make_float3(a.w + m, a.w + m, a.w + m);
    }
    const int i0 = vox_lo(c.x - e.x, 0), i1 = vox_hi(c.x + e.x, 0);
    const int j0 = vox_lo(c.y - e.y, 1), j1 = vox_hi(c.y + e.y, 1);
    const int k0 = vox_lo(c.z - e.z, 2), k1 = vox_hi(c.z + e.z, 2);
    if (i1 < i0 || j1 < j0 || k1 < k0) continue;
    const int ni = i1 - i0 + 1, nj = j1 - j0 + 1, nk = k1 - k0 + 1;
    for (int t = lane; t < ni * nj * nk; t += 32) {
      const int i = i0 + t % ni, j = j0 + (t / ni) % nj, k = k0 + t / (ni * nj);
      const float px = grid_origin(0) + (i + 0.5f) * kCell;
      const float py = grid_origin(1) + (j + 0.5f) * kCell;
      const float pz = grid_origin(2) + (k + 0.5f) * kCell;
      if (sphere_hits_env(px, py, pz, kOccRadius, one.data, one.n_aabb, one.n_obb, one.n_cyl, one.n_sph))
        grid[i + kGrid * j + kGrid * kGrid * k] = 1;
    }
  }
}

// One feature row per sample (rows past B are zero): occupancy of the
// sample's scene, then normalised start and goal, each zero-padded to 32.
__global__ void features_kernel(const uint8_t* __restrict__ occ, const int* __restrict__ scene_of,
                                const int* __restrict__ rows, const float* __restrict__ qs,
                                const float* __restrict__ qg, const float* __restrict__ lo,
                                const float* __restrict__ span, int B, int dof, bf16* __restrict__ x) {
  const int b = blockIdx.x;
  bf16* dst = x + (size_t)b * kIn;
  if (b >= B) {
    for (int c = threadIdx.x; c < kIn; c += blockDim.x) dst[c] = __float2bfloat16_rn(0.f);
    return;
  }
  const int r = rows ? rows[b] : b;
  const int s = scene_of ? scene_of[r] : r;
  const uint8_t* o = occ + (size_t)s * kVox;
  for (int c = threadIdx.x; c < kIn; c += blockDim.x) {
    float v;
    if (c < kVox) {
      v = o[c] ? 1.f : 0.f;
    } else {
      const int j = (c - kVox) % kQPad;
      const float* q = (c < kVox + kQPad) ? qs : qg;
      v = (j < dof) ? 2.f * (q[(size_t)r * dof + j] - lo[j]) / span[j] - 1.f : 0.f;
    }
    dst[c] = __float2bfloat16_rn(v);
  }
}

// Occupancy part of the first layer for a few environments, W[:, :4096] x_occ,
// read straight from the 0/1 grids: one warp per output feature streams its
// weight row once (16-byte loads) and sums the weights of occupied voxels for
// every environment; fixed order, so the result is deterministic.
constexpr int kGemvMaxEnvs = 32;

__global__ void __launch_bounds__(256) l1_occ_gemv_kernel(const uint8_t* __restrict__ occ, int U,
                                                           const bf16* __restrict__ w, float* __restrict__ out) {
  __shared__ uint32_t bits[kGemvMaxEnvs][kVox / 32];
  for (int t = threadIdx.x; t < U * (kVox / 32); t += blockDim.x) {
    const int u = t / (kVox / 32), word = t % (kVox / 32);
    const uint8_t* o = occ + (size_t)u * kVox + word * 32;
    uint32_t b = 0;
    for (int i = 0; i < 32; ++i) b |= (o[i] ? 1u : 0u) << i;
    bits[u][word] = b;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= kHid0) return;
  // the whole 8 KB weight row in flight at once: 16 loads of 16 bytes per lane
  const uint4* row = reinterpret_cast<const uint4*>(w + (size_t)j * kIn);
  uint4 raw[kVox / 256];
#pragma unroll
  for (int it = 0; it < kVox / 256; ++it) raw[it] = __ldg(row + it * 32 + lane);
  for (int u0 = 0; u0 < U; u0 += 8) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int it = 0; it < kVox / 256; ++it) {
      const int c0 = it * 256 + lane * 8;  // this lane's 8 consecutive voxels
      const bf16* wv = reinterpret_cast<const bf16*>(&raw[it]);
      float wf[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) wf[i] = __bfloat162float(wv[i]);
#pragma unroll
      for (int du = 0; du < 8; ++du) {
        if (u0 + du < U) {
          const uint32_t b8 = bits[u0 + du][c0 / 32] >> (c0 % 32);
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[du] += ((b8 >> i) & 1u) ? wf[i] : 0.f;
        }
      }
    }
#pragma unroll
    for (int du = 0; du < 8; ++du) {
      float v = acc[du];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && u0 + du < U) out[(size_t)(u0 + du) * kHid0 + j] = v;
    }
  }
}

// Occupancy rows (one per distinct environment) as BF16 inputs of the
// occupancy part of the first layer, for batches with many environments.
__global__ void occ_bf16_kernel(const uint8_t* __restrict__ occ, bf16* __restrict__ x) {
  const size_t base = (size_t)blockIdx.x * kVox;
  for (int c = threadIdx.x; c < kVox; c += blockDim.x) x[base + c] = __float2bfloat16_rn(occ[base + c] ? 1.f : 0.f);
}

// Mixture negative log-likelihood of each sample's target and its gradient
// with respect to the head output (scaled by 1/B).  One warp per sample;
// lane k < 8 owns component k.
__global__ void mixture_loss_kernel(const float* __restrict__ out, int P, const float* __restrict__ target,
                                    const int* __restrict__ rows, const float* __restrict__ lo,
                                    const float* __restrict__ span, int B, int dof, float invB,
                                    float* __restrict__ dout32, bf16* __restrict__ dout16,
                                    float* __restrict__ loss_sum) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= B) return;
  const int r = rows ? rows[warp] : warp;
  const float* o = out + (size_t)warp * P;
  const bool comp = lane < kK;
  const int k = comp ? lane : 0;
  const float logit = comp ? o[k] : -INFINITY;
  float mx = logit;
  for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, off));
  float se = comp ? expf(logit - mx) : 0.f;
  for (int off = 16; off; off >>= 1) se += __shfl_xor_sync(kFull, se, off);
  const float logpi = logit - mx - logf(se);
  float a = -INFINITY;
  if (comp) {
    a = logpi - 0.5f * dof * 1.8378770664093453f;  // log(2 pi)
    for (int j = 0; j < dof; ++j) {
      const float u = 2.f * (target[(size_t)r * dof + j] - lo[j]) / span[j] - 1.f;
      const float ls = fminf(fmaxf(o[kK + kK * dof + k * dof + j], kLogSigMin), kLogSigMax);
      const float z = (u - o[kK + k * dof + j]) * expf(-ls);
      a += -0.5f * z * z - ls;
    }
  }
  float am = a;
  for (int off = 16; off; off >>= 1) am = fmaxf(am, __shfl_xor_sync(kFull, am, off));
  float sa = comp ? expf(a - am) : 0.f;
  for (int off = 16; off; off >>= 1) sa += __shfl_xor_sync(kFull, sa, off);
  const float lse = am + logf(sa);
  float* d32 = dout32 + (size_t)warp * P;
  bf16* d16 = dout16 + (size_t)warp * P;
  if (comp) {
    const float gamma = expf(a - lse), pi = expf(logpi);
    const float gl = (pi - gamma) * invB;
    d32[k] = gl;
    d16[k] = __float2bfloat16_rn(gl);
    for (int j = 0; j < dof; ++j) {
      const float u = 2.f * (target[(size_t)r * dof + j] - lo[j]) / span[j] - 1.f;
      const float raw = o[kK + kK * dof + k * dof + j];
      const float ls = fminf(fmaxf(raw, kLogSigMin), kLogSigMax);
      const float isig = expf(-ls);
      const float z = (u - o[kK + k * dof + j]) * isig;
      const float gm = -gamma * z * isig * invB;
      const float gs = (raw > kLogSigMin && raw < kLogSigMax) ? -gamma * (z * z - 1.f) * invB : 0.f;
      d32[kK + k * dof + j] = gm;
      d16[kK + k * dof + j] = __float2bfloat16_rn(gm);
      d32[kK + kK * dof + k * dof + j] = gs;
      d16[kK + kK * dof + k * dof + j] = __float2bfloat16_rn(gs);
    }
  }
  if (lane == 0) atomicAdd(loss_sum, -lse * invB);
}

// dZ = dH * [H > 0] in FP32 and BF16.
__global__ void relu_back_kernel(const float* __restrict__ dh, const bf16* __restrict__ h, size_t n,
                                 float* __restrict__ dz32, bf16* __restrict__ dz16) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = (__bfloat162float(h[i]) > 0.f) ? dh[i] : 0.f;
    dz32[i] = v;
    dz16[i] = __float2bfloat16_rn(v);
  }
}

// out[c] = sum over rows of g[r, c].
__global__ void colsum_kernel(const float* __restrict__ g, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += g[(size_t)r * cols + c];
  out[c] = s;
}

// out[c, r] = in[r, c] (BF16, 32 x 32 tiles through shared memory).
__global__ void transpose_kernel(const bf16* __restrict__ in, int rows, int cols, bf16* __restrict__ out) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[(size_t)c * rows + r] = tile[threadIdx.x][k];
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ in, size_t n, bf16* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// Adam with bias-corrected moments: c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

}  // namespace
}  // namespace prrtc

using namespace prrtc;

// ------------------------------------------------------------------ handle
namespace prrtc {
namespace {
// One staged inference batch: offsets into the staging block and its shape.
struct Pending {
  size_t o_env = 0, o_map = 0, o_rows = 0, o_qs = 0, o_qg = 0, bytes = 0;
  int B = 0, rows = 0, U = 0;
  uint64_t sig = 0;
};
}  // namespace
}  // namespace prrtc

struct prrtc_proposal {
  int device = -1;
  int dof = 0, P = 0;
  int in_dim[4], out_dim[4];
  size_t w_off[4], b_off[4], n_params = 0;
  float* master = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16* w16[4] = {};
  bf16* w16t[4] = {};
  bf16* wtile[3] = {};  // layers 2, 3 and the head, tiled for the fused inference kernel
  int step = 0;
  float lo[kMaxDof], span[kMaxDof];
  float* d_lims = nullptr;  // lo[16] | span[16]
  cudaStream_t stream = nullptr;
  // batch scratch
  int cap = 0;
  bf16 *x16 = nullptr, *xT = nullptr, *h16[3] = {}, *hT[3] = {}, *d16 = nullptr, *dT = nullptr, *z16[3] = {},
       *zT[3] = {};
  float *out32 = nullptr, *d32 = nullptr, *dh32 = nullptr, *z32[3] = {}, *loss = nullptr;
  // sample data
  uint8_t* occ = nullptr;
  size_t occ_cap = 0;
  float *qs = nullptr, *qg = nullptr, *tgt = nullptr;
  int *scene_of = nullptr, *rows = nullptr;
  size_t q_cap = 0, qg_cap = 0, tgt_cap = 0, scene_cap = 0, rows_cap = 0;
  EnvView* envs = nullptr;
  size_t envs_cap = 0;
  float** gmm_rows = nullptr;
  size_t gmm_rows_cap = 0;
  cudaEvent_t done = nullptr;
  // inference for planning: the per-call inputs staged in one pinned buffer
  // and copied with one transfer; the kernel chain replayed as a CUDA graph
  unsigned char* h_stage = nullptr;
  size_t h_stage_cap = 0;
  unsigned char* d_stage = nullptr;
  size_t d_stage_cap = 0;
  uint8_t* inf_occ = nullptr;
  size_t inf_occ_cap = 0;
  // first layer split by distinct environment (occupancy part once per environment)
  bf16* xo16 = nullptr;    // [envs x kVox]
  size_t xo16_cap = 0;
  float* h1o32 = nullptr;  // [envs x kHid0]
  size_t h1o32_cap = 0;
  bf16* atile[3] = {};     // tiled hidden activations, 128-row tiles
  int last_infer_B = 0;    // problems of the last staged inference batch
  size_t atile_cap[3] = {};
  Pending pend;            // the staged, not yet submitted, inference batch
  bool pend_ok = false;
  cudaEvent_t inf_ev[2] = {};  // timing of the last submitted chain
  bool inf_timed = false;
  cudaGraphExec_t infer_exec = nullptr;
  uint64_t infer_sig = 0;  // signature of the buffers baked into infer_exec
  uint64_t seen_sig = 0;   // signature of the last chain run eagerly
};

namespace {

}  // namespace
extern "C" void prrtc_internal_set_error(const char* msg);
extern "C" int prrtc_internal_env_view(const prrtc_env* env, EnvView* view, int* device);
namespace {

int mlp_fail(int code, const char* msg) {
  prrtc_internal_set_error(msg);
  return code;
}

#define MCK(call)                                                           \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) return mlp_fail(PRRTC_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
int grow(T** p, size_t* cap, size_t need) {
  if (*p && *cap >= need) return PRRTC_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, std::max<size_t>(need, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return mlp_fail(PRRTC_ERR_OOM, "device allocation failed");
  }
  *cap = need;
  return PRRTC_OK;
}

void free_scratch(prrtc_proposal* p) {
  cudaFree(p->x16); cudaFree(p->xT); cudaFree(p->d16); cudaFree(p->dT);
  cudaFree(p->out32); cudaFree(p->d32); cudaFree(p->dh32); cudaFree(p->loss);
  for (int l = 0; l < 3; ++l) {
    cudaFree(p->h16[l]); cudaFree(p->hT[l]); cudaFree(p->z16[l]); cudaFree(p->zT[l]); cudaFree(p->z32[l]);
    p->h16[l] = p->hT[l] = p->z16[l] = p->zT[l] = nullptr;
    p->z32[l] = nullptr;
  }
  p->x16 = p->xT = p->d16 = p->dT = nullptr;
  p->out32 = p->d32 = p->dh32 = p->loss = nullptr;
  p->cap = 0;
}

// Batch scratch for up to `rows` rows (a multiple of 8).
int ensure_scratch(prrtc_proposal* p, int rows) {
  if (p->cap >= rows) return PRRTC_OK;
  free_scratch(p);
  const int P = p->P;
  const int hid[3] = {kHid0, kHid1, kHid2};
  bool ok = cudaMalloc(&p->x16, (size_t)rows * kIn * 2) == cudaSuccess &&
            cudaMalloc(&p->xT, (size_t)rows * kIn * 2) == cudaSuccess &&
            cudaMalloc(&p->d16, (size_t)rows * P * 2) == cudaSuccess &&
            cudaMalloc(&p->dT, (size_t)rows * P * 2) == cudaSuccess &&
            cudaMalloc(&p->out32, (size_t)rows * P * 4) == cudaSuccess &&
            cudaMalloc(&p->d32, (size_t)rows * P * 4) == cudaSuccess &&
            cudaMalloc(&p->dh32, (size_t)rows * kHid0 * 4) == cudaSuccess &&
            cudaMalloc(&p->loss, 4) == cudaSuccess;
  for (int l = 0; l < 3 && ok; ++l)
    ok = cudaMalloc(&p->h16[l], (size_t)rows * hid[l] * 2) == cudaSuccess &&
         cudaMalloc(&p->hT[l], (size_t)rows * hid[l] * 2) == cudaSuccess &&
         cudaMalloc(&p->z16[l], (size_t)rows * hid[l] * 2) == cudaSuccess &&
         cudaMalloc(&p->zT[l], (size_t)rows * hid[l] * 2) == cudaSuccess &&
         cudaMalloc(&p->z32[l], (size_t)rows * hid[l] * 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_scratch(p);
    return mlp_fail(PRRTC_ERR_OOM, "scratch allocation failed");
  }
  p->cap = rows;
  return PRRTC_OK;
}

int transpose(const bf16* in, int rows, int cols, bf16* out, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  transpose_kernel<<<grid, block, 0, s>>>(in, rows, cols, out);
  return cudaGetLastError() == cudaSuccess ? PRRTC_OK : PRRTC_ERR_CUDA;
}

// BF16 copies of the weights and their transposes from the FP32 masters.
int refresh_weights(prrtc_proposal* p) {
  for (int l = 0; l < 4; ++l) {
    const size_t n = (size_t)p->out_dim[l] * p->in_dim[l];
    to_bf16_kernel<<<blocks_for(n), 256, 0, p->stream>>>(p->master + p->w_off[l], n, p->w16[l]);
    int rc = transpose(p->w16[l], p->out_dim[l], p->in_dim[l], p->w16t[l], p->stream);
    if (rc) return rc;
    if (l > 0 && (rc = mlp_tile_weights(p->w16[l], p->out_dim[l], p->in_dim[l], p->wtile[l - 1], p->stream)))
      return rc;
  }
  return cudaGetLastError() == cudaSuccess ? PRRTC_OK : PRRTC_ERR_CUDA;
}

int gemm(const bf16* a, const bf16* b, int M, int N, int K, const float* bias, int relu, float* c32, bf16* c16,
         cudaStream_t s) {
  return gemm_bf16(a, b, M, N, K, bias, relu, c32, N, c16, N, s);
}

// Forward of `rows` feature rows already in x16 (or, from layer 1 on, first
// activations already in h16[0]); out32 receives the head.
int forward_rows(prrtc_proposal* p, int rows, int first_layer = 0) {
  const cudaStream_t s = p->stream;
  int rc;
  const bf16* in = first_layer == 0 ? p->x16 : p->h16[first_layer - 1];
  for (int l = first_layer; l < 3; ++l) {
    if ((rc = gemm(in, p->w16[l], rows, p->out_dim[l], p->in_dim[l], p->master + p->b_off[l], 1, nullptr, p->h16[l],
                   s)))
      return rc;
    in = p->h16[l];
  }
  return gemm(in, p->w16[3], rows, p->P, p->in_dim[3], p->master + p->b_off[3], 0, p->out32, nullptr, s);
}

// Gradients of the mean NLL for `B` samples (rows padded to `rows`) into p->grad.
int backward_rows(prrtc_proposal* p, int B, int rows) {
  const cudaStream_t s = p->stream;
  const int P = p->P;
  int rc;
  // head: dW4 = dout^T h3, db4 = colsum(dout), dh3 = dout W4
  if ((rc = transpose(p->d16, rows, P, p->dT, s))) return rc;
  const bf16* hprev[4] = {p->x16, p->h16[0], p->h16[1], p->h16[2]};
  bf16* hprevT[4] = {p->xT, p->hT[0], p->hT[1], p->hT[2]};
  const bf16* dz16 = p->d16;
  const bf16* dzT = p->dT;
  const float* dz32 = p->d32;
  for (int l = 3; l >= 0; --l) {
    const int in = p->in_dim[l], out = p->out_dim[l];
    if ((rc = transpose(hprev[l], rows, in, hprevT[l], s))) return rc;
    // dW_l [out x in] = dZ^T [out x rows] * (H^T [in x rows])^T
    if ((rc = gemm(dzT, hprevT[l], out, in, rows, nullptr, 0, p->grad + p->w_off[l], nullptr, s))) return rc;
    colsum_kernel<<<(out + 127) / 128, 128, 0, s>>>(dz32, rows, out, p->grad + p->b_off[l]);
    if (l == 0) break;
    // dH_{l-1} [rows x in] = dZ [rows x out] * (W^T [in x out])^T
    if ((rc = gemm(dz16, p->w16t[l], rows, in, out, nullptr, 0, p->dh32, nullptr, s))) return rc;
    const size_t n = (size_t)rows * in;
    relu_back_kernel<<<blocks_for(n), 256, 0, s>>>(p->dh32, p->h16[l - 1], n, p->z32[l - 1], p->z16[l - 1]);
    if ((rc = transpose(p->z16[l - 1], rows, in, p->zT[l - 1], s))) return rc;
    dz16 = p->z16[l - 1];
    dzT = p->zT[l - 1];
    dz32 = p->z32[l - 1];
  }
  (void)B;
  return cudaGetLastError() == cudaSuccess ? PRRTC_OK : PRRTC_ERR_CUDA;
}

int upload_samples(prrtc_proposal* p, const uint8_t* occ, int n_occ, const float* qs, const float* qg,
                   const float* tgt, int n) {
  int rc;
  if ((rc = grow(&p->occ, &p->occ_cap, (size_t)n_occ * kVox))) return rc;
  if ((rc = grow(&p->qs, &p->q_cap, (size_t)n * p->dof))) return rc;
  if ((rc = grow(&p->qg, &p->qg_cap, (size_t)n * p->dof))) return rc;
  if (tgt && (rc = grow(&p->tgt, &p->tgt_cap, (size_t)n * p->dof))) return rc;
  MCK(cudaMemcpyAsync(p->occ, occ, (size_t)n_occ * kVox, cudaMemcpyHostToDevice, p->stream));
  MCK(cudaMemcpyAsync(p->qs, qs, (size_t)n * p->dof * 4, cudaMemcpyHostToDevice, p->stream));
  MCK(cudaMemcpyAsync(p->qg, qg, (size_t)n * p->dof * 4, cudaMemcpyHostToDevice, p->stream));
  if (tgt) MCK(cudaMemcpyAsync(p->tgt, tgt, (size_t)n * p->dof * 4, cudaMemcpyHostToDevice, p->stream));
  return PRRTC_OK;
}

int check_gemm_error() {
  const int e = gemm_take_error();
  return e ? mlp_fail(e, "a tensor-core kernel wait gave up") : PRRTC_OK;
}

// FNV-1a over the values that a captured inference chain bakes in.
uint64_t chain_signature(std::initializer_list<uint64_t> vals) {
  uint64_t h = 1469598103934665603ull;
  for (uint64_t v : vals) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xffu;
      h *= 1099511628211ull;
    }
  }
  return h;
}

// Kernel chain of one inference batch on p->stream: occupancy grids of the
// U distinct environments, the occupancy part of the first layer once per
// environment, then one fused launch for the rest of the network and the
// mixture parameters in the planner's rows.
int enqueue_inference(prrtc_proposal* p, const EnvView* d_envs, int U, const int* d_row_env, float* const* d_rows,
                      const float* d_qs, const float* d_qg, int B, int rows) {
  const cudaStream_t s = p->stream;
  MCK(cudaMemsetAsync(p->inf_occ, 0, (size_t)U * kVox, s));
  occupancy_scatter_kernel<<<dim3(4, U), 256, 0, s>>>(d_envs, p->inf_occ);
  int rc;
  if (U <= kGemvMaxEnvs) {
    l1_occ_gemv_kernel<<<kHid0 / 8, 256, 0, s>>>(p->inf_occ, U, p->w16[0], p->h1o32);
  } else {
    occ_bf16_kernel<<<U, 256, 0, s>>>(p->inf_occ, p->xo16);
    if ((rc = gemm_bf16_ld(p->xo16, kVox, p->w16[0], kIn, U, kHid0, kVox, nullptr, 0, p->h1o32, kHid0, nullptr, 0, s,
                           0)))
      return rc;
  }
  MCK(cudaGetLastError());
  MlpInferArgs a{};
  a.rows = rows;
  a.B = B;
  a.dof = p->dof;
  a.h0 = kHid0;
  a.h1 = kHid1;
  a.h2 = kHid2;
  a.head = p->P;
  a.qpad = kQPad;
  a.h1o = p->h1o32;
  a.row_env = d_row_env;
  a.qs = d_qs;
  a.qg = d_qg;
  a.lo = p->d_lims;
  a.span = p->d_lims + kMaxDof;
  a.wq = p->w16t[0] + (size_t)kVox * kHid0;
  for (int l = 0; l < 3; ++l) {
    a.w[l] = p->wtile[l];
    a.act[l] = p->atile[l];
  }
  for (int l = 0; l < 4; ++l) a.bias[l] = p->master + p->b_off[l];
  a.gmm_rows = d_rows;
  a.mix_k = kK;
  a.gmm_dof = kMaxDof;
  a.logsig_lo = kLogSigMin;
  a.logsig_hi = kLogSigMax;
  return mlp_infer(a, s);
}

}  // namespace

// Implemented in prrtc_gemm.cu: bumped whenever a split-K workspace moves.
namespace prrtc {
uint64_t gemm_workspace_epoch();
}

namespace {

int grow_pinned(unsigned char** p, size_t* cap, size_t need) {
  if (*p && *cap >= need) return PRRTC_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(p, need) != cudaSuccess) {
    cudaGetLastError();
    return mlp_fail(PRRTC_ERR_OOM, "pinned staging allocation failed");
  }
  *cap = need;
  return PRRTC_OK;
}

}  // namespace

// Internal, two halves of one inference batch.  Stage: the host work -- group
// the problems by environment, fill the pinned staging block -- for `B`
// problems whose mixtures go to the device rows gmm_rows[b] (the planner's
// layout).  Submit: the device work -- one staging copy, the kernel chain
// (eager, captured on the second call with the same buffers, replayed after)
// -- ordered before later work on `stream`.  Used by prrtc_plan_batch_learned
// (which stages before its timed device work begins) and the serving loop.
int prrtc_internal_proposal_stage(prrtc_proposal* p, const EnvView* envs, const float* qs_host, const float* qg_host,
                                  int B, float* const* gmm_rows) {
  if (!p || B <= 0) return PRRTC_ERR_INVALID_ARG;
  cudaGetLastError();
  p->pend_ok = false;
  const int rows = (B + 7) & ~7;
  int rc;
  if ((rc = ensure_scratch(p, rows))) return rc;
  // distinct environments of the batch (by their device data) and each
  // problem's index among them
  std::vector<EnvView> uniq;
  std::vector<int> row_env(rows, 0);
  {
    std::map<std::pair<const void*, const void*>, int> seen;
    for (int b = 0; b < B; ++b) {
      const auto key = std::make_pair(static_cast<const void*>(envs[b].data),
                                      static_cast<const void*>(envs[b].esdf.v));
      auto it = seen.find(key);
      if (it == seen.end()) {
        it = seen.emplace(key, (int)uniq.size()).first;
        uniq.push_back(envs[b]);
      }
      row_env[b] = it->second;
    }
  }
  const int U = (int)uniq.size();
  if ((rc = grow(&p->inf_occ, &p->inf_occ_cap, (size_t)U * kVox))) return rc;
  if (U > kGemvMaxEnvs && (rc = grow(&p->xo16, &p->xo16_cap, (size_t)U * kVox))) return rc;
  if ((rc = grow(&p->h1o32, &p->h1o32_cap, (size_t)U * kHid0))) return rc;
  {
    const size_t m_pad = (size_t)((rows + 127) / 128) * 128;
    const int width[3] = {kHid0, kHid1, kHid2};
    for (int l = 0; l < 3; ++l)
      if ((rc = grow(&p->atile[l], &p->atile_cap[l], m_pad * width[l]))) return rc;
  }
  // one staging block: env views | row -> env | planner row pointers | starts | goals
  auto up16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  Pending& q = p->pend;
  q.o_env = 0;
  q.o_map = up16(q.o_env + (size_t)U * sizeof(EnvView));
  q.o_rows = up16(q.o_map + (size_t)rows * sizeof(int));
  q.o_qs = up16(q.o_rows + (size_t)B * sizeof(float*));
  q.o_qg = up16(q.o_qs + (size_t)B * p->dof * sizeof(float));
  q.bytes = up16(q.o_qg + (size_t)B * p->dof * sizeof(float));
  if ((rc = grow_pinned(&p->h_stage, &p->h_stage_cap, q.bytes))) return rc;
  if ((rc = grow(&p->d_stage, &p->d_stage_cap, q.bytes))) return rc;
  // the previous call's copy may still be reading the pinned block
  MCK(cudaStreamSynchronize(p->stream));
  std::memcpy(p->h_stage + q.o_env, uniq.data(), (size_t)U * sizeof(EnvView));
  std::memcpy(p->h_stage + q.o_map, row_env.data(), (size_t)rows * sizeof(int));
  std::memcpy(p->h_stage + q.o_rows, gmm_rows, (size_t)B * sizeof(float*));
  std::memcpy(p->h_stage + q.o_qs, qs_host, (size_t)B * p->dof * sizeof(float));
  std::memcpy(p->h_stage + q.o_qg, qg_host, (size_t)B * p->dof * sizeof(float));
  q.B = B;
  q.rows = rows;
  q.U = U;
  p->last_infer_B = B;
  q.sig = chain_signature(
      {(uint64_t)B, (uint64_t)rows, (uint64_t)U, (uint64_t)(uintptr_t)p->xo16,
       (uint64_t)(uintptr_t)p->h1o32, (uint64_t)(uintptr_t)p->w16t[0], (uint64_t)(uintptr_t)p->atile[0],
       (uint64_t)(uintptr_t)p->atile[1], (uint64_t)(uintptr_t)p->atile[2], (uint64_t)(uintptr_t)p->wtile[0],
       (uint64_t)(uintptr_t)p->wtile[1], (uint64_t)(uintptr_t)p->wtile[2],
       (uint64_t)(uintptr_t)p->d_stage, (uint64_t)(uintptr_t)p->inf_occ,
       (uint64_t)(uintptr_t)p->x16, (uint64_t)(uintptr_t)p->h16[0], (uint64_t)(uintptr_t)p->h16[1],
       (uint64_t)(uintptr_t)p->h16[2], (uint64_t)(uintptr_t)p->out32, (uint64_t)(uintptr_t)p->w16[0],
       (uint64_t)(uintptr_t)p->w16[1], (uint64_t)(uintptr_t)p->w16[2], (uint64_t)(uintptr_t)p->w16[3],
       (uint64_t)(uintptr_t)p->master, (uint64_t)(uintptr_t)p->d_lims, gemm_workspace_epoch()});
  p->pend_ok = true;
  return PRRTC_OK;
}

int prrtc_internal_proposal_submit(prrtc_proposal* p, cudaStream_t stream) {
  if (!p || !p->pend_ok) return PRRTC_ERR_INVALID_ARG;
  p->pend_ok = false;
  const Pending& q = p->pend;
  int rc;
  MCK(cudaEventRecord(p->inf_ev[0], p->stream));
  MCK(cudaMemcpyAsync(p->d_stage, p->h_stage, q.bytes, cudaMemcpyHostToDevice, p->stream));
  const EnvView* d_envs = reinterpret_cast<const EnvView*>(p->d_stage + q.o_env);
  const int* d_row_env = reinterpret_cast<const int*>(p->d_stage + q.o_map);
  float* const* d_rows = reinterpret_cast<float* const*>(p->d_stage + q.o_rows);
  const float* d_qs = reinterpret_cast<const float*>(p->d_stage + q.o_qs);
  const float* d_qg = reinterpret_cast<const float*>(p->d_stage + q.o_qg);
  if (p->infer_exec && p->infer_sig == q.sig) {
    MCK(cudaGraphLaunch(p->infer_exec, p->stream));
  } else if (p->seen_sig == q.sig) {
    // second call with the same buffers: capture the chain (no allocation can
    // happen inside it now) and replay it from here on
    if (p->infer_exec) {
      cudaGraphExecDestroy(p->infer_exec);
      p->infer_exec = nullptr;
    }
    MCK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_inference(p, d_envs, q.U, d_row_env, d_rows, d_qs, d_qg, q.B, q.rows);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(p->stream, &graph);
    if (rc || ce != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : mlp_fail(PRRTC_ERR_CUDA, "inference capture failed");
    }
    const cudaError_t ie = cudaGraphInstantiate(&p->infer_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      p->infer_exec = nullptr;
      return mlp_fail(PRRTC_ERR_CUDA, "inference graph instantiation failed");
    }
    p->infer_sig = q.sig;
    MCK(cudaGraphLaunch(p->infer_exec, p->stream));
  } else {
    if ((rc = enqueue_inference(p, d_envs, q.U, d_row_env, d_rows, d_qs, d_qg, q.B, q.rows))) return rc;
    p->seen_sig = q.sig;
  }
  MCK(cudaEventRecord(p->inf_ev[1], p->stream));
  // the planner runs on another stream: order it after this work
  MCK(cudaEventRecord(p->done, p->stream));
  MCK(cudaStreamWaitEvent(stream, p->done, 0));
  p->inf_timed = true;
  return PRRTC_OK;
}

int prrtc_internal_proposal_mixtures(prrtc_proposal* p, const EnvView* envs, const float* qs_host,
                                     const float* qg_host, int B, float* const* gmm_rows, cudaStream_t stream) {
  const int rc = prrtc_internal_proposal_stage(p, envs, qs_host, qg_host, B, gmm_rows);
  return rc ? rc : prrtc_internal_proposal_submit(p, stream);
}

// Device time of the last submitted inference (staging copy and chain), ms;
// waits for it.  0 when none was submitted since the last query.
float prrtc_internal_proposal_infer_ms(prrtc_proposal* p) {
  if (!p || !p->inf_timed) return 0.f;
  p->inf_timed = false;
  float ms = 0.f;
  if (cudaEventSynchronize(p->inf_ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(&ms, p->inf_ev[0], p->inf_ev[1]) != cudaSuccess) {
    cudaGetLastError();
    return 0.f;
  }
  return ms;
}

extern "C" {

int prrtc_proposal_create(int32_t dof, const float* lower, const float* upper, const float* params,
                          prrtc_proposal** out) {
  cudaGetLastError();  // start from a clean error state
  if (!out || dof < 1 || dof > kMaxDof || !lower || !upper) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  *out = nullptr;
  int dev = -1, count = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
    return mlp_fail(PRRTC_ERR_NO_DEVICE, "no CUDA device");
  for (int j = 0; j < dof; ++j)
    if (!(upper[j] > lower[j])) return mlp_fail(PRRTC_ERR_INVALID_ARG, "joint limits must have upper > lower");
  if (mlp_check_shapes(kHid0, kHid1, kHid2, head_pad(dof))) return mlp_fail(PRRTC_ERR_UNSUPPORTED, "layer widths");
  prrtc_proposal* p = new prrtc_proposal();
  p->device = dev;
  p->dof = dof;
  p->P = head_pad(dof);
  const int dims[5] = {kIn, kHid0, kHid1, kHid2, p->P};
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    p->in_dim[l] = dims[l];
    p->out_dim[l] = dims[l + 1];
    p->w_off[l] = off;
    off += (size_t)dims[l + 1] * dims[l];
    p->b_off[l] = off;
    off += dims[l + 1];
  }
  p->n_params = off;
  for (int j = 0; j < kMaxDof; ++j) {
    p->lo[j] = j < dof ? lower[j] : 0.f;
    p->span[j] = j < dof ? upper[j] - lower[j] : 1.f;
  }
  bool ok = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreate(&p->inf_ev[0]) == cudaSuccess && cudaEventCreate(&p->inf_ev[1]) == cudaSuccess &&
            cudaMalloc(&p->master, off * 4) == cudaSuccess && cudaMalloc(&p->grad, off * 4) == cudaSuccess &&
            cudaMalloc(&p->m, off * 4) == cudaSuccess && cudaMalloc(&p->v, off * 4) == cudaSuccess &&
            cudaMalloc(&p->d_lims, 2 * kMaxDof * 4) == cudaSuccess;
  for (int l = 0; l < 4 && ok; ++l)
    ok = cudaMalloc(&p->w16[l], (size_t)dims[l + 1] * dims[l] * 2) == cudaSuccess &&
         cudaMalloc(&p->w16t[l], (size_t)dims[l + 1] * dims[l] * 2) == cudaSuccess &&
         (l == 0 || cudaMalloc(&p->wtile[l - 1], (size_t)dims[l + 1] * dims[l] * 2) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    prrtc_proposal_destroy(p);
    return mlp_fail(PRRTC_ERR_OOM, "proposal allocation failed");
  }
  float lims[2 * kMaxDof];
  std::memcpy(lims, p->lo, sizeof(p->lo));
  std::memcpy(lims + kMaxDof, p->span, sizeof(p->span));
  bool ok2 = cudaMemcpy(p->d_lims, lims, sizeof(lims), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(p->m, 0, off * 4) == cudaSuccess && cudaMemset(p->v, 0, off * 4) == cudaSuccess &&
             cudaMemset(p->grad, 0, off * 4) == cudaSuccess &&
             (params ? cudaMemcpy(p->master, params, off * 4, cudaMemcpyHostToDevice)
                     : cudaMemset(p->master, 0, off * 4)) == cudaSuccess;
  if (!ok2 || refresh_weights(p) != PRRTC_OK || cudaStreamSynchronize(p->stream) != cudaSuccess) {
    prrtc_proposal_destroy(p);
    return mlp_fail(PRRTC_ERR_CUDA, "proposal initialisation failed");
  }
  *out = p;
  return PRRTC_OK;
}

void prrtc_proposal_destroy(prrtc_proposal* p) {
  if (!p) return;
  free_scratch(p);
  cudaFree(p->master); cudaFree(p->grad); cudaFree(p->m); cudaFree(p->v); cudaFree(p->d_lims);
  for (int l = 0; l < 4; ++l) {
    cudaFree(p->w16[l]);
    cudaFree(p->w16t[l]);
    if (l > 0) cudaFree(p->wtile[l - 1]);
  }
  cudaFree(p->occ); cudaFree(p->qs); cudaFree(p->qg); cudaFree(p->tgt); cudaFree(p->scene_of); cudaFree(p->rows);
  cudaFree(p->envs); cudaFree(p->gmm_rows);
  cudaFree(p->d_stage); cudaFree(p->inf_occ);
  cudaFree(p->xo16); cudaFree(p->h1o32);
  for (bf16* t : p->atile) cudaFree(t);
  if (p->h_stage) cudaFreeHost(p->h_stage);
  if (p->infer_exec) cudaGraphExecDestroy(p->infer_exec);
  if (p->done) cudaEventDestroy(p->done);
  for (cudaEvent_t e : p->inf_ev)
    if (e) cudaEventDestroy(e);
  if (p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

int prrtc_proposal_info(const prrtc_proposal* p, int32_t* dof, int32_t* head, int64_t* n_params, int32_t* step) {
  if (!p) return mlp_fail(PRRTC_ERR_INVALID_ARG, "null proposal");
  if (dof) *dof = p->dof;
  if (head) *head = p->P;
  if (n_params) *n_params = (int64_t)p->n_params;
  if (step) *step = p->step;
  return PRRTC_OK;
}

int prrtc_proposal_get_params(const prrtc_proposal* p, float* params, float* grads) {
  if (!p) return mlp_fail(PRRTC_ERR_INVALID_ARG, "null proposal");
  if (params) MCK(cudaMemcpy(params, p->master, p->n_params * 4, cudaMemcpyDeviceToHost));
  if (grads) MCK(cudaMemcpy(grads, p->grad, p->n_params * 4, cudaMemcpyDeviceToHost));
  return PRRTC_OK;
}

int prrtc_proposal_forward(prrtc_proposal* p, const uint8_t* occ, const float* q_start, const float* q_goal,
                           int32_t B, float* out) {
  cudaGetLastError();  // start from a clean error state
  if (!p || !occ || !q_start || !q_goal || !out || B < 1) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  const int rows = (B + 7) & ~7;
  int rc;
  if ((rc = ensure_scratch(p, rows))) return rc;
  if ((rc = upload_samples(p, occ, B, q_start, q_goal, nullptr, B))) return rc;
  features_kernel<<<rows, 256, 0, p->stream>>>(p->occ, nullptr, nullptr, p->qs, p->qg, p->d_lims, p->d_lims + kMaxDof,
                                               B, p->dof, p->x16);
  if ((rc = forward_rows(p, rows))) return rc;
  MCK(cudaMemcpyAsync(out, p->out32, (size_t)B * p->P * 4, cudaMemcpyDeviceToHost, p->stream));
  MCK(cudaStreamSynchronize(p->stream));
  return check_gemm_error();
}

namespace {

// BF16 device rows [n x width] (row stride `ld` elements) -> FP32 host rows.
int bf16_rows_to_host(const bf16* d, int n, int width, int ld, float* out, cudaStream_t s) {
  if (!out) return PRRTC_OK;
  std::vector<uint16_t> raw((size_t)n * ld);
  MCK(cudaMemcpyAsync(raw.data(), d, raw.size() * 2, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < width; ++c) {
      const uint32_t bits = (uint32_t)raw[(size_t)r * ld + c] << 16;
      std::memcpy(out + (size_t)r * width + c, &bits, 4);
    }
  return PRRTC_OK;
}

}  // namespace

int prrtc_proposal_forward_layers(prrtc_proposal* p, const uint8_t* occ, const float* q_start, const float* q_goal,
                                  int32_t B, float* x, float* h1, float* h2, float* h3, float* out) {
  cudaGetLastError();
  if (!p || !occ || !q_start || !q_goal || B < 1) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  const int rows = (B + 7) & ~7;
  int rc;
  if ((rc = ensure_scratch(p, rows))) return rc;
  if ((rc = upload_samples(p, occ, B, q_start, q_goal, nullptr, B))) return rc;
  features_kernel<<<rows, 256, 0, p->stream>>>(p->occ, nullptr, nullptr, p->qs, p->qg, p->d_lims, p->d_lims + kMaxDof,
                                               B, p->dof, p->x16);
  if ((rc = forward_rows(p, rows))) return rc;
  if ((rc = check_gemm_error())) return rc;
  if ((rc = bf16_rows_to_host(p->x16, B, kIn, kIn, x, p->stream))) return rc;
  float* hs[3] = {h1, h2, h3};
  for (int l = 0; l < 3; ++l)
    if ((rc = bf16_rows_to_host(p->h16[l], B, p->out_dim[l], p->out_dim[l], hs[l], p->stream))) return rc;
  if (out) {
    MCK(cudaMemcpyAsync(out, p->out32, (size_t)B * p->P * 4, cudaMemcpyDeviceToHost, p->stream));
    MCK(cudaStreamSynchronize(p->stream));
  }
  return PRRTC_OK;
}

int prrtc_proposal_inference_layers(prrtc_proposal* p, int32_t B, float* h1, float* h2, float* h3) {
  if (!p || B < 1 || B > p->last_infer_B) return mlp_fail(PRRTC_ERR_INVALID_ARG, "no inference batch of that size");
  MCK(cudaStreamSynchronize(p->stream));
  const int width[3] = {kHid0, kHid1, kHid2};
  float* outs[3] = {h1, h2, h3};
  const int tiles = (B + 127) / 128;
  for (int l = 0; l < 3; ++l) {
    if (!outs[l]) continue;
    // [row tile][64-column k-block] blocks of 128 rows x 128 bytes, 16-byte
    // unit u of row i stored at unit u ^ (i % 8)
    const size_t elems = (size_t)tiles * 128 * width[l];
    std::vector<uint16_t> raw(elems);
    MCK(cudaMemcpy(raw.data(), p->atile[l], elems * 2, cudaMemcpyDeviceToHost));
    const int kbs = width[l] / 64;
    for (int r = 0; r < B; ++r) {
      const int mt = r / 128, i = r % 128;
      for (int c = 0; c < width[l]; ++c) {
        const int kb = c / 64, cc = c % 64;
        const size_t byte = ((size_t)mt * kbs + kb) * (128 * 128) + (size_t)i * 128 +
                            ((size_t)((cc >> 3) ^ (i & 7)) << 4) + ((size_t)(cc & 7) << 1);
        const uint32_t bits = (uint32_t)raw[byte / 2] << 16;
        std::memcpy(outs[l] + (size_t)r * width[l] + c, &bits, 4);
      }
    }
  }
  return PRRTC_OK;
}

// One step on a batch: gradients into the proposal (readable with
// prrtc_proposal_get_params) and, when lr > 0, an Adam update.
static int step_on_rows(prrtc_proposal* p, const int* scene_of, const int* rows_dev, int B, float lr,
                        float* loss_host) {
  const int rows = (B + 7) & ~7;
  int rc;
  const cudaStream_t s = p->stream;
  features_kernel<<<rows, 256, 0, s>>>(p->occ, scene_of, rows_dev, p->qs, p->qg, p->d_lims, p->d_lims + kMaxDof, B,
                                       p->dof, p->x16);
  if ((rc = forward_rows(p, rows))) return rc;
  MCK(cudaMemsetAsync(p->d32, 0, (size_t)rows * p->P * 4, s));
  MCK(cudaMemsetAsync(p->d16, 0, (size_t)rows * p->P * 2, s));
  MCK(cudaMemsetAsync(p->loss, 0, 4, s));
  mixture_loss_kernel<<<(B * 32 + 255) / 256, 256, 0, s>>>(p->out32, p->P, p->tgt, rows_dev, p->d_lims,
                                                            p->d_lims + kMaxDof, B, p->dof, 1.f / (float)B, p->d32,
                                                            p->d16, p->loss);
  if ((rc = backward_rows(p, B, rows))) return rc;
  if (lr > 0.f) {
    p->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)p->step)), c2 = 1.f / (1.f - std::pow(b2, (float)p->step));
    adam_kernel<<<blocks_for(p->n_params), 256, 0, s>>>(p->master, p->grad, p->m, p->v, p->n_params, lr, b1, b2,
                                                         1e-8f, c1, c2);
    if ((rc = refresh_weights(p))) return rc;
  }
  if (loss_host) MCK(cudaMemcpyAsync(loss_host, p->loss, 4, cudaMemcpyDeviceToHost, s));
  return cudaGetLastError() == cudaSuccess ? PRRTC_OK : PRRTC_ERR_CUDA;
}

static int step_on_rows_direct(prrtc_proposal* p, int B, float* loss) {
  return step_on_rows(p, nullptr, nullptr, B, 0.f, loss);
}

int prrtc_proposal_grads(prrtc_proposal* p, const uint8_t* occ, const float* q_start, const float* q_goal,
                         const float* target, int32_t B, float* loss) {
  cudaGetLastError();  // start from a clean error state
  if (!p || !occ || !q_start || !q_goal || !target || B < 1) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  const int rows = (B + 7) & ~7;
  int rc;
  if ((rc = ensure_scratch(p, rows))) return rc;
  if ((rc = upload_samples(p, occ, B, q_start, q_goal, target, B))) return rc;
  if ((rc = step_on_rows_direct(p, B, loss))) return rc;
  MCK(cudaStreamSynchronize(p->stream));
  return check_gemm_error();
}

int prrtc_proposal_train(prrtc_proposal* p, const uint8_t* occ, int32_t n_scenes, const int32_t* scene_of,
                         const float* q_start, const float* q_goal, const float* target, int32_t n_samples,
                         int32_t batch, int32_t steps, float lr, uint64_t seed, float* losses) {
  cudaGetLastError();  // start from a clean error state
  if (!p || !occ || n_scenes < 1 || !scene_of || !q_start || !q_goal || !target || n_samples < 1 || batch < 1 ||
      steps < 0 || !(lr > 0.f))
    return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  for (int i = 0; i < n_samples; ++i)
    if (scene_of[i] < 0 || scene_of[i] >= n_scenes) return mlp_fail(PRRTC_ERR_INVALID_ARG, "scene index out of range");
  const int B = std::min(batch, n_samples);
  const int rows = (B + 7) & ~7;
  int rc;
  if ((rc = ensure_scratch(p, rows))) return rc;
  if ((rc = upload_samples(p, occ, n_scenes, q_start, q_goal, target, n_samples))) return rc;
  if ((rc = grow(&p->scene_of, &p->scene_cap, (size_t)n_samples))) return rc;
  MCK(cudaMemcpyAsync(p->scene_of, scene_of, (size_t)n_samples * 4, cudaMemcpyHostToDevice, p->stream));
  // sample order: a seeded permutation per epoch, consumed batch by batch
  std::vector<int> order(n_samples);
  std::mt19937_64 rng(seed);
  std::vector<int> idx((size_t)steps * B);
  size_t pos = order.size();
  for (size_t k = 0; k < idx.size(); ++k) {
    if (pos == order.size()) {
      for (int i = 0; i < n_samples; ++i) order[i] = i;
      std::shuffle(order.begin(), order.end(), rng);
      pos = 0;
    }
    idx[k] = order[pos++];
  }
  if ((rc = grow(&p->rows, &p->rows_cap, std::max<size_t>(idx.size(), 1)))) return rc;
  if (!idx.empty())
    MCK(cudaMemcpyAsync(p->rows, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, p->stream));
  std::vector<float> host_loss(std::max(steps, 1));
  for (int t = 0; t < steps; ++t)
    if ((rc = step_on_rows(p, p->scene_of, p->rows + (size_t)t * B, B, lr, losses ? &host_loss[t] : nullptr)))
      return rc;
  MCK(cudaStreamSynchronize(p->stream));
  if (losses)
    for (int t = 0; t < steps; ++t) losses[t] = host_loss[t];
  return check_gemm_error();
}

int prrtc_occupancy(const prrtc_env* env, uint8_t* out) {
  if (!env || !out) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  EnvView ev{};
  int dev = -1;
  int rc = prrtc_internal_env_view(env, &ev, &dev);
  if (rc) return rc;
  uint8_t* d = nullptr;
  EnvView* dv = nullptr;
  MCK(cudaMalloc(&d, kVox));
  if (cudaMalloc(&dv, sizeof(EnvView)) != cudaSuccess) {
    cudaFree(d);
    return mlp_fail(PRRTC_ERR_OOM, "device allocation failed");
  }
  cudaError_t e = cudaMemcpy(dv, &ev, sizeof(EnvView), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d, 0, kVox);
  if (e == cudaSuccess) {
    occupancy_scatter_kernel<<<dim3(4, 1), 256>>>(dv, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d, kVox, cudaMemcpyDeviceToHost);
  cudaFree(d);
  cudaFree(dv);
  if (e != cudaSuccess) return mlp_fail(PRRTC_ERR_CUDA, cudaGetErrorString(e));
  return PRRTC_OK;
}

int prrtc_proposal_mixtures(prrtc_proposal* p, const prrtc_env* const* envs, const float* q_start,
                            const float* q_goal, int32_t B, float* out) {
  cudaGetLastError();
  if (!p || !envs || !q_start || !q_goal || !out || B < 1) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  const int dof = p->dof;
  for (size_t i = 0; i < (size_t)B * dof; ++i)
    if (!std::isfinite(q_start[i]) || !std::isfinite(q_goal[i]))
      return mlp_fail(PRRTC_ERR_INVALID_ARG, "non-finite start or goal");
  std::vector<EnvView> views(B);
  for (int b = 0; b < B; ++b) {
    if (!envs[b]) return mlp_fail(PRRTC_ERR_INVALID_ARG, "null environment");
    int dev = -1;
    int rc = prrtc_internal_env_view(envs[b], &views[b], &dev);
    if (rc) return rc;
    if (dev != p->device) return mlp_fail(PRRTC_ERR_INVALID_ARG, "environment on another device");
  }
  float* d = nullptr;
  MCK(cudaMalloc(&d, (size_t)B * kGmmStride * sizeof(float)));
  std::vector<float*> rows(B);
  for (int b = 0; b < B; ++b) rows[b] = d + (size_t)b * kGmmStride;
  int rc = prrtc_internal_proposal_mixtures(p, views.data(), q_start, q_goal, B, rows.data(), p->stream);
  std::vector<float> padded((size_t)B * kGmmStride);
  cudaError_t e = cudaSuccess;
  if (!rc) e = cudaMemcpyAsync(padded.data(), d, padded.size() * sizeof(float), cudaMemcpyDeviceToHost, p->stream);
  if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  cudaFree(d);
  if (rc) return rc;
  if (e != cudaSuccess) return mlp_fail(PRRTC_ERR_CUDA, cudaGetErrorString(e));
  if ((rc = check_gemm_error())) return rc;
  // the planner's padded rows -> [logits | means (8 x dof) | log-sigmas (8 x dof)]
  const int stride = kK + 2 * kK * dof;
  for (int b = 0; b < B; ++b) {
    const float* g = padded.data() + (size_t)b * kGmmStride;
    float* o = out + (size_t)b * stride;
    for (int k = 0; k < kK; ++k) {
      o[k] = g[k];
      for (int j = 0; j < dof; ++j) {
        o[kK + k * dof + j] = g[kK + k * kMaxDof + j];
        o[kK + kK * dof + k * dof + j] = g[kK + kK * kMaxDof + k * kMaxDof + j];
      }
    }
  }
  return PRRTC_OK;
}

// File: "PRRTCMLP" | version | dof | head | n_params | step | lo[16] | span[16]
// | master | m | v  (FP32, little-endian).
int prrtc_proposal_save(const prrtc_proposal* p, const char* path) {
  if (!p || !path) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  std::vector<float> buf(p->n_params * 3);
  MCK(cudaMemcpy(buf.data(), p->master, p->n_params * 4, cudaMemcpyDeviceToHost));
  MCK(cudaMemcpy(buf.data() + p->n_params, p->m, p->n_params * 4, cudaMemcpyDeviceToHost));
  MCK(cudaMemcpy(buf.data() + 2 * p->n_params, p->v, p->n_params * 4, cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return mlp_fail(PRRTC_ERR_INVALID_ARG, "cannot open file");
  const char magic[8] = {'P', 'R', 'R', 'T', 'C', 'M', 'L', 'P'};
  const int64_t hdr[5] = {1, p->dof, p->P, (int64_t)p->n_params, p->step};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, 8, 5, f) == 5 &&
            std::fwrite(p->lo, 4, kMaxDof, f) == (size_t)kMaxDof && std::fwrite(p->span, 4, kMaxDof, f) == (size_t)kMaxDof &&
            std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? PRRTC_OK : mlp_fail(PRRTC_ERR_INVALID_ARG, "write failed");
}

int prrtc_proposal_load(const char* path, prrtc_proposal** out) {
  if (!path || !out) return mlp_fail(PRRTC_ERR_INVALID_ARG, "bad arguments");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return mlp_fail(PRRTC_ERR_INVALID_ARG, "cannot open file");
  char magic[8];
  int64_t hdr[5];
  float lo[kMaxDof], span[kMaxDof];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "PRRTCMLP", 8) == 0 && std::fread(hdr, 8, 5, f) == 5 &&
            hdr[0] == 1 && hdr[1] >= 1 && hdr[1] <= kMaxDof && std::fread(lo, 4, kMaxDof, f) == (size_t)kMaxDof &&
            std::fread(span, 4, kMaxDof, f) == (size_t)kMaxDof;
  if (!ok) {
    std::fclose(f);
    return mlp_fail(PRRTC_ERR_INVALID_ARG, "not a proposal file");
  }
  const int dof = (int)hdr[1];
  float up[kMaxDof];
  for (int j = 0; j < kMaxDof; ++j) up[j] = lo[j] + span[j];
  prrtc_proposal* p = nullptr;
  int rc = prrtc_proposal_create(dof, lo, up, nullptr, &p);
  if (rc) {
    std::fclose(f);
    return rc;
  }
  if ((int64_t)p->n_params != hdr[3] || p->P != hdr[2]) {
    std::fclose(f);
    prrtc_proposal_destroy(p);
    return mlp_fail(PRRTC_ERR_INVALID_ARG, "size mismatch");
  }
  std::vector<float> buf(p->n_params * 3);
  ok = std::fread(buf.data(), 4, buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) {
    prrtc_proposal_destroy(p);
    return mlp_fail(PRRTC_ERR_INVALID_ARG, "truncated file");
  }
  std::memcpy(p->lo, lo, sizeof(lo));
  std::memcpy(p->span, span, sizeof(span));
  float lims[2 * kMaxDof];
  std::memcpy(lims, lo, sizeof(lo));
  std::memcpy(lims + kMaxDof, span, sizeof(span));
  bool ok2 = cudaMemcpy(p->d_lims, lims, sizeof(lims), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(p->master, buf.data(), p->n_params * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(p->m, buf.data() + p->n_params, p->n_params * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(p->v, buf.data() + 2 * p->n_params, p->n_params * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  p->step = (int)hdr[4];
  if (!ok2 || refresh_weights(p) || cudaStreamSynchronize(p->stream) != cudaSuccess) {
    prrtc_proposal_destroy(p);
    return mlp_fail(PRRTC_ERR_CUDA, "upload failed");
  }
  *out = p;
  return PRRTC_OK;
}

}  // extern "C"
