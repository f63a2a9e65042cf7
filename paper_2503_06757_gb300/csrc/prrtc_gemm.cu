// prrtc_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores for the
// learned sampling proposal's dense layers:  C[M,N] = A[M,K] * B[N,K]^T with
// FP32 accumulation in tensor memory, optional bias + ReLU and FP32 / BF16
// outputs.
//
// Persistent kernel, one CTA per SM.  A work unit is one 128 x 256 output tile
// over a range of K (split-K when the tiles alone cannot fill the GPU):
//   warp 0    -- one lane issues TMA loads of the 128 x 64 A and 256 x 64 B
//                tiles (128-byte swizzle) into a 4-stage shared-memory ring;
//   warp 1    -- allocates all 512 TMEM columns (two 256-column
//                accumulators); one lane issues tcgen05.mma (M=128, N=256,
//                K=16, kind::f16) four times per stage, commits each stage
//                back to the producer and each finished unit to the epilogue;
//   warps 2-5 -- read an accumulator with tcgen05.ld (each warp owns one
//                32-lane quarter of TMEM), run the epilogue, and hand the
//                accumulator back, so the epilogue of one unit overlaps the
//                main loop of the next.
// The epilogue stages each 32 x 32 chunk in a swizzled shared-memory tile and
// writes it with a TMA bulk tensor store (the TMA engine clips the matrix
// edges).  With split-K each unit writes its FP32 partial tile to a workspace
// and a second kernel sums the partials in split order (deterministic) and
// applies bias, ReLU and the output conversions.
// Every mbarrier wait is bounded; a wait that gives up records an error, the
// roles stop, and the CTA still frees its tensor memory.
//
// The same file holds the fused inference kernel of the proposal (one launch
// for layers 1 (second half), 2, 3 and the head; see mlp_infer_kernel).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>

#include "prrtc.h"
#include "prrtc_launch.h"

namespace prrtc {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_TILE_BYTES = 32 * 128;   // one 32 x 32 FP32 chunk (or 32 x 32 BF16 in its first half)
constexpr int EPI_BUFS = 2;                 // staging tiles per epilogue warp (double buffered)
// ring | barriers (1 KB) | staging tiles, plus 1 KB for aligning the base
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 1024 + 4 * EPI_BUFS * EPI_TILE_BYTES;
constexpr int THREADS = 192;
constexpr int EPI_WARPS = 4;
constexpr uint32_t TMEM_COLS = 2 * BN;  // two accumulators
constexpr uint32_t kPolls = 1u << 26;
constexpr int kMinKTilesPerSplit = 4;
constexpr int kMaxSplits = 16;

__device__ int g_gemm_error;

struct Epilogue {
  int M, N, K;
  const float* bias;
  int relu;
  int has_c32, has_c16;  // outputs written through the c32 / c16 tensor maps
  int splits;            // > 1: raw partials through the workspace map, rows split * m_pad + row
  int m_tiles, n_tiles, k_tiles;
  int m_pad;             // rows of one split's partial (M rounded up to the tile), so that the
                         // clipped-off rows of an edge tile never reach the next split's rows
};

// Output tensor maps of one launch: workspace (FP32, rows = splits * m_pad),
// FP32 output and BF16 output; boxes of 32 x 32 elements, 128- / 64-byte
// swizzle matching the staging layout below.
struct OutMaps {
  CUtensorMap ws, c32, c16;
};

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// start address, stride between 8-row groups (1024 B), descriptor version 1,
// swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused with 128 B swizzle, K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // 128 B swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity) {
  if (mbar_wait(bar, parity, kPolls)) return true;
  atomicExch(&g_gemm_error, PRRTC_ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Work unit -> tile and K range.  Tiles go in groups of kGroupM row tiles:
// m fastest inside a group, then n, then the next group, so that the tiles in
// flight at once (one per SM) share a slab of A rows and a few B columns that
// stay in L2 instead of sweeping all of A for every column of B.
constexpr int kGroupM = 16;
struct Unit {
  int m0, n0, split, kt0, kt1;
};

__device__ __forceinline__ Unit unit_of(const Epilogue& ep, int u) {
  Unit w;
  const int tile = u / ep.splits;
  w.split = u - tile * ep.splits;
  const int span = kGroupM * ep.n_tiles;
  const int first_m = (tile / span) * kGroupM;
  const int gm = min(ep.m_tiles - first_m, kGroupM);
  const int in = tile - (tile / span) * span;
  w.m0 = (first_m + in % gm) * BM;
  w.n0 = (in / gm) * BN;
  const int base = ep.k_tiles / ep.splits, rem = ep.k_tiles % ep.splits;
  w.kt0 = w.split * base + min(w.split, rem);
  w.kt1 = w.kt0 + base + (w.split < rem ? 1 : 0);
  return w;
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most one committed bulk store still reads shared memory.
__device__ __forceinline__ void bulk_wait_read_le1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Stage one 32 x 32 chunk held one row per lane (lane = row, values v[0..31]
// = columns) into a shared-memory tile laid out as the TMA engine expects
// with the store map's swizzle, then let lane 0 store it with one bulk
// tensor copy.  FP32 rows are 128 bytes (128-byte swizzle: 16-byte unit u of
// row r sits at unit u ^ (r % 8)); BF16 rows are 64 bytes (64-byte swizzle:
// unit u ^ ((r / 2) % 4)).  Each store instruction of the warp touches every
// bank group once, and the TMA engine clips rows and columns outside the
// matrix.  `buf` alternates between the warp's two staging tiles.
__device__ __forceinline__ void stage_and_store(const CUtensorMap* map, unsigned char* tiles, int& buf, bool bf16,
                                                int x, int y, int lane, const float (&f)[32]) {
  unsigned char* tile = tiles + buf * EPI_TILE_BYTES;
  if (lane == 0) bulk_wait_read_le1();  // the store issued from this tile two rounds ago has read it
  __syncwarp();
  if (!bf16) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float4* dst = reinterpret_cast<float4*>(tile + lane * 128 + ((u ^ (lane & 7)) << 4));
      *dst = make_float4(f[4 * u], f[4 * u + 1], f[4 * u + 2], f[4 * u + 3]);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint4 pk;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(f[8 * u], f[8 * u + 1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(f[8 * u + 2], f[8 * u + 3]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(f[8 * u + 4], f[8 * u + 5]);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(f[8 * u + 6], f[8 * u + 7]);
      pk.x = *reinterpret_cast<uint32_t*>(&h0);
      pk.y = *reinterpret_cast<uint32_t*>(&h1);
      pk.z = *reinterpret_cast<uint32_t*>(&h2);
      pk.w = *reinterpret_cast<uint32_t*>(&h3);
      *reinterpret_cast<uint4*>(tile + lane * 64 + ((u ^ ((lane >> 1) & 3)) << 4)) = pk;
    }
  }
  fence_proxy_async_smem();  // make the generic-proxy writes visible to the TMA engine
  __syncwarp();
  if (lane == 0) {
    tma_store_2d(map, tile, x, y);
    bulk_commit();
  }
  buf ^= 1;
}

// Epilogue of one 32 x 32 chunk (rows row0.., columns col0..; lane = row).
__device__ __forceinline__ void store_chunk(const Epilogue& ep, const OutMaps& om, unsigned char* tiles, int& buf,
                                            int split, int row0, int col0, int lane, const uint32_t (&v)[32]) {
  float f[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]);
  if (ep.splits > 1) {  // raw partial; the reduction kernel finishes it
    stage_and_store(&om.ws, tiles, buf, false, col0, split * ep.m_pad + row0, lane, f);
    return;
  }
  if (ep.bias) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (col0 + j < ep.N) f[j] += ep.bias[col0 + j];
  }
  if (ep.relu) {
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = fmaxf(f[j], 0.f);
  }
  if (ep.has_c32) stage_and_store(&om.c32, tiles, buf, false, col0, row0, lane, f);
  if (ep.has_c16) stage_and_store(&om.c16, tiles, buf, true, col0, row0, lane, f);
}

__global__ void __launch_bounds__(THREADS, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ OutMaps om, Epilogue ep) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;    // [2] epilogue -> MMA
  uint64_t* roles_done = acc_empty + 2;  // every warp of the CTA -> TMEM release
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(roles_done + 1);
  unsigned char* epi_tiles = smem + STAGES * STAGE_BYTES + 256 + 768;  // 1024-aligned staging tiles
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_units = ep.m_tiles * ep.n_tiles * ep.splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], EPI_WARPS);
    }
    mbar_init(roles_done, THREADS / 32);
    s_abort = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  // Role loops run on all 32 lanes of a warp (lane 0 waits and issues, the
  // warp reconverges every step), so every warp reaches the final CTA barrier
  // converged.
  if (warp == 0) {
    int it = 0;  // stage counter across units
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const Unit w = unit_of(ep, u);
      for (int kt = w.kt0; kt < w.kt1; ++kt, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        int got = 0;
        if (lane == 0) got = (!*abort_flag && wait_bar(&empty[s], ph ^ 1u)) ? 1 : 0;
        got = __shfl_sync(kFull, got, 0);
        if (!got) {
          if (lane == 0) *abort_flag = 1;
          ok = false;
          break;
        }
        if (lane == 0) {
          unsigned char* a = smem + s * STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
          tma_load_2d(a, &tmA, &full[s], kt * BK, w.m0);
          tma_load_2d(a + A_BYTES, &tmB, &full[s], kt * BK, w.n0);
        }
        __syncwarp();
      }
    }
  } else if (warp == 1) {
    const uint32_t idesc = idesc_bf16(BM, BN);
    int it = 0, i = 0;  // stage counter, local unit counter
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++i) {
      const Unit w = unit_of(ep, u);
      const int acc = i & 1;
      // wait until the epilogue has drained this accumulator (first use passes)
      int got = 0;
      if (lane == 0) got = (!*abort_flag && wait_bar(&acc_empty[acc], ((uint32_t)(i >> 1) & 1u) ^ 1u)) ? 1 : 0;
      got = __shfl_sync(kFull, got, 0);
      if (!got) {
        if (lane == 0) *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)(acc * BN);
      for (int kt = w.kt0; kt < w.kt1; ++kt, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        got = 0;
        if (lane == 0) got = wait_bar(&full[s], ph) ? 1 : 0;
        got = __shfl_sync(kFull, got, 0);
        if (!got) {
          if (lane == 0) *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after();
        if (lane == 0) {
          const uint32_t a = smem_u32(smem + s * STAGE_BYTES);
          const uint32_t b = a + A_BYTES;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            mma_bf16(d, smem_desc(a + 32u * k), smem_desc(b + 32u * k), idesc, (kt > w.kt0 || k > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(&acc_full[acc]);
      __syncwarp();
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    unsigned char* tiles = epi_tiles + (warp - 2) * EPI_BUFS * EPI_TILE_BYTES;
    int buf = 0;
    int i = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++i) {
      const Unit w = unit_of(ep, u);
      const int acc = i & 1;
      int ok = 0;
      if (lane == 0) ok = wait_bar(&acc_full[acc], (uint32_t)(i >> 1) & 1u) ? 1 : 0;
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) {
        if (lane == 0) *abort_flag = 1;
        break;
      }
      fence_after();
      const int row0 = w.m0 + 32 * q;
      for (int c = 0; c < BN; c += 32) {
        uint32_t v[32];
        __syncwarp();
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + c), v);
        const int col0 = w.n0 + c;
        if (row0 < ep.M && col0 < ep.N) store_chunk(ep, om, tiles, buf, w.split, row0, col0, lane, v);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
    }
    if (lane == 0) bulk_wait_all();  // every bulk store of this warp has landed
    __syncwarp();
  }
  // Join: each warp signals that its role is over (its tensor-memory reads
  // have completed); the allocating warp frees tensor memory only after all
  // of them.  If the join times out the memory is still freed: the kernel is
  // ending and the error word is set.
  __syncwarp();
  fence_before();
  if (lane == 0) mbar_arrive(roles_done);
  if (warp == 1) {
    int joined = 0;
    if (lane == 0) joined = wait_bar(roles_done, 0) ? 1 : 0;
    joined = __shfl_sync(kFull, joined, 0);
    (void)joined;
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Sum of the split-K partials (split s at rows s * m_pad ..) in split order,
// then bias, ReLU and outputs; four columns per thread (N is a multiple of 8).
__global__ void splitk_reduce_kernel(const float* __restrict__ ws, int splits, int M, int m_pad, int N,
                                     const float* __restrict__ bias, int relu, float* __restrict__ c32, int ldc32,
                                     __nv_bfloat16* __restrict__ c16, int ldc16) {
  const int n4 = N >> 2;
  const size_t total = (size_t)M * n4;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(t / n4), col = (int)(t % n4) * 4;
    float4 acc = *reinterpret_cast<const float4*>(ws + (size_t)row * N + col);
    for (int s = 1; s < splits; ++s) {
      const float4 p = *reinterpret_cast<const float4*>(ws + ((size_t)s * m_pad + row) * N + col);
      acc.x += p.x;
      acc.y += p.y;
      acc.z += p.z;
      acc.w += p.w;
    }
    if (bias) {
      acc.x += bias[col];
      acc.y += bias[col + 1];
      acc.z += bias[col + 2];
      acc.w += bias[col + 3];
    }
    if (relu) {
      acc.x = fmaxf(acc.x, 0.f);
      acc.y = fmaxf(acc.y, 0.f);
      acc.z = fmaxf(acc.z, 0.f);
      acc.w = fmaxf(acc.w, 0.f);
    }
    if (c32) *reinterpret_cast<float4*>(c32 + (size_t)row * ldc32 + col) = acc;
    if (c16) {
      __nv_bfloat162 h0 = __floats2bfloat162_rn(acc.x, acc.y), h1 = __floats2bfloat162_rn(acc.z, acc.w);
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t*>(&h0);
      pk.y = *reinterpret_cast<uint32_t*>(&h1);
      *reinterpret_cast<uint2*>(c16 + (size_t)row * ldc16 + col) = pk;
    }
  }
}

// ------------------------------------------------------------ fused inference
// The learned proposal's forward pass for planning, after the occupancy part
// of the first layer, in one launch.  A cluster of kIC CTAs owns 128 problem
// rows; CTA r of the cluster owns 1/kIC of every layer's output columns:
//   layer 1 (CUDA cores): h1[:, r-th eighth] = ReLU(b1 + occupancy part of
//            the row's environment + start / goal columns);
//   layers 2, 3, head (tensor cores): the row tile of the previous
//            activations times this CTA's slice of the weights, FP32
//            accumulator in TMEM, bias (+ ReLU) -- or, for the head, the
//            mixture parameters written into the planner's rows.
// Operands live in global memory pre-tiled: one 64-column k-block of 128
// activation rows, or of this CTA's weight rows, is one contiguous block in
// the 128-byte-swizzled layout the MMA reads.  Every CTA of the cluster reads
// the same activation tile and its own weight slice, each with a plain bulk
// copy into its own shared memory (no copy writes into a peer's shared
// memory).  A stage is refilled once this CTA's MMAs have released it.  Each
// layer's writer produces exactly the k-blocks of the next layer's input that
// its columns cover.  Between layers every thread
// of the cluster makes its global writes visible to the async proxy (the next
// layer's bulk copies) and meets the cluster barrier; the barriers sit
// outside the role branches, so every thread meets each one even after a
// bounded mbarrier wait has given up.
constexpr int kIC = 8;
constexpr int kIThreads = 192;
constexpr int kIStages = 4;
constexpr int kIKB = 2;      // 64-column k-blocks per pipeline stage
constexpr int kIBRows = 64;  // most weight rows one CTA takes per layer
constexpr int kIStageBytes = kIKB * (A_BYTES + kIBRows * BK * 2);  // A tiles, then B tiles
constexpr int kIQMax = 32;   // start + goal inputs
constexpr int kIL0Cols = 128;
constexpr int kIBiasMax = kIL0Cols + 3 * kIBRows;  // this CTA's bias slices of all four layers
// ring (whose first bytes hold layer 1's inputs and weights until the ring's
// first use) | barriers | bias slices and env rows, plus alignment
constexpr int kISmemBytes = kIStages * kIStageBytes + 1024 + kIBiasMax * 4 + BM * 4 + 1024;
static_assert((BM * kIQMax + kIQMax * kIL0Cols) * 4 <= kIStages * kIStageBytes, "layer-1 scratch fits the ring");
constexpr uint32_t kITmemCols = 256;

// Byte offset of element (i, c) inside one k-block tile (rows of 64 BF16 =
// 128 bytes; 16-byte unit u of row i stored at unit u ^ (i % 8)), the layout
// a TMA load with 128-byte swizzle would produce and the MMA descriptors read.
__host__ __device__ __forceinline__ uint32_t tile_off(int i, int c) {
  return (uint32_t)i * 128u + ((((uint32_t)c >> 3) ^ ((uint32_t)i & 7u)) << 4) + (((uint32_t)c & 7u) << 1);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Global writes of this thread -> visible to the cluster's async-proxy reads
// after the barrier; every thread of the cluster calls it.
__device__ __forceinline__ void cluster_publish() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Weight matrix [N x K] (BF16, row-major) -> tiles [kIC slices][K/64 k-blocks]
// of N/kIC rows each, in the tile layout above.
__global__ void tile_weights_kernel(const __nv_bfloat16* __restrict__ w, int N, int K, __nv_bfloat16* __restrict__ out) {
  const int nc = N / kIC, kts = K / BK;
  const size_t total = (size_t)N * K;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(t / K), k = (int)(t % K);
    const int r = n / nc, i = n % nc, kt = k / BK, c = k % BK;
    unsigned char* tile = reinterpret_cast<unsigned char*>(out) + ((size_t)r * kts + kt) * (size_t)nc * 128;
    *reinterpret_cast<__nv_bfloat16*>(tile + tile_off(i, c)) = w[t];
  }
}

__global__ void __cluster_dims__(kIC, 1, 1) __launch_bounds__(kIThreads, 1)
    mlp_infer_kernel(const MlpInferArgs args) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kIStages * kIStageBytes);
  uint64_t* empty = full + kIStages;
  uint64_t* acc_full = empty + kIStages;  // [3] MMA -> epilogue, once per layer
  uint64_t* roles_done = acc_full + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(roles_done + 1);
  float* s_x = reinterpret_cast<float*>(smem);                                  // [BM][kIQMax], layer 1 only
  float* s_w = s_x + BM * kIQMax;                                               // [kIQMax][kIL0Cols], layer 1 only
  float* s_b = reinterpret_cast<float*>(smem + kIStages * kIStageBytes + 1024);  // [kIBiasMax] bias slices
  int* s_e = reinterpret_cast<int*>(s_b + kIBiasMax);                           // [BM]
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const int r = (int)rank;
  const int mt = (int)(blockIdx.x / kIC), m0 = mt * BM;
  const int dof = args.dof, nq = 2 * dof;
  const int n_out[3] = {args.h1, args.h2, args.head};
  const int k_in[3] = {args.h0, args.h1, args.h2};

  if (threadIdx.x == 0) {
    for (int i = 0; i < kIStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);  // this CTA's MMA commit
    }
    for (int l = 0; l < 3; ++l) mbar_init(&acc_full[l], 1);
    mbar_init(roles_done, kIThreads / 32);
    s_abort = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kITmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // ---- layer 1 on the CUDA cores: columns c0 .. c0 + 127 of this row tile
  const int c0 = r * kIL0Cols;
  for (int i = threadIdx.x; i < BM; i += kIThreads) {
    const int row = m0 + i;
    s_e[i] = row < args.B ? args.row_env[row] : -1;
    s_b[i] = args.bias[0][c0 + i];
  }
  // bias slices of layers 2, 3 and the head at s_b + kIL0Cols + l * kIBRows
  for (int i = threadIdx.x; i < 3 * kIBRows; i += kIThreads) {
    const int l = i / kIBRows, j = i % kIBRows, nc = n_out[l] / kIC;
    if (j < nc) s_b[kIL0Cols + i] = args.bias[l + 1][r * nc + j];
  }
  for (int i = threadIdx.x; i < BM * nq; i += kIThreads) {
    const int rr = i / nq, c = i % nq, row = m0 + rr;
    float v = 0.f;
    if (row < args.B) {
      const int j = c < dof ? c : c - dof;
      const float* q = c < dof ? args.qs : args.qg;
      v = __bfloat162float(__float2bfloat16_rn(2.f * (q[(size_t)row * dof + j] - args.lo[j]) / args.span[j] - 1.f));
    }
    s_x[rr * kIQMax + c] = v;
  }
  const __nv_bfloat16* wq = static_cast<const __nv_bfloat16*>(args.wq);
  for (int i = threadIdx.x; i < nq * kIL0Cols; i += kIThreads) {
    const int c = i / kIL0Cols, jj = i % kIL0Cols;
    const int wrow = c < dof ? c : args.qpad + (c - dof);
    s_w[c * kIL0Cols + jj] = __bfloat162float(wq[(size_t)wrow * args.h0 + c0 + jj]);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_flag = &s_abort;
  {
    // item = (row, 8 columns): one 16-byte unit of the tiled output; all 128
    // rows of the tile are written (rows past B as zeros).  Groups of items
    // per thread put their loads in flight together.
    unsigned char* h1 = static_cast<unsigned char*>(args.act[0]) + ((size_t)mt * (args.h0 / BK)) * (BM * 128);
    constexpr int kUnits = kIL0Cols / 8, kItems = BM * kUnits, kGroup = 6;
    for (int base = threadIdx.x; base < kItems; base += kIThreads * kGroup) {
      float4 h[kGroup][2];
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int i = base + u * kIThreads, rr = i / kUnits, j8 = (i % kUnits) * 8;
        h[u][0] = h[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < kItems && s_e[rr] >= 0) {
          const float4* src = reinterpret_cast<const float4*>(args.h1o + (size_t)s_e[rr] * args.h0 + c0 + j8);
          h[u][0] = __ldg(src);
          h[u][1] = __ldg(src + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int i = base + u * kIThreads, rr = i / kUnits, j8 = (i % kUnits) * 8;
        if (i >= kItems) continue;
        uint4 pk = make_uint4(0u, 0u, 0u, 0u);
        if (s_e[rr] >= 0) {
          float v[8] = {h[u][0].x, h[u][0].y, h[u][0].z, h[u][0].w, h[u][1].x, h[u][1].y, h[u][1].z, h[u][1].w};
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] += s_b[j8 + e];
          for (int c = 0; c < nq; ++c) {
            const float x = s_x[rr * kIQMax + c];
            const float* w = s_w + c * kIL0Cols + j8;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = fmaf(w[e], x, v[e]);
          }
          pk = make_uint4(pack_bf16x2(fmaxf(v[0], 0.f), fmaxf(v[1], 0.f)), pack_bf16x2(fmaxf(v[2], 0.f), fmaxf(v[3], 0.f)),
                          pack_bf16x2(fmaxf(v[4], 0.f), fmaxf(v[5], 0.f)), pack_bf16x2(fmaxf(v[6], 0.f), fmaxf(v[7], 0.f)));
        }
        const int col = c0 + j8;  // k-block col / 64 of the next layer, unit (col % 64) / 8
        *reinterpret_cast<uint4*>(h1 + (size_t)(col / BK) * (BM * 128) + tile_off(rr, col % BK)) = pk;
      }
    }
  }
  __syncwarp();
  // the ring held layer 1's scratch: order these generic accesses before the
  // bulk copies that will overwrite it
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  cluster_publish();

  // ---- layers 2, 3 and the head on the tensor cores
  int it_p = 0, it_m = 0;  // stage counters of the producer and the MMA issuer
  uint32_t tcol = 0;       // TMEM column of this layer's accumulator
  for (int l = 0; l < 3; ++l) {
    const int nc = n_out[l] / kIC, n0 = r * nc, kts = k_in[l] / BK, stages = kts / kIKB;
    if (warp == 0) {
      const uint32_t b_bytes = (uint32_t)(nc * BK * 2);
      const unsigned char* a_src = static_cast<const unsigned char*>(args.act[l]) + (size_t)mt * kts * (BM * 128);
      const unsigned char* b_src = static_cast<const unsigned char*>(args.w[l]) + (size_t)r * kts * b_bytes;
      for (int ks = 0; ks < stages; ++ks, ++it_p) {
        const int st = it_p % kIStages;
        const uint32_t ph = (uint32_t)(it_p / kIStages) & 1u;
        int got = 0;
        if (lane == 0) got = (!*abort_flag && wait_bar(&empty[st], ph ^ 1u)) ? 1 : 0;
        got = __shfl_sync(kFull, got, 0);
        if (!got) {
          if (lane == 0) *abort_flag = 1;
          break;
        }
        if (lane == 0) {
          unsigned char* a = smem + st * kIStageBytes;
          mbar_arrive_expect_tx(&full[st], (uint32_t)(kIKB * (A_BYTES + b_bytes)));
          // the stage's 128-row activation k-blocks (contiguous), then this
          // CTA's weight k-blocks
          bulk_g2s(a, a_src + (size_t)ks * kIKB * (BM * 128), (uint32_t)(kIKB * A_BYTES), &full[st]);
          bulk_g2s(a + kIKB * A_BYTES, b_src + (size_t)ks * kIKB * b_bytes, kIKB * b_bytes, &full[st]);
        }
        __syncwarp();
      }
    } else if (warp == 1) {
      const uint32_t idesc = idesc_bf16(BM, nc);
      const uint32_t b_bytes = (uint32_t)(nc * BK * 2);
      bool ok = true;
      for (int ks = 0; ks < stages; ++ks, ++it_m) {
        const int st = it_m % kIStages;
        const uint32_t ph = (uint32_t)(it_m / kIStages) & 1u;
        int got = 0;
        if (lane == 0) got = (!*abort_flag && wait_bar(&full[st], ph)) ? 1 : 0;
        got = __shfl_sync(kFull, got, 0);
        if (!got) {
          if (lane == 0) *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after();
        if (lane == 0) {
          const uint32_t a = smem_u32(smem + st * kIStageBytes);
          const uint32_t b = a + kIKB * A_BYTES;
#pragma unroll
          for (int j = 0; j < kIKB; ++j)
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
              mma_bf16(tmem + tcol, smem_desc(a + j * A_BYTES + 32u * k), smem_desc(b + j * b_bytes + 32u * k), idesc,
                       (ks > 0 || j > 0 || k > 0) ? 1u : 0u);
          mma_commit(&empty[st]);
        }
        __syncwarp();
      }
      if (ok && lane == 0) mma_commit(&acc_full[l]);
      __syncwarp();
    } else {
      const int q = warp & 3;  // TMEM lane quarter this warp may access
      const int i = 32 * q + lane, row = m0 + i;
      int ok = 0;
      if (lane == 0) ok = (!*abort_flag && wait_bar(&acc_full[l], 0u)) ? 1 : 0;
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) {
        if (lane == 0) *abort_flag = 1;
      } else {
        fence_after();
        const float* bias = s_b + kIL0Cols + l * kIBRows;  // this CTA's slice: column n0 + j at j
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + tcol;
        if (l < 2) {
          // columns n0 .. n0 + 63 = k-block r of the next layer's input: row i
          // of that tile is this lane's 128 bytes
          unsigned char* tile = static_cast<unsigned char*>(args.act[l + 1]) +
                                ((size_t)mt * (n_out[l] / BK) + (size_t)(n0 / BK)) * (BM * 128);
          for (int c = 0; c < nc; c += 32) {
            uint32_t v[32];
            __syncwarp();
            tmem_ld32(taddr + (uint32_t)c, v);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              uint4 pk;
              const int j = c + 8 * u;
              pk.x = pack_bf16x2(fmaxf(__uint_as_float(v[8 * u]) + bias[j], 0.f),
                                 fmaxf(__uint_as_float(v[8 * u + 1]) + bias[j + 1], 0.f));
              pk.y = pack_bf16x2(fmaxf(__uint_as_float(v[8 * u + 2]) + bias[j + 2], 0.f),
                                 fmaxf(__uint_as_float(v[8 * u + 3]) + bias[j + 3], 0.f));
              pk.z = pack_bf16x2(fmaxf(__uint_as_float(v[8 * u + 4]) + bias[j + 4], 0.f),
                                 fmaxf(__uint_as_float(v[8 * u + 5]) + bias[j + 5], 0.f));
              pk.w = pack_bf16x2(fmaxf(__uint_as_float(v[8 * u + 6]) + bias[j + 6], 0.f),
                                 fmaxf(__uint_as_float(v[8 * u + 7]) + bias[j + 7], 0.f));
              *reinterpret_cast<uint4*>(tile + tile_off(i, j)) = pk;
            }
          }
        } else {
          // head columns n0 .. n0 + nc - 1 -> the planner's mixture row
          const int K = args.mix_k, G = args.gmm_dof;
          const int head = K * (1 + 2 * dof);
          float* g = row < args.B ? args.gmm_rows[row] : nullptr;
          for (int c = 0; c < nc; c += 16) {
            uint32_t v[16];
            __syncwarp();
            tmem_ld16(taddr + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int t = n0 + c + j;
              if (!g || t >= head) continue;
              const float val = __uint_as_float(v[j]) + bias[c + j];
              if (t < K) {
                g[t] = val;
              } else if (t < K + K * dof) {
                const int k = (t - K) / dof, jj = (t - K) % dof;
                g[K + k * G + jj] = val;
              } else {
                const int k = (t - K - K * dof) / dof, jj = (t - K - K * dof) % dof;
                g[K + K * G + k * G + jj] = fminf(fmaxf(val, args.logsig_lo), args.logsig_hi);
              }
            }
          }
        }
      }
    }
    tcol += (uint32_t)nc;
    if (l < 2) {
      __syncwarp();
      fence_before();
      cluster_publish();
      fence_after();
    }
  }
  // drain: the last release of every stage has arrived, so no MMA reads
  // this CTA's shared memory any more
  if (warp == 0) {
    if (lane == 0) {  // bounded waits, also after an abort
      for (int st = 0; st < kIStages && st < it_p; ++st) {
        const int uses = (it_p - 1 - st) / kIStages + 1;
        if (!wait_bar(&empty[st], (uint32_t)(uses - 1) & 1u)) break;
      }
    }
    __syncwarp();
  }
  cluster_sync_all();
  // join, then the allocating warp frees tensor memory (as in the GEMM)
  __syncwarp();
  fence_before();
  if (lane == 0) mbar_arrive(roles_done);
  if (warp == 1) {
    int joined = 0;
    if (lane == 0) joined = wait_bar(roles_done, 0) ? 1 : 0;
    joined = __shfl_sync(kFull, joined, 0);
    (void)joined;
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kITmemCols) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return g_encode;
}

// Row-major [rows x K] BF16 matrix with row stride ld elements, K
// contiguous; boxes of 64 x box_rows.
bool make_tmap(CUtensorMap* tm, const void* ptr, int rows, int K, int ld, int box_rows) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output matrix [rows x cols] with row stride ld elements (FP32 or BF16),
// boxes of 32 x 32 with the swizzle of the epilogue's staging tiles.
bool make_out_tmap(CUtensorMap* tm, const void* ptr, int rows, int cols, int ld, bool bf16) {
  auto enc = encoder();
  if (!enc) return false;
  const int es_bytes = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * es_bytes};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t es[2] = {1, 1};
  return enc(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr),
             dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             bf16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Encoded tensor maps by (device, address, rows, inner extent, row stride,
// kind, box rows): the MLP calls the same few layouts every step, and encoding
// costs host time.  kind 0: BF16 operand (boxes of 64 x box rows), 2: FP32
// output, 3: BF16 output.
struct MapKey {
  int dev;
  const void* ptr;
  int rows, cols, ld, kind, box;
  bool operator<(const MapKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (ptr != o.ptr) return ptr < o.ptr;
    if (rows != o.rows) return rows < o.rows;
    if (cols != o.cols) return cols < o.cols;
    if (ld != o.ld) return ld < o.ld;
    if (kind != o.kind) return kind < o.kind;
    return box < o.box;
  }
};
std::mutex g_map_mu;
std::map<MapKey, CUtensorMap> g_maps;
constexpr size_t kMaxCachedMaps = 256;

bool cached_map(CUtensorMap* tm, const void* ptr, int rows, int cols, int ld, int kind, int box = 0) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  const MapKey key{dev, ptr, rows, cols, ld, kind, box};
  std::lock_guard<std::mutex> lk(g_map_mu);
  auto it = g_maps.find(key);
  if (it != g_maps.end()) {
    *tm = it->second;
    return true;
  }
  const bool ok = kind == 0 ? make_tmap(tm, ptr, rows, cols, ld, box) : make_out_tmap(tm, ptr, rows, cols, ld, kind == 3);
  if (!ok) return false;
  if (g_maps.size() >= kMaxCachedMaps) g_maps.clear();
  g_maps.emplace(key, *tm);
  return true;
}

// Split-K workspace per (device, stream), grown on demand.
struct Workspace {
  float* ptr = nullptr;
  size_t floats = 0;
};
std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;
std::atomic<uint64_t> g_ws_epoch{0};  // bumped whenever a workspace is (re)allocated

float* workspace(size_t floats, cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace& w = g_ws[{dev, stream}];
  if (w.floats >= floats && w.ptr) return w.ptr;
  if (w.ptr) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) return nullptr;  // earlier launches may still read it
    cudaFree(w.ptr);
    w.ptr = nullptr;
    w.floats = 0;
  }
  g_ws_epoch.fetch_add(1);
  if (cudaMalloc(&w.ptr, floats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    w.ptr = nullptr;
    return nullptr;
  }
  w.floats = floats;
  return w.ptr;
}

int g_sms = 0;

}  // namespace

// Host launcher used by the MLP code and the C ABI entry point.  splits_hint:
// 0 = choose (split K while the tiles fill less than one wave), else forced.
int gemm_bf16_ld(const void* a, int lda, const void* b, int ldb, int M, int N, int K, const float* bias, int relu,
                 float* c32, int ldc32, void* c16, int ldc16, cudaStream_t stream, int splits_hint) {
  if (M <= 0 || N <= 0 || K <= 0 || !a || !b || (!c32 && !c16)) return PRRTC_ERR_INVALID_ARG;
  if (K % 8 || N % 8 || (c32 && ldc32 % 4) || (c16 && ldc16 % 8)) return PRRTC_ERR_UNSUPPORTED;
  if (lda < K || ldb < K || lda % 8 || ldb % 8) return PRRTC_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) return PRRTC_ERR_INVALID_ARG;
  if ((c32 && (reinterpret_cast<uintptr_t>(c32) & 15)) || (c16 && (reinterpret_cast<uintptr_t>(c16) & 15)))
    return PRRTC_ERR_INVALID_ARG;
  CUtensorMap ta, tb;
  if (!cached_map(&ta, a, M, K, lda, 0, BM) || !cached_map(&tb, b, N, K, ldb, 0, BN)) return PRRTC_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess)
      return PRRTC_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    attr = true;
  }
  Epilogue ep{M, N, K, bias, relu, c32 ? 1 : 0, c16 ? 1 : 0, 1, 0, 0, 0, 0};
  OutMaps om;
  std::memset(&om, 0, sizeof(om));
  if (c32 && !cached_map(&om.c32, c32, M, N, ldc32, 2)) return PRRTC_ERR_CUDA;
  if (c16 && !cached_map(&om.c16, c16, M, N, ldc16, 3)) return PRRTC_ERR_CUDA;
  ep.m_tiles = (M + BM - 1) / BM;
  ep.n_tiles = (N + BN - 1) / BN;
  ep.k_tiles = (K + BK - 1) / BK;
  ep.m_pad = ep.m_tiles * BM;
  const int tiles = ep.m_tiles * ep.n_tiles;
  const int sms = g_sms > 0 ? g_sms : 1;
  int splits = splits_hint;
  if (splits <= 0) {
    splits = 1;
    while (splits < kMaxSplits && tiles * (splits * 2) <= sms && ep.k_tiles / (splits * 2) >= kMinKTilesPerSplit)
      splits *= 2;
  }
  splits = std::max(1, std::min(splits, std::min(kMaxSplits, ep.k_tiles)));
  ep.splits = splits;
  float* ws = nullptr;
  if (splits > 1) {
    ws = workspace((size_t)splits * ep.m_pad * N, stream);
    if (!ws) return PRRTC_ERR_OOM;
    if (!cached_map(&om.ws, ws, splits * ep.m_pad, N, N, 2)) return PRRTC_ERR_CUDA;
  }
  const int units = tiles * splits;
  const int grid = std::min(units, sms);
  gemm_bf16_kernel<<<grid, THREADS, SMEM_BYTES, stream>>>(ta, tb, om, ep);
  if (cudaGetLastError() != cudaSuccess) return PRRTC_ERR_CUDA;
  if (splits > 1) {
    const size_t work = (size_t)M * (N / 4);
    const int blocks = (int)std::min<size_t>((work + 255) / 256, (size_t)sms * 8);
    splitk_reduce_kernel<<<blocks, 256, 0, stream>>>(ws, splits, M, ep.m_pad, N, bias, relu, c32, ldc32,
                                                     static_cast<__nv_bfloat16*>(c16), ldc16);
    if (cudaGetLastError() != cudaSuccess) return PRRTC_ERR_CUDA;
  }
  return PRRTC_OK;
}

int gemm_bf16_split(const void* a, const void* b, int M, int N, int K, const float* bias, int relu, float* c32,
                    int ldc32, void* c16, int ldc16, cudaStream_t stream, int splits_hint) {
  return gemm_bf16_ld(a, K, b, K, M, N, K, bias, relu, c32, ldc32, c16, ldc16, stream, splits_hint);
}

int gemm_bf16(const void* a, const void* b, int M, int N, int K, const float* bias, int relu, float* c32, int ldc32,
              void* c16, int ldc16, cudaStream_t stream) {
  return gemm_bf16_split(a, b, M, N, K, bias, relu, c32, ldc32, c16, ldc16, stream, 0);
}

int mlp_check_shapes(int h0, int h1, int h2, int head) {
  if (h0 != kIC * kIL0Cols || h1 % (BK * kIKB) || h2 % (BK * kIKB) || h0 % (BK * kIKB)) return PRRTC_ERR_UNSUPPORTED;
  const int n_out[3] = {h1, h2, head};
  int cols = 0;
  for (int l = 0; l < 3; ++l) {
    if (n_out[l] % (kIC * 16) || n_out[l] / kIC > kIBRows) return PRRTC_ERR_UNSUPPORTED;
    cols += n_out[l] / kIC;
  }
  return cols <= (int)kITmemCols ? PRRTC_OK : PRRTC_ERR_UNSUPPORTED;
}

int mlp_tile_weights(const void* w, int N, int K, void* out, cudaStream_t stream) {
  if (N % (kIC * 16) || K % BK || (reinterpret_cast<uintptr_t>(out) & 15)) return PRRTC_ERR_UNSUPPORTED;
  const size_t total = (size_t)N * K;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  tile_weights_kernel<<<blocks, 256, 0, stream>>>(static_cast<const __nv_bfloat16*>(w), N, K,
                                                  static_cast<__nv_bfloat16*>(out));
  return cudaGetLastError() == cudaSuccess ? PRRTC_OK : PRRTC_ERR_CUDA;
}

int mlp_infer(const MlpInferArgs& a, cudaStream_t stream) {
  if (a.rows <= 0 || a.B <= 0 || a.B > a.rows || a.dof < 1 || 2 * a.dof > kIQMax || a.dof > a.gmm_dof)
    return PRRTC_ERR_INVALID_ARG;
  int rc = mlp_check_shapes(a.h0, a.h1, a.h2, a.head);
  if (rc) return rc;
  if (a.mix_k * (1 + 2 * a.dof) > a.head) return PRRTC_ERR_INVALID_ARG;
  for (int l = 0; l < 3; ++l)
    if (reinterpret_cast<uintptr_t>(a.act[l]) & 15 || reinterpret_cast<uintptr_t>(a.w[l]) & 15)
      return PRRTC_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(a.h1o) & 15) return PRRTC_ERR_INVALID_ARG;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kISmemBytes) !=
        cudaSuccess)
      return PRRTC_ERR_CUDA;
    attr = true;
  }
  const int m_tiles = (a.rows + BM - 1) / BM;
  mlp_infer_kernel<<<m_tiles * kIC, kIThreads, kISmemBytes, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? PRRTC_OK : PRRTC_ERR_CUDA;
}

// Changes whenever a split-K workspace is allocated or moved: work captured
// into a CUDA graph before the change may point at a freed workspace.
uint64_t gemm_workspace_epoch() { return g_ws_epoch.load(); }

// Reads and clears the kernel's error word (synchronous).
int gemm_take_error() {
  int e = 0, z = 0;
  if (cudaMemcpyFromSymbol(&e, g_gemm_error, sizeof(int)) != cudaSuccess) return PRRTC_ERR_CUDA;
  if (e) cudaMemcpyToSymbol(g_gemm_error, &z, sizeof(int));
  return e;
}

}  // namespace prrtc

extern "C" int prrtc_gemm_bf16(const void* a, const void* b, int32_t M, int32_t N, int32_t K, const float* bias,
                               int32_t relu, float* c32, void* c16, void* stream) {
  return prrtc::gemm_bf16(a, b, M, N, K, bias, relu, c32, N, c16, N, static_cast<cudaStream_t>(stream));
}

extern "C" int prrtc_gemm_bf16_splitk(const void* a, const void* b, int32_t M, int32_t N, int32_t K,
                                      const float* bias, int32_t relu, float* c32, void* c16, int32_t splits,
                                      void* stream) {
  if (splits < 0) return PRRTC_ERR_INVALID_ARG;
  return prrtc::gemm_bf16_split(a, b, M, N, K, bias, relu, c32, N, c16, N, static_cast<cudaStream_t>(stream), splits);
}

extern "C" int prrtc_gemm_error(void) { return prrtc::gemm_take_error(); }
