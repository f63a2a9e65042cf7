// prrtc_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores for the
// learned sampling proposal's dense layers:  C[M,N] = A[M,K] * B[N,K]^T with
// FP32 accumulation in tensor memory, optional bias + ReLU and FP32 / BF16
// outputs.
//
// One CTA computes a 128 x 128 tile:
//   warp 0  -- one lane issues TMA loads of 128 x 64 BF16 tiles of A and B
//              (128-byte swizzle) into a 4-stage shared-memory ring;
//   warp 1  -- allocates 128 TMEM columns; one lane issues tcgen05.mma
//              (M=128, N=128, K=16, kind::f16) four times per stage and
//              commits each stage back to the producer;
//   warps 2-5 -- wait for the final commit, read the accumulator with
//              tcgen05.ld (each warp owns one 32-lane quarter of TMEM) and
//              run the epilogue.
// Every mbarrier wait is bounded; a wait that gives up records an error and
// the CTA still frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "prrtc.h"
#include "prrtc_device.cuh"

namespace prrtc {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = BN;
constexpr uint32_t kPolls = 1u << 26;

__device__ int g_gemm_error;

struct Epilogue {
  int M, N, K;
  const float* bias;
  int relu;
  float* c32;
  int ldc32;
  __nv_bfloat16* c16;
  int ldc16;
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

// Epilogue of one 32-column chunk of one output row: bias, ReLU, stores.
__device__ __forceinline__ void store_chunk(const Epilogue& ep, int row, int col0, const uint32_t (&v)[32]) {
  float f[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float x = __uint_as_float(v[j]);
    if (ep.bias && col0 + j < ep.N) x += ep.bias[col0 + j];
    if (ep.relu) x = fmaxf(x, 0.f);
    f[j] = x;
  }
  const bool full_chunk = col0 + 32 <= ep.N;
  if (ep.c32) {
    float* dst = ep.c32 + (size_t)row * ep.ldc32 + col0;
    if (full_chunk) {
#pragma unroll
      for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(f[j], f[j + 1], f[j + 2], f[j + 3]);
    } else {
      for (int j = 0; j < 32 && col0 + j < ep.N; ++j) dst[j] = f[j];
    }
  }
  if (ep.c16) {
    __nv_bfloat16* dst = ep.c16 + (size_t)row * ep.ldc16 + col0;
    if (full_chunk) {
#pragma unroll
      for (int j = 0; j < 32; j += 8) {
        uint4 pk;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(f[j], f[j + 1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(f[j + 2], f[j + 3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(f[j + 4], f[j + 5]);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(f[j + 6], f[j + 7]);
        pk.x = *reinterpret_cast<uint32_t*>(&h0);
        pk.y = *reinterpret_cast<uint32_t*>(&h1);
        pk.z = *reinterpret_cast<uint32_t*>(&h2);
        pk.w = *reinterpret_cast<uint32_t*>(&h3);
        *reinterpret_cast<uint4*>(dst + j) = pk;
      }
    } else {
      for (int j = 0; j < 32 && col0 + j < ep.N; ++j) dst[j] = __float2bfloat16_rn(f[j]);
    }
  }
}

__global__ void __launch_bounds__(THREADS, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Epilogue ep) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int k_tiles = (ep.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
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

  if (warp == 0) {
    if (lane == 0) {
      for (int kt = 0; kt < k_tiles; ++kt) {
        const int s = kt % STAGES;
        const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
        if (!wait_bar(&empty[s], ph ^ 1u)) break;
        unsigned char* a = smem + s * STAGE_BYTES;
        mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
        tma_load_2d(a, &tmA, &full[s], kt * BK, m0);
        tma_load_2d(a + A_BYTES, &tmB, &full[s], kt * BK, n0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, BN);
      bool ok = true;
      for (int kt = 0; kt < k_tiles; ++kt) {
        const int s = kt % STAGES;
        const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
        if (!wait_bar(&full[s], ph)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t a = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t b = a + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          mma_bf16(tmem, smem_desc(a + 32u * k), smem_desc(b + 32u * k), idesc, (kt > 0 || k > 0) ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(done);
    }
  } else {
    int ok = 0;
    if (lane == 0) ok = wait_bar(done, 0) ? 1 : 0;
    ok = __shfl_sync(kFull, ok, 0);
    if (ok) {
      fence_after();
      const int q = warp & 3;  // TMEM lane quarter this warp may access
      const int row = m0 + 32 * q + lane;
      for (int c = 0; c < BN; c += 32) {
        uint32_t v[32];
        __syncwarp();
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
        const int col0 = n0 + c;
        if (row < ep.M && col0 < ep.N) store_chunk(ep, row, col0, v);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
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

// Row-major [rows x K] BF16 matrix, K contiguous; boxes of 64 x 128.
bool make_tmap(CUtensorMap* tm, const void* ptr, int rows, int K) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, 128};
  cuuint32_t es[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Host launcher used by the MLP code and the C ABI entry point.
int gemm_bf16(const void* a, const void* b, int M, int N, int K, const float* bias, int relu, float* c32, int ldc32,
              void* c16, int ldc16, cudaStream_t stream) {
  if (M <= 0 || N <= 0 || K <= 0 || !a || !b || (!c32 && !c16)) return PRRTC_ERR_INVALID_ARG;
  if (K % 8 || N % 8 || (c32 && ldc32 % 4) || (c16 && ldc16 % 8)) return PRRTC_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) return PRRTC_ERR_INVALID_ARG;
  if ((c32 && (reinterpret_cast<uintptr_t>(c32) & 15)) || (c16 && (reinterpret_cast<uintptr_t>(c16) & 15)))
    return PRRTC_ERR_INVALID_ARG;
  CUtensorMap ta, tb;
  if (!make_tmap(&ta, a, M, K) || !make_tmap(&tb, b, N, K)) return PRRTC_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess)
      return PRRTC_ERR_CUDA;
    attr = true;
  }
  Epilogue ep{M, N, K, bias, relu, c32, ldc32, static_cast<__nv_bfloat16*>(c16), ldc16};
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  gemm_bf16_kernel<<<grid, THREADS, SMEM_BYTES, stream>>>(ta, tb, ep);
  return cudaGetLastError() == cudaSuccess ? PRRTC_OK : PRRTC_ERR_CUDA;
}

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

extern "C" int prrtc_gemm_error(void) { return prrtc::gemm_take_error(); }
