// prrtc_device.cuh -- device-side data layouts and the collision-checking core
// of the pRRTC hot path for sm_103a.
//
// Mapping (GB300-first, differs from the paper's 4-threads-per-state layout of
// Sec. III-A): one warp checks one candidate edge, one lane per interpolated
// state (Alg. 2: all N_cc states of the edge in parallel).  Each lane runs the
// forward kinematics of its own state in registers, tests every sphere of the
// link it just placed against every obstacle primitive held in shared memory
// (broadcast reads, no bank conflicts), and the warp votes with __any_sync
// after every sphere so that the whole edge stops at the first collision
// (Sec. III-A, early exit).  Self-collision pairs are tested afterwards from
// the sphere centres the lane staged in shared memory.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace prrtc {

constexpr int kMaxDof = 16;
constexpr int kMaxDistinctSpheres = 64;
constexpr int kMaxDistinctPairs = 3072;
constexpr unsigned kFull = 0xffffffffu;

enum JointType : int { kRevZ = 0, kRevY = 1, kPrismZ = 2, kPrismX = 3, kPrismY = 4, kRevX = 5 };

// Robot sphere model, compact and merged (coincident equal-radius spheres on
// one frame collapse to one).  Spheres are sorted by frame so that the FK loop
// meets each frame's spheres right after placing the frame.
struct RobotHeader {
  int dof;
  int dpad;            // tree row stride in floats: dof rounded up to a multiple of 4
  int n_spheres;       // distinct spheres
  int n_pairs;         // distinct self-collision pairs
  int n_raw;           // spheres as given
  int pad_[3];
  int jtype[kMaxDof];
  int jparent[kMaxDof];
  float jlen[kMaxDof];
  float lo[kMaxDof];
  float span[kMaxDof];  // upper - lower
  float4 jbase[kMaxDof];
  int sph_begin[kMaxDof + 1];
  int pad2_[3];
  float4 sph[kMaxDistinctSpheres];   // offset xyz in the frame, radius
};

// Pair table follows the header in device memory: pair[k] = i | (j << 16),
// thr[k] = (r_i + r_j)^2, sorted by i.
struct RobotDev {
  RobotHeader h;
  uint32_t pair[kMaxDistinctPairs];
  float thr[kMaxDistinctPairs];
  int16_t raw_to_distinct[128];
};

// Environment: one float4 array laid out as
//   [AABB x2: centre|0, half|0][OBB x5: centre, half, R^T rows][CYL x2:
//   centre|radius, axis|half_len][SPH x1: centre|radius].
struct EnvView {
  const float4* data;
  int n_aabb, n_obb, n_cyl, n_sph;
  __host__ __device__ int n_float4() const { return 2 * n_aabb + 5 * n_obb + 2 * n_cyl + n_sph; }
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products,
// key bumped by the two Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// ------------------------------------------------------------------ counters
struct WorkCount {
  unsigned long long sphere_tests = 0;  // lane-level sphere passes over the environment
  unsigned long long pair_tests = 0;    // lane-level self pair tests
  unsigned long long fk_states = 0;     // lane-level FK evaluations
};

// ------------------------------------------------------------------ env tests
// Does a sphere (centre c, radius r) touch any primitive?  Strict test on the
// squared distance to each primitive (touching counts as free).
__device__ __forceinline__ bool sphere_hits_env(float cx, float cy, float cz, float r, const float4* __restrict__ env,
                                                int n_aabb, int n_obb, int n_cyl, int n_sph) {
  const float r2 = r * r;
  bool hit = false;
  const float4* e = env;
#pragma unroll 4
  for (int o = 0; o < n_aabb; ++o) {
    const float4 c = e[2 * o], h = e[2 * o + 1];
    const float dx = fmaxf(fabsf(cx - c.x) - h.x, 0.f);
    const float dy = fmaxf(fabsf(cy - c.y) - h.y, 0.f);
    const float dz = fmaxf(fabsf(cz - c.z) - h.z, 0.f);
    hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < r2;
  }
  e += 2 * n_aabb;
#pragma unroll 2
  for (int o = 0; o < n_obb; ++o) {
    const float4 c = e[5 * o], h = e[5 * o + 1], a = e[5 * o + 2], b = e[5 * o + 3], d = e[5 * o + 4];
    const float vx = cx - c.x, vy = cy - c.y, vz = cz - c.z;
    const float lx = fmaf(a.x, vx, fmaf(a.y, vy, a.z * vz));
    const float ly = fmaf(b.x, vx, fmaf(b.y, vy, b.z * vz));
    const float lz = fmaf(d.x, vx, fmaf(d.y, vy, d.z * vz));
    const float dx = fmaxf(fabsf(lx) - h.x, 0.f);
    const float dy = fmaxf(fabsf(ly) - h.y, 0.f);
    const float dz = fmaxf(fabsf(lz) - h.z, 0.f);
    hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < r2;
  }
  e += 5 * n_obb;
#pragma unroll 2
  for (int o = 0; o < n_cyl; ++o) {
    const float4 c = e[2 * o], a = e[2 * o + 1];
    const float vx = cx - c.x, vy = cy - c.y, vz = cz - c.z;
    const float z = fmaf(a.x, vx, fmaf(a.y, vy, a.z * vz));
    const float wx = fmaf(-z, a.x, vx), wy = fmaf(-z, a.y, vy), wz = fmaf(-z, a.z, vz);
    const float rho2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
    const float rho = rho2 > 0.f ? rho2 * rsqrtf(rho2) : 0.f;
    const float er = fmaxf(rho - c.w, 0.f);
    const float ez = fmaxf(fabsf(z) - a.w, 0.f);
    hit |= fmaf(er, er, ez * ez) < r2;
  }
  e += 2 * n_cyl;
#pragma unroll 4
  for (int o = 0; o < n_sph; ++o) {
    const float4 s = e[o];
    const float dx = cx - s.x, dy = cy - s.y, dz = cz - s.z;
    const float rr = r + s.w;
    hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
  }
  return hit;
}

// ------------------------------------------------------------------ FK + CC
// Joint-value sources for state_collides: lane-private values staged in
// shared memory ([joint][lane]) or a point on a warp-uniform edge a -> b
// (both held in shared memory) at parameter t, exactly b at the endpoint.
struct LaneQ {
  const float* q;  // [kMaxDof][32]
  int lane;
  __device__ __forceinline__ float operator()(int i) const { return q[i * 32 + lane]; }
};

struct EdgeQ {
  const float* a;
  const float* b;
  float t;
  bool end;
  __device__ __forceinline__ float operator()(int i) const { return end ? b[i] : fmaf(t, b[i] - a[i], a[i]); }
};

// Collision test of one configuration per lane.  `stage` is this warp's
// [n_spheres][3][32] shared-memory buffer of sphere centres.  With kWarpVote
// the whole warp returns true as soon as any active lane collides (the edge
// verdict), otherwise each lane returns its own verdict and the warp runs to
// completion.  The joint loop is a runtime loop so that the obstacle loops
// exist once in the code.
template <bool kWarpVote, class QS>
__device__ __forceinline__ bool state_collides(const RobotHeader* __restrict__ R, const uint32_t* __restrict__ pair,
                                               const float* __restrict__ thr, const float4* __restrict__ env,
                                               int n_aabb, int n_obb, int n_cyl, int n_sph, float* __restrict__ stage,
                                               const QS& qs, bool active, int lane, WorkCount& wc) {
  const int dof = R->dof;
  float ax = 1.f, ay = 0.f, az = 0.f;  // rotation column 0 (local x in world)
  float bx = 0.f, by = 1.f, bz = 0.f;  // column 1
  float cx = 0.f, cy = 0.f, cz = 1.f;  // column 2
  float px = 0.f, py = 0.f, pz = 0.f;
  bool hit = false;
  wc.fk_states += active;
#pragma unroll 1
  for (int i = 0; i < dof; ++i) {
    if (R->jparent[i] < 0) {
      ax = 1.f; ay = 0.f; az = 0.f;
      bx = 0.f; by = 1.f; bz = 0.f;
      cx = 0.f; cy = 0.f; cz = 1.f;
      const float4 b = R->jbase[i];
      px = b.x; py = b.y; pz = b.z;
    }
    const int ty = R->jtype[i];
    const float qi = qs(i);
    if (ty == kRevZ || ty == kRevY || ty == kRevX) {
      float s, c;
      sincosf(qi, &s, &c);
      if (ty == kRevZ) {  // R * Rz: col0' = c col0 + s col1, col1' = -s col0 + c col1
        const float nx = fmaf(c, ax, s * bx), ny = fmaf(c, ay, s * by), nz = fmaf(c, az, s * bz);
        bx = fmaf(c, bx, -s * ax); by = fmaf(c, by, -s * ay); bz = fmaf(c, bz, -s * az);
        ax = nx; ay = ny; az = nz;
      } else if (ty == kRevY) {  // R * Ry: col0' = c col0 - s col2, col2' = s col0 + c col2
        const float nx = fmaf(c, ax, -s * cx), ny = fmaf(c, ay, -s * cy), nz = fmaf(c, az, -s * cz);
        cx = fmaf(c, cx, s * ax); cy = fmaf(c, cy, s * ay); cz = fmaf(c, cz, s * az);
        ax = nx; ay = ny; az = nz;
      } else {  // R * Rx: col1' = c col1 + s col2, col2' = -s col1 + c col2
        const float nx = fmaf(c, bx, s * cx), ny = fmaf(c, by, s * cy), nz = fmaf(c, bz, s * cz);
        cx = fmaf(c, cx, -s * bx); cy = fmaf(c, cy, -s * by); cz = fmaf(c, cz, -s * bz);
        bx = nx; by = ny; bz = nz;
      }
    } else if (ty == kPrismZ) {
      px = fmaf(qi, cx, px); py = fmaf(qi, cy, py); pz = fmaf(qi, cz, pz);
    } else if (ty == kPrismX) {
      px = fmaf(qi, ax, px); py = fmaf(qi, ay, py); pz = fmaf(qi, az, pz);
    } else {
      px = fmaf(qi, bx, px); py = fmaf(qi, by, py); pz = fmaf(qi, bz, pz);
    }
    const float L = R->jlen[i];
    px = fmaf(L, cx, px); py = fmaf(L, cy, py); pz = fmaf(L, cz, pz);

    const int s1 = R->sph_begin[i + 1];
    for (int s = R->sph_begin[i]; s < s1; ++s) {
      const float4 o = R->sph[s];
      const float sx = fmaf(ax, o.x, fmaf(bx, o.y, fmaf(cx, o.z, px)));
      const float sy = fmaf(ay, o.x, fmaf(by, o.y, fmaf(cy, o.z, py)));
      const float sz = fmaf(az, o.x, fmaf(bz, o.y, fmaf(cz, o.z, pz)));
      float* st = stage + s * 96 + lane;
      st[0] = sx;
      st[32] = sy;
      st[64] = sz;
      hit |= sphere_hits_env(sx, sy, sz, o.w, env, n_aabb, n_obb, n_cyl, n_sph);
      wc.sphere_tests += active;
      if (kWarpVote) {
        if (__any_sync(kFull, hit && active)) return true;
      }
    }
  }
  const int np = R->n_pairs;
  int last_i = -1;
  float ix = 0.f, iy = 0.f, iz = 0.f;
  for (int k = 0; k < np; ++k) {
    const uint32_t pr = pair[k];
    const int i = (int)(pr & 0xffffu), j = (int)(pr >> 16);
    if (i != last_i) {
      const float* si = stage + i * 96 + lane;
      ix = si[0]; iy = si[32]; iz = si[64];
      last_i = i;
    }
    const float* sj = stage + j * 96 + lane;
    const float dx = ix - sj[0], dy = iy - sj[32], dz = iz - sj[64];
    hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < thr[k];
    if (kWarpVote && (k & 15) == 15) {
      if (__any_sync(kFull, hit && active)) {
        wc.pair_tests += (unsigned long long)(k + 1) * active;
        return true;
      }
    }
  }
  wc.pair_tests += (unsigned long long)np * active;
  if (kWarpVote) return __any_sync(kFull, hit && active);
  return hit;
}

// Byte size of a warp's sphere-centre staging buffer.
__host__ __device__ inline int stage_bytes(int n_spheres) { return n_spheres * 96 * (int)sizeof(float); }

// Shared-memory image of a robot: header, then pairs, then thresholds.
__host__ __device__ inline int robot_smem_bytes(int n_pairs) {
  int b = (int)sizeof(RobotHeader) + n_pairs * 8;
  return (b + 15) & ~15;
}

// ------------------------------------------------------------------ TMA staging
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Bounded wait for the phase with parity `phase`; returns false on give-up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint32_t max_polls) {
  for (uint32_t k = 0; k < max_polls; ++k) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 1-D bulk copy global -> shared through the TMA engine (16-byte aligned
// addresses, size a multiple of 16), completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

}  // namespace prrtc
