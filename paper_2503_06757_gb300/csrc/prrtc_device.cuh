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
//
// Two-stage check (Sec. III-A, hierarchical): a frame with several spheres is
// first tested through one bounding sphere against every primitive; its fine
// spheres then meet only the primitives that the bounding sphere of some lane
// touched.  Each bounding sphere contains its fine spheres with a margin far
// above FP32 rounding, so the verdicts equal those of the one-stage check.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace prrtc {

constexpr int kMaxDof = 16;
constexpr int kMaxDistinctSpheres = 64;
constexpr int kMaxDistinctPairs = 3072;
constexpr int kMaxPairBlocks = 144;  // link pairs with self-collision pairs: <= 16 * 17 / 2
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
  int two_stage;       // 1: frames with a bounding sphere are checked in two stages
  int n_blocks;        // self-collision pair blocks (one per pair of links)
  int pad_;
  int jtype[kMaxDof];
  int jparent[kMaxDof];
  float jlen[kMaxDof];
  float lo[kMaxDof];
  float span[kMaxDof];  // upper - lower
  float4 jbase[kMaxDof];
  int sph_begin[kMaxDof + 1];
  int pad2_[3];
  float4 sph[kMaxDistinctSpheres];   // offset xyz in the frame, radius
  float4 coarse[kMaxDof];            // bounding sphere of frame i's spheres (radius 0: none)
  // Group sphere of frame i for the self-collision first stage: its bounding
  // sphere, or its only sphere, or radius 0 (no spheres).  Centres are staged
  // after the fine spheres (stage slot n_spheres + i).
  float4 grp[kMaxDof];
  // Self-collision pair blocks: the pairs between the spheres of links fa and
  // fb are pair[begin .. end); thr = (R_fa + R_fb)^2 of the group spheres, or
  // +inf when the block is tested without a first stage.
  uint32_t blk_frames[kMaxPairBlocks];  // fa | fb << 16
  uint32_t blk_range[kMaxPairBlocks];   // begin | end << 16
  float blk_thr[kMaxPairBlocks];
};

// Pair table follows the header in device memory: pair[k] = i | (j << 16),
// thr[k] = (r_i + r_j)^2, sorted by i.
struct RobotDev {
  RobotHeader h;
  uint32_t pair[kMaxDistinctPairs];
  float thr[kMaxDistinctPairs];
  int16_t raw_to_distinct[128];
};

// Euclidean signed distance field on a voxel grid (the paper's ESDF maps):
// values at voxel centres (ox, oy, oz) + (index + 1/2) * voxel, index
// i + nx*(j + ny*k); v == null when the environment has none.
struct EsdfGrid {
  const float* v;
  float ox, oy, oz, inv_voxel;
  int nx, ny, nz, pad_;
};

// Environment: one float4 array laid out as
//   [AABB x2: centre|0, half|0][OBB x5: centre, half, R^T rows][CYL x2:
//   centre|radius, axis|half_len][SPH x1: centre|radius],
// plus an optional distance field (read from global memory / L2).
struct EnvView {
  const float4* data;
  int n_aabb, n_obb, n_cyl, n_sph;
  EsdfGrid esdf;
  __host__ __device__ int n_float4() const { return 2 * n_aabb + 5 * n_obb + 2 * n_cyl + n_sph; }
};

// Trilinear read of the distance field at p: continuous index
// u = (p - origin) / voxel - 1/2 per axis, clamped to [0, n - 1], base
// min(floor(u), n - 2); blends along x, then y, then z.  Out of line, so that
// environments without a field pay no registers for it.
static __device__ __noinline__ float esdf_read(const EsdfGrid& g, float px, float py, float pz) {
  float u = fminf(fmaxf(fmaf(px - g.ox, g.inv_voxel, -0.5f), 0.f), (float)(g.nx - 1));
  float w = fminf(fmaxf(fmaf(py - g.oy, g.inv_voxel, -0.5f), 0.f), (float)(g.ny - 1));
  float z = fminf(fmaxf(fmaf(pz - g.oz, g.inv_voxel, -0.5f), 0.f), (float)(g.nz - 1));
  const int i0 = min((int)u, g.nx - 2), j0 = min((int)w, g.ny - 2), k0 = min((int)z, g.nz - 2);
  const float tx = u - (float)i0, ty = w - (float)j0, tz = z - (float)k0;
  const float* b = g.v + (size_t)i0 + (size_t)g.nx * ((size_t)j0 + (size_t)g.ny * (size_t)k0);
  const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
  float c00 = __ldg(b), c01 = __ldg(b + sy), c10 = __ldg(b + sz), c11 = __ldg(b + sz + sy);
  c00 = fmaf(tx, __ldg(b + 1) - c00, c00);
  c01 = fmaf(tx, __ldg(b + sy + 1) - c01, c01);
  c10 = fmaf(tx, __ldg(b + sz + 1) - c10, c10);
  c11 = fmaf(tx, __ldg(b + sz + sy + 1) - c11, c11);
  const float y0 = fmaf(ty, c01 - c00, c00), y1 = fmaf(ty, c11 - c10, c10);
  return fmaf(tz, y1 - y0, y0);
}

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
// Work counters of one warp, kept in shared memory and updated by lane 0 with
// warp-uniform increments (uniform work x active lanes), so that they hold no
// registers in the checking loops.  The planner's per-iteration counters
// follow the collision-checking ones.
struct WarpCount {
  unsigned long long sphere_tests;  // lane-level sphere passes over the environment
  unsigned long long pair_tests;    // lane-level self pair tests
  unsigned long long fk_states;     // lane-level FK evaluations
  unsigned long long prim[4];       // second-stage sphere-primitive tests per type
  unsigned long long edges, edge_states, nn_nodes, iterations, insert_fail, dd_rejected;
  unsigned long long verdict_states;  // states whose verdict was established (early-exit states excluded)
  unsigned long long aborted;         // set when an edge check stopped because the problem was solved
  unsigned long long pad_;
};
static_assert(sizeof(WarpCount) == 128, "per-warp counter block is 128 bytes");

__device__ __forceinline__ void warp_count_clear(WarpCount* wc, int lane) {
  if (lane < 16) reinterpret_cast<unsigned long long*>(wc)[lane] = 0ull;
  __syncwarp();
}

// ------------------------------------------------------------------ env tests
// Squared distance from a point to one primitive (0 inside).  AABB: centre |
// half extents; OBB: centre | half extents | rows of R^T; capped cylinder:
// centre | radius, unit axis | half length.
__device__ __forceinline__ float d2_aabb(const float4* __restrict__ e, float px, float py, float pz) {
  const float4 c = e[0], h = e[1];
  const float dx = fmaxf(fabsf(px - c.x) - h.x, 0.f);
  const float dy = fmaxf(fabsf(py - c.y) - h.y, 0.f);
  const float dz = fmaxf(fabsf(pz - c.z) - h.z, 0.f);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

__device__ __forceinline__ float d2_obb(const float4* __restrict__ e, float px, float py, float pz) {
  const float4 c = e[0], h = e[1], a = e[2], b = e[3], d = e[4];
  const float vx = px - c.x, vy = py - c.y, vz = pz - c.z;
  const float lx = fmaf(a.x, vx, fmaf(a.y, vy, a.z * vz));
  const float ly = fmaf(b.x, vx, fmaf(b.y, vy, b.z * vz));
  const float lz = fmaf(d.x, vx, fmaf(d.y, vy, d.z * vz));
  const float dx = fmaxf(fabsf(lx) - h.x, 0.f);
  const float dy = fmaxf(fabsf(ly) - h.y, 0.f);
  const float dz = fmaxf(fabsf(lz) - h.z, 0.f);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

__device__ __forceinline__ float d2_cyl(const float4* __restrict__ e, float px, float py, float pz) {
  const float4 c = e[0], a = e[1];
  const float vx = px - c.x, vy = py - c.y, vz = pz - c.z;
  const float z = fmaf(a.x, vx, fmaf(a.y, vy, a.z * vz));
  const float wx = fmaf(-z, a.x, vx), wy = fmaf(-z, a.y, vy), wz = fmaf(-z, a.z, vz);
  const float rho2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
  const float rho = rho2 > 0.f ? rho2 * rsqrtf(rho2) : 0.f;
  const float er = fmaxf(rho - c.w, 0.f);
  const float ez = fmaxf(fabsf(z) - a.w, 0.f);
  return fmaf(er, er, ez * ez);
}

// Strict sphere tests (touching counts as free), one primitive type each; a
// sphere obstacle compares against the sum of the radii.
enum PrimKind : int { kAabb = 0, kObb = 1, kCyl = 2, kSph = 3 };
template <int K> struct Prim;
template <> struct Prim<kAabb> {
  static constexpr int kUnroll = 4;
  static constexpr int kStride = 2;
  __device__ static __forceinline__ bool hit(const float4* e, float x, float y, float z, float r) {
    return d2_aabb(e, x, y, z) < r * r;
  }
};
template <> struct Prim<kObb> {
  static constexpr int kUnroll = 2;
  static constexpr int kStride = 5;
  __device__ static __forceinline__ bool hit(const float4* e, float x, float y, float z, float r) {
    return d2_obb(e, x, y, z) < r * r;
  }
};
template <> struct Prim<kCyl> {
  static constexpr int kUnroll = 2;
  static constexpr int kStride = 2;
  __device__ static __forceinline__ bool hit(const float4* e, float x, float y, float z, float r) {
    return d2_cyl(e, x, y, z) < r * r;
  }
};
template <> struct Prim<kSph> {
  static constexpr int kUnroll = 4;
  static constexpr int kStride = 1;
  __device__ static __forceinline__ bool hit(const float4* e, float x, float y, float z, float r) {
    const float4 s = e[0];
    const float dx = x - s.x, dy = y - s.y, dz = z - s.z;
    const float rr = r + s.w;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
  }
};

// Does a sphere (centre c, radius r) touch any primitive?
__device__ __forceinline__ bool sphere_hits_env(float cx, float cy, float cz, float r, const float4* __restrict__ env,
                                                int n_aabb, int n_obb, int n_cyl, int n_sph) {
  bool hit = false;
  const float4* e = env;
#pragma unroll 4
  for (int o = 0; o < n_aabb; ++o) hit |= Prim<kAabb>::hit(e + 2 * o, cx, cy, cz, r);
  e += 2 * n_aabb;
#pragma unroll 2
  for (int o = 0; o < n_obb; ++o) hit |= Prim<kObb>::hit(e + 5 * o, cx, cy, cz, r);
  e += 5 * n_obb;
#pragma unroll 2
  for (int o = 0; o < n_cyl; ++o) hit |= Prim<kCyl>::hit(e + 2 * o, cx, cy, cz, r);
  e += 2 * n_cyl;
#pragma unroll 4
  for (int o = 0; o < n_sph; ++o) hit |= Prim<kSph>::hit(e + o, cx, cy, cz, r);
  return hit;
}

// Two-stage test of one frame against the primitives of one type (Sec. III-A,
// hierarchical check): the frame's bounding sphere (bx, by, bz, br) against
// every primitive, 32 at a time; the flags of all active lanes are OR-ed, and
// the frame's fine spheres s0..s1-1 (centres staged in `stage`) are tested
// against the flagged primitives only.  The flag set is warp-uniform, so the
// second stage runs without divergence.  Returns this lane's fine verdict and
// adds the number of flagged primitives to *flagged.
template <int K>
__device__ __forceinline__ bool frame_two_stage(const float4* __restrict__ prims, int n, float bx, float by, float bz,
                                                float br, const float* __restrict__ stage,
                                                const float4* __restrict__ sph, int s0, int s1, bool active, int lane,
                                                uint32_t& flagged) {
  bool hit = false;
  for (int base = 0; base < n; base += 32) {
    const int m = min(32, n - base);
    uint32_t flags = 0;
#pragma unroll Prim<K>::kUnroll
    for (int k = 0; k < m; ++k)
      flags |= (uint32_t)Prim<K>::hit(prims + Prim<K>::kStride * (base + k), bx, by, bz, br) << k;
    flags = __reduce_or_sync(kFull, active ? flags : 0u);
    flagged += (uint32_t)__popc(flags);
    while (flags) {
      const int k = __ffs(flags) - 1;
      flags &= flags - 1;
      const float4* pk = prims + Prim<K>::kStride * (base + k);
      for (int s = s0; s < s1; ++s) {
        const float* st = stage + s * 96 + lane;
        hit |= Prim<K>::hit(pk, st[0], st[32], st[64], sph[s].w);
      }
    }
  }
  return hit;
}

// Packs a verdict (bit 63) and four per-type test counts (15 bits each,
// saturated; AABB lowest).
__device__ __forceinline__ unsigned long long pack_tests(bool hit, const uint32_t (&t)[4]) {
  unsigned long long r = (unsigned long long)hit << 63;
#pragma unroll
  for (int k = 0; k < 4; ++k) r |= (unsigned long long)min(t[k], 0x7fffu) << (15 * k);
  return r;
}

// Both stages of one frame against the whole environment, kept out of line so
// that the register budget of the caller is not set by it.  Returns the
// lane's verdict and its second-stage tests per primitive type (pack_tests).
static __device__ __noinline__ unsigned long long env_two_stage(const float4* __restrict__ env, int n_aabb, int n_obb,
                                                         int n_cyl, int n_sph, float bx, float by, float bz, float br,
                                                         const float* __restrict__ stage,
                                                         const float4* __restrict__ sph, int s0, int s1, bool active,
                                                         int lane) {
  uint32_t f[4] = {0, 0, 0, 0};
  bool hit = false;
  const float4* e = env;
  hit |= frame_two_stage<kAabb>(e, n_aabb, bx, by, bz, br, stage, sph, s0, s1, active, lane, f[kAabb]);
  e += 2 * n_aabb;
  hit |= frame_two_stage<kObb>(e, n_obb, bx, by, bz, br, stage, sph, s0, s1, active, lane, f[kObb]);
  e += 5 * n_obb;
  hit |= frame_two_stage<kCyl>(e, n_cyl, bx, by, bz, br, stage, sph, s0, s1, active, lane, f[kCyl]);
  e += 2 * n_cyl;
  hit |= frame_two_stage<kSph>(e, n_sph, bx, by, bz, br, stage, sph, s0, s1, active, lane, f[kSph]);
#pragma unroll
  for (int k = 0; k < 4; ++k) f[k] *= (uint32_t)(s1 - s0);
  return pack_tests(hit, f);
}

// Three-stage test of one frame for a warp whose lanes hold the states of
// one edge (the planner).  Stage A: one sphere (ux, uy, uz, ur) around every
// active lane's bounding sphere against the primitives, one primitive per
// lane.  Stage B: each lane's bounding sphere (bx, by, bz, br) against the
// primitives stage A touched.  Stage C: the fine spheres against the
// primitives some lane's bounding sphere touched.  Each sphere contains the
// next with a margin, so the verdict equals the one-stage test.  The
// lane-level tests of the three stages are added to *tests.
//
// Stages B and C of one primitive type for one batch of 32 primitives whose
// stage-A candidates are `cand`.
template <int K>
__device__ __forceinline__ bool frame_stages_bc(const float4* __restrict__ prims, int base, uint32_t cand, float bx,
                                                float by, float bz, float br, const float* __restrict__ stage,
                                                const float4* __restrict__ sph, int s0, int s1, bool active, int lane,
                                                uint32_t& tests) {
  bool hit = false;
  tests += 1u + (uint32_t)__popc(cand);
  uint32_t flags = 0;
  while (cand) {
    const int b = __ffs(cand) - 1;
    cand &= cand - 1;
    flags |= (uint32_t)Prim<K>::hit(prims + Prim<K>::kStride * (base + b), bx, by, bz, br) << b;
  }
  flags = __reduce_or_sync(kFull, active ? flags : 0u);
  tests += (uint32_t)(s1 - s0) * (uint32_t)__popc(flags);
  while (flags) {
    const int b = __ffs(flags) - 1;
    flags &= flags - 1;
    const float4* pk = prims + Prim<K>::kStride * (base + b);
    for (int s = s0; s < s1; ++s) {
      const float* st = stage + s * 96 + lane;
      hit |= Prim<K>::hit(pk, st[0], st[32], st[64], sph[s].w);
    }
  }
  return hit;
}

// The three stages of one frame (warp = one edge), out of line; same return.
// Stage A of all four primitive types runs first, kHalves x 32 primitives of
// each type per round (one or two per lane), so that a lane's tests of a round
// are independent; stages B and C then take the round's candidates in order.
// One instance per tile size: each planner kernel holds only the one it uses.
// kObb = false: the instance of the lean planner, whose batches hold no
// oriented boxes (their tests are not compiled in).
template <int kHalves, bool kObb>
static __device__ __noinline__ unsigned long long env_three_stage(const float4* __restrict__ env, int n_aabb,
                                                           int n_obb, int n_cyl, int n_sph, float ux, float uy,
                                                           float uz, float ur, float bx, float by, float bz, float br,
                                                           const float* __restrict__ stage,
                                                           const float4* __restrict__ sph, int s0, int s1,
                                                           bool active, int lane) {
  if (!kObb) n_obb = 0;
  uint32_t t[4] = {0, 0, 0, 0};
  bool hit = false;
  const float4* ea = env;
  const float4* eo = ea + 2 * n_aabb;
  const float4* ec = eo + 5 * n_obb;
  const float4* es = ec + 2 * n_cyl;
  const int nmax = max(max(n_aabb, n_obb), max(n_cyl, n_sph));
  for (int base = 0; base < nmax; base += 32 * kHalves) {
    bool na[kHalves], no[kHalves], nc[kHalves], ns[kHalves];
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      const int k = base + 32 * h + lane;
      na[h] = k < n_aabb && Prim<kAabb>::hit(ea + 2 * k, ux, uy, uz, ur);
      no[h] = k < n_obb && Prim<kObb>::hit(eo + 5 * k, ux, uy, uz, ur);
      nc[h] = k < n_cyl && Prim<kCyl>::hit(ec + 2 * k, ux, uy, uz, ur);
      ns[h] = k < n_sph && Prim<kSph>::hit(es + k, ux, uy, uz, ur);
    }
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      const int b0 = base + 32 * h;
      const uint32_t ca = __ballot_sync(kFull, na[h]), co = __ballot_sync(kFull, no[h]);
      const uint32_t cc = __ballot_sync(kFull, nc[h]), cs = __ballot_sync(kFull, ns[h]);
      // a type without stage-A candidates (warp-uniform) needs no stages B and C
      if (b0 < n_aabb) {
        if (ca) hit |= frame_stages_bc<kAabb>(ea, b0, ca, bx, by, bz, br, stage, sph, s0, s1, active, lane, t[kAabb]);
        else t[kAabb] += 1u;
      }
      if (b0 < n_obb) {
        if (co) hit |= frame_stages_bc<kObb>(eo, b0, co, bx, by, bz, br, stage, sph, s0, s1, active, lane, t[kObb]);
        else t[kObb] += 1u;
      }
      if (b0 < n_cyl) {
        if (cc) hit |= frame_stages_bc<kCyl>(ec, b0, cc, bx, by, bz, br, stage, sph, s0, s1, active, lane, t[kCyl]);
        else t[kCyl] += 1u;
      }
      if (b0 < n_sph) {
        if (cs) hit |= frame_stages_bc<kSph>(es, b0, cs, bx, by, bz, br, stage, sph, s0, s1, active, lane, t[kSph]);
        else t[kSph] += 1u;
      }
    }
  }
  return pack_tests(hit, t);
}

// Order-preserving map of binary32 to uint32 (and back): larger floats give
// larger keys, so integer warp reductions take exact float minima and maxima.
__device__ __forceinline__ uint32_t f2key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Sphere around the active lanes' spheres (centre (x, y, z), common radius r):
// centre of the lanes' bounding box, radius half its diagonal + r, enlarged by
// 1e-5 m and one part in 10^6 so that FP32 rounding keeps every lane inside.
// The box comes from six integer min / max warp reductions (exact).
__device__ __forceinline__ float4 warp_enclosing_sphere(float x, float y, float z, float r, bool active) {
  const float lx = key2f(__reduce_min_sync(kFull, f2key(active ? x : INFINITY)));
  const float ly = key2f(__reduce_min_sync(kFull, f2key(active ? y : INFINITY)));
  const float lz = key2f(__reduce_min_sync(kFull, f2key(active ? z : INFINITY)));
  const float hx = key2f(__reduce_max_sync(kFull, f2key(active ? x : -INFINITY)));
  const float hy = key2f(__reduce_max_sync(kFull, f2key(active ? y : -INFINITY)));
  const float hz = key2f(__reduce_max_sync(kFull, f2key(active ? z : -INFINITY)));
  const float dx = hx - lx, dy = hy - ly, dz = hz - lz;
  const float half = 0.5f * sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  return make_float4(0.5f * (lx + hx), 0.5f * (ly + hy), 0.5f * (lz + hz), (half + r) * 1.000001f + 1e-5f);
}

// ------------------------------------------------------------------ FK + CC
// Joint-value sources for state_collides: lane-private values staged in
// shared memory ([joint][lane]) or a point on a warp-uniform edge a -> b
// (both held in shared memory) at parameter t, exactly b at the endpoint.
struct LaneQ {
  const float* q;  // [kMaxDof][32]
  int lane;
  __device__ __forceinline__ float operator()(int i) const { return q[i * 32 + lane]; }
  __device__ __forceinline__ int poll() const { return 0; }
};

struct EdgeQ {
  const float* a;
  const float* b;
  float t;
  bool end;
  const int* solved;  // the problem's solved flag: once set, the edge's verdict no longer matters
  __device__ __forceinline__ float operator()(int i) const { return end ? b[i] : fmaf(t, b[i] - a[i], a[i]); }
  __device__ __forceinline__ int poll() const { return *reinterpret_cast<const volatile int*>(solved); }
};

// Collision test of one configuration per lane.  `stage` is this warp's
// [n_spheres + dof][3][32] shared-memory buffer of sphere centres (and, with
// kWarpVote, link group centres).  Without kWarpVote each lane tests its own
// state link by link, in chain order, and returns its own verdict.  With
// kWarpVote the lanes are the states of one edge: the joint loop only places
// and stages every sphere, then the links are tested against the environment
// from the distal end back (three stages per link) and the whole warp returns
// true as soon as any active lane collides (the edge verdict).  The joint loop
// is a runtime loop so that the obstacle loops exist once in the code.
template <bool kWarpVote, int kTile = 32, bool kLean = false, class QS>
__device__ __forceinline__ bool state_collides(const RobotHeader* __restrict__ R, const uint32_t* __restrict__ pair,
                                               const float* __restrict__ thr, const float4* __restrict__ env,
                                               int n_aabb, int n_obb, int n_cyl, int n_sph, const EsdfGrid& grid,
                                               float* __restrict__ stage, const QS& qs, bool active, int lane,
                                               WarpCount* wc) {
  static_assert(kTile == 32 || kTile == 64, "obstacle tile is 32 or 64 primitives per type");
  // kLean: an instance for batches without distance fields whose links all have
  // bounding spheres (the host checks); the other paths are not compiled in.
  const bool has_grid = !kLean && grid.v != nullptr;
  const bool has_prims = (n_aabb | n_obb | n_cyl | n_sph) != 0;
  const int dof = R->dof;
  // edge warps read the problem's solved flag now and look at it after
  // placing the spheres (the load's latency hides behind the FK)
  const int solved_early = (kWarpVote && lane == 0) ? qs.poll() : 0;
  // uniform work of this call, multiplied by the active lanes on the way out
  const unsigned long long na = (unsigned long long)__popc(__ballot_sync(kFull, active));
  uint32_t passes = 0, pairs = 0;
  uint32_t fine[4] = {0, 0, 0, 0};
  auto flush = [&]() {
    if (wc && lane == 0) {
      wc->fk_states += na;
      wc->sphere_tests += na * passes;
      wc->pair_tests += na * pairs;
#pragma unroll
      for (int k = 0; k < 4; ++k) wc->prim[k] += na * fine[k];
    }
  };
  float ax = 1.f, ay = 0.f, az = 0.f;  // rotation column 0 (local x in world)
  float bx = 0.f, by = 1.f, bz = 0.f;  // column 1
  float cx = 0.f, cy = 0.f, cz = 1.f;  // column 2
  float px = 0.f, py = 0.f, pz = 0.f;
  bool hit = false;
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
      // the hardware sine/cosine (absolute error about 2^-21 on [-pi, pi]: sphere
      // centres within about 1e-6 m of exact FK); the library routine beyond
      if (kLean || fabsf(qi) <= 3.2f)  // lean batches keep revolute joints within +-3.2
        __sincosf(qi, &s, &c);
      else
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

    const int s0 = R->sph_begin[i], s1 = R->sph_begin[i + 1];
    const float4 cb = R->coarse[i];
    const bool two = R->two_stage && cb.w > 0.f && has_prims;  // uniform
    const float4 gs = R->grp[i];
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (gs.w > 0.f) {  // group sphere of this link (equals cb when the link has a bounding sphere)
      gx = fmaf(ax, gs.x, fmaf(bx, gs.y, fmaf(cx, gs.z, px)));
      gy = fmaf(ay, gs.x, fmaf(by, gs.y, fmaf(cy, gs.z, py)));
      gz = fmaf(az, gs.x, fmaf(bz, gs.y, fmaf(cz, gs.z, pz)));
      if (kWarpVote) {  // staged for the self-collision first stage (edge warps only)
        float* gst = stage + (R->n_spheres + i) * 96 + lane;
        gst[0] = gx;
        gst[32] = gy;
        gst[64] = gz;
      }
    }
    for (int s = s0; s < s1; ++s) {
      const float4 o = R->sph[s];
      const float sx = fmaf(ax, o.x, fmaf(bx, o.y, fmaf(cx, o.z, px)));
      const float sy = fmaf(ay, o.x, fmaf(by, o.y, fmaf(cy, o.z, py)));
      const float sz = fmaf(az, o.x, fmaf(bz, o.y, fmaf(cz, o.z, pz)));
      float* st = stage + s * 96 + lane;
      st[0] = sx;
      st[32] = sy;
      st[64] = sz;
      if (kWarpVote) continue;  // edge warps test the environment in a second pass, distal links first
      if (has_grid) hit |= esdf_read(grid, sx, sy, sz) < o.w;  // the distance field, sphere by sphere
      if (!two) {
        hit |= sphere_hits_env(sx, sy, sz, o.w, env, n_aabb, n_obb, n_cyl, n_sph);
        passes++;
      }
    }
    if (two && !kWarpVote) {
      passes++;
      const unsigned long long r =
          env_two_stage(env, n_aabb, n_obb, n_cyl, n_sph, gx, gy, gz, cb.w, stage, R->sph, s0, s1, active, lane);
      hit |= (r >> 63) != 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) fine[k] += (uint32_t)((r >> (15 * k)) & 0x7fffu);
    }
  }
  if (kWarpVote) {
    // Another warp has solved the problem: the verdict no longer matters, and
    // the warp leaves with "collides" so that it stops at its next check.
    if (__shfl_sync(kFull, solved_early, 0)) {
      if (wc && lane == 0) wc->aborted = 1;
      flush();
      return true;
    }
    // The lanes are the states of one edge, all placed and staged above.  Test
    // the links against the environment from the last one back: collisions
    // come mostly at the distal links, and the first hit ends the check.  The
    // verdict is the OR of the same tests in any order.
    for (int i = dof - 1; i >= 0; --i) {
      const int s0 = R->sph_begin[i], s1 = R->sph_begin[i + 1];
      if (s0 == s1) continue;
      const float4 cb = R->coarse[i];
      const bool two = kLean || (R->two_stage && cb.w > 0.f && has_prims);  // uniform
      if (two) {
        if (has_grid) {
          for (int s = s0; s < s1; ++s) {
            const float* st = stage + s * 96 + lane;
            hit |= esdf_read(grid, st[0], st[32], st[64]) < R->sph[s].w;
          }
        }
        // the link's bounding sphere, staged as its group centre
        const float* gst = stage + (R->n_spheres + i) * 96 + lane;
        const float gx = gst[0], gy = gst[32], gz = gst[64];
        const float4 u = warp_enclosing_sphere(gx, gy, gz, cb.w, active);
        const unsigned long long r = env_three_stage<kTile / 32, !kLean>(env, n_aabb, n_obb, n_cyl, n_sph, u.x, u.y, u.z,
                                                                 u.w, gx, gy, gz, cb.w, stage, R->sph, s0, s1,
                                                                 active, lane);
        hit |= (r >> 63) != 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) fine[k] += (uint32_t)((r >> (15 * k)) & 0x7fffu);
      } else {
        for (int s = s0; s < s1; ++s) {
          const float4 o = R->sph[s];
          const float* st = stage + s * 96 + lane;
          const float sx = st[0], sy = st[32], sz = st[64];
          if (has_grid) hit |= esdf_read(grid, sx, sy, sz) < o.w;
          hit |= sphere_hits_env(sx, sy, sz, o.w, env, n_aabb, n_obb, n_cyl, n_sph);
          passes++;
        }
      }
      if (__any_sync(kFull, hit && active)) {
        flush();
        return true;
      }
    }
  }
  // Self-collision by link-pair blocks: when the lanes are the states of one
  // edge, a block's fine sphere pairs run only if the group spheres of its two
  // links overlap for some active lane (the group spheres contain the fine
  // ones, so the verdict is that of testing every pair).  Lanes holding
  // unrelated states would nearly always find one overlap, so they test every
  // pair.  Pairs within a block are sorted by their first sphere.
  const int nb = R->n_blocks;
  const int grp_base = R->n_spheres;  // stage slot of frame 0's group centre
  for (int b = 0; b < nb; ++b) {
    const uint32_t fr = R->blk_frames[b], rg = R->blk_range[b];
    const float bt = R->blk_thr[b];
    if (kWarpVote && bt < INFINITY) {
      const float* ga = stage + (grp_base + (int)(fr & 0xffffu)) * 96 + lane;
      const float* gb = stage + (grp_base + (int)(fr >> 16)) * 96 + lane;
      const float dx = ga[0] - gb[0], dy = ga[32] - gb[32], dz = ga[64] - gb[64];
      const bool near = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < bt;
      pairs++;
      if (!__any_sync(kFull, near && active)) continue;
    }
    const int k0 = (int)(rg & 0xffffu), k1 = (int)(rg >> 16);
    pairs += (uint32_t)(k1 - k0);
    int last_i = -1;
    float ix = 0.f, iy = 0.f, iz = 0.f;
    for (int k = k0; k < k1; ++k) {
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
    }
    if (kWarpVote) {
      if (__any_sync(kFull, hit && active)) {
        flush();
        return true;
      }
    }
  }
  flush();
  if (kWarpVote) return __any_sync(kFull, hit && active);
  return hit;
}

// Byte size of a warp's staging buffer of sphere centres: the robot's
// distinct spheres, then one group centre per frame (`slots` = spheres + dof).
__host__ __device__ inline int stage_bytes(int slots) { return slots * 96 * (int)sizeof(float); }

// Shared-memory image of a robot: header, then pairs, then thresholds.
__host__ __device__ inline int robot_smem_bytes(int n_pairs) {
  int b = (int)sizeof(RobotHeader) + n_pairs * 8;
  return (b + 15) & ~15;
}

// One configuration q [dof] checked by a whole warp (start / goal checks):
// every lane runs the same FK, lane l places spheres l, l + 32, ... , tests
// them against every primitive (or the distance field) and stages their
// centres (3 floats each at stage[3 s]); after a warp barrier lane l tests
// self pairs l, l + 32, ....  Each test is the arithmetic of state_collides's
// one-stage path, which the bounding-sphere stages reproduce exactly, so the
// verdict is the same.  Returns the warp-wide verdict.
static __device__ __noinline__ bool config_collides_warp(const RobotHeader* __restrict__ R, const uint32_t* __restrict__ pair,
                                                  const float* __restrict__ thr, const float4* __restrict__ env,
                                                  int n_aabb, int n_obb, int n_cyl, int n_sph, const EsdfGrid& grid,
                                                  float* __restrict__ stage, const float* __restrict__ q, int lane) {
  const bool has_grid = grid.v != nullptr;
  const int dof = R->dof;
  const float qv = lane < dof ? q[lane] : 0.f;  // one load per lane, broadcast per joint below
  float ax = 1.f, ay = 0.f, az = 0.f;
  float bx = 0.f, by = 1.f, bz = 0.f;
  float cx = 0.f, cy = 0.f, cz = 1.f;
  float px = 0.f, py = 0.f, pz = 0.f;
  bool hit = false;
  for (int i = 0; i < dof; ++i) {
    if (R->jparent[i] < 0) {
      ax = 1.f; ay = 0.f; az = 0.f;
      bx = 0.f; by = 1.f; bz = 0.f;
      cx = 0.f; cy = 0.f; cz = 1.f;
      const float4 b = R->jbase[i];
      px = b.x; py = b.y; pz = b.z;
    }
    const int ty = R->jtype[i];
    const float qi = __shfl_sync(kFull, qv, i);
    if (ty == kRevZ || ty == kRevY || ty == kRevX) {
      float s, c;
      sincosf(qi, &s, &c);
      if (ty == kRevZ) {
        const float nx = fmaf(c, ax, s * bx), ny = fmaf(c, ay, s * by), nz = fmaf(c, az, s * bz);
        bx = fmaf(c, bx, -s * ax); by = fmaf(c, by, -s * ay); bz = fmaf(c, bz, -s * az);
        ax = nx; ay = ny; az = nz;
      } else if (ty == kRevY) {
        const float nx = fmaf(c, ax, -s * cx), ny = fmaf(c, ay, -s * cy), nz = fmaf(c, az, -s * cz);
        cx = fmaf(c, cx, s * ax); cy = fmaf(c, cy, s * ay); cz = fmaf(c, cz, s * az);
        ax = nx; ay = ny; az = nz;
      } else {
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
    const int s0 = R->sph_begin[i], s1 = R->sph_begin[i + 1];
    for (int s = s0 + lane; s < s1; s += 32) {
      const float4 o = R->sph[s];
      const float sx = fmaf(ax, o.x, fmaf(bx, o.y, fmaf(cx, o.z, px)));
      const float sy = fmaf(ay, o.x, fmaf(by, o.y, fmaf(cy, o.z, py)));
      const float sz = fmaf(az, o.x, fmaf(bz, o.y, fmaf(cz, o.z, pz)));
      stage[3 * s] = sx;
      stage[3 * s + 1] = sy;
      stage[3 * s + 2] = sz;
      if (has_grid) hit |= esdf_read(grid, sx, sy, sz) < o.w;
      hit |= sphere_hits_env(sx, sy, sz, o.w, env, n_aabb, n_obb, n_cyl, n_sph);
    }
  }
  __syncwarp();
  const int np = R->n_pairs;
  for (int k = lane; k < np; k += 32) {
    const uint32_t pr = pair[k];
    const int i = (int)(pr & 0xffffu), j = (int)(pr >> 16);
    const float dx = stage[3 * i] - stage[3 * j], dy = stage[3 * i + 1] - stage[3 * j + 1],
                dz = stage[3 * i + 2] - stage[3 * j + 2];
    hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < thr[k];
  }
  __syncwarp();
  return __any_sync(kFull, hit);
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
