// prrtc_plan.cu -- the pRRTC expansion loop on the device (Alg. 1 with
// Alg. 2), batched over many problems in one persistent launch.
//
// Layout (GB300-first):
//   * A block stages one problem's robot tables and obstacle set in shared
//     memory (TMA bulk copies) and runs `warps` independent workers on it.  A
//     worker is one warp executing Alg. 1 iterations: the paper's block-level
//     parallel iterations (Sec. III) map to warps, its thread-level NN and CC
//     to lanes.
//   * Blocks take problems from a device work queue (an atomic ticket) and,
//     when their problem is solved or out of budget, move to the next unsolved
//     one, so hard problems soak up the blocks freed by easy ones.
//   * Both trees of a problem live in global memory (L2-resident at these
//     sizes).  Rows start as NaN; a worker reserves a row with one atomicAdd,
//     writes the parent, fences, then the coordinates.  Readers scan with L2
//     loads and skip rows whose distance is NaN, so a row is used only once
//     all its coordinates are final (each word changes NaN -> value once).
//   * Serial mode runs one worker per problem; it performs exactly the
//     iterations of the serial Alg. 1 in order.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <map>
#include <mutex>

#include "prrtc.h"
#include "prrtc_launch.h"

namespace prrtc {

namespace {

static_assert(sizeof(RobotHeader) % 16 == 0, "robot header must stay 16-byte aligned for TMA");
static_assert(offsetof(RobotDev, pair) % 16 == 0 && offsetof(RobotDev, thr) % 16 == 0, "TMA alignment");

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// Time slice of a resumable launch spent?
__device__ __forceinline__ bool slice_over(const PlanGlobals* g) {
  return g->slice_ns && globaltimer_ns() - g->t0 > g->slice_ns;
}


// Halton point `index`, coordinate j (the paper's sampler, Sec. IV-A): the
// radical inverse of index in the j-th prime base -- its base-p digits
// mirrored about the radix point -- formed as an exact integer fraction and
// divided once in FP64.  The primes 2..53 are packed six bits each.
__device__ __forceinline__ float halton_coord(uint32_t index, int j) {
  constexpr uint64_t kPrimesLo = 0x7574d134b1c50c2ull;  // 2, 3, 5, ..., 29
  constexpr uint64_t kPrimesHi = 0xd6fae995full;        // 31, 37, 41, 43, 47, 53
  const uint32_t b = (uint32_t)((j < 10 ? (kPrimesLo >> (6 * j)) : (kPrimesHi >> (6 * (j - 10)))) & 63u);
  uint64_t num = 0, den = 1;
  for (uint32_t i = index; i; i /= b) {
    num = num * b + i % b;
    den *= b;
  }
  return (float)((double)num / (double)den);
}

// Warp-uniform vectors of one worker, in shared memory; lane j owns element j.
struct WarpVecs {
  float* rnd;   // sample c_rand
  float* a;     // edge start
  float* b;     // edge end
};
constexpr int kWarpVecFloats = 3 * kMaxDof;
constexpr int kCountFloats = (int)(sizeof(WarpCount) / sizeof(float));

struct Ctx {
  const PlanGlobals* g;
  const ProblemDesc* D;
  ProblemState* S;
  const RobotHeader* R;
  const uint32_t* pair;
  const float* thr;
  const float4* env;
  float* stage;
  WarpVecs v;
  WarpCount* cnt;  // this warp's counters (shared memory, lane 0 writes)
  int lane;
};

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(kFull, x, off);
  return x;
}

// Element `lane` of row `idx` (0 for lanes past the row width).
__device__ __forceinline__ float row_elem(const float* __restrict__ nodes, int idx, int dpad, int lane) {
  return lane < dpad ? __ldcg(nodes + (size_t)idx * dpad + lane) : 0.f;
}

// NEAREST_NEIGHBOR (Sec. III-C): each lane scans a strided slice of the
// tree, then a butterfly reduction over the warp; ties go to the lowest index.
// Rows are dpad floats (4, 8, 12 or 16) read as float4 from L2.
__device__ __noinline__ int nearest(const float* __restrict__ nodes, int n, int dpad, const float* __restrict__ qv,
                                    int lane, unsigned long long* nn_nodes) {
  float q[kMaxDof];
#pragma unroll
  for (int j = 0; j < kMaxDof; ++j) q[j] = (j < dpad) ? qv[j] : 0.f;
  const int nq = dpad >> 2;
  float best = FLT_MAX;
  int bi = INT_MAX;
  int i = lane;
  for (; i + 32 < n; i += 64) {
    const float4* r0 = reinterpret_cast<const float4*>(nodes + (size_t)i * dpad);
    const float4* r1 = reinterpret_cast<const float4*>(nodes + (size_t)(i + 32) * dpad);
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDof / 4; ++k) {
      if (k < nq) {
        const float4 a = __ldcg(r0 + k), b = __ldcg(r1 + k);
        float t;
        t = q[4 * k + 0] - a.x; d0 = fmaf(t, t, d0);
        t = q[4 * k + 1] - a.y; d0 = fmaf(t, t, d0);
        t = q[4 * k + 2] - a.z; d0 = fmaf(t, t, d0);
        t = q[4 * k + 3] - a.w; d0 = fmaf(t, t, d0);
        t = q[4 * k + 0] - b.x; d1 = fmaf(t, t, d1);
        t = q[4 * k + 1] - b.y; d1 = fmaf(t, t, d1);
        t = q[4 * k + 2] - b.z; d1 = fmaf(t, t, d1);
        t = q[4 * k + 3] - b.w; d1 = fmaf(t, t, d1);
      }
    }
    if (d0 < best) { best = d0; bi = i; }
    if (d1 < best) { best = d1; bi = i + 32; }
  }
  if (i < n) {
    const float4* r0 = reinterpret_cast<const float4*>(nodes + (size_t)i * dpad);
    float d0 = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDof / 4; ++k) {
      if (k < nq) {
        const float4 a = __ldcg(r0 + k);
        float t;
        t = q[4 * k + 0] - a.x; d0 = fmaf(t, t, d0);
        t = q[4 * k + 1] - a.y; d0 = fmaf(t, t, d0);
        t = q[4 * k + 2] - a.z; d0 = fmaf(t, t, d0);
        t = q[4 * k + 3] - a.w; d0 = fmaf(t, t, d0);
      }
    }
    if (d0 < best) { best = d0; bi = i; }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const float ob = __shfl_xor_sync(kFull, best, off);
    const int oi = __shfl_xor_sync(kFull, bi, off);
    if (ob < best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) *nn_nodes += (unsigned long long)n;
  return bi;
}

// Alg. 2 lines 3-5: the N states a + (k/N)(b - a), k = 1..N, of the edge held
// in c.v.a / c.v.b, one per lane (several passes if N > 32); false at the
// first colliding state.  kTile: obstacles per type per first-stage round.
template <int kTile, bool kLean>
__device__ __forceinline__ bool edge_free(const Ctx& c, int N) {
  if (c.lane == 0) {
    c.cnt->edges++;
    c.cnt->edge_states += (unsigned long long)N;
  }
  const float fN = (float)N;
  for (int base = 0; base < N; base += 32) {
    const int k = base + c.lane + 1;
    const bool active = k <= N;
    const int kk = active ? k : N;
    const EdgeQ qs{c.v.a, c.v.b, __fdiv_rn((float)kk, fN), kk == N, &c.S->solved};
    if (state_collides<true, kTile, kLean>(c.R, c.pair, c.thr, c.env, c.D->env.n_aabb, c.D->env.n_obb, c.D->env.n_cyl,
                                    c.D->env.n_sph, c.D->env.esdf, c.stage, qs, active, c.lane, c.cnt)) {
      __syncwarp();  // lane 0 may have just set the flag
      if (c.cnt->aborted) {
        // the problem was solved meanwhile and the check stopped early: this
        // edge is not counted as checked
        __syncwarp();
        if (c.lane == 0) {
          c.cnt->aborted = 0;
          c.cnt->edges--;
          c.cnt->edge_states -= (unsigned long long)N;
        }
        __syncwarp();
        return false;
      }
      // the states of earlier passes were all shown free, and one state of this
      // pass collides; the other states of the pass stopped early
      if (c.lane == 0) c.cnt->verdict_states += (unsigned long long)base + 1ull;
      return false;
    }
  }
  if (c.lane == 0) c.cnt->verdict_states += (unsigned long long)N;
  return true;
}

// Append the row held by lane j's `val` (element j) to tree t; returns its
// index or -1 when the tree is full.
__device__ __forceinline__ int insert(const Ctx& c, int t, float val, int parent) {
  int idx = 0;
  if (c.lane == 0) idx = atomicAdd(&c.S->count[t], 1);
  idx = __shfl_sync(kFull, idx, 0);
  if (idx >= c.D->cap) {
    if (c.lane == 0) c.cnt->insert_fail++;
    return -1;
  }
  if (c.lane == 0) {
    __stcg(c.D->parent[t] + idx, parent);
    __threadfence();
  }
  __syncwarp();
  if (c.lane < c.D->dpad) __stcg(c.D->nodes[t] + (size_t)idx * c.D->dpad + c.lane, val);
  __syncwarp();
  return idx;
}

// Parent of a node, waiting (bounded) for a row still being written.
__device__ __forceinline__ int parent_of(const int* par, int node, int* err) {
  int p = ld_volatile(par + node);
  for (int spin = 0; p == kUnsetParent && spin < (1 << 20); ++spin) p = ld_volatile(par + node);
  if (p == kUnsetParent) *err = 1;
  return p;
}

// PATH(T_a, T_b) by the winning warp: root(T_a) .. join .. root(T_b).  The two
// join rows hold the same configuration; the copy in T_b is dropped when T_a
// was extended and vice versa, so the path lists each waypoint once.
// Out of line: it runs once per solved problem, and kept inline its code (about
// a fifth of the planner's) would sit inside the hot iteration loop.
__device__ __noinline__ void extract_path(const Ctx& c, int s, int js, int jo) {
  const ProblemDesc* D = c.D;
  int err = 0;
  if (c.g->debug_wait_polls) {
    // test hook: the bounded wait of a parent walk, on a flag nothing sets
    if (c.lane == 0) {
      const volatile int* f = &c.S->never_set;
      for (uint32_t k = 0; *f == 0 && k < c.g->debug_wait_polls; ++k) {
      }
      err = (*f == 0) ? 1 : 0;
    }
    err = __shfl_sync(kFull, err, 0);
  }
  // the T_a-side chain (root first) then the T_b-side chain without its join row
  const int a_join = (s == 0) ? js : jo;
  const int b_join = (s == 0) ? jo : js;
  // Lane 0 walks T_a from its join row to the root and lane 1 T_b, at the same
  // time; each records the rows it visits in the warp's staging area (the
  // sphere-centre scratch, free now) while they fit, so that the path can be
  // laid out without a second walk.  When both trees' parent arrays fit in
  // half of the area, the warp first copies them there with coalesced loads
  // and the walks run in shared memory (a walk in global memory pays one L2
  // round trip per step).  Every row on a chain had its parent written before
  // it was linked; an entry still unset in the copy falls back to the global
  // read.
  const int area = (c.R->n_spheres + c.R->dof) * 96;  // ints
  int n0 = 0, n1 = 0;
  if (c.lane == 0) {
    n0 = min(ld_relaxed(&c.S->count[0]), D->cap);
    n1 = min(ld_relaxed(&c.S->count[1]), D->cap);
  }
  n0 = __shfl_sync(kFull, n0, 0);
  n1 = __shfl_sync(kFull, n1, 0);
  const bool in_smem = n0 + n1 <= area / 2;
  int* sp = reinterpret_cast<int*>(c.stage);
  if (in_smem) {
    for (int k = c.lane; k < n0; k += 32) sp[k] = __ldcg(D->parent[0] + k);
    for (int k = c.lane; k < n1; k += 32) sp[n0 + k] = __ldcg(D->parent[1] + k);
    __syncwarp();
  }
  const int rec_cap = in_smem ? area / 4 : area / 2;  // ints per side
  int* rec_base = reinterpret_cast<int*>(c.stage) + (in_smem ? area / 2 : 0);
  int* rec = rec_base + (c.lane & 1) * rec_cap;
  int n = 0;
  if (c.lane < 2) {
    const int t = c.lane, nt = t == 0 ? n0 : n1;
    const int* par = D->parent[t];
    const int* spt = sp + (t == 0 ? 0 : n0);
    int x = t == 0 ? a_join : b_join;
    while (x >= 0 && n <= D->cap) {
      if (n < rec_cap) rec[n] = x;
      ++n;
      int p = kUnsetParent;
      if (in_smem && x < nt) p = spt[x];
      x = (p != kUnsetParent) ? p : parent_of(par, x, &err);
    }
  }
  const int na = __shfl_sync(kFull, n, 0), nb = __shfl_sync(kFull, n, 1);
  err = __reduce_or_sync(kFull, err);
  const int K = na + nb - 1;
  if (c.lane == 0) c.S->path_n = K;
  if (err || na > D->cap || nb > D->cap) {
    if (c.lane == 0) {
      c.S->path_status = PRRTC_ERR_TIMEOUT;
      atomicExch(&const_cast<PlanGlobals*>(c.g)->error, PRRTC_ERR_TIMEOUT);
    }
    return;
  }
  if (K > c.g->path_cap) {
    if (c.lane == 0) c.S->path_status = PRRTC_PATH_OVERFLOW;
    return;
  }
  __syncwarp();
  const int* rec_a = rec_base;
  const int* rec_b = rec_a + rec_cap;
  if (na <= rec_cap) {
    for (int r = c.lane; r < na; r += 32) D->path_idx[r] = rec_a[na - 1 - r];
  } else if (c.lane == 0) {  // a chain longer than the record: walk it again
    int pos = na - 1;
    for (int x = a_join; x >= 0 && pos >= 0; x = parent_of(D->parent[0], x, &err)) D->path_idx[pos--] = x;
  }
  if (nb <= rec_cap) {
    for (int k = c.lane; k < nb - 1; k += 32) D->path_idx[na + k] = (1 << 30) | rec_b[k + 1];
  } else if (c.lane == 1) {
    int pos = na;
    for (int x = parent_of(D->parent[1], b_join, &err); x >= 0 && pos < K; x = parent_of(D->parent[1], x, &err))
      D->path_idx[pos++] = (1 << 30) | x;
  }
  __threadfence_block();
  __syncwarp();
  const int dof = D->dof, dpad = D->dpad;
  double seg = 0.0;
  for (int r = c.lane; r < K; r += 32) {
    const int code = D->path_idx[r];
    const float* row = D->nodes[code >> 30] + (size_t)(code & ((1 << 30) - 1)) * dpad;
    for (int j = 0; j < dof; ++j) D->path[(size_t)r * dof + j] = __ldcg(row + j);
    if (r > 0) {
      const int pc = D->path_idx[r - 1];
      const float* prow = D->nodes[pc >> 30] + (size_t)(pc & ((1 << 30) - 1)) * dpad;
      double s2 = 0.0;
      for (int j = 0; j < dof; ++j) {
        const double d = (double)__ldcg(row + j) - (double)__ldcg(prow + j);
        s2 += d * d;
      }
      seg += sqrt(s2);
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) seg += __shfl_xor_sync(kFull, seg, off);
  if (c.lane == 0) {
    c.S->cost = seg;
    c.S->path_status = err ? PRRTC_ERR_TIMEOUT : PRRTC_SOLVED;
    if (err) atomicExch(&const_cast<PlanGlobals*>(c.g)->error, PRRTC_ERR_TIMEOUT);
  }
}

// Draw from a learned mixture (element `lane` of the configuration): the
// component from word 21 against the cumulative softmax of the logits, then
// z_j from Box-Muller on words 22 + 2m, 23 + 2m (m = j / 2; words >= 32 come
// from Philox blocks 8-9), u_j = mean + exp(log_sigma) z_j, mapped from [-1, 1]
// to the joint limits and clamped to them.
__device__ __forceinline__ float mixture_draw(const float* __restrict__ gmm, const RobotHeader* R, uint32_t pid,
                                              uint32_t it, uint2 key, uint32_t w, int lane, int dof) {
  uint32_t w2 = 0;
  {
    const uint4 ph = philox4x32_10(make_uint4(pid, it, 8u + (uint32_t)((lane >> 2) & 1), 0u), key);
    w2 = ((lane & 3) == 0) ? ph.x : ((lane & 3) == 1) ? ph.y : ((lane & 3) == 2) ? ph.z : ph.w;
  }
  const float uk = u24(__shfl_sync(kFull, w, 21));
  float mx = -INFINITY;
#pragma unroll
  for (int k = 0; k < kMixK; ++k) mx = fmaxf(mx, gmm[k]);
  float tot = 0.f;
#pragma unroll
  for (int k = 0; k < kMixK; ++k) tot += expf(gmm[k] - mx);
  int comp = kMixK - 1;
  float cum = 0.f;
#pragma unroll
  for (int k = 0; k < kMixK; ++k) {
    cum += expf(gmm[k] - mx) / tot;
    if (uk < cum && comp == kMixK - 1 && k < kMixK - 1) comp = k;
  }
  const int m = lane >> 1;
  const int ia = 22 + 2 * m, ib = 23 + 2 * m;
  const uint32_t a_lo = __shfl_sync(kFull, w, ia & 31), a_hi = __shfl_sync(kFull, w2, (ia - 32) & 31);
  const uint32_t b_lo = __shfl_sync(kFull, w, ib & 31), b_hi = __shfl_sync(kFull, w2, (ib - 32) & 31);
  if (lane >= dof) return 0.f;
  const uint32_t wa = ia < 32 ? a_lo : a_hi, wb = ib < 32 ? b_lo : b_hi;
  const float u1 = (float)((wa >> 8) + 1u) * (1.0f / 16777216.0f);
  const float u2 = (float)(wb >> 8) * (1.0f / 16777216.0f);
  const float rad = sqrtf(-2.f * logf(u1));
  float sn, cs;
  sincospif(2.f * u2, &sn, &cs);
  const float z = (lane & 1) ? rad * sn : rad * cs;
  const float un = fmaf(expf(gmm[kMixK + kMixK * kMaxDof + comp * kMaxDof + lane]), z, gmm[kMixK + comp * kMaxDof + lane]);
  const float lo = R->lo[lane], span = R->span[lane];
  return fminf(fmaxf(fmaf(0.5f * (un + 1.f), span, lo), lo), lo + span);
}

// Alg. 1 line 4, RANDOM_CONFIG for iteration `it` (element `lane` of the
// sample): Philox words of counter {pid, it, blk, 0}, lane l holding word l
// (blocks 0..7).  Word 0 draws the goal bias (the root of T_o, tree `o`),
// words 1..dof the uniform configuration; with a learned mixture, word 20
// draws learned-vs-uniform, word 21 the component, words 22.. Box-Muller
// pairs.  The Halton sampler takes point it + 1 + offset instead of the
// uniform words (point 0 is the origin of the unit cube).
template <bool kLean>
__device__ __forceinline__ float random_config(const Ctx& c, int it, int o, bool* goal_sample) {
  const PlanGlobals* g = c.g;
  const ProblemDesc* D = c.D;
  const RobotHeader* R = c.R;
  const int lane = c.lane, dof = D->dof;
  const uint2 key = make_uint2(D->key_lo, D->key_hi);
  const uint4 ph = philox4x32_10(make_uint4(D->pid, (uint32_t)it, (uint32_t)(lane >> 2), 0u), key);
  const uint32_t w = ((lane & 3) == 0) ? ph.x : ((lane & 3) == 1) ? ph.y : ((lane & 3) == 2) ? ph.z : ph.w;
  const uint32_t w0 = __shfl_sync(kFull, w, 0);
  const uint32_t wj = __shfl_sync(kFull, w, (lane + 1) & 31);
  const uint32_t wl = __shfl_sync(kFull, w, 20);
  *goal_sample = (w0 >> 8) < g->bias_thr;
  if (*goal_sample) return row_elem(D->nodes[o], 0, D->dpad, lane);
  if (!kLean && D->gmm && (wl >> 8) < g->learned_thr)
    return mixture_draw(D->gmm, R, D->pid, (uint32_t)it, key, w, lane, dof);
  if (!kLean && g->sampler == PRRTC_SAMPLER_HALTON)
    return (lane < dof) ? fmaf(halton_coord((uint32_t)it + 1u + g->halton_offset, lane), R->span[lane], R->lo[lane])
                        : 0.f;
  return (lane < dof) ? fmaf(u24(wj), R->span[lane], R->lo[lane]) : 0.f;
}

// Alg. 1 iterations of one worker warp on one problem until it is solved,
// out of budget or out of time.  Lane j holds element j of every vector.
template <int kTile, bool kLean>
__device__ void worker(const Ctx& c) {
  const PlanGlobals* g = c.g;
  const ProblemDesc* D = c.D;
  ProblemState* S = c.S;
  const int lane = c.lane;
  const int dpad = D->dpad;
  const int cap = D->cap;
  const float range = g->range;
  const float res = g->resolution;
  const int n_full = g->n_full;
  const bool mine = lane < dpad;
  int claim_next = 0, claim_left = 0;  // iteration ids claimed by lane 0 and not yet run
  for (;;) {
    int stop = 0, it = 0;
    if (lane == 0) {
      // a spent time slice stops the worker before it takes an iteration
      // ticket; the problem resumes in the next launch of a resumable batch
      stop = ld_volatile(&S->done) | ld_volatile(&S->solved) | (slice_over(g) ? 1 : 0);
      if (!stop) {
        if (claim_left == 0) {  // `expansions` consecutive ids per claim of the counter
          claim_next = atomicAdd(&S->iter, g->expansions);
          claim_left = g->expansions;
        }
        it = claim_next++;
        --claim_left;
      }
    }
    stop = __shfl_sync(kFull, stop, 0);
    if (stop) break;
    it = __shfl_sync(kFull, it, 0);
    if (it >= g->max_iters) {
      if (lane == 0) atomicExch(&S->done, 1);
      break;
    }
    // Every value a warp-wide decision rests on is read by lane 0 and broadcast:
    // lanes that load a counter or a clock themselves may see different values
    // (other warps change them, and the lanes need not load in one instruction).
    int late = 0;
    if (lane == 0) late = g->time_limit_ns && globaltimer_ns() - g->t0 > g->time_limit_ns;
    if (__shfl_sync(kFull, late, 0)) {
      if (lane == 0) {
        S->timed_out = 1;
        atomicExch(&S->done, 1);
      }
      break;
    }
    if (lane == 0) c.cnt->iterations++;

    // Alg. 1 line 3: extend the smaller tree (ties: T_a).
    int na = 0, nb = 0;
    if (lane == 0) {
      na = min(ld_relaxed(&S->count[0]), cap);
      nb = min(ld_relaxed(&S->count[1]), cap);
    }
    na = __shfl_sync(kFull, na, 0);
    nb = __shfl_sync(kFull, nb, 0);
    const int s = (na <= nb) ? 0 : 1;
    const int o = 1 - s;
    const int n_s = s ? nb : na;

    // line 4: RANDOM_CONFIG
    bool goal_sample;
    const float crand = random_config<kLean>(c, it, o, &goal_sample);
    if (mine) c.v.rnd[lane] = crand;
    __syncwarp();

    // line 5: nearest node of T_s.
    const int nn = nearest(D->nodes[s], n_s, dpad, c.v.rnd, lane, &c.cnt->nn_nodes);
    const float cnn = row_elem(D->nodes[s], nn, dpad, lane);

    // Alg. 2: steer from c_nn toward c_rand by at most delta.
    const float diff = crand - cnn;
    const float d2 = warp_sum(diff * diff);
    if (!(d2 > 0.f)) continue;
    const float dist = __fsqrt_rn(d2);
    // Dynamic-domain sampling (Yershova et al. 2005): a random sample farther
    // than the nearest node's radius ends the iteration.  NaN = unbounded
    // (every comparison with NaN is false).
    const bool dd = !kLean && g->dd_radius > 0.f;  // lean batches have it off
    if (dd && !goal_sample) {
      float rad = 0.f;
      if (lane == 0) rad = __ldcg(D->radius[s] + nn);  // other warps adapt it
      if (dist > __shfl_sync(kFull, rad, 0)) {
        if (lane == 0) c.cnt->dd_rejected++;
        continue;
      }
    }
    float cnew;
    int N;
    if (dist > range) {
      cnew = fmaf(diff, __fdiv_rn(range, dist), cnn);
      N = n_full;
    } else {
      cnew = crand;
      N = (int)ceilf(__fdiv_rn(dist, res));
    }
    if (N < 1) N = 1;
    if (mine) {
      c.v.a[lane] = cnn;
      c.v.b[lane] = cnew;
    }
    __syncwarp();

    // Phase 0 checks and adds c_new (Alg. 1 lines 5-7); phase i >= 1 is the
    // i-th greedy connect step toward c_nno (lines 9-15).  One edge check
    // site serves both.
    int prev = nn;        // row the current edge starts from (tree s)
    int nno = -1, n_ext = 0;
    float ct = 0.f, Dd = 0.f;
    float bval = cnew;    // element `lane` of the edge end
    bool connected = false;
    for (int phase = 0;; ++phase) {
      if (phase > 0) {
        int solved = 0;
        if (lane == 0) solved = ld_volatile(&S->solved);
        if (__shfl_sync(kFull, solved, 0)) break;
      }
      const bool free_edge = edge_free<kTile, kLean>(c, N);
      if (phase == 0 && dd && lane == 0) {
        // adaptive radius of the nearest node (Jaillet et al. 2005): a bounded
        // radius grows after a free extension; a collision bounds an unbounded
        // radius to dd_radius and shrinks a bounded one, not below the floor
        float* rp = D->radius[s] + nn;
        const float r = __ldcg(rp);
        if (free_edge) {
          if (!isnan(r)) __stcg(rp, r * (1.f + g->dd_alpha));
        } else {
          __stcg(rp, isnan(r) ? g->dd_radius : fmaxf(r * (1.f - g->dd_alpha), g->dd_min_radius));
        }
      }
      if (!free_edge) break;
      const int added = insert(c, s, bval, prev);
      if (added < 0) break;
      prev = added;
      if (phase == 0) {
        // line 8: nearest node of T_o to c_new, and the connect length.
        int n_o = 0;
        if (lane == 0) n_o = min(ld_relaxed(&S->count[o]), cap);
        n_o = __shfl_sync(kFull, n_o, 0);
        nno = nearest(D->nodes[o], n_o, dpad, c.v.b, lane, &c.cnt->nn_nodes);
        ct = row_elem(D->nodes[o], nno, dpad, lane);
        const float dd = ct - cnew;
        Dd = __fsqrt_rn(warp_sum(dd * dd));
        n_ext = (Dd > 0.f) ? (int)ceilf(__fdiv_rn(Dd, range)) : 0;
      }
      if (phase == n_ext) {
        connected = true;
        break;
      }
      // next connect step: from the row just added toward c_new + (i delta / D)(c_nno - c_new)
      const int i = phase + 1;
      if (i < n_ext) {
        bval = fmaf(__fdiv_rn((float)i * range, Dd), ct - cnew, cnew);
        N = n_full;
      } else {
        bval = ct;
        const float len = Dd - (float)(n_ext - 1) * range;
        N = (int)ceilf(__fdiv_rn(len, res));
        if (N < 1) N = 1;
      }
      if (mine) {
        c.v.a[lane] = c.v.b[lane];
        c.v.b[lane] = bval;
      }
      __syncwarp();
    }
    if (!connected) continue;

    // line 16: the trees meet -- the first worker to claim the problem writes PATH.
    int won = 0;
    if (lane == 0) won = (atomicCAS(&S->solved, 0, 1) == 0);
    won = __shfl_sync(kFull, won, 0);
    if (won) {
      if (lane == 0) {
        S->t_solve = globaltimer_ns();
        S->s_tree = s;
        S->join_s = prev;
        S->join_o = nno;
      }
      extract_path(c, s, prev, nno);
      __threadfence();
      if (lane == 0) atomicExch(&S->done, 1);
    }
    break;
  }
}

// ------------------------------------------------------------------ lockstep rounds
// The concurrency of Sec. III on a fixed schedule (PRRTC_MODE_LOCKSTEP): in
// round r, worker b runs iteration r B + b against the trees as they stood
// when the round began, holding its new rows back in its slice of D->held;
// at the end of the round the rows are appended in worker order and the
// connected worker that checked the fewest edges (ties: lowest b) wins.
// Virtual worker b runs on warp b % warps of the problem's block.

// One worker's record for a round (kHeldMeta ints of D->held_meta).
struct LockstepHeld {
  int n;          // rows held back
  int nn;         // snapshot row of T_s the first row extends
  int nno;        // snapshot row of T_o the connect aims at
  int connected;  // the connect reached c_nno
  int edges;      // edges this iteration checked
  int dd_node;    // node whose dynamic-domain radius the extension updates, -1 none
  int dd_free;    // that edge was free
  int offset;     // first row of this worker among the round's appended rows
};
static_assert(sizeof(LockstepHeld) == kHeldMeta * sizeof(int), "lockstep record layout");

// Alg. 1 lines 4-15 of iteration `it` against T_s = tree s (its first n_s
// rows) and T_o (its first n_o rows); new rows go to `rows` (held_rows x
// dpad), the outcome to *h (written by lane 0).
__device__ void lockstep_iteration(const Ctx& c, int it, int s, int n_s, int n_o, LockstepHeld* h, float* rows) {
  const PlanGlobals* g = c.g;
  const ProblemDesc* D = c.D;
  const int lane = c.lane, dpad = D->dpad, cap = D->cap;
  const int o = 1 - s;
  const bool mine = lane < dpad;
  const float range = g->range, res = g->resolution;
  const bool dd = g->dd_radius > 0.f;
  int n = 0, nn = -1, nno = -1, connected = 0, edges = 0, dd_node = -1, dd_free = 0;
  if (lane == 0) c.cnt->iterations++;
  do {
    bool goal_sample;
    const float crand = random_config<false>(c, it, o, &goal_sample);
    if (mine) c.v.rnd[lane] = crand;
    __syncwarp();
    // line 5: nearest node of T_s as the round found it
    nn = nearest(D->nodes[s], n_s, dpad, c.v.rnd, lane, &c.cnt->nn_nodes);
    const float cnn = row_elem(D->nodes[s], nn, dpad, lane);
    const float diff = crand - cnn;
    const float d2 = warp_sum(diff * diff);
    if (!(d2 > 0.f)) break;
    const float dist = __fsqrt_rn(d2);
    if (dd && !goal_sample && dist > __ldcg(D->radius[s] + nn)) {  // NaN radius: unbounded
      if (lane == 0) c.cnt->dd_rejected++;
      break;
    }
    float cnew;
    int N;
    if (dist > range) {
      cnew = fmaf(diff, __fdiv_rn(range, dist), cnn);
      N = g->n_full;
    } else {
      cnew = crand;
      N = (int)ceilf(__fdiv_rn(dist, res));
    }
    if (N < 1) N = 1;
    if (mine) {
      c.v.a[lane] = cnn;
      c.v.b[lane] = cnew;
    }
    __syncwarp();
    // phase 0: the extension (Alg. 2); phase i >= 1: greedy connect step i
    float ct = 0.f, Dd = 0.f, bval = cnew;
    int n_ext = 0;
    for (int phase = 0;; ++phase) {
      const bool free_edge = edge_free<32, false>(c, N);  // lockstep: 32-obstacle tiles
      ++edges;
      if (phase == 0 && dd) {
        dd_node = nn;
        dd_free = free_edge ? 1 : 0;
      }
      if (!free_edge) break;
      // line 7 / 13, held back; a tree full counting this worker's rows takes no more
      if (n_s + n >= cap) break;
      if (n >= D->held_rows) {  // the host sizes held_rows for the longest connect
        if (lane == 0) atomicExch(&const_cast<PlanGlobals*>(g)->error, PRRTC_ERR_DEVICE_INDEX);
        break;
      }
      if (mine) __stcg(rows + (size_t)n * dpad + lane, bval);
      ++n;
      if (phase == 0) {
        // line 8: nearest node of T_o (as the round found it) to c_new
        nno = nearest(D->nodes[o], n_o, dpad, c.v.b, lane, &c.cnt->nn_nodes);
        ct = row_elem(D->nodes[o], nno, dpad, lane);
        const float dv = ct - cnew;
        Dd = __fsqrt_rn(warp_sum(dv * dv));
        n_ext = (Dd > 0.f) ? (int)ceilf(__fdiv_rn(Dd, range)) : 0;
      }
      if (phase == n_ext) {
        connected = 1;
        break;
      }
      const int i = phase + 1;
      if (i < n_ext) {
        bval = fmaf(__fdiv_rn((float)i * range, Dd), ct - cnew, cnew);
        N = g->n_full;
      } else {
        bval = ct;
        const float len = Dd - (float)(n_ext - 1) * range;
        N = (int)ceilf(__fdiv_rn(len, res));
        if (N < 1) N = 1;
      }
      if (mine) {
        c.v.a[lane] = c.v.b[lane];
        c.v.b[lane] = bval;
      }
      __syncwarp();
    }
  } while (false);
  __syncwarp();
  if (lane == 0) {
    h->n = n;
    h->nn = nn;
    h->nno = nno;
    h->connected = connected;
    h->edges = edges;
    h->dd_node = dd_node;
    h->dd_free = dd_free;
  }
  __syncwarp();
}

// Rounds of one problem by every warp of the block (block-uniform control
// flow: every thread meets every barrier).
__device__ void lockstep_problem(const Ctx& c, int warp, int nwarps) {
  __shared__ int s_it0, s_s, s_ns, s_no, s_stop, s_nb, s_winner, s_total;
  PlanGlobals* g = const_cast<PlanGlobals*>(c.g);
  const ProblemDesc* D = c.D;
  ProblemState* S = c.S;
  LockstepHeld* meta = reinterpret_cast<LockstepHeld*>(D->held_meta);
  const int B = g->workers, dpad = D->dpad, cap = D->cap, lane = c.lane;
  const size_t held_stride = (size_t)D->held_rows * dpad;
  for (;;) {
    if (threadIdx.x == 0) {
      int stop = ld_volatile(&S->done) | ld_volatile(&S->solved) | (slice_over(g) ? 1 : 0);
      const int it0 = S->iter;
      if (!stop && it0 >= g->max_iters) {
        atomicExch(&S->done, 1);
        stop = 1;
      }
      if (!stop && g->time_limit_ns && globaltimer_ns() - g->t0 > g->time_limit_ns) {
        S->timed_out = 1;
        atomicExch(&S->done, 1);
        stop = 1;
      }
      // line 3 at the start of the round: every worker extends the smaller tree
      const int na = min(S->count[0], cap), nb = min(S->count[1], cap);
      s_s = (na <= nb) ? 0 : 1;
      s_ns = s_s ? nb : na;
      s_no = s_s ? na : nb;
      s_it0 = it0;
      s_nb = min(B, g->max_iters - it0);
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    const int it0 = s_it0, s = s_s, n_s = s_ns, n_o = s_no, nb = s_nb;
    for (int b = warp; b < nb; b += nwarps)
      lockstep_iteration(c, it0 + b, s, n_s, n_o, meta + b, D->held + (size_t)b * held_stride);
    __syncthreads();
    // end of the round: radius updates and row offsets in worker order, the winner
    if (threadIdx.x == 0) {
      float* rad = D->radius[s];
      int total = 0, winner = -1;
      for (int b = 0; b < nb; ++b) {
        LockstepHeld& h = meta[b];
        if (h.dd_node >= 0) {
          const float r = __ldcg(rad + h.dd_node);
          if (h.dd_free) {
            if (!isnan(r)) __stcg(rad + h.dd_node, r * (1.f + g->dd_alpha));
          } else {
            __stcg(rad + h.dd_node, isnan(r) ? g->dd_radius : fmaxf(r * (1.f - g->dd_alpha), g->dd_min_radius));
          }
        }
        h.offset = total;
        total += h.n;
        const bool all_in = n_s + total <= cap;
        if (h.connected && all_in && (winner < 0 || h.edges < meta[winner].edges)) winner = b;
      }
      s_total = total;
      s_winner = winner;
      S->iter = it0 + nb;
    }
    __syncthreads();
    // append the held rows: row k of worker b at n_s + offset + k, hanging
    // from the worker's previous row (k > 0) or its snapshot row nn
    for (int b = warp; b < nb; b += nwarps) {
      const LockstepHeld h = meta[b];
      const float* src = D->held + (size_t)b * held_stride;
      for (int k = 0; k < h.n; ++k) {
        const int idx = n_s + h.offset + k;
        if (idx >= cap) {
          if (lane == 0) c.cnt->insert_fail++;
          break;
        }
        if (lane == 0) __stcg(D->parent[s] + idx, k == 0 ? h.nn : idx - 1);
        if (lane < dpad) __stcg(D->nodes[s] + (size_t)idx * dpad + lane, __ldcg(src + (size_t)k * dpad + lane));
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) S->count[s] = min(n_s + s_total, cap);
    __syncthreads();
    const int w = s_winner;
    if (w >= 0) {
      if (warp == 0) {
        const LockstepHeld h = meta[w];
        const int join_s = n_s + h.offset + h.n - 1;
        if (lane == 0) {
          S->solved = 1;
          S->t_solve = globaltimer_ns();
          S->s_tree = s;
          S->join_s = join_s;
          S->join_o = h.nno;
        }
        __syncwarp();
        extract_path(c, s, join_s, h.nno);
        __threadfence();
        if (lane == 0) atomicExch(&S->done, 1);
      }
      __syncthreads();
      break;
    }
  }
}

__device__ int pick_problem(PlanGlobals* g, const ProblemState* states) {
  const int P = g->n_problems;
  if (slice_over(g)) return -1;
  const int t = atomicAdd(&g->cursor, 1);
  if (g->mode != PRRTC_MODE_ASYNC) return t < P ? (g->active ? g->active[t] : t) : -1;
  for (int k = 0; k < P; ++k) {
    const int i = (t + k) % P;
    const int p = g->active ? g->active[i] : i;
    if (!ld_volatile(&states[p].done)) return p;
  }
  return -1;
}

// The planner launch: blocks take problems from the work queue, stage each
// problem's robot and environment in shared memory and run its workers --
// independent warps (async and serial modes) or the lockstep rounds.
template <bool kLockstep, int kTile, bool kLean>
__device__ __forceinline__ void plan_body(PlanGlobals* __restrict__ g, const ProblemDesc* __restrict__ descs,
                                          ProblemState* __restrict__ states, int robot_bytes, int env_bytes,
                                          int warp_floats) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_prob;
  __shared__ int s_ok;
  __shared__ const RobotDev* s_robot;
  __shared__ const float4* s_env;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) {
    atomicMin(&g->t0, globaltimer_ns());
    mbar_init(&bar, 1);
    s_robot = nullptr;
    s_env = nullptr;
  }
  __syncthreads();
  uint32_t phase = 0;
  for (;;) {
    if (threadIdx.x == 0) s_prob = pick_problem(g, states);
    __syncthreads();
    const int p = s_prob;
    if (p < 0) break;
    const ProblemDesc* D = descs + p;
    const int np_pad = (D->n_pairs + 3) & ~3;
    RobotHeader* R = reinterpret_cast<RobotHeader*>(smem);
    uint32_t* pair = reinterpret_cast<uint32_t*>(smem + sizeof(RobotHeader));
    float* thr = reinterpret_cast<float*>(pair + np_pad);
    float4* senv = reinterpret_cast<float4*>(smem + robot_bytes);
    const int env_f4 = D->env.n_float4();
    // Stage robot and environment unless the block already holds them.
    const bool restage = (s_robot != D->robot) || (s_env != D->env.data);
    __syncthreads();
    if (restage) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        const uint32_t bytes = (uint32_t)sizeof(RobotHeader) + 8u * (uint32_t)np_pad + 16u * (uint32_t)env_f4;
        mbar_arrive_expect_tx(&bar, bytes);
        bulk_g2s(R, &D->robot->h, sizeof(RobotHeader), &bar);
        if (np_pad) {
          bulk_g2s(pair, D->robot->pair, 4u * np_pad, &bar);
          bulk_g2s(thr, D->robot->thr, 4u * np_pad, &bar);
        }
        if (env_f4) bulk_g2s(senv, D->env.data, 16u * env_f4, &bar);
      }
      if (threadIdx.x == 0) {
        s_ok = mbar_wait(&bar, phase, 1u << 26) ? 1 : 0;
        if (!s_ok) {
          atomicExch(&g->error, PRRTC_ERR_TIMEOUT);
          // the block leaves: first give its bulk copies (bounded) time to land
          mbar_wait(&bar, phase, 1u << 26);
        }
        s_robot = D->robot;
        s_env = D->env.data;
      }
      phase ^= 1u;
      __syncthreads();
      if (!s_ok) break;  // block-uniform: every thread leaves the same way
    }
    Ctx c;
    c.g = g;
    c.D = D;
    c.S = states + p;
    c.R = R;
    c.pair = pair;
    c.thr = thr;
    c.env = senv;
    // per-warp area: counters (128 B), the three vectors, sphere-centre staging
    float* warp_area = reinterpret_cast<float*>(smem + robot_bytes + env_bytes) + warp * (warp_floats);
    c.cnt = reinterpret_cast<WarpCount*>(warp_area);
    warp_count_clear(c.cnt, lane);
    float* vecs = warp_area + kCountFloats;
    c.v.rnd = vecs;
    c.v.a = vecs + kMaxDof;
    c.v.b = vecs + 2 * kMaxDof;
    c.stage = vecs + kWarpVecFloats;
    c.lane = lane;
    if constexpr (kLockstep)
      lockstep_problem(c, warp, blockDim.x >> 5);
    else
      worker<kTile, kLean>(c);
    // flush this warp's counters into the problem
    __syncwarp();
    if (lane < 14) {
      ProblemState* S = states + p;
      const WarpCount& w = *c.cnt;
      unsigned long long* dst[14] = {&S->sphere_tests, &S->pair_tests,  &S->fk_states,     &S->prim_tests[0],
                                     &S->prim_tests[1], &S->prim_tests[2], &S->prim_tests[3], &S->edges,
                                     &S->edge_states,  &S->nn_nodes,    &S->iterations,    &S->insert_fail,
                                     &S->dd_rejected,  &S->verdict_states};
      const unsigned long long val = reinterpret_cast<const unsigned long long*>(&w)[lane];
      if (val) atomicAdd(dst[lane], val);
    }
    __syncthreads();
  }
}

// One instance per obstacle tile (32 or 64 primitives per type per first-stage
// round) and feature set: the launched kernel holds only the check code of its
// tile, and the lean instances (kLean) leave out the learned mixture draw, the
// Halton sampler, distance fields, oriented boxes and links without a bounding
// sphere, for batches that use none of them (fewer instructions to fetch on
// the hot path), and dynamic-domain sampling and the wide-range sine/cosine
// (revolute joints beyond +-3.2 rad) as well.
template <int kTile, bool kLean>
__global__ void __maxnreg__(128) plan_kernel(PlanGlobals* __restrict__ g, const ProblemDesc* __restrict__ descs,
                                             ProblemState* __restrict__ states, int robot_bytes, int env_bytes,
                                             int warp_floats) {
  plan_body<false, kTile, kLean>(g, descs, states, robot_bytes, env_bytes, warp_floats);
}
template __global__ void plan_kernel<32, false>(PlanGlobals*, const ProblemDesc*, ProblemState*, int, int, int);
template __global__ void plan_kernel<64, false>(PlanGlobals*, const ProblemDesc*, ProblemState*, int, int, int);
template __global__ void plan_kernel<32, true>(PlanGlobals*, const ProblemDesc*, ProblemState*, int, int, int);
template __global__ void plan_kernel<64, true>(PlanGlobals*, const ProblemDesc*, ProblemState*, int, int, int);

__global__ void __maxnreg__(128) lockstep_kernel(PlanGlobals* __restrict__ g, const ProblemDesc* __restrict__ descs,
                                                 ProblemState* __restrict__ states, int robot_bytes, int env_bytes,
                                                 int warp_floats) {
  plan_body<true, 32, false>(g, descs, states, robot_bytes, env_bytes, warp_floats);
}

// Reject a start or goal in collision (Alg. 1 lines 1-2): warp 0 checks the
// start and warp 1 the goal, each with the whole warp; the verdicts meet in
// shared memory.
__device__ bool endpoint_collides(const ProblemDesc* D, int which, const RobotHeader* R, const uint32_t* pair,
                                  const float* thr, const float4* env, float* stage) {
  return config_collides_warp(R, pair, thr, env, D->env.n_aabb, D->env.n_obb, D->env.n_cyl, D->env.n_sph, D->env.esdf,
                              stage, which == 0 ? D->q_start : D->q_goal, threadIdx.x & 31);
}

// One block per problem: clear the rows the previous launch wrote (back to
// NaN / unset parent), insert the roots, reset the counters, check start and
// goal.  Robot and environment are staged in shared
// memory (bulk copies, overlapping the clearing) for the endpoint check;
// should the copy not complete in time the check reads them from global, the
// timeout is recorded in *error (nullable), and the block waits once more
// (bounded) for its copies before it exits.
__global__ void setup_kernel(const ProblemDesc* __restrict__ descs, ProblemState* __restrict__ states,
                             const int* __restrict__ idx, int robot_bytes, int env_bytes, int* error) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_hit[2];
  __shared__ int s_late;
  const int p = idx ? idx[blockIdx.x] : blockIdx.x;
  const ProblemDesc* D = descs + p;
  ProblemState* S = states + p;
  const int dpad = D->dpad;
  const int np_pad = (D->n_pairs + 3) & ~3;
  const int env_f4 = D->env.n_float4();
  RobotHeader* sR = reinterpret_cast<RobotHeader*>(smem);
  uint32_t* spair = reinterpret_cast<uint32_t*>(smem + sizeof(RobotHeader));
  float* sthr = reinterpret_cast<float*>(spair + np_pad);
  float4* senv = reinterpret_cast<float4*>(smem + robot_bytes);
  if (threadIdx.x == 0) {
    s_late = 0;
    mbar_init(&bar, 1);
    fence_proxy_async_smem();
    const uint32_t bytes = (uint32_t)sizeof(RobotHeader) + 8u * (uint32_t)np_pad + 16u * (uint32_t)env_f4;
    mbar_arrive_expect_tx(&bar, bytes);
    bulk_g2s(sR, &D->robot->h, sizeof(RobotHeader), &bar);
    if (np_pad) {
      bulk_g2s(spair, D->robot->pair, 4u * np_pad, &bar);
      bulk_g2s(sthr, D->robot->thr, 4u * np_pad, &bar);
    }
    if (env_f4) bulk_g2s(senv, D->env.data, 16u * env_f4, &bar);
  }
  for (int t = 0; t < 2; ++t) {
    const int rows = S->used_rows[t];
    const size_t nf = (size_t)rows * S->used_dpad;
    const uint32_t nan_bits = 0xffffffffu;
    uint32_t* nodes = reinterpret_cast<uint32_t*>(D->nodes[t]);
    for (size_t k = threadIdx.x; k < nf; k += blockDim.x) nodes[k] = nan_bits;
    uint32_t* radius = reinterpret_cast<uint32_t*>(D->radius[t]);
    for (int k = threadIdx.x; k < rows; k += blockDim.x) {
      D->parent[t][k] = kUnsetParent;
      radius[k] = nan_bits;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int j = threadIdx.x;
    if (j < dpad) {
      D->nodes[0][j] = (j < D->dof) ? D->q_start[j] : 0.f;
      D->nodes[1][j] = (j < D->dof) ? D->q_goal[j] : 0.f;
    }
    if (j == 0) {
      D->parent[0][0] = kRootParent;
      D->parent[1][0] = kRootParent;
      S->iter = 0;
      S->count[0] = 1;
      S->count[1] = 1;
      S->solved = 0;
      S->done = 0;
      S->timed_out = 0;
      S->pre_status = 0;
      S->s_tree = -1;
      S->join_s = S->join_o = -1;
      S->path_n = 0;
      S->path_status = -100;
      S->cost = 0.0;
      S->t_solve = 0;
      S->edges = S->edge_states = S->sphere_tests = S->pair_tests = 0;
      S->fk_states = S->nn_nodes = S->iterations = S->insert_fail = 0;
      S->dd_rejected = 0;
      S->verdict_states = 0;
      S->prim_tests[0] = S->prim_tests[1] = S->prim_tests[2] = S->prim_tests[3] = 0;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 2) {
    int ok = 0;
    if (lane == 0) {
      ok = mbar_wait(&bar, 0, 1u << 26) ? 1 : 0;
      if (!ok) s_late = 1;
    }
    ok = __shfl_sync(kFull, ok, 0);
    // each warp's sphere centres: 3 floats per sphere
    float* stage = reinterpret_cast<float*>(smem + robot_bytes + env_bytes) + warp * 3 * D->n_spheres;
    const bool hit = ok ? endpoint_collides(D, warp, sR, spair, sthr, senv, stage)
                        : endpoint_collides(D, warp, &D->robot->h, D->robot->pair, D->robot->thr, D->env.data, stage);
    if (lane == 0) s_hit[warp] = hit ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_hit[0]) S->pre_status = PRRTC_START_IN_COLLISION;
    else if (s_hit[1]) S->pre_status = PRRTC_GOAL_IN_COLLISION;
    if (s_hit[0] | s_hit[1]) S->done = 1;
    if (s_late) {
      if (error) atomicExch(error, PRRTC_ERR_TIMEOUT);
      mbar_wait(&bar, 0, 1u << 26);  // the staged copies, before the block exits
    }
  }
}

// After the plan: record which rows were written so the next setup clears them.
__global__ void record_usage_kernel(const ProblemDesc* __restrict__ descs, ProblemState* __restrict__ states, int n,
                                    const int* __restrict__ idx) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int p = idx ? idx[t] : t;
  const ProblemDesc* D = descs + p;
  ProblemState* S = states + p;
  S->used_rows[0] = min(S->count[0], D->cap);
  S->used_rows[1] = min(S->count[1], D->cap);
  S->used_dpad = D->dpad;
}

__global__ void gather_paths_kernel(const ProblemDesc* __restrict__ descs, const int* __restrict__ offsets, int n,
                                    float* __restrict__ out) {
  const int p = blockIdx.x;
  if (p >= n) return;
  const int begin = offsets[p], count = offsets[p + 1] - begin;
  const float* src = descs[p].path;
  for (int k = threadIdx.x; k < count; k += blockDim.x) out[(size_t)begin + k] = src[k];
}

// The first `rows` path rows of every solved problem into a fixed slot of
// `stride` floats per problem, so that a batch's paths come back with its
// results in one copy (no gather sized on the host in between).
__global__ void gather_heads_kernel(const ProblemDesc* __restrict__ descs, const ProblemState* __restrict__ states,
                                    int n, int rows, int stride, float* __restrict__ out) {
  const int p = blockIdx.x;
  if (p >= n) return;
  const ProblemState& S = states[p];
  const int m = (S.solved && S.path_status == PRRTC_SOLVED) ? min(S.path_n, rows) : 0;
  const int count = m * descs[p].dof;
  const float* src = descs[p].path;
  float* dst = out + (size_t)p * stride;
  for (int k = threadIdx.x; k < count; k += blockDim.x) dst[k] = src[k];
}

}  // namespace

cudaError_t launch_setup(const ProblemDesc* desc, ProblemState* state, int n, int max_spheres, int max_pairs,
                         int max_env_f4, cudaStream_t stream, const int* idx, int* error) {
  if (n <= 0) return cudaSuccess;
  const int robot_bytes = robot_smem_bytes((max_pairs + 3) & ~3);
  const int env_bytes = max_env_f4 * 16;
  const int smem = robot_bytes + env_bytes + stage_bytes(max_spheres);
  cudaError_t e = cudaFuncSetAttribute(setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  setup_kernel<<<n, 256, smem, stream>>>(desc, state, idx, robot_bytes, env_bytes, error);
  return cudaGetLastError();
}

// Resident planner blocks per SM for a block shape, cached: the occupancy
// query and the shared-memory attribute cost host time on every call.
static const void* plan_kernel_fn(bool lockstep, int tile, bool lean) {
  if (lockstep) return reinterpret_cast<const void*>(lockstep_kernel);
  if (lean)
    return tile == 64 ? reinterpret_cast<const void*>(plan_kernel<64, true>)
                      : reinterpret_cast<const void*>(plan_kernel<32, true>);
  return tile == 64 ? reinterpret_cast<const void*>(plan_kernel<64, false>)
                    : reinterpret_cast<const void*>(plan_kernel<32, false>);
}

int resident_blocks_per_sm(int warps, int smem, bool lockstep, int tile, bool lean) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  static std::map<int, int> attr_smem;  // per (device, kernel): the attribute value set so far
  int dev = 0;
  cudaGetDevice(&dev);
  const int kid = 5 * dev + (lockstep ? 4 : (tile == 64 ? 1 : 0) + (lean ? 2 : 0));
  const std::pair<int, int> key{warps + 64 * kid, smem};
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const void* fn = plan_kernel_fn(lockstep, tile, lean);
  if (smem > attr_smem[kid]) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr_smem[kid] = smem;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
  if (per_sm < 1) per_sm = 1;
  cache.emplace(key, per_sm);
  return per_sm;
}

PlanLaunch plan_launch_config(int n_problems, int mode, int blocks, int warps, int max_spheres, int max_pairs,
                              int max_env_f4, int sm_count, int workers) {
  PlanLaunch c{};
  c.lockstep = mode == PRRTC_MODE_LOCKSTEP;
  if (mode == PRRTC_MODE_SERIAL)
    c.warps = 1;
  else if (c.lockstep)  // no more warps than the round has workers
    c.warps = std::min(warps > 0 ? warps : 8, std::max(workers, 1));
  else
    c.warps = warps > 0 ? warps : 4;
  if (c.warps > 16) c.warps = 16;
  c.robot_bytes = robot_smem_bytes((max_pairs + 3) & ~3);
  c.env_bytes = max_env_f4 * 16;
  c.stage_bytes = (int)sizeof(WarpCount) + kWarpVecFloats * (int)sizeof(float) + stage_bytes(max_spheres);  // per warp
  c.smem = c.robot_bytes + c.env_bytes + c.warps * c.stage_bytes;
  // both tile instances take the same registers (capped) and shared memory
  const int per_sm = resident_blocks_per_sm(c.warps, c.smem, c.lockstep, 32, false);
  int resident = per_sm * sm_count;
  if (blocks > 0) {
    c.grid = blocks;
  } else if (mode != PRRTC_MODE_ASYNC) {  // one block per problem
    c.grid = n_problems < resident ? n_problems : resident;
  } else if (n_problems == 1) {
    // one problem: 256 concurrent workers (the paper's saturation point, Sec. IV-C)
    c.grid = 256 / c.warps;
    if (c.grid > resident) c.grid = resident;
  } else {
    c.grid = resident;
  }
  if (c.grid < 1) c.grid = 1;
  return c;
}

cudaError_t launch_plan(const PlanGlobals* g, const ProblemDesc* desc, ProblemState* state, const PlanLaunch& cfg,
                        int obstacle_tile, bool lean, cudaStream_t stream) {
  // sets the shared-memory attribute once per size and kernel
  resident_blocks_per_sm(cfg.warps, cfg.smem, cfg.lockstep, obstacle_tile, lean);
  cudaError_t e;
  if (cfg.lockstep)
    lockstep_kernel<<<cfg.grid, cfg.warps * 32, cfg.smem, stream>>>(const_cast<PlanGlobals*>(g), desc, state,
                                                                    cfg.robot_bytes, cfg.env_bytes,
                                                                    cfg.stage_bytes / (int)sizeof(float));
  else {
    auto* fn = lean ? (obstacle_tile == 64 ? plan_kernel<64, true> : plan_kernel<32, true>)
                    : (obstacle_tile == 64 ? plan_kernel<64, false> : plan_kernel<32, false>);
    fn<<<cfg.grid, cfg.warps * 32, cfg.smem, stream>>>(const_cast<PlanGlobals*>(g), desc, state, cfg.robot_bytes,
                                                       cfg.env_bytes, cfg.stage_bytes / (int)sizeof(float));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_record_usage(const ProblemDesc* desc, ProblemState* state, int n, cudaStream_t stream,
                                const int* idx) {
  if (n <= 0) return cudaSuccess;
  record_usage_kernel<<<(n + 127) / 128, 128, 0, stream>>>(desc, state, n, idx);
  return cudaGetLastError();
}

cudaError_t launch_gather_heads(const ProblemDesc* desc, const ProblemState* state, int n, int rows, int stride,
                                float* out, cudaStream_t stream) {
  if (n <= 0 || rows <= 0) return cudaSuccess;
  gather_heads_kernel<<<n, 128, 0, stream>>>(desc, state, n, rows, stride, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_paths(const ProblemDesc* desc, const int* offsets, int n, float* out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  gather_paths_kernel<<<n, 128, 0, stream>>>(desc, offsets, n, out);
  return cudaGetLastError();
}

}  // namespace prrtc
