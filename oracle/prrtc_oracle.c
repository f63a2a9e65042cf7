/*
 * prrtc_oracle.c -- plain, slow FP64 CPU oracle of the pRRTC hot path.
 *
 * TEST INFRASTRUCTURE: loaded only by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg.  Shares no code with the CUDA path.  Every
 * step below is written as the definition it implements, in binary64, with no
 * blocking, fusion or reordering beyond what that definition states.
 * Interface and paper citations: prrtc_oracle.h.
 */
#include "prrtc_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ------------------------------------------------------------------ Philox */
/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): each round multiplies counter words 0
 * and 2 by two fixed odd constants, swaps the halves and xors in the key;
 * the key is bumped by the two Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_philox_blocks(const uint32_t* ctr, int32_t n, const uint32_t key[2], uint32_t* out) {
  for (int32_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * (size_t)i, key, out + 4 * (size_t)i);
}

/* Word w of the stream for (problem, it): block w/4 of Philox with counter
 * {problem, it, w/4, 0}. */
static uint32_t sample_word(uint64_t seed, uint32_t problem, uint32_t it, int w) {
  uint32_t ctr[4] = {problem, it, (uint32_t)(w / 4), 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[w % 4];
}

/* A 32-bit word mapped to [0,1) with 24 bits: (w >> 8) * 2^-24. */
static double unit24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* RANDOM_CONFIG of Alg. 1 (Halton in the paper, Philox here). */
int orc_sample(const orc_robot* r, uint64_t seed, uint32_t problem, uint32_t it,
               double goal_bias, double* q) {
  double u0 = unit24(sample_word(seed, problem, it, 0));
  if (u0 < goal_bias) return 1;
  for (int j = 0; j < r->dof; ++j) {
    double u = unit24(sample_word(seed, problem, it, j + 1));
    q[j] = r->lower[j] + u * (r->upper[j] - r->lower[j]);
  }
  return 0;
}

/* Learned proposal draw (the mixture proposal of the learned sampler; not in the paper).
 * Words 20.. of the iteration's stream (Philox blocks 5-9): word 20 decides
 * learned vs uniform, word 21 picks the component, then Box-Muller pairs
 * (u1 from (w >> 8) + 1, so u1 is in (0, 1]) give standard normals. */
int orc_sample_learned(const orc_robot* r, uint64_t seed, uint32_t problem, uint32_t it, double goal_bias,
                       const double* gmm, double learned_ratio, double amb_rel, double* q, int* amb) {
  const int d = r->dof;
  const int K = 8;
  if (amb) *amb = 0;
  double u0 = unit24(sample_word(seed, problem, it, 0));
  if (u0 < goal_bias) return 1;
  if (gmm && unit24(sample_word(seed, problem, it, 20)) < learned_ratio) {
    const double* logits = gmm;
    const double* mean = gmm + K;
    const double* logsig = gmm + K + K * d;
    double mx = logits[0];
    for (int k = 1; k < K; ++k) mx = fmax(mx, logits[k]);
    double pk[8], tot = 0.0;
    for (int k = 0; k < K; ++k) {
      pk[k] = exp(logits[k] - mx);
      tot += pk[k];
    }
    double uk = unit24(sample_word(seed, problem, it, 21));
    int comp = K - 1;
    double cum = 0.0;
    for (int k = 0; k < K; ++k) {
      cum += pk[k] / tot;
      if (amb && fabs(uk - cum) <= amb_rel) *amb = 1;
      if (uk < cum) {
        comp = k;
        break;
      }
    }
    for (int j = 0; j < d; ++j) {
      int m = j / 2;
      uint32_t wa = sample_word(seed, problem, it, 22 + 2 * m);
      uint32_t wb = sample_word(seed, problem, it, 23 + 2 * m);
      double u1 = (double)((wa >> 8) + 1u) * (1.0 / 16777216.0);
      double u2 = (double)(wb >> 8) * (1.0 / 16777216.0);
      double rad = sqrt(-2.0 * log(u1));
      double z = (j % 2 == 0) ? rad * cos(2.0 * M_PI * u2) : rad * sin(2.0 * M_PI * u2);
      double ls = fmin(fmax(logsig[comp * d + j], -5.0), 2.0);
      double un = mean[comp * d + j] + exp(ls) * z;
      double v = r->lower[j] + 0.5 * (un + 1.0) * (r->upper[j] - r->lower[j]);
      q[j] = fmin(fmax(v, r->lower[j]), r->upper[j]);
    }
    return 2;
  }
  for (int j = 0; j < d; ++j) {
    double u = unit24(sample_word(seed, problem, it, j + 1));
    q[j] = r->lower[j] + u * (r->upper[j] - r->lower[j]);
  }
  return 0;
}

/* Halton (1960): coordinate j of point `index` is the radical inverse of index
 * in the j-th prime base.  Written as the mirrored digit string: with index =
 * sum_k d_k b^k (m digits), the value is (sum_k d_k b^(m-1-k)) / b^m, formed
 * exactly in integers and divided once. */
void orc_halton(uint32_t index, int32_t dim, double* u) {
  static const uint32_t primes[16] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53};
  for (int32_t j = 0; j < dim && j < 16; ++j) {
    const uint64_t b = primes[j];
    uint64_t num = 0, den = 1;
    for (uint64_t i = index; i > 0; i /= b) {
      num = num * b + i % b;
      den *= b;
    }
    u[j] = (double)num / (double)den;
  }
}

void orc_occupancy(const orc_env* e, const double origin[3], double cell, int32_t n, double radius,
                   uint8_t* out) {
  for (int32_t k = 0; k < n; ++k)
    for (int32_t j = 0; j < n; ++j)
      for (int32_t i = 0; i < n; ++i) {
        double p[3] = {origin[0] + (i + 0.5) * cell, origin[1] + (j + 0.5) * cell, origin[2] + (k + 0.5) * cell};
        double best = DBL_MAX;
        for (int o = 0; o < e->n_box; ++o) best = fmin(best, orc_sd_box(e->box + 15 * o, p));
        for (int o = 0; o < e->n_cyl; ++o) best = fmin(best, orc_sd_cyl(e->cyl + 8 * o, p));
        for (int o = 0; o < e->n_sph; ++o) best = fmin(best, orc_sd_sph(e->sph + 4 * o, p));
        out[i + n * j + n * n * k] = (uint8_t)(best < radius);
      }
}

/* ------------------------------------------------------- ESDF */
static double min_signed_distance(const orc_env* e, const double p[3]) {
  double best = DBL_MAX;
  for (int o = 0; o < e->n_box; ++o) best = fmin(best, orc_sd_box(e->box + 15 * o, p));
  for (int o = 0; o < e->n_cyl; ++o) best = fmin(best, orc_sd_cyl(e->cyl + 8 * o, p));
  for (int o = 0; o < e->n_sph; ++o) best = fmin(best, orc_sd_sph(e->sph + 4 * o, p));
  return best;
}

void orc_voxelize(const orc_env* e, const double origin[3], double voxel, const int32_t dims[3], uint8_t* occ) {
  for (int32_t k = 0; k < dims[2]; ++k)
    for (int32_t j = 0; j < dims[1]; ++j)
      for (int32_t i = 0; i < dims[0]; ++i) {
        double p[3] = {origin[0] + (i + 0.5) * voxel, origin[1] + (j + 0.5) * voxel, origin[2] + (k + 0.5) * voxel};
        occ[i + (size_t)dims[0] * (j + (size_t)dims[1] * k)] = (uint8_t)(min_signed_distance(e, p) < 0.0);
      }
}

double orc_esdf_at(const uint8_t* occ, const int32_t dims[3], double voxel, int32_t vi, int32_t vj, int32_t vk) {
  const int32_t nx = dims[0], ny = dims[1], nz = dims[2];
  const size_t n = (size_t)nx * ny * nz;
  const double diag = voxel * sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
  const uint8_t mine = occ[vi + (size_t)nx * (vj + (size_t)ny * vk)] != 0;
  double best2 = -1.0; /* squared distance in voxel units to the nearest voxel of the other kind */
  for (size_t u = 0; u < n; ++u) {
    if ((occ[u] != 0) == mine) continue;
    const double di = (double)((int32_t)(u % nx) - vi);
    const double dj = (double)((int32_t)((u / nx) % ny) - vj);
    const double dk = (double)((int32_t)(u / ((size_t)nx * ny)) - vk);
    const double d2 = di * di + dj * dj + dk * dk;
    if (best2 < 0.0 || d2 < best2) best2 = d2;
  }
  const double mag = best2 < 0.0 ? diag : voxel * sqrt(best2);
  return mine ? -mag : mag;
}

void orc_esdf(const uint8_t* occ, const int32_t dims[3], double voxel, double* out) {
  const int32_t nx = dims[0], ny = dims[1], nz = dims[2];
  for (int32_t k = 0; k < nz; ++k)
    for (int32_t j = 0; j < ny; ++j)
      for (int32_t i = 0; i < nx; ++i)
        out[i + (size_t)nx * (j + (size_t)ny * k)] = orc_esdf_at(occ, dims, voxel, i, j, k);
}

double orc_esdf_query(const double* esdf, const double origin[3], double voxel, const int32_t dims[3],
                      const double p[3]) {
  int32_t base[3];
  double t[3];
  for (int a = 0; a < 3; ++a) {
    double u = (p[a] - origin[a]) / voxel - 0.5;
    u = fmin(fmax(u, 0.0), (double)(dims[a] - 1));
    int32_t i0 = (int32_t)floor(u);
    if (i0 > dims[a] - 2) i0 = dims[a] - 2;
    base[a] = i0;
    t[a] = u - (double)i0;
  }
  const int32_t nx = dims[0], ny = dims[1];
  double c[2][2];
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj) {
      const size_t row = (size_t)nx * ((size_t)(base[1] + dj) + (size_t)ny * (size_t)(base[2] + dk));
      const double a = esdf[row + base[0]], b = esdf[row + base[0] + 1];
      c[dk][dj] = a + t[0] * (b - a); /* along x */
    }
  const double y0 = c[0][0] + t[1] * (c[0][1] - c[0][0]); /* along y, k = base */
  const double y1 = c[1][0] + t[1] * (c[1][1] - c[1][0]); /* along y, k = base + 1 */
  return y0 + t[2] * (y1 - y0);                          /* along z */
}

/* ------------------------------------------------------- forward kinematics */
static void mat4_identity(double M[16]) {
  memset(M, 0, 16 * sizeof(double));
  M[0] = M[5] = M[10] = M[15] = 1.0;
}

static void mat4_mul(const double A[16], const double B[16], double C[16]) {
  double T[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
      T[4 * i + j] = s;
    }
  memcpy(C, T, sizeof(T));
}

static void mat4_translation(double x, double y, double z, double M[16]) {
  mat4_identity(M);
  M[3] = x;
  M[7] = y;
  M[11] = z;
}

/* Joint transform J_i(q): rotation about a local axis or translation along it. */
static void joint_transform(int32_t type, double q, double M[16]) {
  mat4_identity(M);
  double c = cos(q), s = sin(q);
  if (type == ORC_REV_Z) {
    M[0] = c;  M[1] = -s;
    M[4] = s;  M[5] = c;
  } else if (type == ORC_REV_Y) {
    M[0] = c;  M[2] = s;
    M[8] = -s; M[10] = c;
  } else if (type == ORC_REV_X) {
    M[5] = c;  M[6] = -s;
    M[9] = s;  M[10] = c;
  } else if (type == ORC_PRISM_X) {
    M[3] = q;
  } else if (type == ORC_PRISM_Y) {
    M[7] = q;
  } else {
    M[11] = q;
  }
}

/* Frame i = T_parent * J_i(q_i) * Trans(0, 0, L_i); sphere centre = T_f * [off, 1]. */
void orc_fk(const orc_robot* r, const double* q, double* centres, double* frames) {
  int d = r->dof;
  double* T = (double*)malloc((size_t)d * 16 * sizeof(double));
  for (int i = 0; i < d; ++i) {
    double P[16], J[16], L[16], tmp[16];
    int par = r->joint_parent[i];
    if (par < 0)
      mat4_translation(r->joint_base[3 * i], r->joint_base[3 * i + 1], r->joint_base[3 * i + 2], P);
    else
      memcpy(P, T + 16 * par, sizeof(P));
    joint_transform(r->joint_type[i], q[i], J);
    mat4_translation(0.0, 0.0, r->link_length[i], L);
    mat4_mul(P, J, tmp);
    mat4_mul(tmp, L, T + 16 * i);
  }
  for (int s = 0; s < r->n_spheres; ++s) {
    const double* F = T + 16 * r->sphere_frame[s];
    const double* o = r->sphere_offset + 3 * s;
    for (int k = 0; k < 3; ++k)
      centres[3 * s + k] = F[4 * k] * o[0] + F[4 * k + 1] * o[1] + F[4 * k + 2] * o[2] + F[4 * k + 3];
  }
  if (frames) memcpy(frames, T, (size_t)d * 16 * sizeof(double));
  free(T);
}

/* ------------------------------------------------------- signed distances */
double orc_sd_box(const double* b, const double p[3]) {
  const double* c = b;
  const double* h = b + 3;
  const double* R = b + 6; /* world = R * local + c, row-major */
  double v[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
  double excess[3];
  for (int k = 0; k < 3; ++k) {
    double local = R[0 * 3 + k] * v[0] + R[1 * 3 + k] * v[1] + R[2 * 3 + k] * v[2];
    excess[k] = fabs(local) - h[k];
  }
  double outside = sqrt(fmax(excess[0], 0.0) * fmax(excess[0], 0.0) +
                        fmax(excess[1], 0.0) * fmax(excess[1], 0.0) +
                        fmax(excess[2], 0.0) * fmax(excess[2], 0.0));
  double inside = fmin(fmax(excess[0], fmax(excess[1], excess[2])), 0.0);
  return outside + inside;
}

double orc_sd_cyl(const double* cy, const double p[3]) {
  const double* c = cy;
  const double* a = cy + 3;
  double radius = cy[6], half = cy[7];
  double v[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
  double z = v[0] * a[0] + v[1] * a[1] + v[2] * a[2];
  double w[3] = {v[0] - z * a[0], v[1] - z * a[1], v[2] - z * a[2]};
  double rho = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double dr = rho - radius;
  double dz = fabs(z) - half;
  if (dr <= 0.0 && dz <= 0.0) return fmax(dr, dz);
  double er = fmax(dr, 0.0), ez = fmax(dz, 0.0);
  return sqrt(er * er + ez * ez);
}

double orc_sd_sph(const double* s, const double p[3]) {
  double v[3] = {p[0] - s[0], p[1] - s[1], p[2] - s[2]};
  return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) - s[3];
}

/* ------------------------------------------------------------ clearance */
double orc_clearance(const orc_robot* r, const orc_env* e, const double* q,
                     double* env_c, double* self_c) {
  int S = r->n_spheres;
  double* C = (double*)malloc((size_t)(S > 0 ? S : 1) * 3 * sizeof(double));
  orc_fk(r, q, C, NULL);
  double ce = DBL_MAX, cs = DBL_MAX;
  for (int s = 0; s < S; ++s) {
    const double* p = C + 3 * s;
    double rs = r->sphere_radius[s];
    for (int o = 0; o < e->n_box; ++o) ce = fmin(ce, orc_sd_box(e->box + 15 * o, p) - rs);
    for (int o = 0; o < e->n_cyl; ++o) ce = fmin(ce, orc_sd_cyl(e->cyl + 8 * o, p) - rs);
    for (int o = 0; o < e->n_sph; ++o) ce = fmin(ce, orc_sd_sph(e->sph + 4 * o, p) - rs);
    if (e->esdf) ce = fmin(ce, orc_esdf_query(e->esdf, e->esdf_origin, e->esdf_voxel, e->esdf_dims, p) - rs);
  }
  for (int k = 0; k < r->n_pairs; ++k) {
    int i = r->pairs[2 * k], j = r->pairs[2 * k + 1];
    double dx = C[3 * i] - C[3 * j], dy = C[3 * i + 1] - C[3 * j + 1], dz = C[3 * i + 2] - C[3 * j + 2];
    cs = fmin(cs, sqrt(dx * dx + dy * dy + dz * dz) - r->sphere_radius[i] - r->sphere_radius[j]);
  }
  free(C);
  if (env_c) *env_c = ce;
  if (self_c) *self_c = cs;
  return fmin(ce, cs);
}

void orc_check_states(const orc_robot* r, const orc_env* e, const double* Q, int32_t n,
                      uint8_t* free_out, double* clearance_out) {
  for (int32_t i = 0; i < n; ++i) {
    double c = orc_clearance(r, e, Q + (size_t)i * r->dof, NULL, NULL);
    if (free_out) free_out[i] = (uint8_t)(c >= 0.0);
    if (clearance_out) clearance_out[i] = c;
  }
}

/* ------------------------------------------------------------- planner */
typedef struct tree {
  double* q;      /* [cap*d] */
  int32_t* parent;
  double* radius; /* [cap] dynamic-domain radius, INFINITY = unbounded */
  int32_t n, cap, d;
} tree;

static int tree_add(tree* t, const double* q, int32_t parent) {
  if (t->n >= t->cap) return -1;
  memcpy(t->q + (size_t)t->n * t->d, q, (size_t)t->d * sizeof(double));
  t->parent[t->n] = parent;
  t->radius[t->n] = INFINITY;
  return t->n++;
}

static double dist2(const double* a, const double* b, int d) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) s += (a[j] - b[j]) * (a[j] - b[j]);
  return s;
}

typedef struct plan_ctx {
  const orc_robot* r;
  const orc_env* e;
  const orc_params* p;
  orc_result* res;
  int32_t it;
  double* scratch; /* d doubles */
} plan_ctx;

static void note_amb(plan_ctx* c, int kind) {
  if (c->res->first_amb_iter < 0) {
    c->res->first_amb_iter = c->it;
    c->res->first_amb_kind = kind;
  }
}

/* ceil(x), noting an ambiguity when x lies next to an integer.  `exact` marks
 * arguments that are the same in every precision (delta / resolution of a
 * clamped step), which cannot flip. */
static int32_t ceil_checked(plan_ctx* c, double x, int exact) {
  double nearest = floor(x + 0.5);
  if (!exact && x > 0.0 && fabs(x - nearest) <= c->p->amb_rel * fmax(1.0, x)) note_amb(c, ORC_AMB_CEIL);
  return (int32_t)ceil(x);
}

/* NEAREST_NEIGHBOR (Sec. III-C): argmin of squared L2 distance, lowest index
 * on ties; a near tie is noted as ambiguous. */
static int32_t nearest(plan_ctx* c, const tree* t, const double* q) {
  int32_t best = -1;
  double bd = DBL_MAX, second = DBL_MAX;
  for (int32_t i = 0; i < t->n; ++i) {
    double dd = dist2(t->q + (size_t)i * t->d, q, t->d);
    if (dd < bd) {
      second = bd;
      bd = dd;
      best = i;
    } else if (dd < second) {
      second = dd;
    }
  }
  if (t->n > 1 && second - bd <= c->p->amb_rel * bd + 1e-12) note_amb(c, ORC_AMB_NN_TIE);
  return best;
}

/* Check the n_states interpolated states a + (k/n)(b - a), k = 1..n (Alg. 2,
 * with the endpoint b included and a excluded).  Returns 1 when all are free. */
static int check_edge(plan_ctx* c, const double* a, const double* b, int32_t n_states) {
  int d = c->r->dof;
  double* s = c->scratch;
  int marginal = 0;
  c->res->edges_checked++;
  c->res->edge_states += n_states;
  int valid = 1;
  for (int32_t k = 1; k <= n_states; ++k) {
    double t = (double)k / (double)n_states;
    for (int j = 0; j < d; ++j) s[j] = (k == n_states) ? b[j] : a[j] + t * (b[j] - a[j]);
    double cl = orc_clearance(c->r, c->e, s, NULL, NULL);
    c->res->states_checked++;
    if (fabs(cl) <= c->p->amb_band) marginal = 1;
    if (cl < 0.0) valid = 0;
    if (cl < -c->p->amb_band) {
      marginal = 0; /* robustly invalid whatever the marginal states do */
      break;
    }
  }
  if (marginal) note_amb(c, ORC_AMB_CLEARANCE);
  return valid;
}

static int32_t chain_to_root(const tree* t, int32_t node, int32_t* out, int32_t cap) {
  int32_t n = 0;
  while (node >= 0) {
    if (n < cap) out[n] = node;
    n++;
    node = t->parent[node];
  }
  return n;
}

/* PATH(T_a, T_b): root(T_a) .. join_a, then join_b .. root(T_b); the two join
 * nodes hold the same configuration, so one copy is dropped. */
static void build_path(plan_ctx* c, const tree* A, const tree* B, int32_t ja, int32_t jb) {
  orc_result* res = c->res;
  int d = c->r->dof;
  int32_t ca_cap = A->n, cb_cap = B->n;
  int32_t* ca = (int32_t*)malloc((size_t)(ca_cap > 0 ? ca_cap : 1) * sizeof(int32_t));
  int32_t* cb = (int32_t*)malloc((size_t)(cb_cap > 0 ? cb_cap : 1) * sizeof(int32_t));
  int32_t na = chain_to_root(A, ja, ca, ca_cap);
  int32_t nb = chain_to_root(B, jb, cb, cb_cap);
  int32_t total = na + nb - 1;
  res->path_n = total;
  res->cost = 0.0;
  const double* prev = NULL;
  int32_t w = 0;
  for (int32_t k = na - 1; k >= 0; --k) { /* root(T_a) .. join_a */
    const double* q = A->q + (size_t)ca[k] * d;
    if (prev) res->cost += sqrt(dist2(prev, q, d));
    if (res->path && w < c->p->path_capacity) memcpy(res->path + (size_t)w * d, q, (size_t)d * sizeof(double));
    w++;
    prev = q;
  }
  for (int32_t k = 1; k < nb; ++k) { /* skip join_b (same configuration as join_a) */
    const double* q = B->q + (size_t)cb[k] * d;
    res->cost += sqrt(dist2(prev, q, d));
    if (res->path && w < c->p->path_capacity) memcpy(res->path + (size_t)w * d, q, (size_t)d * sizeof(double));
    w++;
    prev = q;
  }
  res->status = (total > c->p->path_capacity) ? ORC_PATH_OVERFLOW : ORC_SOLVED;
  free(ca);
  free(cb);
}

/* ------------------------------------------------------- lockstep rounds */
/* The concurrent iterations of Sec. III on a fixed schedule: B workers per
 * round, worker b running iteration r B + b against the trees as they stood
 * when round r began.  A worker's new rows are held back until the round
 * ends: row 0 (c_new) hangs from snapshot row nn of T_s, row k from row k-1
 * (the greedy connect's steps). */
typedef struct held {
  int32_t n, cap_rows;
  double* q;      /* [cap_rows * dof] */
  int32_t nn;     /* snapshot row of T_s that row 0 extends */
  int32_t nno;    /* snapshot row of T_o the connect aims at */
  int connected;  /* the connect reached c_nno */
  int32_t dd_node; /* node whose dynamic-domain radius the extension updates, -1 none */
  int dd_free;     /* that extension's edge was free */
  int64_t edges;   /* edges this iteration checked (the extension and each connect step) */
} held;

static void held_push(held* h, const double* q, int d) {
  if (h->n == h->cap_rows) {
    h->cap_rows = h->cap_rows ? 2 * h->cap_rows : 8;
    h->q = (double*)realloc(h->q, (size_t)h->cap_rows * d * sizeof(double));
  }
  memcpy(h->q + (size_t)h->n * d, q, (size_t)d * sizeof(double));
  h->n++;
}

/* Alg. 1 lines 4-15 for iteration `it` against the views vs / vo (T_s and T_o
 * with their sizes at the start of the round), the new rows held in h. */
static void lockstep_iteration(plan_ctx* ctx, const tree* vs, const tree* vo, int32_t it, held* h,
                               double* c_rand, double* c_new, double* c_ext, double* c_tgt) {
  const orc_robot* r = ctx->r;
  const orc_params* p = ctx->p;
  const int d = r->dof;
  const double delta = p->range, resol = p->resolution;
  h->n = 0;
  h->nn = h->nno = -1;
  h->connected = 0;
  h->dd_node = -1;
  h->dd_free = 0;
  const int64_t edges_before = ctx->res->edges_checked;
  ctx->it = it;
  /* line 4: RANDOM_CONFIG (goal bias toward the opposite root, learned or uniform) */
  int amb_k = 0;
  int kind = orc_sample_learned(r, p->seed, p->problem, (uint32_t)it, p->goal_bias, p->gmm,
                                p->gmm ? p->learned_ratio : 0.0, p->amb_rel, c_rand, &amb_k);
  if (amb_k) note_amb(ctx, ORC_AMB_COMPONENT);
  if (kind == 1) memcpy(c_rand, vo->q, (size_t)d * sizeof(double));
  if (kind == 0 && p->sampler == ORC_SAMPLER_HALTON) {
    orc_halton((uint32_t)it + 1u + p->halton_offset, d, c_rand);
    for (int j = 0; j < d; ++j) c_rand[j] = r->lower[j] + c_rand[j] * (r->upper[j] - r->lower[j]);
  }
  /* line 5: nearest node of T_s as the round found it */
  int32_t nn = nearest(ctx, vs, c_rand);
  const double* c_nn = vs->q + (size_t)nn * d;
  double dist = sqrt(dist2(c_rand, c_nn, d));
  if (dist <= 0.0) return;
  const int dd = p->dd_radius > 0.0;
  if (dd && kind != 1) {
    double rad = vs->radius[nn];
    if (isfinite(rad) && fabs(dist - rad) <= p->amb_rel * rad) note_amb(ctx, ORC_AMB_DOMAIN);
    if (dist > rad) {
      ctx->res->dd_rejected++;
      return;
    }
  }
  /* Alg. 2: steer by at most delta, check ceil(len / resolution) states */
  if (fabs(dist - delta) <= p->amb_rel * delta) note_amb(ctx, ORC_AMB_STEER);
  double len;
  int clamped = (dist > delta);
  if (clamped) {
    for (int j = 0; j < d; ++j) c_new[j] = c_nn[j] + (c_rand[j] - c_nn[j]) * (delta / dist);
    len = delta;
  } else {
    memcpy(c_new, c_rand, (size_t)d * sizeof(double));
    len = dist;
  }
  int32_t n_states = ceil_checked(ctx, len / resol, clamped);
  int edge_ok = check_edge(ctx, c_nn, c_new, n_states);
  if (dd) {
    h->dd_node = nn;
    h->dd_free = edge_ok;
  }
  h->edges = ctx->res->edges_checked - edges_before;
  if (!edge_ok) return;
  /* line 7, held back; a tree that is full counting this worker's own rows
   * takes nothing more */
  if (vs->n + h->n >= vs->cap) return;
  held_push(h, c_new, d);
  h->nn = nn;
  /* line 8: nearest node of T_o (as the round found it) to c_new */
  int32_t nno = nearest(ctx, vo, c_new);
  memcpy(c_tgt, vo->q + (size_t)nno * d, (size_t)d * sizeof(double));
  h->nno = nno;
  /* lines 9-15: greedy connect, the same steps as the serial form */
  double D = sqrt(dist2(c_tgt, c_new, d));
  int32_t n_ext = (D > 0.0) ? ceil_checked(ctx, D / delta, 0) : 0;
  for (int32_t i = 1; i <= n_ext; ++i) {
    double step_len;
    if (i < n_ext) {
      double f = (double)i * delta / D;
      for (int j = 0; j < d; ++j) c_ext[j] = c_new[j] + f * (c_tgt[j] - c_new[j]);
      step_len = delta;
    } else {
      memcpy(c_ext, c_tgt, (size_t)d * sizeof(double));
      step_len = D - (double)(n_ext - 1) * delta;
    }
    int32_t ns = ceil_checked(ctx, step_len / resol, i < n_ext);
    if (ns < 1) ns = 1;
    int ok = check_edge(ctx, h->q + (size_t)(h->n - 1) * d, c_ext, ns);
    h->edges = ctx->res->edges_checked - edges_before;
    if (!ok) return;
    if (vs->n + h->n >= vs->cap) return;
    held_push(h, c_ext, d);
  }
  h->connected = 1;
}

/* End of a round: the dynamic-domain radius updates, then every worker's
 * held rows, in worker order.  Among the workers whose connect reached its
 * target with all their rows in the tree, the one a concurrent run would
 * finish first wins: fewest edges checked in its iteration, ties to the
 * lowest worker.  Returns the winner (-1: none); *join_s is its last row's
 * index in T_s. */
static int lockstep_commit(tree* Ts, held* hs, int nb, const orc_params* p, int32_t* join_s) {
  for (int b = 0; b < nb; ++b) {
    if (hs[b].dd_node < 0) continue;
    double* rad = &Ts->radius[hs[b].dd_node];
    if (hs[b].dd_free) {
      if (isfinite(*rad)) *rad *= 1.0 + p->dd_alpha;
    } else if (isinf(*rad)) {
      *rad = p->dd_radius;
    } else {
      *rad = fmax(*rad * (1.0 - p->dd_alpha), p->dd_min_radius);
    }
  }
  int winner = -1;
  for (int b = 0; b < nb; ++b) {
    int32_t prev = hs[b].nn;
    int all_in = 1;
    for (int32_t k = 0; k < hs[b].n; ++k) {
      int32_t idx = tree_add(Ts, hs[b].q + (size_t)k * Ts->d, prev);
      if (idx < 0) {
        all_in = 0;
        break;
      }
      prev = idx;
    }
    if (hs[b].connected && all_in && (winner < 0 || hs[b].edges < hs[winner].edges)) {
      winner = b;
      *join_s = prev;
    }
  }
  return winner;
}

static void plan_lockstep(plan_ctx* ctx, tree* A, tree* B, double* c_rand, double* c_new, double* c_ext,
                          double* c_tgt) {
  const orc_params* p = ctx->p;
  orc_result* res = ctx->res;
  const int32_t nw = p->workers;
  held* hs = (held*)calloc((size_t)nw, sizeof(held));
  res->status = ORC_NO_SOLUTION;
  for (int64_t it0 = 0; it0 < p->max_iters; it0 += nw) {
    /* line 3 at the start of the round: every worker extends the smaller tree */
    int s_is_a = (A->n <= B->n);
    tree* Ts = s_is_a ? A : B;
    tree* To = s_is_a ? B : A;
    const tree vs = *Ts, vo = *To;  /* the trees as the round found them */
    int nb = (int)((p->max_iters - it0) < nw ? (p->max_iters - it0) : nw);
    for (int b = 0; b < nb; ++b)
      lockstep_iteration(ctx, &vs, &vo, (int32_t)(it0 + b), &hs[b], c_rand, c_new, c_ext, c_tgt);
    res->iterations = (int32_t)(it0 + nb);
    int32_t js = -1;
    int w = lockstep_commit(Ts, hs, nb, p, &js);
    if (w >= 0) {
      /* line 16: the winner's last row coincides with row nno of T_o */
      res->join_a = s_is_a ? js : hs[w].nno;
      res->join_b = s_is_a ? hs[w].nno : js;
      res->n_a = A->n;
      res->n_b = B->n;
      build_path(ctx, A, B, res->join_a, res->join_b);
      break;
    }
  }
  if (res->status == ORC_NO_SOLUTION) {
    res->n_a = A->n;
    res->n_b = B->n;
  }
  for (int b = 0; b < nw; ++b) free(hs[b].q);
  free(hs);
}

int32_t orc_plan(const orc_robot* r, const orc_env* e, const double* q_start,
                 const double* q_goal, const orc_params* p, orc_result* res) {
  int d = r->dof;
  res->status = ORC_NO_SOLUTION;
  res->iterations = 0;
  res->n_a = res->n_b = 0;
  res->join_a = res->join_b = -1;
  res->path_n = 0;
  res->first_amb_iter = -1;
  res->first_amb_kind = ORC_AMB_NONE;
  res->cost = 0.0;
  res->edges_checked = res->states_checked = res->edge_states = 0;
  res->dd_rejected = 0;
  if (d <= 0 || p->tree_capacity < 1 || p->range <= 0.0 || p->resolution <= 0.0) {
    res->status = ORC_BAD_INPUT;
    return res->status;
  }
  for (int i = 0; i < d; ++i)
    if (r->joint_parent[i] >= i || r->joint_type[i] < 0 || r->joint_type[i] > ORC_REV_X) {
      res->status = ORC_BAD_INPUT;
      return res->status;
    }

  /* Alg. 1: reject a start or goal in collision up front. */
  if (orc_clearance(r, e, q_start, NULL, NULL) < 0.0) {
    res->status = ORC_START_IN_COLLISION;
    return res->status;
  }
  if (orc_clearance(r, e, q_goal, NULL, NULL) < 0.0) {
    res->status = ORC_GOAL_IN_COLLISION;
    return res->status;
  }

  size_t cap = (size_t)p->tree_capacity;
  tree A = {res->nodes_a, res->parent_a, res->radius_a, 0, p->tree_capacity, d};
  tree B = {res->nodes_b, res->parent_b, res->radius_b, 0, p->tree_capacity, d};
  int own_a = 0, own_b = 0, own_ra = 0, own_rb = 0;
  if (!A.q) { A.q = (double*)malloc(cap * d * sizeof(double)); A.parent = (int32_t*)malloc(cap * sizeof(int32_t)); own_a = 1; }
  if (!B.q) { B.q = (double*)malloc(cap * d * sizeof(double)); B.parent = (int32_t*)malloc(cap * sizeof(int32_t)); own_b = 1; }
  if (!A.radius) { A.radius = (double*)malloc(cap * sizeof(double)); own_ra = 1; }
  if (!B.radius) { B.radius = (double*)malloc(cap * sizeof(double)); own_rb = 1; }
  const int dd = p->dd_radius > 0.0;

  double* c_rand = (double*)malloc((size_t)d * sizeof(double));
  double* c_new = (double*)malloc((size_t)d * sizeof(double));
  double* c_ext = (double*)malloc((size_t)d * sizeof(double));
  double* c_tgt = (double*)malloc((size_t)d * sizeof(double));
  double* scratch = (double*)malloc((size_t)d * sizeof(double));
  plan_ctx ctx = {r, e, p, res, 0, scratch};

  /* Alg. 1 lines 1-2: T_a <- {c_start}, T_b <- {c_goal}; roots have parent -1. */
  tree_add(&A, q_start, -1);
  tree_add(&B, q_goal, -1);

  if (p->workers >= 1) {
    plan_lockstep(&ctx, &A, &B, c_rand, c_new, c_ext, c_tgt);
    goto done;
  }
  const double delta = p->range, resol = p->resolution;
  for (int32_t it = 0; it < p->max_iters; ++it) {
    ctx.it = it;
    res->iterations = it + 1;
    /* line 3: T_s = smaller tree, T_o = larger; ties extend T_a. */
    int s_is_a = (A.n <= B.n);
    tree* Ts = s_is_a ? &A : &B;
    tree* To = s_is_a ? &B : &A;
    /* line 4: RANDOM_CONFIG, with goal bias toward the opposite root (and the
     * learned proposal when one is given). */
    int amb_k = 0;
    int kind = orc_sample_learned(r, p->seed, p->problem, (uint32_t)it, p->goal_bias, p->gmm,
                                  p->gmm ? p->learned_ratio : 0.0, p->amb_rel, c_rand, &amb_k);
    if (amb_k) note_amb(&ctx, ORC_AMB_COMPONENT);
    if (kind == 1) memcpy(c_rand, To->q, (size_t)d * sizeof(double));
    if (kind == 0 && p->sampler == ORC_SAMPLER_HALTON) {
      /* the paper's sampler: Halton point it + 1 + offset (index 0 is the origin) */
      orc_halton((uint32_t)it + 1u + p->halton_offset, d, c_rand);
      for (int j = 0; j < d; ++j) c_rand[j] = r->lower[j] + c_rand[j] * (r->upper[j] - r->lower[j]);
    }
    /* line 5: NEAREST_NEIGHBOR in T_s. */
    int32_t nn = nearest(&ctx, Ts, c_rand);
    const double* c_nn = Ts->q + (size_t)nn * d;
    /* Alg. 2 line 2: INTERPOLATE -- step from c_nn toward c_rand by at most delta. */
    double dist = sqrt(dist2(c_rand, c_nn, d));
    if (dist <= 0.0) continue; /* no motion: nothing to add */
    /* dynamic domain: a random sample outside the nearest node's radius is rejected */
    if (dd && kind != 1) {
      double rad = Ts->radius[nn];
      if (isfinite(rad) && fabs(dist - rad) <= p->amb_rel * rad) note_amb(&ctx, ORC_AMB_DOMAIN);
      if (dist > rad) {
        res->dd_rejected++;
        continue;
      }
    }
    if (fabs(dist - delta) <= p->amb_rel * delta) note_amb(&ctx, ORC_AMB_STEER);
    double len;
    int clamped = (dist > delta);
    if (clamped) {
      for (int j = 0; j < d; ++j) c_new[j] = c_nn[j] + (c_rand[j] - c_nn[j]) * (delta / dist);
      len = delta;
    } else {
      memcpy(c_new, c_rand, (size_t)d * sizeof(double));
      len = dist;
    }
    /* Alg. 2 lines 3-5: N_cc = ceil(len / resolution) states, all must be free. */
    int32_t n_states = ceil_checked(&ctx, len / resol, clamped);
    int edge_ok = check_edge(&ctx, c_nn, c_new, n_states);
    if (dd) {
      /* radius of the nearest node after its extension (adaptive dynamic domain) */
      double* rad = &Ts->radius[nn];
      if (edge_ok) {
        if (isfinite(*rad)) *rad *= 1.0 + p->dd_alpha;
      } else if (isinf(*rad)) {
        *rad = p->dd_radius;
      } else {
        *rad = fmax(*rad * (1.0 - p->dd_alpha), p->dd_min_radius);
      }
    }
    if (!edge_ok) continue;
    /* line 7: add c_new to T_s. */
    int32_t idx_new = tree_add(Ts, c_new, nn);
    if (idx_new < 0) continue;
    /* line 8: nearest node of T_o to c_new. */
    int32_t nno = nearest(&ctx, To, c_new);
    memcpy(c_tgt, To->q + (size_t)nno * d, (size_t)d * sizeof(double));
    /* lines 9-15: greedy connect in n_ext = ceil(D / delta) steps of length
     * delta along (c_tgt - c_new)/D; the last step lands on c_tgt. */
    double D = sqrt(dist2(c_tgt, c_new, d));
    int32_t n_ext = (D > 0.0) ? ceil_checked(&ctx, D / delta, 0) : 0;
    int32_t prev = idx_new;
    int connected = 1;
    for (int32_t i = 1; i <= n_ext; ++i) {
      double step_len;
      if (i < n_ext) {
        double f = (double)i * delta / D;
        for (int j = 0; j < d; ++j) c_ext[j] = c_new[j] + f * (c_tgt[j] - c_new[j]);
        step_len = delta;
      } else {
        memcpy(c_ext, c_tgt, (size_t)d * sizeof(double));
        step_len = D - (double)(n_ext - 1) * delta;
      }
      int32_t ns = ceil_checked(&ctx, step_len / resol, i < n_ext);
      if (ns < 1) ns = 1;
      const double* from = Ts->q + (size_t)prev * d;
      if (!check_edge(&ctx, from, c_ext, ns)) {
        connected = 0;
        break;
      }
      int32_t added = tree_add(Ts, c_ext, prev);
      if (added < 0) {
        connected = 0;
        break;
      }
      prev = added;
    }
    if (connected) {
      /* line 16: PATH -- the last node of T_s coincides with node nno of T_o. */
      int32_t ja = s_is_a ? prev : nno;
      int32_t jb = s_is_a ? nno : prev;
      res->join_a = ja;
      res->join_b = jb;
      res->n_a = A.n;
      res->n_b = B.n;
      build_path(&ctx, &A, &B, ja, jb);
      goto done;
    }
  }
  res->n_a = A.n;
  res->n_b = B.n;
  res->status = ORC_NO_SOLUTION;
done:
  free(c_rand);
  free(c_new);
  free(c_ext);
  free(c_tgt);
  free(scratch);
  if (own_a) { free(A.q); free(A.parent); }
  if (own_b) { free(B.q); free(B.parent); }
  if (own_ra) free(A.radius);
  if (own_rb) free(B.radius);
  return res->status;
}

int32_t orc_revalidate(const orc_robot* r, const orc_env* e, const double* path,
                       int32_t n, double res, double* min_clearance) {
  int d = r->dof;
  double mc = DBL_MAX;
  int32_t bad = 0;
  double* s = (double*)malloc((size_t)d * sizeof(double));
  if (n > 0) mc = fmin(mc, orc_clearance(r, e, path, NULL, NULL));
  for (int32_t k = 0; k + 1 < n; ++k) {
    const double* a = path + (size_t)k * d;
    const double* b = path + (size_t)(k + 1) * d;
    double len = sqrt(dist2(a, b, d));
    int32_t m = (int32_t)ceil(len / res);
    if (m < 1) m = 1;
    int seg_bad = 0;
    for (int32_t j = 1; j <= m; ++j) {
      double t = (double)j / (double)m;
      for (int i = 0; i < d; ++i) s[i] = a[i] + t * (b[i] - a[i]);
      double c = orc_clearance(r, e, s, NULL, NULL);
      mc = fmin(mc, c);
      if (c < 0.0) seg_bad = 1;
    }
    bad += seg_bad;
  }
  free(s);
  if (min_clearance) *min_clearance = mc;
  return bad;
}

/* ------------------------------------------------------------- batch */
typedef struct batch_ctx {
  orc_problem* problems;
  int32_t n;
  int32_t next;
  pthread_mutex_t lock;
} batch_ctx;

static double now_seconds(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void* batch_worker(void* arg) {
  batch_ctx* b = (batch_ctx*)arg;
  for (;;) {
    pthread_mutex_lock(&b->lock);
    int32_t i = b->next++;
    pthread_mutex_unlock(&b->lock);
    if (i >= b->n) break;
    orc_problem* pr = &b->problems[i];
    double t0 = now_seconds();
    orc_plan(pr->robot, pr->env, pr->q_start, pr->q_goal, &pr->params, pr->result);
    pr->seconds = now_seconds() - t0;
  }
  return NULL;
}

void orc_plan_batch(orc_problem* problems, int32_t n, int32_t threads) {
  batch_ctx b;
  b.problems = problems;
  b.n = n;
  b.next = 0;
  pthread_mutex_init(&b.lock, NULL);
  if (threads < 1) threads = 1;
  pthread_t* th = (pthread_t*)malloc((size_t)threads * sizeof(pthread_t));
  for (int32_t t = 0; t < threads; ++t) pthread_create(&th[t], NULL, batch_worker, &b);
  for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&b.lock);
}
