// prrtc_esdf.cu -- Euclidean signed distance fields on a voxel grid for the
// collision check against distance maps (the paper's ESDF setting, Sec. III-A
// and its real-world experiments): voxelisation of primitive obstacles and
// the signed distance transform of an occupancy grid.
//
// The transform is exact: squared distances between voxel centres are
// integers, and the squared Euclidean distance separates into three 1-D
// minimisations (along x, then y, then z) of f(j) + (i - j)^2.  Each pass
// computes, for every voxel, both the distance to the nearest occupied voxel
// (read by free voxels) and to the nearest free voxel (read by occupied
// ones).  A thread per voxel scans its line; neighbouring threads scan the
// same line positions, so the reads are broadcast (x) or coalesced (y, z).
#include "prrtc.h"
#include "prrtc_launch.h"

namespace prrtc {
namespace {

constexpr int kInf = 1 << 29;  // "no site on this line"; + n^2 cannot overflow

__global__ void voxelize_kernel(EnvView env, float ox, float oy, float oz, float voxel, int nx, int ny, int nz,
                                uint8_t* __restrict__ occ) {
  const size_t V = (size_t)nx * ny * nz;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((size_t)nx * ny));
    const float px = ox + ((float)i + 0.5f) * voxel, py = oy + ((float)j + 0.5f) * voxel,
                pz = oz + ((float)k + 0.5f) * voxel;
    bool inside = false;
    const float4* e = env.data;
    for (int o = 0; o < env.n_aabb; ++o) {
      const float4 c = e[2 * o], h = e[2 * o + 1];
      inside |= fabsf(px - c.x) < h.x && fabsf(py - c.y) < h.y && fabsf(pz - c.z) < h.z;
    }
    e += 2 * env.n_aabb;
    for (int o = 0; o < env.n_obb; ++o) {
      const float4 c = e[5 * o], h = e[5 * o + 1], a = e[5 * o + 2], b = e[5 * o + 3], d = e[5 * o + 4];
      const float vx = px - c.x, vy = py - c.y, vz = pz - c.z;
      const float lx = fmaf(a.x, vx, fmaf(a.y, vy, a.z * vz));
      const float ly = fmaf(b.x, vx, fmaf(b.y, vy, b.z * vz));
      const float lz = fmaf(d.x, vx, fmaf(d.y, vy, d.z * vz));
      inside |= fabsf(lx) < h.x && fabsf(ly) < h.y && fabsf(lz) < h.z;
    }
    e += 5 * env.n_obb;
    for (int o = 0; o < env.n_cyl; ++o) {
      const float4 c = e[2 * o], a = e[2 * o + 1];
      const float vx = px - c.x, vy = py - c.y, vz = pz - c.z;
      const float z = fmaf(a.x, vx, fmaf(a.y, vy, a.z * vz));
      const float wx = fmaf(-z, a.x, vx), wy = fmaf(-z, a.y, vy), wz = fmaf(-z, a.z, vz);
      inside |= fabsf(z) < a.w && fmaf(wx, wx, fmaf(wy, wy, wz * wz)) < c.w * c.w;
    }
    e += 2 * env.n_cyl;
    for (int o = 0; o < env.n_sph; ++o) {
      const float4 s = e[o];
      const float dx = px - s.x, dy = py - s.y, dz = pz - s.z;
      inside |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < s.w * s.w;
    }
    occ[v] = inside ? 1 : 0;
  }
}

// Pass along x: squared distance along the row to the nearest occupied
// (.x) and nearest free (.y) voxel.
__global__ void edt_x_kernel(const uint8_t* __restrict__ occ, int nx, size_t V, int2* __restrict__ out) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % nx);
    const uint8_t* row = occ + (v - i);
    int bo = kInf, bf = kInf;
    for (int ii = 0; ii < nx; ++ii) {
      const int d = (i - ii) * (i - ii);
      if (row[ii]) bo = min(bo, d);
      else bf = min(bf, d);
    }
    out[v] = make_int2(bo, bf);
  }
}

// Pass along an axis of length n and element stride `stride` (y: nx, z:
// nx*ny): out(v) = min over positions t of in(t) + (pos(v) - t)^2.
__global__ void edt_axis_kernel(const int2* __restrict__ in, int n, size_t stride, size_t V, int2* __restrict__ out) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    const int pos = (int)((v / stride) % n);
    const int2* line = in + (v - (size_t)pos * stride);
    int bo = kInf, bf = kInf;
    for (int t = 0; t < n; ++t) {
      const int2 f = line[(size_t)t * stride];
      const int d = (pos - t) * (pos - t);
      if (f.x < kInf) bo = min(bo, f.x + d);
      if (f.y < kInf) bf = min(bf, f.y + d);
    }
    out[v] = make_int2(bo, bf);
  }
}

// Signed field: free voxels +voxel * sqrt(d2 to occupied), occupied voxels
// -voxel * sqrt(d2 to free); +/- the grid diagonal when no such voxel exists.
__global__ void esdf_final_kernel(const uint8_t* __restrict__ occ, const int2* __restrict__ d2, size_t V, float voxel,
                                  float diag, float* __restrict__ out) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    const int2 d = d2[v];
    const int q = occ[v] ? d.y : d.x;
    const float mag = q >= kInf ? diag : voxel * sqrtf((float)q);
    out[v] = occ[v] ? -mag : mag;
  }
}

int grid_for(size_t V) {
  const size_t blocks = (V + 255) / 256;
  return (int)(blocks < 65535 ? blocks : 65535);
}

}  // namespace

cudaError_t launch_voxelize(const EnvView& env, const float origin[3], float voxel, const int dims[3], uint8_t* occ,
                            cudaStream_t stream) {
  const size_t V = (size_t)dims[0] * dims[1] * dims[2];
  if (V == 0) return cudaSuccess;
  voxelize_kernel<<<grid_for(V), 256, 0, stream>>>(env, origin[0], origin[1], origin[2], voxel, dims[0], dims[1],
                                                   dims[2], occ);
  return cudaGetLastError();
}

cudaError_t launch_esdf(const uint8_t* occ, const int dims[3], float voxel, int2* tmp_a, int2* tmp_b, float* out,
                        cudaStream_t stream) {
  const size_t V = (size_t)dims[0] * dims[1] * dims[2];
  if (V == 0) return cudaSuccess;
  const int g = grid_for(V);
  edt_x_kernel<<<g, 256, 0, stream>>>(occ, dims[0], V, tmp_a);
  edt_axis_kernel<<<g, 256, 0, stream>>>(tmp_a, dims[1], (size_t)dims[0], V, tmp_b);
  edt_axis_kernel<<<g, 256, 0, stream>>>(tmp_b, dims[2], (size_t)dims[0] * dims[1], V, tmp_a);
  const float diag = voxel * sqrtf((float)dims[0] * dims[0] + (float)dims[1] * dims[1] + (float)dims[2] * dims[2]);
  esdf_final_kernel<<<g, 256, 0, stream>>>(occ, tmp_a, V, voxel, diag, out);
  return cudaGetLastError();
}

}  // namespace prrtc
