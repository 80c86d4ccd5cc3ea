// Mesh resolver of Sec. 3 ("Urban model resolving"): cell porosity from
// closed triangle meshes.  A point is inside an object when it lies in the
// object's axis-aligned bounding box and a ray from it crosses the object's
// triangles an odd number of times (even-odd rule); crossings by the
// Moller-Trumbore test (1997), here without the division by the
// determinant: the barycentric and distance tests compare against |det|.
// A cell's porosity is the mean over a uniform sub-grid of sub^3 points of
// the minimum inside porosity of the objects containing the point (1 in the
// open), the volume fraction outside the solids of the cut-cell treatment.
// A point's classification is integer work decided by floating point, so
// every product and sum is a separate round-to-nearest FP64 operation in a
// fixed order (the _rn intrinsics are never fused into FMAs).
#pragma once
#include <cuda_runtime.h>

#include "uf_device.cuh"

namespace uf {

// Ray direction: no zero component, so no face of an axis-aligned box is
// parallel to it.
constexpr double RAY_X = 0.5741, RAY_Y = 0.6219, RAY_Z = 0.5327;

struct MeshObject {
  int first, count;     // triangles [first, first + count)
  double phi_in;        // porosity inside
  double lo[3], hi[3];  // bounding box [m]
  int clo[3], chi[3];   // cells [clo, chi] per axis whose closed box meets the bounding box
};

__device__ __forceinline__ double dot3_rn(double ax, double ay, double az, double bx, double by, double bz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)), __dmul_rn(az, bz));
}

// Triangles [first, first + count) crossed by the ray p + t RAY, t > 0.
__device__ __forceinline__ int ray_crossings(double px, double py, double pz, const double* __restrict__ tri,
                                             int first, int count) {
  int n = 0;
  for (int e = first; e < first + count; ++e) {
    const double* v = tri + 9 * (size_t)e;
    const double e1x = __dsub_rn(v[3], v[0]), e1y = __dsub_rn(v[4], v[1]), e1z = __dsub_rn(v[5], v[2]);
    const double e2x = __dsub_rn(v[6], v[0]), e2y = __dsub_rn(v[7], v[1]), e2z = __dsub_rn(v[8], v[2]);
    // q = RAY x e2, det = e1 . q
    const double qx = __dsub_rn(__dmul_rn(RAY_Y, e2z), __dmul_rn(RAY_Z, e2y));
    const double qy = __dsub_rn(__dmul_rn(RAY_Z, e2x), __dmul_rn(RAY_X, e2z));
    const double qz = __dsub_rn(__dmul_rn(RAY_X, e2y), __dmul_rn(RAY_Y, e2x));
    const double det = dot3_rn(e1x, e1y, e1z, qx, qy, qz);
    if (det == 0.0) continue;
    const double s = det > 0.0 ? 1.0 : -1.0;
    const double adet = __dmul_rn(det, s);
    const double tx = __dsub_rn(px, v[0]), ty = __dsub_rn(py, v[1]), tz = __dsub_rn(pz, v[2]);
    const double u = __dmul_rn(dot3_rn(tx, ty, tz, qx, qy, qz), s);
    // r = t x e1
    const double rx = __dsub_rn(__dmul_rn(ty, e1z), __dmul_rn(tz, e1y));
    const double ry = __dsub_rn(__dmul_rn(tz, e1x), __dmul_rn(tx, e1z));
    const double rz = __dsub_rn(__dmul_rn(tx, e1y), __dmul_rn(ty, e1x));
    const double w = __dmul_rn(dot3_rn(RAY_X, RAY_Y, RAY_Z, rx, ry, rz), s);
    const double t = __dmul_rn(dot3_rn(e2x, e2y, e2z, rx, ry, rz), s);
    if (u >= 0.0 && u <= adet && w >= 0.0 && __dadd_rn(u, w) <= adet && t > 0.0) ++n;
  }
  return n;
}

// One warp per cell, eight cells per block of 256 threads (blockIdx.x
// enumerates cells x fastest).  Lane 0 lists the objects whose box meets
// the cell (all of them past MESH_LIST) from their integer cell ranges: a
// cell in the open is 1 at once.
// The lanes then classify the sub^3 sample points 32 at a time, and lane 0
// adds each round's values in sample order (c, b, a), so the sum is the
// same sequence of roundings whatever the lane count.  Skipping an object
// whose box misses the cell changes no decision: no sample point can lie in
// its box.
constexpr int MESH_LIST = 64;
constexpr int MESH_WARPS = 8;

template <typename T>
__global__ void __launch_bounds__(32 * MESH_WARPS) k_mesh_phi(int nx, int ny, int nz, int P, double h, int sub,
                                                              const double* __restrict__ tri,
                                                              const MeshObject* __restrict__ obj, int nobj,
                                                              T* __restrict__ phi) {
  __shared__ int s_list[MESH_WARPS][MESH_LIST];
  __shared__ int s_n[MESH_WARPS];
  __shared__ double s_val[MESH_WARPS][32];
  __shared__ double s_off[16];          // sample offsets (a + 1/2) / sub within a cell
  if (threadIdx.x < sub) s_off[threadIdx.x] = __ddiv_rn(__dadd_rn((double)threadIdx.x, 0.5), (double)sub);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long cell = (long long)blockIdx.x * MESH_WARPS + warp;
  if (cell >= (long long)nx * ny * nz) return;      // whole warps leave together
  const int i = (int)(cell % nx), j = (int)((cell / nx) % ny), k = (int)(cell / ((long long)nx * ny));
  const size_t c_out = (size_t)i + (size_t)P * ((size_t)j + (size_t)ny * k);
  if (lane == 0) {
    int nl = 0;
    for (int o = 0; o < nobj; ++o) {
      const MeshObject& m = obj[o];
      if (i < m.clo[0] || i > m.chi[0] || j < m.clo[1] || j > m.chi[1] || k < m.clo[2] || k > m.chi[2]) continue;
      if (nl == MESH_LIST) {
        nl = -1;                        // too many: visit every object
        break;
      }
      s_list[warp][nl++] = o;
    }
    s_n[warp] = nl;
  }
  __syncwarp();
  const int nl = s_n[warp];
  if (nl == 0) {                        // the open: every point is 1, and so is their mean
    if (lane == 0) phi[c_out] = T(1);
    return;
  }
  const int n_obj = nl < 0 ? nobj : nl;
  const int npts = sub * sub * sub;
  double acc = 0.0;
  for (int base = 0; base < npts; base += 32) {
    const int e = base + lane;
    double val = 1.0;
    if (e < npts) {
      const int a = e % sub, b = (e / sub) % sub, c = e / (sub * sub);
      const double px = __dmul_rn(__dadd_rn((double)i, s_off[a]), h);
      const double py = __dmul_rn(__dadd_rn((double)j, s_off[b]), h);
      const double pz = __dmul_rn(__dadd_rn((double)k, s_off[c]), h);
      for (int q = 0; q < n_obj; ++q) {
        const MeshObject& m = obj[nl < 0 ? q : s_list[warp][q]];
        if (px < m.lo[0] || px > m.hi[0] || py < m.lo[1] || py > m.hi[1] || pz < m.lo[2] || pz > m.hi[2]) continue;
        if (ray_crossings(px, py, pz, tri, m.first, m.count) & 1) val = fmin(val, m.phi_in);
      }
    }
    s_val[warp][lane] = val;
    __syncwarp();
    if (lane == 0)
      for (int l = 0; l < 32 && base + l < npts; ++l) acc = __dadd_rn(acc, s_val[warp][l]);
    __syncwarp();
  }
  if (lane == 0) phi[c_out] = (T)__ddiv_rn(acc, (double)npts);
}

}  // namespace uf
