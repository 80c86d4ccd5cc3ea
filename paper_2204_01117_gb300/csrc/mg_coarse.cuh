// The coarse part of the multigrid V-cycle in one launch: a thread-block
// cluster runs the down and up legs of levels cs .. lt-1 and, on its first
// CTA, the shared-memory tail of levels lt .. nl-1.
//
// The per-level kernels (k_mg_down, k_mg_up) need one launch per level and
// leg, and on the coarse levels each launch is a few microseconds of
// latency for little work.  Here each level's leg is two phases over all the
// cluster's threads, separated by cluster barriers (barrier.cluster, with
// release/acquire semantics); the level arrays stay in global memory, which
// the L2 holds:
//   down, level m:  x = presmoothed r (from zero);  | r_{m+1} = R (r - A x)
//   up, level m:    u = relax(x + P e_{m+1});       | t_m = relax(u)
// Every value is formed by the expressions of k_mg_down / k_mg_up: the same
// neighbour sums in the same order (zero outside the level), the same
// restriction order over the children, the same smoother functions.  So the
// V-cycle is bit for bit the one of the per-level kernels, and a grid in a
// batch (which keeps those) still computes what it computes alone.
//
// Cells of a level go to CTA rank r by z plane (k = r, r + CL, ...) and to
// threads by a 32 x 32 layout in the plane; reads of data other CTAs wrote
// in this launch go through the L2 (ld.global.cg).  No CTA returns early
// unless all do (the convergence flag, set before the launch), so every CTA
// reaches every cluster barrier.
#pragma once
#include <cooperative_groups.h>

#include "mg_fused.cuh"

namespace uf {

constexpr int CT = TAIL_T;   // threads per CTA (CTA 0 also runs the tail)

template <typename T>
struct CoarseArgs {
  Level<T> lv[MAX_LEVELS];
  T* lu[MAX_LEVELS];   // scratch of the first post-smoothing pass of each level
  int cs, lt;          // levels cs .. lt-1 here, lt .. nl-1 in the tail
};

// Diagonal of a level operator as the per-level kernels form it: the x-y
// part (pos_xy) plus the z part (diag_z).
template <typename T>
__device__ __forceinline__ T diag_xyz(const Level<T>& L, int i, int j, int k) {
  T D = T(2) * (L.wx + L.wy);
  if (i == 0 && !(L.out_mask & 1)) D -= L.wx;
  if (i == L.nx - 1 && !(L.out_mask & 2)) D -= L.wx;
  if (j == 0 && !(L.out_mask & 4)) D -= L.wy;
  if (j == L.ny - 1 && !(L.out_mask & 8)) D -= L.wy;
  return D + diag_z(L, k);
}

template <typename F>
__device__ __forceinline__ void cluster_cells(int nx, int ny, int nz, int rank, int nrank, F f) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = rank; k < nz; k += nrank)
    for (int j = ty; j < ny; j += 32)
      for (int i = tx; i < nx; i += 32) f(i, j, k);
}

template <typename T>
__device__ __forceinline__ T ldl(const T* p) { return __ldcg(p); }

// q = r / D on level L, zero outside.
template <typename T>
__device__ __forceinline__ T q_at(const Level<T>& L, int i, int j, int k) {
  if (!in_level(L, i, j, k)) return T(0);
  return ldl(L.r + lidx(L, i, j, k)) * rdiag(diag_xyz(L, i, j, k));
}
template <typename T>
__device__ __forceinline__ T x_at(const Level<T>& L, int i, int j, int k) {
  return in_level(L, i, j, k) ? ldl(L.x + lidx(L, i, j, k)) : T(0);
}

template <typename T>
__device__ __forceinline__ T coarse_resid(const Level<T>& L, int i, int j, int k) {
  const T D = diag_xyz(L, i, j, k);
  const T xv = ldl(L.x + lidx(L, i, j, k));
  const T q = ldl(L.r + lidx(L, i, j, k)) * rdiag(D);
  return resid(D, q, xv,
               nb6(L.wx, x_at(L, i - 1, j, k), x_at(L, i + 1, j, k), L.wy, x_at(L, i, j - 1, k), x_at(L, i, j + 1, k),
                   L.wz, x_at(L, i, j, k - 1), x_at(L, i, j, k + 1)));
}

// to_tail: C is the tail's first level, whose right-hand side the tail
// forms itself from L's residual under linear transfers.
template <typename T, int SM>
__device__ __forceinline__ void coarse_down(const Level<T>& L, const Level<T>& C, const SmoothW<T>& W, bool to_tail,
                                            int rank, int nrank, cooperative_groups::cluster_group& cl) {
  // pre-smoothing from zero (computeX of mg_down_body)
  cluster_cells(L.nx, L.ny, L.nz, rank, nrank, [&](int i, int j, int k) {
    const T qc = q_at(L, i, j, k);
    const T s = nb6(L.wx, q_at(L, i - 1, j, k), q_at(L, i + 1, j, k), L.wy, q_at(L, i, j - 1, k), q_at(L, i, j + 1, k),
                    L.wz, q_at(L, i, j, k - 1), q_at(L, i, j, k + 1));
    L.x[lidx(L, i, j, k)] = presmooth<SM>(qc, s, diag_xyz(L, i, j, k), W, ((i + j + k) & 1) == 0);
  });
  cl.sync();
  if (L.lin) {   // residual into L.t, then the linear restriction (as k_restrict_lin)
    cluster_cells(L.nx, L.ny, L.nz, rank, nrank,
                  [&](int i, int j, int k) { L.t[lidx(L, i, j, k)] = coarse_resid(L, i, j, k); });
    cl.sync();
    if (!to_tail) {
      cluster_cells(C.nx, C.ny, C.nz, rank, nrank, [&](int ci, int cj, int ck) {
        C.r[lidx(C, ci, cj, ck)] =
            restrict_lin(L, C, ci, cj, ck, [&](int i, int j, int k) { return ldl(L.t + lidx(L, i, j, k)); });
      });
      cl.sync();
    }
    return;
  }
  // residual and summed restriction (children in the order of mg_down_body)
  const int fx = L.cx ? 2 : 1, fy = L.cy ? 2 : 1;
  cluster_cells(C.nx, C.ny, C.nz, rank, nrank, [&](int ci, int cj, int ck) {
    T sum = 0;
    for (int dz = L.cz ? 1 : 0; dz >= 0; --dz) {
      const int k = L.cz ? 2 * ck + 1 - dz : ck;
      for (int dy = 0; dy < fy; ++dy)
        for (int dx = 0; dx < fx; ++dx) {
          const int i = ci * fx + dx, j = cj * fy + dy;
          sum += in_level(L, i, j, k) ? coarse_resid(L, i, j, k) : T(0);
        }
    }
    C.r[lidx(C, ci, cj, ck)] = sum;
  });
  cl.sync();
}

template <typename T, int SM>
__device__ __forceinline__ void coarse_up(const Level<T>& L, const Level<T>& C, T* U, const SmoothW<T>& W, int rank,
                                          int nrank, cooperative_groups::cluster_group& cl) {
  // t = x + P e, zero outside (commitT of mg_up_body)
  auto t_at = [&](int i, int j, int k) -> T {
    if (!in_level(L, i, j, k)) return T(0);
    if (L.lin)
      return ldl(L.x + lidx(L, i, j, k)) +
             prolong_lin(L, C, i, j, k, [&](int a, int b, int c) { return ldl(C.t + lidx(C, a, b, c)); });
    const int pi = L.cx ? i >> 1 : i, pj = L.cy ? j >> 1 : j, pk = L.cz ? k >> 1 : k;
    return ldl(L.x + lidx(L, i, j, k)) + ldl(C.t + lidx(C, pi, pj, pk));
  };
  cluster_cells(L.nx, L.ny, L.nz, rank, nrank, [&](int i, int j, int k) {
    const T tc = t_at(i, j, k);
    const T s = nb6(L.wx, t_at(i - 1, j, k), t_at(i + 1, j, k), L.wy, t_at(i, j - 1, k), t_at(i, j + 1, k), L.wz,
                    t_at(i, j, k - 1), t_at(i, j, k + 1));
    const size_t c = lidx(L, i, j, k);
    U[c] = relax<SM>(tc, ldl(L.r + c), s, diag_xyz(L, i, j, k), W.w1, ((i + j + k) & 1) == 1);
  });
  cl.sync();
  auto u_at = [&](int i, int j, int k) -> T { return in_level(L, i, j, k) ? ldl(U + lidx(L, i, j, k)) : T(0); };
  cluster_cells(L.nx, L.ny, L.nz, rank, nrank, [&](int i, int j, int k) {
    const T uc = u_at(i, j, k);
    const T s = nb6(L.wx, u_at(i - 1, j, k), u_at(i + 1, j, k), L.wy, u_at(i, j - 1, k), u_at(i, j + 1, k), L.wz,
                    u_at(i, j, k - 1), u_at(i, j, k + 1));
    const size_t c = lidx(L, i, j, k);
    L.t[c] = relax<SM>(uc, ldl(L.r + c), s, diag_xyz(L, i, j, k), W.w2, ((i + j + k) & 1) == 0);
  });
  cl.sync();
}

template <typename T, int SM>
__global__ void __launch_bounds__(CT) k_mg_coarse(const __grid_constant__ CoarseArgs<T> A,
                                                 const __grid_constant__ TailArgs<T> tail, SmoothW<T> W,
                                                 const SolveState* st) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  if (st->converged) return;   // set before this launch: the same in every CTA
  const int rank = (int)cl.block_rank(), nrank = (int)cl.num_blocks();
  for (int m = A.cs; m < A.lt; ++m) coarse_down<T, SM>(A.lv[m], A.lv[m + 1], W, m + 1 == A.lt, rank, nrank, cl);
  if (rank == 0) mg_tail_body<T, SM>(tail, W, st, vblock());
  cl.sync();
  for (int m = A.lt - 1; m >= A.cs; --m) coarse_up<T, SM>(A.lv[m], A.lv[m + 1], A.lu[m], W, rank, nrank, cl);
}

}  // namespace uf
