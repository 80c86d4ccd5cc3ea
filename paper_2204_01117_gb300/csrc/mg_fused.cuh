// Fused multigrid V-cycle and CG kernels (shared-memory tiles).
//
// Each block owns a TX x TY x TZ tile of a level (thread (tx, ty) owns the
// column of TZ cells at x = tx, y = ty) and stages the tile plus a halo in
// shared memory, so that two dependent smoothing passes and the residual run
// without another trip to global memory:
//
//   k_mg_down  : [finest level: CG update x += a d, r -= a q, ||r||^2]
//                pre-smoothing from a zero guess, residual, summed
//                restriction to the next level.            reads r (q, x, d)
//   k_mg_up    : coarse-grid correction (piecewise-constant prolongation) and
//                the post-smoothing passes; on the finest level also r.z and
//                the CG beta.                              reads x_pre, e, r
//   k_mg_tail  : one block runs the whole V-cycle below a level that fits in
//                shared memory; coarsest level by its dense FP64 inverse.
//   k_cg_dir_q : d = z + beta d_old and q = A d, plus d.q and alpha.
//
// Cells outside the domain are staged as zeros, so every neighbour sum is
// the same branch-free 6-term expression: with zero ghosts,
// A x = D_c x_c - sum_6 w_a x_nb holds for the BC-aware operator because
// the diagonal D_c already counts only interior and outlet faces.
//
// Smoothers (template SM): damped Jacobi, two sweeps before and after the
// coarse correction, or red-black Gauss-Seidel, red then black before and
// black then red after (the adjoint order).  Either way the V-cycle is a
// symmetric positive definite preconditioner for CG.
#pragma once
#include "solver_kernels.cuh"

namespace uf {

enum Smoother { SM_JACOBI = 0, SM_RBGS = 1 };

constexpr int TX = 32, TY = 8, TZ = 4;
constexpr int H2X = TX + 4, H2Y = TY + 4, H2Z = TZ + 4, H2P = H2X * H2Y, H2N = H2P * H2Z;   // halo 2
constexpr int H1X = TX + 2, H1Y = TY + 2, H1Z = TZ + 2, H1P = H1X * H1Y, H1N = H1P * H1Z;   // halo 1
constexpr int TN = TX * TY * TZ;
constexpr int FT = TX * TY;   // 256 threads per fused block

template <typename T>
__device__ __forceinline__ bool in_level(const Level<T>& L, int i, int j, int k) {
  return i >= 0 && j >= 0 && k >= 0 && i < L.nx && j < L.ny && k < L.nz;
}

// Diagonal of the level operator: 2 (wx + wy + wz) minus the weight of every
// wall / inlet face (dp/dn = 0).
template <typename T>
__device__ __forceinline__ T diag_of(const Level<T>& L, int i, int j, int k) {
  T D = T(2) * (L.wx + L.wy + L.wz);
  if (i == 0 && !(L.out_mask & 1)) D -= L.wx;
  if (i == L.nx - 1 && !(L.out_mask & 2)) D -= L.wx;
  if (j == 0 && !(L.out_mask & 4)) D -= L.wy;
  if (j == L.ny - 1 && !(L.out_mask & 8)) D -= L.wy;
  if (k == 0 && !(L.out_mask & 16)) D -= L.wz;
  if (k == L.nz - 1 && !(L.out_mask & 32)) D -= L.wz;
  return D;
}

// sum_6 w_a s[nb] for a staged array with plane pitch P and row pitch X.
template <typename T, int X, int P>
__device__ __forceinline__ T nbs(const Level<T>& L, const T* s, int b) {
  return L.wx * (s[b - 1] + s[b + 1]) + L.wy * (s[b - X] + s[b + X]) + L.wz * (s[b - P] + s[b + P]);
}

// Two positions per thread cover a W x H plane (W*H <= 2*FT).
struct PlaneMap {
  int x0, y0, x1, y1;
  bool has1;
};
template <int W, int H>
__device__ __forceinline__ PlaneMap plane_map() {
  static_assert(W * H <= 2 * FT && W * H >= FT, "plane map covers two positions per thread");
  PlaneMap m;
  const int t = threadIdx.x, t1 = t + FT;
  m.x0 = t % W;
  m.y0 = t / W;
  m.has1 = t1 < W * H;
  m.x1 = t1 % W;
  m.y1 = t1 / W;
  return m;
}

// Pre-smoothing from zero with q = r/D staged: Jacobi x2 = w(2-w) q_c +
// w^2/D_c sum w_a q_nb;  RBGS red q_c, black q_c + sum w_a q_nb / D_c.
template <int SM, typename T>
__device__ __forceinline__ T presmooth(T qc, T s, T D, T omega, bool red) {
  if (SM == SM_JACOBI) return omega * (T(2) - omega) * qc + omega * omega * s / D;
  return red ? qc : qc + s / D;
}
// Post-smoothing pass on t: Jacobi t + w (r - D t + s)/D; RBGS relaxes the
// colour `relax` and keeps the other.
template <int SM, typename T>
__device__ __forceinline__ T relax(T tc, T rc, T s, T D, T omega, bool active) {
  if (SM == SM_JACOBI) return tc + omega * (rc - D * tc + s) / D;
  return active ? (rc + s) / D : tc;
}

// ------------------------------------------------------------ down -------
template <typename T, int SM, bool CG>
__global__ void __launch_bounds__(FT) k_mg_down(Level<T> F, Level<T> C, T omega, T* __restrict__ x,
                                               const T* d0, const T* d1, const T* __restrict__ q,
                                               double* partials, SolveState* st, cudaGraphConditionalHandle cond,
                                               int use_cond) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Sq = reinterpret_cast<T*>(smem_raw);   // H2N: r/D on tile + halo 2 (0 outside)
  T* Sx = Sq + H2N;                          // H1N: pre-smoothed x on tile + halo 1 (0 outside)
  T* Ss = Sx + H1N;                          // TN : fine residual of owned cells
  __shared__ double sh[32];
  __shared__ bool last;
  if (!CG && st->converged) return;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * TZ;
  const int tid = threadIdx.x, tx = tid & (TX - 1), ty = tid / TX;
  const int it0 = st->iter;
  const T* r_in = level_r(F, it0);
  T* r_out = level_r(F, it0 + 1);
  T alpha = 0;
  const T* dn = nullptr;
  if (CG) {
    dn = (it0 & 1) ? d0 : d1;
    alpha = (T)st->alpha;
  }
  // 1. q = r/D (CG-updated r on the finest level) on tile + halo 2
  {
    const PlaneMap m = plane_map<H2X, H2Y>();
#pragma unroll 2
    for (int ez = 0; ez < H2Z; ++ez) {
      const int gk = k0 - 2 + ez;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !m.has1) break;
        const int ex = h ? m.x1 : m.x0, ey = h ? m.y1 : m.y0;
        const int gi = i0 - 2 + ex, gj = j0 - 2 + ey;
        T v = 0;
        if (in_level(F, gi, gj, gk)) {
          const size_t c = lidx(F, gi, gj, gk);
          T rv = r_in[c];
          if (CG) rv -= alpha * q[c];
          v = rv / diag_of(F, gi, gj, gk);
        }
        Sq[ex + H2X * ey + H2P * ez] = v;
      }
    }
  }
  const int gi = i0 + tx, gj = j0 + ty;
  const bool col_in = gi < F.nx && gj < F.ny;
  double acc = 0.0;
  if (CG && col_in) {   // owned cells: r and x updates, ||r||^2
#pragma unroll
    for (int z = 0; z < TZ; ++z) {
      const int gk = k0 + z;
      if (gk < F.nz) {
        const size_t c = lidx(F, gi, gj, gk);
        const T rv = r_in[c] - alpha * q[c];
        r_out[c] = rv;
        x[c] += alpha * dn[c];
        acc += (double)rv * (double)rv;
      }
    }
  }
  __syncthreads();
  // 2. pre-smoothed x on tile + halo 1
  {
    const PlaneMap m = plane_map<H1X, H1Y>();
#pragma unroll 2
    for (int ez = 0; ez < H1Z; ++ez) {
      const int gk = k0 - 1 + ez;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !m.has1) break;
        const int ex = h ? m.x1 : m.x0, ey = h ? m.y1 : m.y0;
        const int hi = i0 - 1 + ex, hj = j0 - 1 + ey;
        T v = 0;
        if (in_level(F, hi, hj, gk)) {
          const int b = (ex + 1) + H2X * (ey + 1) + H2P * (ez + 1);
          v = presmooth<SM>(Sq[b], nbs<T, H2X, H2P>(F, Sq, b), diag_of(F, hi, hj, gk), omega,
                            ((hi + hj + gk) & 1) == 0);
        }
        Sx[ex + H1X * ey + H1P * ez] = v;
      }
    }
  }
  __syncthreads();
  // 3. owned cells: store x_pre; residual r - A x = D (q - x) + sum w x_nb
#pragma unroll
  for (int z = 0; z < TZ; ++z) {
    const int gk = k0 + z;
    T res = 0;
    if (col_in && gk < F.nz) {
      const int b1 = (tx + 1) + H1X * (ty + 1) + H1P * (z + 1);
      const int b2 = (tx + 2) + H2X * (ty + 2) + H2P * (z + 2);
      const T xc = Sx[b1];
      F.x[lidx(F, gi, gj, gk)] = xc;
      res = diag_of(F, gi, gj, gk) * (Sq[b2] - xc) + nbs<T, H1X, H1P>(F, Sx, b1);
    }
    Ss[tx + TX * (ty + TY * z)] = res;
  }
  __syncthreads();
  // 4. restriction: coarse cells of this tile sum their children in order
  const int fx = F.cx ? 2 : 1, fy = F.cy ? 2 : 1, fz = F.cz ? 2 : 1;
  const int cnx = TX / fx, cny = TY / fy, cnz = TZ / fz;
  for (int e = tid; e < cnx * cny * cnz; e += FT) {
    const int cxl = e % cnx, cyl = (e / cnx) % cny, czl = e / (cnx * cny);
    const int ci = i0 / fx + cxl, cj = j0 / fy + cyl, ck = k0 / fz + czl;
    if (!in_level(C, ci, cj, ck)) continue;
    T s = 0;
    for (int dz = 0; dz < fz; ++dz)
      for (int dy = 0; dy < fy; ++dy)
        for (int dx = 0; dx < fx; ++dx) s += Ss[(cxl * fx + dx) + TX * ((cyl * fy + dy) + TY * (czl * fz + dz))];
    C.r[lidx(C, ci, cj, ck)] = s;
  }
  if (CG) {
    acc = block_sum<FT>(acc, sh);
    const double vals[1] = {acc};
    if (publish_partials<1>(partials, &st->ticket[3], vals, &last)) {
      double tot[1];
      reduce_partials_sum<FT, 1>(partials, tot, sh);
      if (tid == 0) {
        const double rr = tot[0];
        st->rr = rr;
        st->iter = it0 + 1;
        st->total_iters += 1;
        if (!(rr == rr) || isinf(rr)) {
          st->status = DEV_NAN;
          if (st->sticky == 0) st->sticky = DEV_NAN;
          st->converged = 1;
        } else if (rr <= st->tol2 * st->bb) {
          st->converged = 1;
        } else if (it0 + 1 >= st->max_iter) {
          st->status = DEV_NOT_CONVERGED;
          if (st->sticky == 0) st->sticky = DEV_NOT_CONVERGED;
          st->converged = 1;
        }
        if (st->converged && use_cond) cudaGraphSetConditional(cond, 0);
        st->ticket[3] = 0u;
      }
    }
  }
}

// -------------------------------------------------------------- up -------
// t = x_pre + e(parent); two post-smoothing passes; output to `out`
// (F.t on coarse levels, z on the finest).  FINEST: also r.z, beta.
template <typename T, int SM, bool FINEST>
__global__ void __launch_bounds__(FT) k_mg_up(Level<T> F, Level<T> C, T omega, T* __restrict__ out, int mode,
                                             double* partials, SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* St = reinterpret_cast<T*>(smem_raw);   // H2N: corrected x on tile + halo 2 (0 outside)
  T* Su = St + H2N;                          // H1N: after the first pass (0 outside)
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->converged) return;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * TZ;
  const int tid = threadIdx.x, tx = tid & (TX - 1), ty = tid / TX;
  const T* rcur = level_r(F, st->iter);
  {
    const PlaneMap m = plane_map<H2X, H2Y>();
#pragma unroll 2
    for (int ez = 0; ez < H2Z; ++ez) {
      const int gk = k0 - 2 + ez;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !m.has1) break;
        const int ex = h ? m.x1 : m.x0, ey = h ? m.y1 : m.y0;
        const int hi = i0 - 2 + ex, hj = j0 - 2 + ey;
        T v = 0;
        if (in_level(F, hi, hj, gk)) {
          const int pi = F.cx ? hi >> 1 : hi, pj = F.cy ? hj >> 1 : hj, pk = F.cz ? gk >> 1 : gk;
          v = F.x[lidx(F, hi, hj, gk)] + C.t[lidx(C, pi, pj, pk)];
        }
        St[ex + H2X * ey + H2P * ez] = v;
      }
    }
  }
  __syncthreads();
  // first pass over tile + halo 1 (Jacobi sweep / black cells)
  {
    const PlaneMap m = plane_map<H1X, H1Y>();
#pragma unroll 2
    for (int ez = 0; ez < H1Z; ++ez) {
      const int gk = k0 - 1 + ez;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !m.has1) break;
        const int ex = h ? m.x1 : m.x0, ey = h ? m.y1 : m.y0;
        const int hi = i0 - 1 + ex, hj = j0 - 1 + ey;
        T v = 0;
        if (in_level(F, hi, hj, gk)) {
          const int b = (ex + 1) + H2X * (ey + 1) + H2P * (ez + 1);
          v = relax<SM>(St[b], rcur[lidx(F, hi, hj, gk)], nbs<T, H2X, H2P>(F, St, b), diag_of(F, hi, hj, gk), omega,
                        ((hi + hj + gk) & 1) == 1);
        }
        Su[ex + H1X * ey + H1P * ez] = v;
      }
    }
  }
  __syncthreads();
  const int gi = i0 + tx, gj = j0 + ty;
  double acc = 0.0;
  if (gi < F.nx && gj < F.ny) {
#pragma unroll
    for (int z = 0; z < TZ; ++z) {
      const int gk = k0 + z;
      if (gk >= F.nz) break;
      const int b = (tx + 1) + H1X * (ty + 1) + H1P * (z + 1);
      const size_t c = lidx(F, gi, gj, gk);
      const T rc = rcur[c];
      const T zv = relax<SM>(Su[b], rc, nbs<T, H1X, H1P>(F, Su, b), diag_of(F, gi, gj, gk), omega,
                             ((gi + gj + gk) & 1) == 0);
      out[c] = zv;
      if (FINEST) acc += (double)rc * (double)zv;
    }
  }
  if (FINEST) {
    acc = block_sum<FT>(acc, sh);
    const double vals[1] = {acc};
    if (publish_partials<1>(partials, &st->ticket[0], vals, &last)) {
      double tot[1];
      reduce_partials_sum<FT, 1>(partials, tot, sh);
      if (tid == 0) {
        finish_rz(st, tot[0], mode);
        st->ticket[0] = 0u;
      }
    }
  }
}

// ------------------------------------------------------------ tail -------
// Levels lt..nl-1 live in shared memory, each as three arrays (r, a, u)
// with a one-cell zero border ((nx+2)(ny+2)(nz+2) elements, x fastest), so
// the stencils need no bounds checks.  One block of TAIL_T threads runs the
// V-cycle below level lt: input r of level lt (global), output its
// corrected x into levels[lt].t (global).  `a` holds the pre-smoothed x,
// then the corrected t, then the final result.
constexpr int TAIL_T = 1024;
constexpr int MAX_LEVELS = 16;

template <typename T>
struct TailArgs {
  Level<T> lv[MAX_LEVELS];
  int lt, nl;
  int off[MAX_LEVELS];   // element offset of each tail level's three bordered arrays
  const double* ainv;
  int n_coarse;
};

template <typename T, int SM>
__global__ void __launch_bounds__(TAIL_T) k_mg_tail(TailArgs<T> A, T omega, const SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  if (st->converged) return;
  const int tid = threadIdx.x;
  // zero every array (borders stay zero)
  {
    const int m = A.nl - 1;
    const Level<T>& L = A.lv[m];
    const int tot = A.off[m] + 3 * (L.nx + 2) * (L.ny + 2) * (L.nz + 2);
    for (int e = tid; e < tot; e += TAIL_T) S[e] = T(0);
  }
  __syncthreads();
  auto geom = [&](int m, int& X, int& P, int& NB) {
    const Level<T>& L = A.lv[m];
    X = L.nx + 2;
    P = X * (L.ny + 2);
    NB = P * (L.nz + 2);
  };
  {
    const Level<T>& L = A.lv[A.lt];
    int X, P, NB;
    geom(A.lt, X, P, NB);
    T* r = S + A.off[A.lt];
    const int n = L.nx * L.ny * L.nz;
    for (int e = tid; e < n; e += TAIL_T) {
      const int i = e % L.nx, j = (e / L.nx) % L.ny, k = e / (L.nx * L.ny);
      r[(i + 1) + X * (j + 1) + P * (k + 1)] = L.r[lidx(L, i, j, k)];
    }
  }
  __syncthreads();
  for (int m = A.lt; m < A.nl - 1; ++m) {
    const Level<T>& L = A.lv[m];
    const Level<T>& Cc = A.lv[m + 1];
    int X, P, NB, CX, CP, CNB;
    geom(m, X, P, NB);
    geom(m + 1, CX, CP, CNB);
    T* r = S + A.off[m];
    T* a = r + NB;
    T* u = a + NB;   // u holds r/D during the down leg
    const int n = L.nx * L.ny * L.nz;
    for (int e = tid; e < n; e += TAIL_T) {
      const int i = e % L.nx, j = (e / L.nx) % L.ny, k = e / (L.nx * L.ny);
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      u[b] = r[b] / diag_of(L, i, j, k);
    }
    __syncthreads();
    for (int e = tid; e < n; e += TAIL_T) {
      const int i = e % L.nx, j = (e / L.nx) % L.ny, k = e / (L.nx * L.ny);
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      const T s = L.wx * (u[b - 1] + u[b + 1]) + L.wy * (u[b - X] + u[b + X]) + L.wz * (u[b - P] + u[b + P]);
      a[b] = presmooth<SM>(u[b], s, diag_of(L, i, j, k), omega, ((i + j + k) & 1) == 0);
    }
    __syncthreads();
    T* rc = S + A.off[m + 1];
    const int nc = Cc.nx * Cc.ny * Cc.nz;
    for (int e = tid; e < nc; e += TAIL_T) {
      const int ci = e % Cc.nx, cj = (e / Cc.nx) % Cc.ny, ck = e / (Cc.nx * Cc.ny);
      const int i0 = L.cx ? 2 * ci : ci, i1 = L.cx ? min(2 * ci + 1, L.nx - 1) : ci;
      const int j0 = L.cy ? 2 * cj : cj, j1 = L.cy ? min(2 * cj + 1, L.ny - 1) : cj;
      const int k0 = L.cz ? 2 * ck : ck, k1 = L.cz ? min(2 * ck + 1, L.nz - 1) : ck;
      T s = 0;
      for (int kk = k0; kk <= k1; ++kk)
        for (int jj = j0; jj <= j1; ++jj)
          for (int ii = i0; ii <= i1; ++ii) {
            const int b = (ii + 1) + X * (jj + 1) + P * (kk + 1);
            const T nb = L.wx * (a[b - 1] + a[b + 1]) + L.wy * (a[b - X] + a[b + X]) + L.wz * (a[b - P] + a[b + P]);
            s += r[b] - diag_of(L, ii, jj, kk) * a[b] + nb;
          }
      rc[(ci + 1) + CX * (cj + 1) + CP * (ck + 1)] = s;
    }
    __syncthreads();
  }
  // coarsest level: a = A^-1 r (FP64 dense inverse), one warp per row
  {
    const int m = A.nl - 1;
    const Level<T>& L = A.lv[m];
    int X, P, NB;
    geom(m, X, P, NB);
    const T* r = S + A.off[m];
    T* a = S + A.off[m] + NB;
    const int n = A.n_coarse, warp = tid >> 5, lane = tid & 31;
    for (int row = warp; row < n; row += TAIL_T / 32) {
      double s = 0.0;
      for (int c = lane; c < n; c += 32) {
        const int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
        s += A.ainv[(size_t)row * n + c] * (double)r[(i + 1) + X * (j + 1) + P * (k + 1)];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const int i = row % L.nx, j = (row / L.nx) % L.ny, k = row / (L.nx * L.ny);
        a[(i + 1) + X * (j + 1) + P * (k + 1)] = (T)s;
      }
    }
  }
  __syncthreads();
  for (int m = A.nl - 2; m >= A.lt; --m) {
    const Level<T>& L = A.lv[m];
    int X, P, NB, CX, CP, CNB;
    geom(m, X, P, NB);
    geom(m + 1, CX, CP, CNB);
    T* r = S + A.off[m];
    T* a = r + NB;
    T* u = a + NB;
    const T* ec = S + A.off[m + 1] + CNB;
    const int n = L.nx * L.ny * L.nz;
    for (int e = tid; e < n; e += TAIL_T) {   // t = x + P e (in place)
      const int i = e % L.nx, j = (e / L.nx) % L.ny, k = e / (L.nx * L.ny);
      const int pi = L.cx ? i >> 1 : i, pj = L.cy ? j >> 1 : j, pk = L.cz ? k >> 1 : k;
      a[(i + 1) + X * (j + 1) + P * (k + 1)] += ec[(pi + 1) + CX * (pj + 1) + CP * (pk + 1)];
    }
    __syncthreads();
    for (int e = tid; e < n; e += TAIL_T) {
      const int i = e % L.nx, j = (e / L.nx) % L.ny, k = e / (L.nx * L.ny);
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      const T s = L.wx * (a[b - 1] + a[b + 1]) + L.wy * (a[b - X] + a[b + X]) + L.wz * (a[b - P] + a[b + P]);
      u[b] = relax<SM>(a[b], r[b], s, diag_of(L, i, j, k), omega, ((i + j + k) & 1) == 1);
    }
    __syncthreads();
    for (int e = tid; e < n; e += TAIL_T) {
      const int i = e % L.nx, j = (e / L.nx) % L.ny, k = e / (L.nx * L.ny);
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      const T s = L.wx * (u[b - 1] + u[b + 1]) + L.wy * (u[b - X] + u[b + X]) + L.wz * (u[b - P] + u[b + P]);
      a[b] = relax<SM>(u[b], r[b], s, diag_of(L, i, j, k), omega, ((i + j + k) & 1) == 0);
    }
    __syncthreads();
  }
  {
    const Level<T>& L = A.lv[A.lt];
    int X, P, NB;
    geom(A.lt, X, P, NB);
    const T* a = S + A.off[A.lt] + NB;
    const int n = L.nx * L.ny * L.nz;
    for (int e = tid; e < n; e += TAIL_T) {
      const int i = e % L.nx, j = (e / L.nx) % L.ny, k = e / (L.nx * L.ny);
      L.t[lidx(L, i, j, k)] = a[(i + 1) + X * (j + 1) + P * (k + 1)];
    }
  }
}

// ------------------------------------------- CG direction + SpMV --------
// d = z (first iteration) or z + beta d_old over tile + halo 1 in shared
// memory; q = A d on the owned cells; d.q and alpha = rz / d.q.
template <typename T>
__global__ void __launch_bounds__(FT) k_cg_dir_q(Level<T> L, const T* __restrict__ z, T* d0, T* d1,
                                                T* __restrict__ q, double* partials, SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Sd = reinterpret_cast<T*>(smem_raw);   // H1N (0 outside)
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->converged) return;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * TZ;
  const int tid = threadIdx.x, tx = tid & (TX - 1), ty = tid / TX;
  const int it = st->iter;
  const T* dold = (it & 1) ? d1 : d0;
  T* dnew = (it & 1) ? d0 : d1;
  const T beta = it == 0 ? T(0) : (T)st->beta;
  {
    const PlaneMap m = plane_map<H1X, H1Y>();
#pragma unroll 2
    for (int ez = 0; ez < H1Z; ++ez) {
      const int gk = k0 - 1 + ez;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !m.has1) break;
        const int ex = h ? m.x1 : m.x0, ey = h ? m.y1 : m.y0;
        const int hi = i0 - 1 + ex, hj = j0 - 1 + ey;
        T v = 0;
        if (in_level(L, hi, hj, gk)) {
          const size_t c = lidx(L, hi, hj, gk);
          v = it == 0 ? z[c] : z[c] + beta * dold[c];
        }
        Sd[ex + H1X * ey + H1P * ez] = v;
      }
    }
  }
  __syncthreads();
  const int gi = i0 + tx, gj = j0 + ty;
  double acc = 0.0;
  if (gi < L.nx && gj < L.ny) {
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      const int gk = k0 + zz;
      if (gk >= L.nz) break;
      const int b = (tx + 1) + H1X * (ty + 1) + H1P * (zz + 1);
      const T dc = Sd[b];
      const T qv = diag_of(L, gi, gj, gk) * dc - nbs<T, H1X, H1P>(L, Sd, b);
      const size_t c = lidx(L, gi, gj, gk);
      dnew[c] = dc;
      q[c] = qv;
      acc += (double)dc * (double)qv;
    }
  }
  acc = block_sum<FT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[2], vals, &last)) {
    double tot[1];
    reduce_partials_sum<FT, 1>(partials, tot, sh);
    if (tid == 0) {
      st->dq = tot[0];
      st->alpha = st->rz / tot[0];
      st->ticket[2] = 0u;
    }
  }
}

}  // namespace uf
