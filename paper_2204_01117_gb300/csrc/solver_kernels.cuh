// Pressure Poisson solve (arXiv 2204.01117, Sec. 3: "the pressure Poisson
// equation is solved by the conjugate gradient algorithm"; App. A.3): matrix-
// free preconditioned CG on the 7-point operator A whose coefficients do not
// depend on the geometry (buildings enter through drag, Sec. 3), with FP64
// inner products and residual norms.
//
// Preconditioners:
//   * MG   - one geometric multigrid V-cycle (cell-centred 2x2x2 agglomeration,
//            summed restriction R, piecewise-constant prolongation P = R^T,
//            rediscretised coarse operators, red-black Gauss-Seidel or
//            damped-Jacobi smoothing, dense FP64 inverse on the coarsest
//            level); kernels in mg_fused.cuh.  Symmetric and positive
//            definite, so CG stays CG.  This replaces the paper's
//            approximate inverse as the default.
//   * AI1  - the paper's first-order approximate inverse M^-1 = K^T K,
//            K = sqrt(2-w) Dbar^-1/2 (I - L Dbar^-1), Dbar = D/w (Sec. 3,
//            "Approximate Inverse Preconditioner"), applied matrix-free
//            (see k_precond_simple for the sparsity reading).
//   * JACOBI, NONE.
//
// Operator on a level: for each of the six faces of a cell, an interior face
// adds w_a (x_c - x_nb), a face on an outlet side adds w_a x_c (p = 0 in the
// ghost cell), an inlet or wall face adds nothing (dp/dn = 0).  w_a = 1 on
// the finest level; on a coarse level w_a = (fine cells per coarse cell) /
// (coarsening factor along a)^2, the integer stencil of the coarse spacing
// scaled to the summed restriction.
#pragma once
#include "step_kernels.cuh"

namespace uf {

template <typename T>
struct Level {
  int nx, ny, nz, P;
  int cx, cy, cz;      // 1 if the next coarser level halves this axis
  T wx, wy, wz;
  int out_mask;        // bit s (0..5 = x-,x+,y-,y+,z-,z+) set: outlet side
  T* r;
  T* x;
  T* t;
  T* r_alt;            // finest level of the fused V-cycle: r ping-pongs with the CG iteration parity
  int lin;             // multigrid: 1 if the transfers to the next coarser level are cell-centred
                       // linear (restriction = transpose of the prolongation), 0 piecewise constant
  T* e;                // lin: the prolonged coarse correction P t_{l+1} on this level
};

// Residual buffer holding the current r after `iter` CG iterations.
template <typename T>
__device__ __forceinline__ T* level_r(const Level<T>& L, int iter) {
  return (L.r_alt && (iter & 1)) ? L.r_alt : L.r;
}

template <typename T>
__device__ __forceinline__ size_t lidx(const Level<T>& L, int i, int j, int k) {
  UF_BOUNDS(i >= 0 && i < L.P && j >= 0 && j < L.ny && k >= 0 && k < L.nz, BA_LEVEL, i, j, k);
  return (size_t)i + (size_t)L.P * ((size_t)j + (size_t)L.ny * k);
}

template <typename T>
__device__ __forceinline__ T level_diag(const Level<T>& L, int i, int j, int k) {
  T d = 0;
  d += (i > 0 || (L.out_mask & 1)) ? L.wx : T(0);
  d += (i < L.nx - 1 || (L.out_mask & 2)) ? L.wx : T(0);
  d += (j > 0 || (L.out_mask & 4)) ? L.wy : T(0);
  d += (j < L.ny - 1 || (L.out_mask & 8)) ? L.wy : T(0);
  d += (k > 0 || (L.out_mask & 16)) ? L.wz : T(0);
  d += (k < L.nz - 1 || (L.out_mask & 32)) ? L.wz : T(0);
  return d;
}

// (A x)(i,j,k) for a value functor val(i,j,k).
template <typename T, typename F>
__device__ __forceinline__ T level_apply(const Level<T>& L, int i, int j, int k, const F& val) {
  const T xc = val(i, j, k);
  T acc = 0;
  if (i > 0) acc += L.wx * (xc - val(i - 1, j, k)); else if (L.out_mask & 1) acc += L.wx * xc;
  if (i < L.nx - 1) acc += L.wx * (xc - val(i + 1, j, k)); else if (L.out_mask & 2) acc += L.wx * xc;
  if (j > 0) acc += L.wy * (xc - val(i, j - 1, k)); else if (L.out_mask & 4) acc += L.wy * xc;
  if (j < L.ny - 1) acc += L.wy * (xc - val(i, j + 1, k)); else if (L.out_mask & 8) acc += L.wy * xc;
  if (k > 0) acc += L.wz * (xc - val(i, j, k - 1)); else if (L.out_mask & 16) acc += L.wz * xc;
  if (k < L.nz - 1) acc += L.wz * (xc - val(i, j, k + 1)); else if (L.out_mask & 32) acc += L.wz * xc;
  return acc;
}

// level_apply on the pressure store: the same stencil, with each
// neighbour difference taken on the stored pairs (ps_diff).
template <typename T>
__device__ __forceinline__ T level_apply_store(const Level<T>& L, int i, int j, int k, const PStore<T>* __restrict__ g) {
  const PStore<T> gc = g[lidx(L, i, j, k)];
  const T xc = (T)ps_value(gc);
  auto d = [&](int a, int b2, int c2) { return (T)ps_diff(gc, g[lidx(L, a, b2, c2)]); };
  T acc = 0;
  if (i > 0) acc += L.wx * d(i - 1, j, k); else if (L.out_mask & 1) acc += L.wx * xc;
  if (i < L.nx - 1) acc += L.wx * d(i + 1, j, k); else if (L.out_mask & 2) acc += L.wx * xc;
  if (j > 0) acc += L.wy * d(i, j - 1, k); else if (L.out_mask & 4) acc += L.wy * xc;
  if (j < L.ny - 1) acc += L.wy * d(i, j + 1, k); else if (L.out_mask & 8) acc += L.wy * xc;
  if (k > 0) acc += L.wz * d(i, j, k - 1); else if (L.out_mask & 16) acc += L.wz * xc;
  if (k < L.nz - 1) acc += L.wz * d(i, j, k + 1); else if (L.out_mask & 32) acc += L.wz * xc;
  return acc;
}

// Cell loop of a 32x8 thread tile over the z planes [z0, z1) of a block.
#define UF_CELL_LOOP_VB(L, vb)                                              \
  const int i = (vb).x * BX + threadIdx.x, j = (vb).y * BY + threadIdx.y;   \
  const bool inside = i < (L).nx && j < (L).ny;                             \
  const int z0 = (vb).z * zc, z1 = min((L).nz, z0 + zc);
#define UF_CELL_LOOP(L) UF_CELL_LOOP_VB(L, vblock())

// Clears the WHILE condition of the graph that drives the CG loop once the
// solve is done: at once for a single grid; for a batch, when the last of
// its instances finishes (`left` counts the unfinished ones and each
// instance decrements it exactly once).
__device__ __forceinline__ void signal_converged(cudaGraphConditionalHandle cond, int use_cond, int* left) {
  if (left) {
    if (atomicSub(left, 1) == 1 && use_cond) cudaGraphSetConditional(cond, 0);
  } else if (use_cond) {
    cudaGraphSetConditional(cond, 0);
  }
}

// ------------------------------------------------------------ CG kernels --

// r = b - A x from the warm start in x.  With g != nullptr the solve is for
// the correction to the guess g held in the pressure store (the pressure
// extrapolated in time, see pressure_commit_body) instead: r = b - A g and
// x = 0.  A zero right-hand side gives x = 0.
template <typename T>
__device__ __forceinline__ void cg_init_body(const Level<T>& L, const T* __restrict__ b, T* __restrict__ x,
                                             const PStore<T>* __restrict__ g, int zc,
                                             double* partials, SolveState* st, cudaGraphConditionalHandle cond,
                                             int use_cond, int* left, const VBlock& vb) {
  __shared__ double sh[32];
  __shared__ bool last;
  UF_CELL_LOOP_VB(L, vb);
  const bool zero_rhs = st->bb == 0.0;
  double acc = 0.0;
  DotAcc<T> dacc;
  if (inside) {
    for (int k = z0; k < z1; ++k) {
      const size_t c = lidx(L, i, j, k);
      if (zero_rhs) {
        x[c] = T(0);
        L.r[c] = T(0);
      } else if (g) {
        const T rv = b[c] - level_apply_store(L, i, j, k, g);
        x[c] = T(0);
        L.r[c] = rv;
        dacc.add(rv, rv);
      } else {
        const T ax = level_apply(L, i, j, k, [&](int a, int b2, int c2) { return x[lidx(L, a, b2, c2)]; });
        const T rv = b[c] - ax;
        L.r[c] = rv;
        dacc.add(rv, rv);
      }
    }
  }
  acc += dacc.value();
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[1], vals, &last, vb)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh, vb.n);
    if (thread_linear_id() == 0) {
      st->rr = tot[0];
      st->rr0 = tot[0];
      if (zero_rhs || (st->rule == 0 && tot[0] <= st->tol2 * st->bb)) {
        st->converged = 1;
        signal_converged(cond, use_cond, left);
      }
      st->ticket[1] = 0u;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_cg_init(Level<T> L, const T* __restrict__ b, T* __restrict__ x,
                                                const PStore<T>* __restrict__ g, int zc, double* partials,
                                                SolveState* st, cudaGraphConditionalHandle cond, int use_cond) {
  cg_init_body<T>(L, b, x, g, zc, partials, st, cond, use_cond, nullptr, vblock());
}


// d = z (first iteration) or z + beta d_old;  q = A d;  dq = d.q; alpha = rz/dq.
// d ping-pongs between two buffers by iteration parity.
template <typename T>
__global__ void __launch_bounds__(NT) k_cg_direction_spmv(Level<T> L, const T* __restrict__ z, T* d0, T* d1,
                                                          T* __restrict__ q, int zc, double* partials,
                                                          SolveState* st) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->converged) return;
  UF_CELL_LOOP(L);
  const int it = st->iter;
  const T* dold = (it & 1) ? d1 : d0;
  T* dnew = (it & 1) ? d0 : d1;
  const T beta = it == 0 ? T(0) : (T)st->beta;
  const bool first = it == 0;
  auto dn = [&](int a, int b2, int c2) {
    const size_t c = lidx(L, a, b2, c2);
    return first ? z[c] : z[c] + beta * dold[c];
  };
  double acc = 0.0;
  DotAcc<T> dacc;
  if (inside) {
    for (int k = z0; k < z1; ++k) {
      const size_t c = lidx(L, i, j, k);
      const T dc = dn(i, j, k);
      const T qv = level_apply(L, i, j, k, dn);
      dnew[c] = dc;
      q[c] = qv;
      dacc.add(dc, qv);
    }
  }
  acc += dacc.value();
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[2], vals, &last)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh);
    if (thread_linear_id() == 0) {
      st->dq = tot[0];
      st->alpha = st->rz / tot[0];
      st->ticket[2] = 0u;
    }
  }
}

// x += alpha d;  r -= alpha q;  rr = r.r;  convergence test ||r|| <= tol ||b||.
template <typename T>
__global__ void __launch_bounds__(NT) k_cg_update(Level<T> L, T* __restrict__ x, const T* d0, const T* d1,
                                                  const T* __restrict__ q, int zc, double* partials, SolveState* st,
                                                  cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->converged) return;
  UF_CELL_LOOP(L);
  const int it = st->iter;
  const T* d = (it & 1) ? d0 : d1;
  const T alpha = (T)st->alpha;
  double acc = 0.0;
  DotAcc<T> dacc;
  if (inside) {
    for (int k = z0; k < z1; ++k) {
      const size_t c = lidx(L, i, j, k);
      x[c] += alpha * d[c];
      const T rv = L.r[c] - alpha * q[c];
      L.r[c] = rv;
      dacc.add(rv, rv);
    }
  }
  acc += dacc.value();
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[3], vals, &last)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh);
    if (thread_linear_id() == 0) {
      const double rr = tot[0];
      st->rr = rr;
      st->iter = it + 1;
      st->total_iters += 1;
      if (!(rr == rr) || isinf(rr)) {
        st->status = DEV_NAN;
        if (st->sticky == 0) st->sticky = DEV_NAN;
        st->converged = 1;
      } else if (st->rule == 0 && rr <= st->tol2 * st->bb) {
        st->converged = 1;
      } else if (it + 1 >= st->max_iter) {
        st->status = DEV_NOT_CONVERGED;
        if (st->sticky == 0) st->sticky = DEV_NOT_CONVERGED;
        st->converged = 1;
      }
      if (st->converged && use_cond) cudaGraphSetConditional(cond, 0);
      st->ticket[3] = 0u;
    }
  }
}

// Finishes a preconditioner application: rz_new = r.z; mode 0 (set-up) stores
// it, mode 1 (iteration) also forms beta = rz_new / rz_old.
__device__ __forceinline__ void finish_rz(SolveState* st, double rz_new, int mode) {
  if (mode == 1) st->beta = rz_new / st->rz;
  st->rz = rz_new;
}

// ----------------------------------------------- simple preconditioners --
// kind 0: z = r (plain CG);  kind 1: z = r / D (Jacobi);
// kind 2: the first-order approximate inverse of Sec. 3, M^-1 = K^T K with
// K = sqrt(2-w) Dbar^-1/2 (I - L Dbar^-1), Dbar = D/w, L the strictly lower
// triangle of A (lexicographic order, x fastest).  The product is applied
// as written, without dropping the entries of K^T K that fall outside the
// 7-point pattern: dropping them leaves an indefinite M^-1 for w above
// about 1.2 on this operator, while the untruncated product is SPD for
// 0 < w < 2 and has its best condition number near w = 1.65, where App. A.3
// places the optimum.  Matrix-free: y = K r needs r at the cell and its three
// lower neighbours, z = K^T y needs y at the cell and its three upper
// neighbours; y is recomputed there.
template <typename T>
__device__ __forceinline__ T ai1_K(const Level<T>& L, const T* __restrict__ r, T w, int i, int j, int k) {
  // (K r)_c = sqrt(2-w) / sqrt(Dbar_c) * (r_c + sum_{lower m} w_m r_m / Dbar_m)
  T acc = r[lidx(L, i, j, k)];
  if (i > 0) acc += L.wx * r[lidx(L, i - 1, j, k)] * w / level_diag(L, i - 1, j, k);
  if (j > 0) acc += L.wy * r[lidx(L, i, j - 1, k)] * w / level_diag(L, i, j - 1, k);
  if (k > 0) acc += L.wz * r[lidx(L, i, j, k - 1)] * w / level_diag(L, i, j, k - 1);
  return sqrt((T(2) - w) * w / level_diag(L, i, j, k)) * acc;
}

template <typename T>
__device__ __forceinline__ T ai1_apply(const Level<T>& L, const T* __restrict__ r, T w, int i, int j, int k) {
  // (K^T y)_c = sqrt(2-w)/sqrt(Dbar_c) y_c + sqrt(2-w)/Dbar_c * sum_{upper m} w_m y_m / sqrt(Dbar_m)
  const T s = sqrt(T(2) - w);
  const T Dc = level_diag(L, i, j, k) / w;
  T up = 0;
  if (i < L.nx - 1) up += L.wx * ai1_K(L, r, w, i + 1, j, k) * rsqrt(level_diag(L, i + 1, j, k) / w);
  if (j < L.ny - 1) up += L.wy * ai1_K(L, r, w, i, j + 1, k) * rsqrt(level_diag(L, i, j + 1, k) / w);
  if (k < L.nz - 1) up += L.wz * ai1_K(L, r, w, i, j, k + 1) * rsqrt(level_diag(L, i, j, k + 1) / w);
  return s * rsqrt(Dc) * ai1_K(L, r, w, i, j, k) + s / Dc * up;
}

// Second-order approximate inverse (Sec. 3): K = sqrt(2-w) Dbar^-1/2
// (I + N + N^2) with N = -L Dbar^-1 (strictly lower, entries w_a / Dbar of
// the lower neighbour), M^-1 = K^T K applied without truncation, as for the
// first order.  Two passes: y = K r into a scratch vector (k_ai2_K), then
// z = K^T y (k_precond_simple, kind 3).
//   (K r)_c   = s Dbar_c^-1/2 (r_c + g_c + sum_{lower m} w g_m / Dbar_m),
//               g = N r: g_c = sum_{lower n} w r_n / Dbar_n;
//   (K^T y)_c = s (v_c + h_c + sum_{upper m} w h_m / Dbar_c),
//               v = Dbar^-1/2 y, h = N^T v: h_c = sum_{upper m} w v_m / Dbar_c.
template <typename T>
__device__ __forceinline__ T ai_lower_sum(const Level<T>& L, const T* __restrict__ r, T w, int i, int j, int k) {
  T g = 0;
  if (i > 0) g += L.wx * r[lidx(L, i - 1, j, k)] * w / level_diag(L, i - 1, j, k);
  if (j > 0) g += L.wy * r[lidx(L, i, j - 1, k)] * w / level_diag(L, i, j - 1, k);
  if (k > 0) g += L.wz * r[lidx(L, i, j, k - 1)] * w / level_diag(L, i, j, k - 1);
  return g;
}
template <typename T>
__device__ __forceinline__ T ai_upper_v(const Level<T>& L, const T* __restrict__ y, T w, int i, int j, int k) {
  // sum_{upper m} w_a v_m, v_m = y_m sqrt(w / D_m)
  T h = 0;
  if (i < L.nx - 1) h += L.wx * y[lidx(L, i + 1, j, k)] * sqrt(w / level_diag(L, i + 1, j, k));
  if (j < L.ny - 1) h += L.wy * y[lidx(L, i, j + 1, k)] * sqrt(w / level_diag(L, i, j + 1, k));
  if (k < L.nz - 1) h += L.wz * y[lidx(L, i, j, k + 1)] * sqrt(w / level_diag(L, i, j, k + 1));
  return h;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_ai2_K(Level<T> L, T w, T* __restrict__ y, int zc, const SolveState* st) {
  if (st->converged) return;
  UF_CELL_LOOP(L);
  if (!inside) return;
  for (int k = z0; k < z1; ++k) {
    T acc = L.r[lidx(L, i, j, k)] + ai_lower_sum(L, L.r, w, i, j, k);
    if (i > 0) acc += L.wx * ai_lower_sum(L, L.r, w, i - 1, j, k) * w / level_diag(L, i - 1, j, k);
    if (j > 0) acc += L.wy * ai_lower_sum(L, L.r, w, i, j - 1, k) * w / level_diag(L, i, j - 1, k);
    if (k > 0) acc += L.wz * ai_lower_sum(L, L.r, w, i, j, k - 1) * w / level_diag(L, i, j, k - 1);
    y[lidx(L, i, j, k)] = sqrt((T(2) - w) * w / level_diag(L, i, j, k)) * acc;
  }
}

template <typename T>
__device__ __forceinline__ T ai2_KT(const Level<T>& L, const T* __restrict__ y, T w, int i, int j, int k) {
  const T s = sqrt(T(2) - w);
  const T wD = w / level_diag(L, i, j, k);   // 1 / Dbar_c
  T hh = 0;                                  // sum_{upper m} w_a h_m
  if (i < L.nx - 1) hh += L.wx * (w / level_diag(L, i + 1, j, k)) * ai_upper_v(L, y, w, i + 1, j, k);
  if (j < L.ny - 1) hh += L.wy * (w / level_diag(L, i, j + 1, k)) * ai_upper_v(L, y, w, i, j + 1, k);
  if (k < L.nz - 1) hh += L.wz * (w / level_diag(L, i, j, k + 1)) * ai_upper_v(L, y, w, i, j, k + 1);
  const T v = y[lidx(L, i, j, k)] * sqrt(wD);
  const T h = wD * ai_upper_v(L, y, w, i, j, k);
  return s * (v + h + wD * hh);
}

// z = M^-1 r for the simple preconditioners and rz = r.z (kind 0: copy,
// 1: Jacobi, 2: AI1, 3: AI2 from y = K r in L.t).  Under the stop rule of
// App. A.3 (st->rule 1) the convergence test r.z <= tol ||b||^2 happens
// here, where r.z is formed.
template <typename T>
__global__ void __launch_bounds__(NT) k_precond_simple(Level<T> L, int kind, T w, T* __restrict__ z, int zc, int mode,
                                                       double* partials, SolveState* st,
                                                       cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->converged) return;
  UF_CELL_LOOP(L);
  double acc = 0.0;
  DotAcc<T> dacc;
  if (inside) {
    for (int k = z0; k < z1; ++k) {
      const size_t c = lidx(L, i, j, k);
      const T rv = L.r[c];
      T zv;
      if (kind == 0) {
        zv = rv;
      } else if (kind == 1) {
        zv = rv / level_diag(L, i, j, k);
      } else if (kind == 2) {
        zv = ai1_apply(L, L.r, w, i, j, k);
      } else {
        zv = ai2_KT(L, L.t, w, i, j, k);
      }
      z[c] = zv;
      dacc.add(L.r[c], zv);
    }
  }
  acc += dacc.value();
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[0], vals, &last)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh);
    if (thread_linear_id() == 0) {
      finish_rz(st, tot[0], mode);
      if (st->rule == 1 && tot[0] <= st->tol2 * st->bb) {
        st->converged = 1;
        if (use_cond) cudaGraphSetConditional(cond, 0);
      }
      st->ticket[0] = 0u;
    }
  }
}

// y = A x on a level (diagnostic / test entry point).
template <typename T>
__global__ void __launch_bounds__(NT) k_apply_level(Level<T> L, const T* __restrict__ x, T* __restrict__ y, int zc) {
  UF_CELL_LOOP(L);
  if (!inside) return;
  for (int k = z0; k < z1; ++k)
    y[lidx(L, i, j, k)] = level_apply(L, i, j, k, [&](int a, int b2, int c2) { return x[lidx(L, a, b2, c2)]; });
}

// ||b||^2 and a fresh solver state for a stand-alone solve of A p = b.
template <typename T>
__global__ void __launch_bounds__(NT) k_solve_reset(Level<T> L, const T* __restrict__ b, int zc, double* partials,
                                                    SolveState* st) {
  __shared__ double sh[32];
  __shared__ bool last;
  UF_CELL_LOOP(L);
  DotAcc<T> dacc;
  if (inside)
    for (int k = z0; k < z1; ++k) {
      const T bv = b[lidx(L, i, j, k)];
      dacc.add(bv, bv);
    }
  double acc = block_sum<NT>(dacc.value(), sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[0], vals, &last)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh);
    if (thread_linear_id() == 0) {
      st->bb = tot[0];
      st->iter = 0;
      st->converged = 0;
      st->status = DEV_OK;
      st->ticket[0] = 0u;
    }
  }
}

// Fixed right-hand side for timing solves: values in [-1, 1) from the
// 32-bit finaliser of MurmurHash3 (A. Appleby) applied to the cell index.
__device__ __forceinline__ unsigned int fmix32(unsigned int h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
template <typename T>
__global__ void __launch_bounds__(NT) k_tune_rhs(Level<T> L, T* __restrict__ b, int zc) {
  UF_CELL_LOOP(L);
  if (!inside) return;
  for (int k = z0; k < z1; ++k) {
    const unsigned int id = (unsigned int)(i + L.nx * (j + L.ny * k));
    b[lidx(L, i, j, k)] = T((double)fmix32(id * 2654435761u + 12345u) * (2.0 / 4294967296.0) - 1.0);
  }
}

}  // namespace uf
