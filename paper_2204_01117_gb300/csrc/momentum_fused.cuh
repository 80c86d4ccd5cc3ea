// Fused diffusion, porosity drag, velocity BCs and pressure right-hand side
// (a3-a6: Eq. momen_drag's (nu + nu_t) lap u; the forward-Euler drag step
// and the BC rules of Sec. 3; b = -(rho h / dt) h div u).
//
// One z-marching kernel per 32 x 8 column of cells replaces k_diffuse,
// k_drag_bc and k_pressure_rhs.  Per block, in shared memory:
//   * the advected velocity (u~, v~, w~), nu_t and the drag coefficient c on
//     the column plus a halo of 2 (36 x 12, a ring of 5 planes), copied one
//     plane ahead with cp.async;
//   * the diffused velocity u2 of the three components on the column plus a
//     halo of 1 (34 x 10, a ring of 2 planes);
//   * the dragged velocity u3 of the plane's x and y faces, for the fluxes.
// Per plane k: u2 on plane k+1, sync, u3 on the faces of plane k (u, v) and
// on the w faces of plane k+1, sync, b of plane k and ||b||^2.
//
// Boundary faces of u~ and u2 (never stored between sub-steps) come from
// the BC rules at the moment they are read, as in the unfused kernels.
// Every value is formed by the expressions of k_diffuse, k_drag_bc and
// k_pressure_rhs; the block and z-chunk decomposition is that of
// k_pressure_rhs (chunk_grid), so ||b||^2 is summed in the same order.  The
// results, ||b||^2 included, are bit for bit those of the three kernels.
//
// Tape (the adjoint): when u2t is not null, u2 of every interior face the
// block owns is also written to (u2t, v2t, w2t).
#pragma once
#include "advect_fused.cuh"

namespace uf {

constexpr int DR = 5;   // ring of staged planes
constexpr int UR = 2;   // ring of u2 planes
// staged fields, in this order, each [DR][MWP]
constexpr int DF_U = 0, DF_V = 1, DF_W = 2, DF_NUT = 3, DF_C = 4, DF_N = 5;

template <typename T>
struct MomentumArgs {
  StepParams<T> p;
  const T* ut;
  const T* vt;
  const T* wt;       // advected velocity (interior faces)
  const T* nut;      // eddy viscosity (cells)
  const T* cc;       // drag coefficient (cells)
  T* u;
  T* v;
  T* w;              // out: u3 on every face
  T* b;              // out: right-hand side
  T* u2t;
  T* v2t;
  T* w2t;            // optional tape of u2 (interior faces)
  int zc;
  double* partials;
  SolveState* st;
};

template <typename T>
constexpr size_t momentum_fused_smem() {
  return sizeof(T) * ((size_t)DF_N * DR * MWP + (size_t)3 * UR * MHP + (size_t)(MX + 1) * MY + (size_t)MX * (MY + 1));
}

// Shared-memory view of one block's planes.
template <typename T>
struct MView {
  T* sD;    // [DF_N][DR][MWP]
  T* sU2;   // [3][UR][MHP]
  T* sU3;   // (MX+1) x MY  u3 of the plane's x faces
  T* sV3;   // MX x (MY+1)  u3 of the plane's y faces
  int i0, j0;
  __device__ __forceinline__ const T* D(int f, int k) const {   // plane k of staged field f
    return sD + (f * DR + (k + 4 * DR) % DR) * MWP;
  }
  __device__ __forceinline__ T* U2(int q, int k) const { return sU2 + (q * UR + (k & 1)) * MHP; }
  // window indices of lattice point (i, j)
  __device__ __forceinline__ int sidx(int i, int j) const { return (i - i0 + 2) + MWX * (j - j0 + 2); }
  __device__ __forceinline__ int hidx(int i, int j) const { return (i - i0 + 1) + MHX * (j - j0 + 1); }
};

// Diffusion of one interior face (the expressions of diffuse_body).  Fm,
// Fc, Fp: planes k-1, k, k+1 of the component's staged u~; Nm, Nc: planes
// k-1, k of nu_t; s: the face's index in the staged window.  Boundary
// faces of u~ come from the BC rules (inflow value, the adjacent interior
// face at an outlet, 0 at a wall).
template <int Q, typename T>
__device__ __forceinline__ T diffuse_at(const StepParams<T>& p, T c, const T* Fm, const T* Fc, const T* Fp,
                                        const T* Nm, const T* Nc, int s, int i, int j, int k) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const T x0 = Fc[s];
  if (Q == 0) {
    const T inflow = p.prof[k] * p.dirx;
    const T xm = i - 1 == 0 ? normal_face(p.side[0], Fc[s], inflow) : Fc[s - 1];
    const T xp = i + 1 == nx ? normal_face(p.side[1], Fc[s], inflow) : Fc[s + 1];
    const T ym = j > 0 ? Fc[s - MWX] : tangential_ghost(p.side[2], x0, inflow);
    const T yp = j < ny - 1 ? Fc[s + MWX] : tangential_ghost(p.side[3], x0, inflow);
    const T zm = k > 0 ? Fm[s] : tangential_ghost(p.side[4], x0, T(0));
    const T zp = k < nz - 1 ? Fp[s] : tangential_ghost(p.side[5], x0, T(0));
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (Nc[s - 1] + Nc[s]);
    return x0 + c * (p.nu + nf) * lap;
  } else if (Q == 1) {
    const T inflow = p.prof[k] * p.diry;
    const T xm = i > 0 ? Fc[s - 1] : tangential_ghost(p.side[0], x0, inflow);
    const T xp = i < nx - 1 ? Fc[s + 1] : tangential_ghost(p.side[1], x0, inflow);
    const T ym = j - 1 == 0 ? normal_face(p.side[2], Fc[s], inflow) : Fc[s - MWX];
    const T yp = j + 1 == ny ? normal_face(p.side[3], Fc[s], inflow) : Fc[s + MWX];
    const T zm = k > 0 ? Fm[s] : tangential_ghost(p.side[4], x0, T(0));
    const T zp = k < nz - 1 ? Fp[s] : tangential_ghost(p.side[5], x0, T(0));
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (Nc[s - MWX] + Nc[s]);
    return x0 + c * (p.nu + nf) * lap;
  } else {
    const T xm = i > 0 ? Fc[s - 1] : tangential_ghost(p.side[0], x0, T(0));
    const T xp = i < nx - 1 ? Fc[s + 1] : tangential_ghost(p.side[1], x0, T(0));
    const T ym = j > 0 ? Fc[s - MWX] : tangential_ghost(p.side[2], x0, T(0));
    const T yp = j < ny - 1 ? Fc[s + MWX] : tangential_ghost(p.side[3], x0, T(0));
    const T zm = k - 1 == 0 ? T(0) : Fm[s];
    const T zp = k + 1 == nz ? T(0) : Fp[s];
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (Nm[s] + Nc[s]);
    return x0 + c * (p.nu + nf) * lap;
  }
}

// u2 read at a face with the BC rules on boundary faces; U, Vp, W: the u2
// plane of the u, v or w lattice, h: the face's index in the halo-1 window.
template <typename T>
__device__ __forceinline__ T u2f(const StepParams<T>& p, const T* U, int h, int i, int k) {
  if (i == 0) return normal_face(p.side[0], U[h + 1], p.prof[k] * p.dirx);
  if (i == p.nx) return normal_face(p.side[1], U[h - 1], p.prof[k] * p.dirx);
  return U[h];
}
template <typename T>
__device__ __forceinline__ T v2f(const StepParams<T>& p, const T* Vp, int h, int j, int k) {
  if (j == 0) return normal_face(p.side[2], Vp[h + MHX], p.prof[k] * p.diry);
  if (j == p.ny) return normal_face(p.side[3], Vp[h - MHX], p.prof[k] * p.diry);
  return Vp[h];
}
template <typename T>
__device__ __forceinline__ T w2f(const StepParams<T>& p, const T* W, int h, int k) {
  return (k == 0 || k == p.nz) ? T(0) : W[h];
}

// Drag of one interior face of u2 (the expressions of drag_u/v/w).  u and v
// faces of plane k: A = u2 planes at k, B = at k + 1, C0 = c at plane k.
// w faces of plane k: A = u2 planes at k, B = at k - 1, C0 = c at k - 1,
// C1 = c at k.  h, s: the face's index in the halo-1 and staged windows.
template <int Q, typename T>
__device__ __forceinline__ T drag_at(const StepParams<T>& p, T dt, const T* const* A, const T* const* B, const T* C0,
                                     const T* C1, int h, int s, int i, int j, int k) {
  if (Q == 0) {
    const T q = A[0][h];
    const T vb = T(0.25) * (v2f(p, A[1], h - 1, j, k) + v2f(p, A[1], h, j, k) + v2f(p, A[1], h - 1 + MHX, j + 1, k) +
                            v2f(p, A[1], h + MHX, j + 1, k));
    const T wb = T(0.25) * (w2f(p, A[2], h - 1, k) + w2f(p, A[2], h, k) + w2f(p, B[2], h - 1, k + 1) +
                            w2f(p, B[2], h, k + 1));
    const T sp = sqrt(q * q + vb * vb + wb * wb);
    const T cf = T(0.5) * (C0[s - 1] + C0[s]);
    return fmax(T(0), T(1) - dt * cf * sp) * q;
  } else if (Q == 1) {
    const T q = A[1][h];
    const T ub = T(0.25) * (u2f(p, A[0], h - MHX, i, k) + u2f(p, A[0], h + 1 - MHX, i + 1, k) + u2f(p, A[0], h, i, k) +
                            u2f(p, A[0], h + 1, i + 1, k));
    const T wb = T(0.25) * (w2f(p, A[2], h - MHX, k) + w2f(p, A[2], h, k) + w2f(p, B[2], h - MHX, k + 1) +
                            w2f(p, B[2], h, k + 1));
    const T sp = sqrt(ub * ub + q * q + wb * wb);
    const T cf = T(0.5) * (C0[s - MWX] + C0[s]);
    return fmax(T(0), T(1) - dt * cf * sp) * q;
  } else {
    const T q = A[2][h];
    const T ub = T(0.25) * (u2f(p, B[0], h, i, k - 1) + u2f(p, B[0], h + 1, i + 1, k - 1) + u2f(p, A[0], h, i, k) +
                            u2f(p, A[0], h + 1, i + 1, k));
    const T vb = T(0.25) * (v2f(p, B[1], h, j, k - 1) + v2f(p, B[1], h + MHX, j + 1, k - 1) + v2f(p, A[1], h, j, k) +
                            v2f(p, A[1], h + MHX, j + 1, k));
    const T sp = sqrt(ub * ub + vb * vb + q * q);
    const T cf = T(0.5) * (C0[s] + C1[s]);
    return fmax(T(0), T(1) - dt * cf * sp) * q;
  }
}

// u3 of a u / v face (boundary faces from the BC rule on the dragged
// interior neighbour, as drag_bc_body) and of a w face.  The face whose drag
// is formed is chosen first, so the drag expression is inlined once.
template <typename T>
__device__ __forceinline__ T u3_at(const StepParams<T>& p, T dt, const T* const* A, const T* const* B, const T* C0,
                                   int h, int s, int i, int j, int k) {
  const int sh = i == 0 ? 1 : (i == p.nx ? -1 : 0);
  const T dr = drag_at<0>(p, dt, A, B, C0, C0, h + sh, s + sh, i + sh, j, k);
  if (sh == 0) return dr;
  return normal_face(p.side[i == 0 ? 0 : 1], dr, p.prof[k] * p.dirx);
}
template <typename T>
__device__ __forceinline__ T v3_at(const StepParams<T>& p, T dt, const T* const* A, const T* const* B, const T* C0,
                                   int h, int s, int i, int j, int k) {
  const int sh = j == 0 ? 1 : (j == p.ny ? -1 : 0);
  const T dr = drag_at<1>(p, dt, A, B, C0, C0, h + sh * MHX, s + sh * MWX, i, j + sh, k);
  if (sh == 0) return dr;
  return normal_face(p.side[j == 0 ? 2 : 3], dr, p.prof[k] * p.diry);
}
template <typename T>
__device__ __forceinline__ T w3_at(const StepParams<T>& p, T dt, const T* const* A, const T* const* B, const T* C0,
                                   const T* C1, int h, int s, int i, int j, int k) {
  return (k == 0 || k == p.nz) ? T(0) : drag_at<2>(p, dt, A, B, C0, C1, h, s, i, j, k);
}

// Starts the copy of plane kk of the five staged fields into its ring slot.
template <typename T>
__device__ __forceinline__ void stage_momentum(const MomentumArgs<T>& M, T* sD, int i0, int j0, int kk) {
  const StepParams<T>& p = M.p;
  if (kk < 0 || kk > p.nz) return;
  const int slot = (kk + 4 * DR) % DR;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = threadIdx.x + h * MT;
    if (t >= MWP) break;
    const int gx = i0 - 2 + t % MWX, gy = j0 - 2 + t / MWX;
    if (gx < 0 || gy < 0) continue;
    if (kk < p.nz) {
      if (gx <= p.nx && gy < p.ny) cp_async_elem(sD + (DF_U * DR + slot) * MWP + t, M.ut + idx_u(p, gx, gy, kk));
      if (gx < p.nx && gy <= p.ny) cp_async_elem(sD + (DF_V * DR + slot) * MWP + t, M.vt + idx_v(p, gx, gy, kk));
      if (gx < p.nx && gy < p.ny) {
        cp_async_elem(sD + (DF_NUT * DR + slot) * MWP + t, M.nut + idx_c(p, gx, gy, kk));
        cp_async_elem(sD + (DF_C * DR + slot) * MWP + t, M.cc + idx_c(p, gx, gy, kk));
      }
    }
    if (gx < p.nx && gy < p.ny) cp_async_elem(sD + (DF_W * DR + slot) * MWP + t, M.wt + idx_c(p, gx, gy, kk));
  }
}

// u2 of the three components on plane m over the halo-1 window; only
// interior faces are formed (boundary faces come from the BC rules).
template <typename T>
__device__ __forceinline__ void u2_plane(const MomentumArgs<T>& M, const MView<T>& V, T c, int m, int k0, int kend) {
  const StepParams<T>& p = M.p;
  if (m < 0 || m > p.nz) return;
  const T* Nm = V.D(DF_NUT, m - 1);
  const T* Nc = V.D(DF_NUT, m);
#pragma unroll 1
  for (int it = threadIdx.x; it < 3 * MHP; it += MT) {
    const int q = it >= 2 * MHP ? 2 : (it >= MHP ? 1 : 0), t = it - q * MHP;
    const int wx = t % MHX, wy = t / MHX;
    const int gi = V.i0 - 1 + wx, gj = V.j0 - 1 + wy;
    if (gi < 0 || gj < 0) continue;
    const int s = (wx + 1) + MWX * (wy + 1);
    const int f = DF_U + q;
    const T* Fm = V.D(f, m - 1);
    const T* Fc = V.D(f, m);
    const T* Fp = V.D(f, m + 1);
    T val;
    if (q == 0) {
      if (!(gi > 0 && gi < p.nx && gj < p.ny && m < p.nz)) continue;
      val = diffuse_at<0>(p, c, Fm, Fc, Fp, Nm, Nc, s, gi, gj, m);
    } else if (q == 1) {
      if (!(gi < p.nx && gj > 0 && gj < p.ny && m < p.nz)) continue;
      val = diffuse_at<1>(p, c, Fm, Fc, Fp, Nm, Nc, s, gi, gj, m);
    } else {
      if (!(gi < p.nx && gj < p.ny && m > 0 && m < p.nz)) continue;
      val = diffuse_at<2>(p, c, Fm, Fc, Fp, Nm, Nc, s, gi, gj, m);
    }
    V.U2(q, m)[t] = val;
    if (M.u2t) {   // tape of the owned interior faces
      const bool ox = gi >= V.i0 && gi < V.i0 + MX, oy = gj >= V.j0 && gj < V.j0 + MY, oz = m >= k0 && m < kend;
      if (ox && oy && oz) {
        if (q == 0) M.u2t[idx_u(p, gi, gj, m)] = val;
        else if (q == 1) M.v2t[idx_v(p, gi, gj, m)] = val;
        else M.w2t[idx_c(p, gi, gj, m)] = val;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void momentum_fused_body(const MomentumArgs<T>& M, const VBlock& vb) {
  extern __shared__ __align__(16) unsigned char mom_smem[];
  __shared__ double sh[32];
  __shared__ bool last;
  const StepParams<T>& p = M.p;
  MView<T> V;
  V.sD = reinterpret_cast<T*>(mom_smem);
  V.sU2 = V.sD + DF_N * DR * MWP;
  V.sU3 = V.sU2 + 3 * UR * MHP;
  V.sV3 = V.sU3 + (MX + 1) * MY;
  V.i0 = vb.x * MX;
  V.j0 = vb.y * MY;
  const int k0 = vb.z * M.zc, kend = min(p.nz, k0 + M.zc);
  const int tid = threadIdx.x, tx = tid % MX, ty = tid / MX;
  const int gi = V.i0 + tx, gj = V.j0 + ty;
  const bool own_c = gi < p.nx && gj < p.ny;
  const T dt = *p.dtT;
  const T c = dt * p.inv_h * p.inv_h;
  const T sc = -p.rho * p.h / *p.dtT;
  for (int kk = k0 - 2; kk <= k0 + 2; ++kk) stage_momentum(M, V.sD, V.i0, V.j0, kk);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  u2_plane(M, V, c, k0 - 1, k0, kend);
  u2_plane(M, V, c, k0, k0, kend);
  __syncthreads();
  const int h_own = V.hidx(gi, gj), s_own = V.sidx(gi, gj);
  // w3 of the column's bottom face (owned when k0 is this chunk's first plane)
  T w3lo = T(0);
  if (own_c) {
    const T* A[3] = {V.U2(0, k0), V.U2(1, k0), V.U2(2, k0)};
    const T* B[3] = {V.U2(0, k0 - 1), V.U2(1, k0 - 1), V.U2(2, k0 - 1)};
    w3lo = w3_at(p, dt, A, B, V.D(DF_C, k0 - 1), V.D(DF_C, k0), h_own, s_own, gi, gj, k0);
    M.w[idx_c(p, gi, gj, k0)] = w3lo;
  }
  DotAcc<T> dacc;
  for (int k = k0; k < kend; ++k) {
    cp_async_wait_all();
    __syncthreads();
    stage_momentum(M, V.sD, V.i0, V.j0, k + 3);
    cp_async_commit();
    u2_plane(M, V, c, k + 1, k0, kend);
    __syncthreads();
    // u3 of plane k's x faces i0..i0+MX and y faces j0..j0+MY, w3 of plane k+1
    const T* A[3] = {V.U2(0, k), V.U2(1, k), V.U2(2, k)};
    const T* B[3] = {V.U2(0, k + 1), V.U2(1, k + 1), V.U2(2, k + 1)};
    const T* Ck = V.D(DF_C, k);
    for (int it = tid; it < (MX + 1) * MY; it += MT) {
      const int fx = it % (MX + 1), fy = it / (MX + 1);
      const int fi = V.i0 + fx, fj = V.j0 + fy;
      if (fi <= p.nx && fj < p.ny) {
        const T val = u3_at(p, dt, A, B, Ck, (fx + 1) + MHX * (fy + 1), (fx + 2) + MWX * (fy + 2), fi, fj, k);
        V.sU3[it] = val;
        const bool own = fi < V.i0 + MX || fi == p.nx;
        if (own) M.u[idx_u(p, fi, fj, k)] = val;
      }
    }
    for (int it = tid; it < MX * (MY + 1); it += MT) {
      const int fx = it % MX, fy = it / MX;
      const int fi = V.i0 + fx, fj = V.j0 + fy;
      if (fi < p.nx && fj <= p.ny) {
        const T val = v3_at(p, dt, A, B, Ck, (fx + 1) + MHX * (fy + 1), (fx + 2) + MWX * (fy + 2), fi, fj, k);
        V.sV3[it] = val;
        const bool own = fj < V.j0 + MY || fj == p.ny;
        if (own) M.v[idx_v(p, fi, fj, k)] = val;
      }
    }
    T w3hi = T(0);
    if (own_c) {
      w3hi = w3_at(p, dt, B, A, Ck, V.D(DF_C, k + 1), h_own, s_own, gi, gj, k + 1);
      if (k + 1 < kend || k + 1 == p.nz) M.w[idx_c(p, gi, gj, k + 1)] = w3hi;
    }
    __syncthreads();
    if (own_c) {
      // cell_flux: u(i+1)-u(i) + v(j+1)-v(j) + w(k+1)-w(k)
      const T flux = V.sU3[(tx + 1) + (MX + 1) * ty] - V.sU3[tx + (MX + 1) * ty] + V.sV3[tx + MX * (ty + 1)] -
                     V.sV3[tx + MX * ty] + w3hi - w3lo;
      const T bv = sc * flux;
      M.b[idx_c(p, gi, gj, k)] = bv;
      dacc.add(bv, bv);
    }
    w3lo = w3hi;
  }
  cp_async_wait_all();
  double acc = 0.0;
  acc += dacc.value();
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(M.partials, &M.st->ticket[0], vals, &last, vb)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(M.partials, tot, sh, vb.n);
    if (thread_linear_id() == 0) {
      M.st->bb = tot[0];
      M.st->iter = 0;
      M.st->converged = 0;
      M.st->status = DEV_OK;
      M.st->ticket[0] = 0u;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(MT) k_momentum_fused(const __grid_constant__ MomentumArgs<T> M) {
  momentum_fused_body<T>(M, vblock());
}

}  // namespace uf
