// Fused MacCormack advection of the three velocity components (a2: Sec. 3,
// "Discretization and Numerical Integration", after Selle et al. 2008).
//
// One kernel runs both semi-Lagrangian passes.  A block owns a 32 x 8 column
// of lattice points (the same index range on the u, v and w lattices) and
// marches along z.  It stages, in shared memory:
//   * the time-level-n fields u, v, w on the column plus a halo of 2
//     (36 x 12 per plane, a ring of 8 planes per component, 5 of them live), copied one
//     plane ahead with cp.async;
//   * the forward-step values phi^ = phi(x - dt u(x)) of each component on
//     the column plus a halo of 1 (34 x 10 per plane, a ring of 4 planes, 3 live).
// The backward step, the correction phi* = phi^ + (phi - phi^(x + dt u(x)))/2
// and the clamp to the range of the forward sample's 8 values then read
// both from shared memory.  Per plane: two barriers (see advect_fused_body).
//
// Every value is formed by the same expressions as the two-kernel form
// (k_advect_forward, k_advect_backward) from the same inputs: displacement(),
// axis_cell() and trilerp() are shared, only the memory the corners come
// from differs.  The results are bit for bit those of the two kernels.
//
// A sample whose corners are not all in the staged window reads global
// memory instead (a displacement of a cell or more, possible with a fixed
// time step); a backward sample whose corners are not all in the phi^ window
// recomputes phi^ at its corners from global memory.  With the CFL time
// step the displacement stays below half a cell and neither happens.
//
// Tape (the adjoint's recompute sweep): when A.uh is not null, phi^ at every
// lattice point the block owns is also written to A.uh, A.vh, A.wh.
//
// When A.nut is not null the kernel also forms the eddy viscosity (a1) of
// the cells it owns from the staged time-level-n velocity, bit for bit what
// k_eddy_viscosity gives (strain_sq_acc rounds explicitly), which the step
// then does not launch.
#pragma once
#include "step_kernels.cuh"

namespace uf {

constexpr int MX = 32, MY = 8, MT = MX * MY;                    // owned column, threads per block
constexpr int MWX = MX + 4, MWY = MY + 4, MWP = MWX * MWY;      // window of the fields (halo 2)
constexpr int MHX = MX + 2, MHY = MY + 2, MHP = MHX * MHY;      // window of phi^ (halo 1)
// ring depths (planes): 5 and 3 are live; powers of two make the slot of plane
// kk (kk >= -2) a bit mask instead of a division
constexpr int MFR = 8, MHR = 4;
static_assert((MFR & (MFR - 1)) == 0 && (MHR & (MHR - 1)) == 0, "ring depths are powers of two");
#ifndef UF_ADVECT_MINB
#define UF_ADVECT_MINB 2   // resident blocks per SM the register budget is sized for
#endif

template <typename T>
constexpr size_t advect_fused_smem() {
  return sizeof(T) * 3 * ((size_t)MFR * MWP + (size_t)MHR * MHP);
}

// Staged planes [zlo, zhi] of a W x H window with lattice origin (ox, oy),
// held in a ring of R planes (R a power of two: plane kk in slot kk & (R - 1)).
template <typename T, int W, int H, int R>
struct Win {
  const T* ring;
  int ox, oy, zlo, zhi;
  __device__ __forceinline__ const T* plane(int kk) const { return ring + (kk & (R - 1)) * (W * H); }
  __device__ __forceinline__ bool holds(int i0, int i1, int j0, int j1, int k0, int k1) const {
    return i0 >= ox && i1 < ox + W && j0 >= oy && j1 < oy + H && k0 >= zlo && k1 <= zhi;
  }
  __device__ __forceinline__ void corners(int i0, int i1, int j0, int j1, int k0, int k1, T (&f)[8]) const {
    const T* p0 = plane(k0);
    const T* p1 = plane(k1);
    const int x0 = i0 - ox, x1 = i1 - ox, r0 = W * (j0 - oy), r1 = W * (j1 - oy);
    f[0] = p0[r0 + x0]; f[1] = p0[r0 + x1]; f[2] = p0[r1 + x0]; f[3] = p0[r1 + x1];
    f[4] = p1[r0 + x0]; f[5] = p1[r0 + x1]; f[6] = p1[r1 + x0]; f[7] = p1[r1 + x1];
  }
  __device__ __forceinline__ T at(int i, int j, int kk) const { return plane(kk)[(i - ox) + W * (j - oy)]; }
};

// Trilinear sample of a lattice field whose window is staged (global
// memory for corners outside the window).
template <typename T, bool RANGE, int W, int H, int R>
__device__ __forceinline__ T wsample(const T* __restrict__ g, Lattice L, const Win<T, W, H, R>& win, int ia, T oa,
                                     int ib, T ob, int ic, T oc, T* mn = nullptr, T* mx = nullptr) {
  int i0, i1, j0, j1, k0, k1;
  T ta, tb, tc;
  axis_cell(ia, oa, L.Lx, i0, i1, ta);
  axis_cell(ib, ob, L.Ly, j0, j1, tb);
  axis_cell(ic, oc, L.Lz, k0, k1, tc);
  T f[8];
  if (win.holds(i0, i1, j0, j1, k0, k1)) win.corners(i0, i1, j0, j1, k0, k1, f);
  else corners_global(g, L, i0, i1, j0, j1, k0, k1, f);
  return trilerp<T, RANGE>(f, ta, tb, tc, mn, mx);
}

// The three staged component windows of the fields.
template <typename T>
struct FWins {
  Win<T, MWX, MWY, MFR> c[3];
};

// phi^ at a lattice point from global memory only (the fallback of a
// backward sample that leaves the phi^ window): the forward step of
// advect_forward_body.
template <typename T>
__device__ __noinline__ T fh_global(const AdvectArgs<T>& A, int q, Lattice L, const T* __restrict__ F, int i, int j,
                                    int k, T s) {
  T d[3];
  displacement(A, q, i, j, k, s, d);
  return sample<T, false>(F, L, i, -d[0], j, -d[1], k, -d[2]);
}

// Per-component accessors (Q known at compile time).
template <int Q, typename T>
__device__ __forceinline__ Lattice lat_of(const AdvectArgs<T>& A) { return Q == 0 ? A.Lu : (Q == 1 ? A.Lv : A.Lw); }
template <int Q, typename T>
__device__ __forceinline__ const T* field_of(const AdvectArgs<T>& A) { return Q == 0 ? A.u : (Q == 1 ? A.v : A.w); }
template <int Q, typename T>
__device__ __forceinline__ T* fhat_of(const AdvectArgs<T>& A) { return Q == 0 ? A.uh : (Q == 1 ? A.vh : A.wh); }
template <int Q, typename T>
__device__ __forceinline__ T* out_of(const AdvectArgs<T>& A) { return Q == 0 ? A.ut : (Q == 1 ? A.vt : A.wt); }

// Asynchronous copy of one value global -> shared (cp.async, L1-allocating).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(sizeof(T)));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Starts the copy of plane kk of the three fields into its ring slot: the
// window positions tid and tid + MT of each component that lie on its lattice.
template <typename T>
__device__ __forceinline__ void stage_plane(const AdvectArgs<T>& A, T* sF, int i0, int j0, int kk) {
  if (kk < 0) return;
  const int slot = kk & (MFR - 1);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = threadIdx.x + h * MT;
    if (t >= MWP) break;
    const int gx = i0 - 2 + t % MWX, gy = j0 - 2 + t / MWX;
    if (gx < 0 || gy < 0) continue;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const Lattice L = q == 0 ? A.Lu : (q == 1 ? A.Lv : A.Lw);
      const T* F = q == 0 ? A.u : (q == 1 ? A.v : A.w);
      if (gx < L.Lx && gy < L.Ly && kk < L.Lz)
        cp_async_elem(sF + (q * MFR + slot) * MWP + t, F + (size_t)kk * ((size_t)L.P * L.Ly) + gx + (size_t)L.P * gy);
    }
  }
}

// Trilinear sample whose corners are all staged (the cross-component
// samples at half-cell offsets: within one cell of a point of the phi^
// window, whose planes the window always holds).
template <typename T, int W, int H, int R>
__device__ __forceinline__ T ssample(Lattice L, const Win<T, W, H, R>& win, int ia, T oa, int ib, T ob, int ic, T oc) {
  int i0, i1, j0, j1, k0, k1;
  T ta, tb, tc;
  axis_cell(ia, oa, L.Lx, i0, i1, ta);
  axis_cell(ib, ob, L.Ly, j0, j1, tb);
  axis_cell(ic, oc, L.Lz, k0, k1, tc);
  T f[8];
  win.corners(i0, i1, j0, j1, k0, k1, f);
  return trilerp<T, false>(f, ta, tb, tc, nullptr, nullptr);
}

// Displacement at a point of the phi^ window, the expressions of
// displacement() with the corners from the staged windows.
template <int Q, typename T>
__device__ __forceinline__ void displacement_s(const AdvectArgs<T>& A, const FWins<T>& Wn, int i, int j, int k, T s,
                                               T d[3]) {
  if (Q == 0) {   // u point (i, j+1/2, k+1/2)
    d[0] = s * Wn.c[0].at(i, j, k);
    d[1] = s * ssample(A.Lv, Wn.c[1], i, T(-0.5), j, T(0.5), k, T(0));
    d[2] = s * ssample(A.Lw, Wn.c[2], i, T(-0.5), j, T(0), k, T(0.5));
  } else if (Q == 1) {   // v point (i+1/2, j, k+1/2)
    d[0] = s * ssample(A.Lu, Wn.c[0], i, T(0.5), j, T(-0.5), k, T(0));
    d[1] = s * Wn.c[1].at(i, j, k);
    d[2] = s * ssample(A.Lw, Wn.c[2], i, T(0), j, T(-0.5), k, T(0.5));
  } else {   // w point (i+1/2, j+1/2, k)
    d[0] = s * ssample(A.Lu, Wn.c[0], i, T(0.5), j, T(0), k, T(-0.5));
    d[1] = s * ssample(A.Lv, Wn.c[1], i, T(0), j, T(0.5), k, T(-0.5));
    d[2] = s * Wn.c[2].at(i, j, k);
  }
}

// Per owned point and component, what the phi^ phase leaves for the
// backward step of the next plane: the displacement and the range of the
// forward sample's 8 values (the forward value itself is phi^ there).
// Ring of 2 planes: [plane & 1][component][value][MT].
constexpr int MKEEP = 5;
template <typename T>
constexpr size_t advect_keep_elems() { return (size_t)2 * 3 * MKEEP * MT; }

// phi^ of component Q at window position t (lattice point (gi, gj, m));
// stored in its ring slot (0 off the lattice), kept for owned points, taped.
template <int Q, typename T>
__device__ __forceinline__ void fhat_point(const AdvectArgs<T>& A, const FWins<T>& Wn, T* sH, T* sK, int m, int t,
                                           T s, int i0, int j0, int k0, int kend) {
  const Lattice L = lat_of<Q>(A);
  const int gi = i0 - 1 + t % MHX, gj = j0 - 1 + t / MHX;
  T val = T(0);
  if (gi >= 0 && gj >= 0 && m >= 0 && gi < L.Lx && gj < L.Ly && m < L.Lz) {
    T d[3], mn, mx;
    displacement_s<Q>(A, Wn, gi, gj, m, s, d);
    val = wsample<T, true>(field_of<Q>(A), L, Wn.c[Q], gi, -d[0], gj, -d[1], m, -d[2], &mn, &mx);
    const bool inx = gi >= i0 && gi < i0 + MX, iny = gj >= j0 && gj < j0 + MY;
    if (inx && iny) {
      T* kp = sK + ((m & 1) * 3 + Q) * MKEEP * MT + (gi - i0) + MX * (gj - j0);
      kp[0] = d[0]; kp[MT] = d[1]; kp[2 * MT] = d[2]; kp[3 * MT] = mn; kp[4 * MT] = mx;
    }
    T* tape = fhat_of<Q>(A);
    if (tape) {
      // owned: inside the column, or the lattice's last point beyond it
      const bool ox = inx || (gi >= i0 + MX && i0 + MX >= A.nx);
      const bool oy = iny || (gj >= j0 + MY && j0 + MY >= A.ny);
      const bool oz = (m >= k0 && m < kend) || (m >= kend && kend == A.nz);
      if (ox && oy && oz) tape[(size_t)gi + (size_t)L.P * ((size_t)gj + (size_t)L.Ly * m)] = val;
    }
  }
  sH[(Q * MHR + (m & (MHR - 1))) * MHP + t] = val;
}

// phi^ on plane m over the halo-1 window: 3 x MHP items (component,
// position) spread evenly over the threads.
template <typename T>
__device__ __forceinline__ void fhat_plane(const AdvectArgs<T>& A, T* sF, T* sH, T* sK, int m, int zlo, int zhi, T s,
                                           int i0, int j0, int k0, int kend) {
  FWins<T> Wn;
#pragma unroll
  for (int q = 0; q < 3; ++q) Wn.c[q] = Win<T, MWX, MWY, MFR>{sF + q * MFR * MWP, i0 - 2, j0 - 2, zlo, zhi};
#pragma unroll 1
  for (int it = threadIdx.x; it < 3 * MHP; it += MT) {
    if (it < MHP) fhat_point<0>(A, Wn, sH, sK, m, it, s, i0, j0, k0, kend);
    else if (it < 2 * MHP) fhat_point<1>(A, Wn, sH, sK, m, it - MHP, s, i0, j0, k0, kend);
    else fhat_point<2>(A, Wn, sH, sK, m, it - 2 * MHP, s, i0, j0, k0, kend);
  }
}

// Backward step, correction and clamp of component Q at the owned point
// (gi, gj, k): phi* = phi^ + (phi - phi^(x + dt u(x)))/2, clamped.
template <int Q, typename T>
__device__ __forceinline__ void maccormack_point(const AdvectArgs<T>& A, const T* sF, const T* sH, const T* sK,
                                                 int gi, int gj, int k, T s, int i0, int j0) {
  const bool interior = Q == 0 ? (gi > 0 && gi < A.nx && gj < A.ny)
                               : (Q == 1 ? (gi < A.nx && gj > 0 && gj < A.ny) : (gi < A.nx && gj < A.ny && k > 0 && k < A.nz));
  if (!interior) return;
  const Lattice L = lat_of<Q>(A);
  const int o = (gi - i0) + MX * (gj - j0);
  const T* kp = sK + ((k & 1) * 3 + Q) * MKEEP * MT + o;
  const T d0 = kp[0], d1 = kp[MT], d2 = kp[2 * MT], mn = kp[3 * MT], mx = kp[4 * MT];
  const Win<T, MHX, MHY, MHR> Hw{sH + Q * MHR * MHP, i0 - 1, j0 - 1, k - 1, k + 1};
  const T fwd = Hw.at(gi, gj, k);
  int a0, a1, b0, b1, c0, c1;
  T ta, tb, tc;
  axis_cell(gi, d0, L.Lx, a0, a1, ta);
  axis_cell(gj, d1, L.Ly, b0, b1, tb);
  axis_cell(k, d2, L.Lz, c0, c1, tc);
  T f[8];
  if (Hw.holds(a0, a1, b0, b1, c0, c1)) {
    Hw.corners(a0, a1, b0, b1, c0, c1, f);
  } else {
    const T* F = field_of<Q>(A);
    f[0] = fh_global(A, Q, L, F, a0, b0, c0, s); f[1] = fh_global(A, Q, L, F, a1, b0, c0, s);
    f[2] = fh_global(A, Q, L, F, a0, b1, c0, s); f[3] = fh_global(A, Q, L, F, a1, b1, c0, s);
    f[4] = fh_global(A, Q, L, F, a0, b0, c1, s); f[5] = fh_global(A, Q, L, F, a1, b0, c1, s);
    f[6] = fh_global(A, Q, L, F, a0, b1, c1, s); f[7] = fh_global(A, Q, L, F, a1, b1, c1, s);
  }
  const T bwd = trilerp<T, false>(f, ta, tb, tc, nullptr, nullptr);
  const T own = sF[(Q * MFR + (k & (MFR - 1))) * MWP + (gi - i0 + 2) + MWX * (gj - j0 + 2)];
  const T r = fwd + T(0.5) * (own - bwd);
  out_of<Q>(A)[(size_t)gi + (size_t)L.P * ((size_t)gj + (size_t)L.Ly * k)] = fmin(fmax(r, mn), mx);
}

// Eddy viscosity of cell (gi, gj, k) (the expressions of
// eddy_viscosity_body) with the faces strain_sq reads taken from the staged
// windows: planes k-1 .. k+2 of the fields are complete here.
template <typename T>
__device__ __forceinline__ void eddy_point(const AdvectArgs<T>& A, const T* sF, int gi, int gj, int k, int i0, int j0) {
  auto at = [&](int q, int a, int b, int c) {
    return sF[(q * MFR + (c & (MFR - 1))) * MWP + (a - i0 + 2) + MWX * (b - j0 + 2)];
  };
  const T S2 = strain_sq_acc<T>(
      A.sp, gi, gj, k, [&](int a, int b, int c) { return at(0, a, b, c); },
      [&](int a, int b, int c) { return at(1, a, b, c); }, [&](int a, int b, int c) { return at(2, a, b, c); });
  const size_t c = idx_c(A.sp, gi, gj, k);
  A.nut[c] = limited_nut(A.sp, A.kf[c], A.om[c], S2, *A.dtT);
}

template <typename T>
constexpr size_t advect_fused_smem_total() {
  return advect_fused_smem<T>() + sizeof(T) * advect_keep_elems<T>();
}

// Pipeline per output plane k:  wait for plane k+2 of the fields, sync,
// start the copy of plane k+3 (into the slot of k-2, which no one reads any
// more), phi^ of plane k+1, sync, phi* of plane k.  The phi^ phase reads
// the fields on planes [k-1, k+2].
template <typename T>
__device__ __forceinline__ void advect_fused_body(const AdvectArgs<T>& A, int zc, const VBlock& vb) {
  extern __shared__ __align__(16) unsigned char adv_smem[];
  T* sF = reinterpret_cast<T*>(adv_smem);   // [3][MFR][MWP]
  T* sH = sF + 3 * MFR * MWP;               // [3][MHR][MHP]
  T* sK = sH + 3 * MHR * MHP;               // [2][3][MKEEP][MT]
  const int i0 = vb.x * MX, j0 = vb.y * MY, k0 = vb.z * zc;
  const int kend = min(A.nz, k0 + zc);
  const T s = *A.dtT * A.inv_h;
  for (int kk = k0 - 2; kk <= k0 + 2; ++kk) stage_plane(A, sF, i0, j0, kk);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  fhat_plane(A, sF, sH, sK, k0 - 1, k0 - 2, k0 + 2, s, i0, j0, k0, kend);
  fhat_plane(A, sF, sH, sK, k0, k0 - 2, k0 + 2, s, i0, j0, k0, kend);
  const int gi = i0 + (int)threadIdx.x % MX, gj = j0 + (int)threadIdx.x / MX;
  for (int k = k0; k < kend; ++k) {
    cp_async_wait_all();
    __syncthreads();
    stage_plane(A, sF, i0, j0, k + 3);
    cp_async_commit();
    fhat_plane(A, sF, sH, sK, k + 1, k - 1, k + 2, s, i0, j0, k0, kend);
    __syncthreads();
    maccormack_point<0>(A, sF, sH, sK, gi, gj, k, s, i0, j0);
    maccormack_point<1>(A, sF, sH, sK, gi, gj, k, s, i0, j0);
    maccormack_point<2>(A, sF, sH, sK, gi, gj, k, s, i0, j0);
    if (A.nut && gi < A.nx && gj < A.ny) eddy_point(A, sF, gi, gj, k, i0, j0);
  }
  cp_async_wait_all();
}

template <typename T>
__global__ void __launch_bounds__(MT, UF_ADVECT_MINB) k_advect_fused(const __grid_constant__ AdvectArgs<T> A, int zc) {
  advect_fused_body<T>(A, zc, vblock());
}

}  // namespace uf
