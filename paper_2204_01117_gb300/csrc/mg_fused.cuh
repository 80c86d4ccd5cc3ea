// Fused multigrid V-cycle and CG kernels (shared-memory tiles).
//
// Each block owns a TX x TY x TZ tile of a level (thread (tx, ty) owns the
// column of TZ cells at x = tx, y = ty) and stages the tile plus a halo in
// shared memory, so that two dependent smoothing passes and the residual run
// without another trip to global memory:
//
//   (k_mg_down, k_mg_up and k_cg_dir_q march along z with rolling planes.)
//   k_mg_down  : [finest level: CG update x += a d, r -= a q, ||r||^2]
//                pre-smoothing from a zero guess, residual, summed
//                restriction to the next level (under linear transfers: the
//                residual, stored for k_restrict_lin).     reads r (q, x, d)
//   k_mg_up    : coarse-grid correction (piecewise-constant prolongation, or
//                the correction k_prolong_lin prolonged linearly) and the
//                post-smoothing passes; on the finest level also r.z and the
//                CG beta.                                  reads x_pre, e, r
//   k_restrict_lin, k_prolong_lin : the linear transfers between levels
//                below the finest, one pass each.
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

// Per-thread precomputation for a plane position (x, y) of a staged region
// with origin (ox, oy): x-y validity, 32-bit offset within a z plane, and
// the x-y part of the diagonal; per plane only the z terms remain.
template <typename T>
struct PosXY {
  bool ok;
  int off;
  T dxy;
};
template <typename T>
__device__ __forceinline__ PosXY<T> pos_xy(const Level<T>& L, int gx, int gy) {
  PosXY<T> r;
  r.ok = gx >= 0 && gy >= 0 && gx < L.nx && gy < L.ny;
  r.off = r.ok ? gx + L.P * gy : 0;
  T D = T(2) * (L.wx + L.wy);
  if (gx == 0 && !(L.out_mask & 1)) D -= L.wx;
  if (gx == L.nx - 1 && !(L.out_mask & 2)) D -= L.wx;
  if (gy == 0 && !(L.out_mask & 4)) D -= L.wy;
  if (gy == L.ny - 1 && !(L.out_mask & 8)) D -= L.wy;
  r.dxy = D;
  return r;
}
// z part of the diagonal for plane k.
template <typename T>
__device__ __forceinline__ T diag_z(const Level<T>& L, int k) {
  T D = T(2) * L.wz;
  if (k == 0 && !(L.out_mask & 16)) D -= L.wz;
  if (k == L.nz - 1 && !(L.out_mask & 32)) D -= L.wz;
  return D;
}

// Weights of the two weighted-Jacobi sweeps x <- x + w_k D^-1 (r - A x)
// (k = 1, 2).  From x = 0 the pair gives x2 = pa q + pb D^-1 sum w_a q_nb
// with q = r/D, pa = w1 + w2 - w1 w2 and pb = w1 w2.  Damped Jacobi: w1 = w2
// = w.  Chebyshev: the roots of the degree-2 Chebyshev polynomial on the
// high-frequency range of D^-1 A (see the host side).  The two factors
// commute, so post-smoothing with the same weights keeps the V-cycle
// symmetric.
template <typename T>
struct SmoothW {
  T pa, pb;   // pre-smoothing from zero
  T w1, w2;   // post-smoothing passes
};

// Reciprocal of a diagonal entry for the smoothers.  FP32: the hardware
// approximation rcp.approx.ftz (at most 1 ulp off), one instruction where an
// IEEE division is a subroutine; the smoother only needs a fixed diagonal
// scaling, and the same scaling in every sweep keeps the V-cycle symmetric.
// FP64: exact.
__device__ __forceinline__ float rdiag(float D) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(D));
  return r;
}
__device__ __forceinline__ double rdiag(double D) { return 1.0 / D; }

// (add_rn, mul_rn, fma_rn: uf_device.cuh.)  The smoother and residual
// expressions below are shared by the per-level kernels and the cluster
// V-cycle and spelled with them, so both compute them alike, bit for bit.

// w_x (a1 + a2) + w_y (b1 + b2) + w_z (c1 + c2): the weighted sum of the six
// neighbours of a cell (x pair, y pair, z pair).
template <typename T>
__device__ __forceinline__ T nb6(T wx, T a1, T a2, T wy, T b1, T b2, T wz, T c1, T c2) {
  return fma_rn(wz, add_rn(c1, c2), fma_rn(wy, add_rn(b1, b2), mul_rn(wx, add_rn(a1, a2))));
}
// Residual r - A x at a cell, with q = r/D: D (q - x) + sum_6 w x_nb.
template <typename T>
__device__ __forceinline__ T resid(T D, T q, T x, T nbsum) {
  return fma_rn(D, add_rn(q, -x), nbsum);
}

// Cell-centred linear transfers between a level (n_f cells along an axis)
// and the next coarser one (n_c = ceil(n_f / 2)).  Prolongation along a
// halved axis: fine cell i takes 3/4 of its parent p = i/2 and 1/4 of the
// parent's neighbour on its own side (p - 1 for even i, p + 1 for odd i);
// beyond the level that neighbour is a ghost, the parent mirrored (dp/dn =
// 0: weight 3/4 + 1/4 on p) or negated on an outlet side (p = 0 on the
// face: 3/4 - 1/4).  An axis that is not halved maps cell to cell.  The
// restriction is the transpose: coarse cell p gathers its children 2p and
// 2p + 1 (3/4, or the ghost-folded weight at the level's ends) and the
// outer neighbours 2p - 1 and 2p + 2 (1/4).
// A prolongation value is one FMA chain over the slots inside the level, z
// outermost, then y, then x (slot s is cell base + s); a restriction value
// is four such chains, one per z slot, added in slot order (restrict_lin).
// The arithmetic is explicitly rounded, and every weight and every product
// of three is exact in binary, so a value is the same bit for bit wherever
// it is formed (the pass kernels, the tail, the batch, the cluster V-cycle).
struct Taps {
  int base;    // cell index of slot 0
  int valid;   // bit s: slot s takes part
  float w[4];
};
// Prolongation taps of fine cell i along an axis (slots p - 1, p, p + 1).
__device__ __forceinline__ Taps taps_p(int i, int halved, int nc, bool out_lo, bool out_hi) {
  Taps t;
  t.w[0] = t.w[2] = t.w[3] = 0.25f;
  if (!halved) {
    t.base = i - 1; t.valid = 2; t.w[1] = 1.0f;
    return t;
  }
  const int p = i >> 1;
  t.base = p - 1;
  if (i & 1) {   // neighbour p + 1
    const bool in = p + 1 < nc;
    t.valid = in ? 6 : 2;
    t.w[1] = in ? 0.75f : (out_hi ? 0.5f : 1.0f);
  } else {       // neighbour p - 1
    const bool in = p >= 1;
    t.valid = in ? 3 : 2;
    t.w[1] = in ? 0.75f : (out_lo ? 0.5f : 1.0f);
  }
  return t;
}
// Restriction taps of coarse cell p along an axis of nf fine cells (slots
// 2p - 1, 2p, 2p + 1, 2p + 2).
__device__ __forceinline__ Taps taps_r(int p, int halved, int nf, int nc, bool out_lo, bool out_hi) {
  Taps t;
  t.w[0] = t.w[3] = 0.25f;
  if (!halved) {
    t.base = p - 1; t.valid = 2; t.w[1] = 1.0f; t.w[2] = 0.0f;
    return t;
  }
  t.base = 2 * p - 1;
  t.valid = (p >= 1 ? 1 : 0) | 2 | (2 * p + 1 < nf ? 4 : 0) | (2 * p + 2 < nf ? 8 : 0);
  t.w[1] = p == 0 ? (out_lo ? 0.5f : 1.0f) : 0.75f;
  t.w[2] = p == nc - 1 ? (out_hi ? 0.5f : 1.0f) : 0.75f;
  return t;
}
// (loops unrolled over the four slots and predicated, so the taps stay in
// registers)
template <typename T, typename Get>
__device__ __forceinline__ T tap_sum(const Taps& tx, const Taps& ty, const Taps& tz, Get get) {
  T acc = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (!((tz.valid >> c) & 1)) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (!((ty.valid >> b) & 1)) continue;
      const T wzy = (T)tz.w[c] * (T)ty.w[b];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (!((tx.valid >> a) & 1)) continue;
        acc = fma_rn(wzy * (T)tx.w[a], get(tx.base + a, ty.base + b, tz.base + c), acc);
      }
    }
  }
  return acc;
}
// (P e)(i, j, k) on fine level F from the coarse values get(ci, cj, ck) of C.
template <typename T, typename Get>
__device__ __forceinline__ T prolong_lin(const Level<T>& F, const Level<T>& C, int i, int j, int k, Get get) {
  const int m = F.out_mask;
  return tap_sum<T>(taps_p(i, F.cx, C.nx, m & 1, m & 2), taps_p(j, F.cy, C.ny, m & 4, m & 8),
                    taps_p(k, F.cz, C.nz, m & 16, m & 32), get);
}
// (R r)(ci, cj, ck) on coarse level C from the fine values get(i, j, k) of F,
// as four partial sums, one per z slot (each an FMA chain over y, then x),
// added in slot order: ((P0 + P1) + P2) + P3 (an absent slot is 0).  The
// partials can be formed by four threads (k_restrict_lin, the tail) or one
// after another (restrict_lin), with the same result.
template <typename T, typename Get>
__device__ __forceinline__ T restrict_partial(const Level<T>& F, const Level<T>& C, int ci, int cj, int ck, int c,
                                              Get get) {
  const int m = F.out_mask;
  const Taps tz = taps_r(ck, F.cz, F.nz, C.nz, m & 16, m & 32);
  if (!((tz.valid >> c) & 1)) return T(0);
  const Taps tx = taps_r(ci, F.cx, F.nx, C.nx, m & 1, m & 2), ty = taps_r(cj, F.cy, F.ny, C.ny, m & 4, m & 8);
  const T wz = (T)(c == 0 ? tz.w[0] : c == 1 ? tz.w[1] : c == 2 ? tz.w[2] : tz.w[3]);   // (no indexed array)
  T acc = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (!((ty.valid >> b) & 1)) continue;
    const T wzy = wz * (T)ty.w[b];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (!((tx.valid >> a) & 1)) continue;
      acc = fma_rn(wzy * (T)tx.w[a], get(tx.base + a, ty.base + b, tz.base + c), acc);
    }
  }
  return acc;
}
template <typename T>
__device__ __forceinline__ T combine_partials(T p0, T p1, T p2, T p3) {
  return add_rn(add_rn(add_rn(p0, p1), p2), p3);
}
template <typename T, typename Get>
__device__ __forceinline__ T restrict_lin(const Level<T>& F, const Level<T>& C, int ci, int cj, int ck, Get get) {
  return combine_partials(restrict_partial(F, C, ci, cj, ck, 0, get), restrict_partial(F, C, ci, cj, ck, 1, get),
                          restrict_partial(F, C, ci, cj, ck, 2, get), restrict_partial(F, C, ci, cj, ck, 3, get));
}
// The same with the four partials on four adjacent lanes (lane & 3 = slot;
// every lane of the warp calls this): returns the sum on every lane.
template <typename T>
__device__ __forceinline__ T quad_combine(T part) {
  const int qb = (threadIdx.x & 31) & ~3;
  const T p0 = __shfl_sync(0xffffffffu, part, qb), p1 = __shfl_sync(0xffffffffu, part, qb + 1);
  const T p2 = __shfl_sync(0xffffffffu, part, qb + 2), p3 = __shfl_sync(0xffffffffu, part, qb + 3);
  return combine_partials(p0, p1, p2, p3);
}

// Pre-smoothing from zero with q = r/D staged: weighted Jacobi x2 = pa q_c +
// pb/D_c sum w_a q_nb;  RBGS red q_c, black q_c + sum w_a q_nb / D_c.
template <int SM, typename T>
__device__ __forceinline__ T presmooth(T qc, T s, T D, const SmoothW<T>& W, bool red) {
  if (SM == SM_JACOBI) return fma_rn(W.pa, qc, mul_rn(mul_rn(W.pb, s), rdiag(D)));
  return red ? qc : fma_rn(s, rdiag(D), qc);
}
// Post-smoothing pass on t: weighted Jacobi t + w (r - D t + s)/D; RBGS
// relaxes the colour `relax` and keeps the other.
template <int SM, typename T>
__device__ __forceinline__ T relax(T tc, T rc, T s, T D, T omega, bool active) {
  if (SM == SM_JACOBI) return fma_rn(mul_rn(omega, add_rn(fma_rn(-D, tc, rc), s)), rdiag(D), tc);
  return active ? mul_rn(add_rn(rc, s), rdiag(D)) : tc;
}

// ------------------------------------------------------------ down -------
// Blocks own a 32 x 8 column of cells and march along z over `zc` planes
// (zc even), keeping rolling planes in shared memory: q = r/D on the tile
// plus a halo of 2 (ring of 4 planes), the pre-smoothed x on the tile plus a
// halo of 1 (ring of 3), and the residual of the current z pair.  Per plane:
// load q(k+2); pre-smooth x(k+1); residual of plane k; after every pair of
// planes, restrict it.  CG = true (finest level inside the CG loop): the
// kernel first applies x += alpha d, r -= alpha q (r ping-pongs), reduces
// ||r||^2 and runs the convergence test.
constexpr int QX = TX + 4, QY = TY + 4, QP = QX * QY;   // 36 x 12 plane (halo 2)
constexpr int XX = TX + 2, XY = TY + 2, XP = XX * XY;   // 34 x 10 plane (halo 1)

__device__ __forceinline__ int ring3(int k) { return ((k % 3) + 3) % 3; }
__device__ __forceinline__ int ring4(int k) { return (k + 4) & 3; }

template <typename T, int SM, bool CG>
__device__ __forceinline__ void mg_down_body(const Level<T>& F, const Level<T>& C, const SmoothW<T>& W, int zc, T* __restrict__ x,
                                             const T* d0, const T* d1, const T* __restrict__ q, double* partials,
                                             SolveState* st, cudaGraphConditionalHandle cond, int use_cond,
                                             int* left, const VBlock& vb) {
  __shared__ T sQ[4][QP];
  __shared__ T sX[3][XP];
  __shared__ T sR[2][FT];
  __shared__ double sh[32];
  __shared__ bool last;
  // (a converged solve skips the whole cycle; in a batch, the instances
  // that converged wait here for the others)
  if (st->converged) return;
  const int i0 = vb.x * TX, j0 = vb.y * TY, k0 = vb.z * zc;
  const int kend = min(F.nz, k0 + zc);
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
  const size_t PS = (size_t)F.P * F.ny;   // z-plane stride
  // per-thread positions: two in the halo-2 plane, two in the halo-1 plane
  const PlaneMap mq = plane_map<QX, QY>();
  const PlaneMap mx = plane_map<XX, XY>();
  PosXY<T> pq[2], px[2];
  int sq[2], sx[2], sxq[2], par[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int qx = h ? mq.x1 : mq.x0, qy = h ? mq.y1 : mq.y0;
    pq[h] = pos_xy(F, i0 - 2 + qx, j0 - 2 + qy);
    if (h == 1 && !mq.has1) pq[h].ok = false;
    sq[h] = qx + QX * qy;
    const int xx = h ? mx.x1 : mx.x0, xy = h ? mx.y1 : mx.y0;
    px[h] = pos_xy(F, i0 - 1 + xx, j0 - 1 + xy);
    if (h == 1 && !mx.has1) px[h].ok = false;
    sx[h] = xx + XX * xy;
    sxq[h] = (xx + 1) + QX * (xy + 1);
    par[h] = (i0 - 1 + xx + j0 - 1 + xy) & 1;
  }
  const int gi = i0 + tx, gj = j0 + ty;
  const PosXY<T> po = pos_xy(F, gi, gj);
  const int opar = (gi + gj) & 1;
  // q-plane staging: a load stage (global -> registers) and a commit stage
  // (registers -> shared), one iteration apart, so that the loads of plane
  // k+3 are in flight while planes k+1 and k are processed.
  T pr[2], pqv[2];
  auto issueQ = [&](int k) {
    const bool kin = (unsigned)k < (unsigned)F.nz;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      pr[h] = 0;
      pqv[h] = 0;
      if (kin && pq[h].ok) {
        const size_t c = (size_t)k * PS + pq[h].off;
        pr[h] = r_in[c];
        if (CG) pqv[h] = q[c];
      }
    }
  };
  auto commitQ = [&](int k) {
    T* dst = sQ[ring4(k)];
    const bool kin = (unsigned)k < (unsigned)F.nz;
    const T dz = diag_z(F, k);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !mq.has1) break;
      dst[sq[h]] = (kin && pq[h].ok) ? (CG ? pr[h] - alpha * pqv[h] : pr[h]) * rdiag(pq[h].dxy + dz) : T(0);
    }
  };
  auto computeX = [&](int k, int slot) {
    T* dst = sX[slot];
    const T* qm = sQ[ring4(k - 1)];
    const T* qc = sQ[ring4(k)];
    const T* qp = sQ[ring4(k + 1)];
    const bool kin = (unsigned)k < (unsigned)F.nz;
    const T dz = diag_z(F, k);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !mx.has1) break;
      T v = 0;
      if (kin && px[h].ok) {
        const int b = sxq[h];
        const T s = nb6(F.wx, qc[b - 1], qc[b + 1], F.wy, qc[b - QX], qc[b + QX], F.wz, qm[b], qp[b]);
        v = presmooth<SM>(qc[b], s, px[h].dxy + dz, W, ((par[h] + k) & 1) == 0);
      }
      dst[sx[h]] = v;
    }
  };
  const int fx = F.cx ? 2 : 1, fy = F.cy ? 2 : 1;
  const int cnx = TX / fx, cny = TY / fy;
  double acc = 0.0;
  DotAcc<T> dacc;

  issueQ(k0 - 2); commitQ(k0 - 2);
  issueQ(k0 - 1); commitQ(k0 - 1);
  issueQ(k0); commitQ(k0);
  issueQ(k0 + 1);
  // ring slots of the pre-smoothed planes k - 1, k, k + 1, rotated once per plane
  int xs_m = ring3(k0 - 1), xs_c = ring3(k0), xs_p = ring3(k0 + 1);
  __syncthreads();
  computeX(k0 - 1, xs_m);
  commitQ(k0 + 1);
  issueQ(k0 + 2);
  __syncthreads();
  computeX(k0, xs_c);
  __syncthreads();
  // a z-coarsened level of odd extent ends on a pair whose second plane is
  // outside the domain (its residual is zero)
  const int klast = (F.cz && (kend & 1)) ? kend + 1 : kend;
  const int b1 = (tx + 1) + XX * (ty + 1);
  const int b2 = (tx + 2) + QX * (ty + 2);
  for (int k = k0; k < klast; ++k) {
    const bool own = po.ok && k < F.nz;
    // owned-cell operands of this plane, loaded ahead of the barriers
    T o_r = 0, o_q = 0, o_x = 0, o_d = 0;
    const size_t oc = (size_t)k * PS + po.off;
    if (CG && own) {
      o_r = r_in[oc];
      o_q = q[oc];
      o_x = x[oc];
      o_d = dn[oc];
    }
    commitQ(k + 2);
    issueQ(k + 3);
    __syncthreads();
    computeX(k + 1, xs_p);
    __syncthreads();
    T res = 0;
    if (own) {
      const T* xm = sX[xs_m];
      const T* xc = sX[xs_c];
      const T* xp = sX[xs_p];
      const T xv = xc[b1];
      F.x[oc] = xv;
      res = resid(po.dxy + diag_z(F, k), sQ[ring4(k)][b2], xv,
                  nb6(F.wx, xc[b1 - 1], xc[b1 + 1], F.wy, xc[b1 - XX], xc[b1 + XX], F.wz, xm[b1], xp[b1]));
      if (CG) {
        const T rv = o_r - alpha * o_q;
        r_out[oc] = rv;
        x[oc] = o_x + alpha * o_d;
        dacc.add(rv, rv);
      }
    }
    (void)opar;
    if (!CG && F.lin) {   // linear transfers: the restriction runs as its own pass over the stored residual
      if (own) F.t[oc] = res;
    } else {
      sR[k & 1][tid] = res;
      if (!F.cz || (k & 1)) {
        __syncthreads();
        const int kc = F.cz ? (k >> 1) : k;
        for (int e = tid; e < cnx * cny; e += FT) {
          const int cxl = e % cnx, cyl = e / cnx;
          const int ci = i0 / fx + cxl, cj = j0 / fy + cyl;
          if (!in_level(C, ci, cj, kc)) continue;
          T sum = 0;
          for (int dz = F.cz ? 1 : 0; dz >= 0; --dz)
            for (int dy = 0; dy < fy; ++dy)
              for (int dx = 0; dx < fx; ++dx) sum += sR[(k - dz) & 1][(cxl * fx + dx) + TX * (cyl * fy + dy)];
          C.r[lidx(C, ci, cj, kc)] = sum;
        }
      }
    }
    const int xs_t = xs_m;
    xs_m = xs_c;
    xs_c = xs_p;
    xs_p = xs_t;
  }
  if (CG) {
    acc += dacc.value();
    acc = block_sum<FT>(acc, sh);
    const double vals[1] = {acc};
    if (publish_partials<1>(partials, &st->ticket[3], vals, &last, vb)) {
      double tot[1];
      reduce_partials_sum<FT, 1>(partials, tot, sh, vb.n);
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
        if (st->converged) signal_converged(cond, use_cond, left);
        st->ticket[3] = 0u;
      }
    }
  }
}

template <typename T, int SM, bool CG>
__global__ void __launch_bounds__(FT) k_mg_down(Level<T> F, Level<T> C, SmoothW<T> W, int zc, T* __restrict__ x,
                                               const T* d0, const T* d1, const T* __restrict__ q,
                                               double* partials, SolveState* st, cudaGraphConditionalHandle cond,
                                               int use_cond) {
  mg_down_body<T, SM, CG>(F, C, W, zc, x, d0, d1, q, partials, st, cond, use_cond, nullptr, vblock());
}


// ------------------------------------------------------- restriction -----
// Linear transfers (F.lin): the down kernel of F stores its residual in F.t;
// before the down kernel of the next level C, C.r = R F.t, and before the
// up kernel of F, F.e = P C.t (the up kernel reads it as it would read the
// parent's value).  One thread per cell of the level written (k_restrict_lin,
// k_prolong_lin), or, in a batch, per column of a march tile of level C.
template <typename T>
__device__ __forceinline__ void restrict_lin_at(const Level<T>& F, const Level<T>& C, int ci, int cj, int ck) {
  C.r[lidx(C, ci, cj, ck)] = restrict_lin(F, C, ci, cj, ck, [&](int i, int j, int k) { return F.t[lidx(F, i, j, k)]; });
}
template <typename T>
__device__ __forceinline__ void prolong_lin_at(const Level<T>& F, const Level<T>& C, int i, int j, int k) {
  F.e[lidx(F, i, j, k)] = prolong_lin(F, C, i, j, k, [&](int a, int b, int c) { return C.t[lidx(C, a, b, c)]; });
}

// Four threads per coarse cell (one per z slot of the restriction).
template <typename T>
__global__ void __launch_bounds__(FT) k_restrict_lin(Level<T> F, Level<T> C, const SolveState* st) {
  if (st->converged) return;
  const long long e = ((long long)blockIdx.x * FT + threadIdx.x) >> 2;
  const int slot = threadIdx.x & 3;
  const bool in = e < (long long)C.nx * C.ny * C.nz;
  const int ci = in ? (int)(e % C.nx) : 0, cj = in ? (int)((e / C.nx) % C.ny) : 0;
  const int ck = in ? (int)(e / ((long long)C.nx * C.ny)) : 0;
  const T part = in ? restrict_partial(F, C, ci, cj, ck, slot, [&](int i, int j, int k) { return F.t[lidx(F, i, j, k)]; })
                    : T(0);
  const T sum = quad_combine(part);   // (every lane of the warp takes part)
  if (in && slot == 0) C.r[lidx(C, ci, cj, ck)] = sum;
}
template <typename T>
__global__ void __launch_bounds__(FT) k_prolong_lin(Level<T> F, Level<T> C, const SolveState* st) {
  if (st->converged) return;
  const long long e = (long long)blockIdx.x * FT + threadIdx.x;
  if (e >= (long long)F.nx * F.ny * F.nz) return;
  const int i = (int)(e % F.nx), j = (int)((e / F.nx) % F.ny), k = (int)(e / ((long long)F.nx * F.ny));
  prolong_lin_at(F, C, i, j, k);
}

// The same over a march tile of level C (batched launches).
template <typename T>
__device__ __forceinline__ void restrict_lin_body(const Level<T>& F, const Level<T>& C, int zc, const SolveState* st,
                                                  const VBlock& vb) {
  if (st->converged) return;
  const int ci = vb.x * TX + (threadIdx.x & (TX - 1)), cj = vb.y * TY + threadIdx.x / TX;
  const int k0 = vb.z * zc, kend = min(C.nz, k0 + zc);
  if (ci >= C.nx || cj >= C.ny) return;
  for (int ck = k0; ck < kend; ++ck) restrict_lin_at(F, C, ci, cj, ck);
}
template <typename T>
__device__ __forceinline__ void prolong_lin_body(const Level<T>& F, const Level<T>& C, int zc, const SolveState* st,
                                                 const VBlock& vb) {
  if (st->converged) return;
  const int ci = vb.x * TX + (threadIdx.x & (TX - 1)), cj = vb.y * TY + threadIdx.x / TX;
  const int k0 = vb.z * zc, kend = min(C.nz, k0 + zc);
  if (ci >= C.nx || cj >= C.ny) return;
  const int fx = F.cx ? 2 : 1, fy = F.cy ? 2 : 1, fz = F.cz ? 2 : 1;
  for (int ck = k0; ck < kend; ++ck)
    for (int dz = 0; dz < fz; ++dz)
      for (int dy = 0; dy < fy; ++dy)
        for (int dx = 0; dx < fx; ++dx) {
          const int i = ci * fx + dx, j = cj * fy + dy, k = ck * fz + dz;
          if (in_level(F, i, j, k)) prolong_lin_at(F, C, i, j, k);
        }
}

// -------------------------------------------------------------- up -------
// Same z-march: t = x_pre + e(parent) on tile + halo 2 (ring of 4), first
// post-smoothing pass on tile + halo 1 (ring of 3), second pass on the owned
// plane, written to `out` (F.t on coarse levels, z on the finest).
// FINEST: also r.z and the CG beta.  Global loads run one plane ahead.
template <typename T, int SM, bool FINEST>
__device__ __forceinline__ void mg_up_body(const Level<T>& F, const Level<T>& C, const SmoothW<T>& W, int zc, T* __restrict__ out,
                                           int mode, double* partials, SolveState* st, const VBlock& vb) {
  __shared__ T sT[4][QP];
  __shared__ T sU[3][XP];
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->converged) return;
  const int i0 = vb.x * TX, j0 = vb.y * TY, k0 = vb.z * zc;
  const int kend = min(F.nz, k0 + zc);
  const int tid = threadIdx.x, tx = tid & (TX - 1), ty = tid / TX;
  const T* rcur = level_r(F, st->iter);
  const size_t PS = (size_t)F.P * F.ny, PSC = (size_t)C.P * C.ny;
  const PlaneMap mq = plane_map<QX, QY>();
  const PlaneMap mx = plane_map<XX, XY>();
  PosXY<T> pt[2], pu[2];
  int st_[2], su[2], sut[2], par[2], poff[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int qx = h ? mq.x1 : mq.x0, qy = h ? mq.y1 : mq.y0;
    const int hi = i0 - 2 + qx, hj = j0 - 2 + qy;
    pt[h] = pos_xy(F, hi, hj);
    if (h == 1 && !mq.has1) pt[h].ok = false;
    st_[h] = qx + QX * qy;
    poff[h] = pt[h].ok ? (F.cx ? hi >> 1 : hi) + C.P * (F.cy ? hj >> 1 : hj) : 0;
    const int xx = h ? mx.x1 : mx.x0, xy = h ? mx.y1 : mx.y0;
    pu[h] = pos_xy(F, i0 - 1 + xx, j0 - 1 + xy);
    if (h == 1 && !mx.has1) pu[h].ok = false;
    su[h] = xx + XX * xy;
    sut[h] = (xx + 1) + QX * (xy + 1);
    par[h] = (i0 - 1 + xx + j0 - 1 + xy) & 1;
  }
  const int gi = i0 + tx, gj = j0 + ty;
  const PosXY<T> po = pos_xy(F, gi, gj);
  const int opar = (gi + gj) & 1;
  T px[2], pe[2];   // t-plane loads in flight
  T pr[2];          // r on the halo-1 plane in flight
  auto issueT = [&](int k) {
    const bool kin = (unsigned)k < (unsigned)F.nz;
    const int pk = F.cz ? k >> 1 : k;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      px[h] = 0;
      pe[h] = 0;
      if (kin && pt[h].ok) {
        px[h] = F.x[(size_t)k * PS + pt[h].off];
        // (linear transfers: the prolonged correction, formed before this kernel)
        pe[h] = F.lin ? F.e[(size_t)k * PS + pt[h].off] : C.t[(size_t)pk * PSC + poff[h]];
      }
    }
  };
  auto commitT = [&](int k) {
    T* dst = sT[ring4(k)];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !mq.has1) break;
      dst[st_[h]] = px[h] + pe[h];
    }
  };
  auto issueR = [&](int k) {
    const bool kin = (unsigned)k < (unsigned)F.nz;
#pragma unroll
    for (int h = 0; h < 2; ++h) pr[h] = (kin && pu[h].ok) ? rcur[(size_t)k * PS + pu[h].off] : T(0);
  };
  auto computeU = [&](int k, int slot) {
    T* dst = sU[slot];
    const T* tm = sT[ring4(k - 1)];
    const T* tc = sT[ring4(k)];
    const T* tp = sT[ring4(k + 1)];
    const bool kin = (unsigned)k < (unsigned)F.nz;
    const T dz = diag_z(F, k);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !mx.has1) break;
      T v = 0;
      if (kin && pu[h].ok) {
        const int b = sut[h];
        const T s = nb6(F.wx, tc[b - 1], tc[b + 1], F.wy, tc[b - QX], tc[b + QX], F.wz, tm[b], tp[b]);
        v = relax<SM>(tc[b], pr[h], s, pu[h].dxy + dz, W.w1, ((par[h] + k) & 1) == 1);
      }
      dst[su[h]] = v;
    }
  };
  double acc = 0.0;
  DotAcc<T> dacc;
  issueT(k0 - 2); commitT(k0 - 2);
  issueT(k0 - 1); commitT(k0 - 1);
  issueT(k0); commitT(k0);
  issueT(k0 + 1);
  issueR(k0 - 1);
  // ring slots of the relaxed planes k - 1, k, k + 1, rotated once per plane
  int us_m = ring3(k0 - 1), us_c = ring3(k0), us_p = ring3(k0 + 1);
  __syncthreads();
  computeU(k0 - 1, us_m);
  commitT(k0 + 1);
  issueT(k0 + 2);
  issueR(k0);
  __syncthreads();
  computeU(k0, us_c);
  issueR(k0 + 1);
  __syncthreads();
  const int b = (tx + 1) + XX * (ty + 1);
  for (int k = k0; k < kend; ++k) {
    T o_r = 0;
    const size_t oc = (size_t)k * PS + po.off;
    if (po.ok) o_r = rcur[oc];
    commitT(k + 2);
    issueT(k + 3);
    __syncthreads();
    computeU(k + 1, us_p);
    issueR(k + 2);
    __syncthreads();
    if (po.ok) {
      const T* um = sU[us_m];
      const T* uc = sU[us_c];
      const T* up = sU[us_p];
      const T s = nb6(F.wx, uc[b - 1], uc[b + 1], F.wy, uc[b - XX], uc[b + XX], F.wz, um[b], up[b]);
      const T zv = relax<SM>(uc[b], o_r, s, po.dxy + diag_z(F, k), W.w2, ((opar + k) & 1) == 0);
      out[oc] = zv;
      if (FINEST) dacc.add(o_r, zv);
    }
    const int us_t = us_m;
    us_m = us_c;
    us_c = us_p;
    us_p = us_t;
  }
  if (FINEST) {
    acc += dacc.value();
    acc = block_sum<FT>(acc, sh);
    const double vals[1] = {acc};
    if (publish_partials<1>(partials, &st->ticket[0], vals, &last, vb)) {
      double tot[1];
      reduce_partials_sum<FT, 1>(partials, tot, sh, vb.n);
      if (tid == 0) {
        finish_rz(st, tot[0], mode);
        st->ticket[0] = 0u;
      }
    }
  }
}

template <typename T, int SM, bool FINEST>
__global__ void __launch_bounds__(FT) k_mg_up(Level<T> F, Level<T> C, SmoothW<T> W, int zc, T* __restrict__ out, int mode,
                                             double* partials, SolveState* st) {
  mg_up_body<T, SM, FINEST>(F, C, W, zc, out, mode, partials, st, vblock());
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

// The cells of an nx x ny x nz tail level spread over the TAIL_T threads
// laid out 16 x 16 x 4 (x fastest): thread (tx, ty, tz) takes i = tx, tx +
// 16, ..., j = ty, ty + 16, ..., k = tz, tz + 4, ...  No division by the
// level's extents (an integer division by a run-time value is a long
// instruction sequence, and the tail would take several per cell and pass).
template <typename F>
__device__ __forceinline__ void tail_cells(int nx, int ny, int nz, F f) {
  static_assert(TAIL_T == 16 * 16 * 4, "tail thread layout");
  const int tx = threadIdx.x & 15, ty = (threadIdx.x >> 4) & 15, tz = threadIdx.x >> 8;
  for (int k = tz; k < nz; k += 4)
    for (int j = ty; j < ny; j += 16)
      for (int i = tx; i < nx; i += 16) f(i, j, k);
}

// The cells of level C, four threads per cell (slot = lane & 3): part(i, j,
// k, slot) forms a partial on each, and put(i, j, k, sum) stores their sum
// (quad_combine; the loop runs over whole warps so that every lane takes
// part in the shuffles).
template <typename T, typename Part, typename Put>
__device__ __forceinline__ void tail_quads(const Level<T>& C, Part part, Put put) {
  const int nc = C.nx * C.ny * C.nz, n4 = ((4 * nc + 31) / 32) * 32;
  for (int e = threadIdx.x; e < n4; e += TAIL_T) {
    const int cell = e >> 2;
    const bool in = cell < nc;
    const int i = in ? cell % C.nx : 0, j = in ? (cell / C.nx) % C.ny : 0, k = in ? cell / (C.nx * C.ny) : 0;
    const T sum = quad_combine(in ? part(i, j, k, e & 3) : T(0));
    if (in && (e & 3) == 0) put(i, j, k, sum);
  }
}

template <typename T>
struct TailArgs {
  Level<T> lv[MAX_LEVELS];
  int lt, nl;
  int off[MAX_LEVELS];   // element offset of each tail level's three bordered arrays
  int cr_off;            // byte offset of the compact FP64 right-hand side of the coarsest solve
  const double* ainv;
  int n_coarse;
  int rin;   // linear transfers above the tail: 1 = form the first level's right-hand side from the
             // residual of the level above here, 0 = it is in lv[lt].r already
};

template <typename T, int SM>
__device__ __forceinline__ void mg_tail_body(const TailArgs<T>& A, const SmoothW<T>& W, const SolveState* st,
                                             const VBlock& vb) {
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
    if (A.rin && A.lt > 0 && A.lv[A.lt - 1].lin) {   // the linear restriction of the level above's residual
      const Level<T>& Fa = A.lv[A.lt - 1];
      tail_quads(L, [&](int i, int j, int k, int slot) {
        return restrict_partial(Fa, L, i, j, k, slot, [&](int a, int b, int c) { return Fa.t[lidx(Fa, a, b, c)]; });
      }, [&](int i, int j, int k, T sum) { r[(i + 1) + X * (j + 1) + P * (k + 1)] = sum; });
    } else {
      tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
        r[(i + 1) + X * (j + 1) + P * (k + 1)] = L.r[lidx(L, i, j, k)];
      });
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
    tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      u[b] = r[b] * rdiag(diag_of(L, i, j, k));
    });
    __syncthreads();
    tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      const T s = L.wx * (u[b - 1] + u[b + 1]) + L.wy * (u[b - X] + u[b + X]) + L.wz * (u[b - P] + u[b + P]);
      a[b] = presmooth<SM>(u[b], s, diag_of(L, i, j, k), W, ((i + j + k) & 1) == 0);
    });
    __syncthreads();
    T* rc = S + A.off[m + 1];
    if (L.lin) {
      // residual of every cell into u (no longer needed), then the linear restriction
      tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
        const int b = (i + 1) + X * (j + 1) + P * (k + 1);
        const T nb = nb6(L.wx, a[b - 1], a[b + 1], L.wy, a[b - X], a[b + X], L.wz, a[b - P], a[b + P]);
        u[b] = add_rn(fma_rn(-diag_of(L, i, j, k), a[b], r[b]), nb);
      });
      __syncthreads();
      tail_quads(Cc, [&](int ci, int cj, int ck, int slot) {
        return restrict_partial(L, Cc, ci, cj, ck, slot,
                                [&](int i, int j, int k) { return u[(i + 1) + X * (j + 1) + P * (k + 1)]; });
      }, [&](int ci, int cj, int ck, T sum) { rc[(ci + 1) + CX * (cj + 1) + CP * (ck + 1)] = sum; });
      __syncthreads();
      continue;
    }
    tail_cells(Cc.nx, Cc.ny, Cc.nz, [&](int ci, int cj, int ck) {
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
    });
    __syncthreads();
  }
  // coarsest level: a = A^-1 r with the FP64 dense inverse.  r is first
  // copied into a compact FP64 vector placed after the tail's arrays; then
  // groups of 8 lanes take a row each, every lane a stride-8 set of columns,
  // and the group's partial sums meet by shuffles.
  {
    const int m = A.nl - 1;
    const Level<T>& L = A.lv[m];
    int X, P, NB;
    geom(m, X, P, NB);
    const T* r = S + A.off[m];
    T* a = S + A.off[m] + NB;
    const int n = A.n_coarse;
    double* cr = reinterpret_cast<double*>(smem_raw + A.cr_off);
    tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
      cr[i + L.nx * (j + L.ny * k)] = (double)r[(i + 1) + X * (j + 1) + P * (k + 1)];
    });
    __syncthreads();
    constexpr int G = 8;
    const int lane = tid % G;
    for (int row = tid / G; row < ((n + (TAIL_T / G) - 1) / (TAIL_T / G)) * (TAIL_T / G); row += TAIL_T / G) {
      double sum = 0.0;
      if (row < n) {
        const double* arow = A.ainv + (size_t)row * n;
        for (int c = lane; c < n; c += G) sum += arow[c] * cr[c];
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (row < n && lane == 0) {
        const int i = row % L.nx, j = (row / L.nx) % L.ny, k = row / (L.nx * L.ny);
        a[(i + 1) + X * (j + 1) + P * (k + 1)] = (T)sum;
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
    const Level<T>& Cc = A.lv[m + 1];
    tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {   // t = x + P e (in place)
      T e;
      if (L.lin) {
        e = prolong_lin(L, Cc, i, j, k, [&](int a2, int b2, int c2) { return ec[(a2 + 1) + CX * (b2 + 1) + CP * (c2 + 1)]; });
      } else {
        const int pi = L.cx ? i >> 1 : i, pj = L.cy ? j >> 1 : j, pk = L.cz ? k >> 1 : k;
        e = ec[(pi + 1) + CX * (pj + 1) + CP * (pk + 1)];
      }
      a[(i + 1) + X * (j + 1) + P * (k + 1)] += e;
    });
    __syncthreads();
    tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      const T s = L.wx * (a[b - 1] + a[b + 1]) + L.wy * (a[b - X] + a[b + X]) + L.wz * (a[b - P] + a[b + P]);
      u[b] = relax<SM>(a[b], r[b], s, diag_of(L, i, j, k), W.w1, ((i + j + k) & 1) == 1);
    });
    __syncthreads();
    tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
      const int b = (i + 1) + X * (j + 1) + P * (k + 1);
      const T s = L.wx * (u[b - 1] + u[b + 1]) + L.wy * (u[b - X] + u[b + X]) + L.wz * (u[b - P] + u[b + P]);
      a[b] = relax<SM>(u[b], r[b], s, diag_of(L, i, j, k), W.w2, ((i + j + k) & 1) == 0);
    });
    __syncthreads();
  }
  {
    const Level<T>& L = A.lv[A.lt];
    int X, P, NB;
    geom(A.lt, X, P, NB);
    const T* a = S + A.off[A.lt] + NB;
    tail_cells(L.nx, L.ny, L.nz, [&](int i, int j, int k) {
      L.t[lidx(L, i, j, k)] = a[(i + 1) + X * (j + 1) + P * (k + 1)];
    });
    if (A.lt > 0 && A.lv[A.lt - 1].lin) {   // the level above's prolonged correction
      const Level<T>& Fa = A.lv[A.lt - 1];
      tail_cells(Fa.nx, Fa.ny, Fa.nz, [&](int i, int j, int k) {
        Fa.e[lidx(Fa, i, j, k)] =
            prolong_lin(Fa, L, i, j, k, [&](int a2, int b2, int c2) { return a[(a2 + 1) + X * (b2 + 1) + P * (c2 + 1)]; });
      });
    }
  }
}

template <typename T, int SM>
__global__ void __launch_bounds__(TAIL_T) k_mg_tail(TailArgs<T> A, SmoothW<T> W, const SolveState* st) {
  mg_tail_body<T, SM>(A, W, st, vblock());
}


// ------------------------------------------- CG direction + SpMV --------
// d = z (first iteration) or z + beta d_old, staged per z plane on the tile
// plus a halo of 1 (ring of 4 planes, one barrier per plane, loads one plane
// ahead); q = A d on the owned cells; d.q and alpha = rz / d.q.
// q is formed as a sum of differences w (d_c - d_nb): the CG directions turn
// smooth as the iteration proceeds, and the form D d_c - sum w d_nb would then
// lose about eps * |D d| to cancellation in FP32 -- an error the recursive
// residual never sees, which caps the attainable accuracy of the pressure.
// A Neumann neighbour takes d_c (its term is exactly zero); an outlet
// neighbour is the staged zero ghost (term w d_c).
template <typename T>
__device__ __forceinline__ void cg_dir_q_body(const Level<T>& L, int zc, const T* __restrict__ z, T* d0, T* d1,
                                              T* __restrict__ q, double* partials, SolveState* st, const VBlock& vb) {
  __shared__ T sD[4][XP];
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->converged) return;
  const int i0 = vb.x * TX, j0 = vb.y * TY, k0 = vb.z * zc;
  const int kend = min(L.nz, k0 + zc);
  const int tid = threadIdx.x, tx = tid & (TX - 1), ty = tid / TX;
  const int it = st->iter;
  const T* dold = (it & 1) ? d1 : d0;
  T* dnew = (it & 1) ? d0 : d1;
  const T beta = it == 0 ? T(0) : (T)st->beta;
  const size_t PS = (size_t)L.P * L.ny;
  const PlaneMap mx = plane_map<XX, XY>();
  PosXY<T> pd[2];
  int sd[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int xx = h ? mx.x1 : mx.x0, xy = h ? mx.y1 : mx.y0;
    pd[h] = pos_xy(L, i0 - 1 + xx, j0 - 1 + xy);
    if (h == 1 && !mx.has1) pd[h].ok = false;
    sd[h] = xx + XX * xy;
  }
  T pz[2], pdv[2];
  auto issueD = [&](int k) {
    const bool kin = (unsigned)k < (unsigned)L.nz;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      pz[h] = 0;
      pdv[h] = 0;
      if (kin && pd[h].ok) {
        const size_t c = (size_t)k * PS + pd[h].off;
        pz[h] = z[c];
        if (it != 0) pdv[h] = dold[c];
      }
    }
  };
  auto commitD = [&](int k) {
    T* dst = sD[ring4(k)];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !mx.has1) break;
      dst[sd[h]] = pz[h] + beta * pdv[h];
    }
  };
  const int gi = i0 + tx, gj = j0 + ty;
  const PosXY<T> po = pos_xy(L, gi, gj);
  const int b = (tx + 1) + XX * (ty + 1);
  const bool nxm = gi == 0 && !(L.out_mask & 1), nxp = gi == L.nx - 1 && !(L.out_mask & 2);
  const bool nym = gj == 0 && !(L.out_mask & 4), nyp = gj == L.ny - 1 && !(L.out_mask & 8);
  DotAcc<T> dacc;
  issueD(k0 - 1); commitD(k0 - 1);
  issueD(k0); commitD(k0);
  issueD(k0 + 1);
  for (int k = k0; k < kend; ++k) {
    commitD(k + 1);
    issueD(k + 2);
    __syncthreads();
    if (po.ok) {
      const T* dm = sD[ring4(k - 1)];
      const T* dc = sD[ring4(k)];
      const T* dp = sD[ring4(k + 1)];
      const T dv = dc[b];
      const T xm = nxm ? dv : dc[b - 1], xp = nxp ? dv : dc[b + 1];
      const T ym = nym ? dv : dc[b - XX], yp = nyp ? dv : dc[b + XX];
      const T zm = (k == 0 && !(L.out_mask & 16)) ? dv : dm[b];
      const T zp = (k == L.nz - 1 && !(L.out_mask & 32)) ? dv : dp[b];
      const T qv = L.wx * ((dv - xm) + (dv - xp)) + L.wy * ((dv - ym) + (dv - yp)) + L.wz * ((dv - zm) + (dv - zp));
      const size_t c = (size_t)k * PS + po.off;
      dnew[c] = dv;
      q[c] = qv;
      dacc.add(dv, qv);
    }
  }
  double acc = block_sum<FT>(dacc.value(), sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[2], vals, &last, vb)) {
    double tot[1];
    reduce_partials_sum<FT, 1>(partials, tot, sh, vb.n);
    if (tid == 0) {
      st->dq = tot[0];
      st->alpha = st->rz / tot[0];
      st->ticket[2] = 0u;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(FT) k_cg_dir_q(Level<T> L, int zc, const T* __restrict__ z, T* d0, T* d1,
                                                T* __restrict__ q, double* partials, SolveState* st) {
  cg_dir_q_body<T>(L, zc, z, d0, d1, q, partials, st, vblock());
}


}  // namespace uf
