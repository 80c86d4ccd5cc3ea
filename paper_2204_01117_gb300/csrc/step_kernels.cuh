// Momentum, projection and turbulence kernels of one RANS time step
// (arXiv 2204.01117, Sec. 3).  Each kernel is templated on the field type
// T (float: FP32 bulk arithmetic; double: FP64 throughout); every global
// reduction accumulates in FP64.
//
// Thread mapping: blocks of 32 x 8 threads tile the x-y plane of a lattice
// (a warp reads 32 consecutive x values: 128-byte coalesced rows); blockIdx.z
// walks the z planes.
#pragma once
#include "uf_device.cuh"

namespace uf {

constexpr int BX = 32, BY = 8, NT = BX * BY;

// ------------------------------------------------------------- a0: dt ---
// dt = CFL h / max(|u|,|v|,|w|) over every face (all three lattices, padding
// included: padding is zero).
// max |a_i| over an array (16-byte aligned): 16-byte loads, four of them in
// flight per thread and iteration, then the elements past the last whole
// vector.  The maximum does not depend on the order, so the result is exact.
__device__ __forceinline__ float absmax4(float4 a) { return fmax(fmax(fabsf(a.x), fabsf(a.y)), fmax(fabsf(a.z), fabsf(a.w))); }
__device__ __forceinline__ double absmax4(double2 a) { return fmax(fabs(a.x), fabs(a.y)); }
template <typename T>
__device__ __forceinline__ T absmax_span(const T* __restrict__ a, size_t n, size_t t0, size_t stride, T mt) {
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr size_t W = 16 / sizeof(T);
  const size_t nv = n / W;
  const V* av = reinterpret_cast<const V*>(a);
  size_t q = t0;
  for (; q + 3 * stride < nv; q += 4 * stride) {
    const V a0 = av[q], a1 = av[q + stride], a2 = av[q + 2 * stride], a3 = av[q + 3 * stride];
    mt = fmax(mt, (T)fmax(fmax(absmax4(a0), absmax4(a1)), fmax(absmax4(a2), absmax4(a3))));
  }
  for (; q < nv; q += stride) mt = fmax(mt, (T)absmax4(av[q]));
  for (size_t e = nv * W + t0; e < n; e += stride) mt = fmax(mt, fabs(a[e]));
  return mt;
}

template <typename T>
__device__ __forceinline__ void cfl_dt_body(const T* __restrict__ u, size_t nu, const T* __restrict__ v, size_t nv,
                                            const T* __restrict__ w, size_t nw, double cfl_h, double* partials,
                                            unsigned int* ticket, double* dt_out, T* dtT_out, const VBlock& vb) {
  __shared__ double sh[32];
  __shared__ bool last;
  T mt = 0;   // max in the field type (exact), one conversion per thread
  const size_t stride = (size_t)vb.n * blockDim.x;
  const size_t t0 = vb.lin * (size_t)blockDim.x + threadIdx.x;
  mt = absmax_span(u, nu, t0, stride, mt);
  mt = absmax_span(v, nv, t0, stride, mt);
  mt = absmax_span(w, nw, t0, stride, mt);
  double m = block_max<256>((double)mt, sh);
  const double vals[1] = {m};
  if (publish_partials<1>(partials, ticket, vals, &last, vb)) {
    const double mx = reduce_partials_max<256>(partials, sh, vb.n);
    if (threadIdx.x == 0) {
      if (mx > 0.0) {
        *dt_out = cfl_h / mx;
        *dtT_out = (T)(cfl_h / mx);
      }
      *ticket = 0u;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_cfl_dt(const T* __restrict__ u, size_t nu, const T* __restrict__ v,
                                                size_t nv, const T* __restrict__ w, size_t nw, double cfl_h,
                                                double* partials, unsigned int* ticket, double* dt_out,
                                                T* dtT_out) {
  cfl_dt_body<T>(u, nu, v, nv, w, nw, cfl_h, partials, ticket, dt_out, dtT_out, vblock());
}

// ----------------------------------------------- a1: strain + nu_t ------
// S_ij S_ij at a cell from a staggered field whose boundary faces are all
// stored: diagonal terms from the two faces of the cell, off-diagonal terms
// from central differences of cell-averaged velocities (one-sided at the
// domain edge, zero for an extent of 1).
// uf(a, b, c), vf, wf: the face velocities; from global memory (strain_sq)
// or from staged windows (the fused advection), with the same result: the
// sum of squares is spelled with explicitly rounded operations, the rest
// has nothing the compiler could fuse.
template <typename T, typename UF, typename VF, typename WF>
__device__ __forceinline__ T strain_sq_acc(const StepParams<T>& p, int i, int j, int k, UF uf, VF vf, WF wf) {
  const T ih = p.inv_h;
  auto uc = [&](int a, int b, int c) { return T(0.5) * (uf(a, b, c) + uf(a + 1, b, c)); };
  auto vc = [&](int a, int b, int c) { return T(0.5) * (vf(a, b, c) + vf(a, b + 1, c)); };
  auto wc = [&](int a, int b, int c) { return T(0.5) * (wf(a, b, c) + wf(a, b, c + 1)); };
  const int im = i > 0 ? i - 1 : i, ip = i < p.nx - 1 ? i + 1 : i;
  const int jm = j > 0 ? j - 1 : j, jp = j < p.ny - 1 ? j + 1 : j;
  const int km = k > 0 ? k - 1 : k, kp = k < p.nz - 1 ? k + 1 : k;
  const T sx = (ip > im) ? ih / T(ip - im) : T(0);
  const T sy = (jp > jm) ? ih / T(jp - jm) : T(0);
  const T sz = (kp > km) ? ih / T(kp - km) : T(0);
  const T sxx = (uf(i + 1, j, k) - uf(i, j, k)) * ih;
  const T syy = (vf(i, j + 1, k) - vf(i, j, k)) * ih;
  const T szz = (wf(i, j, k + 1) - wf(i, j, k)) * ih;
  const T du_dy = (uc(i, jp, k) - uc(i, jm, k)) * sy;
  const T du_dz = (uc(i, j, kp) - uc(i, j, km)) * sz;
  const T dv_dx = (vc(ip, j, k) - vc(im, j, k)) * sx;
  const T dv_dz = (vc(i, j, kp) - vc(i, j, km)) * sz;
  const T dw_dx = (wc(ip, j, k) - wc(im, j, k)) * sx;
  const T dw_dy = (wc(i, jp, k) - wc(i, jm, k)) * sy;
  const T sxy = T(0.5) * (du_dy + dv_dx), sxz = T(0.5) * (du_dz + dw_dx), syz = T(0.5) * (dv_dz + dw_dy);
  const T diag = fma_rn(szz, szz, fma_rn(syy, syy, mul_rn(sxx, sxx)));
  const T off = fma_rn(syz, syz, fma_rn(sxz, sxz, mul_rn(sxy, sxy)));
  return fma_rn(T(2), off, diag);
}
template <typename T>
__device__ __forceinline__ T strain_sq(const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
                                       const StepParams<T>& p, int i, int j, int k) {
  return strain_sq_acc<T>(
      p, i, j, k, [&](int a, int b, int c) { return u[idx_u(p, a, b, c)]; },
      [&](int a, int b, int c) { return v[idx_v(p, a, b, c)]; }, [&](int a, int b, int c) { return w[idx_c(p, a, b, c)]; });
}

// k-omega eddy viscosity with the strain limiter on omega (Sec. 3) and the
// von Neumann viscosity limiter h^2/(6 dt) - nu, clamped at zero.
template <typename T>
__device__ __forceinline__ T limited_nut(const StepParams<T>& p, T kv, T omv, T S2, T dt) {
  const T om_t = fmax(omv, p.C_lim * sqrt(S2) / sqrt(p.C_mu * T(0.5)));
  T nut = kv / om_t;
  nut = fmin(nut, p.h * p.h / (T(6) * dt) - p.nu);
  return nut > T(0) ? nut : T(0);
}

template <typename T>
__device__ __forceinline__ void eddy_viscosity_body(const StepParams<T>& p, const T* __restrict__ u,
                                                    const T* __restrict__ v, const T* __restrict__ w,
                                                    const T* __restrict__ kf, const T* __restrict__ om,
                                                    T* __restrict__ nut, const VBlock& vb) {
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y, k = vb.z;
  if (i >= p.nx || j >= p.ny) return;
  const T dt = *p.dtT;
  const size_t c = idx_c(p, i, j, k);
  nut[c] = limited_nut(p, kf[c], om[c], strain_sq(u, v, w, p, i, j, k), dt);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_eddy_viscosity(StepParams<T> p, const T* __restrict__ u,
                                                       const T* __restrict__ v, const T* __restrict__ w,
                                                       const T* __restrict__ kf, const T* __restrict__ om,
                                                       T* __restrict__ nut) {
  eddy_viscosity_body<T>(p, u, v, w, kf, om, nut, vblock());
}


// ------------------------------------------------ a2: MacCormack advection
struct Lattice {
  int Lx, Ly, Lz, P;
};

template <typename T>
__device__ __forceinline__ T lerp_(T a, T b, T t) { return a + t * (b - a); }

// A lattice coordinate is passed as an integer lattice index plus a small
// offset (the displacement, or a half-cell shift): the cell then follows
// from integer arithmetic and the weight t is rounded relative to the
// offset, not to the index.  Formed as one floating-point number x = base +
// off, it would be rounded to eps |x| -- 3e-5 of a cell at index 512 in
// FP32 -- at every backtrace.  Clamped to [0, n - 1] as x would be.
template <typename T>
__device__ __forceinline__ void axis_cell(int base, T off, int n, int& i0, int& i1, T& t) {
  const T fo = floor(off);
  int f = base + (int)fo;
  T tt = off - fo;
  if (f < 0) {                       // below the lattice
    f = 0;
    tt = T(0);
  } else if (f >= n - 1) {           // at or beyond the last point
    f = n >= 2 ? n - 2 : 0;
    tt = n >= 2 ? T(1) : T(0);
  }
  i0 = f;
  i1 = min(f + 1, n - 1);
  t = tt;
}
// base + off inside [0, n - 1] (the sample is not clamped along the axis)
template <typename T>
__device__ __forceinline__ bool axis_inside(int base, T off, int n) {
  const T fo = floor(off);
  const int f = base + (int)fo;
  return f >= 0 && (f < n - 1 || (f == n - 1 && off == fo));
}

// Trilinear interpolation of the 8 corner values f[a + 2b + 4c] with
// weights (ta, tb, tc), as nested lerps along x, then y, then z; optionally
// the range of the 8 values.  Every semi-Lagrangian sample of the step goes
// through this one expression, whatever memory the corners come from.
template <typename T, bool RANGE>
__device__ __forceinline__ T trilerp(const T (&f)[8], T ta, T tb, T tc, T* mn, T* mx) {
  if (RANGE) {
    *mn = fmin(fmin(fmin(f[0], f[1]), fmin(f[2], f[3])), fmin(fmin(f[4], f[5]), fmin(f[6], f[7])));
    *mx = fmax(fmax(fmax(f[0], f[1]), fmax(f[2], f[3])), fmax(fmax(f[4], f[5]), fmax(f[6], f[7])));
  }
  const T x00 = lerp_(f[0], f[1], ta), x10 = lerp_(f[2], f[3], ta);
  const T x01 = lerp_(f[4], f[5], ta), x11 = lerp_(f[6], f[7], ta);
  return lerp_(lerp_(x00, x10, tb), lerp_(x01, x11, tb), tc);
}

// The 8 corners of a sample from global memory.
template <typename T>
__device__ __forceinline__ void corners_global(const T* __restrict__ F, Lattice L, int i0, int i1, int j0, int j1,
                                               int k0, int k1, T (&f)[8]) {
  const size_t r00 = (size_t)L.P * ((size_t)j0 + (size_t)L.Ly * k0);
  const size_t r10 = (size_t)L.P * ((size_t)j1 + (size_t)L.Ly * k0);
  const size_t r01 = (size_t)L.P * ((size_t)j0 + (size_t)L.Ly * k1);
  const size_t r11 = (size_t)L.P * ((size_t)j1 + (size_t)L.Ly * k1);
  f[0] = F[r00 + i0]; f[1] = F[r00 + i1]; f[2] = F[r10 + i0]; f[3] = F[r10 + i1];
  f[4] = F[r01 + i0]; f[5] = F[r01 + i1]; f[6] = F[r11 + i0]; f[7] = F[r11 + i1];
}

// Trilinear sample at lattice coordinates (ia + oa, ib + ob, ic + oc),
// clamped to the lattice; optionally the range of the 8 values used.
template <typename T, bool RANGE>
__device__ __forceinline__ T sample(const T* __restrict__ F, Lattice L, int ia, T oa, int ib, T ob, int ic, T oc,
                                    T* mn = nullptr, T* mx = nullptr) {
  int i0, i1, j0, j1, k0, k1;
  T ta, tb, tc;
  axis_cell(ia, oa, L.Lx, i0, i1, ta);
  axis_cell(ib, ob, L.Ly, j0, j1, tb);
  axis_cell(ic, oc, L.Lz, k0, k1, tc);
  T f[8];
  corners_global(F, L, i0, i1, j0, j1, k0, k1, f);
  return trilerp<T, RANGE>(f, ta, tb, tc, mn, mx);
}

template <typename T>
struct AdvectArgs {
  const T* u;
  const T* v;
  const T* w;         // velocity of time level n (all faces stored)
  T* uh;
  T* vh;
  T* wh;              // forward-step fields (all lattice points)
  T* ut;
  T* vt;
  T* wt;              // MacCormack result (interior faces only)
  Lattice Lu, Lv, Lw;
  int nx, ny, nz;
  const T* dtT;
  T inv_h;
  // fused advection only: with nut set, it also forms the eddy viscosity of
  // the cells (a1, from the time-level-n velocity it stages) from kf, om
  T* nut;
  const T* kf;
  const T* om;
  StepParams<T> sp;
};

// Displacement in lattice units (dt/h * velocity) at a lattice point of
// component q, every component sampled from time level n.
template <typename T>
__device__ __forceinline__ void displacement(const AdvectArgs<T>& A, int q, int i, int j, int k, T s, T d[3]) {
  if (q == 0) {   // u point (i, j+1/2, k+1/2)
    d[0] = s * A.u[(size_t)i + (size_t)A.Lu.P * ((size_t)j + (size_t)A.Lu.Ly * k)];
    d[1] = s * sample<T, false>(A.v, A.Lv, i, T(-0.5), j, T(0.5), k, T(0));
    d[2] = s * sample<T, false>(A.w, A.Lw, i, T(-0.5), j, T(0), k, T(0.5));
  } else if (q == 1) {   // v point (i+1/2, j, k+1/2)
    d[0] = s * sample<T, false>(A.u, A.Lu, i, T(0.5), j, T(-0.5), k, T(0));
    d[1] = s * A.v[(size_t)i + (size_t)A.Lv.P * ((size_t)j + (size_t)A.Lv.Ly * k)];
    d[2] = s * sample<T, false>(A.w, A.Lw, i, T(0), j, T(-0.5), k, T(0.5));
  } else {   // w point (i+1/2, j+1/2, k)
    d[0] = s * sample<T, false>(A.u, A.Lu, i, T(0.5), j, T(0), k, T(-0.5));
    d[1] = s * sample<T, false>(A.v, A.Lv, i, T(0), j, T(0.5), k, T(-0.5));
    d[2] = s * A.w[(size_t)i + (size_t)A.Lw.P * ((size_t)j + (size_t)A.Lw.Ly * k)];
  }
}

// blockIdx.z enumerates the planes of u (nz of them), then v (nz), then w (nz+1).
__device__ __forceinline__ void plane_of(int bz, int nz, int& q, int& k) {
  if (bz < nz) { q = 0; k = bz; }
  else if (bz < 2 * nz) { q = 1; k = bz - nz; }
  else { q = 2; k = bz - 2 * nz; }
}

// Forward semi-Lagrangian step phi^ = phi(x - dt u(x)) at every lattice point.
template <typename T>
__device__ __forceinline__ void advect_forward_body(const AdvectArgs<T>& A, const VBlock& vb) {
  int q, k;
  plane_of(vb.z, A.nz, q, k);
  const Lattice L = q == 0 ? A.Lu : (q == 1 ? A.Lv : A.Lw);
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y;
  if (i >= L.Lx || j >= L.Ly) return;
  const T s = *A.dtT * A.inv_h;
  const T* F = q == 0 ? A.u : (q == 1 ? A.v : A.w);
  T* Fh = q == 0 ? A.uh : (q == 1 ? A.vh : A.wh);
  T d[3];
  displacement(A, q, i, j, k, s, d);
  Fh[(size_t)i + (size_t)L.P * ((size_t)j + (size_t)L.Ly * k)] =
      sample<T, false>(F, L, i, -d[0], j, -d[1], k, -d[2]);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_advect_forward(AdvectArgs<T> A) {
  advect_forward_body<T>(A, vblock());
}


// Backward step, MacCormack correction and clamp on interior faces:
// phi* = phi^ + (phi - phi^(x + dt u(x)))/2, clamped to the range of the 8
// values of the forward sample (Selle et al. 2008).
template <typename T>
__device__ __forceinline__ void advect_backward_body(const AdvectArgs<T>& A, const VBlock& vb) {
  int q, k;
  plane_of(vb.z, A.nz, q, k);
  const Lattice L = q == 0 ? A.Lu : (q == 1 ? A.Lv : A.Lw);
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y;
  if (i >= L.Lx || j >= L.Ly) return;
  const bool interior = q == 0 ? (i > 0 && i < A.nx) : (q == 1 ? (j > 0 && j < A.ny) : (k > 0 && k < A.nz));
  if (!interior) return;
  const T s = *A.dtT * A.inv_h;
  const T* F = q == 0 ? A.u : (q == 1 ? A.v : A.w);
  const T* Fh = q == 0 ? A.uh : (q == 1 ? A.vh : A.wh);
  T* Ft = q == 0 ? A.ut : (q == 1 ? A.vt : A.wt);
  T d[3];
  displacement(A, q, i, j, k, s, d);
  T mn, mx;
  const T fwd = sample<T, true>(F, L, i, -d[0], j, -d[1], k, -d[2], &mn, &mx);
  const T bwd = sample<T, false>(Fh, L, i, d[0], j, d[1], k, d[2]);
  const size_t id = (size_t)i + (size_t)L.P * ((size_t)j + (size_t)L.Ly * k);
  T r = fwd + T(0.5) * (F[id] - bwd);
  Ft[id] = fmin(fmax(r, mn), mx);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_advect_backward(AdvectArgs<T> A) {
  advect_backward_body<T>(A, vblock());
}


// ------------------------------------------------- a3: diffusion ---------
// Explicit (nu + nu_t) lap(u) on each face lattice; nu_t at a face is the
// mean of its two cells.  Input boundary faces come from the BC rules, the
// ghosts beyond tangential sides from the side's BC.  Writes interior faces.
template <typename T>
__device__ __forceinline__ void diffuse_body(const StepParams<T>& p, const T* __restrict__ ui,
                                             const T* __restrict__ vi, const T* __restrict__ wi,
                                             const T* __restrict__ nut, T* __restrict__ uo, T* __restrict__ vo,
                                             T* __restrict__ wo, const VBlock& vb) {
  int q, k;
  plane_of(vb.z, p.nz, q, k);
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y;
  const T dt = *p.dtT;
  const T c = dt * p.inv_h * p.inv_h;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (q == 0) {
    if (i < 1 || i >= nx || j >= ny) return;
    const T x0 = ui[idx_u(p, i, j, k)];
    const T inflow = p.prof[k] * p.dirx;
    const T xm = u_face(ui, p, i - 1, j, k), xp = u_face(ui, p, i + 1, j, k);
    const T ym = j > 0 ? ui[idx_u(p, i, j - 1, k)] : tangential_ghost(p.side[2], x0, inflow);
    const T yp = j < ny - 1 ? ui[idx_u(p, i, j + 1, k)] : tangential_ghost(p.side[3], x0, inflow);
    const T zm = k > 0 ? ui[idx_u(p, i, j, k - 1)] : tangential_ghost(p.side[4], x0, T(0));
    const T zp = k < nz - 1 ? ui[idx_u(p, i, j, k + 1)] : tangential_ghost(p.side[5], x0, T(0));
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (nut[idx_c(p, i - 1, j, k)] + nut[idx_c(p, i, j, k)]);
    uo[idx_u(p, i, j, k)] = x0 + c * (p.nu + nf) * lap;
  } else if (q == 1) {
    if (i >= nx || j < 1 || j >= ny) return;
    const T x0 = vi[idx_v(p, i, j, k)];
    const T inflow = p.prof[k] * p.diry;
    const T xm = i > 0 ? vi[idx_v(p, i - 1, j, k)] : tangential_ghost(p.side[0], x0, inflow);
    const T xp = i < nx - 1 ? vi[idx_v(p, i + 1, j, k)] : tangential_ghost(p.side[1], x0, inflow);
    const T ym = v_face(vi, p, i, j - 1, k), yp = v_face(vi, p, i, j + 1, k);
    const T zm = k > 0 ? vi[idx_v(p, i, j, k - 1)] : tangential_ghost(p.side[4], x0, T(0));
    const T zp = k < nz - 1 ? vi[idx_v(p, i, j, k + 1)] : tangential_ghost(p.side[5], x0, T(0));
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (nut[idx_c(p, i, j - 1, k)] + nut[idx_c(p, i, j, k)]);
    vo[idx_v(p, i, j, k)] = x0 + c * (p.nu + nf) * lap;
  } else {
    if (i >= nx || j >= ny || k < 1 || k >= nz) return;
    const T x0 = wi[idx_c(p, i, j, k)];
    const T xm = i > 0 ? wi[idx_c(p, i - 1, j, k)] : tangential_ghost(p.side[0], x0, T(0));
    const T xp = i < nx - 1 ? wi[idx_c(p, i + 1, j, k)] : tangential_ghost(p.side[1], x0, T(0));
    const T ym = j > 0 ? wi[idx_c(p, i, j - 1, k)] : tangential_ghost(p.side[2], x0, T(0));
    const T yp = j < ny - 1 ? wi[idx_c(p, i, j + 1, k)] : tangential_ghost(p.side[3], x0, T(0));
    const T zm = w_face(wi, p, i, j, k - 1), zp = w_face(wi, p, i, j, k + 1);
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (nut[idx_c(p, i, j, k - 1)] + nut[idx_c(p, i, j, k)]);
    wo[idx_c(p, i, j, k)] = x0 + c * (p.nu + nf) * lap;
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_diffuse(StepParams<T> p, const T* __restrict__ ui, const T* __restrict__ vi,
                                                const T* __restrict__ wi, const T* __restrict__ nut,
                                                T* __restrict__ uo, T* __restrict__ vo, T* __restrict__ wo) {
  diffuse_body<T>(p, ui, vi, wi, nut, uo, vo, wo, vblock());
}


// ---------------------------------------------- a4 + a5: drag and BCs ----
// Forward-Euler porosity drag u <- max(0, 1 - dt c U) u (Sec. 3) with c the
// mean drag coefficient of the two adjacent cells and U the speed from the
// face value and 4-point averages of the other two components.
template <typename T>
__device__ __forceinline__ T drag_u(const StepParams<T>& p, const T* __restrict__ u, const T* __restrict__ v,
                                    const T* __restrict__ w, const T* __restrict__ cc, T dt, int i, int j, int k) {
  const T q = u[idx_u(p, i, j, k)];
  const T vb = T(0.25) * (v_face(v, p, i - 1, j, k) + v_face(v, p, i, j, k) + v_face(v, p, i - 1, j + 1, k) +
                          v_face(v, p, i, j + 1, k));
  const T wb = T(0.25) * (w_face(w, p, i - 1, j, k) + w_face(w, p, i, j, k) + w_face(w, p, i - 1, j, k + 1) +
                          w_face(w, p, i, j, k + 1));
  const T sp = sqrt(q * q + vb * vb + wb * wb);
  const T cf = T(0.5) * (cc[idx_c(p, i - 1, j, k)] + cc[idx_c(p, i, j, k)]);
  return fmax(T(0), T(1) - dt * cf * sp) * q;
}
template <typename T>
__device__ __forceinline__ T drag_v(const StepParams<T>& p, const T* __restrict__ u, const T* __restrict__ v,
                                    const T* __restrict__ w, const T* __restrict__ cc, T dt, int i, int j, int k) {
  const T q = v[idx_v(p, i, j, k)];
  const T ub = T(0.25) * (u_face(u, p, i, j - 1, k) + u_face(u, p, i + 1, j - 1, k) + u_face(u, p, i, j, k) +
                          u_face(u, p, i + 1, j, k));
  const T wb = T(0.25) * (w_face(w, p, i, j - 1, k) + w_face(w, p, i, j, k) + w_face(w, p, i, j - 1, k + 1) +
                          w_face(w, p, i, j, k + 1));
  const T sp = sqrt(ub * ub + q * q + wb * wb);
  const T cf = T(0.5) * (cc[idx_c(p, i, j - 1, k)] + cc[idx_c(p, i, j, k)]);
  return fmax(T(0), T(1) - dt * cf * sp) * q;
}
template <typename T>
__device__ __forceinline__ T drag_w(const StepParams<T>& p, const T* __restrict__ u, const T* __restrict__ v,
                                    const T* __restrict__ w, const T* __restrict__ cc, T dt, int i, int j, int k) {
  const T q = w[idx_c(p, i, j, k)];
  const T ub = T(0.25) * (u_face(u, p, i, j, k - 1) + u_face(u, p, i + 1, j, k - 1) + u_face(u, p, i, j, k) +
                          u_face(u, p, i + 1, j, k));
  const T vb = T(0.25) * (v_face(v, p, i, j, k - 1) + v_face(v, p, i, j + 1, k - 1) + v_face(v, p, i, j, k) +
                          v_face(v, p, i, j + 1, k));
  const T sp = sqrt(ub * ub + vb * vb + q * q);
  const T cf = T(0.5) * (cc[idx_c(p, i, j, k - 1)] + cc[idx_c(p, i, j, k)]);
  return fmax(T(0), T(1) - dt * cf * sp) * q;
}

// Writes every face of the output: drag on interior faces; on boundary faces
// the BC value, where an outlet face copies its (dragged) interior neighbour.
template <typename T>
__device__ __forceinline__ void drag_bc_body(const StepParams<T>& p, const T* __restrict__ ui,
                                             const T* __restrict__ vi, const T* __restrict__ wi,
                                             const T* __restrict__ cc, T* __restrict__ uo, T* __restrict__ vo,
                                             T* __restrict__ wo, const VBlock& vb) {
  int q, k;
  plane_of(vb.z, p.nz, q, k);
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y;
  const T dt = *p.dtT;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (q == 0) {
    if (i > nx || j >= ny) return;
    T r;
    if (i == 0) r = normal_face(p.side[0], drag_u(p, ui, vi, wi, cc, dt, 1, j, k), p.prof[k] * p.dirx);
    else if (i == nx) r = normal_face(p.side[1], drag_u(p, ui, vi, wi, cc, dt, nx - 1, j, k), p.prof[k] * p.dirx);
    else r = drag_u(p, ui, vi, wi, cc, dt, i, j, k);
    uo[idx_u(p, i, j, k)] = r;
  } else if (q == 1) {
    if (i >= nx || j > ny) return;
    T r;
    if (j == 0) r = normal_face(p.side[2], drag_v(p, ui, vi, wi, cc, dt, i, 1, k), p.prof[k] * p.diry);
    else if (j == ny) r = normal_face(p.side[3], drag_v(p, ui, vi, wi, cc, dt, i, ny - 1, k), p.prof[k] * p.diry);
    else r = drag_v(p, ui, vi, wi, cc, dt, i, j, k);
    vo[idx_v(p, i, j, k)] = r;
  } else {
    if (i >= nx || j >= ny) return;
    wo[idx_c(p, i, j, k)] = (k == 0 || k == nz) ? T(0) : drag_w(p, ui, vi, wi, cc, dt, i, j, k);
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_drag_bc(StepParams<T> p, const T* __restrict__ ui, const T* __restrict__ vi,
                                                const T* __restrict__ wi, const T* __restrict__ cc,
                                                T* __restrict__ uo, T* __restrict__ vo, T* __restrict__ wo) {
  drag_bc_body<T>(p, ui, vi, wi, cc, uo, vo, wo, vblock());
}


// ------------------------------------------- a6: pressure right-hand side
// b = -(rho h / dt) (u(i+1)-u(i) + v(j+1)-v(j) + w(k+1)-w(k)), the
// right-hand side of A p = b for the integer 7-point operator A.
template <typename T>
__device__ __forceinline__ T cell_flux(const StepParams<T>& p, const T* __restrict__ u, const T* __restrict__ v,
                                       const T* __restrict__ w, int i, int j, int k) {
  return u[idx_u(p, i + 1, j, k)] - u[idx_u(p, i, j, k)] + v[idx_v(p, i, j + 1, k)] - v[idx_v(p, i, j, k)] +
         w[idx_c(p, i, j, k + 1)] - w[idx_c(p, i, j, k)];
}

// Solver scalars shared by the pressure-solve kernels (device memory).
struct SolveState {
  double bb, rr, rz, dq, alpha, beta, rr0;
  double tol2;   // stop rule 0: tol^2 (rr <= tol2 bb); rule 1: tol (rz <= tol2 bb)
  int iter, converged, status, max_iter, sticky;
  int rule;      // 0: ||r|| <= tol ||b||;  1: r.z <= tol ||b||^2 (App. A.3)
  unsigned int ticket[4];
  long long total_iters;   // CG iterations since the grid was created
};

// b = -(rho h / dt) (sum of the face fluxes of the cell), the right-hand
// side of A p = b on the integer stencil, and ||b||^2 for the CG stop rule.
template <typename T>
__device__ __forceinline__ void pressure_rhs_body(const StepParams<T>& p, const T* __restrict__ u,
                                                  const T* __restrict__ v, const T* __restrict__ w, T* __restrict__ b,
                                                  int zc, double* partials, SolveState* st, const VBlock& vb) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y;
  const int z0 = vb.z * zc, z1 = min(p.nz, z0 + zc);
  double acc = 0.0;
  DotAcc<T> dacc;
  if (i < p.nx && j < p.ny) {
    const T sc = -p.rho * p.h / *p.dtT;
    for (int k = z0; k < z1; ++k) {
      const T bv = sc * cell_flux(p, u, v, w, i, j, k);
      b[idx_c(p, i, j, k)] = bv;
      dacc.add(bv, bv);
    }
  }
  acc += dacc.value();
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, &st->ticket[0], vals, &last, vb)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh, vb.n);
    if (thread_linear_id() == 0) {
      st->bb = tot[0];
      st->iter = 0;
      st->converged = 0;
      st->status = DEV_OK;
      st->ticket[0] = 0u;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_pressure_rhs(StepParams<T> p, const T* __restrict__ u, const T* __restrict__ v,
                                                     const T* __restrict__ w, T* __restrict__ b, int zc,
                                                     double* partials, SolveState* st) {
  pressure_rhs_body<T>(p, u, v, w, b, zc, partials, st, vblock());
}

// After the pressure solve.  The solve works on the correction delta to the
// guess g = 2 p^n - p^{n-1} (the pressure extrapolated in time, see
// cg_init_body), which is small; this kernel forms p^{n+1} = g + delta in
// the pressure store (PStore), the next guess 2 p^{n+1} - p^n in gs, and
// leaves p^{n+1} rounded to the grid precision in delta, the copy the field
// accessors read.  A zero right-hand side gives p = 0.
template <typename T>
__device__ __forceinline__ void pressure_commit_body(const StepParams<T>& p, T* __restrict__ delta,
                                                     PStore<T>* __restrict__ pn, PStore<T>* __restrict__ gs,
                                                     const SolveState* st, const VBlock& vb) {
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y, k = vb.z;
  if (i >= p.nx || j >= p.ny) return;
  const size_t c = idx_c(p, i, j, k);
  PStore<T> v, g;
  ps_commit(gs[c], pn[c], delta[c], st->bb == 0.0, &v, &g);
  pn[c] = v;
  gs[c] = g;
  delta[c] = (T)ps_value(v);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_pressure_commit(StepParams<T> p, T* __restrict__ delta,
                                                        PStore<T>* __restrict__ pn, PStore<T>* __restrict__ gs,
                                                        const SolveState* st) {
  pressure_commit_body<T>(p, delta, pn, gs, st, vblock());
}

// A pressure set from outside (grid precision, in pg) becomes the stored
// state with no history: pn = gs = pg.  to_store = 0 rounds pn back into pg.
template <typename T>
__global__ void k_pressure_sync(T* __restrict__ pg, PStore<T>* __restrict__ pn, PStore<T>* __restrict__ gs, size_t n,
                                int to_store) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  if (to_store) {
    const PStore<T> v = ps_from(pg[q]);
    pn[q] = v;
    gs[q] = v;
  } else {
    pg[q] = (T)ps_value(pn[q]);
  }
}


// --------------------------------------------------------- a8: projection
// u -= dt/(rho h) (p(c+) - p(c-)) on interior faces and on faces of outlet
// sides (outer neighbour: the p = 0 ghost cell).  In place.  The difference
// is taken on the pressure store (PStore).
template <typename T>
__device__ __forceinline__ void project_body(const StepParams<T>& p, const PStore<T>* __restrict__ pr,
                                             T* __restrict__ u, T* __restrict__ v, T* __restrict__ w,
                                             const VBlock& vb) {
  int q, k;
  plane_of(vb.z, p.nz, q, k);
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y;
  const T g = *p.dtT / (p.rho * p.h);
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (q == 0) {
    if (i > nx || j >= ny) return;
    T dp;
    if (i == 0) { if (p.side[0] != OUTFLOW) return; dp = (T)ps_value(pr[idx_c(p, 0, j, k)]); }
    else if (i == nx) { if (p.side[1] != OUTFLOW) return; dp = -(T)ps_value(pr[idx_c(p, nx - 1, j, k)]); }
    else dp = (T)ps_diff(pr[idx_c(p, i, j, k)], pr[idx_c(p, i - 1, j, k)]);
    u[idx_u(p, i, j, k)] -= g * dp;
  } else if (q == 1) {
    if (i >= nx || j > ny) return;
    T dp;
    if (j == 0) { if (p.side[2] != OUTFLOW) return; dp = (T)ps_value(pr[idx_c(p, i, 0, k)]); }
    else if (j == ny) { if (p.side[3] != OUTFLOW) return; dp = -(T)ps_value(pr[idx_c(p, i, ny - 1, k)]); }
    else dp = (T)ps_diff(pr[idx_c(p, i, j, k)], pr[idx_c(p, i, j - 1, k)]);
    v[idx_v(p, i, j, k)] -= g * dp;
  } else {
    if (i >= nx || j >= ny || k < 1 || k >= nz) return;
    w[idx_c(p, i, j, k)] -= g * (T)ps_diff(pr[idx_c(p, i, j, k)], pr[idx_c(p, i, j, k - 1)]);
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_project(StepParams<T> p, const PStore<T>* __restrict__ pr, T* __restrict__ u,
                                                T* __restrict__ v, T* __restrict__ w) {
  project_body<T>(p, pr, u, v, w, vblock());
}

// The same projection with one thread per lattice column (i, j) of plane k
// for the faces i, j and k of cell (i, j, k): the x, y and z faces that the
// per-face form (project_body, blockIdx.z over the three components) gives
// to three threads, with the same expression per face.  Grid (nx + 1, ny + 1)
// columns by nz planes.
template <typename T>
__global__ void __launch_bounds__(NT) k_project_cells(StepParams<T> p, const PStore<T>* __restrict__ pr,
                                                      T* __restrict__ u, T* __restrict__ v, T* __restrict__ w) {
  const VBlock vb = vblock();
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y, k = vb.z;
  const T g = *p.dtT / (p.rho * p.h);
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (i <= nx && j < ny) {   // x face (i, j, k)
    bool on = true;
    T dp = 0;
    if (i == 0) { on = p.side[0] == OUTFLOW; if (on) dp = (T)ps_value(pr[idx_c(p, 0, j, k)]); }
    else if (i == nx) { on = p.side[1] == OUTFLOW; if (on) dp = -(T)ps_value(pr[idx_c(p, nx - 1, j, k)]); }
    else dp = (T)ps_diff(pr[idx_c(p, i, j, k)], pr[idx_c(p, i - 1, j, k)]);
    if (on) u[idx_u(p, i, j, k)] -= g * dp;
  }
  if (i < nx && j <= ny) {   // y face (i, j, k)
    bool on = true;
    T dp = 0;
    if (j == 0) { on = p.side[2] == OUTFLOW; if (on) dp = (T)ps_value(pr[idx_c(p, i, 0, k)]); }
    else if (j == ny) { on = p.side[3] == OUTFLOW; if (on) dp = -(T)ps_value(pr[idx_c(p, i, ny - 1, k)]); }
    else dp = (T)ps_diff(pr[idx_c(p, i, j, k)], pr[idx_c(p, i, j - 1, k)]);
    if (on) v[idx_v(p, i, j, k)] -= g * dp;
  }
  if (i < nx && j < ny && k >= 1)   // z face (i, j, k); k < nz here
    w[idx_c(p, i, j, k)] -= g * (T)ps_diff(pr[idx_c(p, i, j, k)], pr[idx_c(p, i, j, k - 1)]);
}


// ------------------------------------------------------- a9: k-omega -----
// Forward Euler for k and omega after the projection (Sec. 3): first-order
// upwind advection with the cell-centre velocity, 7-point diffusion with
// (nu + sigma* nu_t) and (nu + sigma nu_t), sources P_k - C_mu k omega and
// 2 alpha |S|^2 - beta omega^2 with P_k = 2 nu_t |S|^2, |S|^2 = S_ij S_ij of
// the projected velocity.  Ghosts: inlet values on inlet sides, zero
// gradient elsewhere.  Floors k_min, omega_min.
template <typename T>
__device__ __forceinline__ void turbulence_body(const StepParams<T>& p, const T* __restrict__ u,
                                                const T* __restrict__ v, const T* __restrict__ w,
                                                const T* __restrict__ ki, const T* __restrict__ oi,
                                                T* __restrict__ ko, T* __restrict__ oo, const VBlock& vb) {
  const int i = vb.x * BX + threadIdx.x, j = vb.y * BY + threadIdx.y, k = vb.z;
  if (i >= p.nx || j >= p.ny) return;
  const T dt = *p.dtT;
  const size_t c = idx_c(p, i, j, k);
  const T kc = ki[c], oc = oi[c];
  const T S2 = strain_sq(u, v, w, p, i, j, k);
  const T nut = limited_nut(p, kc, oc, S2, dt);
  const T vel[3] = {T(0.5) * (u[idx_u(p, i, j, k)] + u[idx_u(p, i + 1, j, k)]),
                    T(0.5) * (v[idx_v(p, i, j, k)] + v[idx_v(p, i, j + 1, k)]),
                    T(0.5) * (w[idx_c(p, i, j, k)] + w[idx_c(p, i, j, k + 1)])};
  const int pos[3] = {i, j, k}, ext[3] = {p.nx, p.ny, p.nz};
  T adv_k = 0, adv_o = 0, lap_k = T(-6) * kc, lap_o = T(-6) * oc;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const size_t stride = ax == 0 ? 1 : (ax == 1 ? (size_t)p.Pc : (size_t)p.Pc * p.ny);
    const bool has_m = pos[ax] > 0, has_p = pos[ax] < ext[ax] - 1;
    const int sm = p.side[2 * ax], sp = p.side[2 * ax + 1];
    const T km = has_m ? ki[c - stride] : (sm == INFLOW ? p.k_in : kc);
    const T kp = has_p ? ki[c + stride] : (sp == INFLOW ? p.k_in : kc);
    const T om_m = has_m ? oi[c - stride] : (sm == INFLOW ? p.om_in : oc);
    const T om_p = has_p ? oi[c + stride] : (sp == INFLOW ? p.om_in : oc);
    lap_k += km + kp;
    lap_o += om_m + om_p;
    if (vel[ax] > T(0)) {
      adv_k += vel[ax] * (kc - km) * p.inv_h;
      adv_o += vel[ax] * (oc - om_m) * p.inv_h;
    } else if (vel[ax] < T(0)) {
      adv_k += vel[ax] * (kp - kc) * p.inv_h;
      adv_o += vel[ax] * (om_p - oc) * p.inv_h;
    }
  }
  const T ih2 = p.inv_h * p.inv_h;
  const T Pk = T(2) * nut * S2;
  const T rk = -adv_k + Pk - p.C_mu * kc * oc + (p.nu + p.sigma_star * nut) * lap_k * ih2;
  const T ro = -adv_o + T(2) * p.alpha * S2 - p.beta * oc * oc + (p.nu + p.sigma * nut) * lap_o * ih2;
  ko[c] = fmax(kc + dt * rk, p.k_min);
  oo[c] = fmax(oc + dt * ro, p.om_min);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_turbulence(StepParams<T> p, const T* __restrict__ u, const T* __restrict__ v,
                                                   const T* __restrict__ w, const T* __restrict__ ki,
                                                   const T* __restrict__ oi, T* __restrict__ ko, T* __restrict__ oo) {
  turbulence_body<T>(p, u, v, w, ki, oi, ko, oo, vblock());
}


// ------------------------------------------------------ a10: objective ---
// Sum over cells whose centre height lies in [z_lo, z_hi] of
// max(|u_c| - u_hi, 0)^2 + max(u_lo - |u_c|, 0)^2, cell-centre velocity from
// face averages; FP64 accumulation.
template <typename T>
__global__ void __launch_bounds__(NT) k_objective(StepParams<T> p, const T* __restrict__ u, const T* __restrict__ v,
                                                  const T* __restrict__ w, int k_lo, int k_hi, int zc, double u_hi,
                                                  double u_lo, double* partials, unsigned int* ticket, double* out) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int z0 = k_lo + blockIdx.z * zc, z1 = min(k_hi + 1, z0 + zc);
  double acc = 0.0;
  if (i < p.nx && j < p.ny) {
    for (int k = z0; k < z1; ++k) {
      const double uc = 0.5 * ((double)u[idx_u(p, i, j, k)] + (double)u[idx_u(p, i + 1, j, k)]);
      const double vc = 0.5 * ((double)v[idx_v(p, i, j, k)] + (double)v[idx_v(p, i, j + 1, k)]);
      const double wc = 0.5 * ((double)w[idx_c(p, i, j, k)] + (double)w[idx_c(p, i, j, k + 1)]);
      const double s = sqrt(uc * uc + vc * vc + wc * wc);
      const double hi = fmax(s - u_hi, 0.0), lo = fmax(u_lo - s, 0.0);
      acc += hi * hi + lo * lo;
    }
  }
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, ticket, vals, &last)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh);
    if (thread_linear_id() == 0) {
      *out = tot[0];
      *ticket = 0u;
    }
  }
}

// Sum of the cell-centre speed |u_c| over the cell box [i0, i1] x [j0, j1] x
// [k0, k1] (one target region of the region-average objective of Sec. 6,
// "Avoiding Heat Pockets"); deterministic FP64 reduction into *out.
template <typename T>
__global__ void __launch_bounds__(NT) k_box_speed(StepParams<T> p, const T* __restrict__ u, const T* __restrict__ v,
                                                  const T* __restrict__ w, int i0, int i1, int j0, int j1, int k0,
                                                  int k1, int zc, double* partials, unsigned int* ticket,
                                                  double* out) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int i = i0 + blockIdx.x * BX + threadIdx.x, j = j0 + blockIdx.y * BY + threadIdx.y;
  const int z0 = k0 + blockIdx.z * zc, z1 = min(k1 + 1, z0 + zc);
  double acc = 0.0;
  if (i <= i1 && j <= j1) {
    for (int k = z0; k < z1; ++k) {
      const double uc = 0.5 * ((double)u[idx_u(p, i, j, k)] + (double)u[idx_u(p, i + 1, j, k)]);
      const double vc = 0.5 * ((double)v[idx_v(p, i, j, k)] + (double)v[idx_v(p, i, j + 1, k)]);
      const double wc = 0.5 * ((double)w[idx_c(p, i, j, k)] + (double)w[idx_c(p, i, j, k + 1)]);
      acc += sqrt(uc * uc + vc * vc + wc * wc);
    }
  }
  acc = block_sum<NT>(acc, sh);
  const double vals[1] = {acc};
  if (publish_partials<1>(partials, ticket, vals, &last)) {
    double tot[1];
    reduce_partials_sum<NT, 1>(partials, tot, sh);
    if (thread_linear_id() == 0) {
      *out = tot[0];
      *ticket = 0u;
    }
  }
}

// ---------------------------------------------------- diagnostics --------
// Partial sums of (h div u)^2 and |u_c|^2 over all cells.
template <typename T>
__global__ void __launch_bounds__(NT) k_divergence(StepParams<T> p, const T* __restrict__ u, const T* __restrict__ v,
                                                   const T* __restrict__ w, int zc, double* partials,
                                                   unsigned int* ticket, double* out2) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int z0 = blockIdx.z * zc, z1 = min(p.nz, z0 + zc);
  double a = 0.0, b = 0.0;
  if (i < p.nx && j < p.ny) {
    for (int k = z0; k < z1; ++k) {
      const double f = (double)cell_flux(p, u, v, w, i, j, k);
      a += f * f;
      const double uc = 0.5 * ((double)u[idx_u(p, i, j, k)] + (double)u[idx_u(p, i + 1, j, k)]);
      const double vc = 0.5 * ((double)v[idx_v(p, i, j, k)] + (double)v[idx_v(p, i, j + 1, k)]);
      const double wc = 0.5 * ((double)w[idx_c(p, i, j, k)] + (double)w[idx_c(p, i, j, k + 1)]);
      b += uc * uc + vc * vc + wc * wc;
    }
  }
  a = block_sum<NT>(a, sh);
  b = block_sum<NT>(b, sh);
  const double vals[2] = {a, b};
  if (publish_partials<2>(partials, ticket, vals, &last)) {
    reduce_partials_sum<NT, 2>(partials, out2, sh);
    if (thread_linear_id() == 0) *ticket = 0u;
  }
}

// Initial fields: the inflow profile on every face with the BC values on
// boundary faces, k and omega at the inlet values, p = 0.
template <typename T>
__global__ void __launch_bounds__(NT) k_init_fields(StepParams<T> p, T* __restrict__ u, T* __restrict__ v,
                                                    T* __restrict__ w, T* __restrict__ kf, T* __restrict__ om,
                                                    T* __restrict__ pr) {
  int q, k;
  plane_of(blockIdx.z, p.nz, q, k);
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (q == 0) {
    if (i > nx || j >= ny) return;
    const T in = p.prof[k] * p.dirx;
    T val = in;
    if (i == 0) val = normal_face(p.side[0], in, in);
    if (i == nx) val = normal_face(p.side[1], in, in);
    u[idx_u(p, i, j, k)] = val;
    if (i < nx) {
      const size_t c = idx_c(p, i, j, k);
      kf[c] = p.k_in;
      om[c] = p.om_in;
      pr[c] = T(0);
    }
  } else if (q == 1) {
    if (i >= nx || j > ny) return;
    const T in = p.prof[k] * p.diry;
    T val = in;
    if (j == 0) val = normal_face(p.side[2], in, in);
    if (j == ny) val = normal_face(p.side[3], in, in);
    v[idx_v(p, i, j, k)] = val;
  } else {
    if (i >= nx || j >= ny) return;
    w[idx_c(p, i, j, k)] = T(0);
  }
}

// ---------------------------------------------------- porosity -> drag ---
// c = C_d a ((1 - phi)/(phi + e))^b per cell (Sec. 3 footnote), computed in
// FP64 and stored in the field type.
template <typename T>
__global__ void k_drag_coeff(const T* __restrict__ phi, T* __restrict__ cc, size_t n, double Cd, double a, double b,
                             double e) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double ph = (double)phi[q];
  double ratio = (1.0 - ph) / (ph + e);
  if (ratio < 0.0) ratio = 0.0;
  cc[q] = (T)(Cd * a * pow(ratio, b));
}

// Dense <-> padded layout of one field (lx values per row, ly * lz rows; the
// padded rows have pitch P).  to_padded: dst[r P + i] = src[r lx + i], else
// the reverse.
template <typename T>
__global__ void __launch_bounds__(256) k_repack(const T* __restrict__ src, T* __restrict__ dst, int lx, int rows,
                                                int P, int to_padded) {
  const size_t n = (size_t)lx * rows;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / lx, i = e - r * lx;
    if (to_padded) dst[r * P + i] = src[e];
    else dst[e] = src[r * P + i];
  }
}

}  // namespace uf
