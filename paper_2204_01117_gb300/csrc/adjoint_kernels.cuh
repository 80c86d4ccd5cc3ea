// Discrete adjoint of one RANS time step (the transpose of the forward
// kernels in step_kernels.cuh, in reverse order) and of the objective.
//
// The paper computes design gradients by forward differences (Sec. 5,
// "Gradient-descent"; it names the adjoint method as the costlier
// alternative); this file provides the reverse-mode alternative.  Every
// kernel below is the exact transpose of the linearisation of one forward
// kernel at the forward state, with the branch the forward took (clamps,
// limiters, upwind side, porosity-drag cut-off, MacCormack clamp) deciding
// the derivative.  The time step is fixed (no derivative through the CFL
// condition).  One thread handles one forward output element, recomputes
// that element's forward locals and scatters lambda * d(out)/d(in) into
// the adjoint arrays of the inputs with atomicAdd (adjoint arrays start at
// zero).
#pragma once
#include "step_kernels.cuh"

namespace uf {

template <typename T>
__device__ __forceinline__ void aadd(T* p, T v) {
  atomicAdd(p, v);
}

// Transposes of the boundary-rule face reads (u_face / v_face / w_face).
template <typename T>
__device__ __forceinline__ void u_face_adj(T* lu, const StepParams<T>& p, int i, int j, int k, T val) {
  if (i == 0) {
    if (p.side[0] == OUTFLOW) aadd(&lu[idx_u(p, 1, j, k)], val);
    return;
  }
  if (i == p.nx) {
    if (p.side[1] == OUTFLOW) aadd(&lu[idx_u(p, p.nx - 1, j, k)], val);
    return;
  }
  aadd(&lu[idx_u(p, i, j, k)], val);
}
template <typename T>
__device__ __forceinline__ void v_face_adj(T* lv, const StepParams<T>& p, int i, int j, int k, T val) {
  if (j == 0) {
    if (p.side[2] == OUTFLOW) aadd(&lv[idx_v(p, i, 1, k)], val);
    return;
  }
  if (j == p.ny) {
    if (p.side[3] == OUTFLOW) aadd(&lv[idx_v(p, i, p.ny - 1, k)], val);
    return;
  }
  aadd(&lv[idx_v(p, i, j, k)], val);
}
template <typename T>
__device__ __forceinline__ void w_face_adj(T* lw, const StepParams<T>& p, int i, int j, int k, T val) {
  if (k == 0 || k == p.nz) return;
  aadd(&lw[idx_c(p, i, j, k)], val);
}
// Transpose of tangential_ghost(side, q, inflow) with respect to q.
template <typename T>
__device__ __forceinline__ T ghost_coef(int side) {
  return side == INFLOW ? T(0) : (side == NOSLIP ? T(-1) : T(1));
}

// ---------------------------------------------------------------- strain --
// Transpose of strain_sq: scatters lam * dS2/d(face) into the face adjoints.
template <typename T>
__device__ __forceinline__ void strain_sq_adj(T* lu, T* lv, T* lw, const T* __restrict__ u, const T* __restrict__ v,
                                              const T* __restrict__ w, const StepParams<T>& p, int i, int j, int k,
                                              T lam) {
  if (lam == T(0)) return;
  const T ih = p.inv_h;
  auto uc = [&](int a, int b, int c) { return T(0.5) * (u[idx_u(p, a, b, c)] + u[idx_u(p, a + 1, b, c)]); };
  auto vc = [&](int a, int b, int c) { return T(0.5) * (v[idx_v(p, a, b, c)] + v[idx_v(p, a, b + 1, c)]); };
  auto wc = [&](int a, int b, int c) { return T(0.5) * (w[idx_c(p, a, b, c)] + w[idx_c(p, a, b, c + 1)]); };
  auto uc_adj = [&](int a, int b, int c, T g) {
    aadd(&lu[idx_u(p, a, b, c)], T(0.5) * g);
    aadd(&lu[idx_u(p, a + 1, b, c)], T(0.5) * g);
  };
  auto vc_adj = [&](int a, int b, int c, T g) {
    aadd(&lv[idx_v(p, a, b, c)], T(0.5) * g);
    aadd(&lv[idx_v(p, a, b + 1, c)], T(0.5) * g);
  };
  auto wc_adj = [&](int a, int b, int c, T g) {
    aadd(&lw[idx_c(p, a, b, c)], T(0.5) * g);
    aadd(&lw[idx_c(p, a, b, c + 1)], T(0.5) * g);
  };
  const int im = i > 0 ? i - 1 : i, ip = i < p.nx - 1 ? i + 1 : i;
  const int jm = j > 0 ? j - 1 : j, jp = j < p.ny - 1 ? j + 1 : j;
  const int km = k > 0 ? k - 1 : k, kp = k < p.nz - 1 ? k + 1 : k;
  const T sx = (ip > im) ? ih / T(ip - im) : T(0);
  const T sy = (jp > jm) ? ih / T(jp - jm) : T(0);
  const T sz = (kp > km) ? ih / T(kp - km) : T(0);
  const T sxx = (u[idx_u(p, i + 1, j, k)] - u[idx_u(p, i, j, k)]) * ih;
  const T syy = (v[idx_v(p, i, j + 1, k)] - v[idx_v(p, i, j, k)]) * ih;
  const T szz = (w[idx_c(p, i, j, k + 1)] - w[idx_c(p, i, j, k)]) * ih;
  const T du_dy = (uc(i, jp, k) - uc(i, jm, k)) * sy;
  const T du_dz = (uc(i, j, kp) - uc(i, j, km)) * sz;
  const T dv_dx = (vc(ip, j, k) - vc(im, j, k)) * sx;
  const T dv_dz = (vc(i, j, kp) - vc(i, j, km)) * sz;
  const T dw_dx = (wc(ip, j, k) - wc(im, j, k)) * sx;
  const T dw_dy = (wc(i, jp, k) - wc(i, jm, k)) * sy;
  const T sxy = T(0.5) * (du_dy + dv_dx), sxz = T(0.5) * (du_dz + dw_dx), syz = T(0.5) * (dv_dz + dw_dy);
  // S2 = sxx^2 + syy^2 + szz^2 + 2 (sxy^2 + sxz^2 + syz^2)
  const T gxx = lam * T(2) * sxx, gyy = lam * T(2) * syy, gzz = lam * T(2) * szz;
  const T gxy = lam * T(2) * sxy, gxz = lam * T(2) * sxz, gyz = lam * T(2) * syz;   // d/d(du_dy) etc.
  aadd(&lu[idx_u(p, i + 1, j, k)], gxx * ih);
  aadd(&lu[idx_u(p, i, j, k)], -gxx * ih);
  aadd(&lv[idx_v(p, i, j + 1, k)], gyy * ih);
  aadd(&lv[idx_v(p, i, j, k)], -gyy * ih);
  aadd(&lw[idx_c(p, i, j, k + 1)], gzz * ih);
  aadd(&lw[idx_c(p, i, j, k)], -gzz * ih);
  if (sy != T(0)) { uc_adj(i, jp, k, gxy * sy); uc_adj(i, jm, k, -gxy * sy); }
  if (sx != T(0)) { vc_adj(ip, j, k, gxy * sx); vc_adj(im, j, k, -gxy * sx); }
  if (sz != T(0)) { uc_adj(i, j, kp, gxz * sz); uc_adj(i, j, km, -gxz * sz); }
  if (sx != T(0)) { wc_adj(ip, j, k, gxz * sx); wc_adj(im, j, k, -gxz * sx); }
  if (sz != T(0)) { vc_adj(i, j, kp, gyz * sz); vc_adj(i, j, km, -gyz * sz); }
  if (sy != T(0)) { wc_adj(i, jp, k, gyz * sy); wc_adj(i, jm, k, -gyz * sy); }
}

// limited_nut with its partial derivatives (the forward's branch decides).
template <typename T>
__device__ __forceinline__ T limited_nut_d(const StepParams<T>& p, T kv, T omv, T S2, T dt, T& dk, T& dom, T& dS2) {
  const T strain_om = p.C_lim * sqrt(S2) / sqrt(p.C_mu * T(0.5));
  const bool om_branch = !(strain_om > omv);   // fmax(omv, strain_om) returns omv unless strain_om is larger
  const T om_t = om_branch ? omv : strain_om;
  const T raw = kv / om_t;
  const T lim = p.h * p.h / (T(6) * dt) - p.nu;
  dk = dom = dS2 = T(0);
  const T nut = fmin(raw, lim);
  if (!(nut > T(0))) return T(0);
  if (raw < lim) {
    dk = T(1) / om_t;
    const T d_omt = -kv / (om_t * om_t);
    if (om_branch) dom = d_omt;
    else if (S2 > T(0)) dS2 = d_omt * (p.C_lim / sqrt(p.C_mu * T(0.5))) * T(0.5) / sqrt(S2);
  }
  return nut;
}

// ------------------------------------------------------- a9 transpose ----
// Adjoint of k_turbulence.  In: lk1, lo1 (adjoints of k^{n+1}, omega^{n+1}).
// Scatters into lk0, lo0 (adjoints of k^n, omega^n) and into the face
// adjoints of the projected velocity (lu1, lv1, lw1).
template <typename T>
__global__ void __launch_bounds__(NT) k_turbulence_adj(StepParams<T> p, const T* __restrict__ u, const T* __restrict__ v,
                                                       const T* __restrict__ w, const T* __restrict__ ki,
                                                       const T* __restrict__ oi, const T* __restrict__ lk1,
                                                       const T* __restrict__ lo1, T* lk0, T* lo0, T* lu1, T* lv1,
                                                       T* lw1) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= p.nx || j >= p.ny) return;
  const T dt = *p.dtT;
  const size_t c = idx_c(p, i, j, k);
  const T kc = ki[c], oc = oi[c];
  const T S2 = strain_sq(u, v, w, p, i, j, k);
  T dnk, dno, dnS;
  const T nut = limited_nut_d(p, kc, oc, S2, dt, dnk, dno, dnS);
  const T vel[3] = {T(0.5) * (u[idx_u(p, i, j, k)] + u[idx_u(p, i + 1, j, k)]),
                    T(0.5) * (v[idx_v(p, i, j, k)] + v[idx_v(p, i, j + 1, k)]),
                    T(0.5) * (w[idx_c(p, i, j, k)] + w[idx_c(p, i, j, k + 1)])};
  const int pos[3] = {i, j, k}, ext[3] = {p.nx, p.ny, p.nz};
  size_t strides[3] = {1, (size_t)p.Pc, (size_t)p.Pc * p.ny};
  // forward recomputation (same operation order as k_turbulence)
  T km[3], kp[3], om[3], op[3];
  T adv_k = 0, adv_o = 0, lap_k = T(-6) * kc, lap_o = T(-6) * oc;
  for (int ax = 0; ax < 3; ++ax) {
    const bool hm = pos[ax] > 0, hp = pos[ax] < ext[ax] - 1;
    const int sm = p.side[2 * ax], sp = p.side[2 * ax + 1];
    km[ax] = hm ? ki[c - strides[ax]] : (sm == INFLOW ? p.k_in : kc);
    kp[ax] = hp ? ki[c + strides[ax]] : (sp == INFLOW ? p.k_in : kc);
    om[ax] = hm ? oi[c - strides[ax]] : (sm == INFLOW ? p.om_in : oc);
    op[ax] = hp ? oi[c + strides[ax]] : (sp == INFLOW ? p.om_in : oc);
    lap_k += km[ax] + kp[ax];
    lap_o += om[ax] + op[ax];
    if (vel[ax] > T(0)) {
      adv_k += vel[ax] * (kc - km[ax]) * p.inv_h;
      adv_o += vel[ax] * (oc - om[ax]) * p.inv_h;
    } else if (vel[ax] < T(0)) {
      adv_k += vel[ax] * (kp[ax] - kc) * p.inv_h;
      adv_o += vel[ax] * (op[ax] - oc) * p.inv_h;
    }
  }
  const T ih2 = p.inv_h * p.inv_h;
  const T Pk = T(2) * nut * S2;
  const T rk = -adv_k + Pk - p.C_mu * kc * oc + (p.nu + p.sigma_star * nut) * lap_k * ih2;
  const T ro = -adv_o + T(2) * p.alpha * S2 - p.beta * oc * oc + (p.nu + p.sigma * nut) * lap_o * ih2;
  const T gk = (kc + dt * rk > p.k_min) ? lk1[c] : T(0);
  const T go = (oc + dt * ro > p.om_min) ? lo1[c] : T(0);
  if (gk == T(0) && go == T(0)) return;
  const T lrk = gk * dt, lro = go * dt;
  T l_kc = gk, l_oc = go, l_nut = 0, l_S2 = 0;
  l_nut += lrk * T(2) * S2;
  l_S2 += lrk * T(2) * nut;
  l_kc += -lrk * p.C_mu * oc;
  l_oc += -lrk * p.C_mu * kc;
  l_nut += lrk * p.sigma_star * lap_k * ih2;
  const T l_lapk = lrk * (p.nu + p.sigma_star * nut) * ih2;
  l_S2 += lro * T(2) * p.alpha;
  l_oc += -lro * T(2) * p.beta * oc;
  l_nut += lro * p.sigma * lap_o * ih2;
  const T l_lapo = lro * (p.nu + p.sigma * nut) * ih2;
  l_kc += T(-6) * l_lapk;
  l_oc += T(-6) * l_lapo;
  for (int ax = 0; ax < 3; ++ax) {
    const bool hm = pos[ax] > 0, hp = pos[ax] < ext[ax] - 1;
    const int sm = p.side[2 * ax], sp = p.side[2 * ax + 1];
    // neighbour contributions: l_km, l_kp, l_om, l_op
    T l_km = l_lapk, l_kp = l_lapk, l_om = l_lapo, l_op = l_lapo;
    T l_vel = 0;
    if (vel[ax] > T(0)) {
      // -adv: -(vel (kc - km) / h)
      l_kc += -lrk * vel[ax] * p.inv_h;
      l_km += lrk * vel[ax] * p.inv_h;
      l_oc += -lro * vel[ax] * p.inv_h;
      l_om += lro * vel[ax] * p.inv_h;
      l_vel += -lrk * (kc - km[ax]) * p.inv_h - lro * (oc - om[ax]) * p.inv_h;
    } else if (vel[ax] < T(0)) {
      l_kp += -lrk * vel[ax] * p.inv_h;
      l_kc += lrk * vel[ax] * p.inv_h;
      l_op += -lro * vel[ax] * p.inv_h;
      l_oc += lro * vel[ax] * p.inv_h;
      l_vel += -lrk * (kp[ax] - kc) * p.inv_h - lro * (op[ax] - oc) * p.inv_h;
    }
    if (hm) { aadd(&lk0[c - strides[ax]], l_km); aadd(&lo0[c - strides[ax]], l_om); }
    else if (sm != INFLOW) { l_kc += l_km; l_oc += l_om; }
    if (hp) { aadd(&lk0[c + strides[ax]], l_kp); aadd(&lo0[c + strides[ax]], l_op); }
    else if (sp != INFLOW) { l_kc += l_kp; l_oc += l_op; }
    if (l_vel != T(0)) {
      const T hv = T(0.5) * l_vel;
      if (ax == 0) { aadd(&lu1[idx_u(p, i, j, k)], hv); aadd(&lu1[idx_u(p, i + 1, j, k)], hv); }
      else if (ax == 1) { aadd(&lv1[idx_v(p, i, j, k)], hv); aadd(&lv1[idx_v(p, i, j + 1, k)], hv); }
      else { aadd(&lw1[idx_c(p, i, j, k)], hv); aadd(&lw1[idx_c(p, i, j, k + 1)], hv); }
    }
  }
  l_kc += l_nut * dnk;
  l_oc += l_nut * dno;
  l_S2 += l_nut * dnS;
  aadd(&lk0[c], l_kc);
  aadd(&lo0[c], l_oc);
  strain_sq_adj(lu1, lv1, lw1, u, v, w, p, i, j, k, l_S2);
}

// ------------------------------------------------------- a8 transpose ----
// u1 = u3 + G A^-1 Dv u3 (projection with its scaling), so
// lambda_u3 = lambda + Dv^T mu with A mu = G^T lambda.
// k_proj_adj_rhs: b(c) = G^T lambda: + lambda on the low face of c, - on
// the high face, projected faces only.  It also sets the initial guess of
// the solve, mu <- 2 mu - mu_prev (linear extrapolation along the reverse
// sweep, as for the forward pressure), keeping mu in mu_prev.
template <typename T>
__global__ void __launch_bounds__(NT) k_proj_adj_rhs(StepParams<T> p, const T* __restrict__ lu, const T* __restrict__ lv,
                                                     const T* __restrict__ lw, T* __restrict__ b, T* __restrict__ mu,
                                                     T* __restrict__ mu_prev) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= p.nx || j >= p.ny) return;
  auto proj_u = [&](int ii) { return (ii > 0 && ii < p.nx) || (ii == 0 && p.side[0] == OUTFLOW) || (ii == p.nx && p.side[1] == OUTFLOW); };
  auto proj_v = [&](int jj) { return (jj > 0 && jj < p.ny) || (jj == 0 && p.side[2] == OUTFLOW) || (jj == p.ny && p.side[3] == OUTFLOW); };
  auto proj_w = [&](int kk) { return kk > 0 && kk < p.nz; };
  T s = 0;
  if (proj_u(i)) s += lu[idx_u(p, i, j, k)];
  if (proj_u(i + 1)) s -= lu[idx_u(p, i + 1, j, k)];
  if (proj_v(j)) s += lv[idx_v(p, i, j, k)];
  if (proj_v(j + 1)) s -= lv[idx_v(p, i, j + 1, k)];
  if (proj_w(k)) s += lw[idx_c(p, i, j, k)];
  if (proj_w(k + 1)) s -= lw[idx_c(p, i, j, k + 1)];
  const size_t c = idx_c(p, i, j, k);
  b[c] = s;
  const T m = mu[c];
  mu[c] = T(2) * m - mu_prev[c];
  mu_prev[c] = m;
}

// lambda(f) += mu(c-) - mu(c+) on every face (missing cells count 0).
template <typename T>
__global__ void __launch_bounds__(NT) k_proj_adj_apply(StepParams<T> p, const T* __restrict__ mu, T* lu, T* lv, T* lw) {
  int q, k;
  plane_of(blockIdx.z, p.nz, q, k);
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (q == 0) {
    if (i > nx || j >= ny) return;
    const T mm = i > 0 ? mu[idx_c(p, i - 1, j, k)] : T(0);
    const T mp = i < nx ? mu[idx_c(p, i, j, k)] : T(0);
    lu[idx_u(p, i, j, k)] += mm - mp;
  } else if (q == 1) {
    if (i >= nx || j > ny) return;
    const T mm = j > 0 ? mu[idx_c(p, i, j - 1, k)] : T(0);
    const T mp = j < ny ? mu[idx_c(p, i, j, k)] : T(0);
    lv[idx_v(p, i, j, k)] += mm - mp;
  } else {
    if (i >= nx || j >= ny) return;
    const T mm = k > 0 ? mu[idx_c(p, i, j, k - 1)] : T(0);
    const T mp = k < nz ? mu[idx_c(p, i, j, k)] : T(0);
    lw[idx_c(p, i, j, k)] += mm - mp;
  }
}

// -------------------------------------------------- a4 + a5 transpose ----
// Adjoint of drag_u/v/w at one interior face with output adjoint lam.
template <typename T>
__device__ __forceinline__ void drag_face_adj(const StepParams<T>& p, int comp, const T* __restrict__ u,
                                              const T* __restrict__ v, const T* __restrict__ w, const T* __restrict__ cc,
                                              T dt, int i, int j, int k, T lam, T* lu, T* lv, T* lw, T* lc) {
  T q, ab, bb, cf;
  size_t c0, c1;
  if (comp == 0) {
    q = u[idx_u(p, i, j, k)];
    ab = T(0.25) * (v_face(v, p, i - 1, j, k) + v_face(v, p, i, j, k) + v_face(v, p, i - 1, j + 1, k) + v_face(v, p, i, j + 1, k));
    bb = T(0.25) * (w_face(w, p, i - 1, j, k) + w_face(w, p, i, j, k) + w_face(w, p, i - 1, j, k + 1) + w_face(w, p, i, j, k + 1));
    c0 = idx_c(p, i - 1, j, k);
    c1 = idx_c(p, i, j, k);
  } else if (comp == 1) {
    q = v[idx_v(p, i, j, k)];
    ab = T(0.25) * (u_face(u, p, i, j - 1, k) + u_face(u, p, i + 1, j - 1, k) + u_face(u, p, i, j, k) + u_face(u, p, i + 1, j, k));
    bb = T(0.25) * (w_face(w, p, i, j - 1, k) + w_face(w, p, i, j, k) + w_face(w, p, i, j - 1, k + 1) + w_face(w, p, i, j, k + 1));
    c0 = idx_c(p, i, j - 1, k);
    c1 = idx_c(p, i, j, k);
  } else {
    q = w[idx_c(p, i, j, k)];
    ab = T(0.25) * (u_face(u, p, i, j, k - 1) + u_face(u, p, i + 1, j, k - 1) + u_face(u, p, i, j, k) + u_face(u, p, i + 1, j, k));
    bb = T(0.25) * (v_face(v, p, i, j, k - 1) + v_face(v, p, i, j + 1, k - 1) + v_face(v, p, i, j, k) + v_face(v, p, i, j + 1, k));
    c0 = idx_c(p, i, j, k - 1);
    c1 = idx_c(p, i, j, k);
  }
  const T sp = sqrt(q * q + ab * ab + bb * bb);
  cf = T(0.5) * (cc[c0] + cc[c1]);
  const T fac = T(1) - dt * cf * sp;
  if (!(fac > T(0))) return;   // clamped at zero: no sensitivity
  T dq = fac, dab = 0, dbb = 0;
  if (sp > T(0)) {
    dq -= dt * cf * q * q / sp;
    dab = -dt * cf * q * ab / sp;
    dbb = -dt * cf * q * bb / sp;
  }
  const T dcf = -dt * sp * q;
  aadd(&lc[c0], T(0.5) * lam * dcf);
  aadd(&lc[c1], T(0.5) * lam * dcf);
  const T ga = T(0.25) * lam * dab, gb = T(0.25) * lam * dbb;
  if (comp == 0) {
    aadd(&lu[idx_u(p, i, j, k)], lam * dq);
    v_face_adj(lv, p, i - 1, j, k, ga); v_face_adj(lv, p, i, j, k, ga);
    v_face_adj(lv, p, i - 1, j + 1, k, ga); v_face_adj(lv, p, i, j + 1, k, ga);
    w_face_adj(lw, p, i - 1, j, k, gb); w_face_adj(lw, p, i, j, k, gb);
    w_face_adj(lw, p, i - 1, j, k + 1, gb); w_face_adj(lw, p, i, j, k + 1, gb);
  } else if (comp == 1) {
    aadd(&lv[idx_v(p, i, j, k)], lam * dq);
    u_face_adj(lu, p, i, j - 1, k, ga); u_face_adj(lu, p, i + 1, j - 1, k, ga);
    u_face_adj(lu, p, i, j, k, ga); u_face_adj(lu, p, i + 1, j, k, ga);
    w_face_adj(lw, p, i, j - 1, k, gb); w_face_adj(lw, p, i, j, k, gb);
    w_face_adj(lw, p, i, j - 1, k + 1, gb); w_face_adj(lw, p, i, j, k + 1, gb);
  } else {
    aadd(&lw[idx_c(p, i, j, k)], lam * dq);
    u_face_adj(lu, p, i, j, k - 1, ga); u_face_adj(lu, p, i + 1, j, k - 1, ga);
    u_face_adj(lu, p, i, j, k, ga); u_face_adj(lu, p, i + 1, j, k, ga);
    v_face_adj(lv, p, i, j, k - 1, gb); v_face_adj(lv, p, i, j + 1, k - 1, gb);
    v_face_adj(lv, p, i, j, k, gb); v_face_adj(lv, p, i, j + 1, k, gb);
  }
}

// Adjoint of k_drag_bc.  In: l3 (adjoint of the dragged field, every face).
// An outlet face copied its interior neighbour, so its adjoint joins that
// neighbour's; inlet and wall faces are constants.  Out: l2 (adjoint of the
// diffused field, interior faces), lc (drag coefficient, accumulated).
template <typename T>
__global__ void __launch_bounds__(NT) k_drag_bc_adj(StepParams<T> p, const T* __restrict__ u2, const T* __restrict__ v2,
                                                    const T* __restrict__ w2, const T* __restrict__ cc,
                                                    const T* __restrict__ lu3, const T* __restrict__ lv3,
                                                    const T* __restrict__ lw3, T* lu2, T* lv2, T* lw2, T* lc) {
  int q, k;
  plane_of(blockIdx.z, p.nz, q, k);
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const T dt = *p.dtT;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (q == 0) {
    if (i < 1 || i >= nx || j >= ny) return;
    T lam = lu3[idx_u(p, i, j, k)];
    if (i == 1 && p.side[0] == OUTFLOW) lam += lu3[idx_u(p, 0, j, k)];
    if (i == nx - 1 && p.side[1] == OUTFLOW) lam += lu3[idx_u(p, nx, j, k)];
    if (lam != T(0)) drag_face_adj(p, 0, u2, v2, w2, cc, dt, i, j, k, lam, lu2, lv2, lw2, lc);
  } else if (q == 1) {
    if (i >= nx || j < 1 || j >= ny) return;
    T lam = lv3[idx_v(p, i, j, k)];
    if (j == 1 && p.side[2] == OUTFLOW) lam += lv3[idx_v(p, i, 0, k)];
    if (j == ny - 1 && p.side[3] == OUTFLOW) lam += lv3[idx_v(p, i, ny, k)];
    if (lam != T(0)) drag_face_adj(p, 1, u2, v2, w2, cc, dt, i, j, k, lam, lu2, lv2, lw2, lc);
  } else {
    if (i >= nx || j >= ny || k < 1 || k >= nz) return;
    const T lam = lw3[idx_c(p, i, j, k)];
    if (lam != T(0)) drag_face_adj(p, 2, u2, v2, w2, cc, dt, i, j, k, lam, lu2, lv2, lw2, lc);
  }
}

// ------------------------------------------------------- a3 transpose ----
// Adjoint of k_diffuse.  In: l2 (interior faces).  Out: lt (adjoint of the
// advected field, interior faces), lnut.
template <typename T>
__global__ void __launch_bounds__(NT) k_diffuse_adj(StepParams<T> p, const T* __restrict__ ut, const T* __restrict__ vt,
                                                    const T* __restrict__ wt, const T* __restrict__ nut,
                                                    const T* __restrict__ lu2, const T* __restrict__ lv2,
                                                    const T* __restrict__ lw2, T* lut, T* lvt, T* lwt, T* lnut) {
  int q, k;
  plane_of(blockIdx.z, p.nz, q, k);
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const T dt = *p.dtT;
  const T c = dt * p.inv_h * p.inv_h;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  if (q == 0) {
    if (i < 1 || i >= nx || j >= ny) return;
    const T lam = lu2[idx_u(p, i, j, k)];
    if (lam == T(0)) return;
    const T x0 = ut[idx_u(p, i, j, k)];
    const T inflow = p.prof[k] * p.dirx;
    const T xm = u_face(ut, p, i - 1, j, k), xp = u_face(ut, p, i + 1, j, k);
    const T ym = j > 0 ? ut[idx_u(p, i, j - 1, k)] : tangential_ghost(p.side[2], x0, inflow);
    const T yp = j < ny - 1 ? ut[idx_u(p, i, j + 1, k)] : tangential_ghost(p.side[3], x0, inflow);
    const T zm = k > 0 ? ut[idx_u(p, i, j, k - 1)] : tangential_ghost(p.side[4], x0, T(0));
    const T zp = k < nz - 1 ? ut[idx_u(p, i, j, k + 1)] : tangential_ghost(p.side[5], x0, T(0));
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (nut[idx_c(p, i - 1, j, k)] + nut[idx_c(p, i, j, k)]);
    const T cD = c * (p.nu + nf);
    const T g = lam * cD;
    T l0 = lam * (T(1) - T(6) * cD);
    u_face_adj(lut, p, i - 1, j, k, g);
    u_face_adj(lut, p, i + 1, j, k, g);
    if (j > 0) aadd(&lut[idx_u(p, i, j - 1, k)], g); else l0 += g * ghost_coef<T>(p.side[2]);
    if (j < ny - 1) aadd(&lut[idx_u(p, i, j + 1, k)], g); else l0 += g * ghost_coef<T>(p.side[3]);
    if (k > 0) aadd(&lut[idx_u(p, i, j, k - 1)], g); else l0 += g * ghost_coef<T>(p.side[4]);
    if (k < nz - 1) aadd(&lut[idx_u(p, i, j, k + 1)], g); else l0 += g * ghost_coef<T>(p.side[5]);
    aadd(&lut[idx_u(p, i, j, k)], l0);
    const T ln = T(0.5) * lam * c * lap;
    aadd(&lnut[idx_c(p, i - 1, j, k)], ln);
    aadd(&lnut[idx_c(p, i, j, k)], ln);
  } else if (q == 1) {
    if (i >= nx || j < 1 || j >= ny) return;
    const T lam = lv2[idx_v(p, i, j, k)];
    if (lam == T(0)) return;
    const T x0 = vt[idx_v(p, i, j, k)];
    const T inflow = p.prof[k] * p.diry;
    const T xm = i > 0 ? vt[idx_v(p, i - 1, j, k)] : tangential_ghost(p.side[0], x0, inflow);
    const T xp = i < nx - 1 ? vt[idx_v(p, i + 1, j, k)] : tangential_ghost(p.side[1], x0, inflow);
    const T ym = v_face(vt, p, i, j - 1, k), yp = v_face(vt, p, i, j + 1, k);
    const T zm = k > 0 ? vt[idx_v(p, i, j, k - 1)] : tangential_ghost(p.side[4], x0, T(0));
    const T zp = k < nz - 1 ? vt[idx_v(p, i, j, k + 1)] : tangential_ghost(p.side[5], x0, T(0));
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (nut[idx_c(p, i, j - 1, k)] + nut[idx_c(p, i, j, k)]);
    const T cD = c * (p.nu + nf);
    const T g = lam * cD;
    T l0 = lam * (T(1) - T(6) * cD);
    if (i > 0) aadd(&lvt[idx_v(p, i - 1, j, k)], g); else l0 += g * ghost_coef<T>(p.side[0]);
    if (i < nx - 1) aadd(&lvt[idx_v(p, i + 1, j, k)], g); else l0 += g * ghost_coef<T>(p.side[1]);
    v_face_adj(lvt, p, i, j - 1, k, g);
    v_face_adj(lvt, p, i, j + 1, k, g);
    if (k > 0) aadd(&lvt[idx_v(p, i, j, k - 1)], g); else l0 += g * ghost_coef<T>(p.side[4]);
    if (k < nz - 1) aadd(&lvt[idx_v(p, i, j, k + 1)], g); else l0 += g * ghost_coef<T>(p.side[5]);
    aadd(&lvt[idx_v(p, i, j, k)], l0);
    const T ln = T(0.5) * lam * c * lap;
    aadd(&lnut[idx_c(p, i, j - 1, k)], ln);
    aadd(&lnut[idx_c(p, i, j, k)], ln);
  } else {
    if (i >= nx || j >= ny || k < 1 || k >= nz) return;
    const T lam = lw2[idx_c(p, i, j, k)];
    if (lam == T(0)) return;
    const T x0 = wt[idx_c(p, i, j, k)];
    const T xm = i > 0 ? wt[idx_c(p, i - 1, j, k)] : tangential_ghost(p.side[0], x0, T(0));
    const T xp = i < nx - 1 ? wt[idx_c(p, i + 1, j, k)] : tangential_ghost(p.side[1], x0, T(0));
    const T ym = j > 0 ? wt[idx_c(p, i, j - 1, k)] : tangential_ghost(p.side[2], x0, T(0));
    const T yp = j < ny - 1 ? wt[idx_c(p, i, j + 1, k)] : tangential_ghost(p.side[3], x0, T(0));
    const T zm = w_face(wt, p, i, j, k - 1), zp = w_face(wt, p, i, j, k + 1);
    const T lap = xm + xp + ym + yp + zm + zp - T(6) * x0;
    const T nf = T(0.5) * (nut[idx_c(p, i, j, k - 1)] + nut[idx_c(p, i, j, k)]);
    const T cD = c * (p.nu + nf);
    const T g = lam * cD;
    T l0 = lam * (T(1) - T(6) * cD);
    if (i > 0) aadd(&lwt[idx_c(p, i - 1, j, k)], g); else l0 += g * ghost_coef<T>(p.side[0]);
    if (i < nx - 1) aadd(&lwt[idx_c(p, i + 1, j, k)], g); else l0 += g * ghost_coef<T>(p.side[1]);
    if (j > 0) aadd(&lwt[idx_c(p, i, j - 1, k)], g); else l0 += g * ghost_coef<T>(p.side[2]);
    if (j < ny - 1) aadd(&lwt[idx_c(p, i, j + 1, k)], g); else l0 += g * ghost_coef<T>(p.side[3]);
    w_face_adj(lwt, p, i, j, k - 1, g);
    w_face_adj(lwt, p, i, j, k + 1, g);
    aadd(&lwt[idx_c(p, i, j, k)], l0);
    const T ln = T(0.5) * lam * c * lap;
    aadd(&lnut[idx_c(p, i, j, k - 1)], ln);
    aadd(&lnut[idx_c(p, i, j, k)], ln);
  }
}

// ------------------------------------------------------- a1 transpose ----
// Adjoint of k_eddy_viscosity: lnut -> lk, lo, and the faces of u^n.
template <typename T>
__global__ void __launch_bounds__(NT) k_eddy_viscosity_adj(StepParams<T> p, const T* __restrict__ u,
                                                           const T* __restrict__ v, const T* __restrict__ w,
                                                           const T* __restrict__ kf, const T* __restrict__ om,
                                                           const T* __restrict__ lnut, T* lk, T* lo, T* lu, T* lv,
                                                           T* lw) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= p.nx || j >= p.ny) return;
  const size_t c = idx_c(p, i, j, k);
  const T lam = lnut[c];
  if (lam == T(0)) return;
  const T S2 = strain_sq(u, v, w, p, i, j, k);
  T dk, dom, dS2;
  limited_nut_d(p, kf[c], om[c], S2, *p.dtT, dk, dom, dS2);
  aadd(&lk[c], lam * dk);
  aadd(&lo[c], lam * dom);
  strain_sq_adj(lu, lv, lw, u, v, w, p, i, j, k, lam * dS2);
}

// ------------------------------------------------------- a2 transpose ----
// Trilinear weights and value gradient of sample() at (a, b, c); scatters
// lam * weight into lF when lF != nullptr.  The gradient along a clamped
// axis is zero.
template <typename T>
__device__ __forceinline__ void sample_adj(const T* __restrict__ F, T* lF, Lattice L, int ia, T oa, int ib, T ob,
                                           int ic, T oc, T lam, T grad[3]) {
  const bool fa = L.Lx >= 2 && axis_inside(ia, oa, L.Lx);
  const bool fb = L.Ly >= 2 && axis_inside(ib, ob, L.Ly);
  const bool fc = L.Lz >= 2 && axis_inside(ic, oc, L.Lz);
  int i0, i1, j0, j1, k0, k1;
  T ta, tb, tc;
  axis_cell(ia, oa, L.Lx, i0, i1, ta);
  axis_cell(ib, ob, L.Ly, j0, j1, tb);
  axis_cell(ic, oc, L.Lz, k0, k1, tc);
  const size_t r00 = (size_t)L.P * ((size_t)j0 + (size_t)L.Ly * k0);
  const size_t r10 = (size_t)L.P * ((size_t)j1 + (size_t)L.Ly * k0);
  const size_t r01 = (size_t)L.P * ((size_t)j0 + (size_t)L.Ly * k1);
  const size_t r11 = (size_t)L.P * ((size_t)j1 + (size_t)L.Ly * k1);
  const T a0 = T(1) - ta, b0 = T(1) - tb, c0 = T(1) - tc;
  if (lF && lam != T(0)) {
    aadd(&lF[r00 + i0], lam * a0 * b0 * c0);
    aadd(&lF[r00 + i1], lam * ta * b0 * c0);
    aadd(&lF[r10 + i0], lam * a0 * tb * c0);
    aadd(&lF[r10 + i1], lam * ta * tb * c0);
    aadd(&lF[r01 + i0], lam * a0 * b0 * tc);
    aadd(&lF[r01 + i1], lam * ta * b0 * tc);
    aadd(&lF[r11 + i0], lam * a0 * tb * tc);
    aadd(&lF[r11 + i1], lam * ta * tb * tc);
  }
  if (grad) {
    const T f000 = F[r00 + i0], f100 = F[r00 + i1], f010 = F[r10 + i0], f110 = F[r10 + i1];
    const T f001 = F[r01 + i0], f101 = F[r01 + i1], f011 = F[r11 + i0], f111 = F[r11 + i1];
    grad[0] = fa ? (f100 - f000) * b0 * c0 + (f110 - f010) * tb * c0 + (f101 - f001) * b0 * tc + (f111 - f011) * tb * tc : T(0);
    grad[1] = fb ? (f010 - f000) * a0 * c0 + (f110 - f100) * ta * c0 + (f011 - f001) * a0 * tc + (f111 - f101) * ta * tc : T(0);
    grad[2] = fc ? (f001 - f000) * a0 * b0 + (f101 - f100) * ta * b0 + (f011 - f010) * a0 * tb + (f111 - f110) * ta * tb : T(0);
  }
}

// Transpose of displacement(): scatters s * ld (d(displacement) adjoint)
// into the velocity-lattice adjoints of time level n.
template <typename T>
__device__ __forceinline__ void displacement_adj(const AdvectArgs<T>& A, int q, int i, int j, int k, T s, const T ld[3],
                                                 T* lu, T* lv, T* lw) {
  if (q == 0) {
    aadd(&lu[(size_t)i + (size_t)A.Lu.P * ((size_t)j + (size_t)A.Lu.Ly * k)], s * ld[0]);
    sample_adj<T>(A.v, lv, A.Lv, i, T(-0.5), j, T(0.5), k, T(0), s * ld[1], nullptr);
    sample_adj<T>(A.w, lw, A.Lw, i, T(-0.5), j, T(0), k, T(0.5), s * ld[2], nullptr);
  } else if (q == 1) {
    sample_adj<T>(A.u, lu, A.Lu, i, T(0.5), j, T(-0.5), k, T(0), s * ld[0], nullptr);
    aadd(&lv[(size_t)i + (size_t)A.Lv.P * ((size_t)j + (size_t)A.Lv.Ly * k)], s * ld[1]);
    sample_adj<T>(A.w, lw, A.Lw, i, T(0), j, T(-0.5), k, T(0.5), s * ld[2], nullptr);
  } else {
    sample_adj<T>(A.u, lu, A.Lu, i, T(0.5), j, T(0), k, T(-0.5), s * ld[0], nullptr);
    sample_adj<T>(A.v, lv, A.Lv, i, T(0), j, T(0.5), k, T(-0.5), s * ld[1], nullptr);
    aadd(&lw[(size_t)i + (size_t)A.Lw.P * ((size_t)j + (size_t)A.Lw.Ly * k)], s * ld[2]);
  }
}

// Adjoint arrays for the advection transposes.
template <typename T>
struct AdvectAdj {
  const T* lut;
  const T* lvt;
  const T* lwt;   // adjoint of the MacCormack result (interior faces)
  T* luh;
  T* lvh;
  T* lwh;         // adjoint of the forward-step fields (accumulated)
  T* lu;
  T* lv;
  T* lw;          // adjoint of the velocity of time level n (accumulated)
};

// Pass A: transpose of the backward step, correction and clamp.
template <typename T>
__global__ void __launch_bounds__(NT, 2) k_advect_backward_adj(AdvectArgs<T> A, AdvectAdj<T> J) {
  int q, k;
  plane_of(blockIdx.z, A.nz, q, k);
  const Lattice L = q == 0 ? A.Lu : (q == 1 ? A.Lv : A.Lw);
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= L.Lx || j >= L.Ly) return;
  const bool interior = q == 0 ? (i > 0 && i < A.nx) : (q == 1 ? (j > 0 && j < A.ny) : (k > 0 && k < A.nz));
  if (!interior) return;
  const size_t id = (size_t)i + (size_t)L.P * ((size_t)j + (size_t)L.Ly * k);
  const T lam = q == 0 ? J.lut[id] : (q == 1 ? J.lvt[id] : J.lwt[id]);
  if (lam == T(0)) return;
  const T s = *A.dtT * A.inv_h;
  const T* F = q == 0 ? A.u : (q == 1 ? A.v : A.w);
  const T* Fh = q == 0 ? A.uh : (q == 1 ? A.vh : A.wh);
  T* lF = q == 0 ? J.lu : (q == 1 ? J.lv : J.lw);
  T* lFh = q == 0 ? J.luh : (q == 1 ? J.lvh : J.lwh);
  T d[3];
  displacement(A, q, i, j, k, s, d);
  T mn, mx;
  const T fwd = sample<T, true>(F, L, i, -d[0], j, -d[1], k, -d[2], &mn, &mx);
  const T bwd = sample<T, false>(Fh, L, i, d[0], j, d[1], k, d[2]);
  const T r = fwd + T(0.5) * (F[id] - bwd);
  if (r < mn || r > mx) {
    // clamped: the output is one of the 8 forward-sample values
    const T target = r < mn ? mn : mx;
    int i0, i1, j0, j1, k0, k1;
    T ta, tb, tc;
    axis_cell(i, -d[0], L.Lx, i0, i1, ta);
    axis_cell(j, -d[1], L.Ly, j0, j1, tb);
    axis_cell(k, -d[2], L.Lz, k0, k1, tc);
    const int ii[2] = {i0, i1}, jj[2] = {j0, j1}, kk[2] = {k0, k1};
    for (int cz = 0; cz < 2; ++cz)
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
          const size_t e = (size_t)ii[cx] + (size_t)L.P * ((size_t)jj[cy] + (size_t)L.Ly * kk[cz]);
          if (F[e] == target) {
            aadd(&lF[e], lam);
            return;
          }
        }
    return;
  }
  aadd(&lF[id], T(0.5) * lam);
  T gf[3], gb[3];
  sample_adj<T>(F, lF, L, i, -d[0], j, -d[1], k, -d[2], lam, gf);
  sample_adj<T>(Fh, lFh, L, i, d[0], j, d[1], k, d[2], T(-0.5) * lam, gb);
  // d(fwd)/dd = -grad f, d(bwd)/dd = +grad fh
  const T ld[3] = {-lam * gf[0] - T(0.5) * lam * gb[0], -lam * gf[1] - T(0.5) * lam * gb[1],
                   -lam * gf[2] - T(0.5) * lam * gb[2]};
  displacement_adj(A, q, i, j, k, s, ld, J.lu, J.lv, J.lw);
}

// Pass B: transpose of the forward step at every lattice point.
template <typename T>
__global__ void __launch_bounds__(NT) k_advect_forward_adj(AdvectArgs<T> A, AdvectAdj<T> J) {
  int q, k;
  plane_of(blockIdx.z, A.nz, q, k);
  const Lattice L = q == 0 ? A.Lu : (q == 1 ? A.Lv : A.Lw);
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= L.Lx || j >= L.Ly) return;
  const size_t id = (size_t)i + (size_t)L.P * ((size_t)j + (size_t)L.Ly * k);
  const T lam = q == 0 ? J.luh[id] : (q == 1 ? J.lvh[id] : J.lwh[id]);
  if (lam == T(0)) return;
  const T s = *A.dtT * A.inv_h;
  const T* F = q == 0 ? A.u : (q == 1 ? A.v : A.w);
  T* lF = q == 0 ? J.lu : (q == 1 ? J.lv : J.lw);
  T d[3];
  displacement(A, q, i, j, k, s, d);
  T g[3];
  sample_adj<T>(F, lF, L, i, -d[0], j, -d[1], k, -d[2], lam, g);
  const T ld[3] = {-lam * g[0], -lam * g[1], -lam * g[2]};
  displacement_adj(A, q, i, j, k, s, ld, J.lu, J.lv, J.lw);
}

// ------------------------------------------------------ a10 transpose ----
// Seed of the reverse sweep: dJ/du on every face from the comfort objective.
template <typename T>
__global__ void __launch_bounds__(NT) k_objective_adj(StepParams<T> p, const T* __restrict__ u, const T* __restrict__ v,
                                                      const T* __restrict__ w, int k_lo, int k_hi, double u_hi,
                                                      double u_lo, T* lu, T* lv, T* lw) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = k_lo + blockIdx.z;
  if (i >= p.nx || j >= p.ny || k > k_hi) return;
  const double uc = 0.5 * ((double)u[idx_u(p, i, j, k)] + (double)u[idx_u(p, i + 1, j, k)]);
  const double vc = 0.5 * ((double)v[idx_v(p, i, j, k)] + (double)v[idx_v(p, i, j + 1, k)]);
  const double wc = 0.5 * ((double)w[idx_c(p, i, j, k)] + (double)w[idx_c(p, i, j, k + 1)]);
  const double s = sqrt(uc * uc + vc * vc + wc * wc);
  if (!(s > 0.0)) return;
  const double fp = 2.0 * fmax(s - u_hi, 0.0) - 2.0 * fmax(u_lo - s, 0.0);
  if (fp == 0.0) return;
  const T gx = (T)(0.5 * fp * uc / s), gy = (T)(0.5 * fp * vc / s), gz = (T)(0.5 * fp * wc / s);
  aadd(&lu[idx_u(p, i, j, k)], gx);
  aadd(&lu[idx_u(p, i + 1, j, k)], gx);
  aadd(&lv[idx_v(p, i, j, k)], gy);
  aadd(&lv[idx_v(p, i, j + 1, k)], gy);
  aadd(&lw[idx_c(p, i, j, k)], gz);
  aadd(&lw[idx_c(p, i, j, k + 1)], gz);
}

// Seed of the region-average objective for one region: dL/du_c = coef u_c /
// |u_c| on the cells of the box, coef = 2 (mean speed - u_t) / cell count,
// scattered half to each of the two faces of every component.
template <typename T>
__global__ void __launch_bounds__(NT) k_box_speed_adj(StepParams<T> p, const T* __restrict__ u,
                                                      const T* __restrict__ v, const T* __restrict__ w, int i0, int i1,
                                                      int j0, int j1, int k0, double coef, T* lu, T* lv, T* lw) {
  const int i = i0 + blockIdx.x * BX + threadIdx.x, j = j0 + blockIdx.y * BY + threadIdx.y, k = k0 + blockIdx.z;
  if (i > i1 || j > j1) return;
  const double uc = 0.5 * ((double)u[idx_u(p, i, j, k)] + (double)u[idx_u(p, i + 1, j, k)]);
  const double vc = 0.5 * ((double)v[idx_v(p, i, j, k)] + (double)v[idx_v(p, i, j + 1, k)]);
  const double wc = 0.5 * ((double)w[idx_c(p, i, j, k)] + (double)w[idx_c(p, i, j, k + 1)]);
  const double s = sqrt(uc * uc + vc * vc + wc * wc);
  if (!(s > 0.0)) return;
  const T gx = (T)(0.5 * coef * uc / s), gy = (T)(0.5 * coef * vc / s), gz = (T)(0.5 * coef * wc / s);
  aadd(&lu[idx_u(p, i, j, k)], gx);
  aadd(&lu[idx_u(p, i + 1, j, k)], gx);
  aadd(&lv[idx_v(p, i, j, k)], gy);
  aadd(&lv[idx_v(p, i, j + 1, k)], gy);
  aadd(&lw[idx_c(p, i, j, k)], gz);
  aadd(&lw[idx_c(p, i, j, k + 1)], gz);
}

// dJ/dphi = dJ/dc * dc/dphi with c = C_d a ((1-phi)/(phi+e))^b, in FP64.
template <typename T>
__global__ void k_dphi(const T* __restrict__ phi, const T* __restrict__ lc, T* __restrict__ out, size_t n, double Cd,
                       double a, double b, double e) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double ph = (double)phi[q];
  const double ratio = (1.0 - ph) / (ph + e);
  double dc = 0.0;
  if (ratio > 0.0) dc = Cd * a * b * pow(ratio, b - 1.0) * (-(1.0 + e) / ((ph + e) * (ph + e)));
  out[q] = (T)((double)lc[q] * dc);
}

// ---------------------------------------------- a12: design -> porosity --
// phi = prod_i (1 - chi_i), chi_i = s((x - xa_i)/w) s((xb_i - x)/w)
// s((y - ya_i)/w) s((yb_i - y)/w) s((H_i - z)/w) at cell centres, s the
// logistic function; box i = base box shifted by (dx_i, dy_i), height H_i.
struct DesignBox {
  double xa, xb, ya, yb;   // base footprint [m]
  double H, dx, dy;        // design parameters [m]
};
constexpr int MAX_BOXES = 64;

__device__ __forceinline__ double logistic(double t) { return 1.0 / (1.0 + exp(-t)); }

template <typename T>
__global__ void k_design_phi(int nx, int ny, int nz, int P, double h, const DesignBox* __restrict__ boxes, int nbox,
                             double wdt, T* __restrict__ phi) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= nx || j >= ny) return;
  const double x = (i + 0.5) * h, y = (j + 0.5) * h, z = (k + 0.5) * h;
  double ph = 1.0;
  for (int b = 0; b < nbox; ++b) {
    const DesignBox B = boxes[b];
    const double chi = logistic((x - (B.xa + B.dx)) / wdt) * logistic(((B.xb + B.dx) - x) / wdt) *
                       logistic((y - (B.ya + B.dy)) / wdt) * logistic(((B.yb + B.dy) - y) / wdt) *
                       logistic((B.H - z) / wdt);
    ph *= 1.0 - chi;
  }
  phi[(size_t)i + (size_t)P * ((size_t)j + (size_t)ny * k)] = (T)ph;
}

// Vector-Jacobian product: g[3b + {0,1,2}] += sum_cells lphi dphi/d(H, dx, dy)_b.
template <typename T>
__global__ void __launch_bounds__(NT) k_design_phi_vjp(int nx, int ny, int nz, int P, double h,
                                                       const DesignBox* __restrict__ boxes, int nbox, double wdt,
                                                       const T* __restrict__ lphi, double* g) {
  __shared__ double sg[3 * MAX_BOXES];
  const int tid = threadIdx.x + BX * threadIdx.y;
  for (int e = tid; e < 3 * nbox; e += NT) sg[e] = 0.0;
  __syncthreads();
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i < nx && j < ny) {
    const double lam = (double)lphi[(size_t)i + (size_t)P * ((size_t)j + (size_t)ny * k)];
    if (lam != 0.0) {
      const double x = (i + 0.5) * h, y = (j + 0.5) * h, z = (k + 0.5) * h;
      double chi[MAX_BOXES];
      for (int b = 0; b < nbox; ++b) {
        const DesignBox B = boxes[b];
        chi[b] = logistic((x - (B.xa + B.dx)) / wdt) * logistic(((B.xb + B.dx) - x) / wdt) *
                 logistic((y - (B.ya + B.dy)) / wdt) * logistic(((B.yb + B.dy) - y) / wdt) *
                 logistic((B.H - z) / wdt);
      }
      for (int b = 0; b < nbox; ++b) {
        double others = 1.0;   // prod_{c != b} (1 - chi_c)
        for (int c = 0; c < nbox; ++c)
          if (c != b) others *= 1.0 - chi[c];
        const DesignBox B = boxes[b];
        const double sxa = logistic((x - (B.xa + B.dx)) / wdt), sxb = logistic(((B.xb + B.dx) - x) / wdt);
        const double sya = logistic((y - (B.ya + B.dy)) / wdt), syb = logistic(((B.yb + B.dy) - y) / wdt);
        const double sz = logistic((B.H - z) / wdt);
        // dphi/dchi_b = -others; dchi/dtheta = chi * (dlog s/dtheta)
        const double base = -others * chi[b] * lam / wdt;
        atomicAdd(&sg[3 * b + 0], base * (1.0 - sz));
        atomicAdd(&sg[3 * b + 1], base * (-(1.0 - sxa) + (1.0 - sxb)));
        atomicAdd(&sg[3 * b + 2], base * (-(1.0 - sya) + (1.0 - syb)));
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < 3 * nbox; e += NT)
    if (sg[e] != 0.0) atomicAdd(&g[e], sg[e]);
}

}  // namespace uf
