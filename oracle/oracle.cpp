// UrbanFlow RANS step -- FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
// restatement of one Eulerian RANS time step of "UrbanFlow: Designing
// Comfortable Outdoor Areas" (arXiv 2204.01117).  It exists so that the CUDA
// path can be checked against it.  Only the tests, the smoke check and the
// CPU-baseline leg of the benchmark may load it; the product library never
// links, calls or includes anything from here, and this file includes nothing
// from the product.
//
// Every routine follows the paper's operator-split order (Sec. 3,
// "Discretization and Numerical Integration"):
//   dt (CFL)  ->  eddy viscosity (Eq. nu_t, limiter)  ->  MacCormack advection
//   ->  (nu+nu_t) diffusion  ->  porosity drag (Sec. 3, "Porosity Model",
//   forward-Euler drag equation)  ->  velocity BCs (Sec. 3 BC equations)
//   ->  pressure Poisson solve  ->  projection  ->  k-omega update (Eqs. k,
//   omega, P_k; Table 1 coefficients).
// Where the paper leaves a choice open, the reading used here is stated
// beside the code; the two implementations take the same readings.
//
// Pressure (step a7): the oracle solves A p = b to ||r||/||b|| <= tol
// (default 1e-13) with unpreconditioned CG, i.e. it computes the exact
// discrete solution that any preconditioned solver converges to.
//
// Layout (x fastest, structure of arrays, no ghost layers):
//   u : (nx+1) * ny * nz      u(i,j,k) at x=i h,     y=(j+1/2)h, z=(k+1/2)h
//   v : nx * (ny+1) * nz      v(i,j,k) at x=(i+1/2)h, y=j h,     z=(k+1/2)h
//   w : nx * ny * (nz+1)      w(i,j,k) at x=(i+1/2)h, y=(j+1/2)h, z=k h
//   p, k, omega, phi : nx * ny * nz at cell centres.
//
// Parity status of each routine: see the tests under tests/ (every routine
// below is pinned by at least one closed form, invariant or brute-force check).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

// Parameter block (all SI units).  Field order is this file's own; the
// Python loader mirrors it with ctypes.
struct orc_desc {
  int nx, ny, nz;
  double h;
  double wind_dir_deg, u_ref, z_ref, z0;
  int inflow_loglaw;   // 0: uniform u_ref; 1: log law (Sec. 6.1)
  int ground_noslip;   // 1: no-slip ground; 0: slip ground
  double rho, nu, Cd, a, b, e;          // Sec. 3 footnote + drag equation
  double I, L;                          // inlet turbulence (Sec. 3)
  double C_mu, alpha, beta, sigma, sigma_star, C_lim;  // Table 1
  double cfl, fixed_dt, k_min, omega_min;
  double cg_tol;
  int cg_max_iter;
};

struct orc_stats {
  double dt;
  int cg_iters;
  double cg_rel_residual;
  double div_before;   // ||h div u*||/||u||  before projection
  double div_after;    // ||h div u||/||u||   after projection
};

}  // extern "C"

namespace {

enum Side { INFLOW = 0, OUTFLOW = 1, SLIP = 2, NOSLIP = 3 };

struct Sim {
  orc_desc d;
  int nx, ny, nz;
  double h;
  int side[6];            // x-, x+, y-, y+, z-, z+
  double dirx, diry;      // horizontal wind direction
  std::vector<double> prof;   // inflow speed at cell-centre heights
  double k_in, om_in;
  std::vector<double> u, v, w, p, k, om, phi, c, nut;
  std::vector<double> uh, vh, wh;   // MacCormack forward-step scratch
  double dt;
  orc_stats last;

  size_t nu_() const { return (size_t)(nx + 1) * ny * nz; }
  size_t nv_() const { return (size_t)nx * (ny + 1) * nz; }
  size_t nw_() const { return (size_t)nx * ny * (nz + 1); }
  size_t nc_() const { return (size_t)nx * ny * nz; }
  size_t U(int i, int j, int kk) const { return (size_t)i + (size_t)(nx + 1) * (j + (size_t)ny * kk); }
  size_t V(int i, int j, int kk) const { return (size_t)i + (size_t)nx * (j + (size_t)(ny + 1) * kk); }
  size_t W(int i, int j, int kk) const { return (size_t)i + (size_t)nx * (j + (size_t)ny * kk); }
  size_t C(int i, int j, int kk) const { return (size_t)i + (size_t)nx * (j + (size_t)ny * kk); }
};

// ---------------------------------------------------------------- set-up --

// Log-law inflow (Sec. 6.1): u(z) = (u*/kappa) ln(z/z0) with u* chosen so
// that u(z_ref) = u_ref; clamped at zero below z0.
double inflow_speed(const orc_desc& d, double z) {
  if (!d.inflow_loglaw) return d.u_ref;
  const double kappa = 0.41;
  const double ustar = d.u_ref * kappa / std::log(d.z_ref / d.z0);
  double s = ustar / kappa * std::log(z / d.z0);
  return s > 0.0 ? s : 0.0;
}

void classify_sides(Sim& s) {
  const double th = s.d.wind_dir_deg * M_PI / 180.0;
  s.dirx = std::cos(th);
  s.diry = std::sin(th);
  const double tau = 1e-9;
  // A side is inflow when its inward normal has a positive component along
  // the wind, outflow when negative, slip when the wind is parallel to it.
  const double inward[4] = {s.dirx, -s.dirx, s.diry, -s.diry};
  for (int q = 0; q < 4; ++q)
    s.side[q] = inward[q] > tau ? INFLOW : (inward[q] < -tau ? OUTFLOW : SLIP);
  s.side[4] = s.d.ground_noslip ? NOSLIP : SLIP;
  s.side[5] = SLIP;
}

// Drag coefficient per cell: C_d * a * ((1-phi)/(phi+e))^b  (Sec. 3 footnote
// replacing LAD; drag equation of Sec. 3 "Porosity Model").
double drag_coeff(const orc_desc& d, double ph) {
  double ratio = (1.0 - ph) / (ph + d.e);
  if (ratio < 0.0) ratio = 0.0;
  return d.Cd * d.a * std::pow(ratio, d.b);
}

// ----------------------------------------------------- velocity boundaries --

// Value a boundary face of the normal velocity takes from the BCs of Sec. 3:
// inlet Dirichlet, outlet zero normal derivative (copy of the adjacent
// interior face), walls zero normal velocity.
void apply_velocity_bc(Sim& s) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j) {
      const double inflow = s.prof[kk] * s.dirx;
      // x- side, face i = 0
      switch (s.side[0]) {
        case INFLOW: s.u[s.U(0, j, kk)] = inflow; break;
        case OUTFLOW: s.u[s.U(0, j, kk)] = s.u[s.U(1, j, kk)]; break;
        default: s.u[s.U(0, j, kk)] = 0.0;
      }
      switch (s.side[1]) {
        case INFLOW: s.u[s.U(nx, j, kk)] = inflow; break;
        case OUTFLOW: s.u[s.U(nx, j, kk)] = s.u[s.U(nx - 1, j, kk)]; break;
        default: s.u[s.U(nx, j, kk)] = 0.0;
      }
    }
  for (int kk = 0; kk < nz; ++kk)
    for (int i = 0; i < nx; ++i) {
      const double inflow = s.prof[kk] * s.diry;
      switch (s.side[2]) {
        case INFLOW: s.v[s.V(i, 0, kk)] = inflow; break;
        case OUTFLOW: s.v[s.V(i, 0, kk)] = s.v[s.V(i, 1, kk)]; break;
        default: s.v[s.V(i, 0, kk)] = 0.0;
      }
      switch (s.side[3]) {
        case INFLOW: s.v[s.V(i, ny, kk)] = inflow; break;
        case OUTFLOW: s.v[s.V(i, ny, kk)] = s.v[s.V(i, ny - 1, kk)]; break;
        default: s.v[s.V(i, ny, kk)] = 0.0;
      }
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      s.w[s.W(i, j, 0)] = 0.0;    // ground: no flow through it
      s.w[s.W(i, j, nz)] = 0.0;   // top: slip lid
    }
}

// Ghost value of a velocity component tangential to side `sd`, given the
// adjacent interior value q and the inflow value of that component.
inline double tangential_ghost(int sd_type, double q, double inflow_value) {
  switch (sd_type) {
    case INFLOW: return inflow_value;
    case NOSLIP: return -q;
    default: return q;   // outflow (zero gradient) or slip (mirror)
  }
}

// --------------------------------------------------------------- strain --

// Cell-centred strain-rate tensor S = (grad u + grad u^T)/2 of a staggered
// field: diagonal terms from the two faces of the cell, off-diagonal terms
// from central differences of cell-averaged velocities (one-sided at the
// domain boundary, zero when the extent is 1).  Returns S_ij S_ij.
double strain_sq(const Sim& s, const std::vector<double>& u, const std::vector<double>& v,
                 const std::vector<double>& w, int i, int j, int kk) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  const double h = s.h;
  auto uc = [&](int a, int b, int c) { return 0.5 * (u[s.U(a, b, c)] + u[s.U(a + 1, b, c)]); };
  auto vc = [&](int a, int b, int c) { return 0.5 * (v[s.V(a, b, c)] + v[s.V(a, b + 1, c)]); };
  auto wc = [&](int a, int b, int c) { return 0.5 * (w[s.W(a, b, c)] + w[s.W(a, b, c + 1)]); };
  // derivative of a cell-centred quantity along one axis
  auto dcell = [&](auto f, int axis) {
    int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    int idx = axis == 0 ? i : (axis == 1 ? j : kk);
    if (n < 2) return 0.0;
    int lo = idx > 0 ? idx - 1 : idx;
    int hi = idx < n - 1 ? idx + 1 : idx;
    int a0 = i, b0 = j, c0 = kk, a1 = i, b1 = j, c1 = kk;
    if (axis == 0) { a0 = lo; a1 = hi; }
    if (axis == 1) { b0 = lo; b1 = hi; }
    if (axis == 2) { c0 = lo; c1 = hi; }
    return (f(a1, b1, c1) - f(a0, b0, c0)) / ((hi - lo) * h);
  };
  const double sxx = (u[s.U(i + 1, j, kk)] - u[s.U(i, j, kk)]) / h;
  const double syy = (v[s.V(i, j + 1, kk)] - v[s.V(i, j, kk)]) / h;
  const double szz = (w[s.W(i, j, kk + 1)] - w[s.W(i, j, kk)]) / h;
  const double du_dy = dcell(uc, 1), du_dz = dcell(uc, 2);
  const double dv_dx = dcell(vc, 0), dv_dz = dcell(vc, 2);
  const double dw_dx = dcell(wc, 0), dw_dy = dcell(wc, 1);
  const double sxy = 0.5 * (du_dy + dv_dx);
  const double sxz = 0.5 * (du_dz + dw_dx);
  const double syz = 0.5 * (dv_dz + dw_dy);
  return sxx * sxx + syy * syy + szz * szz + 2.0 * (sxy * sxy + sxz * sxz + syz * syz);
}

// Eddy viscosity of the k-omega closure (Sec. 3): omega~ = max(omega,
// C_lim |S| / sqrt(C_mu/2)), nu_t = k / omega~, then the viscosity limiter
// nu_t <= 1/(2 dt sum h^-2) - nu (von Neumann bound of explicit diffusion;
// h^2/(6 dt) - nu on a uniform grid), clamped at zero.
double eddy_viscosity(const Sim& s, double kv, double omv, double S2, double dt) {
  const double Smag = std::sqrt(S2);
  const double om_t = std::max(omv, s.d.C_lim * Smag / std::sqrt(s.d.C_mu / 2.0));
  double nut = kv / om_t;
  const double lim = s.h * s.h / (6.0 * dt) - s.d.nu;
  nut = std::min(nut, lim);
  return nut > 0.0 ? nut : 0.0;
}

void compute_eddy_viscosity(Sim& s) {
  for (int kk = 0; kk < s.nz; ++kk)
    for (int j = 0; j < s.ny; ++j)
      for (int i = 0; i < s.nx; ++i) {
        const size_t c = s.C(i, j, kk);
        const double S2 = strain_sq(s, s.u, s.v, s.w, i, j, kk);
        s.nut[c] = eddy_viscosity(s, s.k[c], s.om[c], S2, s.dt);
      }
}

// ----------------------------------------------------------------- dt --

double compute_dt(const Sim& s) {
  if (s.d.fixed_dt > 0.0) return s.d.fixed_dt;
  double m = 0.0;
  for (double x : s.u) m = std::max(m, std::fabs(x));
  for (double x : s.v) m = std::max(m, std::fabs(x));
  for (double x : s.w) m = std::max(m, std::fabs(x));
  return s.d.cfl * s.h / m;
}

// ------------------------------------------------------------ advection --

inline double lerp(double a, double b, double t) { return a + t * (b - a); }

// Trilinear sample of a lattice field F of extents (Lx,Ly,Lz) at lattice
// coordinates (a,b,c); coordinates beyond the lattice clamp to it.  Also
// returns the min and max of the 8 lattice values used.
double sample(const std::vector<double>& F, int Lx, int Ly, int Lz, double a, double b, double c,
              double* mn, double* mx) {
  auto axis = [](double x, int n, int* i0, int* i1, double* t) {
    x = std::min(std::max(x, 0.0), (double)(n - 1));
    int f = (int)std::floor(x);
    if (n >= 2) f = std::min(f, n - 2); else f = 0;
    *i0 = f;
    *i1 = std::min(f + 1, n - 1);
    *t = x - f;
  };
  int i0, i1, j0, j1, k0, k1;
  double ta, tb, tc;
  axis(a, Lx, &i0, &i1, &ta);
  axis(b, Ly, &j0, &j1, &tb);
  axis(c, Lz, &k0, &k1, &tc);
  auto at = [&](int i, int j, int k) { return F[(size_t)i + (size_t)Lx * (j + (size_t)Ly * k)]; };
  const double f000 = at(i0, j0, k0), f100 = at(i1, j0, k0);
  const double f010 = at(i0, j1, k0), f110 = at(i1, j1, k0);
  const double f001 = at(i0, j0, k1), f101 = at(i1, j0, k1);
  const double f011 = at(i0, j1, k1), f111 = at(i1, j1, k1);
  if (mn) {
    double lo = f000, hi = f000;
    for (double q : {f100, f010, f110, f001, f101, f011, f111}) { lo = std::min(lo, q); hi = std::max(hi, q); }
    *mn = lo;
    *mx = hi;
  }
  const double x00 = lerp(f000, f100, ta), x10 = lerp(f010, f110, ta);
  const double x01 = lerp(f001, f101, ta), x11 = lerp(f011, f111, ta);
  return lerp(lerp(x00, x10, tb), lerp(x01, x11, tb), tc);
}

// Velocity (in lattice units per step: dt/h * velocity) at a lattice point of
// component `comp` (0=u,1=v,2=w), all three components sampled from the
// time-level-n fields.
void departure_velocity(const Sim& s, int comp, int i, int j, int kk, double out[3]) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  const double sc = s.dt / s.h;
  double U, Vv, Ww;
  if (comp == 0) {   // u point: (i, j+1/2, k+1/2)
    U = s.u[s.U(i, j, kk)];
    Vv = sample(s.v, nx, ny + 1, nz, i - 0.5, j + 0.5, kk, nullptr, nullptr);
    Ww = sample(s.w, nx, ny, nz + 1, i - 0.5, j, kk + 0.5, nullptr, nullptr);
  } else if (comp == 1) {   // v point: (i+1/2, j, k+1/2)
    U = sample(s.u, nx + 1, ny, nz, i + 0.5, j - 0.5, kk, nullptr, nullptr);
    Vv = s.v[s.V(i, j, kk)];
    Ww = sample(s.w, nx, ny, nz + 1, i, j - 0.5, kk + 0.5, nullptr, nullptr);
  } else {   // w point: (i+1/2, j+1/2, k)
    U = sample(s.u, nx + 1, ny, nz, i + 0.5, j, kk - 0.5, nullptr, nullptr);
    Vv = sample(s.v, nx, ny + 1, nz, i, j + 0.5, kk - 0.5, nullptr, nullptr);
    Ww = s.w[s.W(i, j, kk)];
  }
  out[0] = sc * U;
  out[1] = sc * Vv;
  out[2] = sc * Ww;
}

// MacCormack semi-Lagrangian advection (Selle et al. 2008, adopted in
// Sec. 3): forward step phi^ = SL(phi, -dt); backward step phi_v = SL(phi^,
// +dt); phi* = phi^ + (phi - phi_v)/2, clamped to the range of the 8 values
// used by the forward sample.  All components are moved by the velocity of
// time level n.  Only interior faces are written; boundary faces come from
// the BCs afterwards.
void advect(Sim& s) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  struct Comp { std::vector<double>* F; std::vector<double>* Fh; int Lx, Ly, Lz; };
  Comp comps[3] = {{&s.u, &s.uh, nx + 1, ny, nz}, {&s.v, &s.vh, nx, ny + 1, nz}, {&s.w, &s.wh, nx, ny, nz + 1}};
  // forward step on every lattice point (boundary points included: the
  // backward sample may reach them)
  for (int q = 0; q < 3; ++q) {
    Comp& cp = comps[q];
    cp.Fh->assign(cp.F->size(), 0.0);
    for (int kk = 0; kk < cp.Lz; ++kk)
      for (int j = 0; j < cp.Ly; ++j)
        for (int i = 0; i < cp.Lx; ++i) {
          double d3[3];
          departure_velocity(s, q, i, j, kk, d3);
          (*cp.Fh)[(size_t)i + (size_t)cp.Lx * (j + (size_t)cp.Ly * kk)] =
              sample(*cp.F, cp.Lx, cp.Ly, cp.Lz, i - d3[0], j - d3[1], kk - d3[2], nullptr, nullptr);
        }
  }
  // backward step + correction + clamp on interior faces
  std::vector<double> out[3] = {s.u, s.v, s.w};
  for (int q = 0; q < 3; ++q) {
    Comp& cp = comps[q];
    for (int kk = 0; kk < cp.Lz; ++kk)
      for (int j = 0; j < cp.Ly; ++j)
        for (int i = 0; i < cp.Lx; ++i) {
          const bool interior = (q == 0) ? (i > 0 && i < nx) : (q == 1) ? (j > 0 && j < ny) : (kk > 0 && kk < nz);
          if (!interior) continue;
          double d3[3], mn, mx;
          departure_velocity(s, q, i, j, kk, d3);
          const size_t id = (size_t)i + (size_t)cp.Lx * (j + (size_t)cp.Ly * kk);
          const double fwd = sample(*cp.F, cp.Lx, cp.Ly, cp.Lz, i - d3[0], j - d3[1], kk - d3[2], &mn, &mx);
          const double bwd = sample(*cp.Fh, cp.Lx, cp.Ly, cp.Lz, i + d3[0], j + d3[1], kk + d3[2], nullptr, nullptr);
          double r = fwd + 0.5 * ((*cp.F)[id] - bwd);
          r = std::min(std::max(r, mn), mx);
          out[q][id] = r;
        }
  }
  s.u.swap(out[0]);
  s.v.swap(out[1]);
  s.w.swap(out[2]);
}

// ------------------------------------------------------------ diffusion --

// Explicit diffusion (nu + nu_t) lap(u) of each face component (Eq.
// momen_drag), 7-point Laplacian on the component's own lattice.  nu_t at a
// face is the mean of the two cells it separates.  Neighbours along the
// normal axis are faces (boundary faces hold their BC values); neighbours
// beyond a tangential side are ghosts from the BC of that side.
void diffuse(Sim& s) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  const double dth2 = s.dt / (s.h * s.h);
  std::vector<double> un = s.u, vn = s.v, wn = s.w;
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i) {
        const double q = s.u[s.U(i, j, kk)];
        const double inflow = s.prof[kk] * s.dirx;
        const double ym = j > 0 ? s.u[s.U(i, j - 1, kk)] : tangential_ghost(s.side[2], q, inflow);
        const double yp = j < ny - 1 ? s.u[s.U(i, j + 1, kk)] : tangential_ghost(s.side[3], q, inflow);
        const double zm = kk > 0 ? s.u[s.U(i, j, kk - 1)] : tangential_ghost(s.side[4], q, 0.0);
        const double zp = kk < nz - 1 ? s.u[s.U(i, j, kk + 1)] : tangential_ghost(s.side[5], q, 0.0);
        const double lap = s.u[s.U(i - 1, j, kk)] + s.u[s.U(i + 1, j, kk)] + ym + yp + zm + zp - 6.0 * q;
        const double nutf = 0.5 * (s.nut[s.C(i - 1, j, kk)] + s.nut[s.C(i, j, kk)]);
        un[s.U(i, j, kk)] = q + dth2 * (s.d.nu + nutf) * lap;
      }
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double q = s.v[s.V(i, j, kk)];
        const double inflow = s.prof[kk] * s.diry;
        const double xm = i > 0 ? s.v[s.V(i - 1, j, kk)] : tangential_ghost(s.side[0], q, inflow);
        const double xp = i < nx - 1 ? s.v[s.V(i + 1, j, kk)] : tangential_ghost(s.side[1], q, inflow);
        const double zm = kk > 0 ? s.v[s.V(i, j, kk - 1)] : tangential_ghost(s.side[4], q, 0.0);
        const double zp = kk < nz - 1 ? s.v[s.V(i, j, kk + 1)] : tangential_ghost(s.side[5], q, 0.0);
        const double lap = xm + xp + s.v[s.V(i, j - 1, kk)] + s.v[s.V(i, j + 1, kk)] + zm + zp - 6.0 * q;
        const double nutf = 0.5 * (s.nut[s.C(i, j - 1, kk)] + s.nut[s.C(i, j, kk)]);
        vn[s.V(i, j, kk)] = q + dth2 * (s.d.nu + nutf) * lap;
      }
  for (int kk = 1; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double q = s.w[s.W(i, j, kk)];
        const double xm = i > 0 ? s.w[s.W(i - 1, j, kk)] : tangential_ghost(s.side[0], q, 0.0);
        const double xp = i < nx - 1 ? s.w[s.W(i + 1, j, kk)] : tangential_ghost(s.side[1], q, 0.0);
        const double ym = j > 0 ? s.w[s.W(i, j - 1, kk)] : tangential_ghost(s.side[2], q, 0.0);
        const double yp = j < ny - 1 ? s.w[s.W(i, j + 1, kk)] : tangential_ghost(s.side[3], q, 0.0);
        const double lap = xm + xp + ym + yp + s.w[s.W(i, j, kk - 1)] + s.w[s.W(i, j, kk + 1)] - 6.0 * q;
        const double nutf = 0.5 * (s.nut[s.C(i, j, kk - 1)] + s.nut[s.C(i, j, kk)]);
        wn[s.W(i, j, kk)] = q + dth2 * (s.d.nu + nutf) * lap;
      }
  s.u.swap(un);
  s.v.swap(vn);
  s.w.swap(wn);
}

// ----------------------------------------------------------------- drag --

// Forward-Euler porosity drag (Sec. 3): u <- max(0, 1 - dt c U) u with the
// coefficient c averaged from the two adjacent cells and the speed U at the
// face from the face value and 4-point averages of the other components.
void drag(Sim& s) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  const double dt = s.dt;
  std::vector<double> un = s.u, vn = s.v, wn = s.w;
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i) {
        const double q = s.u[s.U(i, j, kk)];
        const double vb = 0.25 * (s.v[s.V(i - 1, j, kk)] + s.v[s.V(i, j, kk)] + s.v[s.V(i - 1, j + 1, kk)] + s.v[s.V(i, j + 1, kk)]);
        const double wb = 0.25 * (s.w[s.W(i - 1, j, kk)] + s.w[s.W(i, j, kk)] + s.w[s.W(i - 1, j, kk + 1)] + s.w[s.W(i, j, kk + 1)]);
        const double speed = std::sqrt(q * q + vb * vb + wb * wb);
        const double cf = 0.5 * (s.c[s.C(i - 1, j, kk)] + s.c[s.C(i, j, kk)]);
        un[s.U(i, j, kk)] = std::max(0.0, 1.0 - dt * cf * speed) * q;
      }
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double q = s.v[s.V(i, j, kk)];
        const double ub = 0.25 * (s.u[s.U(i, j - 1, kk)] + s.u[s.U(i + 1, j - 1, kk)] + s.u[s.U(i, j, kk)] + s.u[s.U(i + 1, j, kk)]);
        const double wb = 0.25 * (s.w[s.W(i, j - 1, kk)] + s.w[s.W(i, j, kk)] + s.w[s.W(i, j - 1, kk + 1)] + s.w[s.W(i, j, kk + 1)]);
        const double speed = std::sqrt(ub * ub + q * q + wb * wb);
        const double cf = 0.5 * (s.c[s.C(i, j - 1, kk)] + s.c[s.C(i, j, kk)]);
        vn[s.V(i, j, kk)] = std::max(0.0, 1.0 - dt * cf * speed) * q;
      }
  for (int kk = 1; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double q = s.w[s.W(i, j, kk)];
        const double ub = 0.25 * (s.u[s.U(i, j, kk - 1)] + s.u[s.U(i + 1, j, kk - 1)] + s.u[s.U(i, j, kk)] + s.u[s.U(i + 1, j, kk)]);
        const double vb = 0.25 * (s.v[s.V(i, j, kk - 1)] + s.v[s.V(i, j + 1, kk - 1)] + s.v[s.V(i, j, kk)] + s.v[s.V(i, j + 1, kk)]);
        const double speed = std::sqrt(ub * ub + vb * vb + q * q);
        const double cf = 0.5 * (s.c[s.C(i, j, kk - 1)] + s.c[s.C(i, j, kk)]);
        wn[s.W(i, j, kk)] = std::max(0.0, 1.0 - dt * cf * speed) * q;
      }
  s.u.swap(un);
  s.v.swap(vn);
  s.w.swap(wn);
}

// ------------------------------------------------------------- pressure --

// Face fluxes of a cell in units of velocity: u(i+1)-u(i)+v(j+1)-v(j)+w(k+1)-w(k)
// (= h div u).
double cell_flux(const Sim& s, int i, int j, int kk) {
  return s.u[s.U(i + 1, j, kk)] - s.u[s.U(i, j, kk)] + s.v[s.V(i, j + 1, kk)] - s.v[s.V(i, j, kk)] +
         s.w[s.W(i, j, kk + 1)] - s.w[s.W(i, j, kk)];
}

// Right-hand side of the pressure Poisson equation (Sec. 3): A p = b with
// b = -(rho h / dt) * (h div u*), so that the projection below makes every
// cell divergence free.
void pressure_rhs(const Sim& s, std::vector<double>& b) {
  b.assign(s.nc_(), 0.0);
  const double sc = -s.d.rho * s.h / s.dt;
  for (int kk = 0; kk < s.nz; ++kk)
    for (int j = 0; j < s.ny; ++j)
      for (int i = 0; i < s.nx; ++i) b[s.C(i, j, kk)] = sc * cell_flux(s, i, j, kk);
}

// Matrix-free 7-point Poisson operator (Sec. 3, BC paragraph): for every
// face of a cell, an interior face contributes (p_c - p_nb); a face on an
// outlet side contributes p_c (the ghost cell beyond it holds p = 0); a face
// on an inlet or wall side contributes nothing (dp/dn = 0).
void apply_A(const Sim& s, const std::vector<double>& x, std::vector<double>& y) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  y.assign(s.nc_(), 0.0);
#pragma omp parallel for schedule(static)
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double pc = x[s.C(i, j, kk)];
        double acc = 0.0;
        auto face = [&](bool inside, int ni, int nj, int nk, int sd) {
          if (inside) acc += pc - x[s.C(ni, nj, nk)];
          else if (s.side[sd] == OUTFLOW) acc += pc;
        };
        face(i > 0, i - 1, j, kk, 0);
        face(i < nx - 1, i + 1, j, kk, 1);
        face(j > 0, i, j - 1, kk, 2);
        face(j < ny - 1, i, j + 1, kk, 3);
        face(kk > 0, i, j, kk - 1, 4);
        face(kk < nz - 1, i, j, kk + 1, 5);
        y[s.C(i, j, kk)] = acc;
      }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double acc = 0.0;
  const long n = (long)a.size();
#pragma omp parallel for reduction(+ : acc) schedule(static)
  for (long i = 0; i < n; ++i) acc += a[i] * b[i];
  return acc;
}

// Plain conjugate gradients (Hestenes-Stiefel) on the SPD system A x = b,
// starting from the given x, stopping at ||r|| <= tol ||b||.
int cg_solve(const Sim& s, const std::vector<double>& b, std::vector<double>& x, double tol, int max_iter,
             double* rel_out) {
  const size_t n = b.size();
  const double bn = std::sqrt(dot(b, b));
  if (bn == 0.0) {
    std::fill(x.begin(), x.end(), 0.0);
    if (rel_out) *rel_out = 0.0;
    return 0;
  }
  std::vector<double> r(n), d(n), q(n);
  apply_A(s, x, q);
  for (size_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  d = r;
  double rr = dot(r, r);
  int it = 0;
  while (std::sqrt(rr) > tol * bn && it < max_iter) {
    apply_A(s, d, q);
    const double alpha = rr / dot(d, q);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n; ++i) {
      x[i] += alpha * d[i];
      r[i] -= alpha * q[i];
    }
    const double rr_new = dot(r, r);
    const double beta = rr_new / rr;
    rr = rr_new;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n; ++i) d[i] = r[i] + beta * d[i];
    ++it;
  }
  if (rel_out) *rel_out = std::sqrt(rr) / bn;
  return it;
}

// Projection (Sec. 3): u -= dt/(rho h) (p_c+ - p_c-) on every face whose
// velocity is not prescribed -- interior faces and faces on outlet sides,
// whose outer neighbour is the p = 0 ghost cell.
void project(Sim& s) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  const double g = s.dt / (s.d.rho * s.h);
  auto P = [&](int i, int j, int kk) { return s.p[s.C(i, j, kk)]; };
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j) {
      for (int i = 1; i < nx; ++i) s.u[s.U(i, j, kk)] -= g * (P(i, j, kk) - P(i - 1, j, kk));
      if (s.side[0] == OUTFLOW) s.u[s.U(0, j, kk)] -= g * (P(0, j, kk) - 0.0);
      if (s.side[1] == OUTFLOW) s.u[s.U(nx, j, kk)] -= g * (0.0 - P(nx - 1, j, kk));
    }
  for (int kk = 0; kk < nz; ++kk)
    for (int i = 0; i < nx; ++i) {
      for (int j = 1; j < ny; ++j) s.v[s.V(i, j, kk)] -= g * (P(i, j, kk) - P(i, j - 1, kk));
      if (s.side[2] == OUTFLOW) s.v[s.V(i, 0, kk)] -= g * (P(i, 0, kk) - 0.0);
      if (s.side[3] == OUTFLOW) s.v[s.V(i, ny, kk)] -= g * (0.0 - P(i, ny - 1, kk));
    }
  for (int kk = 1; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) s.w[s.W(i, j, kk)] -= g * (P(i, j, kk) - P(i, j, kk - 1));
}

// ||h div u||_2 / ||u_cell||_2 over all cells.
double divergence_metric(const Sim& s) {
  double num = 0.0, den = 0.0;
  for (int kk = 0; kk < s.nz; ++kk)
    for (int j = 0; j < s.ny; ++j)
      for (int i = 0; i < s.nx; ++i) {
        const double f = cell_flux(s, i, j, kk);
        num += f * f;
        const double uc = 0.5 * (s.u[s.U(i, j, kk)] + s.u[s.U(i + 1, j, kk)]);
        const double vc = 0.5 * (s.v[s.V(i, j, kk)] + s.v[s.V(i, j + 1, kk)]);
        const double wc = 0.5 * (s.w[s.W(i, j, kk)] + s.w[s.W(i, j, kk + 1)]);
        den += uc * uc + vc * vc + wc * wc;
      }
  return den > 0.0 ? std::sqrt(num / den) : std::sqrt(num);
}

int pressure_solve_project(Sim& s) {
  std::vector<double> b;
  pressure_rhs(s, b);
  s.last.div_before = divergence_metric(s);
  double rel = 0.0;
  s.last.cg_iters = cg_solve(s, b, s.p, s.d.cg_tol, s.d.cg_max_iter, &rel);
  s.last.cg_rel_residual = rel;
  project(s);
  s.last.div_after = divergence_metric(s);
  return s.last.cg_iters;
}

// ----------------------------------------------------------- turbulence --

// k-omega update (Sec. 3, after the projection): forward Euler in time,
// first-order upwind advection with the cell-centre velocity, central
// 7-point diffusion with (nu + sigma* nu_t) for k and (nu + sigma nu_t) for
// omega, sources P_k - C_mu k omega and 2 alpha |S|^2 - beta omega^2, with
// P_k = 2 nu_t |S|^2 and |S|^2 = S_ij S_ij from the projected velocity.
// Ghosts: inlet sides hold the inlet values, every other side is zero
// gradient.  Floors k >= k_min, omega >= omega_min.
void turbulence(Sim& s) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  const double h = s.h, dt = s.dt;
  std::vector<double> kn(s.nc_()), on(s.nc_());
  for (int kk = 0; kk < nz; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t c = s.C(i, j, kk);
        const double kc = s.k[c], oc = s.om[c];
        const double S2 = strain_sq(s, s.u, s.v, s.w, i, j, kk);
        const double nut = eddy_viscosity(s, kc, oc, S2, dt);
        const double vel[3] = {0.5 * (s.u[s.U(i, j, kk)] + s.u[s.U(i + 1, j, kk)]),
                               0.5 * (s.v[s.V(i, j, kk)] + s.v[s.V(i, j + 1, kk)]),
                               0.5 * (s.w[s.W(i, j, kk)] + s.w[s.W(i, j, kk + 1)])};
        // neighbour value of a cell field along axis ax, direction dirn
        auto nb = [&](const std::vector<double>& F, double inlet, int ax, int dirn) {
          int ii = i, jj = j, kq = kk, n, idx, sd;
          if (ax == 0) { ii += dirn; n = nx; idx = ii; sd = dirn < 0 ? 0 : 1; }
          else if (ax == 1) { jj += dirn; n = ny; idx = jj; sd = dirn < 0 ? 2 : 3; }
          else { kq += dirn; n = nz; idx = kq; sd = dirn < 0 ? 4 : 5; }
          if (idx >= 0 && idx < n) return F[s.C(ii, jj, kq)];
          return s.side[sd] == INFLOW ? inlet : F[c];
        };
        double adv_k = 0.0, adv_o = 0.0, lap_k = -6.0 * kc, lap_o = -6.0 * oc;
        for (int ax = 0; ax < 3; ++ax) {
          const double km = nb(s.k, s.k_in, ax, -1), kp = nb(s.k, s.k_in, ax, +1);
          const double om_m = nb(s.om, s.om_in, ax, -1), om_p = nb(s.om, s.om_in, ax, +1);
          lap_k += km + kp;
          lap_o += om_m + om_p;
          if (vel[ax] > 0.0) {
            adv_k += vel[ax] * (kc - km) / h;
            adv_o += vel[ax] * (oc - om_m) / h;
          } else if (vel[ax] < 0.0) {
            adv_k += vel[ax] * (kp - kc) / h;
            adv_o += vel[ax] * (om_p - oc) / h;
          }
        }
        const double Pk = 2.0 * nut * S2;
        const double rk = -adv_k + Pk - s.d.C_mu * kc * oc + (s.d.nu + s.d.sigma_star * nut) * lap_k / (h * h);
        const double ro = -adv_o + 2.0 * s.d.alpha * S2 - s.d.beta * oc * oc + (s.d.nu + s.d.sigma * nut) * lap_o / (h * h);
        kn[c] = std::max(kc + dt * rk, s.d.k_min);
        on[c] = std::max(oc + dt * ro, s.d.omega_min);
      }
  s.k.swap(kn);
  s.om.swap(on);
}

// -------------------------------------------------------------- objective --

// Pedestrian comfort objective: over cells whose centre height lies in
// [1 m, 3 m], sum of max(|u_c| - 4, 0)^2 + max(1 - |u_c|, 0)^2 with the
// cell-centre velocity averaged from the faces.
double objective(const Sim& s, double z_lo, double z_hi, double u_hi, double u_lo) {
  double J = 0.0;
  for (int kk = 0; kk < s.nz; ++kk) {
    const double zc = (kk + 0.5) * s.h;
    if (zc < z_lo || zc > z_hi) continue;
    for (int j = 0; j < s.ny; ++j)
      for (int i = 0; i < s.nx; ++i) {
        const double uc = 0.5 * (s.u[s.U(i, j, kk)] + s.u[s.U(i + 1, j, kk)]);
        const double vc = 0.5 * (s.v[s.V(i, j, kk)] + s.v[s.V(i, j + 1, kk)]);
        const double wc = 0.5 * (s.w[s.W(i, j, kk)] + s.w[s.W(i, j, kk + 1)]);
        const double sp = std::sqrt(uc * uc + vc * vc + wc * wc);
        const double hi = std::max(sp - u_hi, 0.0), lo = std::max(u_lo - sp, 0.0);
        J += hi * hi + lo * lo;
      }
  }
  return J;
}

}  // namespace

// ================================================================ C ABI ==

extern "C" {

enum { ORC_U = 0, ORC_V, ORC_W, ORC_P, ORC_K, ORC_OMEGA, ORC_PHI, ORC_NUT, ORC_C };

void* orc_create(const orc_desc* d) {
  if (!d || d->nx < 2 || d->ny < 2 || d->nz < 1 || !(d->h > 0)) return nullptr;
  Sim* s = new Sim();
  s->d = *d;
  s->nx = d->nx; s->ny = d->ny; s->nz = d->nz; s->h = d->h;
  classify_sides(*s);
  s->prof.resize(d->nz);
  for (int kk = 0; kk < d->nz; ++kk) s->prof[kk] = inflow_speed(*d, (kk + 0.5) * d->h);
  // inlet turbulence (Sec. 3): k = 1.5 (I U_ref)^2, omega = k^(1/2) / (C_mu^(1/4) L)
  s->k_in = 1.5 * (d->I * inflow_speed(*d, d->z_ref)) * (d->I * inflow_speed(*d, d->z_ref));
  s->om_in = std::sqrt(s->k_in) / (std::pow(d->C_mu, 0.25) * d->L);
  s->u.assign(s->nu_(), 0.0); s->v.assign(s->nv_(), 0.0); s->w.assign(s->nw_(), 0.0);
  s->p.assign(s->nc_(), 0.0); s->k.assign(s->nc_(), s->k_in); s->om.assign(s->nc_(), s->om_in);
  s->phi.assign(s->nc_(), 1.0); s->c.assign(s->nc_(), 0.0); s->nut.assign(s->nc_(), 0.0);
  s->dt = 0.0;
  std::memset(&s->last, 0, sizeof(s->last));
  return s;
}

void orc_destroy(void* hnd) { delete (Sim*)hnd; }

int orc_side(void* hnd, int q) { return ((Sim*)hnd)->side[q]; }
double orc_inlet_k(void* hnd) { return ((Sim*)hnd)->k_in; }
double orc_inlet_omega(void* hnd) { return ((Sim*)hnd)->om_in; }
double orc_profile(void* hnd, int kk) { return ((Sim*)hnd)->prof[kk]; }
double orc_drag_coeff(void* hnd, double ph) { return drag_coeff(((Sim*)hnd)->d, ph); }

static std::vector<double>* field_ptr(Sim* s, int f) {
  switch (f) {
    case ORC_U: return &s->u; case ORC_V: return &s->v; case ORC_W: return &s->w;
    case ORC_P: return &s->p; case ORC_K: return &s->k; case ORC_OMEGA: return &s->om;
    case ORC_PHI: return &s->phi; case ORC_NUT: return &s->nut; case ORC_C: return &s->c;
  }
  return nullptr;
}

long orc_field_size(void* hnd, int f) {
  std::vector<double>* p = field_ptr((Sim*)hnd, f);
  return p ? (long)p->size() : -1;
}
int orc_get(void* hnd, int f, double* out) {
  std::vector<double>* p = field_ptr((Sim*)hnd, f);
  if (!p) return -1;
  std::memcpy(out, p->data(), p->size() * sizeof(double));
  return 0;
}
int orc_set(void* hnd, int f, const double* in) {
  Sim* s = (Sim*)hnd;
  std::vector<double>* p = field_ptr(s, f);
  if (!p) return -1;
  std::memcpy(p->data(), in, p->size() * sizeof(double));
  if (f == ORC_PHI)
    for (size_t i = 0; i < s->phi.size(); ++i) s->c[i] = drag_coeff(s->d, s->phi[i]);
  return 0;
}
void orc_set_dt(void* hnd, double dt) { ((Sim*)hnd)->dt = dt; }
double orc_get_dt(void* hnd) { return ((Sim*)hnd)->dt; }

// Sub-steps, each on the current state (exported so that tests can pin them
// one by one).
double orc_compute_dt(void* hnd) { Sim* s = (Sim*)hnd; s->dt = compute_dt(*s); return s->dt; }
void orc_eddy_viscosity(void* hnd) { compute_eddy_viscosity(*(Sim*)hnd); }
void orc_advect(void* hnd) { advect(*(Sim*)hnd); }
void orc_apply_bc(void* hnd) { apply_velocity_bc(*(Sim*)hnd); }
void orc_diffuse(void* hnd) { diffuse(*(Sim*)hnd); }
void orc_drag(void* hnd) { drag(*(Sim*)hnd); }
void orc_pressure_rhs(void* hnd, double* b) {
  Sim* s = (Sim*)hnd;
  std::vector<double> bb;
  pressure_rhs(*s, bb);
  std::memcpy(b, bb.data(), bb.size() * sizeof(double));
}
void orc_apply_A(void* hnd, const double* x, double* y) {
  Sim* s = (Sim*)hnd;
  std::vector<double> xx(x, x + s->nc_()), yy;
  apply_A(*s, xx, yy);
  std::memcpy(y, yy.data(), yy.size() * sizeof(double));
}
int orc_cg(void* hnd, const double* b, double* x, double tol, int max_iter, double* rel) {
  Sim* s = (Sim*)hnd;
  std::vector<double> bb(b, b + s->nc_()), xx(x, x + s->nc_());
  int it = cg_solve(*s, bb, xx, tol, max_iter, rel);
  std::memcpy(x, xx.data(), xx.size() * sizeof(double));
  return it;
}
int orc_pressure_project(void* hnd) { return pressure_solve_project(*(Sim*)hnd); }
void orc_project(void* hnd) { project(*(Sim*)hnd); }
void orc_turbulence(void* hnd) { turbulence(*(Sim*)hnd); }
double orc_divergence(void* hnd) { return divergence_metric(*(Sim*)hnd); }
double orc_objective(void* hnd, double z_lo, double z_hi, double u_hi, double u_lo) {
  return objective(*(Sim*)hnd, z_lo, z_hi, u_hi, u_lo);
}

// Initial state: the inflow profile on every face (Dirichlet values on
// the boundary), one drag step with the CFL time step, the BCs, and one
// projection starting from p = 0.  k and omega take the inlet values.
void orc_init(void* hnd) {
  Sim* s = (Sim*)hnd;
  for (int kk = 0; kk < s->nz; ++kk)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i <= s->nx; ++i) s->u[s->U(i, j, kk)] = s->prof[kk] * s->dirx;
  for (int kk = 0; kk < s->nz; ++kk)
    for (int j = 0; j <= s->ny; ++j)
      for (int i = 0; i < s->nx; ++i) s->v[s->V(i, j, kk)] = s->prof[kk] * s->diry;
  std::fill(s->w.begin(), s->w.end(), 0.0);
  apply_velocity_bc(*s);
  std::fill(s->k.begin(), s->k.end(), s->k_in);
  std::fill(s->om.begin(), s->om.end(), s->om_in);
  std::fill(s->p.begin(), s->p.end(), 0.0);
  s->dt = compute_dt(*s);
  drag(*s);
  apply_velocity_bc(*s);
  pressure_solve_project(*s);
}

// One full time step in the split order of Sec. 3.
int orc_step(void* hnd, orc_stats* st) {
  Sim* s = (Sim*)hnd;
  s->dt = compute_dt(*s);             // a0
  compute_eddy_viscosity(*s);         // a1 (from time level n)
  advect(*s);                         // a2
  apply_velocity_bc(*s);
  diffuse(*s);                        // a3
  apply_velocity_bc(*s);
  drag(*s);                           // a4
  apply_velocity_bc(*s);              // a5
  pressure_solve_project(*s);         // a6-a8 (warm start from p^n)
  turbulence(*s);                     // a9
  s->last.dt = s->dt;
  if (st) *st = s->last;
  return s->last.cg_iters;
}

int orc_run(void* hnd, int nsteps, orc_stats* st) {
  int it = 0;
  for (int n = 0; n < nsteps; ++n) it = orc_step(hnd, st);
  return it;
}

}  // extern "C"
