// Host side of the UrbanFlow RANS step: workspace layout, multigrid
// hierarchy, CUDA-graph capture and the C ABI declared in include/uf.h.
//
// One uf_step replays a CUDA graph captured once per grid (two graphs, one per
// parity of the k/omega ping-pong buffers).  The pressure CG loop sits in a
// conditional WHILE node whose body is {direction + SpMV, update + norm,
// preconditioner}; the update kernel clears the condition when
// ||r|| <= tol ||b||, when the iteration cap is hit or when the residual is not
// finite, so the host never polls inside a step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/uf.h"
#include "grid_base.cuh"
#include "adjoint_kernels.cuh"
#include "advect_fused.cuh"
#include "momentum_fused.cuh"
#include "mg_coarse.cuh"
#include "mesh_kernels.cuh"

namespace {

thread_local std::string g_err;

uf_status fail(uf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define UF_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(UF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int pitch_of(int lx) { return (int)round_up((size_t)lx, 32); }

constexpr int kPartials = 8192;      // doubles per partials buffer
constexpr int kDtBlocks = 1024;
constexpr int kTargetBlocks = 2048;  // blocks of reducing cell kernels
constexpr size_t kTailSmemBudget = 64 * 1024;
constexpr size_t kTailSmemMax = 220 * 1024;   // below the 227 KB per-block opt-in of sm_103a

struct LevelDims {
  int nx, ny, nz, P;
  int fx, fy, fz;   // coarsening factor relative to the finest level
  int cx, cy, cz;   // the next level halves this axis
};

std::vector<LevelDims> mg_hierarchy(int nx, int ny, int nz, int coarse_max) {
  std::vector<LevelDims> L;
  LevelDims d{nx, ny, nz, pitch_of(nx), 1, 1, 1, 0, 0, 0};
  L.push_back(d);
  while (L.size() < 16) {
    LevelDims& f = L.back();
    if (f.nx < 2 && f.ny < 2 && f.nz < 2) break;
    if (L.size() > 1 && (long)f.nx * f.ny * f.nz <= coarse_max) break;
    f.cx = f.nx >= 2; f.cy = f.ny >= 2; f.cz = f.nz >= 2;
    LevelDims c{f.cx ? (f.nx + 1) / 2 : f.nx, f.cy ? (f.ny + 1) / 2 : f.ny, f.cz ? (f.nz + 1) / 2 : f.nz, 0,
                f.fx * (f.cx ? 2 : 1), f.fy * (f.cy ? 2 : 1), f.fz * (f.cz ? 2 : 1), 0, 0, 0};
    c.P = pitch_of(c.nx);
    L.push_back(c);
  }
  return L;
}

// Workspace layout: every buffer 256-byte aligned.
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += round_up(bytes, 256);
    return o;
  }
};

bool desc_valid(const uf_grid_desc* d, std::string* why) {
  if (!d) { *why = "NULL description"; return false; }
  if (d->nx < 2 || d->ny < 2 || d->nz < 1) { *why = "need nx, ny >= 2 and nz >= 1"; return false; }
  if ((long long)d->nx * d->ny * d->nz > (1LL << 31)) { *why = "grid too large"; return false; }
  if (!(d->h > 0)) { *why = "h must be positive"; return false; }
  // every reducing launch keeps at most kPartials blocks (one 32 x 8 tile each)
  if ((long long)((d->nx + 32) / 32) * ((d->ny + 8) / 8) > kPartials / 2) { *why = "nx * ny too large"; return false; }
  if (d->precision != UF_F32 && d->precision != UF_F64) { *why = "precision must be UF_F32 or UF_F64"; return false; }
  if (!(d->u_ref >= 0) || (d->u_ref == 0 && !(d->fixed_dt > 0))) { *why = "u_ref must be > 0 (or fixed_dt > 0)"; return false; }
  if (d->inflow_loglaw && !(d->z0 > 0 && d->z_ref > d->z0)) { *why = "log law needs z_ref > z0 > 0"; return false; }
  if (d->precond < UF_PRECOND_MG || d->precond > UF_PRECOND_AI2) { *why = "unknown preconditioner"; return false; }
  if (d->cg_stop_rule != UF_STOP_RESIDUAL && d->cg_stop_rule != UF_STOP_PAPER) { *why = "unknown stop rule"; return false; }
  if (d->cg_stop_rule == UF_STOP_PAPER && d->precond == UF_PRECOND_MG) {
    *why = "the stop rule of App. A.3 needs the AI, Jacobi or no preconditioner";
    return false;
  }
  if (!(d->cg_tol >= 0) || d->cg_max_iter < 1) { *why = "cg_tol >= 0 and cg_max_iter >= 1 required"; return false; }
  if (d->mg_smoother != UF_SMOOTH_JACOBI && d->mg_smoother != UF_SMOOTH_RBGS && d->mg_smoother != UF_SMOOTH_CHEBY) {
    *why = "unknown smoother";
    return false;
  }
  if (!(d->ai_omega > 0 && d->ai_omega < 2)) { *why = "ai_omega must lie in (0, 2)"; return false; }
  if (!(d->mg_jacobi_omega > 0 && d->mg_jacobi_omega <= 1)) { *why = "mg_jacobi_omega must lie in (0, 1]"; return false; }
  if (d->mg_coarse_max < 1 || d->mg_coarse_max > 1024) { *why = "mg_coarse_max must lie in [1, 1024]"; return false; }
  if (d->mg_transfer != UF_TRANSFER_CONSTANT && d->mg_transfer != UF_TRANSFER_LINEAR) {
    *why = "unknown multigrid transfer";
    return false;
  }
  if (!(d->cfl > 0) && !(d->fixed_dt > 0)) { *why = "cfl or fixed_dt must be positive"; return false; }
  // at least one outlet side, otherwise the pressure operator is singular
  const double th = d->wind_dir_deg * M_PI / 180.0;
  const double cx = std::cos(th), sy = std::sin(th);
  if (!(cx < -1e-9 || cx > 1e-9 || sy < -1e-9 || sy > 1e-9)) { *why = "wind direction undefined"; return false; }
  return true;
}

// Host-side summary of a grid's buffers (offsets into the workspace).
struct Plan;
size_t tail_bytes(const Plan& P, int lt);
void plan_tail(Plan& P, int lt);

struct Plan {
  int T_bytes;
  int nx, ny, nz, Pu, Pc;
  size_t n_u, n_v, n_w, n_c;   // padded element counts
  std::vector<LevelDims> levels;
  int coarse_n;
  // offsets
  size_t u, v, w, uh, vh, wh, ut, vt, wt, u2, v2, w2, k0, k1, o0, o1, cc, phi, nut, p, pd, gd, b, r, r2, z, q, d0, d1;
  int nl;                  // multigrid levels in use (1 without MG)
  int auto_tail_level;     // shallowest level whose tail fits the shared-memory budget
  int min_tail_level;      // shallowest level whose tail fits one block's shared memory
  int tail_level;          // first level run by the shared-memory tail kernel
  size_t tail_smem;        // its dynamic shared memory (bytes)
  size_t tail_cr_off;      // byte offset of the coarsest solve's FP64 right-hand side in it
  std::vector<int> tail_off;
  std::vector<size_t> lr, lx, lt, lu;   // lu: scratch of the cluster V-cycle (levels >= 1)
  size_t prof, dt, dtT, scal, state, partials, ainv, boxes, grad;
  size_t total;
};

Plan make_plan(const uf_grid_desc* d) {
  Plan P;
  P.T_bytes = d->precision == UF_F64 ? 8 : 4;
  P.nx = d->nx; P.ny = d->ny; P.nz = d->nz;
  P.Pu = pitch_of(d->nx + 1);
  P.Pc = pitch_of(d->nx);
  P.n_u = (size_t)P.Pu * d->ny * d->nz;
  P.n_v = (size_t)P.Pc * (d->ny + 1) * d->nz;
  P.n_w = (size_t)P.Pc * d->ny * (d->nz + 1);
  P.n_c = (size_t)P.Pc * d->ny * d->nz;
  Layout L;
  const size_t tb = P.T_bytes;
  P.u = L.take(P.n_u * tb); P.v = L.take(P.n_v * tb); P.w = L.take(P.n_w * tb);
  P.uh = L.take(P.n_u * tb); P.vh = L.take(P.n_v * tb); P.wh = L.take(P.n_w * tb);
  P.ut = L.take(P.n_u * tb); P.vt = L.take(P.n_v * tb); P.wt = L.take(P.n_w * tb);
  P.u2 = L.take(P.n_u * tb); P.v2 = L.take(P.n_v * tb); P.w2 = L.take(P.n_w * tb);
  P.k0 = L.take(P.n_c * tb); P.k1 = L.take(P.n_c * tb);
  P.o0 = L.take(P.n_c * tb); P.o1 = L.take(P.n_c * tb);
  P.cc = L.take(P.n_c * tb); P.phi = L.take(P.n_c * tb); P.nut = L.take(P.n_c * tb);
  P.p = L.take(P.n_c * tb); P.b = L.take(P.n_c * tb); P.r = L.take(P.n_c * tb);
  P.pd = L.take(P.n_c * 2 * tb); P.gd = L.take(P.n_c * 2 * tb);   // pressure store: (hi, lo) pairs or FP64
  P.r2 = L.take(P.n_c * tb);
  P.z = L.take(P.n_c * tb); P.q = L.take(P.n_c * tb);
  P.d0 = L.take(P.n_c * tb); P.d1 = L.take(P.n_c * tb);
  P.levels = mg_hierarchy(d->nx, d->ny, d->nz, d->mg_coarse_max);
  const bool mg = d->precond == UF_PRECOND_MG;
  const size_t nl = mg ? P.levels.size() : 1;
  P.lr.assign(nl, 0); P.lx.assign(nl, 0); P.lt.assign(nl, 0); P.lu.assign(nl, 0);
  for (size_t l = 0; l < nl; ++l) {
    const LevelDims& ld = P.levels[l];
    const size_t n = (size_t)ld.P * ld.ny * ld.nz;
    P.lr[l] = l == 0 ? P.r : L.take(n * tb);
    P.lx[l] = L.take(n * tb);
    P.lt[l] = L.take(n * tb);
    if (l > 0) P.lu[l] = L.take(n * tb);
  }
  const LevelDims& cl = P.levels.back();
  P.coarse_n = mg ? cl.nx * cl.ny * cl.nz : 0;
  // tail: deepest suffix of levels (never the finest) whose three bordered
  // arrays per level fit the shared-memory budget
  P.nl = (int)nl;
  P.auto_tail_level = (int)nl - 1;
  P.min_tail_level = (int)nl - 1;
  if (mg) {
    for (int l = (int)nl - 1; l >= 1; --l) {
      if (tail_bytes(P, l) > kTailSmemBudget) break;
      P.auto_tail_level = l;
    }
    for (int l = (int)nl - 1; l >= 1; --l) {
      if (tail_bytes(P, l) > kTailSmemMax) break;
      P.min_tail_level = l;
    }
  }
  plan_tail(P, P.auto_tail_level);
  P.prof = L.take((size_t)d->nz * tb);
  P.dt = L.take(8);
  P.dtT = L.take(8);
  P.scal = L.take(8 * 8);
  P.state = L.take(sizeof(uf::SolveState));
  P.partials = L.take(sizeof(double) * kPartials * 2);
  P.ainv = L.take(sizeof(double) * (size_t)P.coarse_n * P.coarse_n);
  P.boxes = L.take(sizeof(uf::DesignBox) * uf::MAX_BOXES);
  P.grad = L.take(sizeof(double) * 3 * uf::MAX_BOXES);
  P.total = L.off + 256;
  return P;
}

// Shared memory of a tail starting at level lt: three bordered arrays per level.
size_t tail_bytes(const Plan& P, int lt) {
  size_t n = 0;
  for (int m = lt; m < P.nl; ++m)
    n += 3 * (size_t)(P.levels[m].nx + 2) * (P.levels[m].ny + 2) * (P.levels[m].nz + 2);
  return round_up(n * P.T_bytes, 16) + sizeof(double) * (size_t)P.coarse_n;
}

void plan_tail(Plan& P, int lt) {
  P.tail_level = lt;
  P.tail_off.assign(P.nl, 0);
  if (P.coarse_n == 0) {
    P.tail_smem = 0;
    return;
  }
  size_t off = 0;
  for (int m = lt; m < P.nl; ++m) {
    P.tail_off[m] = (int)off;
    off += 3 * (size_t)(P.levels[m].nx + 2) * (P.levels[m].ny + 2) * (P.levels[m].nz + 2);
  }
  // then the compact FP64 right-hand side of the coarsest solve
  P.tail_cr_off = round_up(off * P.T_bytes, 16);
  P.tail_smem = P.tail_cr_off + sizeof(double) * (size_t)P.coarse_n;
}

// Dense operator of a level (compact order i + nx (j + ny k)).
std::vector<double> dense_level_operator(const LevelDims& ld, double wx, double wy, double wz, int out_mask) {
  const int n = ld.nx * ld.ny * ld.nz;
  std::vector<double> A((size_t)n * n, 0.0);
  auto id = [&](int i, int j, int k) { return i + ld.nx * (j + ld.ny * k); };
  for (int k = 0; k < ld.nz; ++k)
    for (int j = 0; j < ld.ny; ++j)
      for (int i = 0; i < ld.nx; ++i) {
        const int c = id(i, j, k);
        auto face = [&](bool in, int m, double w, int bit) {
          if (in) { A[(size_t)c * n + c] += w; A[(size_t)c * n + m] -= w; }
          else if (out_mask & bit) A[(size_t)c * n + c] += w;
        };
        face(i > 0, i > 0 ? id(i - 1, j, k) : 0, wx, 1);
        face(i < ld.nx - 1, i < ld.nx - 1 ? id(i + 1, j, k) : 0, wx, 2);
        face(j > 0, j > 0 ? id(i, j - 1, k) : 0, wy, 4);
        face(j < ld.ny - 1, j < ld.ny - 1 ? id(i, j + 1, k) : 0, wy, 8);
        face(k > 0, k > 0 ? id(i, j, k - 1) : 0, wz, 16);
        face(k < ld.nz - 1, k < ld.nz - 1 ? id(i, j, k + 1) : 0, wz, 32);
      }
  return A;
}

// Inverse of an SPD matrix by Cholesky factorisation (FP64).
bool spd_inverse(std::vector<double>& A, int n, std::vector<double>& inv) {
  std::vector<double> Lm((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= Lm[(size_t)j * n + k] * Lm[(size_t)j * n + k];
    if (!(s > 0)) return false;
    const double ljj = std::sqrt(s);
    Lm[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= Lm[(size_t)i * n + k] * Lm[(size_t)j * n + k];
      Lm[(size_t)i * n + j] = t / ljj;
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> y(n);
  for (int col = 0; col < n; ++col) {
    for (int i = 0; i < n; ++i) {   // L y = e_col
      double t = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= Lm[(size_t)i * n + k] * y[k];
      y[i] = t / Lm[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {   // L^T x = y
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t -= Lm[(size_t)k * n + i] * inv[(size_t)k * n + col];
      inv[(size_t)i * n + col] = t / Lm[(size_t)i * n + i];
    }
  }
  return true;
}

double inflow_speed(const uf_grid_desc& d, double z) {
  if (!d.inflow_loglaw) return d.u_ref;
  const double kappa = 0.41;
  const double ustar = d.u_ref * kappa / std::log(d.z_ref / d.z0);
  const double s = ustar / kappa * std::log(z / d.z0);
  return s > 0.0 ? s : 0.0;
}

dim3 plane_grid(int lx, int ly, int planes) {
  return dim3((lx + uf::BX - 1) / uf::BX, (ly + uf::BY - 1) / uf::BY, planes);
}

// z-chunking of a cell kernel: returns the grid and the planes per block.
dim3 chunk_grid(int lx, int ly, int lz, int* zc) {
  const int gx = (lx + uf::BX - 1) / uf::BX, gy = (ly + uf::BY - 1) / uf::BY;
  int chunks = std::max(1, std::min(lz, kTargetBlocks / std::max(1, gx * gy)));
  *zc = (lz + chunks - 1) / chunks;
  chunks = (lz + *zc - 1) / *zc;
  return dim3(gx, gy, chunks);
}

}  // namespace

void uf_internal_set_last_error(const char* msg) { g_err = msg ? msg : ""; }

// ======================================================================

namespace {

template <typename T>
class GridImpl final : public uf_grid {
 public:
  uf_grid_desc d;
  Plan P;
  char* ws = nullptr;
  cudaStream_t stream = nullptr, cap = nullptr, cap2 = nullptr;
  uf::StepParams<T> sp;
  std::vector<uf::Level<T>> lv;
  T *u, *v, *w, *uh, *vh, *wh, *ut, *vt, *wt, *u2, *v2, *w2, *kb[2], *ob[2], *cc, *phi, *nut, *p, *b, *r, *r2, *z, *q,
    *d0, *d1, *prof;
  // the pressure p^n and the next solve's guess 2 p^n - p^{n-1} in the
  // pressure store; p holds the solve's correction, then p^{n+1} rounded
  uf::PStore<T> *pd, *gd;
  uf::TailArgs<T> tail;
  T* sol_x = nullptr;   // the solve's unknown (the pressure correction for the step; mu for the adjoint)
  T* sol_b = nullptr;   // its right-hand side
  const uf::PStore<T>* sol_g = nullptr;   // guess of the step's solve (nullptr: warm start in sol_x)
  double *dt, *scal, *partials, *ainv;
  T* dtT;
  uf::SolveState* st;
  cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
  // the same step with the intermediate fields the adjoint tapes (phi^ of
  // the fused advection) written out as well
  cudaGraphExec_t tape_exec[2] = {nullptr, nullptr};
  bool taping = false;
  int unfused = 0;          // tuning: bit mask of fused kernels run as their sub-step kernels
  int advect_zc_tuned = 0;  // tuning: z planes per block of the fused advection (0: automatic)
  int coarse_start_tuned = 0;  // tuning: first MG level of the cluster V-cycle (0 automatic, -1 off)
  int cluster_ctas = 0;        // CTAs per cluster of the coarse V-cycle on this device (0: unavailable)
  cudaGraphExec_t init_exec = nullptr, solve_exec = nullptr;
  int parity = 0;
  bool have_state = false;
  int launches_fixed = 0, launches_per_iter = 0, launches_solve_setup = 0, last_iters = -1;

  ~GridImpl() override {
    for (auto& e : step_exec) if (e) cudaGraphExecDestroy(e);
    for (auto& e : tape_exec) if (e) cudaGraphExecDestroy(e);
    for (auto& e : pool) cudaEventDestroy(e);
    if (init_exec) cudaGraphExecDestroy(init_exec);
    if (solve_exec) cudaGraphExecDestroy(solve_exec);
    if (adj_solve_exec) cudaGraphExecDestroy(adj_solve_exec);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
  }

  template <typename U>
  U* at(size_t off) { return reinterpret_cast<U*>(ws + off); }

  uf_status setup(const uf_grid_desc* desc, void* workspace, cudaStream_t s) {
    d = *desc;
    P = make_plan(desc);
    ws = reinterpret_cast<char*>(round_up(reinterpret_cast<size_t>(workspace), 256));
    stream = s;
    UF_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    UF_CUDA(cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking));
    u = at<T>(P.u); v = at<T>(P.v); w = at<T>(P.w);
    uh = at<T>(P.uh); vh = at<T>(P.vh); wh = at<T>(P.wh);
    ut = at<T>(P.ut); vt = at<T>(P.vt); wt = at<T>(P.wt);
    u2 = at<T>(P.u2); v2 = at<T>(P.v2); w2 = at<T>(P.w2);
    kb[0] = at<T>(P.k0); kb[1] = at<T>(P.k1); ob[0] = at<T>(P.o0); ob[1] = at<T>(P.o1);
    cc = at<T>(P.cc); phi = at<T>(P.phi); nut = at<T>(P.nut); p = at<T>(P.p); b = at<T>(P.b);
    pd = at<uf::PStore<T>>(P.pd); gd = at<uf::PStore<T>>(P.gd);
    sol_x = p;
    sol_b = b;
    sol_g = gd;
    r = at<T>(P.r); r2 = at<T>(P.r2); z = at<T>(P.z); q = at<T>(P.q); d0 = at<T>(P.d0); d1 = at<T>(P.d1);
    prof = at<T>(P.prof);
    dt = at<double>(P.dt); dtT = at<T>(P.dtT); scal = at<double>(P.scal); partials = at<double>(P.partials);
    ainv = at<double>(P.ainv);
    st = at<uf::SolveState>(P.state);
    UF_CUDA(cudaMemsetAsync(ws, 0, P.total - 256, stream));

    // physics parameters
    sp.nx = d.nx; sp.ny = d.ny; sp.nz = d.nz; sp.Pu = P.Pu; sp.Pc = P.Pc;
    const double th = d.wind_dir_deg * M_PI / 180.0;
    const double cx = std::cos(th), sy = std::sin(th), tau = 1e-9;
    const double inward[4] = {cx, -cx, sy, -sy};
    for (int s2 = 0; s2 < 4; ++s2) sp.side[s2] = inward[s2] > tau ? uf::INFLOW : (inward[s2] < -tau ? uf::OUTFLOW : uf::SLIP);
    sp.side[4] = d.ground_noslip ? uf::NOSLIP : uf::SLIP;
    sp.side[5] = uf::SLIP;
    sp.h = (T)d.h; sp.inv_h = (T)(1.0 / d.h);
    sp.dirx = (T)cx; sp.diry = (T)sy;
    sp.rho = (T)d.rho; sp.nu = (T)d.nu;
    sp.C_mu = (T)d.C_mu; sp.alpha = (T)d.alpha; sp.beta = (T)d.beta; sp.sigma = (T)d.sigma;
    sp.sigma_star = (T)d.sigma_star; sp.C_lim = (T)d.C_lim;
    sp.k_min = (T)d.k_min; sp.om_min = (T)d.omega_min;
    const double uin = inflow_speed(d, d.z_ref);
    const double kin = 1.5 * (d.I * uin) * (d.I * uin);
    sp.k_in = (T)kin;
    sp.om_in = (T)(std::sqrt(kin) / (std::pow(d.C_mu, 0.25) * d.L));
    sp.prof = prof;
    sp.dt = dt;
    sp.dtT = dtT;
    std::vector<T> hp(d.nz);
    for (int k = 0; k < d.nz; ++k) hp[k] = (T)inflow_speed(d, (k + 0.5) * d.h);
    UF_CUDA(cudaMemcpyAsync(prof, hp.data(), sizeof(T) * d.nz, cudaMemcpyHostToDevice, stream));
    if (d.fixed_dt > 0) {
      const double fdt = d.fixed_dt;
      const T fdtT = (T)d.fixed_dt;
      UF_CUDA(cudaMemcpyAsync(dt, &fdt, sizeof(double), cudaMemcpyHostToDevice, stream));
      UF_CUDA(cudaMemcpyAsync(dtT, &fdtT, sizeof(T), cudaMemcpyHostToDevice, stream));
    }
    // solver constants
    uf::SolveState s0;
    std::memset(&s0, 0, sizeof(s0));
    const double tol = d.cg_tol > 0 ? d.cg_tol
                       : d.cg_stop_rule == UF_STOP_PAPER ? 1e-5
                       : (d.precision == UF_F64 ? 1e-12 : 1e-7);
    s0.rule = d.cg_stop_rule;
    s0.tol2 = d.cg_stop_rule == UF_STOP_PAPER ? tol : tol * tol;
    s0.max_iter = d.cg_max_iter;
    UF_CUDA(cudaMemcpyAsync(st, &s0, sizeof(s0), cudaMemcpyHostToDevice, stream));
    // porosity 1 everywhere (open air): drag coefficient 0 (already zeroed)
    std::vector<T> ones(P.n_c, T(1));
    UF_CUDA(cudaMemcpyAsync(phi, ones.data(), sizeof(T) * P.n_c, cudaMemcpyHostToDevice, stream));

    // multigrid levels
    int out_mask = 0;
    for (int s2 = 0; s2 < 4; ++s2) if (sp.side[s2] == uf::OUTFLOW) out_mask |= 1 << s2;
    const size_t nl = P.lr.size();
    lv.resize(nl);
    for (size_t l = 0; l < nl; ++l) {
      const LevelDims& ld = P.levels[l];
      uf::Level<T>& L = lv[l];
      L.nx = ld.nx; L.ny = ld.ny; L.nz = ld.nz; L.P = ld.P;
      L.cx = ld.cx; L.cy = ld.cy; L.cz = ld.cz;
      const double cnt = (double)ld.fx * ld.fy * ld.fz;
      L.wx = (T)(cnt / ((double)ld.fx * ld.fx));
      L.wy = (T)(cnt / ((double)ld.fy * ld.fy));
      L.wz = (T)(cnt / ((double)ld.fz * ld.fz));
      L.out_mask = out_mask;
      L.r = at<T>(P.lr[l]); L.x = at<T>(P.lx[l]); L.t = at<T>(P.lt[l]);
      L.r_alt = nullptr;
      // linear transfers below level 1 (the down kernel of such a level
      // keeps its residual in t, which the up leg overwrites later)
      L.lin = d.precond == UF_PRECOND_MG && d.mg_transfer == UF_TRANSFER_LINEAR && l >= 1 && l + 1 < nl;
      L.e = L.lin ? at<T>(P.lu[l]) : nullptr;   // (the cluster V-cycle uses lu only on its own levels)
    }
    if (d.precond == UF_PRECOND_MG) {
      lv[0].r_alt = r2;
      std::memset(&tail, 0, sizeof(tail));
      if (nl > uf::MAX_LEVELS) return fail(UF_ERR_ARG, "too many multigrid levels");
      for (size_t l = 0; l < nl; ++l) { tail.lv[l] = lv[l]; tail.off[l] = P.tail_off[l]; }
      tail.lt = P.tail_level;
      tail.cr_off = (int)P.tail_cr_off;
      tail.nl = (int)nl;
      tail.ainv = ainv;
      tail.n_coarse = P.coarse_n;
      tail.rin = 0;
    }
    UF_CUDA(set_smem_limits());   // every grid: the fused step kernels need more than 48 KB
    if (d.precond == UF_PRECOND_MG) cluster_ctas = probe_cluster();
    if (d.precond == UF_PRECOND_MG) {
      const LevelDims& cl = P.levels.back();
      const uf::Level<T>& L = lv.back();
      std::vector<double> A = dense_level_operator(cl, (double)L.wx, (double)L.wy, (double)L.wz, out_mask);
      std::vector<double> inv;
      if (!spd_inverse(A, P.coarse_n, inv)) return fail(UF_ERR_ARG, "coarsest multigrid operator is not SPD");
      UF_CUDA(cudaMemcpyAsync(ainv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice, stream));
      UF_CUDA(cudaStreamSynchronize(stream));   // host vectors go out of scope
    } else {
      UF_CUDA(cudaStreamSynchronize(stream));
    }
    return UF_OK;
  }

  // ------------------------------------------------------------ recording --
  // Every launch goes through L(): in capture mode it only counts, in the
  // eager profiling mode it also brackets the launch with CUDA events on the
  // launching stream.
  int rec_count = 0;
  bool profiling = false;
  struct Rec {
    std::string name;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;

  cudaEvent_t next_event() {
    if (pool_used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[pool_used++];
  }
  uf_status after_call(uf_status s) override {
#ifdef UF_BOUNDS_CHECK
    uf::BoundsHit h;
    if (uf::bounds_hit_take(stream, &h)) return fail(UF_ERR_BOUNDS, bounds_text(h));
#endif
    return s;
  }

  template <typename F>
  void L(cudaStream_t s, const std::string& name, double bytes, F launch) {
    rec_count++;
    if (!profiling) {
      launch();
      return;
    }
    NvtxRange range(name.c_str());   // eager profiled step: one range per launch
    Rec r{name, bytes, next_event(), next_event()};
    cudaEventRecord(r.a, s);
    launch();
    cudaEventRecord(r.b, s);
    recs.push_back(r);
  }

  double N() const { return (double)d.nx * d.ny * d.nz; }
  double Nl(int l) const { return (double)lv[l].nx * lv[l].ny * lv[l].nz; }
  double tb() const { return (double)sizeof(T); }


  // The dynamic shared-memory limit is an attribute of the kernel, shared by
  // every grid in the process: raise it to the device's opt-in maximum (each
  // launch still asks for its own size), never to one grid's size, which
  // would fail the launches of grids with larger tails.
  cudaError_t set_smem_limits() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && P.tail_smem > (size_t)optin) return cudaErrorInvalidValue;
    auto lim = [&](const void* f) {   // the opt-in maximum less the kernel's static shared memory
      cudaFuncAttributes fa;
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    };
    lim((const void*)uf::k_mg_tail<T, uf::SM_JACOBI>);
    lim((const void*)uf::k_mg_tail<T, uf::SM_RBGS>);
    lim((const void*)uf::k_advect_fused<T>);
    lim((const void*)uf::k_momentum_fused<T>);
    lim((const void*)uf::k_mg_coarse<T, uf::SM_JACOBI>);
    lim((const void*)uf::k_mg_coarse<T, uf::SM_RBGS>);
    return e;
  }

  // z-marching grid of level l: 32 x 8 columns, zc planes (even) per block;
  // by default zc is chosen so that the level still gives a few blocks per
  // SM, else it is the tuned value.  Either way zc is then doubled until the
  // launch has at most kPartials blocks, the capacity of the reduction
  // buffer every block writes one partial sum to.
  int march_zc_tuned[uf::MAX_LEVELS] = {0};
  dim3 march_grid(int l, int* zc) const {
    const uf::Level<T>& L = lv[l];
    const int bx = (L.nx + uf::TX - 1) / uf::TX, by = (L.ny + uf::TY - 1) / uf::TY;
    int z = march_zc_tuned[l];
    if (z <= 0) {
      z = 16;
      while (z > 2 && (long)bx * by * ((L.nz + z - 1) / z) < 456) z /= 2;
    }
    while (z < L.nz && (long long)bx * by * ((L.nz + z - 1) / z) > kPartials) z *= 2;
    *zc = z;
    return dim3(bx, by, (L.nz + z - 1) / z);
  }

  // Fused V-cycle: down kernels to the tail level, the tail, up kernels.
  // mode 1 (inside the CG loop): the finest down kernel also applies the CG
  // update and the convergence test.
  // Weights of the two smoothing sweeps.  Damped Jacobi: both mg_jacobi_omega.
  // Chebyshev: on the 7-point operator, the modes with a high frequency
  // (theta >= pi/2) along at least one axis have eigenvalues of D^-1 A in
  // [1/3, 2]; the weights are the reciprocals of the roots of the degree-2
  // Chebyshev polynomial on that interval, c +- h cos(pi/4), which damp those
  // modes by 1/T2(7/5) = 0.342 per pair of sweeps against (5/7)^2 = 0.510
  // for two sweeps at the best single weight 6/7.
  uf::SmoothW<T> smooth_weights() const {
    double w1 = d.mg_jacobi_omega, w2 = d.mg_jacobi_omega;
    if (d.mg_smoother == UF_SMOOTH_CHEBY) {
      const double lo = 1.0 / 3.0, hi = 2.0, c = 0.5 * (lo + hi), h = 0.5 * (hi - lo), r = std::sqrt(0.5);
      w1 = 1.0 / (c + h * r);
      w2 = 1.0 / (c - h * r);
    }
    uf::SmoothW<T> W;
    W.pa = (T)(w1 + w2 - w1 * w2);
    W.pb = (T)(w1 * w2);
    W.w1 = (T)w1;
    W.w2 = (T)w2;
    return W;
  }

  // CTAs per cluster for the coarse V-cycle: 16 where the device can
  // co-schedule such a cluster of 1024-thread CTAs with the tail's shared
  // memory, else 8, else 0 (per-level kernels only).
  int probe_cluster() {
    for (int ctas : {16, 8}) {
      bool ok = true;
      for (const void* f : {(const void*)uf::k_mg_coarse<T, uf::SM_JACOBI>, (const void*)uf::k_mg_coarse<T, uf::SM_RBGS>}) {
        if (ctas > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) ok = false;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ctas, 1, 1);
        cfg.blockDim = dim3(uf::CT, 1, 1);
        cfg.dynamicSmemBytes = P.tail_smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = ctas;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (ok && (cudaOccupancyMaxActiveClusters(&nclusters, f, &cfg) != cudaSuccess || nclusters < 1)) ok = false;
      }
      cudaGetLastError();   // a refused size is not an error of the grid
      if (ok) return ctas;
    }
    return 0;
  }

  // First level of the cluster V-cycle (below it, the per-level kernels);
  // tail_level when the cluster kernel is not used.
  // Automatic (0) is per-level launches: the cluster runs on 16 SMs at most,
  // and its phases are slower than the per-level kernels on every level but
  // the last one or two before the tail, where the two are about even.
  int coarse_start() const {
    const int lt = P.tail_level;
    if (d.precond != UF_PRECOND_MG || cluster_ctas == 0 || coarse_start_tuned <= 0) return lt;
    return std::min(coarse_start_tuned, lt);
  }

  // Down kernel of level l (mode 1 on the finest level: with the CG update).
  template <int SM>
  void rec_down(cudaStream_t s, int l, int mode, cudaGraphConditionalHandle cond, int use_cond,
                const uf::SmoothW<T>& om) {
    const std::string sl = std::to_string(l);
    int zc;
    const dim3 g = march_grid(l, &zc);
    if (l == 0 && mode == 1)
      L(s, "mg_down_cg_L0", (7 * Nl(0) + Nl(1)) * tb(), [&] {
        uf::k_mg_down<T, SM, true><<<g, uf::FT, 0, s>>>(lv[0], lv[1], om, zc, sol_x, d0, d1, q, partials, st, cond,
                                                       use_cond);
      });
    else
      L(s, "mg_down_L" + sl, (2 * Nl(l) + (lv[l].lin ? Nl(l) : Nl(l + 1))) * tb(), [&] {
        uf::k_mg_down<T, SM, false><<<g, uf::FT, 0, s>>>(lv[l], lv[l + 1], om, zc, nullptr, nullptr, nullptr,
                                                        nullptr, partials, st, cond, 0);
      });
    // linear transfers: the right-hand side of level l + 1 from the stored
    // residual (here also that of the tail's first level: tail.rin = 0)
    if (lv[l].lin && l + 1 <= P.tail_level) {
      const unsigned nb = (unsigned)((4 * Nl(l + 1) + uf::FT - 1) / uf::FT);   // four threads per cell
      L(s, "mg_restrict_L" + std::to_string(l + 1), (Nl(l) + Nl(l + 1)) * tb(), [&] {
        uf::k_restrict_lin<T><<<nb, uf::FT, 0, s>>>(lv[l], lv[l + 1], st);
      });
    }
  }
  // Up kernel of level l (the finest writes z and forms r.z).
  template <int SM>
  void rec_up(cudaStream_t s, int l, int mode, const uf::SmoothW<T>& om) {
    const std::string sl = std::to_string(l);
    // linear transfers: the prolonged correction from level l + 1 (the tail
    // forms that of the level above it)
    if (lv[l].lin && l + 1 < P.tail_level) {
      const unsigned nb = (unsigned)((Nl(l) + uf::FT - 1) / uf::FT);
      L(s, "mg_prolong_L" + sl, (Nl(l) + Nl(l + 1)) * tb(), [&] {
        uf::k_prolong_lin<T><<<nb, uf::FT, 0, s>>>(lv[l], lv[l + 1], st);
      });
    }
    int zc;
    const dim3 g = march_grid(l, &zc);
    if (l == 0)
      L(s, "mg_up_L0", (3 * Nl(0) + Nl(1)) * tb(), [&] {
        uf::k_mg_up<T, SM, true><<<g, uf::FT, 0, s>>>(lv[0], lv[1], om, zc, z, mode, partials, st);
      });
    else
      L(s, "mg_up_L" + sl, (3 * Nl(l) + Nl(l + 1)) * tb(), [&] {
        uf::k_mg_up<T, SM, false><<<g, uf::FT, 0, s>>>(lv[l], lv[l + 1], om, zc, lv[l].t, mode, partials, st);
      });
  }

  template <int SM>
  void rec_vcycle_sm(cudaStream_t s, int mode, cudaGraphConditionalHandle cond, int use_cond) {
    const uf::SmoothW<T> om = smooth_weights();
    const int lt = P.tail_level;
    const int cs = coarse_start();
    for (int l = 0; l < cs; ++l) rec_down<SM>(s, l, mode, cond, use_cond, om);
    if (cs < lt) {   // levels cs .. lt-1 and the tail in one cluster launch
      uf::CoarseArgs<T> ca;
      std::memset(&ca, 0, sizeof(ca));
      for (size_t l = 0; l < lv.size(); ++l) {
        ca.lv[l] = lv[l];
        ca.lu[l] = l > 0 ? at<T>(P.lu[l]) : nullptr;
      }
      ca.cs = cs;
      ca.lt = lt;
      double bytes = (double)P.coarse_n * P.coarse_n * 8 + 2 * Nl(lt) * tb();
      for (int l = cs; l < lt; ++l) bytes += (5 * Nl(l) + 2 * Nl(l + 1)) * tb();
      L(s, "mg_coarse", bytes, [&] {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cluster_ctas, 1, 1);
        cfg.blockDim = dim3(uf::CT, 1, 1);
        cfg.dynamicSmemBytes = P.tail_smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster_ctas;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        uf::TailArgs<T> ta = tail;
        ta.rin = 1;   // the cluster's down legs leave the tail's right-hand side to the tail
        cudaLaunchKernelEx(&cfg, uf::k_mg_coarse<T, SM>, ca, ta, om, (const uf::SolveState*)st);
      });
    } else {
      L(s, "mg_tail", (double)P.coarse_n * P.coarse_n * 8 + 2 * Nl(lt) * tb(),
        [&] { uf::k_mg_tail<T, SM><<<1, uf::TAIL_T, P.tail_smem, s>>>(tail, om, st); });
    }
    for (int l = cs - 1; l >= 0; --l) rec_up<SM>(s, l, mode, om);
  }
  void rec_vcycle(cudaStream_t s, int mode, cudaGraphConditionalHandle cond, int use_cond) {
    if (d.mg_smoother == UF_SMOOTH_RBGS) rec_vcycle_sm<uf::SM_RBGS>(s, mode, cond, use_cond);
    else rec_vcycle_sm<uf::SM_JACOBI>(s, mode, cond, use_cond);
  }

  // Non-multigrid preconditioners: one kernel that also forms r.z (and,
  // under the stop rule of App. A.3, the convergence test); AI2 first forms
  // y = K r in the level's scratch vector.
  void rec_precond(cudaStream_t s, int mode, cudaGraphConditionalHandle cond, int use_cond) {
    const int kind = d.precond == UF_PRECOND_NONE ? 0
                     : d.precond == UF_PRECOND_JACOBI ? 1
                     : d.precond == UF_PRECOND_AI1 ? 2 : 3;
    int zc;
    dim3 g = chunk_grid(lv[0].nx, lv[0].ny, lv[0].nz, &zc);
    if (kind == 3)
      L(s, "precond_ai2_K", 2 * N() * tb(), [&] {
        uf::k_ai2_K<T><<<g, dim3(uf::BX, uf::BY), 0, s>>>(lv[0], (T)d.ai_omega, lv[0].t, zc, st);
      });
    const char* names[4] = {"precond_copy", "precond_jacobi", "precond_ai1", "precond_ai2"};
    L(s, names[kind], 2 * N() * tb(), [&] {
      uf::k_precond_simple<T><<<g, dim3(uf::BX, uf::BY), 0, s>>>(lv[0], kind, (T)d.ai_omega, z, zc, mode, partials, st,
                                                                  cond, use_cond);
    });
  }

  void rec_setup_precond(cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
    if (d.precond == UF_PRECOND_MG) rec_vcycle(s, 0, 0, 0);
    else rec_precond(s, 0, cond, use_cond);
  }

  void rec_cg_init(cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
    int zc;
    dim3 g = chunk_grid(lv[0].nx, lv[0].ny, lv[0].nz, &zc);
    L(s, "cg_init", N() * (3 * tb() + (sol_g ? 2 * tb() : 0.0)), [&] {
      uf::k_cg_init<T><<<g, dim3(uf::BX, uf::BY), 0, s>>>(lv[0], sol_b, sol_x, sol_g, zc, partials, st, cond,
                                                          use_cond);
    });
  }
  void rec_cg_iter(cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
    if (d.precond == UF_PRECOND_MG) {
      int zc;
      const dim3 g = march_grid(0, &zc);
      L(s, "cg_dir_q", 4 * N() * tb(), [&] {
        uf::k_cg_dir_q<T><<<g, uf::FT, 0, s>>>(lv[0], zc, z, d0, d1, q, partials, st);
      });
      rec_vcycle(s, 1, cond, use_cond);
      return;
    }
    int zc;
    dim3 g = chunk_grid(lv[0].nx, lv[0].ny, lv[0].nz, &zc);
    L(s, "cg_direction_spmv", 4 * N() * tb(), [&] {
      uf::k_cg_direction_spmv<T><<<g, dim3(uf::BX, uf::BY), 0, s>>>(lv[0], z, d0, d1, q, zc, partials, st);
    });
    L(s, "cg_update", 6 * N() * tb(), [&] {
      uf::k_cg_update<T><<<g, dim3(uf::BX, uf::BY), 0, s>>>(lv[0], sol_x, d0, d1, q, zc, partials, st, cond, use_cond);
    });
  }

  // Records the CG solve of A p = b (b, bb and the solver state already set
  // by the preceding kernel) as set-up kernels + a conditional while node.
  uf_status rec_solve(cudaStream_t s, cudaGraphConditionalHandle cond, int* setup_count, int* iter_count) {
    const int before = rec_count;
    rec_cg_init(s, cond, 1);
    rec_setup_precond(s, cond, 1);
    *setup_count = rec_count - before;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cgraph;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    UF_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cgraph, &deps, nullptr, &ndeps));
    if (cs != cudaStreamCaptureStatusActive)   // a launch before this point failed
      return fail(UF_ERR_CUDA, std::string("graph capture invalidated: ") + cudaGetErrorString(cudaGetLastError()));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cnode;
    UF_CUDA(cudaGraphAddNode(&cnode, cgraph, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    UF_CUDA(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    UF_CUDA(cudaStreamBeginCaptureToGraph(cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const int b2 = rec_count;
    rec_cg_iter(cap2, cond, 1);
    if (d.precond != UF_PRECOND_MG) rec_precond(cap2, 1, cond, 1);
    *iter_count = rec_count - b2;
    UF_CUDA(cudaStreamEndCapture(cap2, &body));
    return UF_OK;
  }

  // The same solve launched eagerly on `s`; the host polls the convergence
  // flag after every update (profiling mode only).
  uf_status run_solve_eager(cudaStream_t s) {
    int conv = 0;
    rec_cg_init(s, 0, 0);
    UF_CUDA(cudaMemcpyAsync(&conv, &st->converged, sizeof(int), cudaMemcpyDeviceToHost, s));
    UF_CUDA(cudaStreamSynchronize(s));
    if (conv) return UF_OK;
    rec_setup_precond(s, 0, 0);
    for (int it = 0; it < d.cg_max_iter + 1; ++it) {
      rec_cg_iter(s, 0, 0);
      UF_CUDA(cudaMemcpyAsync(&conv, &st->converged, sizeof(int), cudaMemcpyDeviceToHost, s));
      UF_CUDA(cudaStreamSynchronize(s));
      if (conv) break;
      if (d.precond != UF_PRECOND_MG) rec_precond(s, 1, 0, 0);
    }
    return UF_OK;
  }

  uf::AdvectArgs<T> advect_args() {
    uf::AdvectArgs<T> A;
    A.u = u; A.v = v; A.w = w; A.uh = uh; A.vh = vh; A.wh = wh; A.ut = ut; A.vt = vt; A.wt = wt;
    A.Lu = {d.nx + 1, d.ny, d.nz, P.Pu};
    A.Lv = {d.nx, d.ny + 1, d.nz, P.Pc};
    A.Lw = {d.nx, d.ny, d.nz + 1, P.Pc};
    A.nx = d.nx; A.ny = d.ny; A.nz = d.nz;
    A.dtT = dtT;
    A.inv_h = (T)(1.0 / d.h);
    A.nut = nullptr;   // the fused step sets these (eddy viscosity inside the advection)
    A.kf = A.om = nullptr;
    A.sp = sp;
    return A;
  }

  // Fused advection: 32 x 8 columns, zc planes per block (16 unless tuned).
  dim3 advect_grid(int* zc) const {
    const int z = advect_zc_tuned > 0 ? advect_zc_tuned : 16;
    *zc = z;
    return dim3((d.nx + uf::MX - 1) / uf::MX, (d.ny + uf::MY - 1) / uf::MY, (d.nz + z - 1) / z);
  }

  void rec_momentum(cudaStream_t s, const T* kin, const T* oin) {
    const dim3 blk(uf::BX, uf::BY);
    const double faces = 3 * N() * tb(), cells = N() * tb();
    if (!(d.fixed_dt > 0))
      L(s, "cfl_dt", faces, [&] {
        uf::k_cfl_dt<T><<<kDtBlocks, 256, 0, s>>>(u, P.n_u, v, P.n_v, w, P.n_w, d.cfl * d.h, partials, &st->ticket[0], dt, dtT);
      });
    const uf::AdvectArgs<T> A = advect_args();
    const dim3 ga = plane_grid(d.nx + 1, d.ny + 1, 3 * d.nz + 1);
    if (!(unfused & UF_UNFUSED_ADVECT)) {
      // one pass: the eddy viscosity (k, omega -> nu_t) and both MacCormack passes
      uf::AdvectArgs<T> Af = A;
      if (!taping) Af.uh = Af.vh = Af.wh = nullptr;
      Af.nut = nut;
      Af.kf = kin;
      Af.om = oin;
      int zc;
      const dim3 gf = advect_grid(&zc);
      L(s, "advect_fused", 2 * faces + 3 * cells, [&] {
        uf::k_advect_fused<T><<<gf, uf::MT, uf::advect_fused_smem_total<T>(), s>>>(Af, zc);
      });
    } else {
      L(s, "eddy_viscosity", faces + 3 * cells,
        [&] { uf::k_eddy_viscosity<T><<<plane_grid(d.nx, d.ny, d.nz), blk, 0, s>>>(sp, u, v, w, kin, oin, nut); });
      L(s, "advect_forward", 2 * faces, [&] { uf::k_advect_forward<T><<<ga, blk, 0, s>>>(A); });
      L(s, "advect_backward", 3 * faces, [&] { uf::k_advect_backward<T><<<ga, blk, 0, s>>>(A); });
    }
    int zc;
    const dim3 gr = chunk_grid(d.nx, d.ny, d.nz, &zc);
    if (!(unfused & UF_UNFUSED_MOMENTUM)) {
      // one pass: u~, nu_t, c -> u3 (every face), b
      uf::MomentumArgs<T> M;
      M.p = sp; M.ut = ut; M.vt = vt; M.wt = wt; M.nut = nut; M.cc = cc;
      M.u = u; M.v = v; M.w = w; M.b = b;
      M.u2t = taping ? u2 : nullptr; M.v2t = taping ? v2 : nullptr; M.w2t = taping ? w2 : nullptr;
      M.zc = zc; M.partials = partials; M.st = st;
      L(s, "momentum_fused", faces + 2 * cells + faces + cells, [&] {
        uf::k_momentum_fused<T><<<gr, uf::MT, uf::momentum_fused_smem<T>(), s>>>(M);
      });
    } else {
      L(s, "diffuse", 2 * faces + cells, [&] { uf::k_diffuse<T><<<ga, blk, 0, s>>>(sp, ut, vt, wt, nut, u2, v2, w2); });
      L(s, "drag_bc", 2 * faces + cells, [&] { uf::k_drag_bc<T><<<ga, blk, 0, s>>>(sp, u2, v2, w2, cc, u, v, w); });
      L(s, "pressure_rhs", faces + cells,
        [&] { uf::k_pressure_rhs<T><<<gr, blk, 0, s>>>(sp, u, v, w, b, zc, partials, st); });
    }
  }

  void rec_post(cudaStream_t s, const T* kin, const T* oin, T* kout, T* oout) {
    const dim3 blk(uf::BX, uf::BY);
    const double faces = 3 * N() * tb(), cells = N() * tb();
    L(s, "pressure_commit", N() * 10 * tb(),
      [&] { uf::k_pressure_commit<T><<<plane_grid(d.nx, d.ny, d.nz), blk, 0, s>>>(sp, p, pd, gd, st); });
    L(s, "project", 2 * faces + 2 * cells,
      [&] { uf::k_project_cells<T><<<plane_grid(d.nx + 1, d.ny + 1, d.nz), blk, 0, s>>>(sp, pd, u, v, w); });
    L(s, "turbulence", faces + 4 * cells,
      [&] { uf::k_turbulence<T><<<plane_grid(d.nx, d.ny, d.nz), blk, 0, s>>>(sp, u, v, w, kin, oin, kout, oout); });
  }

  // One step launched eagerly with per-launch events; aggregates by name.
  uf_status profile_step(uf_kernel_time* out, int cap_n, int* count, uf_step_stats* stats) override {
    if (!have_state) return fail(UF_ERR_STATE, "no state: call uf_init_state or uf_set_state first");
    recs.clear();
    pool_used = 0;
    profiling = true;
    rec_count = 0;
    const int par = parity;
    rec_momentum(stream, kb[par], ob[par]);
    uf_status s = run_solve_eager(stream);
    if (s == UF_OK) rec_post(stream, kb[par], ob[par], kb[1 - par], ob[1 - par]);
    profiling = false;
    if (s != UF_OK) return s;
    UF_CUDA(cudaStreamSynchronize(stream));
    UF_CUDA(cudaGetLastError());
    parity ^= 1;
    std::vector<uf_kernel_time> agg;
    for (const Rec& r : recs) {
      float ms = 0;
      UF_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      auto it = std::find_if(agg.begin(), agg.end(), [&](const uf_kernel_time& k) { return r.name == k.name; });
      if (it == agg.end()) {
        uf_kernel_time k;
        std::memset(&k, 0, sizeof(k));
        std::snprintf(k.name, sizeof(k.name), "%s", r.name.c_str());
        k.bytes_per_launch = r.bytes;
        agg.push_back(k);
        it = agg.end() - 1;
      }
      it->launches += 1;
      it->total_ms += ms;
    }
    if (count) *count = (int)agg.size();
    if (out)
      for (int i = 0; i < std::min(cap_n, (int)agg.size()); ++i) out[i] = agg[i];
    last_profile_launches = (int)recs.size();
    return check_device(stats);
  }
  int last_profile_launches = 0;

  // ------------------------------------------------------------ adjoint ---
  // Workspace of uf_adjoint_run (caller-allocated): per-step tapes of one
  // checkpoint segment, the checkpoints, the final state and the adjoint
  // arrays.  Offsets in elements of T, every array 64-element aligned.
  struct AdjLayout {
    size_t faceN, cellN, cellD, slot, ckpt, total;
    int C, nseg;
    size_t tape0, ckpt0, fin, lam;
    // offsets inside one tape slot; a slot starts with a checkpoint
    // (faces | k | omega | p^n | guess) so that save_state() fills its head
    size_t s_nut, s_uh, s_ut, s_u2, s_u1;
  };
  static size_t a64(size_t n) { return (n + 63) / 64 * 64; }
  size_t face_set() const { return a64(P.n_u) + a64(P.n_v) + a64(P.n_w); }
  AdjLayout adj_layout(int nsteps, int C) const {
    AdjLayout A;
    A.faceN = face_set();
    A.cellN = a64(P.n_c);
    A.C = C;
    A.nseg = (nsteps + C - 1) / C;
    A.cellD = A.cellN * (sizeof(uf::PStore<T>) / sizeof(T));   // a pressure-store cell array in units of T
    A.ckpt = A.faceN + 2 * A.cellN + 2 * A.cellD;              // faces, k, omega, p^n, guess
    A.s_nut = A.ckpt;
    A.s_uh = A.s_nut + A.cellN;
    A.s_ut = A.s_uh + A.faceN;
    A.s_u2 = A.s_ut + A.faceN;
    A.s_u1 = A.s_u2 + A.faceN;
    A.slot = A.s_u1 + A.faceN;
    A.tape0 = 0;
    A.ckpt0 = A.tape0 + (size_t)C * A.slot;
    A.fin = A.ckpt0 + (size_t)A.nseg * A.ckpt;
    A.lam = A.fin + A.ckpt;
    A.total = A.lam + 5 * A.faceN + 10 * A.cellN;
    return A;
  }
  size_t adjoint_bytes(int nsteps, int C) override {
    if (nsteps < 1 || C < 1) return 0;
    return adj_layout(nsteps, C).total * sizeof(T) + 256;
  }
  struct FaceSet {
    T *u, *v, *w;
  };
  FaceSet faces_at(T* base) const {
    FaceSet f;
    f.u = base;
    f.v = base + a64(P.n_u);
    f.w = f.v + a64(P.n_v);
    return f;
  }
  cudaError_t copy_faces(FaceSet dst, const T* su, const T* sv, const T* sw) {
    cudaError_t e = cudaMemcpyAsync(dst.u, su, P.n_u * sizeof(T), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst.v, sv, P.n_v * sizeof(T), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst.w, sw, P.n_w * sizeof(T), cudaMemcpyDeviceToDevice, stream);
    return e;
  }
  cudaError_t copy_cell(T* dst, const T* src) {
    return cudaMemcpyAsync(dst, src, P.n_c * sizeof(T), cudaMemcpyDeviceToDevice, stream);
  }
  cudaError_t copy_cell_ps(uf::PStore<T>* dst, const uf::PStore<T>* src) {
    return cudaMemcpyAsync(dst, src, P.n_c * sizeof(uf::PStore<T>), cudaMemcpyDeviceToDevice, stream);
  }
  // p (grid precision) -> the pressure store with no history, or back
  cudaError_t pressure_sync(int to_store) {
    uf::k_pressure_sync<T><<<(unsigned)((P.n_c + 255) / 256), 256, 0, stream>>>(p, pd, gd, P.n_c, to_store);
    return cudaGetLastError();
  }
  // checkpoint layout: faces | k | omega | p^n | the next solve's guess (both in the pressure store)
  uf::PStore<T>* ckpt_pressure(T* slot, const AdjLayout& A, int which) const {
    return reinterpret_cast<uf::PStore<T>*>(slot + A.faceN + 2 * A.cellN + (size_t)which * A.cellD);
  }
  cudaError_t save_state(T* slot, const AdjLayout& A) {
    FaceSet f = faces_at(slot);
    cudaError_t e = copy_faces(f, u, v, w);
    if (e == cudaSuccess) e = copy_cell(slot + A.faceN, kb[parity]);
    if (e == cudaSuccess) e = copy_cell(slot + A.faceN + A.cellN, ob[parity]);
    if (e == cudaSuccess) e = copy_cell_ps(ckpt_pressure(slot, A, 0), pd);
    if (e == cudaSuccess) e = copy_cell_ps(ckpt_pressure(slot, A, 1), gd);
    return e;
  }
  cudaError_t load_state(const T* slot, const AdjLayout& A) {
    parity = 0;
    FaceSet f = faces_at(const_cast<T*>(slot));
    cudaError_t e = cudaMemcpyAsync(u, f.u, P.n_u * sizeof(T), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, f.v, P.n_v * sizeof(T), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, f.w, P.n_w * sizeof(T), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = copy_cell(kb[0], slot + A.faceN);
    if (e == cudaSuccess) e = copy_cell(ob[0], slot + A.faceN + A.cellN);
    T* sl = const_cast<T*>(slot);
    if (e == cudaSuccess) e = copy_cell_ps(pd, ckpt_pressure(sl, A, 0));
    if (e == cudaSuccess) e = copy_cell_ps(gd, ckpt_pressure(sl, A, 1));
    if (e == cudaSuccess) e = pressure_sync(0);
    return e;
  }

  cudaGraphExec_t adj_solve_exec = nullptr;
  T* adj_mu = nullptr;
  T* adj_b = nullptr;

  // Adjoint arrays inside the workspace (after the tapes and checkpoints).
  struct AdjArrays {
    FaceSet L0, L1, Lt, L2, Lh;   // adjoints: step input, step output, advected, diffused, forward SL
    T *lk0, *lk1, *lo0, *lo1, *lnut, *lc, *mu, *badj, *lphi, *mu_prev;
  };
  AdjArrays adj_arrays(T* base, const AdjLayout& A) const {
    AdjArrays R;
    T* lam = base + A.lam;
    R.L0 = faces_at(lam);
    R.L1 = faces_at(lam + A.faceN);
    R.Lt = faces_at(lam + 2 * A.faceN);
    R.L2 = faces_at(lam + 3 * A.faceN);
    R.Lh = faces_at(lam + 4 * A.faceN);
    T* cells = lam + 5 * A.faceN;
    R.lk0 = cells; R.lk1 = cells + A.cellN; R.lo0 = cells + 2 * A.cellN; R.lo1 = cells + 3 * A.cellN;
    R.lnut = cells + 4 * A.cellN; R.lc = cells + 5 * A.cellN; R.mu = cells + 6 * A.cellN;
    R.badj = cells + 7 * A.cellN; R.lphi = cells + 8 * A.cellN; R.mu_prev = cells + 9 * A.cellN;
    return R;
  }

  // The adjoint pressure solve: the step's MG-PCG captured with (badj -> mu)
  // in place of (b -> p).
  uf_status ensure_adj_solve(T* mu, T* badj) {
    if (adj_solve_exec && adj_mu == mu && adj_b == badj) return UF_OK;
    if (adj_solve_exec) cudaGraphExecDestroy(adj_solve_exec);
    adj_solve_exec = nullptr;
    sol_x = mu;
    sol_b = badj;
    sol_g = nullptr;
    int nf, ns, ni;
    auto pre = [&](cudaStream_t s2) {
      int zc;
      dim3 g = chunk_grid(d.nx, d.ny, d.nz, &zc);
      uf::k_solve_reset<T><<<g, dim3(uf::BX, uf::BY), 0, s2>>>(lv[0], badj, zc, partials, st);
      rec_count++;
    };
    uf_status s = capture(&adj_solve_exec, pre, [&](cudaStream_t) {}, &nf, &ns, &ni);
    sol_x = p;
    sol_b = b;
    sol_g = gd;
    if (s != UF_OK) return s;
    adj_mu = mu;
    adj_b = badj;
    return UF_OK;
  }

  // Runs one step from the current state and tapes it into slot t.
  uf_status tape_step(T* t, const AdjLayout& A) {
    uf_status bs = build_tape_graphs();
    if (bs != UF_OK) return bs;
    UF_CUDA(save_state(t, A));
    UF_CUDA(cudaGraphLaunch(tape_exec[parity], stream));
    parity ^= 1;
    UF_CUDA(copy_cell(t + A.s_nut, nut));
    UF_CUDA(copy_faces(faces_at(t + A.s_uh), uh, vh, wh));
    UF_CUDA(copy_faces(faces_at(t + A.s_ut), ut, vt, wt));
    UF_CUDA(copy_faces(faces_at(t + A.s_u2), u2, v2, w2));
    UF_CUDA(copy_faces(faces_at(t + A.s_u1), u, v, w));
    return UF_OK;
  }

  // Transpose of the taped step in slot t: from the adjoint of its output
  // (R.L1, R.lk1, R.lo1) to the adjoint of its input (R.L0, R.lk0, R.lo0);
  // dJ/dc accumulates in R.lc.
  uf_status reverse_step(const T* t, const AdjLayout& A, const AdjArrays& R) {
    const size_t faceB = A.faceN * sizeof(T), cellB = A.cellN * sizeof(T);
    const dim3 blk(uf::BX, uf::BY);
    const dim3 gc = plane_grid(d.nx, d.ny, d.nz);
    const dim3 ga = plane_grid(d.nx + 1, d.ny + 1, 3 * d.nz + 1);
    const FaceSet U0 = faces_at(const_cast<T*>(t));
    const T* K0 = t + A.faceN;
    const T* O0 = t + A.faceN + A.cellN;
    const T* NUT = t + A.s_nut;
    const FaceSet UH = faces_at(const_cast<T*>(t) + A.s_uh);
    const FaceSet UT = faces_at(const_cast<T*>(t) + A.s_ut);
    const FaceSet U2 = faces_at(const_cast<T*>(t) + A.s_u2);
    const FaceSet U1 = faces_at(const_cast<T*>(t) + A.s_u1);
    UF_CUDA(cudaMemsetAsync(R.L0.u, 0, faceB, stream));
    UF_CUDA(cudaMemsetAsync(R.Lt.u, 0, 3 * faceB, stream));   // Lt, L2, Lh are contiguous
    UF_CUDA(cudaMemsetAsync(R.lk0, 0, cellB, stream));
    UF_CUDA(cudaMemsetAsync(R.lo0, 0, cellB, stream));
    UF_CUDA(cudaMemsetAsync(R.lnut, 0, cellB, stream));
    // a9^T: k-omega update
    uf::k_turbulence_adj<T><<<gc, blk, 0, stream>>>(sp, U1.u, U1.v, U1.w, K0, O0, R.lk1, R.lo1, R.lk0, R.lo0, R.L1.u,
                                                    R.L1.v, R.L1.w);
    // a8^T: projection (A symmetric: the same MG-PCG)
    uf::k_proj_adj_rhs<T><<<gc, blk, 0, stream>>>(sp, R.L1.u, R.L1.v, R.L1.w, R.badj, R.mu, R.mu_prev);
    UF_CUDA(cudaGraphLaunch(adj_solve_exec, stream));
    uf::k_proj_adj_apply<T><<<ga, blk, 0, stream>>>(sp, R.mu, R.L1.u, R.L1.v, R.L1.w);
    // a4/a5^T: drag and velocity BCs
    uf::k_drag_bc_adj<T><<<ga, blk, 0, stream>>>(sp, U2.u, U2.v, U2.w, cc, R.L1.u, R.L1.v, R.L1.w, R.L2.u, R.L2.v,
                                                 R.L2.w, R.lc);
    // a3^T: diffusion
    uf::k_diffuse_adj<T><<<ga, blk, 0, stream>>>(sp, UT.u, UT.v, UT.w, NUT, R.L2.u, R.L2.v, R.L2.w, R.Lt.u, R.Lt.v,
                                                 R.Lt.w, R.lnut);
    // a2^T: MacCormack advection
    uf::AdvectArgs<T> Aa = advect_args();
    Aa.u = U0.u; Aa.v = U0.v; Aa.w = U0.w;
    Aa.uh = UH.u; Aa.vh = UH.v; Aa.wh = UH.w;
    uf::AdvectAdj<T> Ja{R.Lt.u, R.Lt.v, R.Lt.w, R.Lh.u, R.Lh.v, R.Lh.w, R.L0.u, R.L0.v, R.L0.w};
    uf::k_advect_backward_adj<T><<<ga, blk, 0, stream>>>(Aa, Ja);
    uf::k_advect_forward_adj<T><<<ga, blk, 0, stream>>>(Aa, Ja);
    // a1^T: eddy viscosity
    uf::k_eddy_viscosity_adj<T><<<gc, blk, 0, stream>>>(sp, U0.u, U0.v, U0.w, K0, O0, R.lnut, R.lk0, R.lo0, R.L0.u,
                                                        R.L0.v, R.L0.w);
    UF_CUDA(cudaGetLastError());
    return UF_OK;
  }

  uf_status adjoint_run(void* wsp, size_t bytes, int nsteps, int C, double z_lo, double z_hi, double u_hi, double u_lo,
                        void* dJ_dphi, double* J_out) override {
    uf_objective_desc od;
    std::memset(&od, 0, sizeof(od));
    od.kind = UF_OBJ_COMFORT;
    od.z_lo = z_lo; od.z_hi = z_hi; od.u_hi = u_hi; od.u_lo = u_lo;
    return adjoint_run_ex(wsp, bytes, nsteps, C, &od, dJ_dphi, J_out);
  }

  uf_status adjoint_run_ex(void* wsp, size_t bytes, int nsteps, int C, const uf_objective_desc* od, void* dJ_dphi,
                           double* J_out) override {
    uf_status s0 = check_objective(od);
    if (s0 != UF_OK) return s0;
    if (!(d.fixed_dt > 0)) return fail(UF_ERR_ARG, "uf_adjoint_run needs a fixed time step (fixed_dt > 0)");
    if (!have_state) return fail(UF_ERR_STATE, "no state: call uf_init_state or uf_set_state first");
    if (!wsp || nsteps < 1 || C < 1) return fail(UF_ERR_ARG, "need a workspace, nsteps >= 1 and ckpt_every >= 1");
    if (bytes < adjoint_bytes(nsteps, C)) return fail(UF_ERR_NOMEM, "adjoint workspace smaller than uf_adjoint_workspace_bytes()");
    const AdjLayout A = adj_layout(nsteps, C);
    T* base = reinterpret_cast<T*>(round_up(reinterpret_cast<size_t>(wsp), 256));
    uf_status s = build_step_graphs();
    if (s != UF_OK) return s;
    AdjArrays R = adj_arrays(base, A);
    s = ensure_adj_solve(R.mu, R.badj);
    if (s != UF_OK) return s;
    UF_CUDA(cudaMemsetAsync(base + A.lam, 0, (5 * A.faceN + 10 * A.cellN) * sizeof(T), stream));
    // 1. forward sweep with checkpoints every C steps; the last segment is
    //    taped on the way, so the reverse sweep need not recompute it
    const int last0 = (A.nseg - 1) * C;
    for (int n = 0; n < nsteps; ++n) {
      if (n % C == 0) UF_CUDA(save_state(base + A.ckpt0 + (size_t)(n / C) * A.ckpt, A));
      if (n >= last0) {
        s = tape_step(base + A.tape0 + (size_t)(n - last0) * A.slot, A);
        if (s != UF_OK) return s;
      } else {
        UF_CUDA(cudaGraphLaunch(step_exec[parity], stream));
        parity ^= 1;
      }
    }
    UF_CUDA(save_state(base + A.fin, A));
    s = check_device(nullptr);
    if (s != UF_OK) return s;
    double J = 0.0;
    std::vector<double> means;
    s = objective_ex_means(od, &J, &means);
    if (s != UF_OK) return s;
    if (J_out) *J_out = J;
    // 2. seed: dJ/du of the final state
    s = seed_objective(od, means, R.L1);
    if (s != UF_OK) return s;
    // 3. reverse sweep, one checkpoint segment at a time
    for (int seg = A.nseg - 1; seg >= 0; --seg) {
      const int n0 = seg * C, n1 = std::min(nsteps, n0 + C);
      if (seg < A.nseg - 1) {
        UF_CUDA(load_state(base + A.ckpt0 + (size_t)seg * A.ckpt, A));
        for (int n = n0; n < n1; ++n) {   // recompute the segment, taping each step
          s = tape_step(base + A.tape0 + (size_t)(n - n0) * A.slot, A);
          if (s != UF_OK) return s;
        }
      }
      for (int n = n1 - 1; n >= n0; --n) {
        s = reverse_step(base + A.tape0 + (size_t)(n - n0) * A.slot, A, R);
        if (s != UF_OK) return s;
        std::swap(R.L0, R.L1);
        std::swap(R.lk0, R.lk1);
        std::swap(R.lo0, R.lo1);
      }
      s = check_device(nullptr);
      if (s != UF_OK) return s;
    }
    // 4. dJ/dphi = dJ/dc dc/dphi; leave the grid at the final state
    uf::k_dphi<T><<<(unsigned)((P.n_c + 255) / 256), 256, 0, stream>>>(phi, R.lc, R.lphi, P.n_c, d.Cd, d.a, d.b, d.e);
    UF_CUDA(cudaGetLastError());
    UF_CUDA(load_state(base + A.fin, A));
    if (dJ_dphi) {
      s = copy_out(dJ_dphi, R.lphi, d.nx, d.ny, d.nz, P.Pc);
      if (s != UF_OK) return s;
    }
    return check_device(nullptr);
  }

  // Vector-Jacobian product of one step at the current state; the state is
  // restored afterwards.  Order of the five arrays: u, v, w, k, omega.
  uf_status step_vjp(void* wsp, size_t bytes, const void* const* lam_out, void* const* lam_in, void* lam_phi) override {
    if (!(d.fixed_dt > 0)) return fail(UF_ERR_ARG, "uf_step_vjp needs a fixed time step (fixed_dt > 0)");
    if (!have_state) return fail(UF_ERR_STATE, "no state: call uf_init_state or uf_set_state first");
    if (!wsp || !lam_out || !lam_in) return fail(UF_ERR_ARG, "NULL workspace or cotangent arrays");
    for (int q = 0; q < 5; ++q)
      if (!lam_out[q] || !lam_in[q]) return fail(UF_ERR_ARG, "NULL cotangent array");
    if (bytes < adjoint_bytes(1, 1)) return fail(UF_ERR_NOMEM, "workspace smaller than uf_adjoint_workspace_bytes(g, 1, 1)");
    const AdjLayout A = adj_layout(1, 1);
    T* base = reinterpret_cast<T*>(round_up(reinterpret_cast<size_t>(wsp), 256));
    uf_status s = build_step_graphs();
    if (s != UF_OK) return s;
    AdjArrays R = adj_arrays(base, A);
    s = ensure_adj_solve(R.mu, R.badj);
    if (s != UF_OK) return s;
    UF_CUDA(cudaMemsetAsync(base + A.lam, 0, (5 * A.faceN + 10 * A.cellN) * sizeof(T), stream));
    T* keep = base + A.ckpt0;
    UF_CUDA(save_state(keep, A));
    T* t = base + A.tape0;
    s = tape_step(t, A);
    if (s == UF_OK) s = copy_in(R.L1.u, d.nx + 1, d.ny, d.nz, P.Pu, lam_out[0]);
    if (s == UF_OK) s = copy_in(R.L1.v, d.nx, d.ny + 1, d.nz, P.Pc, lam_out[1]);
    if (s == UF_OK) s = copy_in(R.L1.w, d.nx, d.ny, d.nz + 1, P.Pc, lam_out[2]);
    if (s == UF_OK) s = copy_in(R.lk1, d.nx, d.ny, d.nz, P.Pc, lam_out[3]);
    if (s == UF_OK) s = copy_in(R.lo1, d.nx, d.ny, d.nz, P.Pc, lam_out[4]);
    if (s == UF_OK) s = reverse_step(t, A, R);
    if (s == UF_OK) s = copy_out(lam_in[0], R.L0.u, d.nx + 1, d.ny, d.nz, P.Pu);
    if (s == UF_OK) s = copy_out(lam_in[1], R.L0.v, d.nx, d.ny + 1, d.nz, P.Pc);
    if (s == UF_OK) s = copy_out(lam_in[2], R.L0.w, d.nx, d.ny, d.nz + 1, P.Pc);
    if (s == UF_OK) s = copy_out(lam_in[3], R.lk0, d.nx, d.ny, d.nz, P.Pc);
    if (s == UF_OK) s = copy_out(lam_in[4], R.lo0, d.nx, d.ny, d.nz, P.Pc);
    if (s == UF_OK && lam_phi) {
      uf::k_dphi<T><<<(unsigned)((P.n_c + 255) / 256), 256, 0, stream>>>(phi, R.lc, R.lphi, P.n_c, d.Cd, d.a, d.b,
                                                                         d.e);
      UF_CUDA(cudaGetLastError());
      s = copy_out(lam_phi, R.lphi, d.nx, d.ny, d.nz, P.Pc);
    }
    UF_CUDA(load_state(keep, A));   // the grid keeps its state
    if (s != UF_OK) return s;
    return check_device(nullptr);
  }

  // ---------------------------------------------------- design -> phi ----
  uf_status upload_boxes(int nbox, const double* boxes, const double* theta) {
    if (nbox < 1 || nbox > uf::MAX_BOXES) return fail(UF_ERR_ARG, "nbox must lie in [1, 64]");
    if (!boxes || !theta) return fail(UF_ERR_ARG, "NULL boxes or theta");
    std::vector<uf::DesignBox> hb(nbox);
    for (int i = 0; i < nbox; ++i)
      hb[i] = {boxes[4 * i], boxes[4 * i + 1], boxes[4 * i + 2], boxes[4 * i + 3], theta[3 * i], theta[3 * i + 1],
               theta[3 * i + 2]};
    UF_CUDA(cudaMemcpyAsync(at<uf::DesignBox>(P.boxes), hb.data(), sizeof(uf::DesignBox) * nbox, cudaMemcpyHostToDevice,
                            stream));
    UF_CUDA(cudaStreamSynchronize(stream));
    return UF_OK;
  }
  uf_status design_phi(int nbox, const double* boxes, const double* theta, double width, void* out) override {
    if (!(width > 0)) return fail(UF_ERR_ARG, "width must be positive");
    uf_status s = upload_boxes(nbox, boxes, theta);
    if (s != UF_OK) return s;
    T* dst = out ? q : phi;
    uf::k_design_phi<T><<<plane_grid(d.nx, d.ny, d.nz), dim3(uf::BX, uf::BY), 0, stream>>>(
        d.nx, d.ny, d.nz, P.Pc, d.h, at<uf::DesignBox>(P.boxes), nbox, width, dst);
    UF_CUDA(cudaGetLastError());
    if (out) return copy_out(out, q, d.nx, d.ny, d.nz, P.Pc);
    const size_t n = P.n_c;
    uf::k_drag_coeff<T><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(phi, cc, n, d.Cd, d.a, d.b, d.e);
    UF_CUDA(cudaGetLastError());
    return UF_OK;
  }
  uf_status design_vjp(int nbox, const double* boxes, const double* theta, double width, const void* lphi_in,
                       double* g_out) override {
    if (!(width > 0) || !g_out) return fail(UF_ERR_ARG, "width must be positive and g_out non-NULL");
    uf_status s = upload_boxes(nbox, boxes, theta);
    if (s != UF_OK) return s;
    s = copy_in(q, d.nx, d.ny, d.nz, P.Pc, lphi_in);
    if (s != UF_OK) return s;
    double* g = at<double>(P.grad);
    UF_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * 3 * nbox, stream));
    uf::k_design_phi_vjp<T><<<plane_grid(d.nx, d.ny, d.nz), dim3(uf::BX, uf::BY), 0, stream>>>(
        d.nx, d.ny, d.nz, P.Pc, d.h, at<uf::DesignBox>(P.boxes), nbox, width, q, g);
    UF_CUDA(cudaGetLastError());
    UF_CUDA(cudaMemcpyAsync(g_out, g, sizeof(double) * 3 * nbox, cudaMemcpyDeviceToHost, stream));
    UF_CUDA(cudaStreamSynchronize(stream));
    return UF_OK;
  }

  // Captures pre(s) ; solve ; post(s) into an executable graph.
  template <typename Pre, typename Post>
  uf_status capture(cudaGraphExec_t* exec, Pre pre, Post post, int* n_fixed, int* n_setup, int* n_iter) {
    cudaGraph_t graph = nullptr;
    UF_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    cudaStreamCaptureStatus cs;
    cudaGraph_t cgraph;
    uf_status rs = UF_OK;
    cudaError_t e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cgraph, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle cond;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cgraph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      return fail(UF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    rec_count = 0;
    pre(cap);
    const int fixed_pre = rec_count;
    rs = rec_solve(cap, cond, n_setup, n_iter);
    const int after_solve = rec_count;
    if (rs == UF_OK) post(cap);
    *n_fixed = fixed_pre + (rec_count - after_solve);
    e = cudaStreamEndCapture(cap, &graph);
    if (rs != UF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rs;
    }
    if (e != cudaSuccess) return fail(UF_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(UF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return UF_OK;
  }

  uf_status build_step_graphs() {
    for (int par = 0; par < 2; ++par) {
      if (step_exec[par]) continue;
      T* kin = kb[par];
      T* oin = ob[par];
      T* kout = kb[1 - par];
      T* oout = ob[1 - par];
      int nf, ns, ni;
      uf_status s = capture(&step_exec[par], [&](cudaStream_t st2) { rec_momentum(st2, kin, oin); },
                            [&](cudaStream_t st2) { rec_post(st2, kin, oin, kout, oout); }, &nf, &ns, &ni);
      if (s != UF_OK) return s;
      launches_fixed = nf;
      launches_solve_setup = ns;
      launches_per_iter = ni;
    }
    return UF_OK;
  }

  // The taping variant of the step graphs (the same kernels and arithmetic;
  // the fused kernels also write the intermediate fields the adjoint reads).
  uf_status build_tape_graphs() {
    for (int par = 0; par < 2; ++par) {
      if (tape_exec[par]) continue;
      T* kin = kb[par];
      T* oin = ob[par];
      T* kout = kb[1 - par];
      T* oout = ob[1 - par];
      int nf, ns, ni;
      taping = true;
      uf_status s = capture(&tape_exec[par], [&](cudaStream_t st2) { rec_momentum(st2, kin, oin); },
                            [&](cudaStream_t st2) { rec_post(st2, kin, oin, kout, oout); }, &nf, &ns, &ni);
      taping = false;
      if (s != UF_OK) return s;
    }
    return UF_OK;
  }

  // Drops every captured graph (after a change of the launch tuning).
  void drop_graphs() {
    for (auto& e : step_exec)
      if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    for (auto& e : tape_exec)
      if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    if (init_exec) { cudaGraphExecDestroy(init_exec); init_exec = nullptr; }
    if (solve_exec) { cudaGraphExecDestroy(solve_exec); solve_exec = nullptr; }
    if (adj_solve_exec) { cudaGraphExecDestroy(adj_solve_exec); adj_solve_exec = nullptr; }
    adj_mu = adj_b = nullptr;
  }

  // Tail starting at level lt (clamped to [automatic, coarsest]).
  uf_status set_tail_level(int lt) {
    if (d.precond != UF_PRECOND_MG) return UF_OK;
    lt = std::min(std::max(lt, P.min_tail_level), P.nl - 1);
    plan_tail(P, lt);
    for (int l = 0; l < P.nl; ++l) tail.off[l] = P.tail_off[l];
    tail.lt = lt;
    tail.cr_off = (int)P.tail_cr_off;
    UF_CUDA(set_smem_limits());
    return UF_OK;
  }

  uf_status get_tuning(uf_tuning* t, int* levels) override {
    if (!t) return fail(UF_ERR_ARG, "NULL output");
    std::memset(t, 0, sizeof(*t));
    t->tail_level = P.tail_level;
    for (int l = 0; l < P.nl && l < UF_MAX_LEVELS; ++l) {
      int zc;
      march_grid(l, &zc);
      t->march_zc[l] = d.precond == UF_PRECOND_MG ? zc : 0;
    }
    int azc;
    advect_grid(&azc);
    t->advect_zc = azc;
    t->unfused = unfused;
    t->coarse_start = coarse_start() < P.tail_level ? coarse_start() : -1;
    if (levels) *levels = P.nl;
    return UF_OK;
  }

  uf_status set_tuning(const uf_tuning* t) override {
    if (t) {
      for (int l = 0; l < UF_MAX_LEVELS; ++l) {
        const int z = t->march_zc[l];
        if (z != 0 && (z < 2 || z > 64 || (z & 1))) return fail(UF_ERR_ARG, "march_zc must be 0 or even in [2, 64]");
      }
      if (t->advect_zc < 0 || t->advect_zc > 64) return fail(UF_ERR_ARG, "advect_zc must be in [0, 64]");
      if (t->unfused & ~(UF_UNFUSED_ADVECT | UF_UNFUSED_MOMENTUM)) return fail(UF_ERR_ARG, "unknown bit in unfused");
      if (t->coarse_start < -1 || t->coarse_start >= UF_MAX_LEVELS) return fail(UF_ERR_ARG, "coarse_start out of range");
    }
    drop_graphs();
    advect_zc_tuned = t ? t->advect_zc : 0;
    unfused = t ? t->unfused : 0;
    coarse_start_tuned = t ? t->coarse_start : 0;
    for (int l = 0; l < uf::MAX_LEVELS; ++l) march_zc_tuned[l] = t ? t->march_zc[l] : 0;
    return set_tail_level(t && t->tail_level > 0 ? t->tail_level : P.auto_tail_level);
  }

  // Autotuner: candidates = tail level (automatic and up to two levels
  // deeper) x a uniform tile depth (automatic, 2, 4, 8) x per-level launches
  // or the cluster V-cycle over the last level above the tail (where the
  // device co-schedules the cluster); each is timed over
  // `reps` solves of a synthetic right-hand side from a zero guess, with the
  // unknown and the right-hand side in scratch buffers (ut, uh) that no step
  // keeps between steps.
  uf_status autotune(int reps, uf_tuning* chosen, double* best_ms) override {
    if (reps < 1) return fail(UF_ERR_ARG, "reps >= 1 required");
    if (d.precond != UF_PRECOND_MG) {
      if (chosen) get_tuning(chosen, nullptr);
      if (best_ms) *best_ms = 0.0;
      return UF_OK;
    }
    int zc0;
    dim3 g0 = chunk_grid(d.nx, d.ny, d.nz, &zc0);
    uf::k_tune_rhs<T><<<g0, dim3(uf::BX, uf::BY), 0, stream>>>(lv[0], uh, zc0);
    UF_CUDA(cudaGetLastError());
    cudaEvent_t e0, e1;
    UF_CUDA(cudaEventCreate(&e0));
    UF_CUDA(cudaEventCreate(&e1));
    struct Cand {
      int lt, zc, cs;
    };
    std::vector<Cand> cands;
    for (int lt = P.auto_tail_level; lt <= std::min(P.nl - 1, P.auto_tail_level + 2); ++lt)
      for (int zc : {0, 2, 4, 8}) {
        cands.push_back({lt, zc, -1});
        // the cluster V-cycle over the last level before the tail
        if (d.precond == UF_PRECOND_MG && cluster_ctas > 0 && lt >= 2) cands.push_back({lt, zc, lt - 1});
      }
    double best = 1e300;
    uf_tuning best_t;
    uf_status rs = UF_OK;
    for (const Cand& c : cands) {
      uf_tuning t;
      std::memset(&t, 0, sizeof(t));
      t.tail_level = c.lt;
      for (int l = 0; l < UF_MAX_LEVELS; ++l) t.march_zc[l] = c.zc;
      t.advect_zc = advect_zc_tuned;       // the solve's candidates keep the step's other knobs
      t.unfused = unfused;
      t.coarse_start = c.cs;
      rs = set_tuning(&t);
      if (rs != UF_OK) break;
      cudaGraphExec_t ex = nullptr;
      sol_x = ut;
      sol_b = uh;
      sol_g = nullptr;
      int nf, ns, ni;
      auto pre = [&](cudaStream_t s2) {
        cudaMemsetAsync(ut, 0, P.n_u * sizeof(T), s2);
        int zc;
        dim3 g = chunk_grid(d.nx, d.ny, d.nz, &zc);
        uf::k_solve_reset<T><<<g, dim3(uf::BX, uf::BY), 0, s2>>>(lv[0], uh, zc, partials, st);
        rec_count++;
      };
      rs = capture(&ex, pre, [&](cudaStream_t) {}, &nf, &ns, &ni);
      sol_x = p;
      sol_b = b;
      sol_g = gd;
      if (rs != UF_OK) break;
      cudaError_t e = cudaGraphLaunch(ex, stream);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(ex, stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      cudaGraphExecDestroy(ex);
      if (e != cudaSuccess) {
        rs = fail(UF_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        break;
      }
      const double mean = ms / reps;
      if (mean < best) {
        best = mean;
        get_tuning(&best_t, nullptr);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != UF_OK) return rs;
    rs = check_device(nullptr);
    if (rs != UF_OK) return rs;
    rs = set_tuning(&best_t);
    if (rs != UF_OK) return rs;
    if (chosen) *chosen = best_t;
    if (best_ms) *best_ms = best;
    return UF_OK;
  }

  // ------------------------------------------------------------ batch support
  const uf_grid_desc& desc() const override { return d; }
  bool has_state() const override { return have_state; }
  void advanced(int nsteps) override { parity ^= (nsteps & 1); }
  uf_status read_status(uf_step_stats* out) override { return check_device(out); }

  // Checkpoint / resume: the adjoint's checkpoint layout (faces, k, omega,
  // p^n and the next guess in the pressure store), 256-byte aligned inside
  // the caller's buffer.
  size_t state_bytes() override { return adj_layout(1, 1).ckpt * sizeof(T) + 256; }
  uf_status save_snapshot(void* buf, size_t bytes) override {
    if (!buf) return fail(UF_ERR_ARG, "NULL state buffer");
    if (bytes < state_bytes()) return fail(UF_ERR_NOMEM, "state buffer smaller than uf_state_bytes()");
    if (!have_state) return fail(UF_ERR_STATE, "no state: call uf_init_state or uf_set_state first");
    T* slot = reinterpret_cast<T*>(round_up(reinterpret_cast<size_t>(buf), 256));
    UF_CUDA(save_state(slot, adj_layout(1, 1)));
    return UF_OK;
  }
  uf_status load_snapshot(const void* buf, size_t bytes) override {
    if (!buf) return fail(UF_ERR_ARG, "NULL state buffer");
    if (bytes < state_bytes()) return fail(UF_ERR_NOMEM, "state buffer smaller than uf_state_bytes()");
    const T* slot = reinterpret_cast<const T*>(round_up(reinterpret_cast<size_t>(buf), 256));
    UF_CUDA(load_state(slot, adj_layout(1, 1)));
    have_state = true;
    return UF_OK;
  }

  void fill_view(void* vp) override {
    GridView<T>& V = *reinterpret_cast<GridView<T>*>(vp);
    std::memset(&V, 0, sizeof(V));
    V.d = d;
    V.sp = sp;
    V.adv = advect_args();
    V.u = u; V.v = v; V.w = w; V.uh = uh; V.vh = vh; V.wh = wh; V.ut = ut; V.vt = vt; V.wt = wt;
    V.u2 = u2; V.v2 = v2; V.w2 = w2; V.cc = cc; V.nut = nut; V.p = p; V.pd = pd; V.gd = gd; V.b = b; V.z = z; V.q = q;
    V.d0 = d0; V.d1 = d1;
    V.kb[0] = kb[0]; V.kb[1] = kb[1]; V.ob[0] = ob[0]; V.ob[1] = ob[1];
    V.parity = parity;
    V.n_u = P.n_u; V.n_v = P.n_v; V.n_w = P.n_w;
    V.nl = (int)lv.size();
    for (int l = 0; l < V.nl; ++l) {
      V.lv[l] = lv[l];
      int zc;
      const dim3 g = march_grid(l, &zc);
      V.march_g[l][0] = g.x; V.march_g[l][1] = g.y; V.march_g[l][2] = g.z;
      V.march_zc[l] = zc;
    }
    V.tail_level = P.tail_level;
    V.tail = tail;
    V.tail.rin = 1;   // batched launches form the tail's right-hand side in the tail
    V.tail_smem = P.tail_smem;
    int zc;
    const dim3 gc = chunk_grid(d.nx, d.ny, d.nz, &zc);
    V.chunk_g[0] = gc.x; V.chunk_g[1] = gc.y; V.chunk_g[2] = gc.z;
    V.chunk_zc = zc;
    int azc;
    const dim3 ga = advect_grid(&azc);
    V.adv_g[0] = ga.x; V.adv_g[1] = ga.y; V.adv_g[2] = ga.z;
    V.adv_zc = azc;
    V.dt_blocks = kDtBlocks;
    V.st = st;
    V.partials = partials;
    V.dt = dt;
    V.dtT = dtT;
    V.sw = smooth_weights();
  }

  // ------------------------------------------------------------ entry points
  uf_status copy_in(T* dst, int lx, int ly, int lz, int pitch, const void* src) {
    if (!src) return fail(UF_ERR_ARG, "NULL buffer");
    UF_CUDA(cudaMemcpy2DAsync(dst, (size_t)pitch * sizeof(T), src, (size_t)lx * sizeof(T), (size_t)lx * sizeof(T),
                              (size_t)ly * lz, cudaMemcpyDefault, stream));
    return UF_OK;
  }
  uf_status copy_out(void* dstp, const T* src, int lx, int ly, int lz, int pitch) {
    if (!dstp) return fail(UF_ERR_ARG, "NULL buffer");
    UF_CUDA(cudaMemcpy2DAsync(dstp, (size_t)lx * sizeof(T), src, (size_t)pitch * sizeof(T), (size_t)lx * sizeof(T),
                              (size_t)ly * lz, cudaMemcpyDefault, stream));
    UF_CUDA(cudaStreamSynchronize(stream));
    return UF_OK;
  }

  uf_status set_porosity(const void* src) override {
    uf_status s = copy_in(phi, d.nx, d.ny, d.nz, P.Pc, src);
    if (s != UF_OK) return s;
    const size_t n = P.n_c;
    uf::k_drag_coeff<T><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(phi, cc, n, d.Cd, d.a, d.b, d.e);
    UF_CUDA(cudaGetLastError());
    return UF_OK;
  }

  bool field_geom(int f, T** ptr, int* lx, int* ly, int* lz, int* pitch) {
    *pitch = P.Pc;
    *lx = d.nx; *ly = d.ny; *lz = d.nz;
    switch (f) {
      case UF_FIELD_U: *ptr = u; *lx = d.nx + 1; *pitch = P.Pu; return true;
      case UF_FIELD_V: *ptr = v; *ly = d.ny + 1; return true;
      case UF_FIELD_W: *ptr = w; *lz = d.nz + 1; return true;
      case UF_FIELD_P: *ptr = p; return true;
      case UF_FIELD_K: *ptr = kb[parity]; return true;
      case UF_FIELD_OMEGA: *ptr = ob[parity]; return true;
      case UF_FIELD_PHI: *ptr = phi; return true;
      case UF_FIELD_NUT: *ptr = nut; return true;
    }
    return false;
  }

  uf_status set_state(int f, const void* src) override {
    T* ptr; int lx, ly, lz, pitch;
    if (!field_geom(f, &ptr, &lx, &ly, &lz, &pitch)) return fail(UF_ERR_ARG, "unknown field");
    if (f == UF_FIELD_PHI) return set_porosity(src);
    uf_status s = copy_in(ptr, lx, ly, lz, pitch, src);
    if (s == UF_OK && (f == UF_FIELD_U || f == UF_FIELD_V || f == UF_FIELD_W)) have_state = true;
    if (s == UF_OK && f == UF_FIELD_P) UF_CUDA(pressure_sync(1));   // a new pressure has no history
    return s;
  }

  uf_status get_state(int f, void* dst) override {
    T* ptr; int lx, ly, lz, pitch;
    if (!field_geom(f, &ptr, &lx, &ly, &lz, &pitch)) return fail(UF_ERR_ARG, "unknown field");
    return copy_out(dst, ptr, lx, ly, lz, pitch);
  }

  // ------------------------------------------------- bulk field transfer
  // Staging buffer of each field for uf_set_fields / uf_get_fields: a step
  // scratch array (recomputed by every step) at least as large as the
  // field's dense layout.
  T* staging(int f) {
    switch (f) {
      case UF_FIELD_U: return uh;
      case UF_FIELD_V: return vh;
      case UF_FIELD_W: return wh;
      case UF_FIELD_P: return ut;
      case UF_FIELD_K: return vt;
      case UF_FIELD_OMEGA: return wt;
      case UF_FIELD_PHI: return u2;
      case UF_FIELD_NUT: return v2;
    }
    return nullptr;
  }
  static bool on_device(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  }
  uf_status repack(const T* src, T* dst, int lx, int rows, int pitch, int to_padded) {
    const size_t n = (size_t)lx * rows;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    uf::k_repack<T><<<blocks, 256, 0, stream>>>(src, dst, lx, rows, pitch, to_padded);
    UF_CUDA(cudaGetLastError());
    return UF_OK;
  }

  uf_status set_fields(int n, const int* fields, const void* const* bufs) override {
    if (n < 0 || (n > 0 && (!fields || !bufs))) return fail(UF_ERR_ARG, "NULL field list");
    bool state = false;
    for (int q = 0; q < n; ++q) {
      T* ptr; int lx, ly, lz, pitch;
      if (!field_geom(fields[q], &ptr, &lx, &ly, &lz, &pitch)) return fail(UF_ERR_ARG, "unknown field");
      if (!bufs[q]) return fail(UF_ERR_ARG, "NULL buffer");
    }
    // every host copy first, back to back on the copy engine, then the repacks
    for (int q = 0; q < n; ++q) {
      T* ptr; int lx, ly, lz, pitch;
      field_geom(fields[q], &ptr, &lx, &ly, &lz, &pitch);
      if (!on_device(bufs[q]))
        UF_CUDA(cudaMemcpyAsync(staging(fields[q]), bufs[q], (size_t)lx * ly * lz * sizeof(T), cudaMemcpyHostToDevice,
                                stream));
    }
    for (int q = 0; q < n; ++q) {
      T* ptr; int lx, ly, lz, pitch;
      field_geom(fields[q], &ptr, &lx, &ly, &lz, &pitch);
      T* dst = fields[q] == UF_FIELD_PHI ? phi : ptr;
      const T* src = on_device(bufs[q]) ? reinterpret_cast<const T*>(bufs[q]) : staging(fields[q]);
      uf_status s = repack(src, dst, lx, ly * lz, pitch, 1);
      if (s != UF_OK) return s;
      if (fields[q] == UF_FIELD_PHI) {
        uf::k_drag_coeff<T><<<(unsigned)((P.n_c + 255) / 256), 256, 0, stream>>>(phi, cc, P.n_c, d.Cd, d.a, d.b, d.e);
        UF_CUDA(cudaGetLastError());
      }
      state |= fields[q] == UF_FIELD_U || fields[q] == UF_FIELD_V || fields[q] == UF_FIELD_W;
      if (fields[q] == UF_FIELD_P) UF_CUDA(pressure_sync(1));
    }
    if (state) have_state = true;
    return UF_OK;
  }

  uf_status get_fields(int n, const int* fields, void* const* bufs) override {
    if (n < 0 || (n > 0 && (!fields || !bufs))) return fail(UF_ERR_ARG, "NULL field list");
    for (int q = 0; q < n; ++q) {
      T* ptr; int lx, ly, lz, pitch;
      if (!field_geom(fields[q], &ptr, &lx, &ly, &lz, &pitch)) return fail(UF_ERR_ARG, "unknown field");
      if (!bufs[q]) return fail(UF_ERR_ARG, "NULL buffer");
    }
    // every repack first, then the host copies back to back
    for (int q = 0; q < n; ++q) {
      T* ptr; int lx, ly, lz, pitch;
      field_geom(fields[q], &ptr, &lx, &ly, &lz, &pitch);
      T* dst = on_device(bufs[q]) ? reinterpret_cast<T*>(bufs[q]) : staging(fields[q]);
      uf_status s = repack(ptr, dst, lx, ly * lz, pitch, 0);
      if (s != UF_OK) return s;
    }
    for (int q = 0; q < n; ++q) {
      T* ptr; int lx, ly, lz, pitch;
      field_geom(fields[q], &ptr, &lx, &ly, &lz, &pitch);
      if (!on_device(bufs[q]))
        UF_CUDA(cudaMemcpyAsync(bufs[q], staging(fields[q]), (size_t)lx * ly * lz * sizeof(T), cudaMemcpyDeviceToHost,
                                stream));
    }
    UF_CUDA(cudaStreamSynchronize(stream));
    return UF_OK;
  }

  uf_status init_state() override {
    if (!init_exec) {
      int nf, ns, ni;
      auto pre = [&](cudaStream_t s) {
        const dim3 blk(uf::BX, uf::BY);
        const dim3 ga = plane_grid(d.nx + 1, d.ny + 1, 3 * d.nz + 1);
        cudaMemsetAsync(pd, 0, P.n_c * sizeof(uf::PStore<T>), s);
        cudaMemsetAsync(gd, 0, P.n_c * sizeof(uf::PStore<T>), s);
        uf::k_init_fields<T><<<ga, blk, 0, s>>>(sp, u, v, w, kb[0], ob[0], p);
        rec_count++;
        if (!(d.fixed_dt > 0)) {
          uf::k_cfl_dt<T><<<kDtBlocks, 256, 0, s>>>(u, P.n_u, v, P.n_v, w, P.n_w, d.cfl * d.h, partials, &st->ticket[0], dt, dtT);
          rec_count++;
        }
        uf::k_drag_bc<T><<<ga, blk, 0, s>>>(sp, u, v, w, cc, uh, vh, wh);
        int zc;
        const dim3 gr = chunk_grid(d.nx, d.ny, d.nz, &zc);
        uf::k_pressure_rhs<T><<<gr, blk, 0, s>>>(sp, uh, vh, wh, b, zc, partials, st);
        rec_count += 2;
      };
      auto post = [&](cudaStream_t s) {
        uf::k_pressure_commit<T><<<plane_grid(d.nx, d.ny, d.nz), dim3(uf::BX, uf::BY), 0, s>>>(sp, p, pd, gd, st);
        rec_count++;
      };
      uf_status s = capture(&init_exec, pre, post, &nf, &ns, &ni);
      if (s != UF_OK) return s;
    }
    uf_status s = ensure_solve_exec();
    if (s != UF_OK) return s;
    parity = 0;
    UF_CUDA(cudaGraphLaunch(init_exec, stream));
    s = check_device(nullptr);
    if (s != UF_OK) return s;
    // The solve above held the whole initial pressure in its grid-precision
    // iterate, which bounds its true residual by about eps ||A|| ||p||.  One
    // more solve from the committed pressure (initial residual formed on the
    // pressure store) removes that remainder; then the projection.
    UF_CUDA(copy_cell_ps(gd, pd));
    UF_CUDA(cudaGraphLaunch(solve_exec, stream));
    uf::k_project<T><<<plane_grid(d.nx + 1, d.ny + 1, 3 * d.nz + 1), dim3(uf::BX, uf::BY), 0, stream>>>(sp, pd, uh, vh,
                                                                                                       wh);
    UF_CUDA(cudaGetLastError());
    UF_CUDA(cudaMemcpyAsync(u, uh, P.n_u * sizeof(T), cudaMemcpyDeviceToDevice, stream));
    UF_CUDA(cudaMemcpyAsync(v, vh, P.n_v * sizeof(T), cudaMemcpyDeviceToDevice, stream));
    UF_CUDA(cudaMemcpyAsync(w, wh, P.n_w * sizeof(T), cudaMemcpyDeviceToDevice, stream));
    UF_CUDA(copy_cell_ps(gd, pd));   // no previous pressure: the first guess is p itself
    have_state = true;
    return check_device(nullptr);
  }

  // Reads the solver state; returns the device status as a uf_status.
  uf_status check_device(uf_step_stats* out) {
    uf::SolveState h;
    double hdt = 0;
    UF_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, stream));
    UF_CUDA(cudaMemcpyAsync(&hdt, dt, sizeof(double), cudaMemcpyDeviceToHost, stream));
    UF_CUDA(cudaStreamSynchronize(stream));
    last_iters = h.iter;
    if (out) {
      out->dt = hdt;
      out->cg_iters = h.iter;
      out->cg_rel_residual = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
      out->status = h.status;
      out->cg_iters_total = h.total_iters;
    }
    if (h.sticky != 0) {
      const int code = h.sticky;
      int zero = 0;
      UF_CUDA(cudaMemcpyAsync(&st->sticky, &zero, sizeof(int), cudaMemcpyHostToDevice, stream));
      UF_CUDA(cudaStreamSynchronize(stream));
      if (code == uf::DEV_NOT_CONVERGED) return fail(UF_ERR_NOT_CONVERGED, "pressure CG reached its iteration cap");
      if (code == uf::DEV_NAN) return fail(UF_ERR_NAN, "non-finite residual in the pressure solve");
      return fail(UF_ERR_CUDA, "device reported an error");
    }
    return UF_OK;
  }

  uf_status step(uf_step_stats* out) override {
    if (!have_state) return fail(UF_ERR_STATE, "no state: call uf_init_state or uf_set_state first");
    uf_status s = build_step_graphs();
    if (s != UF_OK) return s;
    UF_CUDA(cudaGraphLaunch(step_exec[parity], stream));
    parity ^= 1;
    if (out) return check_device(out);
    UF_CUDA(cudaGetLastError());
    return UF_OK;
  }

  uf_status run(int nsteps, uf_step_stats* out) override {
    if (nsteps < 0) return fail(UF_ERR_ARG, "nsteps < 0");
    for (int n = 0; n < nsteps; ++n) {
      uf_status s = step(nullptr);
      if (s != UF_OK) return s;
    }
    if (out) return check_device(out);
    return UF_OK;
  }

  // ---------------------------------------------------- mesh resolver ----
  // Porosity of closed triangle meshes (uf_mesh_to_phi): the mesh and the
  // objects' bounding boxes are copied to device memory allocated for the
  // call; the result goes to the grid's porosity (and drag coefficient) or
  // to phi_out.
  uf_status mesh_to_phi(int ntri, const double* tris, int nobj, const int* first, const int* count,
                        const double* phi_in, int sub, void* phi_out) override {
    if (ntri < 0 || nobj < 0 || (ntri > 0 && !tris) || (nobj > 0 && (!first || !count || !phi_in)))
      return fail(UF_ERR_ARG, "NULL mesh arrays");
    if (sub < 1 || sub > 16) return fail(UF_ERR_ARG, "sub-sampling must be 1..16 per axis");
    std::vector<uf::MeshObject> obj(nobj);
    for (int o = 0; o < nobj; ++o) {
      if (first[o] < 0 || count[o] < 1 || (long long)first[o] + count[o] > ntri)
        return fail(UF_ERR_ARG, "object " + std::to_string(o) + " has a triangle range outside the mesh");
      if (!(phi_in[o] >= 0.0 && phi_in[o] <= 1.0))
        return fail(UF_ERR_ARG, "object " + std::to_string(o) + " has a porosity outside [0, 1]");
      uf::MeshObject& m = obj[o];
      m.first = first[o];
      m.count = count[o];
      m.phi_in = phi_in[o];
      for (int a = 0; a < 3; ++a) {
        m.lo[a] = tris[9 * (size_t)m.first + a];
        m.hi[a] = m.lo[a];
      }
      for (size_t e = (size_t)m.first; e < (size_t)m.first + m.count; ++e)
        for (int c = 0; c < 3; ++c)
          for (int a = 0; a < 3; ++a) {
            const double x = tris[9 * e + 3 * c + a];
            if (!std::isfinite(x)) return fail(UF_ERR_ARG, "non-finite vertex coordinate");
            m.lo[a] = std::min(m.lo[a], x);
            m.hi[a] = std::max(m.hi[a], x);
          }
      // cells whose closed box [i h, (i + 1) h] meets [lo, hi], per axis (a
      // contiguous range; empty: clo > chi)
      const int ext[3] = {d.nx, d.ny, d.nz};
      for (int a = 0; a < 3; ++a) {
        m.clo[a] = ext[a];
        m.chi[a] = -1;
        for (int c = 0; c < ext[a]; ++c) {
          const double c0 = (double)c * d.h, c1 = (double)(c + 1) * d.h;
          if (m.hi[a] < c0 || m.lo[a] > c1) continue;
          m.clo[a] = std::min(m.clo[a], c);
          m.chi[a] = std::max(m.chi[a], c);
        }
      }
    }
    double* dtri = nullptr;
    uf::MeshObject* dobj = nullptr;
    const size_t tb_tri = (size_t)std::max(ntri, 1) * 9 * sizeof(double);
    const size_t tb_obj = (size_t)std::max(nobj, 1) * sizeof(uf::MeshObject);
    UF_CUDA(cudaMalloc(&dtri, tb_tri));
    cudaError_t e = cudaMalloc(&dobj, tb_obj);
    if (e == cudaSuccess && ntri > 0)
      e = cudaMemcpyAsync(dtri, tris, (size_t)ntri * 9 * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && nobj > 0)
      e = cudaMemcpyAsync(dobj, obj.data(), nobj * sizeof(uf::MeshObject), cudaMemcpyHostToDevice, stream);
    T* dst = phi_out ? q : phi;
    if (e == cudaSuccess) {
      const long long cells = (long long)d.nx * d.ny * d.nz;
      const unsigned blocks = (unsigned)((cells + uf::MESH_WARPS - 1) / uf::MESH_WARPS);
      uf::k_mesh_phi<T><<<blocks, 32 * uf::MESH_WARPS, 0, stream>>>(d.nx, d.ny, d.nz, P.Pc, d.h, sub, dtri, dobj,
                                                                     nobj, dst);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(dtri);
    if (dobj) cudaFree(dobj);
    UF_CUDA(e);
    if (phi_out) {
      uf_status s = copy_out(phi_out, q, d.nx, d.ny, d.nz, P.Pc);
      if (s != UF_OK) return s;
      UF_CUDA(cudaStreamSynchronize(stream));
      return UF_OK;
    }
    uf::k_drag_coeff<T><<<(unsigned)((P.n_c + 255) / 256), 256, 0, stream>>>(phi, cc, P.n_c, d.Cd, d.a, d.b, d.e);
    UF_CUDA(cudaGetLastError());
    return UF_OK;
  }

  // ------------------------------------------------------ sub-steps ------
  // One sub-step of the step, or its transpose, on dense inputs (test
  // support, uf_substep).  Works in a scratch block of four face sets and
  // eight cell arrays allocated for the call; the projection also uses the
  // solver's arrays and the pressure store, so the grid's state is not
  // kept.
  uf_status substep(int which, int tr, const void* const* in, const void* const* cot, void* const* out) override {
    if (!(d.fixed_dt > 0)) return fail(UF_ERR_ARG, "sub-steps need a fixed time step (fixed_dt > 0)");
    if (!in || !out || (tr && !cot)) return fail(UF_ERR_ARG, "NULL buffer list");
    if (which < UF_SUB_EDDY || which > UF_SUB_TURB) return fail(UF_ERR_ARG, "unknown sub-step");
    const size_t fN = face_set(), cN = a64(P.n_c);
    T* blk = nullptr;
    UF_CUDA(cudaMalloc(&blk, (4 * fN + 8 * cN) * sizeof(T)));
    uf_status s = substep_in(which, tr, in, cot, out, blk, fN, cN);
    cudaError_t e = cudaStreamSynchronize(stream);
    cudaFree(blk);
    if (s != UF_OK) return s;
    UF_CUDA(e);
    return check_device(nullptr);
  }
  uf_status substep_in(int which, int tr, const void* const* in, const void* const* cot, void* const* out, T* blk,
                       size_t fN, size_t cN) {
    FaceSet S[4];
    T* C[8];
    for (int a = 0; a < 4; ++a) S[a] = faces_at(blk + a * fN);
    for (int a = 0; a < 8; ++a) C[a] = blk + 4 * fN + a * cN;
    UF_CUDA(cudaMemsetAsync(blk, 0, (4 * fN + 8 * cN) * sizeof(T), stream));
    auto faces_in = [&](FaceSet f, const void* const* src) -> uf_status {
      uf_status r = copy_in(f.u, d.nx + 1, d.ny, d.nz, P.Pu, src[0]);
      if (r == UF_OK) r = copy_in(f.v, d.nx, d.ny + 1, d.nz, P.Pc, src[1]);
      if (r == UF_OK) r = copy_in(f.w, d.nx, d.ny, d.nz + 1, P.Pc, src[2]);
      return r;
    };
    auto faces_out = [&](void* const* dst, FaceSet f) -> uf_status {
      uf_status r = copy_out(dst[0], f.u, d.nx + 1, d.ny, d.nz, P.Pu);
      if (r == UF_OK) r = copy_out(dst[1], f.v, d.nx, d.ny + 1, d.nz, P.Pc);
      if (r == UF_OK) r = copy_out(dst[2], f.w, d.nx, d.ny, d.nz + 1, P.Pc);
      return r;
    };
    auto cell_in = [&](T* c, const void* src) { return copy_in(c, d.nx, d.ny, d.nz, P.Pc, src); };
    auto cell_out = [&](void* dst, const T* c) { return copy_out(dst, c, d.nx, d.ny, d.nz, P.Pc); };
    const dim3 bk(uf::BX, uf::BY);
    const dim3 gc = plane_grid(d.nx, d.ny, d.nz);
    const dim3 ga = plane_grid(d.nx + 1, d.ny + 1, 3 * d.nz + 1);
    uf_status s = UF_OK;
#define UF_TRY(x) do { s = (x); if (s != UF_OK) return s; } while (0)
    switch (which) {
      case UF_SUB_EDDY: {       // in u, v, w, k, omega -> nu_t
        UF_TRY(faces_in(S[0], in));
        UF_TRY(cell_in(C[0], in[3]));
        UF_TRY(cell_in(C[1], in[4]));
        if (!tr) {
          uf::k_eddy_viscosity<T><<<gc, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[0], C[1], C[2]);
          UF_CUDA(cudaGetLastError());
          return cell_out(out[0], C[2]);
        }
        UF_TRY(cell_in(C[2], cot[0]));
        uf::k_eddy_viscosity_adj<T><<<gc, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[0], C[1], C[2], C[3], C[4],
                                                            S[1].u, S[1].v, S[1].w);
        UF_CUDA(cudaGetLastError());
        UF_TRY(faces_out(out, S[1]));
        UF_TRY(cell_out(out[3], C[3]));
        return cell_out(out[4], C[4]);
      }
      case UF_SUB_ADVECT: {     // in u, v, w -> MacCormack result on interior faces
        UF_TRY(faces_in(S[0], in));
        uf::AdvectArgs<T> Aa = advect_args();
        Aa.u = S[0].u; Aa.v = S[0].v; Aa.w = S[0].w;
        Aa.uh = S[1].u; Aa.vh = S[1].v; Aa.wh = S[1].w;
        Aa.ut = S[2].u; Aa.vt = S[2].v; Aa.wt = S[2].w;
        uf::k_advect_forward<T><<<ga, bk, 0, stream>>>(Aa);
        uf::k_advect_backward<T><<<ga, bk, 0, stream>>>(Aa);
        UF_CUDA(cudaGetLastError());
        if (!tr) return faces_out(out, S[2]);
        UF_TRY(faces_in(S[2], cot));
        uf::AdvectAdj<T> Ja{S[2].u, S[2].v, S[2].w, S[3].u, S[3].v, S[3].w, nullptr, nullptr, nullptr};
        FaceSet L = faces_at(C[0]);   // C[0..] hold a face set: 3 face arrays fit in 8 cell arrays
        UF_CUDA(cudaMemsetAsync(C[0], 0, fN * sizeof(T), stream));
        Ja.lu = L.u; Ja.lv = L.v; Ja.lw = L.w;
        uf::k_advect_backward_adj<T><<<ga, bk, 0, stream>>>(Aa, Ja);
        uf::k_advect_forward_adj<T><<<ga, bk, 0, stream>>>(Aa, Ja);
        UF_CUDA(cudaGetLastError());
        return faces_out(out, L);
      }
      case UF_SUB_DIFFUSE: {    // in u~, v~, w~, nu_t -> u2 (interior faces)
        UF_TRY(faces_in(S[0], in));
        UF_TRY(cell_in(C[0], in[3]));
        if (!tr) {
          uf::k_diffuse<T><<<ga, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[0], S[1].u, S[1].v, S[1].w);
          UF_CUDA(cudaGetLastError());
          return faces_out(out, S[1]);
        }
        UF_TRY(faces_in(S[2], cot));
        uf::k_diffuse_adj<T><<<ga, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[0], S[2].u, S[2].v, S[2].w, S[3].u,
                                                     S[3].v, S[3].w, C[1]);
        UF_CUDA(cudaGetLastError());
        UF_TRY(faces_out(out, S[3]));
        return cell_out(out[3], C[1]);
      }
      case UF_SUB_DRAG_BC: {    // in u2, v2, w2, phi -> u3 (every face)
        UF_TRY(faces_in(S[0], in));
        UF_TRY(cell_in(C[0], in[3]));
        uf::k_drag_coeff<T><<<(unsigned)((P.n_c + 255) / 256), 256, 0, stream>>>(C[0], C[1], P.n_c, d.Cd, d.a, d.b,
                                                                                  d.e);
        if (!tr) {
          uf::k_drag_bc<T><<<ga, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[1], S[1].u, S[1].v, S[1].w);
          UF_CUDA(cudaGetLastError());
          return faces_out(out, S[1]);
        }
        UF_TRY(faces_in(S[2], cot));
        uf::k_drag_bc_adj<T><<<ga, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[1], S[2].u, S[2].v, S[2].w, S[3].u,
                                                     S[3].v, S[3].w, C[2]);
        uf::k_dphi<T><<<(unsigned)((P.n_c + 255) / 256), 256, 0, stream>>>(C[0], C[2], C[3], P.n_c, d.Cd, d.a, d.b,
                                                                            d.e);
        UF_CUDA(cudaGetLastError());
        UF_TRY(faces_out(out, S[3]));
        return cell_out(out[3], C[3]);
      }
      case UF_SUB_PROJECT: {    // in u3, v3, w3 -> projected u1 (pressure solved from zero)
        UF_TRY(faces_in(S[0], in));
        if (!tr) {
          int zc;
          const dim3 gr = chunk_grid(d.nx, d.ny, d.nz, &zc);
          UF_CUDA(cudaMemsetAsync(pd, 0, P.n_c * sizeof(uf::PStore<T>), stream));
          UF_CUDA(cudaMemsetAsync(gd, 0, P.n_c * sizeof(uf::PStore<T>), stream));
          uf::k_pressure_rhs<T><<<gr, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, b, zc, partials, st);
          UF_CUDA(cudaGetLastError());
          UF_TRY(ensure_solve_exec());
          UF_CUDA(cudaGraphLaunch(solve_exec, stream));
          uf::k_project<T><<<ga, bk, 0, stream>>>(sp, pd, S[0].u, S[0].v, S[0].w);
          UF_CUDA(cudaGetLastError());
          return faces_out(out, S[0]);
        }
        UF_TRY(faces_in(S[1], cot));
        T* mu = C[0];
        T* badj = C[1];
        UF_TRY(ensure_adj_solve(mu, badj));
        uf::k_proj_adj_rhs<T><<<gc, bk, 0, stream>>>(sp, S[1].u, S[1].v, S[1].w, badj, mu, C[2]);
        UF_CUDA(cudaGetLastError());
        UF_CUDA(cudaGraphLaunch(adj_solve_exec, stream));
        uf::k_proj_adj_apply<T><<<ga, bk, 0, stream>>>(sp, mu, S[1].u, S[1].v, S[1].w);
        UF_CUDA(cudaGetLastError());
        return faces_out(out, S[1]);
      }
      case UF_SUB_TURB: {       // in u1, v1, w1, k, omega -> k', omega'
        UF_TRY(faces_in(S[0], in));
        UF_TRY(cell_in(C[0], in[3]));
        UF_TRY(cell_in(C[1], in[4]));
        if (!tr) {
          uf::k_turbulence<T><<<gc, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[0], C[1], C[2], C[3]);
          UF_CUDA(cudaGetLastError());
          UF_TRY(cell_out(out[0], C[2]));
          return cell_out(out[1], C[3]);
        }
        UF_TRY(cell_in(C[4], cot[0]));
        UF_TRY(cell_in(C[5], cot[1]));
        uf::k_turbulence_adj<T><<<gc, bk, 0, stream>>>(sp, S[0].u, S[0].v, S[0].w, C[0], C[1], C[4], C[5], C[6], C[7],
                                                        S[1].u, S[1].v, S[1].w);
        UF_CUDA(cudaGetLastError());
        UF_TRY(faces_out(out, S[1]));
        UF_TRY(cell_out(out[3], C[6]));
        return cell_out(out[4], C[7]);
      }
    }
#undef UF_TRY
    return fail(UF_ERR_ARG, "unknown sub-step");
  }

  // ------------------------------------------------------------- objectives
  // Cell index range whose centres lie in [a, b] (m) along an axis of n cells.
  void centre_range(double a, double b, int n, int* lo, int* hi) const {
    *lo = std::max(0, (int)std::ceil(a / d.h - 0.5));
    *hi = std::min(n - 1, (int)std::floor(b / d.h - 0.5));
  }
  struct Box {
    int i0, i1, j0, j1, k0, k1;
    long long cells() const { return (long long)(i1 - i0 + 1) * (j1 - j0 + 1) * (k1 - k0 + 1); }
  };
  Box region_box(const double* r6) const {
    Box B;
    centre_range(r6[0], r6[1], d.nx, &B.i0, &B.i1);
    centre_range(r6[2], r6[3], d.ny, &B.j0, &B.j1);
    centre_range(r6[4], r6[5], d.nz, &B.k0, &B.k1);
    return B;
  }
  uf_status check_objective(const uf_objective_desc* od) const {
    if (!od) return fail(UF_ERR_ARG, "NULL objective");
    if (od->kind == UF_OBJ_COMFORT) return UF_OK;
    if (od->kind != UF_OBJ_REGIONS) return fail(UF_ERR_ARG, "unknown objective kind");
    if (od->nreg < 1 || od->nreg > UF_MAX_REGIONS || !od->regions)
      return fail(UF_ERR_ARG, "regions objective needs 1..8 regions");
    for (int r = 0; r < od->nreg; ++r) {
      const Box B = region_box(od->regions + 6 * r);
      if (B.i1 < B.i0 || B.j1 < B.j0 || B.k1 < B.k0)
        return fail(UF_ERR_ARG, "region " + std::to_string(r) + " holds no cell centre");
    }
    return UF_OK;
  }

  // The objective; for regions also the mean speed of each region.
  uf_status objective_ex_means(const uf_objective_desc* od, double* J, std::vector<double>* means) {
    uf_status s = check_objective(od);
    if (s != UF_OK) return s;
    if (od->kind == UF_OBJ_COMFORT) return objective(od->z_lo, od->z_hi, od->u_hi, od->u_lo, J);
    const dim3 blk(uf::BX, uf::BY);
    for (int r = 0; r < od->nreg; ++r) {
      const Box B = region_box(od->regions + 6 * r);
      int zc;
      dim3 g = chunk_grid(B.i1 - B.i0 + 1, B.j1 - B.j0 + 1, B.k1 - B.k0 + 1, &zc);
      uf::k_box_speed<T><<<g, blk, 0, stream>>>(sp, u, v, w, B.i0, B.i1, B.j0, B.j1, B.k0, B.k1, zc, partials,
                                                 &st->ticket[0], scal + r);
    }
    UF_CUDA(cudaGetLastError());
    double sums[UF_MAX_REGIONS];
    UF_CUDA(cudaMemcpyAsync(sums, scal, sizeof(double) * od->nreg, cudaMemcpyDeviceToHost, stream));
    UF_CUDA(cudaStreamSynchronize(stream));
    double L = 0.0;
    if (means) means->assign(od->nreg, 0.0);
    for (int r = 0; r < od->nreg; ++r) {
      const double m = sums[r] / (double)region_box(od->regions + 6 * r).cells();
      if (means) (*means)[r] = m;
      L += (m - od->u_t) * (m - od->u_t);
    }
    *J = L;
    return UF_OK;
  }
  uf_status objective_ex(const uf_objective_desc* od, double* J) override {
    if (!J) return fail(UF_ERR_ARG, "NULL output");
    return objective_ex_means(od, J, nullptr);
  }

  // dJ/du of the current state into the face adjoints L (accumulated).
  uf_status seed_objective(const uf_objective_desc* od, const std::vector<double>& means, const FaceSet& Lf) {
    const dim3 blk(uf::BX, uf::BY);
    if (od->kind == UF_OBJ_COMFORT) {
      int k_lo = d.nz, k_hi = -1;
      for (int k = 0; k < d.nz; ++k) {
        const double zc = (k + 0.5) * d.h;
        if (zc >= od->z_lo && zc <= od->z_hi) { k_lo = std::min(k_lo, k); k_hi = std::max(k_hi, k); }
      }
      if (k_hi >= k_lo)
        uf::k_objective_adj<T><<<plane_grid(d.nx, d.ny, k_hi - k_lo + 1), blk, 0, stream>>>(
            sp, u, v, w, k_lo, k_hi, od->u_hi, od->u_lo, Lf.u, Lf.v, Lf.w);
    } else {
      for (int r = 0; r < od->nreg; ++r) {
        const Box B = region_box(od->regions + 6 * r);
        const double coef = 2.0 * (means[r] - od->u_t) / (double)B.cells();
        uf::k_box_speed_adj<T><<<plane_grid(B.i1 - B.i0 + 1, B.j1 - B.j0 + 1, B.k1 - B.k0 + 1), blk, 0, stream>>>(
            sp, u, v, w, B.i0, B.i1, B.j0, B.j1, B.k0, coef, Lf.u, Lf.v, Lf.w);
      }
    }
    UF_CUDA(cudaGetLastError());
    return UF_OK;
  }

  uf_status objective(double z_lo, double z_hi, double u_hi, double u_lo, double* J) override {
    if (!J) return fail(UF_ERR_ARG, "NULL output");
    int k_lo = d.nz, k_hi = -1;
    for (int k = 0; k < d.nz; ++k) {
      const double zc = (k + 0.5) * d.h;
      if (zc >= z_lo && zc <= z_hi) { k_lo = std::min(k_lo, k); k_hi = std::max(k_hi, k); }
    }
    if (k_hi < k_lo) { *J = 0.0; return UF_OK; }
    int zc;
    const dim3 go = chunk_grid(d.nx, d.ny, k_hi - k_lo + 1, &zc);
    uf::k_objective<T><<<go, dim3(uf::BX, uf::BY), 0, stream>>>(sp, u, v, w, k_lo, k_hi, zc, u_hi, u_lo, partials,
                                                                 &st->ticket[0], scal);
    UF_CUDA(cudaGetLastError());
    UF_CUDA(cudaMemcpyAsync(J, scal, sizeof(double), cudaMemcpyDeviceToHost, stream));
    UF_CUDA(cudaStreamSynchronize(stream));
    return UF_OK;
  }

  uf_status divergence(double* outv) override {
    if (!outv) return fail(UF_ERR_ARG, "NULL output");
    int zc;
    const dim3 gd = chunk_grid(d.nx, d.ny, d.nz, &zc);
    uf::k_divergence<T><<<gd, dim3(uf::BX, uf::BY), 0, stream>>>(sp, u, v, w, zc, partials, &st->ticket[0], scal + 2);
    UF_CUDA(cudaGetLastError());
    double h2[2];
    UF_CUDA(cudaMemcpyAsync(h2, scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    UF_CUDA(cudaStreamSynchronize(stream));
    *outv = h2[1] > 0 ? std::sqrt(h2[0] / h2[1]) : std::sqrt(h2[0]);
    return UF_OK;
  }

  uf_status apply_poisson(const void* x, void* y) override {
    uf_status s = copy_in(q, d.nx, d.ny, d.nz, P.Pc, x);
    if (s != UF_OK) return s;
    int zc;
    dim3 g = chunk_grid(d.nx, d.ny, d.nz, &zc);
    uf::k_apply_level<T><<<g, dim3(uf::BX, uf::BY), 0, stream>>>(lv[0], q, d0, zc);
    UF_CUDA(cudaGetLastError());
    return copy_out(y, d0, d.nx, d.ny, d.nz, P.Pc);
  }

  // Stand-alone solve of A p = b (b in the grid's b buffer) from the guess
  // in the pressure store, committed into it.
  uf_status ensure_solve_exec() {
    if (solve_exec) return UF_OK;
    int nf, ns, ni;
    auto pre = [&](cudaStream_t s2) {
      int zc;
      dim3 g = chunk_grid(d.nx, d.ny, d.nz, &zc);
      uf::k_solve_reset<T><<<g, dim3(uf::BX, uf::BY), 0, s2>>>(lv[0], b, zc, partials, st);
      rec_count++;
    };
    auto post = [&](cudaStream_t s2) {
      uf::k_pressure_commit<T><<<plane_grid(d.nx, d.ny, d.nz), dim3(uf::BX, uf::BY), 0, s2>>>(sp, p, pd, gd, st);
      rec_count++;
    };
    return capture(&solve_exec, pre, post, &nf, &ns, &ni);
  }

  uf_status poisson_solve(const void* bsrc, int* iters, double* rel) override {
    uf_status s = copy_in(b, d.nx, d.ny, d.nz, P.Pc, bsrc);
    if (s != UF_OK) return s;
    s = ensure_solve_exec();
    if (s != UF_OK) return s;
    UF_CUDA(cudaGraphLaunch(solve_exec, stream));
    UF_CUDA(copy_cell_ps(gd, pd));
    uf_step_stats o;
    s = check_device(&o);
    if (iters) *iters = o.cg_iters;
    if (rel) *rel = o.cg_rel_residual;
    return s;
  }

  uf_status launch_counts(int* fixed, int* per_iter) override {
    uf_status s = build_step_graphs();
    if (s != UF_OK) return s;
    if (fixed) *fixed = launches_fixed + launches_solve_setup;
    if (per_iter) *per_iter = launches_per_iter;
    return UF_OK;
  }

  int last_launches() override {
    if (last_iters < 0) return 0;
    return launches_fixed + launches_solve_setup + last_iters * launches_per_iter;
  }
};

}  // namespace

// ============================================================== C ABI ====

extern "C" {

void uf_default_desc(uf_grid_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->nx = 64; d->ny = 32; d->nz = 16; d->h = 2.0;
  d->precision = UF_F32;
  d->wind_dir_deg = 0.0; d->u_ref = 5.0; d->z_ref = 10.0; d->z0 = 0.5;
  d->inflow_loglaw = 0; d->ground_noslip = 1;
  d->rho = 1.225; d->nu = 1.5e-5; d->Cd = 1.0; d->a = 0.62; d->b = 2.5; d->e = 1e-10;
  d->I = 0.1; d->L = 10.0;
  d->C_mu = 0.09; d->alpha = 0.52; d->beta = 0.0708; d->sigma = 0.5; d->sigma_star = 0.6; d->C_lim = 7.0 / 8.0;
  d->cfl = 0.5; d->fixed_dt = 0.0; d->k_min = 1e-10; d->omega_min = 1e-6;
  d->precond = UF_PRECOND_MG; d->cg_tol = 0.0; d->cg_max_iter = 200;
  d->ai_omega = 1.65; d->mg_jacobi_omega = 6.0 / 7.0; d->mg_coarse_max = 512;
  d->mg_smoother = UF_SMOOTH_CHEBY;
  d->mg_transfer = UF_TRANSFER_LINEAR;
  d->cg_stop_rule = UF_STOP_RESIDUAL;
}

size_t uf_workspace_bytes(const uf_grid_desc* d) {
  std::string why;
  if (!desc_valid(d, &why)) {
    g_err = why;
    return 0;
  }
  return make_plan(d).total;
}

uf_status uf_create_grid(const uf_grid_desc* d, void* d_workspace, size_t bytes, void* stream, uf_grid** out) {
  std::string why;
  if (!out) return fail(UF_ERR_ARG, "NULL output handle");
  *out = nullptr;
  if (!desc_valid(d, &why)) return fail(UF_ERR_ARG, why);
  if (!d_workspace) return fail(UF_ERR_ARG, "NULL workspace");
  if (!stream) return fail(UF_ERR_ARG, "pass a created CUDA stream (the legacy default stream cannot be captured)");
  const Plan P = make_plan(d);
  if (bytes < P.total) return fail(UF_ERR_NOMEM, "workspace smaller than uf_workspace_bytes()");
  uf_grid* g = nullptr;
  uf_status s;
  if (d->precision == UF_F64) {
    auto* gi = new GridImpl<double>();
    s = gi->setup(d, d_workspace, (cudaStream_t)stream);
    g = gi;
  } else {
    auto* gi = new GridImpl<float>();
    s = gi->setup(d, d_workspace, (cudaStream_t)stream);
    g = gi;
  }
  if (s != UF_OK) {
    delete g;
    return s;
  }
  *out = g;
  return UF_OK;
}

uf_status uf_destroy(uf_grid* g) {
  if (!g) return fail(UF_ERR_ARG, "NULL grid");
  delete g;
  return UF_OK;
}

#define UF_NEED(g) if (!(g)) return fail(UF_ERR_ARG, "NULL grid")

// Every entry point that works on a grid runs inside an NVTX range named
// after it (seen by Nsight Systems and other NVTX tools; next to free
// without one), and hands its status to after_call, which in a library built
// with -DUF_BOUNDS_CHECK reports an out-of-bounds index (UF_ERR_BOUNDS).
#define UF_CALL(g, name, expr)         \
  do {                                 \
    UF_NEED(g);                        \
    NvtxRange nvtx_range_(name);       \
    return (g)->after_call(expr);      \
  } while (0)

uf_status uf_set_porosity(uf_grid* g, const void* phi) { UF_CALL(g, "uf_set_porosity", g->set_porosity(phi)); }
uf_status uf_set_state(uf_grid* g, int f, const void* b) { UF_CALL(g, "uf_set_state", g->set_state(f, b)); }
uf_status uf_get_state(uf_grid* g, int f, void* b) { UF_CALL(g, "uf_get_state", g->get_state(f, b)); }
uf_status uf_init_state(uf_grid* g) { UF_CALL(g, "uf_init_state", g->init_state()); }
uf_status uf_step(uf_grid* g, uf_step_stats* s) { UF_CALL(g, "uf_step", g->step(s)); }
uf_status uf_run(uf_grid* g, int n, uf_step_stats* s) { UF_CALL(g, "uf_run", g->run(n, s)); }
uf_status uf_objective(uf_grid* g, double z_lo, double z_hi, double u_hi, double u_lo, double* J) {
  UF_CALL(g, "uf_objective", g->objective(z_lo, z_hi, u_hi, u_lo, J));
}
uf_status uf_divergence(uf_grid* g, double* out) { UF_CALL(g, "uf_divergence", g->divergence(out)); }
uf_status uf_apply_poisson(uf_grid* g, const void* x, void* y) { UF_CALL(g, "uf_apply_poisson", g->apply_poisson(x, y)); }
uf_status uf_poisson_solve(uf_grid* g, const void* b, int* iters, double* rel) {
  UF_CALL(g, "uf_poisson_solve", g->poisson_solve(b, iters, rel));
}
int uf_last_step_launches(uf_grid* g) { return g ? g->last_launches() : 0; }
uf_status uf_launch_counts(uf_grid* g, int* fixed, int* per_iter) { UF_CALL(g, "uf_launch_counts", g->launch_counts(fixed, per_iter)); }
uf_status uf_profile_step(uf_grid* g, uf_kernel_time* out, int capacity, int* count, uf_step_stats* stats) {
  if (capacity < 0) return fail(UF_ERR_ARG, "negative capacity");
  UF_CALL(g, "uf_profile_step", g->profile_step(out, capacity, count, stats));
}
size_t uf_adjoint_workspace_bytes(uf_grid* g, int nsteps, int ckpt_every) {
  return g ? g->adjoint_bytes(nsteps, ckpt_every) : 0;
}
uf_status uf_adjoint_run(uf_grid* g, void* ws, size_t bytes, int nsteps, int ckpt_every, double z_lo, double z_hi,
                         double u_hi, double u_lo, void* dJ_dphi, double* J_out) {
  UF_CALL(g, "uf_adjoint_run", g->adjoint_run(ws, bytes, nsteps, ckpt_every, z_lo, z_hi, u_hi, u_lo, dJ_dphi, J_out));
}
uf_status uf_set_fields(uf_grid* g, int n, const int* fields, const void* const* bufs) {
  UF_CALL(g, "uf_set_fields", g->set_fields(n, fields, bufs));
}
size_t uf_state_bytes(uf_grid* g) { return g ? g->state_bytes() : 0; }
uf_status uf_save_state(uf_grid* g, void* buf, size_t bytes) { UF_CALL(g, "uf_save_state", g->save_snapshot(buf, bytes)); }
uf_status uf_load_state(uf_grid* g, const void* buf, size_t bytes) { UF_CALL(g, "uf_load_state", g->load_snapshot(buf, bytes)); }
uf_status uf_get_fields(uf_grid* g, int n, const int* fields, void* const* bufs) {
  UF_CALL(g, "uf_get_fields", g->get_fields(n, fields, bufs));
}
uf_status uf_objective_ex(uf_grid* g, const uf_objective_desc* obj, double* J_out) {
  UF_CALL(g, "uf_objective_ex", g->objective_ex(obj, J_out));
}
uf_status uf_adjoint_run_ex(uf_grid* g, void* d_ws, size_t bytes, int nsteps, int ckpt_every,
                            const uf_objective_desc* obj, void* dJ_dphi, double* J_out) {
  UF_CALL(g, "uf_adjoint_run_ex", g->adjoint_run_ex(d_ws, bytes, nsteps, ckpt_every, obj, dJ_dphi, J_out));
}
uf_status uf_mesh_to_phi(uf_grid* g, int ntri, const double* tris, int nobj, const int* obj_first,
                         const int* obj_count, const double* obj_phi, int sub, void* phi_out) {
  UF_CALL(g, "uf_mesh_to_phi", g->mesh_to_phi(ntri, tris, nobj, obj_first, obj_count, obj_phi, sub, phi_out));
}
uf_status uf_substep(uf_grid* g, int which, int transpose, const void* const* in, const void* const* cot,
                     void* const* out) {
  UF_CALL(g, "uf_substep", g->substep(which, transpose, in, cot, out));
}
uf_status uf_step_vjp(uf_grid* g, void* d_ws, size_t bytes, const void* const* lam_out, void* const* lam_in,
                      void* lam_phi) {
  UF_CALL(g, "uf_step_vjp", g->step_vjp(d_ws, bytes, lam_out, lam_in, lam_phi));
}
uf_status uf_get_tuning(uf_grid* g, uf_tuning* out, int* levels) {
  UF_CALL(g, "uf_get_tuning", g->get_tuning(out, levels));
}
uf_status uf_set_tuning(uf_grid* g, const uf_tuning* t) {
  UF_CALL(g, "uf_set_tuning", g->set_tuning(t));
}
uf_status uf_autotune(uf_grid* g, int reps, uf_tuning* chosen, double* best_ms) {
  UF_CALL(g, "uf_autotune", g->autotune(reps, chosen, best_ms));
}
uf_status uf_design_to_phi(uf_grid* g, int nbox, const double* boxes, const double* theta, double width, void* phi_out) {
  UF_CALL(g, "uf_design_to_phi", g->design_phi(nbox, boxes, theta, width, phi_out));
}
uf_status uf_design_vjp(uf_grid* g, int nbox, const double* boxes, const double* theta, double width,
                        const void* dJ_dphi, double* dJ_dtheta) {
  UF_CALL(g, "uf_design_vjp", g->design_vjp(nbox, boxes, theta, width, dJ_dphi, dJ_dtheta));
}
const char* uf_last_error(void) { return g_err.c_str(); }
int uf_bounds_checked(void) {
#ifdef UF_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

}  // extern "C"
