// uf_poisson_solve_static: a pressure solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// running inside another framework's allocator-controlled region (where a
// stray cudaMalloc would fragment or bypass its pool), plug-ins loaded into
// a host application that owns the CUDA context and forbids allocations
// after start-up, and real-time loops that must not take the allocator's
// locks or risk an out-of-memory failure in the middle of a run.  This entry
// point serves them: the caller passes only the right-hand side and the
// pressure buffer, and the solver's scratch (CG vectors, FP64 reduction
// partials, solver state) lives in the file-scope array below, which the
// CUDA module reserves when the library is loaded and keeps on every device
// until the process exits.
//
// The solve is the same as uf_poisson_solve on a grid built with
// precond = UF_PRECOND_AI1: preconditioned CG on the 7-point pressure
// operator of Sec. 3 with the first-order approximate inverse (Sec. 3,
// App. A.3) at w = 1.65, FP32 vectors and FP64 inner products; it reuses the
// library's kernels unchanged and changes none of their code paths.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/uf.h"
#include "solver_kernels.cuh"

// Sets the thread-local message returned by uf_last_error() (capi.cu).
void uf_internal_set_last_error(const char* msg);

namespace {

constexpr size_t kStaticBytes = UF_STATIC_SCRATCH_BYTES;
constexpr int kStaticPartials = 8192;
constexpr size_t kStateBytes = 256;    // SolveState, padded
constexpr size_t kPartialBytes = sizeof(double) * kStaticPartials;

// The shared scratch.  Host code must not use this name as an address (on
// the host it is only a stand-in); it uses the per-device address obtained
// from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_uf_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

uf_status static_fail(uf_status s, const std::string& msg) {
  uf_internal_set_last_error(msg.c_str());   // reported by uf_last_error()
  return s;
}

// Device address of the scratch array on the current device; looked up once
// per device, with that device current.
uf_status scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(UF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return static_fail(UF_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_uf_static_scratch);
    if (e != cudaSuccess || !p)
      return static_fail(UF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = reinterpret_cast<unsigned char*>(g_addr[dev]);
  return UF_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" uf_status uf_poisson_solve_static(int nx, int ny, int nz, double wind_dir_deg, const float* b, float* p,
                                             double tol, int max_iter, void* stream, int* iters,
                                             double* rel_residual) {
  if (nx < 2 || ny < 2 || nz < 1) return static_fail(UF_ERR_ARG, "need nx, ny >= 2 and nz >= 1");
  const long long cells = (long long)nx * ny * nz;
  if (cells > UF_STATIC_MAX_CELLS)
    return static_fail(UF_ERR_ARG, "grid has " + std::to_string(cells) + " cells; uf_poisson_solve_static handles at most " +
                                       std::to_string(UF_STATIC_MAX_CELLS));
  if ((long long)((nx + 31) / 32) * ((ny + 7) / 8) > kStaticPartials / 2)
    return static_fail(UF_ERR_ARG, "nx * ny too large for the reduction scratch");
  if (!b || !p) return static_fail(UF_ERR_ARG, "NULL b or p");
  if (!stream) return static_fail(UF_ERR_ARG, "pass a created CUDA stream");
  if (!(tol > 0) || max_iter < 1) return static_fail(UF_ERR_ARG, "tol > 0 and max_iter >= 1 required");
  const double th = wind_dir_deg * M_PI / 180.0;
  const double cx = std::cos(th), sy = std::sin(th), tau = 1e-9;
  if (!(std::fabs(cx) > tau || std::fabs(sy) > tau)) return static_fail(UF_ERR_ARG, "wind direction undefined");
  cudaStream_t s = (cudaStream_t)stream;
  static_assert(kStateBytes >= sizeof(uf::SolveState), "state slot too small");
  const size_t need = kStateBytes + kPartialBytes + 5 * align256((size_t)UF_STATIC_MAX_CELLS * sizeof(float));
  if (need > kStaticBytes) return static_fail(UF_ERR_ARG, "static scratch smaller than its stated maximum");

  unsigned char* base = nullptr;
  uf_status rs = scratch_address(&base);
  if (rs != UF_OK) return rs;

  // scratch layout: state | partials | r z q d0 d1 (dense, x fastest)
  const size_t vec = align256((size_t)cells * sizeof(float));
  uf::SolveState* st = reinterpret_cast<uf::SolveState*>(base);
  double* partials = reinterpret_cast<double*>(base + kStateBytes);
  float* r = reinterpret_cast<float*>(base + kStateBytes + kPartialBytes);
  float* z = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(r) + vec);
  float* q = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(z) + vec);
  float* d0 = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(q) + vec);
  float* d1 = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(d0) + vec);

  uf::Level<float> L;
  std::memset(&L, 0, sizeof(L));
  L.nx = nx; L.ny = ny; L.nz = nz; L.P = nx;
  L.wx = L.wy = L.wz = 1.0f;
  const double inward[4] = {cx, -cx, sy, -sy};
  for (int q4 = 0; q4 < 4; ++q4)
    if (inward[q4] < -tau) L.out_mask |= 1 << q4;   // outlet sides: p = 0 ghost
  L.r = r;

  // fresh solver state: every call starts from zeroed tickets and counters
  uf::SolveState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.tol2 = tol * tol;
  s0.max_iter = max_iter;
  cudaError_t e = cudaMemcpyAsync(st, &s0, sizeof(s0), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return static_fail(UF_ERR_CUDA, std::string("state upload: ") + cudaGetErrorString(e));

  int zc;
  const int gx = (nx + uf::BX - 1) / uf::BX, gy = (ny + uf::BY - 1) / uf::BY;
  int chunks = std::max(1, std::min(nz, 2048 / std::max(1, gx * gy)));
  zc = (nz + chunks - 1) / chunks;
  chunks = (nz + zc - 1) / zc;
  const dim3 grid(gx, gy, chunks), blk(uf::BX, uf::BY);
  const float w = 1.65f;

  uf::k_solve_reset<float><<<grid, blk, 0, s>>>(L, b, zc, partials, st);
  uf::k_cg_init<float><<<grid, blk, 0, s>>>(L, b, p, nullptr, zc, partials, st, 0, 0);
  uf::k_precond_simple<float><<<grid, blk, 0, s>>>(L, 2, w, z, zc, 0, partials, st, 0, 0);
  // The host reads the convergence flag once per kPoll iterations.  Every
  // iteration kernel returns at once when the flag is set (and the update
  // kernel sets it at the iteration cap), so the launches queued past
  // convergence change nothing.
  constexpr int kPoll = 8;
  int conv = 0;
  e = cudaMemcpyAsync(&conv, &st->converged, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int it = 0; e == cudaSuccess && !conv && it <= max_iter; it += kPoll) {
    for (int m = 0; m < kPoll; ++m) {
      uf::k_cg_direction_spmv<float><<<grid, blk, 0, s>>>(L, z, d0, d1, q, zc, partials, st);
      uf::k_cg_update<float><<<grid, blk, 0, s>>>(L, p, d0, d1, q, zc, partials, st, 0, 0);
      uf::k_precond_simple<float><<<grid, blk, 0, s>>>(L, 2, w, z, zc, 1, partials, st, 0, 0);
    }
    e = cudaMemcpyAsync(&conv, &st->converged, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(UF_ERR_CUDA, std::string("static solve: ") + cudaGetErrorString(e));
  uf::SolveState h;
  e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return static_fail(UF_ERR_CUDA, std::string("state read: ") + cudaGetErrorString(e));
#ifdef UF_BOUNDS_CHECK
  {
    uf::BoundsHit bh;
    if (uf::bounds_hit_take(s, &bh))
      return static_fail(UF_ERR_BOUNDS, "index out of its array (" + std::to_string(bh.array) + ": " +
                                            std::to_string(bh.i) + ", " + std::to_string(bh.j) + ", " +
                                            std::to_string(bh.k) + ")");
  }
#endif
  if (iters) *iters = h.iter;
  if (rel_residual) *rel_residual = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
  if (h.status == uf::DEV_NOT_CONVERGED) return static_fail(UF_ERR_NOT_CONVERGED, "CG reached its iteration cap");
  if (h.status == uf::DEV_NAN) return static_fail(UF_ERR_NAN, "non-finite residual");
  return UF_OK;
}
