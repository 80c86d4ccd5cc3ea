// Internal interface between the single-grid API (capi.cu) and the batch
// (batch.cu): the abstract grid behind the opaque uf_grid handle, and a plain
// view of one grid's device state that the batched kernels read.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>

#include "../../include/uf.h"
#include "mg_fused.cuh"
#include "momentum_fused.cuh"

// Launch geometry and buffers of one grid, as its own graphs use them; the
// batch replays the same blocks (same z chunks, same tail level), so a grid
// stepped inside a batch computes exactly what it computes alone.
template <typename T>
struct GridView {
  uf_grid_desc d;
  uf::StepParams<T> sp;
  uf::AdvectArgs<T> adv;
  T *u, *v, *w, *uh, *vh, *wh, *ut, *vt, *wt, *u2, *v2, *w2, *cc, *nut, *p, *b, *z, *q, *d0, *d1;
  uf::PStore<T> *pd, *gd;          // pressure p^n and the next guess (pressure store); p: the correction
  T* kb[2];
  T* ob[2];
  int parity;                      // kb[parity], ob[parity] hold the current k, omega
  size_t n_u, n_v, n_w;            // padded face-lattice sizes
  uf::Level<T> lv[uf::MAX_LEVELS];
  int nl;                          // multigrid levels
  int tail_level;                  // first level of the shared-memory tail
  uf::TailArgs<T> tail;
  size_t tail_smem;
  int march_g[uf::MAX_LEVELS][3];  // blocks of the z-marching level kernels
  int march_zc[uf::MAX_LEVELS];    // z planes per block
  int chunk_g[3], chunk_zc;        // z-chunked reductions over the cells (and the fused momentum pass)
  int adv_g[3], adv_zc;            // blocks and z planes per block of the fused advection
  int dt_blocks;                   // blocks of the CFL reduction
  uf::SolveState* st;
  double* partials;
  double* dt;
  T* dtT;
  uf::SmoothW<T> sw;               // smoother weights
};

// An NVTX range (host side) for the lifetime of a scope.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// The message of a bounds-check record (UF_BOUNDS_CHECK builds).
inline std::string bounds_text(const uf::BoundsHit& h) {
  static const char* arrays[] = {"u lattice", "v lattice", "cell / w lattice", "multigrid level"};
  return std::string("index out of its array: ") + (h.array >= 0 && h.array < 4 ? arrays[h.array] : "?") + " at (" +
         std::to_string(h.i) + ", " + std::to_string(h.j) + ", " + std::to_string(h.k) + ")";
}

struct uf_grid {
  virtual ~uf_grid() {}
  // Status of a finished entry point: s, or UF_ERR_BOUNDS where a library
  // built with -DUF_BOUNDS_CHECK recorded an index outside its array.
  virtual uf_status after_call(uf_status s) { return s; }
  virtual uf_status set_porosity(const void*) = 0;
  virtual uf_status set_state(int, const void*) = 0;
  virtual uf_status get_state(int, void*) = 0;
  virtual uf_status set_fields(int, const int*, const void* const*) = 0;
  virtual uf_status get_fields(int, const int*, void* const*) = 0;
  virtual uf_status init_state() = 0;
  virtual uf_status step(uf_step_stats*) = 0;
  virtual uf_status run(int, uf_step_stats*) = 0;
  virtual uf_status objective(double, double, double, double, double*) = 0;
  virtual uf_status divergence(double*) = 0;
  virtual uf_status apply_poisson(const void*, void*) = 0;
  virtual uf_status poisson_solve(const void*, int*, double*) = 0;
  virtual int last_launches() = 0;
  virtual uf_status launch_counts(int*, int*) = 0;
  virtual uf_status profile_step(uf_kernel_time*, int, int*, uf_step_stats*) = 0;
  virtual size_t adjoint_bytes(int, int) = 0;
  virtual uf_status adjoint_run(void*, size_t, int, int, double, double, double, double, void*, double*) = 0;
  virtual uf_status objective_ex(const uf_objective_desc*, double*) = 0;
  virtual uf_status adjoint_run_ex(void*, size_t, int, int, const uf_objective_desc*, void*, double*) = 0;
  virtual uf_status step_vjp(void*, size_t, const void* const*, void* const*, void*) = 0;
  virtual uf_status substep(int, int, const void* const*, const void* const*, void* const*) = 0;
  virtual uf_status mesh_to_phi(int, const double*, int, const int*, const int*, const double*, int, void*) = 0;
  virtual uf_status design_phi(int, const double*, const double*, double, void*) = 0;
  virtual uf_status design_vjp(int, const double*, const double*, double, const void*, double*) = 0;
  virtual uf_status get_tuning(uf_tuning*, int*) = 0;
  virtual uf_status set_tuning(const uf_tuning*) = 0;
  virtual uf_status autotune(int, uf_tuning*, double*) = 0;
  // batch support
  virtual const uf_grid_desc& desc() const = 0;
  virtual bool has_state() const = 0;
  virtual void fill_view(void* view) = 0;          // GridView<T>* of the grid's precision
  virtual void advanced(int nsteps) = 0;           // the state was stepped nsteps times by a batch
  virtual uf_status read_status(uf_step_stats*) = 0;
  // checkpoint / resume
  virtual size_t state_bytes() = 0;
  virtual uf_status save_snapshot(void*, size_t) = 0;
  virtual uf_status load_snapshot(const void*, size_t) = 0;
};
