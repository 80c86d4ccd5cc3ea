// Batched execution: many independent grids (design variants, wind
// directions, uneven sizes) advance together.  Every phase of the step is one
// persistent launch whose blocks walk a work list of (instance, tile) items;
// one captured CUDA graph holds the whole step, with a single conditional
// WHILE node for all instances' CG loops.
//
// The items of an instance are exactly the blocks its own graph launches
// (same tiles, z chunks and tail level, read from GridView), and every
// reduction still runs over that instance's blocks only, in the same order,
// so an instance computes bit for bit what it computes alone.  Converged
// instances skip their items while the others iterate; the WHILE condition
// clears when the last one finishes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/uf.h"
#include "grid_base.cuh"

// Sets the thread-local message returned by uf_last_error() (capi.cu).
void uf_internal_set_last_error(const char* msg);

struct uf_batch {
  virtual ~uf_batch() {}
  // Status of a finished entry point (see uf_grid::after_call).
  virtual uf_status after_call(uf_status s) { return s; }
  virtual uf_status grid(int, uf_grid**) = 0;
  virtual uf_status run(int, uf_step_stats*) = 0;
  virtual uf_status launch_counts(int*, int*) = 0;
  virtual uf_status autotune(int, int*) = 0;
  virtual uf_status profile_step(uf_kernel_time*, int, int*) = 0;
};

namespace {

using uf::VBlock;

uf_status bfail(uf_status s, const std::string& msg) {
  uf_internal_set_last_error(msg.c_str());
  return s;
}

#define UFB_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bfail(UF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

constexpr int kMaxBatch = UF_MAX_BATCH;

// Work list of one batched launch: entry e covers items [start[e],
// start[e+1]) of instance inst[e], whose blocks form a gx x gy x (count /
// (gx gy)) grid; zc is that instance's z chunk for this launch.
struct LaunchMap {
  int n, total;
  int start[kMaxBatch + 1];
  int inst[kMaxBatch];
  int gx[kMaxBatch], gy[kMaxBatch];
  int zc[kMaxBatch];
  int gz_planes[kMaxBatch];   // plane kernels: planes of instance i (indexed by instance)
};

// Launch kinds: one work list each (march levels: one per level).
enum MapKind { MAP_CFL = 0, MAP_CELL, MAP_FACE, MAP_CHUNK, MAP_TAIL, MAP_ADV, MAP_MARCH0 };
constexpr int kMaps = MAP_MARCH0 + uf::MAX_LEVELS;

__device__ __forceinline__ int map_entry(const LaunchMap* __restrict__ m, int w) {
  int lo = 0, hi = m->n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (m->start[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Persistent loop: block b takes items b, b + gridDim.x, ...  At any moment
// the resident blocks work on one window of neighbouring tiles, so halos are
// shared through L2 and DRAM pages stay local (a contiguous run of items per
// block measured 1.4-1.5x slower on the 32-instance workload).  The item
// index only grows, so the work-list entry is found once and then advanced;
// f(instance, z chunk, block coordinates) runs the kernel body on one item.
template <typename F>
__device__ __forceinline__ void for_items(const LaunchMap* __restrict__ m, F&& f) {
  const int total = m->total;
  int w = blockIdx.x;
  if (w >= total) return;
  int e = map_entry(m, w);
  int s0 = m->start[e], s1 = m->start[e + 1];
  for (; w < total; w += gridDim.x) {
    while (w >= s1) {   // items only move forward
      ++e;
      s0 = s1;
      s1 = m->start[e + 1];
    }
    const int lin = w - s0, gx = m->gx[e], gy = m->gy[e];
    const VBlock vb{lin % gx, (lin / gx) % gy, lin / (gx * gy), lin, s1 - s0};
    f(m->inst[e], m->zc[e], vb);
    __syncthreads();   // the next item reuses the shared memory
  }
}

// Element-wise plane kernels: an item is a 32 x 8 tile over `zc` consecutive
// planes (their results do not depend on how the planes are grouped).
template <typename F>
__device__ __forceinline__ void for_plane_items(const LaunchMap* __restrict__ m, F&& f) {
  for_items(m, [&](int i, int zc, const VBlock& vb) {
    const int p0 = vb.z * zc, p1 = min(p0 + zc, m->gz_planes[i]);
    for (int z = p0; z < p1; ++z) f(i, VBlock{vb.x, vb.y, z, 0, 1});
  });
}

template <typename T>
using View = GridView<T>;

// One batched launch, passed by value in the kernel's parameter space: the
// work list and, per instance, what the kernel body needs.  The instance
// index is uniform across a block, so every field is read from the constant
// bank as the single-grid kernels read their own parameters.
template <typename P>
struct Args {
  LaunchMap m;
  P at[kMaxBatch];
};

template <typename T>
struct CflP {
  const T *u, *v, *w;
  size_t nu, nv, nw;
  double cfl_h;
  double* partials;
  unsigned int* ticket;
  double* dt;
  T* dtT;
};
template <typename T>
struct CellP {   // eddy viscosity, k-omega
  uf::StepParams<T> sp;
  const T *u, *v, *w;
  T* nut;
  T* kb[2];
  T* ob[2];
};
template <typename T>
struct AdvP {
  uf::AdvectArgs<T> a;
};
template <typename T>
struct MomP {    // fused diffusion + drag + BCs + pressure right-hand side
  uf::MomentumArgs<T> M;
};
template <typename T>
struct ProjP {   // projection from the pressure store
  uf::StepParams<T> sp;
  const uf::PStore<T>* pr;
  T *u, *v, *w;
};
template <typename T>
struct CommitP { // p^{n+1} from the solve's correction, in the pressure store
  uf::StepParams<T> sp;
  T* delta;
  uf::PStore<T> *pn, *gs;
  const uf::SolveState* st;
};
template <typename T>
struct CgP {     // CG initial residual, direction + A d
  uf::Level<T> L;
  const T* b;
  T* x;
  const uf::PStore<T>* g;   // guess of the correction solve (pressure store)
  const T* z;
  T *d0, *d1, *q;
  double* partials;
  uf::SolveState* st;
};
template <typename T>
struct MgP {     // V-cycle level kernels
  uf::Level<T> F, C;
  uf::SmoothW<T> sw;
  T* x;
  const T *d0, *d1, *q;
  T* out;
  double* partials;
  uf::SolveState* st;
};

// Minimum resident blocks per SM (second __launch_bounds__ argument): the
// batch's working set exceeds L2, so these kernels wait on DRAM latency and
// gain from more resident warps; measured on the 32-instance workload, 4
// blocks of 256 threads for the fused level kernels and 6 for the plane
// kernels beat the register-unbounded build (small spills included).
template <typename T>
__global__ void __launch_bounds__(256) kb_cfl(const __grid_constant__ Args<CflP<T>> A) {
  for_items(&A.m, [&](int i, int, const VBlock& vb) {
    const CflP<T>& P = A.at[i];
    uf::cfl_dt_body<T>(P.u, P.nu, P.v, P.nv, P.w, P.nw, P.cfl_h, P.partials, P.ticket, P.dt, P.dtT, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT, 6) kb_eddy(const __grid_constant__ Args<CellP<T>> A,
                                                  const int* __restrict__ par) {
  for_plane_items(&A.m, [&](int i, const VBlock& vb) {
    const CellP<T>& P = A.at[i];
    const int a = par[i];
    uf::eddy_viscosity_body<T>(P.sp, P.u, P.v, P.w, P.kb[a], P.ob[a], P.nut, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::MT, UF_ADVECT_MINB) kb_advect_fused(const __grid_constant__ Args<AdvP<T>> A) {
  for_items(&A.m, [&](int i, int zc, const VBlock& vb) { uf::advect_fused_body<T>(A.at[i].a, zc, vb); });
}

template <typename T>
__global__ void __launch_bounds__(uf::MT) kb_momentum_fused(const __grid_constant__ Args<MomP<T>> A) {
  for_items(&A.m, [&](int i, int, const VBlock& vb) { uf::momentum_fused_body<T>(A.at[i].M, vb); });
}

// Opens the batch's CG loop: every instance that takes part is unfinished.
__global__ void kb_begin_solve(int* left, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *left = n;
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_cg_init(const __grid_constant__ Args<CgP<T>> A,
                                                     cudaGraphConditionalHandle cond, int use_cond, int* left) {
  for_items(&A.m, [&](int i, int zc, const VBlock& vb) {
    const CgP<T>& P = A.at[i];
    uf::cg_init_body<T>(P.L, P.b, P.x, P.g, zc, P.partials, P.st, cond, use_cond, left, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::FT) kb_cg_dir_q(const __grid_constant__ Args<CgP<T>> A) {
  for_items(&A.m, [&](int i, int zc, const VBlock& vb) {
    const CgP<T>& P = A.at[i];
    uf::cg_dir_q_body<T>(P.L, zc, P.z, P.d0, P.d1, P.q, P.partials, P.st, vb);
  });
}

template <typename T, int SM, bool CG>
__global__ void __launch_bounds__(uf::FT, 4) kb_mg_down(const __grid_constant__ Args<MgP<T>> A,
                                                     cudaGraphConditionalHandle cond, int use_cond, int* left) {
  for_items(&A.m, [&](int i, int zc, const VBlock& vb) {
    const MgP<T>& P = A.at[i];
    uf::mg_down_body<T, SM, CG>(P.F, P.C, P.sw, zc, P.x, P.d0, P.d1, P.q, P.partials, P.st, cond, use_cond,
                                CG ? left : nullptr, vb);
  });
}

// Linear transfers: the right-hand side of level l + 1 from the residual
// that the down kernel of level l stored (instances without them skip).
template <typename T>
__global__ void __launch_bounds__(uf::FT) kb_restrict_lin(const __grid_constant__ Args<MgP<T>> A) {
  for_items(&A.m, [&](int i, int zc, const VBlock& vb) {
    const MgP<T>& P = A.at[i];
    if (P.F.lin) uf::restrict_lin_body<T>(P.F, P.C, zc, P.st, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::FT) kb_prolong_lin(const __grid_constant__ Args<MgP<T>> A) {
  for_items(&A.m, [&](int i, int zc, const VBlock& vb) {
    const MgP<T>& P = A.at[i];
    if (P.F.lin) uf::prolong_lin_body<T>(P.F, P.C, zc, P.st, vb);
  });
}

template <typename T, int SM>
__global__ void __launch_bounds__(uf::TAIL_T) kb_mg_tail(const View<T>* __restrict__ V,
                                                         const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::mg_tail_body<T, SM>(G.tail, G.sw, G.st, vb);
  });
}

template <typename T, int SM, bool FINEST>
__global__ void __launch_bounds__(uf::FT, 4) kb_mg_up(const __grid_constant__ Args<MgP<T>> A, int mode) {
  for_items(&A.m, [&](int i, int zc, const VBlock& vb) {
    const MgP<T>& P = A.at[i];
    uf::mg_up_body<T, SM, FINEST>(P.F, P.C, P.sw, zc, P.out, mode, P.partials, P.st, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT, 6) kb_pressure_commit(const __grid_constant__ Args<CommitP<T>> A) {
  for_plane_items(&A.m, [&](int i, const VBlock& vb) {
    const CommitP<T>& P = A.at[i];
    uf::pressure_commit_body<T>(P.sp, P.delta, P.pn, P.gs, P.st, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_project(const __grid_constant__ Args<ProjP<T>> A) {
  for_plane_items(&A.m, [&](int i, const VBlock& vb) {
    const ProjP<T>& P = A.at[i];
    uf::project_body<T>(P.sp, P.pr, P.u, P.v, P.w, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT, 6) kb_turbulence(const __grid_constant__ Args<CellP<T>> A,
                                                        const int* __restrict__ par) {
  for_plane_items(&A.m, [&](int i, const VBlock& vb) {
    const CellP<T>& P = A.at[i];
    const int a = par[i], o = a ^ 1;
    uf::turbulence_body<T>(P.sp, P.u, P.v, P.w, P.kb[a], P.ob[a], P.kb[o], P.ob[o], vb);
  });
}

// End of a step: every instance's k and omega now live in the other buffer.
__global__ void kb_flip_parity(int* par, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) par[i] ^= 1;
}

// Device-side tables of a batch: the views, the work lists, the loop counter.
struct TableLayout {
  size_t views, maps, left, par, total;
};
template <typename T>
TableLayout table_layout(int n) {
  TableLayout L;
  L.views = 0;
  L.maps = round256(sizeof(View<T>) * n);
  L.left = L.maps + round256(sizeof(LaunchMap) * kMaps);
  L.par = L.left + 256;
  L.total = L.par + round256(sizeof(int) * kMaxBatch);
  return L;
}

template <typename T>
class BatchImpl final : public uf_batch {
 public:
  int n = 0;
  std::vector<uf_grid*> grids;
  cudaStream_t stream = nullptr, cap = nullptr, cap2 = nullptr;
  char* tables = nullptr;
  TableLayout TL;
  View<T>* d_views = nullptr;
  LaunchMap* d_maps = nullptr;
  int* d_left = nullptr;
  int* d_par = nullptr;                // per instance: which k / omega buffer is current
  std::vector<View<T>> views;          // host copies (parity included)
  std::vector<LaunchMap> maps;
  std::vector<View<T>> built_for;      // views the graph was captured for
  std::vector<int> par_host;
  cudaGraphExec_t exec = nullptr;
  int smoother = UF_SMOOTH_JACOBI;
  int n_fixed = 0, n_iter = 0, max_levels = 0;
  int sms = 0;
  size_t tail_smem = 0;

  ~BatchImpl() override {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
    for (uf_grid* g : grids) uf_destroy(g);
  }

  uf_status setup(int count, const uf_grid_desc* descs, char* ws, size_t bytes, cudaStream_t s) {
    n = count;
    stream = s;
    smoother = descs[0].mg_smoother;
    UFB_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    UFB_CUDA(cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking));
    int dev = 0;
    UFB_CUDA(cudaGetDevice(&dev));
    UFB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
      const size_t gb = round256(uf_workspace_bytes(&descs[i]));
      uf_grid* g = nullptr;
      const uf_status st = uf_create_grid(&descs[i], ws + off, gb, (void*)s, &g);
      if (st != UF_OK) return st;
      grids.push_back(g);
      off += gb;
    }
    tables = ws + off;
    TL = table_layout<T>(n);
    if (off + TL.total > bytes) return bfail(UF_ERR_NOMEM, "batch workspace too small");
    d_views = reinterpret_cast<View<T>*>(tables + TL.views);
    d_maps = reinterpret_cast<LaunchMap*>(tables + TL.maps);
    d_left = reinterpret_cast<int*>(tables + TL.left);
    d_par = reinterpret_cast<int*>(tables + TL.par);
    views.resize(n);
    return UF_OK;
  }

  uf_status grid(int i, uf_grid** out) override {
    if (i < 0 || i >= n || !out) return bfail(UF_ERR_ARG, "instance index out of range");
    *out = grids[i];
    return UF_OK;
  }

  // ----------------------------------------------------------- work lists
  void add_entry(LaunchMap& m, int inst, int gx, int gy, int gz, int zc) {
    const int e = m.n++;
    m.start[e] = m.total;
    m.inst[e] = inst;
    m.gx[e] = gx;
    m.gy[e] = gy;
    m.zc[e] = zc;
    m.total += gx * gy * gz;
    m.start[e + 1] = m.total;
  }

  // Plane kernels: items of kPlanesPerItem planes.
  static constexpr int kPlanesPerItem = 4;
  void add_plane_entry(LaunchMap& m, int inst, int gx, int gy, int planes) {
    m.gz_planes[inst] = planes;
    add_entry(m, inst, gx, gy, (planes + kPlanesPerItem - 1) / kPlanesPerItem, kPlanesPerItem);
  }

  void build_maps() {
    maps.assign(kMaps, LaunchMap());
    for (auto& m : maps) std::memset(&m, 0, sizeof(m));
    max_levels = 0;
    tail_smem = 0;
    for (int i = 0; i < n; ++i) {
      const View<T>& G = views[i];
      const uf_grid_desc& d = G.d;
      if (!(d.fixed_dt > 0)) {
        // the maximum is exact in any block order; fewer blocks than the
        // single-grid launch suffice
        const size_t faces = G.n_u + G.n_v + G.n_w;
        const int blocks = (int)std::min<size_t>(G.dt_blocks, std::max<size_t>(1, faces / (256 * 16)));
        add_entry(maps[MAP_CFL], i, blocks, 1, 1, 0);
      }
      add_plane_entry(maps[MAP_CELL], i, (d.nx + uf::BX - 1) / uf::BX, (d.ny + uf::BY - 1) / uf::BY, d.nz);
      add_plane_entry(maps[MAP_FACE], i, (d.nx + 1 + uf::BX - 1) / uf::BX, (d.ny + 1 + uf::BY - 1) / uf::BY,
                      3 * d.nz + 1);
      add_entry(maps[MAP_CHUNK], i, G.chunk_g[0], G.chunk_g[1], G.chunk_g[2], G.chunk_zc);
      add_entry(maps[MAP_ADV], i, G.adv_g[0], G.adv_g[1], G.adv_g[2], G.adv_zc);
      add_entry(maps[MAP_TAIL], i, 1, 1, 1, 0);
      for (int l = 0; l < G.tail_level; ++l)
        add_entry(maps[MAP_MARCH0 + l], i, G.march_g[l][0], G.march_g[l][1], G.march_g[l][2], G.march_zc[l]);
      max_levels = std::max(max_levels, G.tail_level);
      tail_smem = std::max(tail_smem, G.tail_smem);
    }
  }

  // Blocks of a persistent launch: the items, at most what stays resident.
  template <typename K>
  int grid_of(K kernel, int threads, size_t smem, int items) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    return std::max(1, std::min(items, per_sm * sms));
  }

  const LaunchMap* dm(int kind) const { return d_maps + kind; }
  int items(int kind) const { return maps[kind].total; }

  // ------------------------------------------------------------ recording
  // Every launch goes through L(): it counts, and in the eager profiling
  // mode brackets the launch with CUDA events on the launching stream.
  // Algorithmic bytes per launch: the single-grid figures summed over the
  // instances of the work list.
  int rec = 0;
  bool profiling = false;
  struct Rec {
    std::string name;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;

  template <typename F>
  void L(cudaStream_t s, const std::string& name, double bytes, F launch) {
    rec++;
    if (!profiling) {
      launch();
      return;
    }
    NvtxRange range(name.c_str());   // eager profiled step: one range per launch
    if (pool_used + 2 > pool.size())
      for (int k = 0; k < 2; ++k) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pool.push_back(e);
      }
    Rec r{name, bytes, pool[pool_used], pool[pool_used + 1]};
    pool_used += 2;
    cudaEventRecord(r.a, s);
    launch();
    cudaEventRecord(r.b, s);
    recs.push_back(r);
  }

  // sum over the instances of a work list of f(view)
  template <typename F>
  double sum_over(int kind, F f) const {
    double t = 0;
    const LaunchMap& m = maps[kind];
    for (int e = 0; e < m.n; ++e) t += f(views[m.inst[e]]);
    return t;
  }
  static double cells(const View<T>& G, int l) { return (double)G.lv[l].nx * G.lv[l].ny * G.lv[l].nz; }
  static constexpr double tb = sizeof(T);

  // Parameters of one batched launch: the work list of `kind` and, for each
  // of its instances, fill(P, view).
  template <typename P, typename Fill>
  const Args<P>& args(int kind, Fill fill) {
    static_assert(sizeof(Args<P>) <= 32000, "kernel parameters above the 32 KB limit");
    auto* a = reinterpret_cast<Args<P>*>(arg_buf.data());
    std::memset(a, 0, sizeof(Args<P>));
    a->m = maps[kind];
    for (int e = 0; e < a->m.n; ++e) {
      const int i = a->m.inst[e];
      fill(a->at[i], views[i]);
    }
    return *a;
  }
  std::vector<unsigned char> arg_buf = std::vector<unsigned char>(32768);

  static MgP<T> mg_params(const View<T>& G, int l) {
    MgP<T> P;
    std::memset(&P, 0, sizeof(P));
    P.F = G.lv[l];
    P.C = G.lv[l + 1];
    P.sw = G.sw;
    P.partials = G.partials;
    P.st = G.st;
    return P;
  }

  template <int SM>
  void rec_vcycle(cudaStream_t s, int mode, cudaGraphConditionalHandle cond, int use_cond) {
    const dim3 ft(uf::FT);
    for (int l = 0; l < max_levels; ++l) {
      const int kind = MAP_MARCH0 + l;
      const std::string sl = std::to_string(l);
      if (l == 0 && mode == 1) {
        auto k = kb_mg_down<T, SM, true>;
        const auto& A = args<MgP<T>>(kind, [](MgP<T>& P, const View<T>& G) {
          P = mg_params(G, 0);
          P.x = G.p;
          P.d0 = G.d0;
          P.d1 = G.d1;
          P.q = G.q;
        });
        L(s, "b_mg_down_cg_L0", sum_over(kind, [](const View<T>& G) { return (7 * cells(G, 0) + cells(G, 1)) * tb; }),
          [&] { k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(A, cond, use_cond, d_left); });
      } else {
        auto k = kb_mg_down<T, SM, false>;
        const auto& A = args<MgP<T>>(kind, [l](MgP<T>& P, const View<T>& G) { P = mg_params(G, l); });
        L(s, "b_mg_down_L" + sl,
          sum_over(kind, [l](const View<T>& G) {
            return (2 * cells(G, l) + (G.lv[l].lin ? cells(G, l) : cells(G, l + 1))) * tb;
          }),
          [&] { k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(A, cond, 0, nullptr); });
      }
      // linear transfers: right-hand side of level l + 1 for the instances
      // that keep it outside their tail
      if (l + 1 < max_levels) {
        const int kind1 = MAP_MARCH0 + l + 1;
        const double bytes = sum_over(kind1, [l](const View<T>& G) {
          return G.lv[l].lin ? (cells(G, l) + cells(G, l + 1)) * tb : 0.0;
        });
        if (bytes > 0) {
          auto k = kb_restrict_lin<T>;
          const auto& A = args<MgP<T>>(kind1, [l](MgP<T>& P, const View<T>& G) { P = mg_params(G, l); });
          L(s, "b_mg_restrict_L" + std::to_string(l + 1), bytes,
            [&] { k<<<grid_of(k, uf::FT, 0, items(kind1)), ft, 0, s>>>(A); });
        }
      }
    }
    {
      auto k = kb_mg_tail<T, SM>;
      L(s, "b_mg_tail", sum_over(MAP_TAIL, [](const View<T>& G) {
          return (double)G.tail.n_coarse * G.tail.n_coarse * 8 + 2 * cells(G, G.tail_level) * tb;
        }),
        [&] {
          k<<<grid_of(k, uf::TAIL_T, tail_smem, items(MAP_TAIL)), uf::TAIL_T, tail_smem, s>>>(d_views, dm(MAP_TAIL));
        });
    }
    for (int l = max_levels - 1; l >= 0; --l) {
      const int kind = MAP_MARCH0 + l;
      const std::string sl = std::to_string(l);
      // linear transfers: the prolonged correction of level l for the
      // instances whose level l + 1 lies outside their tail (the tail forms
      // it for the others)
      if (l + 1 < max_levels) {
        const int kind1 = MAP_MARCH0 + l + 1;
        const double pbytes = sum_over(kind1, [l](const View<T>& G) {
          return G.lv[l].lin ? (cells(G, l) + cells(G, l + 1)) * tb : 0.0;
        });
        if (pbytes > 0) {
          auto k = kb_prolong_lin<T>;
          const auto& A = args<MgP<T>>(kind1, [l](MgP<T>& P, const View<T>& G) { P = mg_params(G, l); });
          L(s, "b_mg_prolong_L" + sl, pbytes, [&] { k<<<grid_of(k, uf::FT, 0, items(kind1)), ft, 0, s>>>(A); });
        }
      }
      const double bytes = sum_over(kind, [l](const View<T>& G) { return (3 * cells(G, l) + cells(G, l + 1)) * tb; });
      const auto& A = args<MgP<T>>(kind, [l](MgP<T>& P, const View<T>& G) {
        P = mg_params(G, l);
        P.out = l == 0 ? G.z : G.lv[l].t;
      });
      if (l == 0) {
        auto k = kb_mg_up<T, SM, true>;
        L(s, "b_mg_up_L0", bytes, [&] { k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(A, mode); });
      } else {
        auto k = kb_mg_up<T, SM, false>;
        L(s, "b_mg_up_L" + sl, bytes, [&] { k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(A, mode); });
      }
    }
  }

  void vcycle(cudaStream_t s, int mode, cudaGraphConditionalHandle cond, int use_cond) {
    if (smoother == UF_SMOOTH_RBGS) rec_vcycle<uf::SM_RBGS>(s, mode, cond, use_cond);
    else rec_vcycle<uf::SM_JACOBI>(s, mode, cond, use_cond);
  }

  double plane_bytes(int kind, double per_cell) const {
    return sum_over(kind, [&](const View<T>& G) { return per_cell * cells(G, 0) * tb; });
  }

  static CellP<T> cell_params(const View<T>& G) {
    CellP<T> P;
    std::memset(&P, 0, sizeof(P));
    P.sp = G.sp;
    P.u = G.u; P.v = G.v; P.w = G.w;
    P.nut = G.nut;
    P.kb[0] = G.kb[0]; P.kb[1] = G.kb[1]; P.ob[0] = G.ob[0]; P.ob[1] = G.ob[1];
    return P;
  }
  static CgP<T> cg_params(const View<T>& G) {
    CgP<T> P;
    std::memset(&P, 0, sizeof(P));
    P.L = G.lv[0];
    P.b = G.b; P.x = G.p; P.z = G.z; P.d0 = G.d0; P.d1 = G.d1; P.q = G.q;
    P.g = G.gd;
    P.partials = G.partials;
    P.st = G.st;
    return P;
  }

  template <typename K, typename A>
  void launch_plane(K kernel, int kind, cudaStream_t s, const char* name, double per_cell, const A& a) {
    if (items(kind) == 0) return;
    L(s, name, plane_bytes(kind, per_cell),
      [&] { kernel<<<grid_of(kernel, uf::NT, 0, items(kind)), dim3(uf::BX, uf::BY), 0, s>>>(a); });
  }

  // a0-a6, the CG set-up (initial residual, first V-cycle)
  void rec_pre(cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
    const dim3 blk(uf::BX, uf::BY);
    if (items(MAP_CFL) > 0) {
      auto k = kb_cfl<T>;
      const auto& A = args<CflP<T>>(MAP_CFL, [](CflP<T>& P, const View<T>& G) {
        P.u = G.u; P.v = G.v; P.w = G.w;
        P.nu = G.n_u; P.nv = G.n_v; P.nw = G.n_w;
        P.cfl_h = G.d.cfl * G.d.h;
        P.partials = G.partials;
        P.ticket = &G.st->ticket[0];
        P.dt = G.dt;
        P.dtT = G.dtT;
      });
      L(s, "b_cfl_dt", plane_bytes(MAP_CFL, 3), [&] { k<<<grid_of(k, 256, 0, items(MAP_CFL)), 256, 0, s>>>(A); });
    }
    {
      auto k = kb_eddy<T>;
      const auto& A = args<CellP<T>>(MAP_CELL, [](CellP<T>& P, const View<T>& G) { P = cell_params(G); });
      L(s, "b_eddy_viscosity", plane_bytes(MAP_CELL, 6),
        [&] { k<<<grid_of(k, uf::NT, 0, items(MAP_CELL)), blk, 0, s>>>(A, d_par); });
    }
    {   // both MacCormack passes (the fused kernel of the single grids, bit for bit the two-pass form)
      auto k = kb_advect_fused<T>;
      const auto& A = args<AdvP<T>>(MAP_ADV, [](AdvP<T>& P, const View<T>& G) {
        P.a = G.adv;
        P.a.uh = P.a.vh = P.a.wh = nullptr;   // no tape
      });
      const size_t sm = uf::advect_fused_smem_total<T>();
      L(s, "b_advect_fused", plane_bytes(MAP_ADV, 6),
        [&] { k<<<grid_of(k, uf::MT, sm, items(MAP_ADV)), uf::MT, sm, s>>>(A); });
    }
    {   // diffusion, drag, velocity BCs and the pressure right-hand side in one pass
      auto k = kb_momentum_fused<T>;
      const auto& A = args<MomP<T>>(MAP_CHUNK, [](MomP<T>& P, const View<T>& G) {
        uf::MomentumArgs<T>& M = P.M;
        M.p = G.sp;
        M.ut = G.ut; M.vt = G.vt; M.wt = G.wt; M.nut = G.nut; M.cc = G.cc;
        M.u = G.u; M.v = G.v; M.w = G.w; M.b = G.b;
        M.u2t = M.v2t = M.w2t = nullptr;
        M.zc = G.chunk_zc;
        M.partials = G.partials;
        M.st = G.st;
      });
      const size_t sm = uf::momentum_fused_smem<T>();
      L(s, "b_momentum_fused", plane_bytes(MAP_CHUNK, 9),
        [&] { k<<<grid_of(k, uf::MT, sm, items(MAP_CHUNK)), uf::MT, sm, s>>>(A); });
    }
    L(s, "b_begin_solve", 0, [&] { kb_begin_solve<<<1, 32, 0, s>>>(d_left, n); });
    {
      auto k = kb_cg_init<T>;
      const auto& A = args<CgP<T>>(MAP_CHUNK, [](CgP<T>& P, const View<T>& G) { P = cg_params(G); });
      L(s, "b_cg_init", plane_bytes(MAP_CHUNK, 5),
        [&] { k<<<grid_of(k, uf::NT, 0, items(MAP_CHUNK)), blk, 0, s>>>(A, cond, use_cond, d_left); });
    }
    vcycle(s, 0, cond, use_cond);
  }

  // one CG iteration: direction + A d, then the V-cycle with the CG update
  void rec_iter(cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
    auto k = kb_cg_dir_q<T>;
    const auto& A = args<CgP<T>>(MAP_MARCH0, [](CgP<T>& P, const View<T>& G) { P = cg_params(G); });
    L(s, "b_cg_dir_q", plane_bytes(MAP_MARCH0, 4),
      [&] { k<<<grid_of(k, uf::FT, 0, items(MAP_MARCH0)), dim3(uf::FT), 0, s>>>(A); });
    vcycle(s, 1, cond, use_cond);
  }

  // a8, a9, the k / omega buffer swap
  void rec_post(cudaStream_t s) {
    launch_plane(kb_pressure_commit<T>, MAP_CELL, s, "b_pressure_commit", 10,
                 args<CommitP<T>>(MAP_CELL, [](CommitP<T>& P, const View<T>& G) {
                   P.sp = G.sp;
                   P.delta = G.p;
                   P.pn = G.pd;
                   P.gs = G.gd;
                   P.st = G.st;
                 }));
    launch_plane(kb_project<T>, MAP_FACE, s, "b_project", 8,
                 args<ProjP<T>>(MAP_FACE, [](ProjP<T>& P, const View<T>& G) {
                   P.sp = G.sp;
                   P.pr = G.pd;
                   P.u = G.u; P.v = G.v; P.w = G.w;
                 }));
    {
      auto k = kb_turbulence<T>;
      const auto& A = args<CellP<T>>(MAP_CELL, [](CellP<T>& P, const View<T>& G) { P = cell_params(G); });
      L(s, "b_turbulence", plane_bytes(MAP_CELL, 7),
        [&] { k<<<grid_of(k, uf::NT, 0, items(MAP_CELL)), dim3(uf::BX, uf::BY), 0, s>>>(A, d_par); });
    }
    L(s, "b_flip_parity", 0, [&] { kb_flip_parity<<<(n + 63) / 64, 64, 0, s>>>(d_par, n); });
  }

  uf_status capture() {
    if (exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    UFB_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    cudaStreamCaptureStatus cs;
    cudaGraph_t cgraph;
    cudaError_t e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cgraph, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle cond;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cgraph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      return bfail(UF_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    }
    rec = 0;
    rec_pre(cap, cond, 1);
    const int before_loop = rec;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cgraph, &deps, nullptr, &ndeps);
    if (e == cudaSuccess && cs != cudaStreamCaptureStatusActive) e = cudaGetLastError();   // a launch failed
    if (e == cudaSuccess && cs != cudaStreamCaptureStatusActive) e = cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cnode;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, cgraph, deps, nullptr, ndeps, &np);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        rec_iter(cap2, cond, 1);
        e = cudaStreamEndCapture(cap2, &body);
      }
    }
    const int in_loop = rec - before_loop;
    if (e == cudaSuccess) rec_post(cap);
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(UF_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    n_iter = in_loop;
    n_fixed = rec - in_loop;
    return UF_OK;
  }

  // One batched step launched eagerly with per-launch events; the host
  // polls the unfinished-instance counter before every CG iteration.
  uf_status profile_step(uf_kernel_time* out, int cap_n, int* count) override {
    for (int i = 0; i < n; ++i)
      if (!grids[i]->has_state()) return bfail(UF_ERR_STATE, "instance " + std::to_string(i) + " has no state");
    uf_status s = prepare();
    if (s != UF_OK) return s;
    recs.clear();
    pool_used = 0;
    profiling = true;
    rec_pre(stream, 0, 0);
    int max_it = 1;
    for (const View<T>& G : views) max_it = std::max(max_it, G.d.cg_max_iter);
    for (int it = 0; it <= max_it; ++it) {
      int left = 0;
      cudaError_t e = cudaMemcpyAsync(&left, d_left, sizeof(int), cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) {
        profiling = false;
        return bfail(UF_ERR_CUDA, std::string("profile: ") + cudaGetErrorString(e));
      }
      if (left <= 0) break;
      rec_iter(stream, 0, 0);
    }
    rec_post(stream);
    profiling = false;
    UFB_CUDA(cudaStreamSynchronize(stream));
    UFB_CUDA(cudaGetLastError());
    for (int i = 0; i < n; ++i) grids[i]->advanced(1);
    std::vector<uf_kernel_time> agg;
    for (const Rec& r : recs) {
      float ms = 0;
      UFB_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
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
    uf_status first = UF_OK;
    for (int i = 0; i < n; ++i) {
      const uf_status si = grids[i]->read_status(nullptr);
      if (si != UF_OK && first == UF_OK) first = si;
    }
    return first;
  }

  static bool same_launches(const View<T>& a, const View<T>& b) {
    View<T> x = a, y = b;
    x.parity = y.parity = 0;
    return std::memcmp(&x, &y, sizeof(View<T>)) == 0;
  }

  // Refreshes the device views (parity changes between runs) and re-captures
  // the graph when an instance's buffers or tuning changed.
  uf_status prepare() {
    bool rebuild = !exec || built_for.size() != (size_t)n;
    for (int i = 0; i < n; ++i) {
      grids[i]->fill_view(&views[i]);
      if (!rebuild && !same_launches(views[i], built_for[i])) rebuild = true;
    }
    UFB_CUDA(cudaMemcpyAsync(d_views, views.data(), sizeof(View<T>) * n, cudaMemcpyHostToDevice, stream));
    par_host.resize(n);
    for (int i = 0; i < n; ++i) par_host[i] = views[i].parity;
    UFB_CUDA(cudaMemcpyAsync(d_par, par_host.data(), sizeof(int) * n, cudaMemcpyHostToDevice, stream));
    if (rebuild) {
      build_maps();
      UFB_CUDA(cudaMemcpyAsync(d_maps, maps.data(), sizeof(LaunchMap) * kMaps, cudaMemcpyHostToDevice, stream));
      int dev = 0, optin = 0;
      UFB_CUDA(cudaGetDevice(&dev));
      UFB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      auto lim = [&](const void* f) {   // per kernel, shared by all batches: the device maximum
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      };
      UFB_CUDA(lim((const void*)kb_mg_tail<T, uf::SM_JACOBI>));
      UFB_CUDA(lim((const void*)kb_mg_tail<T, uf::SM_RBGS>));
      auto lim_static = [&](const void* f) {   // less the kernel's static shared memory
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        return e;
      };
      UFB_CUDA(lim_static((const void*)kb_advect_fused<T>));
      UFB_CUDA(lim_static((const void*)kb_momentum_fused<T>));
      UFB_CUDA(cudaStreamSynchronize(stream));
      uf_status s = capture();
      if (s != UF_OK) return s;
      built_for = views;
    }
    UFB_CUDA(cudaStreamSynchronize(stream));   // the host copies may change
    return UF_OK;
  }

  uf_status after_call(uf_status s) override {
#ifdef UF_BOUNDS_CHECK
    uf::BoundsHit h;
    if (uf::bounds_hit_take(stream, &h)) return bfail(UF_ERR_BOUNDS, bounds_text(h));
#endif
    return s;
  }

  uf_status run(int nsteps, uf_step_stats* stats) override {
    if (nsteps < 0) return bfail(UF_ERR_ARG, "nsteps < 0");
    for (int i = 0; i < n; ++i)
      if (!grids[i]->has_state())
        return bfail(UF_ERR_STATE, "instance " + std::to_string(i) + " has no state (uf_init_state or uf_set_state)");
    uf_status s = prepare();
    if (s != UF_OK) return s;
    for (int k = 0; k < nsteps; ++k) UFB_CUDA(cudaGraphLaunch(exec, stream));
    UFB_CUDA(cudaGetLastError());
    for (int i = 0; i < n; ++i) grids[i]->advanced(nsteps);
    if (!stats) return UF_OK;
    uf_status first = UF_OK;
    for (int i = 0; i < n; ++i) {
      const uf_status si = grids[i]->read_status(&stats[i]);
      if (si != UF_OK && first == UF_OK) first = si;
    }
    return first;
  }

  uf_status launch_counts(int* fixed, int* per_iter) override {
    for (int i = 0; i < n; ++i) grids[i]->fill_view(&views[i]);
    if (!exec) {
      uf_status s = prepare();
      if (s != UF_OK) return s;
    }
    if (fixed) *fixed = n_fixed;
    if (per_iter) *per_iter = n_iter;
    return UF_OK;
  }

  // Size class: the number of multigrid levels and the cell count in
  // half-octaves (grids within a factor sqrt(2) of each other share one).
  static std::vector<int> size_class(const View<T>& G) {
    return {G.nl, (int)std::floor(2.0 * std::log2(cells(G, 0)))};
  }

  uf_status autotune(int reps, int* classes) override {
    std::vector<std::vector<int>> keys;
    std::vector<uf_tuning> chosen;
    for (int i = 0; i < n; ++i) {
      grids[i]->fill_view(&views[i]);
      const std::vector<int> key = size_class(views[i]);
      auto it = std::find(keys.begin(), keys.end(), key);
      if (it == keys.end()) {
        uf_tuning t;
        uf_status s = grids[i]->autotune(reps, &t, nullptr);
        if (s != UF_OK) return s;
        keys.push_back(key);
        chosen.push_back(t);
      } else {
        uf_status s = grids[i]->set_tuning(&chosen[it - keys.begin()]);
        if (s != UF_OK) return s;
      }
    }
    if (classes) *classes = (int)keys.size();
    if (exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    return UF_OK;
  }
};

bool batch_descs_valid(int n, const uf_grid_desc* descs, std::string* why) {
  if (n < 1 || n > kMaxBatch) { *why = "batch size must lie in [1, 64]"; return false; }
  if (!descs) { *why = "NULL descriptions"; return false; }
  for (int i = 0; i < n; ++i) {
    if (uf_workspace_bytes(&descs[i]) == 0) { *why = "instance " + std::to_string(i) + ": " + uf_last_error(); return false; }
    if (descs[i].precision != descs[0].precision) { *why = "instances must share the precision"; return false; }
    if (descs[i].precond != UF_PRECOND_MG) { *why = "batched instances use the MG preconditioner"; return false; }
    if (descs[i].mg_smoother != descs[0].mg_smoother) { *why = "instances must share the smoother"; return false; }
  }
  return true;
}

size_t batch_bytes(int n, const uf_grid_desc* descs) {
  size_t b = 0;
  for (int i = 0; i < n; ++i) b += round256(uf_workspace_bytes(&descs[i]));
  const TableLayout TL = descs[0].precision == UF_F64 ? table_layout<double>(n) : table_layout<float>(n);
  return b + TL.total + 256;
}

}  // namespace

extern "C" {

size_t uf_batch_workspace_bytes(int n, const uf_grid_desc* descs) {
  std::string why;
  if (!batch_descs_valid(n, descs, &why)) {
    uf_internal_set_last_error(why.c_str());
    return 0;
  }
  return batch_bytes(n, descs);
}

uf_status uf_batch_create(int n, const uf_grid_desc* descs, void* d_workspace, size_t bytes, void* cuda_stream,
                          uf_batch** out) {
  if (!out) return bfail(UF_ERR_ARG, "NULL output");
  *out = nullptr;
  std::string why;
  if (!batch_descs_valid(n, descs, &why)) return bfail(UF_ERR_ARG, why);
  if (!d_workspace) return bfail(UF_ERR_ARG, "NULL workspace");
  if (bytes < batch_bytes(n, descs)) return bfail(UF_ERR_NOMEM, "workspace smaller than uf_batch_workspace_bytes()");
  char* ws = reinterpret_cast<char*>(round256(reinterpret_cast<size_t>(d_workspace)));
  const size_t usable = bytes - (size_t)(ws - reinterpret_cast<char*>(d_workspace));
  uf_batch* b = nullptr;
  uf_status s;
  if (descs[0].precision == UF_F64) {
    auto* impl = new BatchImpl<double>();
    s = impl->setup(n, descs, ws, usable, (cudaStream_t)cuda_stream);
    b = impl;
  } else {
    auto* impl = new BatchImpl<float>();
    s = impl->setup(n, descs, ws, usable, (cudaStream_t)cuda_stream);
    b = impl;
  }
  if (s != UF_OK) {
    delete b;
    return s;
  }
  *out = b;
  return UF_OK;
}

uf_status uf_batch_grid(uf_batch* b, int i, uf_grid** out) {
  if (!b) return bfail(UF_ERR_ARG, "NULL batch");
  return b->grid(i, out);
}

uf_status uf_batch_run(uf_batch* b, int nsteps, uf_step_stats* stats) {
  if (!b) return bfail(UF_ERR_ARG, "NULL batch");
  NvtxRange range("uf_batch_run");
  return b->after_call(b->run(nsteps, stats));
}

uf_status uf_batch_launch_counts(uf_batch* b, int* fixed, int* per_iter) {
  if (!b) return bfail(UF_ERR_ARG, "NULL batch");
  return b->launch_counts(fixed, per_iter);
}

uf_status uf_batch_autotune(uf_batch* b, int reps, int* classes) {
  if (!b) return bfail(UF_ERR_ARG, "NULL batch");
  if (reps < 1) return bfail(UF_ERR_ARG, "reps >= 1 required");
  NvtxRange range("uf_batch_autotune");
  return b->after_call(b->autotune(reps, classes));
}

uf_status uf_batch_profile_step(uf_batch* b, uf_kernel_time* out, int capacity, int* count) {
  if (!b) return bfail(UF_ERR_ARG, "NULL batch");
  if (capacity < 0) return bfail(UF_ERR_ARG, "negative capacity");
  NvtxRange range("uf_batch_profile_step");
  return b->after_call(b->profile_step(out, capacity, count));
}

uf_status uf_batch_destroy(uf_batch* b) {
  delete b;
  return UF_OK;
}

}  // extern "C"
