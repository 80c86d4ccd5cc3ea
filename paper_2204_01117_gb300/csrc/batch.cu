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
#include <cstring>
#include <string>
#include <vector>

#include "../../include/uf.h"
#include "grid_base.cuh"

// Sets the thread-local message returned by uf_last_error() (capi.cu).
void uf_internal_set_last_error(const char* msg);

struct uf_batch {
  virtual ~uf_batch() {}
  virtual uf_status grid(int, uf_grid**) = 0;
  virtual uf_status run(int, uf_step_stats*) = 0;
  virtual uf_status launch_counts(int*, int*) = 0;
  virtual uf_status autotune(int, int*) = 0;
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
};

// Launch kinds: one work list each (march levels: one per level).
enum MapKind { MAP_CFL = 0, MAP_CELL, MAP_FACE, MAP_CHUNK, MAP_TAIL, MAP_MARCH0 };
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

// Persistent loop: block b takes items b, b + gridDim.x, ...; f(instance,
// z chunk, block coordinates) runs the kernel body on one item.
template <typename F>
__device__ __forceinline__ void for_items(const LaunchMap* __restrict__ m, F&& f) {
  const int total = m->total;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int e = map_entry(m, w);
    const int lin = w - m->start[e], gx = m->gx[e], gy = m->gy[e];
    const VBlock vb{lin % gx, (lin / gx) % gy, lin / (gx * gy), lin, m->start[e + 1] - m->start[e]};
    f(m->inst[e], m->zc[e], vb);
    __syncthreads();   // the next item reuses the shared memory
  }
}

template <typename T>
using View = GridView<T>;

template <typename T>
__global__ void __launch_bounds__(256) kb_cfl(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::cfl_dt_body<T>(G.u, G.n_u, G.v, G.n_v, G.w, G.n_w, G.d.cfl * G.d.h, G.partials, &G.st->ticket[0], G.dt,
                       G.dtT, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_eddy(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::eddy_viscosity_body<T>(G.sp, G.u, G.v, G.w, G.kb[G.parity], G.ob[G.parity], G.nut, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_advect_forward(const View<T>* __restrict__ V,
                                                            const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) { uf::advect_forward_body<T>(V[i].adv, vb); });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_advect_backward(const View<T>* __restrict__ V,
                                                             const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) { uf::advect_backward_body<T>(V[i].adv, vb); });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_diffuse(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::diffuse_body<T>(G.sp, G.ut, G.vt, G.wt, G.nut, G.u2, G.v2, G.w2, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_drag_bc(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::drag_bc_body<T>(G.sp, G.u2, G.v2, G.w2, G.cc, G.u, G.v, G.w, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_pressure_rhs(const View<T>* __restrict__ V,
                                                          const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int zc, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::pressure_rhs_body<T>(G.sp, G.u, G.v, G.w, G.b, zc, G.partials, G.st, vb);
  });
}

// Opens the batch's CG loop: every instance that takes part is unfinished.
__global__ void kb_begin_solve(int* left, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *left = n;
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_cg_init(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m,
                                                     cudaGraphConditionalHandle cond, int* left) {
  for_items(m, [&](int i, int zc, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::cg_init_body<T>(G.lv[0], G.b, G.p, zc, G.partials, G.st, cond, 1, left, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::FT) kb_cg_dir_q(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int zc, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::cg_dir_q_body<T>(G.lv[0], zc, G.z, G.d0, G.d1, G.q, G.partials, G.st, vb);
  });
}

template <typename T, int SM, bool CG>
__global__ void __launch_bounds__(uf::FT) kb_mg_down(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m,
                                                     int l, cudaGraphConditionalHandle cond, int* left) {
  for_items(m, [&](int i, int zc, const VBlock& vb) {
    const View<T>& G = V[i];
    if (CG)
      uf::mg_down_body<T, SM, true>(G.lv[0], G.lv[1], G.omega, zc, G.p, G.d0, G.d1, G.q, G.partials, G.st, cond, 1,
                                     left, vb);
    else
      uf::mg_down_body<T, SM, false>(G.lv[l], G.lv[l + 1], G.omega, zc, nullptr, nullptr, nullptr, nullptr,
                                      G.partials, G.st, cond, 0, nullptr, vb);
  });
}

template <typename T, int SM>
__global__ void __launch_bounds__(uf::TAIL_T) kb_mg_tail(const View<T>* __restrict__ V,
                                                         const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::mg_tail_body<T, SM>(G.tail, G.omega, G.st, vb);
  });
}

template <typename T, int SM, bool FINEST>
__global__ void __launch_bounds__(uf::FT) kb_mg_up(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m,
                                                   int l, int mode) {
  for_items(m, [&](int i, int zc, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::mg_up_body<T, SM, FINEST>(G.lv[l], G.lv[l + 1], G.omega, zc, FINEST ? G.z : G.lv[l].t, mode, G.partials,
                                  G.st, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_project(const View<T>* __restrict__ V, const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    uf::project_body<T>(G.sp, G.p, G.u, G.v, G.w, vb);
  });
}

template <typename T>
__global__ void __launch_bounds__(uf::NT) kb_turbulence(const View<T>* __restrict__ V,
                                                        const LaunchMap* __restrict__ m) {
  for_items(m, [&](int i, int, const VBlock& vb) {
    const View<T>& G = V[i];
    const int a = G.parity, o = a ^ 1;
    uf::turbulence_body<T>(G.sp, G.u, G.v, G.w, G.kb[a], G.ob[a], G.kb[o], G.ob[o], vb);
  });
}

// End of a step: every instance's k and omega now live in the other buffer.
template <typename T>
__global__ void kb_flip_parity(View<T>* V, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) V[i].parity ^= 1;
}

// Device-side tables of a batch: the views, the work lists, the loop counter.
struct TableLayout {
  size_t views, maps, left, total;
};
template <typename T>
TableLayout table_layout(int n) {
  TableLayout L;
  L.views = 0;
  L.maps = round256(sizeof(View<T>) * n);
  L.left = L.maps + round256(sizeof(LaunchMap) * kMaps);
  L.total = L.left + 256;
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
  std::vector<View<T>> views;          // host copies (parity included)
  std::vector<LaunchMap> maps;
  std::vector<View<T>> built_for;      // views the graph was captured for
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
      add_entry(maps[MAP_CELL], i, (d.nx + uf::BX - 1) / uf::BX, (d.ny + uf::BY - 1) / uf::BY, d.nz, 0);
      add_entry(maps[MAP_FACE], i, (d.nx + 1 + uf::BX - 1) / uf::BX, (d.ny + 1 + uf::BY - 1) / uf::BY, 3 * d.nz + 1,
                0);
      add_entry(maps[MAP_CHUNK], i, G.chunk_g[0], G.chunk_g[1], G.chunk_g[2], G.chunk_zc);
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

  // --------------------------------------------------------------- capture
  int rec = 0;

  template <int SM>
  void rec_vcycle(cudaStream_t s, int mode, cudaGraphConditionalHandle cond) {
    const dim3 ft(uf::FT);
    for (int l = 0; l < max_levels; ++l) {
      const int kind = MAP_MARCH0 + l;
      if (l == 0 && mode == 1) {
        auto k = kb_mg_down<T, SM, true>;
        k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(d_views, dm(kind), 0, cond, d_left);
      } else {
        auto k = kb_mg_down<T, SM, false>;
        k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(d_views, dm(kind), l, cond, nullptr);
      }
      rec++;
    }
    {
      auto k = kb_mg_tail<T, SM>;
      k<<<grid_of(k, uf::TAIL_T, tail_smem, items(MAP_TAIL)), uf::TAIL_T, tail_smem, s>>>(d_views, dm(MAP_TAIL));
      rec++;
    }
    for (int l = max_levels - 1; l >= 0; --l) {
      const int kind = MAP_MARCH0 + l;
      if (l == 0) {
        auto k = kb_mg_up<T, SM, true>;
        k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(d_views, dm(kind), 0, mode);
      } else {
        auto k = kb_mg_up<T, SM, false>;
        k<<<grid_of(k, uf::FT, 0, items(kind)), ft, 0, s>>>(d_views, dm(kind), l, mode);
      }
      rec++;
    }
  }

  void vcycle(cudaStream_t s, int mode, cudaGraphConditionalHandle cond) {
    if (smoother == UF_SMOOTH_JACOBI) rec_vcycle<uf::SM_JACOBI>(s, mode, cond);
    else rec_vcycle<uf::SM_RBGS>(s, mode, cond);
  }

  template <typename K>
  void launch_items(K kernel, int kind, int threads, cudaStream_t s, dim3 blk) {
    if (items(kind) == 0) return;
    kernel<<<grid_of(kernel, threads, 0, items(kind)), blk, 0, s>>>(d_views, dm(kind));
    rec++;
  }

  uf_status capture() {
    if (exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    const dim3 blk(uf::BX, uf::BY);
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
    // a0-a6
    launch_items(kb_cfl<T>, MAP_CFL, 256, cap, dim3(256));
    launch_items(kb_eddy<T>, MAP_CELL, uf::NT, cap, blk);
    launch_items(kb_advect_forward<T>, MAP_FACE, uf::NT, cap, blk);
    launch_items(kb_advect_backward<T>, MAP_FACE, uf::NT, cap, blk);
    launch_items(kb_diffuse<T>, MAP_FACE, uf::NT, cap, blk);
    launch_items(kb_drag_bc<T>, MAP_FACE, uf::NT, cap, blk);
    launch_items(kb_pressure_rhs<T>, MAP_CHUNK, uf::NT, cap, blk);
    // a7: CG set-up, then the loop
    kb_begin_solve<<<1, 32, 0, cap>>>(d_left, n);
    rec++;
    {
      auto k = kb_cg_init<T>;
      k<<<grid_of(k, uf::NT, 0, items(MAP_CHUNK)), blk, 0, cap>>>(d_views, dm(MAP_CHUNK), cond, d_left);
      rec++;
    }
    vcycle(cap, 0, cond);
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
        auto k = kb_cg_dir_q<T>;
        k<<<grid_of(k, uf::FT, 0, items(MAP_MARCH0)), dim3(uf::FT), 0, cap2>>>(d_views, dm(MAP_MARCH0));
        rec++;
        vcycle(cap2, 1, cond);
        e = cudaStreamEndCapture(cap2, &body);
      }
    }
    const int in_loop = rec - before_loop;
    // a8, a9, parity
    if (e == cudaSuccess) {
      launch_items(kb_project<T>, MAP_FACE, uf::NT, cap, blk);
      launch_items(kb_turbulence<T>, MAP_CELL, uf::NT, cap, blk);
      kb_flip_parity<T><<<(n + 63) / 64, 64, 0, cap>>>(d_views, n);
      rec++;
    }
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(UF_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    n_iter = in_loop;
    n_fixed = rec - in_loop;
    return UF_OK;
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
      UFB_CUDA(cudaStreamSynchronize(stream));
      uf_status s = capture();
      if (s != UF_OK) return s;
      built_for = views;
    }
    UFB_CUDA(cudaStreamSynchronize(stream));   // the host copies may change
    return UF_OK;
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

  // Size class: the shape of the multigrid hierarchy (level extents).
  static std::vector<int> size_class(const View<T>& G) {
    std::vector<int> k;
    for (int l = 0; l < G.nl; ++l) {
      k.push_back(G.lv[l].nx);
      k.push_back(G.lv[l].ny);
      k.push_back(G.lv[l].nz);
    }
    return k;
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
  return b->run(nsteps, stats);
}

uf_status uf_batch_launch_counts(uf_batch* b, int* fixed, int* per_iter) {
  if (!b) return bfail(UF_ERR_ARG, "NULL batch");
  return b->launch_counts(fixed, per_iter);
}

uf_status uf_batch_autotune(uf_batch* b, int reps, int* classes) {
  if (!b) return bfail(UF_ERR_ARG, "NULL batch");
  if (reps < 1) return bfail(UF_ERR_ARG, "reps >= 1 required");
  return b->autotune(reps, classes);
}

uf_status uf_batch_destroy(uf_batch* b) {
  delete b;
  return UF_OK;
}

}  // extern "C"
