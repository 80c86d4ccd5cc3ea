// Device-side building blocks of the UrbanFlow RANS step (sm_103a).
//
// Grid: uniform staggered MAC grid (Sec. 3, "Discretization and Numerical
// Integration"): u on x-faces, v on y-faces, w on z-faces, p / k / omega /
// porosity at cell centres.  Every lattice is stored x-fastest with its row
// pitch rounded up to 32 elements so that rows start on 128-byte
// boundaries; padding is zero and never written.
//
// Boundary conditions (Sec. 3, "Porosity Model vs. Solid-wall Boundary
// Conditions") are evaluated on the fly by the consumers of a field instead of
// being materialised by separate passes:
//   * normal component on a boundary face: inlet -> inflow profile, outlet ->
//     value of the adjacent interior face (zero normal derivative), slip or
//     no-slip wall -> 0;
//   * tangential ghost beyond a side: inlet -> inflow value, outlet / slip ->
//     mirror of the interior value, no-slip -> its negative.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace uf {

enum SideType { INFLOW = 0, OUTFLOW = 1, SLIP = 2, NOSLIP = 3 };

// Solver state word written by kernels (first error wins).
enum DevStatus { DEV_OK = 0, DEV_NOT_CONVERGED = 4, DEV_NAN = 5 };

template <typename T>
struct StepParams {
  int nx, ny, nz;
  int Pu;     // row pitch of the u lattice (nx+1 rounded up)
  int Pc;     // row pitch of the v, w and cell lattices (nx rounded up)
  int side[6];   // x-, x+, y-, y+, z-, z+
  T h, inv_h;
  T dirx, diry;            // horizontal wind direction (cos, sin)
  T rho, nu;
  T C_mu, alpha, beta, sigma, sigma_star, C_lim;
  T k_min, om_min, k_in, om_in;
  const T* prof;           // inflow speed at the nz cell-centre heights
  const double* dt;        // device scalar: the step's time step (FP64)
  const T* dtT;            // the same time step in the field type (read per cell)
};

// Arithmetic with every operation rounded as written (the compiler fuses no
// multiply into an add on its own): expressions that two kernels must form
// alike, bit for bit, are spelled with these.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ------------------------------------------------------- bounds checks --
// Debug build (compiled with -DUF_BOUNDS_CHECK): every global index the
// index helpers form (idx_u, idx_v, idx_c here, lidx for the multigrid
// levels) is checked against its array: x within the row pitch, y and z
// within the stored rows and planes.  The first violation is recorded in
// uf_bounds_hit (array, i, j, k) and the access is redirected to element 0,
// so the kernel completes; the host reads the record after the call and
// returns UF_ERR_BOUNDS.  Each translation unit has its own record, read by
// its own host code.  The ordinary build compiles none of this.
enum BoundsArray { BA_U = 0, BA_V = 1, BA_CW = 2, BA_LEVEL = 3 };
struct BoundsHit {
  int hit, array, i, j, k;
};
#ifdef UF_BOUNDS_CHECK
static __device__ BoundsHit uf_bounds_hit;
__device__ __forceinline__ void bounds_check(bool ok, int array, int& i, int& j, int& k) {
  if (ok) return;
  if (atomicExch(&uf_bounds_hit.hit, 1) == 0) {
    uf_bounds_hit.array = array;
    uf_bounds_hit.i = i;
    uf_bounds_hit.j = j;
    uf_bounds_hit.k = k;
  }
  i = j = k = 0;
}
// Reads (and clears) this translation unit's record after the work queued
// on stream s; true if an index was out of bounds.
static inline bool bounds_hit_take(cudaStream_t s, BoundsHit* out) {
  const BoundsHit clear = {0, 0, 0, 0, 0};
  if (cudaMemcpyFromSymbolAsync(out, uf_bounds_hit, sizeof(*out), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return false;   // (the CUDA error surfaces in the caller's next check)
  if (!out->hit) return false;
  cudaMemcpyToSymbolAsync(uf_bounds_hit, &clear, sizeof(clear), 0, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  return true;
}
#define UF_BOUNDS(ok, array, i, j, k) ::uf::bounds_check((ok), (array), i, j, k)
#else
#define UF_BOUNDS(ok, array, i, j, k) ((void)0)
#endif

// ------------------------------------------------------------- indexing --
template <typename T>
__device__ __forceinline__ size_t idx_u(const StepParams<T>& p, int i, int j, int k) {
  UF_BOUNDS(i >= 0 && i < p.Pu && j >= 0 && j < p.ny && k >= 0 && k < p.nz, BA_U, i, j, k);
  return (size_t)i + (size_t)p.Pu * ((size_t)j + (size_t)p.ny * k);
}
template <typename T>
__device__ __forceinline__ size_t idx_v(const StepParams<T>& p, int i, int j, int k) {
  UF_BOUNDS(i >= 0 && i < p.Pc && j >= 0 && j <= p.ny && k >= 0 && k < p.nz, BA_V, i, j, k);
  return (size_t)i + (size_t)p.Pc * ((size_t)j + (size_t)(p.ny + 1) * k);
}
template <typename T>   // w lattice and cell lattice share the x-y layout
__device__ __forceinline__ size_t idx_c(const StepParams<T>& p, int i, int j, int k) {
  // (z up to nz: the w lattice's top face; a cell array has nz planes, which
  // this shared helper cannot tell apart)
  UF_BOUNDS(i >= 0 && i < p.Pc && j >= 0 && j < p.ny && k >= 0 && k <= p.nz, BA_CW, i, j, k);
  return (size_t)i + (size_t)p.Pc * ((size_t)j + (size_t)p.ny * k);
}

// ------------------------------------------------------ boundary values --
template <typename T>
__device__ __forceinline__ T normal_face(int side, T adjacent, T inflow) {
  return side == INFLOW ? inflow : (side == OUTFLOW ? adjacent : T(0));
}
template <typename T>
__device__ __forceinline__ T tangential_ghost(int side, T q, T inflow) {
  return side == INFLOW ? inflow : (side == NOSLIP ? -q : q);
}

// Face values with the BC applied on boundary faces (the stored value there
// is never read).
template <typename T>
__device__ __forceinline__ T u_face(const T* __restrict__ u, const StepParams<T>& p, int i, int j, int k) {
  if (i == 0) return normal_face(p.side[0], u[idx_u(p, 1, j, k)], p.prof[k] * p.dirx);
  if (i == p.nx) return normal_face(p.side[1], u[idx_u(p, p.nx - 1, j, k)], p.prof[k] * p.dirx);
  return u[idx_u(p, i, j, k)];
}
template <typename T>
__device__ __forceinline__ T v_face(const T* __restrict__ v, const StepParams<T>& p, int i, int j, int k) {
  if (j == 0) return normal_face(p.side[2], v[idx_v(p, i, 1, k)], p.prof[k] * p.diry);
  if (j == p.ny) return normal_face(p.side[3], v[idx_v(p, i, p.ny - 1, k)], p.prof[k] * p.diry);
  return v[idx_v(p, i, j, k)];
}
template <typename T>
__device__ __forceinline__ T w_face(const T* __restrict__ w, const StepParams<T>& p, int i, int j, int k) {
  if (k == 0 || k == p.nz) return T(0);
  return w[idx_c(p, i, j, k)];
}

// ----------------------------------------------------- dot accumulation --
// Per-thread accumulator of sums of products.  For FP32 fields it is the
// compensated "Dot2" scheme of Ogita, Rump and Oishi (SIAM J. Sci. Comput.
// 26(6), 2005): every product is split exactly into p + e with an FMA, the
// running sum is kept as an unevaluated pair (hi, lo) with Knuth's TwoSum,
// so the result is as accurate as a sum accumulated in twice the working
// precision -- while every operation stays on the FP32 pipes (GB300 issues
// FP64 at 1/64 of the FP32 rate).  The pair is converted to FP64 once per
// thread; block and grid sums are FP64.  For FP64 fields it is a plain
// double sum.
template <typename T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s = fma((double)a, (double)b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);   // a*b = p + pe exactly
    const float t = hi + p;            // TwoSum(hi, p) = t + te exactly
    const float bv = t - hi;
    const float te = (hi - (t - bv)) + (p - bv);
    hi = t;
    lo += te + pe;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ------------------------------------------------------ pressure store --
// The pressure state is stored as an unevaluated pair (hi, lo) of FP32
// values for FP32 grids -- twice the working precision, with every
// operation on the FP32 pipes -- and as a double for FP64 grids.  It grows
// upstream of the outlet to many times the neighbour differences the
// projection uses; a single FP32 value would carry an absolute error of
// eps |p| into every face.  Only differences of neighbouring pressures and
// the commit of a new pressure read it; a difference of two pairs,
// (hi1 - hi2) + (lo1 - lo2), is rounded relative to the difference itself.
template <typename T>
struct PStoreOf { using type = double; };
template <>
struct PStoreOf<float> { using type = float2; };
template <typename T>
using PStore = typename PStoreOf<T>::type;

// Knuth's TwoSum: s + e == a + b exactly in round-to-nearest.  The _rn
// intrinsics keep the compiler from contracting or reordering the steps.
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  return make_float2(s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv)));
}
// Sum of two pairs, renormalised: the accurate double-word addition
// (Dekker 1971; Joldes, Muller and Popescu 2017, Algorithm 6), with TwoSum
// in place of Fast2Sum so that no ordering of magnitudes is assumed.
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  const float2 t = two_sum(a.y, b.y);
  s = two_sum(s.x, __fadd_rn(s.y, t.x));
  return two_sum(s.x, __fadd_rn(s.y, t.y));
}
__device__ __forceinline__ float ps_diff(float2 a, float2 b) {
  return __fadd_rn(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}
__device__ __forceinline__ double ps_diff(double a, double b) { return a - b; }
__device__ __forceinline__ float ps_value(float2 a) { return __fadd_rn(a.x, a.y); }
__device__ __forceinline__ double ps_value(double a) { return a; }
__device__ __forceinline__ float2 ps_from(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ double ps_from(double v) { return v; }
// p^{n+1} = g + delta (zero: p = 0) and the next solve's guess 2 p^{n+1} - p^n.
__device__ __forceinline__ void ps_commit(float2 g, float2 pn, float delta, bool zero, float2* pnew, float2* gnew) {
  const float2 v = zero ? make_float2(0.f, 0.f) : pair_add(g, make_float2(delta, 0.f));
  *pnew = v;
  *gnew = pair_add(make_float2(2.f * v.x, 2.f * v.y), make_float2(-pn.x, -pn.y));
}
__device__ __forceinline__ void ps_commit(double g, double pn, double delta, bool zero, double* pnew, double* gnew) {
  const double v = zero ? 0.0 : g + delta;
  *pnew = v;
  *gnew = 2.0 * v - pn;
}

// ------------------------------------------------------------- reduction --
// Deterministic block + grid reduction in FP64: every block writes one
// partial; the last block to finish (atomic ticket) sums the partials in a
// fixed order and runs `finish(total)` on thread 0.  The ticket is reset by
// the last block, so the kernel can be replayed.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = (lane < NT / 32) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid on thread 0 of the block
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = (lane < NT / 32) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  }
  return t;
}

__device__ __forceinline__ int block_linear_id() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ int grid_blocks() { return gridDim.x * gridDim.y * gridDim.z; }
__device__ __forceinline__ int thread_linear_id() { return threadIdx.x + blockDim.x * threadIdx.y; }

// Coordinates of the block of work a kernel body processes: the launch's own
// block (vblock()) for a single grid, or one item of a batch work list.
// lin / n: linear index and count of the blocks that reduce into the same
// partials buffer (one grid, or one instance of a batch).
struct VBlock {
  int x, y, z;
  int lin, n;
};
__device__ __forceinline__ VBlock vblock() {
  return VBlock{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, block_linear_id(), grid_blocks()};
}

// Publishes this block's partial(s) and returns true in the last of the vb.n
// blocks that share the partials buffer and the ticket.
template <int NV>
__device__ __forceinline__ bool publish_partials(double* partials, unsigned int* ticket, const double* vals,
                                                 bool* sh_last, const VBlock& vb) {
  if (thread_linear_id() == 0) {
    const int b = vb.lin, nb = vb.n;
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[q * nb + b] = vals[q];
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    *sh_last = (t == (unsigned)nb - 1);
  }
  __syncthreads();
  return *sh_last;
}
template <int NV>
__device__ __forceinline__ bool publish_partials(double* partials, unsigned int* ticket, const double* vals,
                                                 bool* sh_last) {
  return publish_partials<NV>(partials, ticket, vals, sh_last, vblock());
}

// In the last block: sum partials[q*nb ..] for q < NV in a fixed order.
template <int NT, int NV>
__device__ __forceinline__ void reduce_partials_sum(const double* partials, double* out, double* sh, int nb) {
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
    for (int b = thread_linear_id(); b < nb; b += NT) s += __ldcg(partials + q * nb + b);
    s = block_sum<NT>(s, sh);
    if (thread_linear_id() == 0) out[q] = s;
  }
}
template <int NT, int NV>
__device__ __forceinline__ void reduce_partials_sum(const double* partials, double* out, double* sh) {
  reduce_partials_sum<NT, NV>(partials, out, sh, grid_blocks());
}
template <int NT>
__device__ __forceinline__ double reduce_partials_max(const double* partials, double* sh, int nb) {
  double s = 0.0;
  for (int b = thread_linear_id(); b < nb; b += NT) s = fmax(s, __ldcg(partials + b));
  return block_max<NT>(s, sh);
}

}  // namespace uf
