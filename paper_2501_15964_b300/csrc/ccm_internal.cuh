// Internal declarations shared by the libccm translation units.
//
// Layout used by every solver kernel: node rows (A, X, gradient, CG vectors)
// and edge rows (multipliers U, projected y, yhat) are stored with a padded
// leading dimension ld = round_up(d, 4); padding elements are zero and stay
// zero under every operation. A "quad" is 4 consecutive elements of a row; a
// group of LANES threads owns one row, lane t holding quads t, t+LANES, ...
// (CH quads per lane), so one float4 (float32 rows) or two double2 (float64
// rows) move a quad, and consecutive lanes touch consecutive 16/32-byte
// pieces of the row (coalesced).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ccm.h"

namespace ccm {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CCM_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t _e = (call);                                             \
    if (_e != cudaSuccess) return ::ccm::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define CCM_TRY(...)                  \
  do {                                \
    int _s = (__VA_ARGS__);           \
    if (_s != CCM_OK) return _s;      \
  } while (0)

// ---------------------------------------------------------------- context
enum Slot : int {
  S_AP, S_X0, S_X1, S_G, S_DX, S_R, S_P0, S_P1, S_Q, S_MINV,
  S_U, S_UT, S_YH, S_ALPHA, S_KIND, S_EDGES, S_CSR_OFF, S_CSR_INC, S_PART, S_CTRL,
  S_SCRATCH0, S_SCRATCH1, S_SCRATCH2, S_SCRATCH3, S_SCRATCH4, S_SCRATCH5,
  S_SCRATCH6, S_SCRATCH7, S_BATCH0, S_BATCH1, S_BATCH2, S_BATCH3, S_META, S_WPART, S_VJPF, S_ADMM,
  S_XF0, S_XF1, S_KNN, S_REORD, S_ORDER, S_ORDER_TMP, S_CO_PARENT, S_CO_AGG, S_CO_A, S_CO_AINV,
  S_CO_YZ, S_CO_U, S_CO_ONES, S_XSTAGE, S_LSTAGE, S_COUNT
};

// Autotuned group shape of the block engine for one (d, precision, degree bucket).
struct BlockTune {
  int d, tc, bucket, L, CH;
};

struct Ctx {
  int device = 0;
  int num_sms = 148;
  size_t l2_bytes = 0;
  void* slot_ptr[S_COUNT] = {};
  size_t slot_size[S_COUNT] = {};
  void* host_pinned = nullptr;   // small pinned buffer for scalar read-back
  cudaStream_t copy_stream = nullptr;  // device-to-host output copies (created at first use)
  cudaEvent_t copy_event = nullptr;
  size_t host_pinned_size = 0;
  std::vector<cudaEvent_t> ev_pool;
  ccm_profile last_profile = {};
  ccm_graph_info last_graph = {};
  int64_t launches = 0;          // kernels launched by this context (all calls)
  // dynamic shared-memory limit already raised per kernel, keyed by the kernel's
  // host address as seen by the launching translation unit (each .cu file holds
  // its own instance of a template kernel, so one kernel name can have several)
  std::vector<std::pair<const void*, size_t>> smem_attr;
  std::vector<BlockTune> block_tune;  // block-engine shapes measured on this context
  // blocks resident on the whole GPU per kernel (occupancy x SMs), keyed like smem_attr
  std::vector<std::pair<const void*, int>> resident;
};

// Blocks of `threads` threads (no dynamic shared memory) that kernel fn can keep
// resident on every SM at once, times the SM count: a grid-stride kernel
// launched with at most this many blocks runs in one wave.
template <typename F>
inline int resident_grid(Ctx* c, F fn, int threads) {
  const void* key = (const void*)fn;
  for (auto& e : c->resident)
    if (e.first == key) return e.second;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0) != cudaSuccess)
    per = 1;
  per = per < 1 ? 1 : (per > 8 ? 8 : per);
  c->resident.emplace_back(key, per * c->num_sms);
  return per * c->num_sms;
}

// Count one kernel launch on context c (for launch statistics).
#define CCM_COUNT(c) ((c)->launches++)

Ctx* ctx_of(ccm_ctx* x);

// Grow-only scratch buffer for one slot (contents not preserved on growth).
int ws_get(Ctx* c, Slot s, size_t bytes, void** out);
int host_scalars(Ctx* c, size_t bytes, void** out);

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Penalty cap: a positive option value as given; otherwise 10 for q = 2 and 1
// for q = 1 and q = inf (the separable-ball norms converged in far fewer Newton
// and CG steps with the lower cap on the measured paths), and never below the
// initial penalty sigma0.
inline double resolve_sigma_max(const ccm_options& o, int q) {
  if (o.sigma_max > 0) return o.sigma_max;
  const double cap = q == 2 ? 10.0 : 1.0;
  return o.sigma0 > cap ? o.sigma0 : cap;
}

// ---------------------------------------------------------------- device helpers
template <typename T> struct Vec4;
template <> struct Vec4<double> {
  __device__ __forceinline__ static void load(const double* p, double (&v)[4]) {
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ __forceinline__ static void store(double* p, const double (&v)[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
};
template <> struct Vec4<float> {
  __device__ __forceinline__ static void load(const float* p, float (&v)[4]) {
    float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  __device__ __forceinline__ static void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

// A row held in registers by one lane: CH quads.
template <typename T, int CH>
struct RowReg {
  T v[CH][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) v[c][e] = T(0);
  }
};

// Load the lane's quads of a row (elements beyond ld are treated as zero).
template <int LANES, int CH, typename S, typename T>
__device__ __forceinline__ void row_load(const S* row, int ld, int lane, T (&out)[CH][4]) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    int q = c * LANES + lane;
    if (4 * q < ld) {
      S tmp[4];
      Vec4<S>::load(row + 4 * q, tmp);
#pragma unroll
      for (int e = 0; e < 4; ++e) out[c][e] = T(tmp[e]);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) out[c][e] = T(0);
    }
  }
}

template <int LANES, int CH, typename S, typename T>
__device__ __forceinline__ void row_store(S* row, int ld, int lane, const T (&in)[CH][4]) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    int q = c * LANES + lane;
    if (4 * q < ld) {
      S tmp[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) tmp[e] = S(in[c][e]);
      Vec4<S>::store(row + 4 * q, tmp);
    }
  }
}

// Sum over the LANES lanes of one group (fixed butterfly: deterministic).
template <int LANES, typename T>
__device__ __forceinline__ T group_sum(T x, unsigned mask) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, LANES);
  return x;
}

template <int LANES>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (LANES >= 32) {
    return 0xffffffffu;
  } else {
    unsigned base = (threadIdx.x & 31) / LANES * LANES;
    return ((1u << LANES) - 1u) << base;
  }
}

// Deterministic grid reduction of NRED doubles.
// Every block reduces its threads' values in a fixed order and writes one
// partial per quantity; the last block to arrive (counter) sums the partials
// in block order and returns true with the totals in `tot` (all its threads).
// The counter is reset by that block, so kernels can be relaunched.
// `nextra` further partial rows (indices gridDim.x .. gridDim.x + nextra - 1,
// written before their writers' blocks arrive) join the final sum in index order.
template <int NRED>
__device__ __forceinline__ bool grid_reduce(double (&acc)[NRED], double* partials,
                                            unsigned* counter, double (&tot)[NRED],
                                            int nextra = 0) {
  __shared__ double sh[32][NRED];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NRED; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
      double v = lane < nwarps ? sh[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) partials[(size_t)blockIdx.x * NRED + k] = v;
    }
    if (lane == 0) {
      __threadfence();
      unsigned prev = atomicAdd(counter, 1u);
      is_last = (prev == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // every thread of the last block sums a strided subset, then a fixed tree
#pragma unroll
  for (int k = 0; k < NRED; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x + nextra; b += blockDim.x)
      v += __ldcg(partials + (size_t)b * NRED + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
      double v = lane < nwarps ? sh[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sh[0][k] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NRED; ++k) tot[k] = sh[0][k];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Cluster labels of X (row stride ldx) on an edge list (labels.cu).
int labels_device(Ctx* c, const double* X, int64_t ldx, int64_t n, int d, const int2* edges,
                  int64_t m, int32_t* labels, int32_t* n_clusters, cudaStream_t s);

// Tensor-core kNN candidates (knn_tc.cu): whether the kernel handles (d, K'),
// and the candidate lists (n x *used_kp, *used_kp >= Kp) with their thresholds.
int knn_tc_supported(int d, int Kp);
int knn_candidates_tc(Ctx* c, const float* At, int ldf, int64_t n, int d, int Kp, int* cand,
                      float* cand_thr, int* used_kp, cudaStream_t s);

// Node relabelling for locality (reorder.cu): perm maps new -> old node, iperm
// old -> new; edges / w are the relabelled, oriented and sorted edge list and its
// weights; eperm maps new -> old edge id, complemented (~id) where the endpoints
// swapped (the edge's B X row changes sign). All device arrays in scratch.
struct Relabel {
  int* perm = nullptr;
  int* iperm = nullptr;
  int2* edges = nullptr;
  double* w = nullptr;
  int* eperm = nullptr;
};
int locality_relabel(Ctx* c, const int2* edges, const double* w, int64_t m, int64_t n,
                     Relabel& r, cudaStream_t s);
// Visiting order of the register-form gathers (reorder.cu): windows of 4,096 nodes
// in index order, by decreasing degree inside a window. ord: device n int32.
int degree_order(Ctx* c, const int64_t* off, int64_t n, int* ord, cudaStream_t s);

// Scan helpers (device-wide exclusive scan of int32 / int64).
int scan_exclusive_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_host,
                       cudaStream_t s);

}  // namespace ccm
