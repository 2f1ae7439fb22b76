// Cluster labels from a solution X: union-find over fused edges.
//
// Sec. 1 assigns a_i and a_j to one cluster when x_i* = x_j*. Fusion rule of
// this library: edge (i, j) is fused when sum_k (x_ik - x_jk)^2, evaluated in
// float64 with one rounding per subtraction, product and addition (features
// in ascending order, no FMA), is <= 1e-12. Clusters are the connected
// components of the fused edges; the label of a node is the rank of its
// cluster's smallest node index.
//
// Union-find: every fused edge hooks the larger of its two roots under the
// smaller with atomicMin, retrying until both endpoints share a root, so each
// component ends with its smallest index as root; a pointer-jumping pass then
// flattens the forest. Roots are ranked with an exclusive scan.
#include "ccm_internal.cuh"

namespace ccm {

__global__ void k_lab_init(int32_t* parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (int32_t)i;
}

__device__ __forceinline__ int32_t lab_find(int32_t* parent, int32_t x, int64_t n, int* err) {
  // parent[x] <= x always and each step moves to a strictly smaller index,
  // so a root is reached within n steps
  for (int64_t guard = 0; guard <= n; ++guard) {
    int32_t p = __ldcg(parent + x);
    if (p == x) return x;
    x = p;
  }
  atomicExch(err, 1);
  return x;
}

__global__ void k_lab_hook(const double* __restrict__ X, int64_t ldx, int d,
                           const int2* __restrict__ edges, int64_t m, int32_t* parent,
                           int64_t n, int* err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int2 ij = edges[e];
    const double* xi = X + (int64_t)ij.x * ldx;
    const double* xj = X + (int64_t)ij.y * ldx;
    // the partial sums of non-negative terms never decrease, so the sum stops as
    // soon as it passes the threshold: the decision is the one of the full sum
    double acc = 0.0;
    for (int k = 0; k < d && acc <= 1e-12; ++k) {
      double dl = __dsub_rn(xi[k], xj[k]);
      acc = __dadd_rn(acc, __dmul_rn(dl, dl));
    }
    if (!(acc <= 1e-12)) continue;
    int32_t a = lab_find(parent, ij.x, n, err), b = lab_find(parent, ij.y, n, err);
    for (int64_t guard = 0; a != b && guard <= n; ++guard) {
      int32_t lo = a < b ? a : b, hi = a < b ? b : a;
      int32_t old = atomicMin(parent + hi, lo);
      if (old == hi) break;                 // hooked hi under lo
      // hi already points below: continue from its current parent
      if (hi == a) a = lab_find(parent, old, n, err);
      else b = lab_find(parent, old, n, err);
    }
  }
}

__global__ void k_lab_flatten(int32_t* parent, int64_t n, int64_t* is_root, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = lab_find(parent, (int32_t)i, n, err);
    is_root[i] = (r == (int32_t)i) ? 1 : 0;
  }
}

__global__ void k_lab_assign(const int32_t* __restrict__ parent, int64_t n,
                             const int64_t* __restrict__ rank, int32_t* __restrict__ labels,
                             int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    // parents were flattened into root pointers by k_lab_flatten's finds only
    // along the path; resolve fully here (read-only)
    int32_t x = (int32_t)i;
    for (int64_t guard = 0; guard <= n; ++guard) {
      int32_t p = parent[x];
      if (p == x) break;
      x = p;
    }
    if (parent[x] != x) atomicExch(err, 1);
    labels[i] = (int32_t)rank[x];
  }
}

int labels_device(Ctx* c, const double* X, int64_t ldx, int64_t n, int d, const int2* edges,
                  int64_t m, int32_t* labels, int32_t* n_clusters, cudaStream_t s) {
  void *p1, *p2, *p3, *p4;
  CCM_TRY(ws_get(c, S_BATCH0, (size_t)n * 4, &p1));
  CCM_TRY(ws_get(c, S_BATCH1, (size_t)n * 8, &p2));
  CCM_TRY(ws_get(c, S_BATCH2, (size_t)n * 8, &p3));
  CCM_TRY(ws_get(c, S_BATCH3, 64, &p4));
  int32_t* parent = (int32_t*)p1;
  int64_t* is_root = (int64_t*)p2;
  int64_t* rank = (int64_t*)p3;
  int* err = (int*)p4;
  CCM_CUDA(cudaMemsetAsync(err, 0, 4, s));
  int blocks_n = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
  int blocks_m = (int)std::min<int64_t>((m + 255) / 256, (int64_t)c->num_sms * 8);
  blocks_n = blocks_n < 1 ? 1 : blocks_n;
  blocks_m = blocks_m < 1 ? 1 : blocks_m;
  k_lab_init<<<blocks_n, 256, 0, s>>>(parent, n);
  CCM_COUNT(c);
  if (m > 0) {
    k_lab_hook<<<blocks_m, 256, 0, s>>>(X, ldx, d, edges, m, parent, n, err);
    CCM_COUNT(c);
  }
  k_lab_flatten<<<blocks_n, 256, 0, s>>>(parent, n, is_root, err);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  int64_t total = 0;
  CCM_TRY(scan_exclusive_i64(c, is_root, rank, n, n_clusters ? &total : nullptr, s));
  k_lab_assign<<<blocks_n, 256, 0, s>>>(parent, n, rank, labels, err);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  if (n_clusters) {
    void* hp;
    CCM_TRY(host_scalars(c, 64, &hp));
    CCM_CUDA(cudaMemcpyAsync(hp, err, 4, cudaMemcpyDeviceToHost, s));
    CCM_CUDA(cudaStreamSynchronize(s));
    if (*(int*)hp) {
      set_error("labels: union-find step bound exceeded");
      return CCM_ERR_TIMEOUT;
    }
    *n_clusters = (int32_t)total;
  }
  return CCM_OK;
}

}  // namespace ccm

using namespace ccm;

extern "C" int ccm_labels(ccm_ctx* x, const double* X, int64_t n, int32_t d,
                          const int32_t* edges, int64_t m, int32_t* labels,
                          int32_t* n_clusters, ccm_stream_t stream) {
  Ctx* c = ctx_of(x);
  if (!c || !X || !labels || n <= 0 || d <= 0 || m < 0 || (m > 0 && !edges) ||
      n > INT32_MAX) {
    set_error("ccm_labels: invalid argument");
    return CCM_ERR_INVALID_ARG;
  }
  if (((uintptr_t)edges) % 8) {
    set_error("ccm_labels: edges must be 8-byte aligned");
    return CCM_ERR_INVALID_ARG;
  }
  CCM_CUDA(cudaSetDevice(c->device));
  int32_t nc = 0;
  CCM_TRY(labels_device(c, X, d, n, d, (const int2*)edges, m, labels, &nc,
                        (cudaStream_t)stream));
  if (n_clusters) *n_clusters = nc;
  return CCM_OK;
}
