// ccm_labels_noalloc: cluster labels without any device allocation.
//
// Same result as ccm_labels (same fusion rule, same canonical numbering), for
// callers that must not allocate device memory: code running inside a memory
// pool or allocator that forbids cudaMalloc/cudaFree, callers that hold a CUDA
// graph capture open on other streams and cannot risk the synchronisation an
// allocation implies, or embedded hosts whose device memory is fully
// pre-reserved. Its scratch lives in a file-scope static __device__ array of
// fixed size (kNoAllocMaxN nodes; every GPU that loads this library keeps that
// array for the life of the process). The caller still passes X, the edges and
// the labels buffer.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress; make that first call before
// any stream capture. Every call reuses the same array, so calls that can
// overlap on the GPU (different streams, or different host threads) race and
// must be serialised by the caller.

#include "ccm_internal.cuh"

namespace ccm {

static constexpr int64_t kNoAllocMaxN = 1 << 18;  // 262,144 nodes (2 MB of scratch)
static constexpr int kNoAllocThreads = 1024;

// scratch: parent[kNoAllocMaxN] int32, rank[kNoAllocMaxN] int32, flags[4] int32
struct NoAllocScratch {
  int32_t parent[kNoAllocMaxN];
  int32_t rank[kNoAllocMaxN];
  int32_t flags[4];  // [0] error, [1] cluster count
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ int32_t na_find(int32_t* parent, int32_t x, int64_t n, int32_t* err) {
  for (int64_t g = 0; g <= n; ++g) {
    int32_t p = __ldcg(parent + x);
    if (p == x) return x;
    x = p;
  }
  atomicExch(err, 1);
  return x;
}

__global__ void k_na_init(NoAllocScratch* sc, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    sc->parent[i] = (int32_t)i;
  if (blockIdx.x == 0 && threadIdx.x < 4) sc->flags[threadIdx.x] = 0;
}

__global__ void k_na_hook(const double* __restrict__ X, int d, const int2* __restrict__ edges,
                          int64_t m, int64_t n, NoAllocScratch* sc) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 ij = edges[e];
    const double* xi = X + (int64_t)ij.x * d;
    const double* xj = X + (int64_t)ij.y * d;
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
      const double dl = __dsub_rn(xi[k], xj[k]);
      acc = __dadd_rn(acc, __dmul_rn(dl, dl));
    }
    if (!(acc <= 1e-12)) continue;
    int32_t a = na_find(sc->parent, ij.x, n, &sc->flags[0]);
    int32_t b = na_find(sc->parent, ij.y, n, &sc->flags[0]);
    for (int64_t g = 0; a != b && g <= n; ++g) {
      const int32_t lo = a < b ? a : b, hi = a < b ? b : a;
      const int32_t old = atomicMin(sc->parent + hi, lo);
      if (old == hi) break;
      if (hi == a) a = na_find(sc->parent, old, n, &sc->flags[0]);
      else b = na_find(sc->parent, old, n, &sc->flags[0]);
    }
  }
}

// flatten to roots and rank the roots with one block (n <= kNoAllocMaxN)
__global__ void __launch_bounds__(kNoAllocThreads)
k_na_rank(int64_t n, NoAllocScratch* sc, int32_t* __restrict__ labels) {
  __shared__ int32_t part[kNoAllocThreads];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    sc->parent[i] = na_find(sc->parent, (int32_t)i, n, &sc->flags[0]);
  __syncthreads();
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t s = threadIdx.x * chunk, e = min(n, s + chunk);
  int32_t cnt = 0;
  for (int64_t i = s; i < e; ++i) cnt += (sc->parent[i] == (int32_t)i) ? 1 : 0;
  part[threadIdx.x] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int32_t x = part[t];
      part[t] = run;
      run += x;
    }
    sc->flags[1] = run;
  }
  __syncthreads();
  int32_t run = part[threadIdx.x];
  for (int64_t i = s; i < e; ++i)
    if (sc->parent[i] == (int32_t)i) sc->rank[i] = run++;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) labels[i] = sc->rank[sc->parent[i]];
}

// Device address of the static scratch on the current device. Looked up on
// every call (a host-side table lookup once the module is loaded; it allocates
// nothing), so a context destroyed and re-created by cudaDeviceReset never
// leaves a stale address behind. The first lookup on a device loads the module
// and is the reason the first call must come before any stream capture.
static int noalloc_scratch(int device, NoAllocScratch** out) {
  if (device < 0) {
    set_error("ccm_labels_noalloc: device %d out of range", device);
    return CCM_ERR_INVALID_ARG;
  }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
  *out = (NoAllocScratch*)ptr;
  return CCM_OK;
}

}  // namespace ccm

using namespace ccm;

extern "C" int ccm_labels_noalloc(const double* X, int64_t n, int32_t d, const int32_t* edges,
                                  int64_t m, int32_t* labels, int32_t* n_clusters,
                                  ccm_stream_t stream) {
  if (!X || !labels || n <= 0 || d <= 0 || m < 0 || (m > 0 && !edges) ||
      ((uintptr_t)edges) % 8) {
    set_error("ccm_labels_noalloc: invalid argument");
    return CCM_ERR_INVALID_ARG;
  }
  if (n > kNoAllocMaxN) {
    set_error("ccm_labels_noalloc: n = %lld exceeds the static scratch maximum %lld",
              (long long)n, (long long)kNoAllocMaxN);
    return CCM_ERR_INVALID_ARG;
  }
  int dev = 0;
  CCM_CUDA(cudaGetDevice(&dev));
  NoAllocScratch* sc = nullptr;
  CCM_TRY(noalloc_scratch(dev, &sc));
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks_n = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024));
  const int blocks_m = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 1024));
  k_na_init<<<blocks_n, 256, 0, s>>>(sc, n);
  if (m > 0) k_na_hook<<<blocks_m, 256, 0, s>>>(X, d, (const int2*)edges, m, n, sc);
  k_na_rank<<<1, kNoAllocThreads, 0, s>>>(n, sc, labels);
  CCM_CUDA(cudaGetLastError());
  int32_t flags[2] = {0, 0};
  CCM_CUDA(cudaMemcpyAsync(flags, sc->flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  if (flags[0]) {
    set_error("ccm_labels_noalloc: union-find step bound exceeded");
    return CCM_ERR_TIMEOUT;
  }
  if (n_clusters) *n_clusters = flags[1];
  return CCM_OK;
}
