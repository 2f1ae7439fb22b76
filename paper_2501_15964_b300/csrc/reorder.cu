// Node relabelling for locality in the gather kernels (grid engine).
//
// The operator, the node gradient and the edge passes gather rows of their
// neighbours (R, yhat, Pi(y), X). When the points arrive in an order unrelated
// to the graph (the Gaussian-mixture workloads draw every point's component at
// random), the two reads of an edge's row, one per endpoint, are far apart in
// time and both come from HBM. Sorting the nodes by connected component of the
// kNN graph (stable: by smallest member, then by index) puts every edge's
// endpoints within one component's index range, so the grid-stride sweeps read
// an edge's rows twice within a short window and the second read hits L2. The
// solve runs on the relabelled problem; inputs are gathered and outputs
// scattered back through the permutations, so callers see the original order.
//
// Everything here is deterministic: components by min-label hooking (every
// component ends labelled by its smallest index) and a stable LSD radix sort
// (8-bit digits; ranks within a 256-item block from warp match masks).
#include <algorithm>

#include "ccm_internal.cuh"

namespace ccm {

// ---------------------------------------------------------------- components
__device__ __forceinline__ int cc_root(const int* parent, int x) {
  int p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

__global__ void k_cc_init(int* __restrict__ parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (int)i;
}

// parent[x] <= x always, so roots only move to smaller indices and the walks end
__global__ void k_cc_hook(const int2* __restrict__ edges, int64_t m, int* parent, int* changed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 ij = edges[e];
    const int a = cc_root(parent, ij.x), b = cc_root(parent, ij.y);
    if (a != b) {
      atomicMin(parent + max(a, b), min(a, b));
      *changed = 1;
    }
  }
}

__global__ void k_cc_flatten(int* parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = cc_root(parent, (int)i);
}

// ---------------------------------------------------------------- radix sort
// One pass of a stable LSD radix sort on the 8-bit digit at `shift`: block b
// holds items [256 b, 256 b + 256); cnt / off are digit-major [digit][block].
template <typename K>
__global__ void k_rs_count(const K* __restrict__ keys, int64_t n, int shift, int nblk,
                           int64_t* __restrict__ cnt) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 255)], 1);
  __syncthreads();
  cnt[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

template <typename K, typename V>
__global__ void k_rs_scatter(const K* __restrict__ kin, const V* __restrict__ vin, int64_t n,
                             int shift, int nblk, const int64_t* __restrict__ off,
                             K* __restrict__ kout, V* __restrict__ vout) {
  __shared__ int wc[8][256];  // per-warp digit counts
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < 8 * 256; t += 256) (&wc[0][0])[t] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const bool valid = i < n;
  // items past the end get a digit no real item has (256 + lane)
  const unsigned dg = valid ? (unsigned)((kin[i] >> shift) & 255) : 256u + lane;
  const unsigned same = __match_any_sync(0xffffffffu, dg);
  const int wrank = __popc(same & ((1u << lane) - 1u));
  if (valid && lane == __ffs(same) - 1) wc[warp][dg] = __popc(same);
  __syncthreads();
  if (valid) {
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wc[w][dg];
    const int64_t dst = off[(int64_t)dg * nblk + blockIdx.x] + before + wrank;
    kout[dst] = kin[i];
    vout[dst] = vin[i];
  }
}

// Stable sort of n (key, value) pairs by the low `bits` bits of the key. The
// buffers ping-pong; returns in *kres / *vres the ones holding the result.
template <typename K, typename V>
static int radix_sort(Ctx* c, K* k0, V* v0, K* k1, V* v1, int64_t n, int bits, int64_t* cnt,
                      int64_t* off, K** kres, V** vres, cudaStream_t s) {
  const int nblk = (int)((n + 255) / 256);
  K* ka = k0;
  V* va = v0;
  K* kb = k1;
  V* vb = v1;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_count<K><<<nblk, 256, 0, s>>>(ka, n, shift, nblk, cnt);
    CCM_COUNT(c);
    CCM_TRY(scan_exclusive_i64(c, cnt, off, (int64_t)256 * nblk, nullptr, s));
    k_rs_scatter<K, V><<<nblk, 256, 0, s>>>(ka, va, n, shift, nblk, off, kb, vb);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  *kres = ka;
  *vres = va;
  return CCM_OK;
}

static int bit_width(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return std::max(b, 1);
}

// ---------------------------------------------------------------- relabelling
__global__ void k_iota(int* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int)i;
}

__global__ void k_widen(const int* __restrict__ v, unsigned long long* __restrict__ k, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    k[i] = (unsigned long long)v[i];
}

__global__ void k_invert(const int* __restrict__ perm, int* __restrict__ iperm, int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    iperm[perm[p]] = (int)p;
}

// new endpoints (lo, hi) of every old edge as the key lo * n + hi; the value is
// the old edge id, complemented when the endpoints swap (B X changes sign there)
__global__ void k_edge_keys(const int2* __restrict__ edges, int64_t m, int64_t n,
                            const int* __restrict__ iperm, unsigned long long* __restrict__ key,
                            int* __restrict__ val) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 ij = edges[e];
    const int a = iperm[ij.x], b = iperm[ij.y];
    const bool flip = a > b;
    key[e] = (unsigned long long)(flip ? b : a) * (unsigned long long)n + (flip ? a : b);
    val[e] = flip ? ~(int)e : (int)e;
  }
}

__global__ void k_edge_emit(const unsigned long long* __restrict__ key,
                            const int* __restrict__ val, const double* __restrict__ w,
                            int64_t m, int64_t n, int2* __restrict__ edges_p,
                            double* __restrict__ w_p) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = key[e];
    edges_p[e] = make_int2((int)(k / (unsigned long long)n), (int)(k % (unsigned long long)n));
    const int v = val[e];
    w_p[e] = w[v < 0 ? ~v : v];
  }
}

// ---------------------------------------------------------------- processing order
// Order in which the register-form gathers visit nodes: windows of 2^wshift
// consecutive nodes in index order, inside a window by decreasing degree (stable).
// The groups of a warp then own nodes of (nearly) equal degree and run their
// incidence loops for the same number of iterations, while the window keeps the
// sweep local in the node order.
__global__ void k_degree_keys(const int64_t* __restrict__ off, int64_t n, int wshift,
                              unsigned long long* __restrict__ key, int* __restrict__ val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t deg = off[i + 1] - off[i];
    const unsigned long long inv = 65535ull - (unsigned long long)(deg < 65535 ? deg : 65535);
    key[i] = ((unsigned long long)(i >> wshift) << 16) | inv;
    val[i] = (int)i;
  }
}

int degree_order(Ctx* c, const int64_t* off, int64_t n, int* ord, cudaStream_t s) {
  const int wshift = 12;
  const int threads = 256;
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->num_sms * 8));
  const int64_t nblk = (n + 255) / 256;
  const size_t b_k = round_up(n * 8, 256), b_v = round_up(n * 4, 256),
               b_c = round_up(256 * nblk * 8, 256);
  void* p;
  CCM_TRY(ws_get(c, S_ORDER_TMP, 2 * b_k + 2 * b_v + 2 * b_c, &p));
  char* q = (char*)p;
  unsigned long long* k0 = (unsigned long long*)q;
  unsigned long long* k1 = (unsigned long long*)(q + b_k);
  int* v0 = (int*)(q + 2 * b_k);
  int* v1 = (int*)(q + 2 * b_k + b_v);
  int64_t* cnt = (int64_t*)(q + 2 * b_k + 2 * b_v);
  int64_t* offs = (int64_t*)(q + 2 * b_k + 2 * b_v + b_c);
  k_degree_keys<<<blocks, threads, 0, s>>>(off, n, wshift, k0, v0);
  CCM_COUNT(c);
  unsigned long long* kr;
  int* vr;
  const int bits = bit_width((((uint64_t)(n - 1)) >> wshift << 16) | 65535ull);
  CCM_TRY(radix_sort(c, k0, v0, k1, v1, n, bits, cnt, offs, &kr, &vr, s));
  CCM_CUDA(cudaMemcpyAsync(ord, vr, n * 4, cudaMemcpyDeviceToDevice, s));
  return CCM_OK;
}

int locality_relabel(Ctx* c, const int2* edges, const double* w, int64_t m, int64_t n,
                     Relabel& r, cudaStream_t s) {
  const int threads = 256;
  auto nb = [&](int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads,
                                                       (int64_t)c->num_sms * 8));
  };
  const int64_t big = std::max(n, m);
  const int64_t nblk = (big + 255) / 256;
  const size_t b_n = round_up(n * 4, 256), b_m = round_up(m * 4, 256);
  const size_t b_k = round_up(big * 8, 256), b_c = round_up(256 * nblk * 8, 256);
  // perm, iperm, parent | edges_p (8m), w_p (8m), eperm | 2 key + 2 value buffers | cnt, off
  const size_t total = 3 * b_n + 2 * round_up(m * 8, 256) + b_m + 2 * b_k + 2 * round_up(big * 4, 256) +
                       2 * b_c + 256;
  void* p;
  CCM_TRY(ws_get(c, S_REORD, total, &p));
  char* q = (char*)p;
  auto take = [&](size_t bytes) {
    char* a = q;
    q += bytes;
    return a;
  };
  r.perm = (int*)take(b_n);
  r.iperm = (int*)take(b_n);
  int* parent = (int*)take(b_n);
  r.edges = (int2*)take(round_up(m * 8, 256));
  r.w = (double*)take(round_up(m * 8, 256));
  r.eperm = (int*)take(b_m);
  unsigned long long* k0 = (unsigned long long*)take(b_k);
  unsigned long long* k1 = (unsigned long long*)take(b_k);
  int* v0 = (int*)take(round_up(big * 4, 256));
  int* v1 = (int*)take(round_up(big * 4, 256));
  int64_t* cnt = (int64_t*)take(b_c);
  int64_t* off = (int64_t*)take(b_c);
  void* pf;
  CCM_TRY(ws_get(c, S_SCRATCH6, 64, &pf));
  int* changed = (int*)pf;
  void* hp;
  CCM_TRY(host_scalars(c, 64, &hp));

  // 1. components: every node labelled by its component's smallest index
  k_cc_init<<<nb(n), threads, 0, s>>>(parent, n);
  CCM_COUNT(c);
  for (int it = 0; it < 64; ++it) {
    CCM_CUDA(cudaMemsetAsync(changed, 0, 4, s));
    k_cc_hook<<<nb(m), threads, 0, s>>>(edges, m, parent, changed);
    CCM_COUNT(c);
    k_cc_flatten<<<nb(n), threads, 0, s>>>(parent, n);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    CCM_CUDA(cudaMemcpyAsync(hp, changed, 4, cudaMemcpyDeviceToHost, s));
    CCM_CUDA(cudaStreamSynchronize(s));
    if (*(int*)hp == 0) break;
  }
  // 2. nodes sorted by (component label, index): stable sort of the labels
  k_iota<<<nb(n), threads, 0, s>>>(v0, n);
  CCM_COUNT(c);
  k_widen<<<nb(n), threads, 0, s>>>(parent, k0, n);  // labels as the sort keys
  CCM_COUNT(c);
  unsigned long long* kr;
  int* vr;
  CCM_TRY(radix_sort(c, k0, v0, k1, v1, n, bit_width((uint64_t)(n - 1)), cnt, off, &kr, &vr, s));
  CCM_CUDA(cudaMemcpyAsync(r.perm, vr, n * 4, cudaMemcpyDeviceToDevice, s));
  k_invert<<<nb(n), threads, 0, s>>>(r.perm, r.iperm, n);
  CCM_COUNT(c);
  // 3. edges relabelled, oriented (lo, hi) and sorted lexicographically
  if (m > 0) {
    k_edge_keys<<<nb(m), threads, 0, s>>>(edges, m, n, r.iperm, k0, v0);
    CCM_COUNT(c);
    const int bits = bit_width((uint64_t)n * (uint64_t)n - 1);
    CCM_TRY(radix_sort(c, k0, v0, k1, v1, m, bits, cnt, off, &kr, &vr, s));
    k_edge_emit<<<nb(m), threads, 0, s>>>(kr, vr, w, m, n, r.edges, r.w);
    CCM_COUNT(c);
    CCM_CUDA(cudaMemcpyAsync(r.eperm, vr, m * 4, cudaMemcpyDeviceToDevice, s));
  }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

}  // namespace ccm
