// Two-level preconditioner of the Newton-CG (grid engine, q = 2).
//
// Where many edges are inside their balls (P_l = I) or outside with P_l close
// to the projection I - yhat yhat^T, the Newton matrix V = I + sigma B^T P B
// restricted to a strongly coupled group of nodes is close to I + sigma L (L a
// graph Laplacian, in every coordinate), and the one-scalar-per-node Jacobi
// preconditioner leaves the group-constant modes of V at relative eigenvalue
// about 1 / (1 + sigma deg). The coarse correction adds one unknown per
// aggregate: a connected component of the strong edges (inside, or outside with
// t_l >= kCoarseStrong) of at least kCoarseMinSize nodes, at most
// kCoarseMaxAgg of the largest:
//
//     M^-1 r = D^-1 r + P A_c^-1 P^T r,    A_c = P^T (I + sigma B^T diag(t) B) P,
//
// with P the n x K 0/1 aggregation matrix, D^-1 = diag(Minv) and the scalar
// t_l = tr(P_l) / d per edge (1 inside, alpha_l (d - 1) / d outside, 0 inert),
// so that A_c = diag(aggregate sizes) + sigma L_agg(t) is the weighted Laplacian
// of the aggregate graph plus a diagonal (edges from an aggregate to a node of
// no aggregate add to its diagonal). A_c is symmetric positive definite and
// strictly diagonally dominant; it is inverted once per Newton step (float32
// Gauss-Jordan in one block, no pivoting), and M^-1 is a fixed symmetric
// positive-definite operator, so plain preconditioned CG applies.
//
// Per CG iteration: y = P^T R (k_co_restrict), z = A_c^-1 y (k_co_apply),
// U = Minv R + P z and gamma = <R, U> (k_co_prolong); the operator then runs on
// U with unit scalars (its Jacobi scaling is already in U).
//
// Measured on the MNIST-shaped path (n = 10,000, d = 784, 50 gammas): 2,353 of
// its 2,911 CG steps fall at the one gamma where 10,000 singletons fuse into
// 3,488 clusters, and there the strong edges form at most 10 aggregates; the
// correction saves 5 % of the CG steps (2,773) and costs more than it saves,
// so it is off by default (options.coarse).
//
// Assembly is deterministic: the coarse matrix is summed in 64-bit fixed point
// (integer atomics), and every other sum runs in a fixed order.
#include <algorithm>
#include <vector>

#include "ccm_internal.cuh"
#include "solve_common.cuh"
#include "coarse.cuh"
#include "ring_kernels.cuh"
#include "ssnal_kernels.cuh"

namespace ccm {

namespace {

constexpr double kFixScale = 1048576.0;  // 2^20: fixed-point scale of the coarse matrix

__device__ __forceinline__ int co_root(const int* parent, int x) {
  int p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

__global__ void k_co_init(int* __restrict__ parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (int)i;
}

// min-label hooking over the strong edges: inside edges (t_l = 1) and outside
// edges with t_l = alpha_l (d - 1) / d >= kCoarseStrong (parent[x] <= x always)
template <typename Tc>
__global__ void k_co_hook(const int2* __restrict__ edges, const uint8_t* __restrict__ kind,
                          const Tc* __restrict__ alpha, float alpha_min, int64_t m, int* parent,
                          int* changed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t kd = kind[e];
    if (!(kd == K_IN || (kd == K_OUT && (float)alpha[e] >= alpha_min))) continue;
    const int2 ij = edges[e];
    const int a = co_root(parent, ij.x), b = co_root(parent, ij.y);
    if (a != b) {
      atomicMin(parent + max(a, b), min(a, b));
      *changed = 1;
    }
  }
}

__global__ void k_co_flatten(int* parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = co_root(parent, (int)i);
}

// Coarse matrix off the diagonal sizes: sigma t_l per edge between different
// aggregates (or from an aggregate to a node of none), in fixed point.
template <typename Tc>
__global__ void k_co_assemble(const int2* __restrict__ edges, const uint8_t* __restrict__ kind,
                              const Tc* __restrict__ alpha, int64_t m, const int* __restrict__ agg,
                              double sigma, int d, int K, unsigned long long* __restrict__ A) {
  const double tr_out = (double)(d - 1) / (double)d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t kd = kind[e];
    const double t = kd == K_IN ? 1.0 : (kd == K_OUT ? (double)alpha[e] * tr_out : 0.0);
    if (!(t > 0.0)) continue;
    const int2 ij = edges[e];
    const int a = agg[ij.x], b = agg[ij.y];
    if (a == b) continue;  // inside one aggregate (or both in none): no coarse term
    const unsigned long long v = (unsigned long long)llrint(sigma * t * kFixScale);
    if (a >= 0) atomicAdd(A + (int64_t)a * K + a, v);
    if (b >= 0) atomicAdd(A + (int64_t)b * K + b, v);
    if (a >= 0 && b >= 0) {
      atomicAdd(A + (int64_t)a * K + b, ~v + 1ull);  // -v in two's complement
      atomicAdd(A + (int64_t)b * K + a, ~v + 1ull);
    }
  }
}

// In-place Gauss-Jordan inversion of A_c = diag(sizes) + fixed-point part, in
// float32 in shared memory (K <= kCoarseMaxAgg), one block of 1024 threads. Without
// pivoting: A_c is strictly diagonally dominant with a positive diagonal.
__global__ void __launch_bounds__(1024)
k_co_invert(const unsigned long long* __restrict__ Afix, const int* __restrict__ mem_off, int K,
            float* __restrict__ Ainv) {
  extern __shared__ float sm[];
  float* M = sm;          // K x K
  float* col = sm + K * K;  // pivot column of the current step
  const int KK = K * K;
  for (int q = threadIdx.x; q < KK; q += blockDim.x) {
    const int r = q / K, cc = q - r * K;
    double v = (double)(long long)Afix[q] / kFixScale;
    if (r == cc) v += (double)(mem_off[r + 1] - mem_off[r]);
    M[q] = (float)v;
  }
  __syncthreads();
  for (int p = 0; p < K; ++p) {
    const float piv = M[p * K + p];
    for (int r = threadIdx.x; r < K; r += blockDim.x) col[r] = M[r * K + p];
    __syncthreads();
    const float ip = 1.0f / piv;
    for (int cc = threadIdx.x; cc < K; cc += blockDim.x)
      M[p * K + cc] = (cc == p ? 1.0f : M[p * K + cc]) * ip;
    __syncthreads();
    for (int q = threadIdx.x; q < KK; q += blockDim.x) {
      const int r = q / K, cc = q - r * K;
      if (r == p) continue;
      M[q] = (cc == p ? 0.0f : M[q]) - col[r] * M[p * K + cc];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < KK; q += blockDim.x) Ainv[q] = M[q];
}

// y = P^T R: block (k, column block) sums the rows of aggregate k's members
// (in member order) for 32 quads of columns; 8 member slices per block joined
// in slice order.
template <typename Tc>
__global__ void __launch_bounds__(256)
k_co_restrict(const Tc* __restrict__ R, const int* __restrict__ mem_off,
              const int* __restrict__ mem, int ld, Tc* __restrict__ y, const Ctl* ctl) {
  if (!ctl->cg.active) return;
  __shared__ Tc part[8][32][4];
  const int k = blockIdx.y;
  const int qd = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int q = blockIdx.x * 32 + qd;  // quad of columns
  const bool live = 4 * q < ld;
  Tc s[4] = {(Tc)0, (Tc)0, (Tc)0, (Tc)0};
  const int b = mem_off[k], e = mem_off[k + 1];
  if (live)
    for (int t = b + slice; t < e; t += 8) {
      Tc v[4];
      Vec4<Tc>::load(R + (int64_t)mem[t] * ld + 4 * q, v);
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] += v[c];
    }
#pragma unroll
  for (int c = 0; c < 4; ++c) part[slice][qd][c] = s[c];
  __syncthreads();
  if (slice == 0 && live) {
#pragma unroll
    for (int sl = 1; sl < 8; ++sl)
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] += part[sl][qd][c];
    Vec4<Tc>::store(y + (int64_t)k * ld + 4 * q, s);
  }
}

// z = A_c^-1 y (K x K times K x ld), one thread per (aggregate, column).
template <typename Tc>
__global__ void __launch_bounds__(256)
k_co_apply(const float* __restrict__ Ainv, const Tc* __restrict__ y, int K, int ld,
           Tc* __restrict__ z, const Ctl* ctl) {
  if (!ctl->cg.active) return;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (col >= ld) return;
  float acc = 0.0f;
  for (int j = 0; j < K; ++j) acc = fmaf(Ainv[k * K + j], (float)y[(int64_t)j * ld + col], acc);
  z[(int64_t)k * ld + col] = (Tc)acc;
}

// U = Minv R + P z; gamma = <R, U> (float-float per thread, then float64 in
// block order); beta = gamma / gamma_prev; stop on a non-positive gamma.
template <typename Tc>
__global__ void __launch_bounds__(256)
k_co_prolong(const Tc* __restrict__ R, const Tc* __restrict__ Minv, const Tc* __restrict__ z,
             const int* __restrict__ agg, int64_t n, int ld, Tc* __restrict__ U,
             double* partials, Ctl* ctl) {
  if (!ctl->cg.active) return;
  Tc g_t = (Tc)0, g_e = (Tc)0;
  const int64_t total = n * ld;
  for (int64_t t4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; t4 < total;
       t4 += (int64_t)gridDim.x * blockDim.x * 4) {
    const int64_t i = t4 / ld;
    const int col = (int)(t4 - i * ld);
    const Tc mi = Minv[i];
    const int a = agg[i];
    Tc r[4], u[4], zz[4] = {(Tc)0, (Tc)0, (Tc)0, (Tc)0};
    Vec4<Tc>::load(R + t4, r);
    if (a >= 0) Vec4<Tc>::load(z + (int64_t)a * ld + col, zz);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      u[k] = mi * r[k] + zz[k];
      dot_acc(g_t, g_e, r[k], u[k]);
    }
    Vec4<Tc>::store(U + t4, u);
  }
  double acc[1] = {(double)g_t + (double)g_e};
  double tot[1];
  // the CG-init counter is free here: that kernel has finished
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_CGI], tot) && threadIdx.x == 0) {
    CgCtl& c = ctl->cg;
    c.beta = (c.it > 0 && c.rz > 0.0) ? tot[0] / c.rz : 0.0;
    c.rz = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) c.active = 0;
  }
}

}  // namespace

// ---------------------------------------------------------------- host side
template <typename Tc>
int coarse_build(Ctx* c, const int2* edges, const uint8_t* kind, const Tc* alpha, int64_t n,
                 int64_t m, double sigma, int d, int ld, CoarsePlan<Tc>& cp, cudaStream_t s) {
  cp.K = 0;
  if (n <= 0 || m <= 0) return CCM_OK;
  const int threads = 256;
  auto nb = [&](int64_t work) {
    return (int)std::max<int64_t>(
        1, std::min<int64_t>((work + threads - 1) / threads, (int64_t)c->num_sms * 4));
  };
  void* p;
  CCM_TRY(ws_get(c, S_CO_PARENT, (size_t)(n + 1) * 4, &p));
  int* parent = (int*)p;
  int* changed = parent + n;
  const float alpha_min = (float)(kCoarseStrong * (double)d / (double)std::max(d - 1, 1));
  // host copies in pageable memory: the context's pinned scalar buffer holds the
  // solver's control block and must not move
  std::vector<int> root((size_t)n);
  int flag = 0;
  // 1. components of the inside edges (every node labelled by its smallest member)
  k_co_init<<<nb(n), threads, 0, s>>>(parent, n);
  CCM_COUNT(c);
  for (int it = 0; it < 64; ++it) {
    CCM_CUDA(cudaMemsetAsync(changed, 0, 4, s));
    k_co_hook<Tc><<<nb(m), threads, 0, s>>>(edges, kind, alpha, alpha_min, m, parent, changed);
    CCM_COUNT(c);
    k_co_flatten<<<nb(n), threads, 0, s>>>(parent, n);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    CCM_CUDA(cudaMemcpyAsync(&flag, changed, 4, cudaMemcpyDeviceToHost, s));
    CCM_CUDA(cudaStreamSynchronize(s));
    if (flag == 0) {
      if (it == 0) return CCM_OK;  // no strong edge: no aggregate
      break;
    }
  }
  // 2. aggregates: components of at least kMinSize nodes, the kMaxAgg largest
  //    (ties by smallest member), numbered by smallest member
  CCM_CUDA(cudaMemcpyAsync(root.data(), parent, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  std::vector<int> size((size_t)n, 0);
  for (int64_t i = 0; i < n; ++i) ++size[(size_t)root[(size_t)i]];
  std::vector<int> cand;
  for (int64_t i = 0; i < n; ++i)
    if (root[(size_t)i] == (int)i && size[(size_t)i] >= kCoarseMinSize) cand.push_back((int)i);
  if (cand.empty()) return CCM_OK;
  if ((int)cand.size() > kCoarseMaxAgg) {
    std::stable_sort(cand.begin(), cand.end(),
                     [&](int a, int b) { return size[(size_t)a] > size[(size_t)b]; });
    cand.resize(kCoarseMaxAgg);
    std::sort(cand.begin(), cand.end());
  }
  const int K = (int)cand.size();
  std::vector<int> kid((size_t)n, -1);  // root -> aggregate
  for (int k = 0; k < K; ++k) kid[(size_t)cand[(size_t)k]] = k;
  // agg (n), then mem_off (K + 1), then mem (members in increasing index)
  std::vector<int> host((size_t)n + (size_t)K + 1 + (size_t)n);
  int* h_agg = host.data();
  int* h_off = h_agg + n;
  int* h_mem = h_off + K + 1;
  std::fill(h_off, h_off + K + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int a = kid[(size_t)root[(size_t)i]];
    h_agg[i] = a;
    if (a >= 0) ++h_off[a + 1];
  }
  for (int k = 0; k < K; ++k) h_off[k + 1] += h_off[k];
  {
    std::vector<int> fill(h_off, h_off + K);
    for (int64_t i = 0; i < n; ++i)
      if (h_agg[i] >= 0) h_mem[fill[(size_t)h_agg[i]]++] = (int)i;
  }
  const int64_t nmem = h_off[K];
  CCM_TRY(ws_get(c, S_CO_AGG, (size_t)(n + K + 1 + nmem) * 4, &p));
  int* d_agg = (int*)p;
  CCM_CUDA(cudaMemcpyAsync(d_agg, host.data(), (size_t)(n + K + 1 + nmem) * 4,
                           cudaMemcpyHostToDevice, s));
  // 3. coarse matrix and its inverse
  CCM_TRY(ws_get(c, S_CO_A, (size_t)K * K * 8, &p));
  unsigned long long* Afix = (unsigned long long*)p;
  CCM_TRY(ws_get(c, S_CO_AINV, (size_t)K * K * 4, &p));
  float* Ainv = (float*)p;
  CCM_CUDA(cudaMemsetAsync(Afix, 0, (size_t)K * K * 8, s));
  k_co_assemble<Tc><<<nb(m), threads, 0, s>>>(edges, kind, alpha, m, d_agg, sigma, d, K, Afix);
  CCM_COUNT(c);
  const size_t smem = ((size_t)K * K + (size_t)K) * 4;
  CCM_TRY(set_smem_limit(c, (const void*)k_co_invert, smem));
  k_co_invert<<<1, 1024, smem, s>>>(Afix, d_agg + n, K, Ainv);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  CCM_TRY(ws_get(c, S_CO_YZ, (size_t)2 * K * ld * sizeof(Tc), &p));
  cp.K = K;
  cp.agg = d_agg;
  cp.mem_off = d_agg + n;
  cp.mem = d_agg + n + K + 1;
  cp.Ainv = Ainv;
  cp.y = (Tc*)p;
  cp.z = cp.y + (size_t)K * ld;
  return CCM_OK;
}

template <typename Tc>
int coarse_precondition(Ctx* c, const CoarsePlan<Tc>& cp, const Tc* R, const Tc* Minv, Tc* U,
                        int64_t n, int ld, double* part, Ctl* ctl, cudaStream_t s) {
  const int qb = (ld / 4 + 31) / 32;
  k_co_restrict<Tc><<<dim3(qb, cp.K), 256, 0, s>>>(R, cp.mem_off, cp.mem, ld, cp.y, ctl);
  CCM_COUNT(c);
  k_co_apply<Tc><<<dim3((ld + 255) / 256, cp.K), 256, 0, s>>>(cp.Ainv, cp.y, cp.K, ld, cp.z, ctl);
  CCM_COUNT(c);
  const int64_t quads = n * ld / 4;
  const int blocks =
      (int)std::max<int64_t>(1, std::min<int64_t>((quads + 255) / 256, (int64_t)c->num_sms * 4));
  k_co_prolong<Tc><<<blocks, 256, 0, s>>>(R, Minv, cp.z, cp.agg, n, ld, U, part, ctl);
  CCM_COUNT(c);
  return CCM_OK;
}

template int coarse_build<float>(Ctx*, const int2*, const uint8_t*, const float*, int64_t,
                                 int64_t, double, int, int, CoarsePlan<float>&, cudaStream_t);
template int coarse_build<double>(Ctx*, const int2*, const uint8_t*, const double*, int64_t,
                                  int64_t, double, int, int, CoarsePlan<double>&, cudaStream_t);
template int coarse_precondition<float>(Ctx*, const CoarsePlan<float>&, const float*,
                                        const float*, float*, int64_t, int, double*, Ctl*,
                                        cudaStream_t);
template int coarse_precondition<double>(Ctx*, const CoarsePlan<double>&, const double*,
                                         const double*, double*, int64_t, int, double*, Ctl*,
                                         cudaStream_t);

}  // namespace ccm
