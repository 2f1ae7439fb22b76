// ccm_path_vjp: gradients of sum_t L_t(X*(gamma_t)) with respect to A and w.
//
// Not in the paper. Away from fusion events the solution is piecewise smooth:
// with clusters c (components of fused edges, the labelling rule of
// labels.cu), assignment Q, sizes M, and the edges N joining two clusters
// (s_l = (x_i - x_j)/||x_i - x_j||, c_l = gamma w_l / ||x_i - x_j||), the
// cluster values solve a smooth problem whose Hessian is
//     H = M (x) I_d + sum_{l in N} c_l (e_c(i) - e_c(j))(e_c(i) - e_c(j))^T (x) (I - s_l s_l^T).
// Implicit differentiation gives H lambda = Q^T G and
//     dL/da_i = lambda_c(i),   dL/dw_l = -gamma s_l^T (lambda_c(i) - lambda_c(j)) (l in N), 0 else.
// H is the Newton-CG operator of the solver applied on the cluster graph with
// alpha_l = c_l, yhat_l = s_l, sigma = 1 and the diagonal M instead of I, so the
// same node-pull kernel (k_cg_matvec) and CG kernels solve it: float32 CG on the
// corrections of a float64 iterative refinement (residuals in float64).
//
// Cluster member lists and the cluster-level incidence lists are built with a
// bitonic sort of (cluster, index) keys, so every sum has a fixed order and the
// result is bitwise reproducible.
#include <algorithm>
#include <cmath>

#include "ccm_internal.cuh"
#include "solve_common.cuh"
#include "ssnal_kernels.cuh"

namespace ccm {

// ---------------------------------------------------------------- bitonic sort
__global__ void k_bitonic_step(unsigned long long* a, int64_t n2, int64_t j, int64_t k) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = i ^ j;
    if (l > i) {
      const unsigned long long x = a[i], y = a[l];
      const bool up = (i & k) == 0;
      if (up ? (x > y) : (x < y)) {
        a[i] = y;
        a[l] = x;
      }
    }
  }
}

// sort keys[0..n2) ascending; n2 must be a power of two (pad with ~0ull)
static int bitonic_sort(Ctx* c, unsigned long long* a, int64_t n2, cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n2 + 255) / 256,
                                                                 (int64_t)c->num_sms * 8));
  for (int64_t k = 2; k <= n2; k <<= 1)
    for (int64_t j = k >> 1; j > 0; j >>= 1) {
      k_bitonic_step<<<blocks, 256, 0, s>>>(a, n2, j, k);
      CCM_COUNT(c);
    }
  CCM_CUDA(cudaGetLastError());
  return CCM_OK;
}

static int64_t pow2_at_least(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ---------------------------------------------------------------- kernels
__global__ void k_vjp_node_keys(const int32_t* __restrict__ lab, int64_t n, int64_t n2,
                                unsigned long long* __restrict__ keys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = (i < n) ? (((unsigned long long)(unsigned)lab[i] << 32) | (unsigned long long)i)
                      : ~0ull;
}

// cluster starts from the sorted node keys: cstart[c] for c in [0, K), cstart[K] = n
__global__ void k_vjp_cstart(const unsigned long long* __restrict__ keys, int64_t n, int64_t K,
                             int64_t* __restrict__ cstart) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned cl = (unsigned)(keys[p] >> 32);
    if (p == 0 || (unsigned)(keys[p - 1] >> 32) != cl) cstart[cl] = p;
    if (p == n - 1) cstart[K] = n;
  }
}

// per edge: N membership, s_l (padded row, float64), c_l; cluster-incidence keys
__global__ void k_vjp_edges(const double* __restrict__ X, int d, int ld,
                            const int2* __restrict__ edges, const double* __restrict__ w,
                            double gamma, const int32_t* __restrict__ lab, int64_t m, int64_t m2,
                            double* __restrict__ S, double* __restrict__ coef,
                            uint8_t* __restrict__ kind, unsigned long long* __restrict__ keys) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m2;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e >= m) {
      keys[2 * e] = ~0ull;
      keys[2 * e + 1] = ~0ull;
      continue;
    }
    const int2 ij = edges[e];
    const int32_t ci = lab[ij.x], cj = lab[ij.y];
    double* srow = S + e * ld;
    if (ci == cj) {
      kind[e] = K_INERT;
      coef[e] = 0.0;
      for (int k = 0; k < ld; ++k) srow[k] = 0.0;
      keys[2 * e] = ~0ull;
      keys[2 * e + 1] = ~0ull;
      continue;
    }
    const double* xi = X + (int64_t)ij.x * d;
    const double* xj = X + (int64_t)ij.y * d;
    double ss = 0.0;
    for (int k = 0; k < d; ++k) {
      const double dl = xi[k] - xj[k];
      ss += dl * dl;
    }
    const double nd = sqrt(ss);
    const double inv = 1.0 / nd;
    for (int k = 0; k < ld; ++k) srow[k] = (k < d) ? (xi[k] - xj[k]) * inv : 0.0;
    kind[e] = K_OUT;
    coef[e] = gamma * w[e] * inv;
    keys[2 * e] = ((unsigned long long)(unsigned)ci << 32) | (unsigned long long)e;
    keys[2 * e + 1] = ((unsigned long long)(unsigned)cj << 32) | (unsigned long long)e;
  }
}

// cluster CSR from the sorted incidence keys (K+1 offsets, entries {edge, other cluster})
__global__ void k_vjp_ccsr(const unsigned long long* __restrict__ keys, int64_t nk,
                           const int2* __restrict__ edges, const int32_t* __restrict__ lab,
                           int64_t K, int64_t* __restrict__ coff, int2* __restrict__ cinc) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nk;
       p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[p];
    if (key == ~0ull) continue;
    const unsigned cl = (unsigned)(key >> 32);
    const int e = (int)(key & 0xffffffffull);
    const int2 ij = edges[e];
    const int32_t ci = lab[ij.x], cj = lab[ij.y];
    cinc[p] = make_int2(e, (int)((unsigned)ci == cl ? cj : ci));
    if (p == 0 || (unsigned)(keys[p - 1] >> 32) != cl) coff[cl] = p;
  }
}

// offsets of clusters with no boundary edge: fill from the right (run once, 1 thread)
__global__ void k_vjp_fix_coff(int64_t* coff, int64_t K, int64_t nvalid) {
  coff[K] = nvalid;
  for (int64_t c = K - 1; c >= 0; --c)
    if (coff[c] < 0) coff[c] = coff[c + 1];
}

// b_c = - sum_{i in c} G_i (the CG init negates: R = -b_neg = Q^T G), D_c = |c|,
// Minv_c = 1/(|c| + sum_l c_l (d-1)/d)
template <int L, int CH>
__global__ void k_vjp_rhs(const double* __restrict__ G, int d, int ld,
                          const unsigned long long* __restrict__ nkeys,
                          const int64_t* __restrict__ cstart, const int64_t* __restrict__ coff,
                          const int2* __restrict__ cinc, const double* __restrict__ coef,
                          int64_t K, double* __restrict__ bneg, double* __restrict__ Dg,
                          double* __restrict__ Minv) {
  const int lane = threadIdx.x % L;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / L;
  const double tr = (double)(d - 1) / (double)d;
  for (int64_t cl = g0; cl < K; cl += ng) {
    for (int c = 0; c < CH; ++c) {
      const int q = c * L + lane;
      if (4 * q >= ld) break;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int64_t p = cstart[cl]; p < cstart[cl + 1]; ++p) {
        const int64_t i = (int64_t)(nkeys[p] & 0xffffffffull);
        const double* g = G + i * d;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4 * q + k < d) acc[k] += g[4 * q + k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) bneg[cl * ld + 4 * q + k] = -acc[k];
    }
    if (lane == 0) {
      const double size = (double)(cstart[cl + 1] - cstart[cl]);
      double diag = size;
      for (int64_t t = coff[cl]; t < coff[cl + 1]; ++t) diag += coef[cinc[t].x] * tr;
      Dg[cl] = size;
      Minv[cl] = 1.0 / diag;
    }
  }
}

// dA_i += lambda_c(i) (first gamma overwrites), dw_l += -gamma s_l.(lambda_ci - lambda_cj)
__global__ void k_vjp_scatter_a(const double* __restrict__ lam, const int32_t* __restrict__ lab,
                                int64_t n, int d, int ld, double* __restrict__ dA, int first) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * d;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / d;
    const int k = (int)(q - i * d);
    const double v = lam[(int64_t)lab[i] * ld + k];
    dA[q] = first ? v : dA[q] + v;
  }
}

__global__ void k_vjp_scatter_w(const double* __restrict__ lam, const int32_t* __restrict__ lab,
                                const int2* __restrict__ edges, const uint8_t* __restrict__ kind,
                                const double* __restrict__ S, int64_t m, int d, int ld,
                                double gamma, double* __restrict__ dw, int first) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (kind[e] == K_OUT) {
      const int2 ij = edges[e];
      const double* li = lam + (int64_t)lab[ij.x] * ld;
      const double* lj = lam + (int64_t)lab[ij.y] * ld;
      const double* s = S + e * ld;
      double dot = 0.0;
      for (int k = 0; k < d; ++k) dot += s[k] * (li[k] - lj[k]);
      v = -gamma * dot;
    }
    dw[e] = first ? v : dw[e] + v;
  }
}

// rneg = bneg + H lambda, the negated residual of H lambda = -bneg (float64),
// and ||rneg||^2 -> ctl->dots[0]. H = M (x) I + sum_{l in N} c_l B_l^T (I - s_l s_l^T) B_l
// on the cluster graph: the operator of k_cg_matvec applied to lambda itself.
template <int L, int CH>
__global__ void __launch_bounds__(256)
k_vjp_residual(const double* __restrict__ lam, const double* __restrict__ bneg,
               const double* __restrict__ Dg, const double* __restrict__ S,
               const double* __restrict__ coef, const int64_t* __restrict__ coff,
               const int2* __restrict__ cinc, int64_t K, int ld, double* __restrict__ rneg,
               double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / L;
  double acc1[1] = {0.0};
  for (int64_t i = g0; i < K; i += ng) {
    double li[CH][4], h[CH][4];
    row_load<L, CH>(lam + i * ld, ld, lane, li);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) h[c][k] = 0.0;
    for (int64_t t = coff[i]; t < coff[i + 1]; ++t) {
      const int2 eo = cinc[t];
      double v[CH][4], sl[CH][4];
      row_load<L, CH>(lam + (int64_t)eo.y * ld, ld, lane, v);
      row_load<L, CH>(S + (int64_t)eo.x * ld, ld, lane, sl);
      double dot = 0.0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          v[c][k] = li[c][k] - v[c][k];
          dot += sl[c][k] * v[c][k];
        }
      dot = group_sum<L>(dot, mask);
      const double a = coef[eo.x];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) h[c][k] += a * (v[c][k] - dot * sl[c][k]);
    }
    double b4[CH][4];
    row_load<L, CH>(bneg + i * ld, ld, lane, b4);
    const double di = Dg[i];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        h[c][k] = b4[c][k] + (di * li[c][k] + h[c][k]);
        acc1[0] += h[c][k] * h[c][k];
      }
    row_store<L, CH>(rneg + i * ld, ld, lane, h);
  }
  double tot[1];
  if (grid_reduce<1>(acc1, partials, &ctl->counter[C_TRIAL], tot) && threadIdx.x == 0)
    ctl->dots[0] = tot[0];
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t count) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    b[q] = (float)a[q];
}

// lambda += delta (float correction into the float64 iterate)
__global__ void k_add_f2d(double* __restrict__ lam, const float* __restrict__ dlt, int64_t count) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    lam[q] += (double)dlt[q];
}

// ---------------------------------------------------------------- host engine
template <int L, int CH>
static int run_vjp(Ctx* c, const double* A, int64_t n, int d, const int2* edges, const double* w,
                   int64_t m, const double* gammas, int T, const double* X, const double* dLdX,
                   double* dLdA, double* dLdw, cudaStream_t s) {
  (void)A;
  const int ld = (int)round_up(d, 4);
  const int threads = 256;
  const int maxb = c->num_sms * 4;
  auto nb = [&](int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, maxb));
  };
  const int gpb = threads / L;
  const int64_t n2 = pow2_at_least(std::max<int64_t>(n, 2));
  const int64_t m2 = pow2_at_least(std::max<int64_t>(m, 1));
  void* p;
  CCM_TRY(ws_get(c, S_P0, (size_t)n2 * 8, &p));
  unsigned long long* nkeys = (unsigned long long*)p;
  CCM_TRY(ws_get(c, S_P1, (size_t)2 * m2 * 8, &p));
  unsigned long long* ekeys = (unsigned long long*)p;
  CCM_TRY(ws_get(c, S_Q, (size_t)n * 4, &p));
  int32_t* lab = (int32_t*)p;
  CCM_TRY(ws_get(c, S_MINV, (size_t)(n + 1) * 8 * 2, &p));
  int64_t* cstart = (int64_t*)p;
  int64_t* coff = cstart + (n + 1);
  CCM_TRY(ws_get(c, S_CSR_INC, (size_t)std::max<int64_t>(2 * m, 1) * 8, &p));
  int2* cinc = (int2*)p;
  CCM_TRY(ws_get(c, S_YH, (size_t)std::max<int64_t>(m, 1) * ld * 8, &p));
  double* S = (double*)p;
  CCM_TRY(ws_get(c, S_ALPHA, (size_t)std::max<int64_t>(m, 1) * 8, &p));
  double* coef = (double*)p;
  CCM_TRY(ws_get(c, S_KIND, (size_t)std::max<int64_t>(m, 1), &p));
  uint8_t* kind = (uint8_t*)p;
  CCM_TRY(ws_get(c, S_AP, (size_t)n * ld * 8, &p));
  double* bneg = (double*)p;
  CCM_TRY(ws_get(c, S_DX, (size_t)n * ld * 8, &p));
  double* lam = (double*)p;
  CCM_TRY(ws_get(c, S_G, (size_t)n * ld * 8, &p));
  double* Qv = (double*)p;  // negated residual of the float64 system
  CCM_TRY(ws_get(c, S_U, (size_t)n * 8 * 2, &p));
  double* Dg = (double*)p;
  double* Minv = Dg + n;
  CCM_TRY(ws_get(c, S_PART, (size_t)kMaxPartBlocksPerSm * c->num_sms * 4 * 8, &p));
  double* part = (double*)p;
  // float32 copies for the correction solves: 5 vectors of n x ld, Minv and D
  // (n each), yhat rows (m x ld), c_l (m), packed incidence coefficients (2 m2)
  const size_t f_vec = (size_t)round_up((int64_t)5 * n * ld + 2 * n, 64) * 4;
  const size_t f_sy = (size_t)round_up(std::max<int64_t>(m, 1) * ld, 64) * 4;
  const size_t f_cf = (size_t)round_up(std::max<int64_t>(m, 1), 64) * 4;
  CCM_TRY(ws_get(c, S_VJPF, f_vec + f_sy + f_cf + (size_t)2 * m2 * sizeof(IncMeta<float>), &p));
  float* vf = (float*)p;
  float* Syf = (float*)((char*)p + f_vec);
  float* coeff = (float*)((char*)p + f_vec + f_sy);
  IncMeta<float>* metaf = (IncMeta<float>*)((char*)p + f_vec + f_sy + f_cf);
  CCM_TRY(ws_get(c, S_CTRL, sizeof(Ctl), &p));
  Ctl* ctl = (Ctl*)p;
  void* hp;
  CCM_TRY(host_scalars(c, sizeof(Ctl) + 64, &hp));
  Ctl* hc = (Ctl*)hp;
  CCM_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));

  for (int t = 0; t < T; ++t) {
    const double gamma = gammas[t];
    const double* Xt = X + (int64_t)t * n * d;
    const double* Gt = dLdX + (int64_t)t * n * d;
    int32_t K = 0;
    CCM_TRY(labels_device(c, Xt, d, n, d, edges, m, lab, &K, s));
    // cluster member lists
    k_vjp_node_keys<<<nb(n2), threads, 0, s>>>(lab, n, n2, nkeys);
    CCM_COUNT(c);
    CCM_TRY(bitonic_sort(c, nkeys, n2, s));
    k_vjp_cstart<<<nb(n), threads, 0, s>>>(nkeys, n, K, cstart);
    CCM_COUNT(c);
    // boundary edges and the cluster CSR
    CCM_CUDA(cudaMemsetAsync(coff, 0xff, (size_t)(K + 1) * 8, s));
    k_vjp_edges<<<nb(m2), threads, 0, s>>>(Xt, d, ld, edges, w, gamma, lab, m, m2, S, coef, kind,
                                            ekeys);
    CCM_COUNT(c);
    CCM_TRY(bitonic_sort(c, ekeys, 2 * m2, s));
    k_vjp_ccsr<<<nb(2 * m2), threads, 0, s>>>(ekeys, 2 * m2, edges, lab, K, coff, cinc);
    CCM_COUNT(c);
    // number of valid incidence keys = 2 |N|: count them from the keys (sorted, invalid last)
    int64_t nvalid = 0;
    {
      // binary search on the host would need the keys; count with a reduction instead
      std::vector<unsigned long long> tail(1);
      int64_t lo = 0, hi = 2 * m2;  // first invalid position by bisection with small copies
      while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        CCM_CUDA(cudaMemcpyAsync(tail.data(), ekeys + mid, 8, cudaMemcpyDeviceToHost, s));
        CCM_CUDA(cudaStreamSynchronize(s));
        if (tail[0] == ~0ull) hi = mid;
        else lo = mid + 1;
      }
      nvalid = lo;
    }
    k_vjp_fix_coff<<<1, 1, 0, s>>>(coff, K, nvalid);
    CCM_COUNT(c);
    k_vjp_rhs<L, CH><<<(int)std::max<int64_t>(1, std::min<int64_t>((K + gpb - 1) / gpb, maxb)),
                       threads, 0, s>>>(Gt, d, ld, nkeys, cstart, coff, cinc, coef, K, bneg, Dg,
                                        Minv);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    // H lambda = Q^T G by mixed-precision iterative refinement: the residual
    // r = Q^T G - H lambda in float64 (k_vjp_residual), the correction H delta = r
    // by float32 CG with the operator kernels (relative tolerance 1e-3, at most 400
    // iterations), lambda += delta in float64; stop at ||r|| <= 1e-11 ||Q^T G||, when a
    // correction no longer halves ||r||, or after 16 corrections.
    const int b_node = (int)std::max<int64_t>(1, std::min<int64_t>((K + gpb - 1) / gpb, maxb));
    const int b_elem = nb((int64_t)K * ld);
    const int b_quad = nb(((int64_t)K * ld + 3) / 4);
    const int64_t kl = (int64_t)K * ld;
    float* Rf = vf;
    float* Pf = Rf + kl;
    float* Sf = Pf + kl;
    float* Wf = Sf + kl;
    float* Df = Wf + kl;
    float* Minvf = Df + kl;
    float* Dgf = Minvf + K;
    k_d2f<<<nb(m * ld), threads, 0, s>>>(S, Syf, m * ld);
    k_d2f<<<nb(m), threads, 0, s>>>(coef, coeff, m);
    k_d2f<<<nb(K), threads, 0, s>>>(Minv, Minvf, K);
    k_d2f<<<nb(K), threads, 0, s>>>(Dg, Dgf, K);
    CCM_COUNT(c); CCM_COUNT(c); CCM_COUNT(c); CCM_COUNT(c);
    CCM_CUDA(cudaMemsetAsync(lam, 0, (size_t)kl * 8, s));
    double r2_0 = -1.0, r2_prev = 0.0;
    for (int ref = 0; ref <= 16; ++ref) {
      k_vjp_residual<L, CH><<<b_node, threads, 0, s>>>(lam, bneg, Dg, S, coef, coff, cinc, K, ld,
                                                       Qv, part, ctl);
      CCM_COUNT(c);
      CCM_CUDA(cudaGetLastError());
      CCM_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
      CCM_CUDA(cudaStreamSynchronize(s));
      const double r2 = hc->dots[0];
      if (r2_0 < 0.0) r2_0 = r2;
      if (!(r2 > 1e-22 * r2_0) || ref == 16 || (ref > 0 && !(r2 < 0.25 * r2_prev))) break;
      r2_prev = r2;
      k_cg_init<float><<<b_elem, threads, 0, s>>>(Qv, Minvf, Rf, Df, K, ld, 1e-3, 400, cinc,
                                                  kind, coeff, metaf, nvalid, part, ctl);
      CCM_COUNT(c);
      CCM_CUDA(cudaGetLastError());
      const int CHUNK = 16;
      for (int chunk = 0; chunk * CHUNK < 400; ++chunk) {
        for (int k = 0; k < CHUNK; ++k) {
          CCM_TRY(launch_matvec_reg<L, CH, float>(c, Rf, Minvf, Dgf, Wf, Syf, metaf, coff, cinc,
                                                  1.0, K, ld, part, ctl, s));
          k_cg_update<float><<<b_quad, threads, 0, s>>>(Df, Pf, Sf, Rf, Wf, Minvf, K, ld, part,
                                                        ctl);
          CCM_COUNT(c);
        }
        CCM_CUDA(cudaGetLastError());
        CCM_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CCM_CUDA(cudaStreamSynchronize(s));
        if (!hc->cg.active) break;
      }
      k_add_f2d<<<b_elem, threads, 0, s>>>(lam, Df, kl);
      CCM_COUNT(c);
    }
    k_vjp_scatter_a<<<nb(n * d), threads, 0, s>>>(lam, lab, n, d, ld, dLdA, t == 0);
    CCM_COUNT(c);
    k_vjp_scatter_w<<<nb(m), threads, 0, s>>>(lam, lab, edges, kind, S, m, d, ld, gamma, dLdw,
                                              t == 0);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
  }
  CCM_CUDA(cudaStreamSynchronize(s));
  return CCM_OK;
}

static int dispatch_vjp(Ctx* c, const double* A, int64_t n, int d, const int2* edges,
                        const double* w, int64_t m, const double* gammas, int T, const double* X,
                        const double* G, double* dA, double* dw, cudaStream_t s) {
  const int nq = (int)(round_up(d, 4) / 4);
#define CCM_VJP(LL, CC) return run_vjp<LL, CC>(c, A, n, d, edges, w, m, gammas, T, X, G, dA, dw, s)
  if (nq <= 1) CCM_VJP(1, 1);
  if (nq <= 2) CCM_VJP(2, 1);
  if (nq <= 4) CCM_VJP(4, 1);
  if (nq <= 8) CCM_VJP(8, 1);
  if (nq <= 16) CCM_VJP(16, 1);
  if (nq <= 32) CCM_VJP(32, 1);
  if (nq <= 64) CCM_VJP(32, 2);
  if (nq <= 128) CCM_VJP(32, 4);
  if (nq <= 256) CCM_VJP(32, 8);
#undef CCM_VJP
  set_error("ccm_path_vjp: d = %d exceeds the maximum %d", d, ccm_max_dim());
  return CCM_ERR_UNSUPPORTED;
}

}  // namespace ccm

using namespace ccm;

extern "C" int ccm_path_vjp(ccm_ctx* x, const double* A, int64_t n, int32_t d,
                            const int32_t* edges, const double* w, int64_t m,
                            const double* gammas, int32_t T, const double* X, const double* U,
                            const double* dLdX, double* dLdA, double* dLdw,
                            ccm_stream_t stream) {
  (void)U;
  Ctx* c = ctx_of(x);
  if (!c || !A || !X || !dLdX || !dLdA || !gammas || n < 1 || d < 1 || m < 0 || T < 1 ||
      (m > 0 && (!edges || !w || !dLdw)) || n > INT32_MAX || m > INT32_MAX / 2) {
    set_error("ccm_path_vjp: invalid argument");
    return CCM_ERR_INVALID_ARG;
  }
  if (d > ccm_max_dim()) {
    set_error("ccm_path_vjp: d = %d exceeds the maximum %d", d, ccm_max_dim());
    return CCM_ERR_UNSUPPORTED;
  }
  for (int t = 0; t < T; ++t)
    if (!(gammas[t] >= 0) || !std::isfinite(gammas[t])) {
      set_error("ccm_path_vjp: gammas must be finite and >= 0");
      return CCM_ERR_INVALID_ARG;
    }
  if (((uintptr_t)edges) % 8) {
    set_error("ccm_path_vjp: edges must be 8-byte aligned");
    return CCM_ERR_INVALID_ARG;
  }
  CCM_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  CCM_TRY(check_edges(c, (const int2*)edges, m, n, w, s));
  return dispatch_vjp(c, A, n, d, (const int2*)edges, w, m, gammas, T, X, dLdX, dLdA, dLdw, s);
}
