// ccm_solve_path_admm: model CCM (q = 2) along a gamma path by ADMM, the
// second of the paper's three solvers (Sec. 1, Table 3), on the same device
// operators as the SSNAL engine.
//
// Splitting z_l = (BX)_l with multiplier U and a fixed penalty sigma:
//   X <- (I + sigma B^T B)^{-1} (A + B^T (sigma Z - U))
//   Z <- prox_{p/sigma}(B X + U / sigma),  p(Z) = sum_l gamma w_l ||z_l||
//   U <- U + sigma (B X - Z)
// The X-step is solved as a correction: with Ut = U + sigma (B X - Z) the
// residual of the X-system at the current X is -(X - A + B^T Ut), the node
// gradient of Ut (k_node_grad / k_node_grad_ring); CG on V = I + sigma B^T B
// (the Newton-CG operator with every edge inside the ball, P_l = I) reduces it
// by a factor 100 and X takes the correction. The Z- and U-steps are one edge
// pass. Every `kCheck` iterations the KKT residuals and the relative gap (the
// stopping rule of ccm_solve_path) are evaluated at (X, U).
#include <algorithm>
#include <cmath>

#include "ccm_internal.cuh"
#include "ring_kernels.cuh"
#include "solve_common.cuh"
#include "ssnal_kernels.cuh"

namespace ccm {

static constexpr int kCheck = 10;  // iterations between KKT evaluations

// Ut_l = u_l + sigma (x_i - x_j - z_l)
template <int LANES, int CH>
__global__ void __launch_bounds__(256)
k_admm_resid(const double* __restrict__ X, const double* __restrict__ Z,
             const double* __restrict__ U, const int2* __restrict__ edges, double sigma,
             double* __restrict__ Ut, int64_t m, int ld) {
  const int lane = threadIdx.x % LANES;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = edges[e];
    double xi[CH][4], xj[CH][4], zu[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, xi);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, xj);
    row_load<LANES, CH>(Z + e * ld, ld, lane, zu);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) xi[c][k] = (xi[c][k] - xj[c][k]) - zu[c][k];
    row_load<LANES, CH>(U + e * ld, ld, lane, zu);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) zu[c][k] = fma(sigma, xi[c][k], zu[c][k]);
    row_store<LANES, CH>(Ut + e * ld, ld, lane, zu);
  }
}

// Z- and U-steps: v = bx + u / sigma, z = max(0, 1 - (r/sigma)/||v||) v,
// u <- u + sigma (bx - z); in place.
template <int LANES, int CH>
__global__ void __launch_bounds__(256)
k_admm_zu(const double* __restrict__ X, double* __restrict__ Z, double* __restrict__ U,
          const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
          double sigma, int64_t m, int ld) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const double isg = 1.0 / sigma;
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = edges[e];
    const double t = gamma * w[e] * isg;
    double bx[CH][4], v[CH][4], u[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, bx);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, v);
    row_load<LANES, CH>(U + e * ld, ld, lane, u);
    double sv = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bx[c][k] -= v[c][k];
        v[c][k] = fma(isg, u[c][k], bx[c][k]);
        sv = fma(v[c][k], v[c][k], sv);
      }
    sv = group_sum<LANES>(sv, mask);
    const double nv = sqrt(sv);
    const double shrink = nv > t ? 1.0 - t / nv : 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[c][k] *= shrink;                                   // z
        u[c][k] = fma(sigma, bx[c][k] - v[c][k], u[c][k]);   // u + sigma (bx - z)
      }
    row_store<LANES, CH>(Z + e * ld, ld, lane, v);
    row_store<LANES, CH>(U + e * ld, ld, lane, u);
  }
}

// Z = B X (start of a cold path)
template <int LANES, int CH>
__global__ void __launch_bounds__(256)
k_admm_bx(const double* __restrict__ X, const int2* __restrict__ edges, double* __restrict__ Z,
          int64_t m, int ld) {
  const int lane = threadIdx.x % LANES;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = edges[e];
    double a[CH][4], b[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, a);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, b);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) a[c][k] -= b[c][k];
    row_store<LANES, CH>(Z + e * ld, ld, lane, a);
  }
}

// Primal residual ||BX - prox_p(BX + U)||^2 and sum_l r_l ||(BX)_l|| at (X, U).
template <int LANES, int CH>
__global__ void __launch_bounds__(256)
k_admm_kkt_edge(const double* __restrict__ X, const double* __restrict__ U,
                const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
                int64_t m, int ld, double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  double acc[2] = {0.0, 0.0};
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = edges[e];
    const double r = gamma * w[e];
    double bx[CH][4], v[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, bx);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, v);
    double sb = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bx[c][k] -= v[c][k];
        sb = fma(bx[c][k], bx[c][k], sb);
      }
    row_load<LANES, CH>(U + e * ld, ld, lane, v);
    double sv = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[c][k] += bx[c][k];
        sv = fma(v[c][k], v[c][k], sv);
      }
    sb = group_sum<LANES>(sb, mask);
    sv = group_sum<LANES>(sv, mask);
    const double nv = sqrt(sv);
    const double shrink = nv > r ? 1.0 - r / nv : 0.0;
    double sres = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double res = fma(-shrink, v[c][k], bx[c][k]);
        sres = fma(res, res, sres);
      }
    acc[0] += sres;
    if (lane == 0) acc[1] += r * sqrt(sb);
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_KKT_E], tot) && threadIdx.x == 0) {
    ctl->kkt[0] = tot[0];
    ctl->kkt[1] = tot[1];
  }
}

// every edge inside the ball: P_l = I in the X-step operator
template <typename Tc>
__global__ void k_admm_inside(uint8_t* __restrict__ kind, Tc* __restrict__ alpha, int64_t m) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    kind[e] = K_IN;
    alpha[e] = (Tc)1;
  }
}

template <int L, int CH, typename Tc>
struct AdmmEngine {
  static int run(Ctx* c, const SolveArgs& a, cudaStream_t s) {
    const int64_t n = a.n, m = a.m;
    const int d = a.d;
    const int ld = (int)round_up(d, 4);
    const int64_t nl = n * ld, ml = m * ld;
    const int threads = 256;
    const int gpb = threads / L;
    const int maxb = c->num_sms * 4;
    auto nb = [&](int64_t work) {
      return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, maxb));
    };
    const int b_edge = (int)std::max<int64_t>(1, std::min<int64_t>((m + gpb - 1) / gpb, maxb));
    const int b_elem = nb(nl);
    const int b_quad = nb((nl + 3) / 4);

    void* p;
    auto get = [&](Slot sl, size_t bytes, void** out) { return ws_get(c, sl, bytes, out); };
    CCM_TRY(get(S_AP, nl * 8, &p)); double* Ap = (double*)p;
    CCM_TRY(get(S_X0, nl * 8, &p)); double* Xa = (double*)p;
    CCM_TRY(get(S_X1, nl * 8, &p)); double* Xb = (double*)p;
    CCM_TRY(get(S_G, nl * 8, &p)); double* G = (double*)p;
    CCM_TRY(get(S_DX, nl * sizeof(Tc), &p)); Tc* Dx = (Tc*)p;
    CCM_TRY(get(S_R, nl * sizeof(Tc), &p)); Tc* R = (Tc*)p;
    CCM_TRY(get(S_P0, nl * sizeof(Tc), &p)); Tc* P = (Tc*)p;
    CCM_TRY(get(S_P1, nl * sizeof(Tc), &p)); Tc* Sv = (Tc*)p;
    CCM_TRY(get(S_Q, nl * sizeof(Tc), &p)); Tc* W = (Tc*)p;
    CCM_TRY(get(S_MINV, n * sizeof(Tc), &p)); Tc* Minv = (Tc*)p;
    CCM_TRY(get(S_U, std::max<int64_t>(ml, 1) * 8, &p)); double* U = (double*)p;
    CCM_TRY(get(S_UT, std::max<int64_t>(ml, 1) * 8, &p)); double* Z = (double*)p;
    CCM_TRY(get(S_ADMM, std::max<int64_t>(ml, 1) * 8, &p)); double* Ut = (double*)p;
    CCM_TRY(get(S_ALPHA, std::max<int64_t>(m, 1) * sizeof(Tc), &p)); Tc* alpha = (Tc*)p;
    CCM_TRY(get(S_KIND, std::max<int64_t>(m, 1), &p)); uint8_t* kind = (uint8_t*)p;
    CCM_TRY(get(S_META, std::max<int64_t>(2 * m, 1) * sizeof(IncMeta<Tc>), &p));
    IncMeta<Tc>* meta = (IncMeta<Tc>*)p;
    CCM_TRY(get(S_PART, (size_t)kMaxPartBlocksPerSm * c->num_sms * 4 * 8, &p));
    double* part = (double*)p;
    CCM_TRY(get(S_CTRL, sizeof(Ctl), &p)); Ctl* ctl = (Ctl*)p;
    void* hp;
    CCM_TRY(host_scalars(c, sizeof(Ctl) + 64, &hp));
    Ctl* hc = (Ctl*)hp;
    const int2* edges = (const int2*)a.edges;

    int64_t* off;
    int2* inc;
    CCM_TRY(build_csr(c, edges, m, n, &off, &inc, s));
    RingPlan rp;
    CCM_TRY(ring_plan<Tc>(c, L, ld, off, n, rp, s));
    CCM_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    k_pad_rows<<<b_elem, threads, 0, s>>>(a.A, Ap, n, d, ld);
    CCM_COUNT(c);
    k_pad_rows<<<b_elem, threads, 0, s>>>(a.X0 ? a.X0 : a.A, Xa, n, d, ld);
    CCM_COUNT(c);
    CCM_CUDA(cudaMemsetAsync(Xb, 0, nl * 8, s));
    if (m > 0) {
      if (a.U0) {
        k_pad_rows<<<nb(ml), threads, 0, s>>>(a.U0, U, m, d, ld);
        CCM_COUNT(c);
      } else {
        CCM_CUDA(cudaMemsetAsync(U, 0, ml * 8, s));
      }
      k_admm_bx<L, CH><<<b_edge, threads, 0, s>>>(Xa, edges, Z, m, ld);
      CCM_COUNT(c);
      k_admm_inside<Tc><<<nb(m), threads, 0, s>>>(kind, alpha, m);
      CCM_COUNT(c);
    }
    k_sumsq<<<b_elem, threads, 0, s>>>(Ap, nl, part, ctl);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    auto readback = [&]() -> int {
      CCM_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
      CCM_CUDA(cudaStreamSynchronize(s));
      return CCM_OK;
    };
    CCM_TRY(readback());
    const double scale = 1.0 + std::sqrt(hc->dots[1]);
    const double sigma = a.opt.sigma0;
    const int max_it = a.opt.max_outer * a.opt.max_newton;
    const int CHUNK = 8;
    double* X = Xa;
    double* Xt = Xb;
    int any_fail = 0;
    for (int t = 0; t < a.T; ++t) {
      const double gamma = a.gammas[t];
      ccm_stats st = {};
      bool converged = false;
      for (int it = 1; it <= max_it; ++it) {
        // X-step as a correction: residual -(X - A + B^T (U + sigma (BX - Z)))
        if (m > 0) {
          k_admm_resid<L, CH><<<b_edge, threads, 0, s>>>(X, Z, U, edges, sigma, Ut, m, ld);
          CCM_COUNT(c);
        }
        CCM_TRY(launch_node_grad<L, CH, Tc>(c, X, Ap, Ut, off, inc, alpha, kind, sigma, d, G, Minv,
                                            rp, n, ld, part, ctl, s));
        k_cg_init<Tc><<<b_elem, threads, 0, s>>>(G, Minv, R, Dx, n, ld, 1e-2, a.opt.max_cg, inc,
                                                 kind, alpha, meta, 2 * m, part, ctl);
        CCM_COUNT(c);
        CCM_CUDA(cudaGetLastError());
        for (int chunk = 0; chunk * CHUNK < a.opt.max_cg; ++chunk) {
          for (int k = 0; k < CHUNK; ++k) {
            CCM_TRY(launch_matvec<L, CH, Tc>(c, R, Minv, nullptr, W, (const Tc*)nullptr, meta, off,
                                              inc, rp, sigma, n, ld, part, ctl, s));
            k_cg_update<Tc><<<b_quad, threads, 0, s>>>(Dx, P, Sv, R, W, Minv, n, ld, part, ctl);
            CCM_COUNT(c);
          }
          CCM_CUDA(cudaGetLastError());
          CCM_TRY(readback());
          if (!hc->cg.active) break;
        }
        st.cg += hc->cg.it;
        k_trial<Tc><<<b_elem, threads, 0, s>>>(X, Dx, G, 1.0, Xt, nl, part, ctl);
        CCM_COUNT(c);
        std::swap(X, Xt);
        if (m > 0) {
          k_admm_zu<L, CH><<<b_edge, threads, 0, s>>>(X, Z, U, edges, a.w, gamma, sigma, m, ld);
          CCM_COUNT(c);
        }
        CCM_CUDA(cudaGetLastError());
        st.outer = it;
        if (it % kCheck != 0 && it != max_it) continue;
        // KKT and gap at (X, U): G = X - A + B^T U, primal residual, objectives
        CCM_TRY(launch_node_grad<L, CH, Tc>(c, X, Ap, U, off, inc, alpha, kind, sigma, d, G, Minv,
                                            rp, n, ld, part, ctl, s));
        if (m > 0) {
          k_admm_kkt_edge<L, CH><<<b_edge, threads, 0, s>>>(X, U, edges, a.w, gamma, m, ld, part,
                                                           ctl);
          CCM_COUNT(c);
        } else {
          CCM_CUDA(cudaMemsetAsync(&ctl->kkt[0], 0, 2 * sizeof(double), s));
        }
        k_kkt_node<<<b_elem, threads, 0, s>>>(X, Ap, G, nl, part, ctl);
        CCM_COUNT(c);
        CCM_CUDA(cudaGetLastError());
        CCM_TRY(readback());
        const double eta_d = std::sqrt(hc->eval[2]) / scale;
        const double eta_p = std::sqrt(hc->kkt[0]) / scale;
        const double fp = hc->eval[1] + hc->kkt[1];
        const double fd = hc->kkt[2] - 0.5 * hc->kkt[3];
        st.eta_d = eta_d;
        st.eta_p = eta_p;
        st.kkt = std::max(eta_d, eta_p);
        st.f_p = fp;
        st.f_d = fd;
        st.gap = std::fabs(fp - fd) / (1.0 + std::fabs(fp) + std::fabs(fd));
        if (st.kkt <= a.tol && st.gap <= a.tol) {
          converged = true;
          break;
        }
      }
      st.sigma = sigma;
      st.status = converged ? CCM_OK : CCM_ERR_NOT_CONVERGED;
      if (!converged) any_fail = 1;
      k_unpad_rows<<<nb(n * d), threads, 0, s>>>(X, a.Xout + (int64_t)t * n * d, n, d, ld);
      CCM_COUNT(c);
      if (a.Uout && m > 0) {
        k_unpad_rows<<<nb(m * d), threads, 0, s>>>(U, a.Uout + (int64_t)t * m * d, m, d, ld);
        CCM_COUNT(c);
      }
      CCM_CUDA(cudaGetLastError());
      if (a.stats) a.stats[t] = st;
    }
    return any_fail ? CCM_ERR_NOT_CONVERGED : CCM_OK;
  }
};

// ---------------------------------------------------------------- fast AMA
// The paper's third solver (Sec. 1, Table 3): projected gradient ascent on the
// dual with Nesterov momentum. For dual-feasible U the primal point is
// X(U) = A - B^T U (the minimiser of the Lagrangian in X), and
//   U_k = Pi(Uh + nu B X(Uh)),   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
//   Uh  = U_k + ((t_k - 1) / t_{k+1}) (U_k - U_{k-1}),
// with the step nu = 1 / max_l (deg_i + deg_j) <= 1 / lambda_max(B^T B). The
// momentum restarts (t = 1) when the step U_k - U_{k-1} turns against the
// extrapolation (<Uh_prev - U_k, U_k - U_{k-1}> > 0). KKT and gap at
// (X(U_k), U_k) every kCheck iterations.

// max over edges of deg_i + deg_j -> *out (one block)
__global__ void k_ama_edge_degree(const int64_t* __restrict__ off, const int2* __restrict__ edges,
                                  int64_t m, unsigned long long* __restrict__ out) {
  unsigned long long mx = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 ij = edges[e];
    const unsigned long long dg = (unsigned long long)((off[ij.x + 1] - off[ij.x]) +
                                                       (off[ij.y + 1] - off[ij.y]));
    mx = dg > mx ? dg : mx;
  }
  atomicMax(out, mx);
}

// X = A - G (G = B^T U from the node pull at X := A)
__global__ void k_ama_primal(const double* __restrict__ Ap, const double* __restrict__ G,
                             double* __restrict__ X, int64_t total) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x)
    X[q] = Ap[q] - G[q];
}

// restart test <Uh - U_k, U_k - U_{k-1}> -> ctl->dots[0]
__global__ void __launch_bounds__(256)
k_ama_restart_dot(const double* __restrict__ Uh, const double* __restrict__ Uk,
                  const double* __restrict__ Up, int64_t total, double* partials, Ctl* ctl) {
  double acc[1] = {0.0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma(Uh[q] - Uk[q], Uk[q] - Up[q], acc[0]);
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_TRIAL], tot) && threadIdx.x == 0)
    ctl->dots[0] = tot[0];
}

// Uh = U_k + theta (U_k - U_{k-1})
__global__ void k_ama_momentum(const double* __restrict__ Uk, const double* __restrict__ Up,
                               double theta, double* __restrict__ Uh, int64_t total) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x)
    Uh[q] = fma(theta, Uk[q] - Up[q], Uk[q]);
}

template <int L, int CH, typename Tc>
struct AmaEngine {
  static int run(Ctx* c, const SolveArgs& a, cudaStream_t s) {
    const int64_t n = a.n, m = a.m;
    const int d = a.d;
    const int ld = (int)round_up(d, 4);
    const int64_t nl = n * ld, ml = m * ld;
    const int threads = 256;
    const int gpb = threads / L;
    const int maxb = c->num_sms * 4;
    auto nb = [&](int64_t work) {
      return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, maxb));
    };
    const int b_edge = (int)std::max<int64_t>(1, std::min<int64_t>((m + gpb - 1) / gpb, maxb));
    const int b_elem = nb(nl);

    void* p;
    auto get = [&](Slot sl, size_t bytes, void** out) { return ws_get(c, sl, bytes, out); };
    CCM_TRY(get(S_AP, nl * 8, &p)); double* Ap = (double*)p;
    CCM_TRY(get(S_X0, nl * 8, &p)); double* X = (double*)p;
    CCM_TRY(get(S_G, nl * 8, &p)); double* G = (double*)p;
    CCM_TRY(get(S_MINV, n * sizeof(Tc), &p)); Tc* Minv = (Tc*)p;
    CCM_TRY(get(S_U, std::max<int64_t>(ml, 1) * 8, &p)); double* Ua = (double*)p;
    CCM_TRY(get(S_UT, std::max<int64_t>(ml, 1) * 8, &p)); double* Ub = (double*)p;
    CCM_TRY(get(S_ADMM, std::max<int64_t>(ml, 1) * 8, &p)); double* Uh = (double*)p;
    CCM_TRY(get(S_YH, std::max<int64_t>(ml, 1) * sizeof(Tc), &p)); Tc* Yh = (Tc*)p;
    CCM_TRY(get(S_ALPHA, std::max<int64_t>(m, 1) * sizeof(Tc), &p)); Tc* alpha = (Tc*)p;
    CCM_TRY(get(S_KIND, std::max<int64_t>(m, 1), &p)); uint8_t* kind = (uint8_t*)p;
    CCM_TRY(get(S_PART, (size_t)kMaxPartBlocksPerSm * c->num_sms * 4 * 8, &p));
    double* part = (double*)p;
    CCM_TRY(get(S_CTRL, sizeof(Ctl), &p)); Ctl* ctl = (Ctl*)p;
    CCM_TRY(get(S_SCRATCH5, 64, &p));
    unsigned long long* dmax = (unsigned long long*)p;
    void* hp;
    CCM_TRY(host_scalars(c, sizeof(Ctl) + 64, &hp));
    Ctl* hc = (Ctl*)hp;
    const int2* edges = (const int2*)a.edges;

    int64_t* off;
    int2* inc;
    CCM_TRY(build_csr(c, edges, m, n, &off, &inc, s));
    RingPlan rp;
    CCM_TRY(ring_plan<Tc>(c, L, ld, off, n, rp, s));
    CCM_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    CCM_CUDA(cudaMemsetAsync(dmax, 0, 8, s));
    k_pad_rows<<<b_elem, threads, 0, s>>>(a.A, Ap, n, d, ld);
    CCM_COUNT(c);
    CCM_CUDA(cudaMemsetAsync(Yh, 0, std::max<int64_t>(ml, 1) * sizeof(Tc), s));
    if (m > 0) {
      if (a.U0) {
        k_pad_rows<<<nb(ml), threads, 0, s>>>(a.U0, Ua, m, d, ld);
        CCM_COUNT(c);
      } else {
        CCM_CUDA(cudaMemsetAsync(Ua, 0, ml * 8, s));
      }
      CCM_CUDA(cudaMemsetAsync(Ub, 0, ml * 8, s));
      k_ama_edge_degree<<<nb(m), threads, 0, s>>>(off, edges, m, dmax);
      CCM_COUNT(c);
    }
    k_sumsq<<<b_elem, threads, 0, s>>>(Ap, nl, part, ctl);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    auto readback = [&]() -> int {
      CCM_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
      CCM_CUDA(cudaStreamSynchronize(s));
      return CCM_OK;
    };
    CCM_TRY(readback());
    const double scale = 1.0 + std::sqrt(hc->dots[1]);
    unsigned long long hdmax = 0;
    CCM_CUDA(cudaMemcpy(&hdmax, dmax, 8, cudaMemcpyDeviceToHost));
    const double nu = 1.0 / (double)std::max<unsigned long long>(hdmax, 1);
    const int max_it = a.opt.max_outer * a.opt.max_newton * 10;
    // node pull at X := A: G = B^T U, eval[2] = ||G||^2
    auto pull = [&](const double* Uc) -> int {
      return launch_node_grad<L, CH, Tc>(c, Ap, Ap, Uc, off, inc, alpha, kind, 1.0, d, G, Minv,
                                         rp, n, ld, part, ctl, s);
    };
    double* Uk = Ua;  // current iterate U_k
    double* Up = Ub;  // previous U_{k-1}
    int any_fail = 0;
    for (int t = 0; t < a.T; ++t) {
      const double gamma = a.gammas[t];
      ccm_stats st = {};
      bool converged = false;
      double tk = 1.0;
      if (m > 0) CCM_CUDA(cudaMemcpyAsync(Uh, Uk, ml * 8, cudaMemcpyDeviceToDevice, s));
      for (int it = 1; it <= max_it; ++it) {
        if (m > 0) {
          // U_k+1 = Pi(Uh + nu B X(Uh)) into Up (it becomes the new U_k)
          CCM_TRY(pull(Uh));
          k_ama_primal<<<b_elem, threads, 0, s>>>(Ap, G, X, nl);
          CCM_COUNT(c);
          k_edge_eval<L, CH, Tc><<<b_edge, threads, 0, s>>>(X, Uh, edges, a.w, gamma, nu, Up, Yh,
                                                            alpha, kind, m, ld, part, ctl);
          CCM_COUNT(c);
          std::swap(Uk, Up);
          // momentum with restart
          k_ama_restart_dot<<<nb(ml), threads, 0, s>>>(Uh, Uk, Up, ml, part, ctl);
          CCM_COUNT(c);
          CCM_TRY(readback());
          double theta = 0.0;
          if (hc->dots[0] > 0.0) {
            tk = 1.0;  // restart
          } else {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * tk * tk));
            theta = (tk - 1.0) / tn;
            tk = tn;
          }
          k_ama_momentum<<<nb(ml), threads, 0, s>>>(Uk, Up, theta, Uh, ml);
          CCM_COUNT(c);
          CCM_CUDA(cudaGetLastError());
        }
        st.outer = it;
        if (it % kCheck != 0 && it != max_it && m > 0) continue;
        // KKT and gap at (X(U_k), U_k)
        CCM_TRY(pull(Uk));
        k_ama_primal<<<b_elem, threads, 0, s>>>(Ap, G, X, nl);
        CCM_COUNT(c);
        if (m > 0) {
          k_admm_kkt_edge<L, CH><<<b_edge, threads, 0, s>>>(X, Uk, edges, a.w, gamma, m, ld, part,
                                                           ctl);
          CCM_COUNT(c);
        } else {
          CCM_CUDA(cudaMemsetAsync(&ctl->kkt[0], 0, 2 * sizeof(double), s));
        }
        k_kkt_node<<<b_elem, threads, 0, s>>>(Ap, Ap, G, nl, part, ctl);  // B^T U = G
        CCM_COUNT(c);
        CCM_CUDA(cudaGetLastError());
        CCM_TRY(readback());
        const double eta_p = std::sqrt(hc->kkt[0]) / scale;
        const double fp = 0.5 * hc->eval[2] + hc->kkt[1];
        const double fd = hc->kkt[2] - 0.5 * hc->kkt[3];
        st.eta_d = 0.0;  // X = A - B^T U exactly
        st.eta_p = eta_p;
        st.kkt = eta_p;
        st.f_p = fp;
        st.f_d = fd;
        st.gap = std::fabs(fp - fd) / (1.0 + std::fabs(fp) + std::fabs(fd));
        if (st.kkt <= a.tol && st.gap <= a.tol) {
          converged = true;
          break;
        }
      }
      st.sigma = nu;
      st.status = converged ? CCM_OK : CCM_ERR_NOT_CONVERGED;
      if (!converged) any_fail = 1;
      k_unpad_rows<<<nb(n * d), threads, 0, s>>>(X, a.Xout + (int64_t)t * n * d, n, d, ld);
      CCM_COUNT(c);
      if (a.Uout && m > 0) {
        k_unpad_rows<<<nb(m * d), threads, 0, s>>>(Uk, a.Uout + (int64_t)t * m * d, m, d, ld);
        CCM_COUNT(c);
      }
      CCM_CUDA(cudaGetLastError());
      if (a.stats) a.stats[t] = st;
    }
    return any_fail ? CCM_ERR_NOT_CONVERGED : CCM_OK;
  }
};

template <typename Tc>
static int run_ama(Ctx* c, const SolveArgs& a, cudaStream_t s) {
  const int nq = (int)(round_up(a.d, 4) / 4);
  if (nq <= 1) return AmaEngine<1, 1, Tc>::run(c, a, s);
  if (nq <= 2) return AmaEngine<2, 1, Tc>::run(c, a, s);
  if (nq <= 4) return AmaEngine<4, 1, Tc>::run(c, a, s);
  if (nq <= 8) return AmaEngine<8, 1, Tc>::run(c, a, s);
  if (nq <= 16) return AmaEngine<16, 1, Tc>::run(c, a, s);
  if (nq <= 32) return AmaEngine<32, 1, Tc>::run(c, a, s);
  if (nq <= 64) return AmaEngine<32, 2, Tc>::run(c, a, s);
  if (nq <= 96) return AmaEngine<32, 3, Tc>::run(c, a, s);
  if (nq <= 128) return AmaEngine<32, 4, Tc>::run(c, a, s);
  if (nq <= 160) return AmaEngine<32, 5, Tc>::run(c, a, s);
  if (nq <= 192) return AmaEngine<32, 6, Tc>::run(c, a, s);
  if (nq <= 224) return AmaEngine<32, 7, Tc>::run(c, a, s);
  if (nq <= 256) return AmaEngine<32, 8, Tc>::run(c, a, s);
  set_error("d = %d exceeds the compiled maximum %d", a.d, ccm_max_dim());
  return CCM_ERR_UNSUPPORTED;
}

template <typename Tc>
static int run_admm(Ctx* c, const SolveArgs& a, cudaStream_t s) {
  const int nq = (int)(round_up(a.d, 4) / 4);
  if (nq <= 1) return AdmmEngine<1, 1, Tc>::run(c, a, s);
  if (nq <= 2) return AdmmEngine<2, 1, Tc>::run(c, a, s);
  if (nq <= 4) return AdmmEngine<4, 1, Tc>::run(c, a, s);
  if (nq <= 8) return AdmmEngine<8, 1, Tc>::run(c, a, s);
  if (nq <= 16) return AdmmEngine<16, 1, Tc>::run(c, a, s);
  if (nq <= 32) return AdmmEngine<32, 1, Tc>::run(c, a, s);
  if (nq <= 64) return AdmmEngine<32, 2, Tc>::run(c, a, s);
  if (nq <= 96) return AdmmEngine<32, 3, Tc>::run(c, a, s);
  if (nq <= 128) return AdmmEngine<32, 4, Tc>::run(c, a, s);
  if (nq <= 160) return AdmmEngine<32, 5, Tc>::run(c, a, s);
  if (nq <= 192) return AdmmEngine<32, 6, Tc>::run(c, a, s);
  if (nq <= 224) return AdmmEngine<32, 7, Tc>::run(c, a, s);
  if (nq <= 256) return AdmmEngine<32, 8, Tc>::run(c, a, s);
  set_error("d = %d exceeds the compiled maximum %d", a.d, ccm_max_dim());
  return CCM_ERR_UNSUPPORTED;
}

}  // namespace ccm

using namespace ccm;

static int solve_path_dual(int which, const char* name, ccm_ctx* x, const double* A, int64_t n, int32_t d,
                                   const int32_t* edges, const double* w, int64_t m,
                                   const double* gammas, int32_t T, int32_t q, double tol,
                                   const ccm_options* opt, double* X, int32_t* labels, double* U,
                                   ccm_stats* stats, ccm_stream_t stream) {
  Ctx* c = ctx_of(x);
  if (!c || !A || !X || !gammas || n < 1 || d < 1 || m < 0 || T < 1 || (m > 0 && (!edges || !w)) ||
      !(tol > 0) || n > INT32_MAX || m > INT32_MAX) {
    set_error("%s: invalid argument", name);
    return CCM_ERR_INVALID_ARG;
  }
  if (q != 2) {
    set_error("%s: only q = 2 is implemented (got q = %d)", name, q);
    return CCM_ERR_UNSUPPORTED;
  }
  if (d > ccm_max_dim()) {
    set_error("%s: d = %d exceeds the maximum %d", name, d, ccm_max_dim());
    return CCM_ERR_UNSUPPORTED;
  }
  for (int t = 0; t < T; ++t) {
    if (!(gammas[t] >= 0) || !std::isfinite(gammas[t]) || (t > 0 && gammas[t] < gammas[t - 1])) {
      set_error("%s: gammas must be finite, >= 0 and non-decreasing", name);
      return CCM_ERR_INVALID_ARG;
    }
  }
  if (((uintptr_t)edges) % 8 || ((uintptr_t)A) % 8 || ((uintptr_t)X) % 8) {
    set_error("%s: misaligned pointer", name);
    return CCM_ERR_INVALID_ARG;
  }
  ccm_options o;
  ccm_default_options(&o);
  if (opt) o = *opt;
  if (o.max_outer < 1 || o.max_newton < 1 || o.max_cg < 1 || !(o.sigma0 > 0)) {
    set_error("%s: invalid options", name);
    return CCM_ERR_INVALID_ARG;
  }
  CCM_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  CCM_TRY(check_edges(c, (const int2*)edges, m, n, w, s));
  SolveArgs a;
  a.A = A; a.n = n; a.d = d; a.edges = edges; a.w = w; a.m = m;
  a.gammas = gammas; a.T = T; a.tol = tol; a.opt = o; a.Xout = X; a.Uout = U;
  a.stats = stats; a.X0 = o.X0; a.U0 = o.U0;
  const int64_t launches0 = c->launches;
  int st;
  if (which == 0)
    st = o.precision == CCM_PREC_FP64 ? run_admm<double>(c, a, s) : run_admm<float>(c, a, s);
  else
    st = o.precision == CCM_PREC_FP64 ? run_ama<double>(c, a, s) : run_ama<float>(c, a, s);
  if (st != CCM_OK && st != CCM_ERR_NOT_CONVERGED) return st;
  if (labels) {
    for (int t = 0; t < T; ++t) {
      int32_t nc = 0;
      CCM_TRY(labels_device(c, X + (int64_t)t * n * d, d, n, d, (const int2*)edges, m,
                            labels + (int64_t)t * n, stats ? &nc : nullptr, s));
      if (stats) stats[t].n_clusters = nc;
    }
  }
  CCM_CUDA(cudaStreamSynchronize(s));
  c->last_profile = ccm_profile{};
  c->last_profile.kernel_launches = c->launches - launches0;
  if (st == CCM_ERR_NOT_CONVERGED)
    set_error("%s: some gamma hit the iteration cap", name);
  return st;
}

extern "C" int ccm_solve_path_admm(ccm_ctx* x, const double* A, int64_t n, int32_t d,
                                   const int32_t* edges, const double* w, int64_t m,
                                   const double* gammas, int32_t T, int32_t q, double tol,
                                   const ccm_options* opt, double* X, int32_t* labels, double* U,
                                   ccm_stats* stats, ccm_stream_t stream) {
  return solve_path_dual(0, "ccm_solve_path_admm", x, A, n, d, edges, w, m, gammas, T, q, tol,
                         opt, X, labels, U, stats, stream);
}

extern "C" int ccm_solve_path_ama(ccm_ctx* x, const double* A, int64_t n, int32_t d,
                                  const int32_t* edges, const double* w, int64_t m,
                                  const double* gammas, int32_t T, int32_t q, double tol,
                                  const ccm_options* opt, double* X, int32_t* labels, double* U,
                                  ccm_stats* stats, ccm_stream_t stream) {
  return solve_path_dual(1, "ccm_solve_path_ama", x, A, n, d, edges, w, m, gammas, T, q, tol, opt,
                         X, labels, U, stats, stream);
}
