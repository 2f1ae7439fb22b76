// Block engine: one thread block runs the whole SSNAL path of one problem.
//
// Used by ccm_solve_path_batched (many independent problems in one persistent
// launch: every block takes the next problem from a device work queue, largest
// first) and by ccm_solve_path for small problems (engine BLOCK, or AUTO when
// the problem is small). All control flow of the method (multiplier updates,
// semismooth-Newton steps, Armijo backtracking, CG) runs on the device; every
// decision is taken from block reductions whose values are identical in all
// threads, so the threads of a block always follow the same path. The
// arithmetic is the one of the grid engine (ssnal_kernels.cuh): same
// definitions, float64 evaluation/KKT, float32 or float64 CG.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "ccm_internal.cuh"
#include "solve_common.cuh"
#include "ssnal_kernels.cuh"

namespace ccm {

static constexpr int BT = 256;  // threads per block

template <typename Tc>
struct BProb {
  // inputs
  const double* A;
  const int2* edges;
  const double* w;
  int64_t n, m;
  // outputs
  double* X_out;       // T x n x d
  int32_t* labels;     // T x n or null
  double* U_out;       // T x m x d or null
  ccm_stats* stats;    // T (device)
  // workspace
  double *Ap, *Xa, *Xb, *G, *Ua, *Ub;
  Tc *Dx, *R, *P0, *P1, *Q, *Minv, *Yh, *alpha;
  uint8_t* kind;
  int64_t* off;
  int2* inc;
  int32_t* parent;
  int64_t* rank;
};

struct BCommon {
  const double* gammas;  // device, T
  int T, d, ld;
  double tol, sigma0, sigma_max;
  int max_outer, max_newton, max_cg;
  const int* order;      // problem order (largest first)
  int P;
  unsigned* queue;       // work counter
};

// ---------------------------------------------------------------- block reductions
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N]) {
  __shared__ double sh[BT / 32][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[warp][k] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double x = 0.0;
#pragma unroll
    for (int w = 0; w < BT / 32; ++w) x += sh[w][k];  // fixed order, same in every thread
    v[k] = x;
  }
  __syncthreads();
}

// exclusive scan of cnt[0..n) (int64) in place, returns the total; block-wide
__device__ int64_t block_scan_excl(int64_t* cnt, int64_t n) {
  __shared__ int64_t part[BT];
  const int64_t chunk = (n + BT - 1) / BT;
  const int64_t s = threadIdx.x * chunk, e = min(n, s + chunk);
  int64_t sum = 0;
  for (int64_t i = s; i < e; ++i) sum += cnt[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int t = 0; t < BT; ++t) {
      int64_t x = part[t];
      part[t] = run;
      run += x;
    }
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = s; i < e; ++i) {
    int64_t x = cnt[i];
    cnt[i] = run;
    run += x;
  }
  __syncthreads();
  __shared__ int64_t total;
  if (threadIdx.x == BT - 1) total = run;
  if (n == 0 && threadIdx.x == 0) total = 0;
  __syncthreads();
  return total;
}

// ---------------------------------------------------------------- per-problem setup
template <typename Tc>
__device__ void b_build_csr(const BProb<Tc>& p) {
  const int64_t n = p.n, m = p.m;
  for (int64_t i = threadIdx.x; i <= n; i += BT) p.off[i] = 0;
  __syncthreads();
  for (int64_t e = threadIdx.x; e < m; e += BT) {
    int2 ij = p.edges[e];
    atomicAdd((unsigned long long*)(p.off + ij.x), 1ull);
    atomicAdd((unsigned long long*)(p.off + ij.y), 1ull);
  }
  __syncthreads();
  block_scan_excl(p.off, n + 1);
  // cursors in parent[] (int32): reuse as per-node fill counters
  for (int64_t i = threadIdx.x; i < n; i += BT) p.parent[i] = 0;
  __syncthreads();
  for (int64_t e = threadIdx.x; e < m; e += BT) {
    int2 ij = p.edges[e];
    int a = atomicAdd(p.parent + ij.x, 1);
    int b = atomicAdd(p.parent + ij.y, 1);
    p.inc[p.off[ij.x] + a] = make_int2((int)e, ij.y);
    p.inc[p.off[ij.y] + b] = make_int2((int)e, ij.x);
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += BT) {
    int64_t b = p.off[i], e = p.off[i + 1];
    for (int64_t s = b + 1; s < e; ++s) {
      int2 key = p.inc[s];
      int64_t t = s - 1;
      while (t >= b && p.inc[t].x > key.x) {
        p.inc[t + 1] = p.inc[t];
        --t;
      }
      p.inc[t + 1] = key;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- phases
// y, kind, alpha, yhat, Pi(y) for every edge; returns (sum h, #outside) via block_sum
template <int L, int CH, typename Tc>
__device__ void b_edge_eval(const BProb<Tc>& p, const double* X, const double* U, double* Ut,
                            double gamma, double sigma, int ld, double (&out)[2]) {
  const int lane = threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  double acc[2] = {0.0, 0.0};
  for (int64_t e = threadIdx.x / L; e < p.m; e += BT / L) {
    int2 ij = p.edges[e];
    double r = gamma * p.w[e];
    double xi[CH][4], xj[CH][4], y[CH][4];
    row_load<L, CH>(X + (int64_t)ij.x * ld, ld, lane, xi);
    row_load<L, CH>(X + (int64_t)ij.y * ld, ld, lane, xj);
    row_load<L, CH>(U + e * ld, ld, lane, y);
    double ss = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        y[c][k] = fma(sigma, xi[c][k] - xj[c][k], y[c][k]);
        ss = fma(y[c][k], y[c][k], ss);
      }
    ss = group_sum<L>(ss, mask);
    double ny = sqrt(ss);
    uint8_t kd;
    double scale, a;
    if (!(r > 0.0)) {
      kd = K_INERT; scale = 0.0; a = 0.0;
    } else if (ny <= r) {
      kd = K_IN; scale = 1.0; a = 1.0;
    } else {
      kd = K_OUT; scale = r / ny; a = r / ny;
    }
    if (lane == 0) {
      acc[0] += (ny <= r) ? 0.5 * ss : r * ny - 0.5 * r * r;
      acc[1] += (kd == K_OUT) ? 1.0 : 0.0;
      p.kind[e] = kd;
      p.alpha[e] = (Tc)a;
    }
    double o[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) o[c][k] = scale * y[c][k];
    row_store<L, CH>(Ut + e * ld, ld, lane, o);
    if (kd == K_OUT) {
      double inv = 1.0 / ny;
      Tc yh[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) yh[c][k] = (Tc)(y[c][k] * inv);
      row_store<L, CH>(p.Yh + e * ld, ld, lane, yh);
    }
  }
  __syncthreads();
  block_sum<2>(acc);
  out[0] = acc[0];
  out[1] = acc[1];
}

// G = X - A + B^T Ut, Minv; returns (||G||^2, 1/2||X-A||^2)
template <int L, int CH, typename Tc>
__device__ void b_node_grad(const BProb<Tc>& p, const double* X, const double* Ut, double sigma,
                            int d, int ld, double (&out)[2]) {
  const int lane = threadIdx.x % L;
  const double tr_out = (double)(d - 1) / (double)d;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = threadIdx.x / L; i < p.n; i += BT / L) {
    double g[CH][4], a[CH][4];
    row_load<L, CH>(X + i * ld, ld, lane, g);
    row_load<L, CH>(p.Ap + i * ld, ld, lane, a);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        g[c][k] -= a[c][k];
        acc[1] += 0.5 * g[c][k] * g[c][k];
      }
    double diag = 0.0;
    for (int64_t t = p.off[i]; t < p.off[i + 1]; ++t) {
      int2 eo = p.inc[t];
      double u[CH][4];
      row_load<L, CH>(Ut + (int64_t)eo.x * ld, ld, lane, u);
      const double sg = (i < eo.y) ? 1.0 : -1.0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[c][k] += sg * u[c][k];
      uint8_t kd = p.kind[eo.x];
      diag += kd == K_IN ? 1.0 : (kd == K_OUT ? (double)p.alpha[eo.x] * tr_out : 0.0);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[0] += g[c][k] * g[c][k];
    row_store<L, CH>(p.G + i * ld, ld, lane, g);
    if (lane == 0) p.Minv[i] = (Tc)(1.0 / (1.0 + sigma * diag));
  }
  __syncthreads();
  block_sum<2>(acc);
  out[0] = acc[0];
  out[1] = acc[1];
}

// q = V p with p = Minv R + beta Pold (written to Pnew); returns <p, q>
template <int L, int CH, typename Tc>
__device__ double b_matvec(const BProb<Tc>& p, const Tc* Pold, Tc* Pnew, Tc beta, bool use_old,
                           double sigma, int ld) {
  const int lane = threadIdx.x % L;
  const unsigned mask = group_mask<L>();
  const Tc sg = (Tc)sigma;
  double acc[1] = {0.0};
  for (int64_t i = threadIdx.x / L; i < p.n; i += BT / L) {
    Tc pi[CH][4], tmp[CH][4], av[CH][4];
    const Tc mi = p.Minv[i];
    row_load<L, CH>(p.R + i * ld, ld, lane, pi);
    if (use_old) row_load<L, CH>(Pold + i * ld, ld, lane, tmp);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        pi[c][k] = mi * pi[c][k] + (use_old ? beta * tmp[c][k] : (Tc)0);
        av[c][k] = (Tc)0;
      }
    row_store<L, CH>(Pnew + i * ld, ld, lane, pi);
    for (int64_t t = p.off[i]; t < p.off[i + 1]; ++t) {
      const int2 eo = p.inc[t];
      const uint8_t kd = p.kind[eo.x];
      if (kd == K_INERT) continue;
      Tc v[CH][4];
      const Tc mo = p.Minv[eo.y];
      row_load<L, CH>(p.R + (int64_t)eo.y * ld, ld, lane, v);
      if (use_old) row_load<L, CH>(Pold + (int64_t)eo.y * ld, ld, lane, tmp);
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          v[c][k] = pi[c][k] - (mo * v[c][k] + (use_old ? beta * tmp[c][k] : (Tc)0));
      if (kd == K_OUT) {
        row_load<L, CH>(p.Yh + (int64_t)eo.x * ld, ld, lane, tmp);
        Tc s = (Tc)0;
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) s += tmp[c][k] * v[c][k];
        s = group_sum<L>(s, mask);
        const Tc a = p.alpha[eo.x];
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) av[c][k] += a * (v[c][k] - s * tmp[c][k]);
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) av[c][k] += v[c][k];
      }
    }
    Tc dot = (Tc)0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        av[c][k] = pi[c][k] + sg * av[c][k];
        dot += pi[c][k] * av[c][k];
      }
    acc[0] += (double)dot;
    row_store<L, CH>(p.Q + i * ld, ld, lane, av);
  }
  __syncthreads();
  block_sum<1>(acc);
  return acc[0];
}

// one SSNAL path for problem p (all threads of the block)
template <int L, int CH, typename Tc>
__device__ void b_solve(const BProb<Tc>& p, const BCommon& cm) {
  const int d = cm.d, ld = cm.ld;
  const int64_t n = p.n, m = p.m, nl = n * ld;
  // setup: padded A, X = A, U = 0, zero padding of the other buffers
  for (int64_t q = threadIdx.x; q < nl; q += BT) {
    int64_t r = q / ld;
    int k = (int)(q - r * ld);
    double a = (k < d) ? p.A[r * d + k] : 0.0;
    p.Ap[q] = a;
    p.Xa[q] = a;
    p.Xb[q] = 0.0;
  }
  for (int64_t q = threadIdx.x; q < m * ld; q += BT) {
    p.Ua[q] = 0.0;
    p.Ub[q] = 0.0;
    p.Yh[q] = (Tc)0;
  }
  __syncthreads();
  b_build_csr(p);
  double nA2[1] = {0.0};
  for (int64_t q = threadIdx.x; q < nl; q += BT) nA2[0] += p.Ap[q] * p.Ap[q];
  block_sum<1>(nA2);
  const double scale = 1.0 + sqrt(nA2[0]);
  double* X = p.Xa;
  double* Xt = p.Xb;
  double* U = p.Ua;
  double* Ut = p.Ub;
  double sigma = cm.sigma0;
  const double tc_floor = sizeof(Tc) == 4 ? 1e-5 : 1e-10;
  for (int t = 0; t < cm.T; ++t) {
    const double gamma = cm.gammas[t];
    ccm_stats st;
    st.status = CCM_ERR_NOT_CONVERGED;
    st.outer = st.newton = st.cg = st.line_search = 0;
    st.n_clusters = 0;
    st.kkt = st.eta_d = st.eta_p = st.gap = st.f_p = st.f_d = 0.0;
    double last_kkt = 1.0, last_etap = -1.0;
    sigma = fmin(sigma, cm.sigma_max);  // a raised cap lasts one gamma
    double cap = cm.sigma_max;
    int at_cap = 0;
    double eps_gap = 1.0;  // inner-tolerance cap from the duality gap
    double phi = 0.0, gn = 0.0, half_xa = 0.0;
    for (int outer = 0; outer < cm.max_outer; ++outer) {
      const double eps_in = fmin(fmax(0.5 * cm.tol, 0.1 * last_kkt), eps_gap);
      double ev[2], nv[2];
      b_edge_eval<L, CH, Tc>(p, X, U, Ut, gamma, sigma, ld, ev);
      b_node_grad<L, CH, Tc>(p, X, Ut, sigma, d, ld, nv);
      phi = nv[1] + ev[0] / sigma;
      gn = sqrt(nv[0]);
      half_xa = nv[1];
      for (int it = 0; it < cm.max_newton; ++it) {
        if (gn / scale <= eps_in) break;
        const double eta = fmin(0.1, fmax(tc_floor, sqrt(gn / scale)));
        // CG init: R = -G, Dx = 0
        double r0[2] = {0.0, 0.0};
        for (int64_t q = threadIdx.x; q < nl; q += BT) {
          Tc r = (Tc)(-p.G[q]);
          p.R[q] = r;
          p.Dx[q] = (Tc)0;
          double rd = (double)r;
          r0[0] += rd * rd;
          r0[1] += rd * rd * (double)p.Minv[q / ld];
        }
        __syncthreads();
        block_sum<2>(r0);
        double rr = r0[0], rz = r0[1];
        const double tol2 = eta * eta * rr;
        double beta = 0.0;
        int cgit = 0;
        Tc* Pa = p.P0;
        Tc* Pb = p.P1;
        bool active = rr > tol2 && rz > 0.0;
        while (active && cgit < cm.max_cg) {
          const double pq = b_matvec<L, CH, Tc>(p, Pa, Pb, (Tc)beta, beta != 0.0, sigma, ld);
          if (!(pq > 0.0) || !isfinite(pq)) break;
          const Tc al = (Tc)(rz / pq);
          double up[2] = {0.0, 0.0};
          for (int64_t q = threadIdx.x; q < nl; q += BT) {
            Tc dx = p.Dx[q] + al * Pb[q];
            Tc r = p.R[q] - al * p.Q[q];
            p.Dx[q] = dx;
            p.R[q] = r;
            double rd = (double)r;
            up[1] += rd * rd;
            up[0] += rd * rd * (double)p.Minv[q / ld];
          }
          __syncthreads();
          block_sum<2>(up);
          ++cgit;
          beta = (rz > 0.0) ? up[0] / rz : 0.0;
          rz = up[0];
          rr = up[1];
          Tc* tmpp = Pa;
          Pa = Pb;
          Pb = tmpp;
          if (!(rr > tol2) || !isfinite(rr) || !(rz > 0.0)) active = false;
        }
        st.cg += cgit;
        // Armijo backtracking along Dx
        double gd[1] = {0.0};
        for (int64_t q = threadIdx.x; q < nl; q += BT) gd[0] += p.G[q] * (double)p.Dx[q];
        block_sum<1>(gd);
        const double slack = 1e-14 * (1.0 + fabs(phi));
        double tstep = 1.0, phit = 0.0, gnt = 0.0, halft = 0.0;
        for (;;) {
          for (int64_t q = threadIdx.x; q < nl; q += BT) Xt[q] = X[q] + tstep * (double)p.Dx[q];
          __syncthreads();
          b_edge_eval<L, CH, Tc>(p, Xt, U, Ut, gamma, sigma, ld, ev);
          b_node_grad<L, CH, Tc>(p, Xt, Ut, sigma, d, ld, nv);
          phit = nv[1] + ev[0] / sigma;
          gnt = sqrt(nv[0]);
          halft = nv[1];
          st.line_search += 1;
          if (phit <= phi + 1e-4 * tstep * gd[0] + slack || tstep < 1e-10) break;
          tstep *= 0.5;
        }
        double* sw = X;
        X = Xt;
        Xt = sw;
        phi = phit;
        gn = gnt;
        half_xa = halft;
        st.newton += 1;
        if (tstep < 1e-10) break;
      }
      // multiplier update and KKT / objectives at (X, U)
      double* sw = U;
      U = Ut;
      Ut = sw;
      double kk[4] = {0.0, 0.0, 0.0, 0.0};
      {
        const int lane = threadIdx.x % L;
        const unsigned mask = group_mask<L>();
        for (int64_t e = threadIdx.x / L; e < m; e += BT / L) {
          int2 ij = p.edges[e];
          double r = gamma * p.w[e];
          double bx[CH][4], v[CH][4];
          row_load<L, CH>(X + (int64_t)ij.x * ld, ld, lane, bx);
          row_load<L, CH>(X + (int64_t)ij.y * ld, ld, lane, v);
          double sb = 0.0;
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              bx[c][k] -= v[c][k];
              sb += bx[c][k] * bx[c][k];
            }
          row_load<L, CH>(U + e * ld, ld, lane, v);
          double sv = 0.0;
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              v[c][k] += bx[c][k];
              sv += v[c][k] * v[c][k];
            }
          sb = group_sum<L>(sb, mask);
          sv = group_sum<L>(sv, mask);
          double nvv = sqrt(sv);
          double shrink = (nvv > r) ? 1.0 - r / nvv : 0.0;
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              double res = bx[c][k] - shrink * v[c][k];
              kk[0] += res * res;
            }
          if (lane == 0) kk[1] += r * sqrt(sb);
        }
        for (int64_t q = threadIdx.x; q < nl; q += BT) {
          double a = p.Ap[q];
          double btu = p.G[q] - (X[q] - a);
          kk[2] += a * btu;
          kk[3] += btu * btu;
        }
        __syncthreads();
        block_sum<4>(kk);
      }
      st.outer += 1;
      const double eta_d = gn / scale;
      const double eta_p = sqrt(kk[0]) / scale;
      const double fp = half_xa + kk[1];
      const double fd = kk[2] - 0.5 * kk[3];
      const double gap = fabs(fp - fd) / (1.0 + fabs(fp) + fabs(fd));
      st.eta_d = eta_d;
      st.eta_p = eta_p;
      st.kkt = fmax(eta_d, eta_p);
      st.f_p = fp;
      st.f_d = fd;
      st.gap = gap;
      if (st.kkt <= cm.tol && gap <= cm.tol) {
        st.status = CCM_OK;
        break;
      }
      // f_p - f_d >= 1/2 ||X - A + B^T U||^2 (U dual feasible): cap the inner tolerance
      if (gap > cm.tol)
        eps_gap = fmin(eps_gap, 0.5 * sqrt(2.0 * cm.tol * (1.0 + fabs(fp) + fabs(fd))) / scale);
      // same penalty rule as the grid engine (cap rises 10x after 20 steps at it)
      if (last_etap >= 0.0 && eta_p > 0.2 * last_etap) sigma = fmin(3.0 * sigma, cap);
      if (sigma >= cap) {
        if (++at_cap >= 20) {
          cap = fmin(10.0 * cap, 1e6);
          at_cap = 0;
        }
      } else {
        at_cap = 0;
      }
      last_etap = eta_p;
      last_kkt = st.kkt;
    }
    st.sigma = sigma;
    // outputs for this gamma
    double* Xo = p.X_out + (int64_t)t * n * d;
    for (int64_t q = threadIdx.x; q < n * d; q += BT) {
      int64_t r = q / d;
      Xo[q] = X[r * ld + (q - r * d)];
    }
    if (p.U_out) {
      double* Uo = p.U_out + (int64_t)t * m * d;
      for (int64_t q = threadIdx.x; q < m * d; q += BT) {
        int64_t r = q / d;
        Uo[q] = U[r * ld + (q - r * d)];
      }
    }
    __syncthreads();
    // labels: union-find over fused edges (same rule as labels.cu)
    int32_t* par = p.parent;
    for (int64_t i = threadIdx.x; i < n; i += BT) par[i] = (int32_t)i;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < m; e += BT) {
      int2 ij = p.edges[e];
      const double* xi = Xo + (int64_t)ij.x * d;
      const double* xj = Xo + (int64_t)ij.y * d;
      double acc = 0.0;
      for (int k = 0; k < d; ++k) {
        double dl = __dsub_rn(xi[k], xj[k]);
        acc = __dadd_rn(acc, __dmul_rn(dl, dl));
      }
      if (!(acc <= 1e-12)) continue;
      int32_t a = ij.x, b = ij.y;
      for (int64_t g = 0; g <= n; ++g) {  // find roots (parent[x] <= x: bounded by n)
        int32_t pa = __ldcg(par + a);
        if (pa == a) break;
        a = pa;
      }
      for (int64_t g = 0; g <= n; ++g) {
        int32_t pb = __ldcg(par + b);
        if (pb == b) break;
        b = pb;
      }
      for (int64_t g = 0; a != b && g <= n; ++g) {
        int32_t lo = a < b ? a : b, hi = a < b ? b : a;
        int32_t old = atomicMin(par + hi, lo);
        if (old == hi) break;
        int32_t x = old;
        for (int64_t h = 0; h <= n; ++h) {
          int32_t px = __ldcg(par + x);
          if (px == x) break;
          x = px;
        }
        if (hi == a) a = x;
        else b = x;
      }
    }
    __syncthreads();
    // roots, ranks
    int64_t* rank = p.rank;
    for (int64_t i = threadIdx.x; i < n; i += BT) {
      int32_t x = (int32_t)i;
      for (int64_t g = 0; g <= n; ++g) {
        int32_t px = __ldcg(par + x);
        if (px == x) break;
        x = px;
      }
      par[i] = x;  // flatten (roots are fixed points)
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += BT) rank[i] = (par[i] == (int32_t)i) ? 1 : 0;
    __syncthreads();
    const int64_t K = block_scan_excl(rank, n);
    if (p.labels)
      for (int64_t i = threadIdx.x; i < n; i += BT)
        p.labels[(int64_t)t * n + i] = (int32_t)rank[par[i]];
    __syncthreads();
    st.n_clusters = (int32_t)K;
    if (threadIdx.x == 0) p.stats[t] = st;
  }
}

template <int L, int CH, typename Tc>
__global__ void __launch_bounds__(BT)
k_block_paths(BProb<Tc>* probs, BCommon cm) {
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) {
      unsigned k = atomicAdd(cm.queue, 1u);
      cur = (k < (unsigned)cm.P) ? cm.order[k] : -1;
    }
    __syncthreads();
    const int pi = cur;
    __syncthreads();
    if (pi < 0) return;
    b_solve<L, CH, Tc>(probs[pi], cm);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host side
template <typename Tc>
static size_t carve_bytes(int64_t n, int64_t m, int ld) {
  auto a = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t nl = (size_t)n * ld, ml = (size_t)std::max<int64_t>(m, 1) * ld;
  size_t b = 0;
  b += 4 * a(nl * 8);                            // Ap, Xa, Xb, G
  b += 2 * a(ml * 8);                            // Ua, Ub
  b += 5 * a(nl * sizeof(Tc));                   // Dx, R, P0, P1, Q
  b += a((size_t)n * sizeof(Tc));                // Minv
  b += a(ml * sizeof(Tc));                       // Yh
  b += a((size_t)std::max<int64_t>(m, 1) * sizeof(Tc));  // alpha
  b += a((size_t)std::max<int64_t>(m, 1));       // kind
  b += a((size_t)(n + 1) * 8);                   // off
  b += a((size_t)std::max<int64_t>(2 * m, 1) * 8);  // inc
  b += a((size_t)n * 4);                         // parent
  b += a((size_t)(n + 1) * 8);                   // rank
  return b;
}

template <typename Tc>
static void carve(BProb<Tc>& p, char*& base, int ld) {
  auto a = [](size_t x) { return (x + 255) / 256 * 256; };
  auto take = [&](size_t bytes) {
    char* r = base;
    base += a(bytes);
    return r;
  };
  size_t nl = (size_t)p.n * ld, ml = (size_t)std::max<int64_t>(p.m, 1) * ld;
  p.Ap = (double*)take(nl * 8);
  p.Xa = (double*)take(nl * 8);
  p.Xb = (double*)take(nl * 8);
  p.G = (double*)take(nl * 8);
  p.Ua = (double*)take(ml * 8);
  p.Ub = (double*)take(ml * 8);
  p.Dx = (Tc*)take(nl * sizeof(Tc));
  p.R = (Tc*)take(nl * sizeof(Tc));
  p.P0 = (Tc*)take(nl * sizeof(Tc));
  p.P1 = (Tc*)take(nl * sizeof(Tc));
  p.Q = (Tc*)take(nl * sizeof(Tc));
  p.Minv = (Tc*)take((size_t)p.n * sizeof(Tc));
  p.Yh = (Tc*)take(ml * sizeof(Tc));
  p.alpha = (Tc*)take((size_t)std::max<int64_t>(p.m, 1) * sizeof(Tc));
  p.kind = (uint8_t*)take((size_t)std::max<int64_t>(p.m, 1));
  p.off = (int64_t*)take((size_t)(p.n + 1) * 8);
  p.inc = (int2*)take((size_t)std::max<int64_t>(2 * p.m, 1) * 8);
  p.parent = (int32_t*)take((size_t)p.n * 4);
  p.rank = (int64_t*)take((size_t)(p.n + 1) * 8);
}

struct HostProblem {
  const double* A;
  const int32_t* edges;
  const double* w;
  int64_t n, m;
  double* X;
  int32_t* labels;
  double* U;
};

template <int L, int CH, typename Tc>
static int run_block_engine(Ctx* c, const std::vector<HostProblem>& hp, int d, const double* gammas,
                            int T, double tol, const ccm_options& o, ccm_stats* stats_host,
                            cudaStream_t s) {
  const int P = (int)hp.size();
  const int ld = (int)round_up(d, 4);
  size_t total = 0;
  std::vector<size_t> sz(P);
  for (int i = 0; i < P; ++i) total += (sz[i] = carve_bytes<Tc>(hp[i].n, hp[i].m, ld));
  void* p;
  CCM_TRY(ws_get(c, S_BATCH0, total, &p));
  char* base = (char*)p;
  std::vector<BProb<Tc>> probs(P);
  for (int i = 0; i < P; ++i) {
    BProb<Tc>& b = probs[i];
    b.A = hp[i].A;
    b.edges = (const int2*)hp[i].edges;
    b.w = hp[i].w;
    b.n = hp[i].n;
    b.m = hp[i].m;
    b.X_out = hp[i].X;
    b.labels = hp[i].labels;
    b.U_out = hp[i].U;
    carve(b, base, ld);
  }
  // device arrays: problems, stats, gammas, order, queue
  CCM_TRY(ws_get(c, S_BATCH1, (size_t)P * sizeof(BProb<Tc>) + (size_t)P * T * sizeof(ccm_stats) +
                                  (size_t)T * 8 + (size_t)P * 4 + 64, &p));
  char* q = (char*)p;
  BProb<Tc>* d_probs = (BProb<Tc>*)q;
  q += (size_t)P * sizeof(BProb<Tc>);
  ccm_stats* d_stats = (ccm_stats*)q;
  q += (size_t)P * T * sizeof(ccm_stats);
  double* d_g = (double*)q;
  q += (size_t)T * 8;
  int* d_order = (int*)q;
  q += (size_t)P * 4;
  unsigned* d_queue = (unsigned*)(((uintptr_t)q + 15) / 16 * 16);
  for (int i = 0; i < P; ++i) probs[i].stats = d_stats + (size_t)i * T;
  std::vector<int> order(P);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return hp[a].m * 4 + hp[a].n > hp[b].m * 4 + hp[b].n;
  });
  CCM_CUDA(cudaMemcpyAsync(d_probs, probs.data(), (size_t)P * sizeof(BProb<Tc>),
                           cudaMemcpyHostToDevice, s));
  CCM_CUDA(cudaMemcpyAsync(d_g, gammas, (size_t)T * 8, cudaMemcpyHostToDevice, s));
  CCM_CUDA(cudaMemcpyAsync(d_order, order.data(), (size_t)P * 4, cudaMemcpyHostToDevice, s));
  CCM_CUDA(cudaMemsetAsync(d_queue, 0, 4, s));
  BCommon cm;
  cm.gammas = d_g;
  cm.T = T;
  cm.d = d;
  cm.ld = ld;
  cm.tol = tol;
  cm.sigma0 = o.sigma0;
  cm.sigma_max = o.sigma_max;
  cm.max_outer = o.max_outer;
  cm.max_newton = o.max_newton;
  cm.max_cg = o.max_cg;
  cm.order = d_order;
  cm.P = P;
  cm.queue = d_queue;
  int per_sm = 0;
  CCM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_block_paths<L, CH, Tc>, BT, 0));
  per_sm = std::max(1, per_sm);
  const int blocks = std::max(1, std::min(P, c->num_sms * per_sm));
  k_block_paths<L, CH, Tc><<<blocks, BT, 0, s>>>(d_probs, cm);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  std::vector<ccm_stats> hs((size_t)P * T);
  CCM_CUDA(cudaMemcpyAsync(hs.data(), d_stats, hs.size() * sizeof(ccm_stats),
                           cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  int fail = 0;
  for (auto& st : hs) fail |= (st.status != CCM_OK);
  if (stats_host) std::copy(hs.begin(), hs.end(), stats_host);
  return fail ? CCM_ERR_NOT_CONVERGED : CCM_OK;
}

// ---------------------------------------------------------------- shapes and autotuning
// A row of nq quads is handled by a group of L lanes with CH quads each (L CH >=
// nq): 32 / L edges (or nodes) per warp. The default takes the narrowest power of
// two L >= nq with CH = 1; the alternatives fold it to L/2 x 2 and L/4 x 4, which
// put more edges in flight per warp and shorten the group sums at the price of
// registers per thread.
template <typename Tc>
static int run_shape(Ctx* c, int L, int CH, const std::vector<HostProblem>& hp, int d,
                     const double* g, int T, double tol, const ccm_options& o, ccm_stats* st,
                     cudaStream_t s) {
#define CCM_SHAPE(LL, CC) \
  if (L == LL && CH == CC) return run_block_engine<LL, CC, Tc>(c, hp, d, g, T, tol, o, st, s);
  CCM_SHAPE(1, 1) CCM_SHAPE(2, 1) CCM_SHAPE(1, 2) CCM_SHAPE(4, 1) CCM_SHAPE(2, 2) CCM_SHAPE(1, 4)
  CCM_SHAPE(8, 1) CCM_SHAPE(4, 2) CCM_SHAPE(2, 4) CCM_SHAPE(16, 1) CCM_SHAPE(8, 2)
  CCM_SHAPE(4, 4) CCM_SHAPE(32, 1) CCM_SHAPE(16, 2) CCM_SHAPE(8, 4)
#undef CCM_SHAPE
  set_error("block engine: no kernel for %d lanes x %d quads", L, CH);
  return CCM_ERR_UNSUPPORTED;
}

static int default_lanes(int d) {
  const int nq = (int)(round_up(d, 4) / 4);
  int L = 1;
  while (L < nq) L <<= 1;
  return L;
}

// Shape for a batch: the measured best of the candidates on a sample of the
// batch, cached per context and (d, precision, mean-degree bucket). Tuning runs
// when the batch has at least kTuneMin problems and options.autotune is set; the
// sample is eight problems spread over the batch's sizes, solved for the first
// three gammas with every candidate (their outputs are overwritten by the run
// that follows). Other batches and single problems use a cached shape for their
// key when there is one, else the default.
static constexpr int kTuneMin = 8;

template <typename Tc>
static int pick_shape(Ctx* c, const std::vector<HostProblem>& hp, int d, const double* g, int T,
                      double tol, const ccm_options& o, cudaStream_t s, int* Lout, int* CHout) {
  const int L0 = default_lanes(d);
  double sn = 0, sm = 0;
  for (auto& p : hp) {
    sn += (double)p.n;
    sm += (double)p.m;
  }
  const double deg = sn > 0 ? 2.0 * sm / sn : 0.0;
  int bucket = 0;
  while ((double)(2 << bucket) <= deg && bucket < 30) ++bucket;
  for (auto& e : c->block_tune)
    if (e.d == d && e.tc == (int)sizeof(Tc) && e.bucket == bucket) {
      *Lout = e.L;
      *CHout = e.CH;
      return CCM_OK;
    }
  *Lout = L0;
  *CHout = 1;
  if (!o.autotune || (int)hp.size() < kTuneMin || L0 < 2) return CCM_OK;
  // sample: eight problems spread over the batch ordered by size
  std::vector<int> order(hp.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return hp[a].m * 4 + hp[a].n > hp[b].m * 4 + hp[b].n;
  });
  std::vector<HostProblem> sample;
  for (int k = 0; k < kTuneMin; ++k) sample.push_back(hp[order[(size_t)k * hp.size() / kTuneMin]]);
  const int Ts = std::min(T, 3);
  std::vector<ccm_stats> st((size_t)sample.size() * Ts);
  if (c->ev_pool.size() < 2) {
    while (c->ev_pool.size() < 2) {
      cudaEvent_t e;
      CCM_CUDA(cudaEventCreate(&e));
      c->ev_pool.push_back(e);
    }
  }
  float best = 0.f;
  for (int f = 1; f <= 4 && L0 / f >= 1; f *= 2) {
    const int L = L0 / f, CH = f;
    CCM_CUDA(cudaEventRecord(c->ev_pool[0], s));
    const int r = run_shape<Tc>(c, L, CH, sample, d, g, Ts, tol, o, st.data(), s);
    if (r != CCM_OK && r != CCM_ERR_NOT_CONVERGED) return r;
    CCM_CUDA(cudaEventRecord(c->ev_pool[1], s));
    CCM_CUDA(cudaEventSynchronize(c->ev_pool[1]));
    float ms = 0.f;
    CCM_CUDA(cudaEventElapsedTime(&ms, c->ev_pool[0], c->ev_pool[1]));
    if (f == 1 || ms < best) {
      best = ms;
      *Lout = L;
      *CHout = CH;
    }
  }
  c->block_tune.push_back(BlockTune{d, (int)sizeof(Tc), bucket, *Lout, *CHout});
  return CCM_OK;
}

template <typename Tc>
static int dispatch_block(Ctx* c, const std::vector<HostProblem>& hp, int d, const double* g,
                          int T, double tol, const ccm_options& o, ccm_stats* st,
                          cudaStream_t s) {
  if (d > 128) {
    set_error("block engine: d = %d above its maximum 128", d);
    return CCM_ERR_UNSUPPORTED;
  }
  int L = 0, CH = 0;
  CCM_TRY(pick_shape<Tc>(c, hp, d, g, T, tol, o, s, &L, &CH));
  c->last_profile.block_lanes = L;
  c->last_profile.block_quads = CH;
  return run_shape<Tc>(c, L, CH, hp, d, g, T, tol, o, st, s);
}

int solve_block(Ctx* c, const std::vector<HostProblem>& hp, int d, const double* gammas, int T,
                double tol, const ccm_options& o, ccm_stats* stats, cudaStream_t s) {
  return o.precision == CCM_PREC_FP64
             ? dispatch_block<double>(c, hp, d, gammas, T, tol, o, stats, s)
             : dispatch_block<float>(c, hp, d, gammas, T, tol, o, stats, s);
}

// single problem through the block engine (ccm_solve_path, small problems)
int solve_single_block(Ctx* c, const SolveArgs& a, int32_t* labels, cudaStream_t s) {
  std::vector<HostProblem> hp(1);
  hp[0] = HostProblem{a.A, a.edges, a.w, a.n, a.m, a.Xout, labels, a.Uout};
  std::vector<ccm_stats> st(a.T);
  int r = solve_block(c, hp, a.d, a.gammas, a.T, a.tol, a.opt, st.data(), s);
  if (a.stats) std::copy(st.begin(), st.end(), a.stats);
  return r;
}

}  // namespace ccm

using namespace ccm;

extern "C" int ccm_solve_path_batched(ccm_ctx* x, int32_t P, const ccm_problem* probs, int32_t d,
                                      const double* gammas, int32_t T, double tol,
                                      const ccm_options* opt, ccm_stats* stats,
                                      ccm_stream_t stream) {
  Ctx* c = ctx_of(x);
  if (!c || P < 1 || !probs || d < 1 || !gammas || T < 1 || !(tol > 0)) {
    set_error("ccm_solve_path_batched: invalid argument");
    return CCM_ERR_INVALID_ARG;
  }
  if (d > 128) {
    set_error("ccm_solve_path_batched: d = %d above the batched maximum 128", d);
    return CCM_ERR_UNSUPPORTED;
  }
  for (int t = 0; t < T; ++t)
    if (!(gammas[t] >= 0) || !std::isfinite(gammas[t]) || (t > 0 && gammas[t] < gammas[t - 1])) {
      set_error("ccm_solve_path_batched: gammas must be finite, >= 0 and non-decreasing");
      return CCM_ERR_INVALID_ARG;
    }
  ccm_options o;
  ccm_default_options(&o);
  if (opt) o = *opt;
  o.sigma_max = resolve_sigma_max(o, 2);
  CCM_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<HostProblem> hp(P);
  for (int i = 0; i < P; ++i) {
    const ccm_problem& q = probs[i];
    if (!q.A || !q.X || q.n < 1 || q.m < 0 || (q.m > 0 && (!q.edges || !q.w)) ||
        q.n > INT32_MAX || ((uintptr_t)q.edges) % 8) {
      set_error("ccm_solve_path_batched: invalid problem %d", i);
      return CCM_ERR_INVALID_ARG;
    }
    CCM_TRY(check_edges(c, (const int2*)q.edges, q.m, q.n, q.w, s));
    hp[i] = HostProblem{q.A, q.edges, q.w, q.n, q.m, q.X, q.labels, nullptr};
  }
  return solve_block(c, hp, d, gammas, T, tol, o, stats, s);
}
