// SSNAL building blocks for model CCM, q = 2 (Sec. 1 names the method); the q = 1
// and q = inf edge passes and their Jacobian kinds are at the end of this file.
//
// Notation (restated from convex analysis; the paper prints no formulas for
// SSNAL): edges l = (i, j), i < j; (BX)_l = x_i - x_j; r_l = gamma w_l;
// Pi = row-wise projection onto {||u_l|| <= r_l}; sigma = AL penalty.
//   y_l        = u_l + sigma (x_i - x_j)
//   phi(X)     = 1/2||X - A||^2 + (1/sigma) sum_l h_l(y_l)  (+ a constant)
//   h_l(y)     = ||y||^2/2 if ||y|| <= r_l, else r_l||y|| - r_l^2/2
//   grad phi   = X - A + B^T Pi(y)
//   V          = I + sigma B^T P B,  P_l = I (||y_l|| <= r_l, r_l > 0),
//                P_l = (r_l/||y_l||)(I - yhat_l yhat_l^T) (||y_l|| > r_l),
//                P_l = 0 (r_l = 0)
// The scatter B^T(.) is a deterministic pull through the CSR of B^T: node i
// visits its incident edges in increasing edge id; the contribution of edge
// l to node i is +(.)_l if i is its first endpoint and -(.)_l otherwise. For the
// operator, both signs give P_l (p_i - p_other), so no sign is needed there.
#pragma once

#include "ccm_internal.cuh"

namespace ccm {

// K_MASK (q = 1 only): P_l = diag(mask) with mask_k = 1 where |y_k| <= r_l; the
// mask row is stored in the yhat slot and alpha holds trace(P_l)/d.
// K_LINF (q = inf only, y_l outside the l1 ball): P_l = diag(mask) - s s^T with
// mask the support S of Pi(y_l) and s = sign(y_l) mask / sqrt(|S|); the unit
// vector s is stored in the yhat slot (mask = s != 0) and alpha holds
// trace(P_l)/d = (|S| - 1)/d (0 when |S| = 1, where P_l = 0).
enum EdgeKind : uint8_t { K_INERT = 0, K_IN = 1, K_OUT = 2, K_MASK = 3, K_LINF = 4 };

// The int32 value of q that selects q = inf.
constexpr int kQInf = CCM_Q_INF;

// Bounds-checked build (CCM_DEBUG_BOUNDS): the kernels that gather through the
// CSR incidence records check each record's edge id and other endpoint against
// the problem's sizes before touching memory; a bad record is skipped and the
// first one is recorded here (no trap), and the host turns it into
// CCM_ERR_BOUNDS. One copy per translation unit; the grid engine's host code
// sets the sizes before its launches (a unit that never sets them, n = 0, is
// not checked).
struct DebugBounds {
  long long n, m;
  int err, where;
  long long index;
};
#ifdef CCM_DEBUG_BOUNDS
static __device__ DebugBounds g_bounds;
__device__ __forceinline__ bool inc_ok(int2 eo, int where, long long idx) {
  if (g_bounds.n == 0) return true;
  const bool ok = eo.x >= 0 && eo.x < g_bounds.m && eo.y >= 0 && eo.y < g_bounds.n;
  if (!ok && atomicCAS(&g_bounds.err, 0, 1) == 0) {
    g_bounds.where = where;
    g_bounds.index = idx;
  }
  return ok;
}
#else
__device__ __forceinline__ bool inc_ok(int2, int, long long) { return true; }
#endif
// Kernels named by DebugBounds::where.
enum BoundsSite { B_CG_INIT = 1, B_MATVEC = 2, B_MATVEC_RING = 3 };

// Device-resident scalars of one solve (one problem).
struct CgCtl {
  double rz, rr, tol2, alpha, beta;
  int it, maxit, active, pad;
};
struct Ctl {
  CgCtl cg;
  double eval[4];   // sum_h, 1/2||X-A||^2, ||G||^2, number of outside edges
  double dots[2];   // <G, Dx>
  double kkt[4];    // ||BX - prox(BX+U)||^2, sum r||BX||, <A, B^T U>, ||B^T U||^2
  unsigned counter[8];
};
enum CounterId { C_EVAL_E = 0, C_EVAL_N, C_CGI, C_MV, C_UPD, C_TRIAL, C_KKT_E, C_KKT_N };

// float64 -> float32 rounding toward zero from the bit fields (IEEE 754
// binary64: sign, 11-bit exponent biased by 1023, 52-bit fraction; binary32:
// 8-bit exponent biased by 127, 23-bit fraction): the high word carries the
// sign, the exponent and 20 fraction bits, the low word the next 3. Values
// below 2^-126 in magnitude go to a signed zero; the yhat components this
// converts are at most 1 in magnitude, so no overflow case arises. Integer
// operations only: on B300 the FP64 pipe (2 operations per clock per SM) is
// the limit of the edge passes, and a conversion instruction would occupy it.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned mag = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float((hi & 0x80000000u) | (e > 896u ? mag : 0u));
}
// float32 -> float64, exact, from the bit fields (normal, finite x only): the
// sign and the 23 fraction bits move over unchanged, the exponent is re-biased
// from 127 to 1023. Integer operations only (see f64_to_f32_rz).
__device__ __forceinline__ double f32_to_f64_normal(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = ((b >> 23) & 0xffu) + 896u;
  const unsigned hi = (b & 0x80000000u) | (e << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// 1/sqrt(s) for s > 0 to about 1e-13 relative: a float32 hardware estimate
// (error about 2^-22 after the truncation of s to float32) refined by one
// Newton step for f(x) = 1/x^2 - s in float64,
//   x1 = x0 + (x0/2)(1 - s x0^2),
// whose relative error is about (3/2) e0^2. That costs four float64 operations
// against the twenty or so of a correctly rounded square root and division,
// which matters on B300 whose FP64 pipe (2 operations per clock per SM) bounds
// the edge passes. Outside [1e-36, 1e36], where the float32 estimate could
// overflow or lose precision, it takes 1/sqrt(s) in float64.
__device__ __forceinline__ double rsqrt_refined(double s) {
  if (!(s > 1e-36 && s < 1e36)) return 1.0 / sqrt(s);
  const double x0 = f32_to_f64_normal(rsqrtf(f64_to_f32_rz(s)));
  const double e = fma(-(s * x0), x0, 1.0);
  return fma(0.5 * x0, e, x0);
}

// Group shape of the q = 2 edge passes for an operator shape (LANES, CH). Those
// passes do per-edge scalar work (three norms, their inverse square roots, the
// ball test, h) in every lane of the edge's group, so for short rows (one quad
// per lane) each lane takes four quads and the group is four times narrower:
// fewer lanes repeat the scalar work and the group sums have fewer levels.
template <int LANES, int CH>
struct EdgeShape {
  static constexpr int L = (CH == 1 && LANES >= 4) ? LANES / 4 : (CH == 1 && LANES == 2 ? 1 : LANES);
  static constexpr int C = CH * LANES / L;
};

// Group shape of the float-float edge passes (ff_kernels.cuh). The KKT pass
// keeps two rows of each edge in registers (bx and u, later y), so where the
// edge shape gives a lane four quads the float-float passes give it two (twice
// the lanes), which keeps two resident blocks per SM for the KKT pass (744
// against 919 us on 1.7 M edges of 13 quads) and shortens the evaluation pass
// as well (400 against 431 us).
template <int LANES, int CH>
struct FfEdgeShape {
  using E = EdgeShape<LANES, CH>;
  static constexpr int L = (E::C == 4 && E::L <= 16) ? 2 * E::L : E::L;
  static constexpr int C = E::C * E::L / L;
};

template <typename Tc>
__device__ __forceinline__ Tc to_operator(double x);
template <>
__device__ __forceinline__ float to_operator<float>(double x) { return f64_to_f32_rz(x); }
template <>
__device__ __forceinline__ double to_operator<double>(double x) { return x; }

// ------------------------------------------------------------ edge evaluation
// For every edge: y, ||y||, kind, Pi(y) -> Ut, yhat -> Yh (outside edges),
// alpha; accumulates sum_l h_l(y_l).
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_edge_eval(const double* __restrict__ X, const double* __restrict__ U,
            const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
            double sigma, double* __restrict__ Ut, Tc* __restrict__ Yh, Tc* __restrict__ alpha,
            uint8_t* __restrict__ kind, int64_t m, int ld, double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  double acc[2] = {0.0, 0.0};
  for (int64_t e = g0; e < m; e += ng) {
    int2 ij = edges[e];
    double r = gamma * w[e];
    double xi[CH][4], xj[CH][4], y[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, xi);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, xj);
    row_load<LANES, CH>(U + e * ld, ld, lane, y);
    double ss = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        y[c][k] = fma(sigma, xi[c][k] - xj[c][k], y[c][k]);
        ss = fma(y[c][k], y[c][k], ss);
      }
    ss = group_sum<LANES>(ss, mask);
    // ||y|| and 1/||y|| from one refined inverse square root (ss = 0: y = 0, inside)
    const double rs = ss > 0.0 ? rsqrt_refined(ss) : 0.0;
    const double ny = ss * rs;
    uint8_t kd;
    double scale, a;
    if (!(r > 0.0)) {
      kd = K_INERT; scale = 0.0; a = 0.0;
    } else if (ny <= r) {
      kd = K_IN; scale = 1.0; a = 1.0;
    } else {
      kd = K_OUT; scale = r * rs; a = scale;
    }
    double h = (ny <= r) ? 0.5 * ss : r * ny - 0.5 * r * r;
    if (lane == 0) {
      acc[0] += h;
      acc[1] += (kd == K_OUT) ? 1.0 : 0.0;
      kind[e] = kd;
      alpha[e] = (Tc)a;
    }
    if (kd == K_IN) {
      row_store<LANES, CH>(Ut + e * ld, ld, lane, y);  // Pi(y) = y inside the ball
    } else {
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) xi[c][k] = scale * y[c][k];
      row_store<LANES, CH>(Ut + e * ld, ld, lane, xi);
    }
    if (kd == K_OUT) {
      // yhat in the operator's precision: for float32 the scaling runs in
      // float32 (FP64 throughput is the limit of this kernel)
      const Tc invc = to_operator<Tc>(rs);
      Tc yh[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) yh[c][k] = to_operator<Tc>(y[c][k]) * invc;
      row_store<LANES, CH>(Yh + e * ld, ld, lane, yh);
    }
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_EVAL_E], tot) && threadIdx.x == 0) {
    ctl->eval[0] = tot[0];
    ctl->eval[3] = tot[1];
  }
}

// ------------------------------------------------------------ node gradient
// G_i = x_i - a_i + sum_l +-Ut_l ; also Jacobi scalars Minv_i = 1/(1 + sigma sum_l t_l)
// with t_l = trace(P_l)/d: 1 (inside), alpha_l (d-1)/d (outside), alpha_l (q = 1
// mask, q = inf l1-ball kinds), 0 (inert).
//
// Register form (rows of at most 32 quads per group). Memory-level parallelism:
// a group reads its node's incidence records LANES at a time, one per lane
// (coalesced), and then gathers kNB incident rows at once before adding them,
// so a lane keeps kNB row loads in flight instead of one. The rows are still
// added one by one in increasing edge id (the same order for every run).
template <int CH>
struct GatherDepth {
  static constexpr int v = CH <= 2 ? 4 : 1;
};

// Group shape of the register-form operator for an operator shape (LANES, CH):
// rows of one quad per lane on 8 or more lanes run on half as many lanes with
// two quads each, which halves the per-incidence overhead (record broadcasts,
// loop control) and the levels of the per-edge group sums (measured: 0.58 ->
// 0.54 ms per launch at n = 200,000, d = 50; the node gradient, whose work is
// per element, was slower in that shape and keeps one quad per lane).
template <int LANES, int CH>
struct GatherShape {
  static constexpr int L = (CH == 1 && LANES >= 8) ? LANES / 2 : LANES;
  static constexpr int C = CH * LANES / L;
};

template <typename Tc>
__device__ __forceinline__ double trace_term(uint8_t kd, Tc al, double tr_out) {
  return kd == K_IN ? 1.0
         : (kd == K_OUT ? (double)al * tr_out
                        : ((kd == K_MASK || kd == K_LINF) ? (double)al : 0.0));
}

template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_node_grad(const double* __restrict__ X, const double* __restrict__ Ap,
            const double* __restrict__ Ut, const int64_t* __restrict__ off,
            const int2* __restrict__ inc, const Tc* __restrict__ alpha,
            const uint8_t* __restrict__ kind, double sigma, int d, double* __restrict__ G,
            Tc* __restrict__ Minv, int64_t n, int ld, double* partials, Ctl* ctl) {
  constexpr int NB = GatherDepth<CH>::v;
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const double tr_out = (double)(d - 1) / (double)d;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = g0; i < n; i += ng) {
    const int64_t b = off[i], eend = off[i + 1];
    double g[CH][4], a4[CH][4];
    row_load<LANES, CH>(X + i * ld, ld, lane, g);
    row_load<LANES, CH>(Ap + i * ld, ld, lane, a4);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        g[c][k] -= a4[c][k];
        acc[1] += 0.5 * g[c][k] * g[c][k];
      }
    double diag = 0.0;
    for (int64_t base = b; base < eend; base += LANES) {
      const int nb = (int)(eend - base < (int64_t)LANES ? eend - base : (int64_t)LANES);
      int2 rec = make_int2(0, 0);
      double tl = 0.0;
      if (lane < nb) {
        rec = inc[base + lane];
        tl = trace_term<Tc>(kind[rec.x], alpha[rec.x], tr_out);
      }
      diag += group_sum<LANES>(tl, mask);
      for (int j = 0; j < nb; j += NB) {
        double u[NB][CH][4];
        double sg[NB];
#pragma unroll
        for (int kk = 0; kk < NB; ++kk) {
          const int ex = __shfl_sync(mask, rec.x, j + kk, LANES);
          const int ey = __shfl_sync(mask, rec.y, j + kk, LANES);
          sg[kk] = (i < ey) ? 1.0 : -1.0;
          if (j + kk < nb) {
            row_load<LANES, CH>(Ut + (int64_t)ex * ld, ld, lane, u[kk]);
          } else {
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) u[kk][c][k] = 0.0;
            sg[kk] = 0.0;
          }
        }
#pragma unroll
        for (int kk = 0; kk < NB; ++kk)
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[c][k] += sg[kk] * u[kk][c][k];
      }
    }
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[0] += g[c][k] * g[c][k];
    row_store<LANES, CH>(G + i * ld, ld, lane, g);
    if (lane == 0) Minv[i] = (Tc)(1.0 / (1.0 + sigma * diag));
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_EVAL_N], tot) && threadIdx.x == 0) {
    ctl->eval[2] = tot[0];
    ctl->eval[1] = tot[1];
  }
}

// ------------------------------------------------------------ CG
// Preconditioned CG on V dx = -G in the Chronopoulos-Gear arrangement, which
// needs one reduction phase per operator application and applies V to
// u = M r (M = diag(Minv), one scalar per node) rather than to the search
// direction, so the operator gathers one vector (R) per neighbour:
//   matvec:  W = V u,  delta = <W, u>,
//            alpha = gamma / (delta - beta gamma / alpha_prev)   (gamma / delta first),
//   update:  P = u + beta P,  S = W + beta S  (S = V P),  dx += alpha P,  r -= alpha S,
//            gamma' = <r, M r>,  beta' = gamma' / gamma.
// In exact arithmetic the iterates equal those of standard preconditioned CG.

// Per-incidence operator coefficients, packed once per Newton step: c = 1
// (inside edge, P_l = I), c = -alpha_l (outside edge, P_l = alpha_l (I - yhat yhat^T)),
// c = 2 (q = 1 mask edge, P_l = diag(mask row)), c = 3 (q = inf edge outside the
// l1 ball, P_l = diag(s != 0) - s s^T), c = 0 (inert edge, or a q = inf edge with
// |S| = 1, where P_l = 0); mo = Minv of the incidence's other endpoint.
template <typename Tc>
struct alignas(2 * sizeof(Tc)) IncMeta {
  Tc c, mo;
};

// Dot products of the CG kernels: float32 products summed in float-float
// (two-product and two-sum on the FP32 pipe); float64 vectors sum plainly.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
  // s + e += x with the rounding error of s + x kept in e (Knuth's two-sum)
  const float t = s + x;
  const float bp = t - s;
  e += (s - (t - bp)) + (x - bp);
  s = t;
}
__device__ __forceinline__ void dot_acc(float& s, float& e, float a, float b) {
  const float p = a * b;
  e += fmaf(a, b, -p);  // exact product error (fused multiply-add)
  two_sum_acc(s, e, p);
}
__device__ __forceinline__ void dot_acc(double& s, double& e, double a, double b) {
  s = fma(a, b, s);
}

// R = -G, Dx = 0; rr = <R,R>, rz = <R, Minv R>; tol2 = eta^2 rr. Also packs the
// incidence coefficients (meta may be null).
template <typename Tc>
__global__ void __launch_bounds__(256)
k_cg_init(const double* __restrict__ G, const Tc* __restrict__ Minv, Tc* __restrict__ R,
          Tc* __restrict__ Dx, int64_t n, int ld, double eta, int maxit,
          const int2* __restrict__ inc, const uint8_t* __restrict__ kind,
          const Tc* __restrict__ alpha, IncMeta<Tc>* __restrict__ meta, int64_t ninc,
          double* partials, Ctl* ctl) {
  // rr = <R, R>, rz = <R, Minv R> as in k_cg_update (float-float sums of the
  // operator-precision products; one row index per quad: ld is a multiple of 4)
  Tc rr_t = (Tc)0, rr_e = (Tc)0, rz_t = (Tc)0, rz_e = (Tc)0;
  const int64_t total = n * ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; t4 < total;
       t4 += stride * 4) {
    double g[4];
    Vec4<double>::load(G + t4, g);
    const Tc mi = Minv[t4 / ld];
    Tc r[4], z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      r[k] = (Tc)(-g[k]);
      z[k] = (Tc)0;
      dot_acc(rr_t, rr_e, r[k], r[k]);
      dot_acc(rz_t, rz_e, mi * r[k], r[k]);
    }
    Vec4<Tc>::store(R + t4, r);
    Vec4<Tc>::store(Dx + t4, z);
  }
  double acc[2] = {(double)rr_t + (double)rr_e, (double)rz_t + (double)rz_e};
  if (meta)
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ninc; t += stride) {
      const int2 eo = inc[t];
      if (!inc_ok(eo, B_CG_INIT, t)) {
        meta[t] = IncMeta<Tc>{(Tc)0, (Tc)0};  // the record is skipped
        continue;
      }
      const uint8_t kd = kind[eo.x];
      IncMeta<Tc> mm;
      mm.c = kd == K_IN ? (Tc)1
             : (kd == K_OUT ? -alpha[eo.x]
                : (kd == K_MASK ? (Tc)2
                   : ((kd == K_LINF && alpha[eo.x] > (Tc)0) ? (Tc)3 : (Tc)0)));
      mm.mo = Minv[eo.y];
      meta[t] = mm;
    }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_CGI], tot) && threadIdx.x == 0) {
    CgCtl& c = ctl->cg;
    c.rr = tot[0];
    c.rz = tot[1];
    c.tol2 = eta * eta * tot[0];
    c.alpha = 0.0;
    c.beta = 0.0;
    c.it = 0;
    c.maxit = maxit;
    c.active = (tot[0] > c.tol2 && maxit > 0 && tot[1] > 0.0) ? 1 : 0;
  }
}

// alpha of the current iteration from delta = <V u, u> (last block of a matvec)
__device__ __forceinline__ void cg_set_alpha(Ctl* ctl, double delta) {
  CgCtl& c = ctl->cg;
  const double den = c.it > 0 ? delta - c.beta * c.rz / c.alpha : delta;
  if (den > 0.0 && isfinite(den)) {
    c.alpha = c.rz / den;
  } else {
    c.alpha = 0.0;
    c.active = 0;  // breakdown: keep the current iterate
  }
}


template <int LANES, int CH, typename Tc>
__device__ __forceinline__ void matvec_term(Tc c, Tc mo, const Tc (&u)[CH][4], const Tc (&v0)[CH][4],
                                            const Tc (&yh)[CH][4], Tc (&accv)[CH][4],
                                            unsigned mask) {
  Tc v[CH][4];
#pragma unroll
  for (int cc = 0; cc < CH; ++cc)
#pragma unroll
    for (int k = 0; k < 4; ++k) v[cc][k] = u[cc][k] - mo * v0[cc][k];
  if (c > (Tc)2.5) {  // q = inf: diag(s != 0) - s s^T
    Tc sdot = (Tc)0;
#pragma unroll
    for (int cc = 0; cc < CH; ++cc)
#pragma unroll
      for (int k = 0; k < 4; ++k) sdot += yh[cc][k] * v[cc][k];
    sdot = group_sum<LANES>(sdot, mask);
#pragma unroll
    for (int cc = 0; cc < CH; ++cc)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        accv[cc][k] += (yh[cc][k] != (Tc)0 ? v[cc][k] : (Tc)0) - sdot * yh[cc][k];
  } else if (c > (Tc)1.5) {  // q = 1: diagonal mask
#pragma unroll
    for (int cc = 0; cc < CH; ++cc)
#pragma unroll
      for (int k = 0; k < 4; ++k) accv[cc][k] += yh[cc][k] * v[cc][k];
  } else if (c < (Tc)0) {  // outside: -c (I - yhat yhat^T)
    Tc sdot = (Tc)0;
#pragma unroll
    for (int cc = 0; cc < CH; ++cc)
#pragma unroll
      for (int k = 0; k < 4; ++k) sdot += yh[cc][k] * v[cc][k];
    sdot = group_sum<LANES>(sdot, mask);
    const Tc a = -c;
#pragma unroll
    for (int cc = 0; cc < CH; ++cc)
#pragma unroll
      for (int k = 0; k < 4; ++k) accv[cc][k] += a * (v[cc][k] - sdot * yh[cc][k]);
  } else if (c > (Tc)0) {  // inside: I
#pragma unroll
    for (int cc = 0; cc < CH; ++cc)
#pragma unroll
      for (int k = 0; k < 4; ++k) accv[cc][k] += v[cc][k];
  }
}

// W = D u + sigma B^T P B u with u = Minv R (D = I, or the diagonal Dg);
// delta = <W, u>. Node-parallel pull over the CSR of B^T: a group of LANES
// threads owns node i and visits its incidences in increasing edge id,
// gathering the other endpoint's R row (and the yhat / mask / s row of the edge
// for the kinds that have one). Like k_node_grad, the group reads its node's
// incidence records and packed coefficients LANES at a time (one per lane) and
// keeps kNB gathered rows in flight; the terms are still added in edge-id
// order. Used for short rows and the adjoint; k_cg_matvec_ring stages long rows
// through shared memory. The dot product <W, u> is accumulated exactly in
// float-float form (two_prod / two_sum) per lane, then in float64.
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_cg_matvec(const Tc* __restrict__ R, const Tc* __restrict__ Minv, const Tc* __restrict__ Dg,
            Tc* __restrict__ W, const Tc* __restrict__ Yh, const IncMeta<Tc>* __restrict__ meta,
            const int64_t* __restrict__ off, const int2* __restrict__ inc, double sigma,
            int64_t n, int ld, double* partials, Ctl* ctl, const int* __restrict__ ord) {
  if (!ctl->cg.active) return;
  constexpr int NB = GatherDepth<CH>::v;
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const Tc sg = (Tc)sigma;
  Tc dot = (Tc)0, dot_e = (Tc)0;  // <W, u> over this thread's elements, float-float
  // Dependent loads are pipelined across the group's nodes and record batches:
  // the next node's row range (and the index of the one after it) is loaded at
  // the start of a node, and every batch of LANES incidence records is loaded
  // one batch ahead (the first batch of the next node during the last batch of
  // this one), so the row gathers wait on at most one round trip to memory.
  auto node_of = [&](int64_t gi) -> int64_t {
    return gi < n ? (ord ? (int64_t)ord[gi] : gi) : 0;
  };
  auto records = [&](int64_t pb, int64_t pe, int2& rec, IncMeta<Tc>& mm) {
    rec = make_int2(0, 0);
    mm.c = (Tc)0;
    mm.mo = (Tc)0;
    if (pb + lane < pe) {
      rec = inc[pb + lane];
      mm = meta[pb + lane];
    }
  };
  int64_t i_cur = node_of(g0);
  int64_t b_cur = g0 < n ? off[i_cur] : 0, e_cur = g0 < n ? off[i_cur + 1] : 0;
  int64_t i_nxt = node_of(g0 + ng);
  int2 rec;
  IncMeta<Tc> mm;
  records(b_cur, e_cur, rec, mm);
  for (int64_t gi = g0; gi < n; gi += ng) {
    const int64_t i = i_cur, b = b_cur, eend = e_cur;
    int64_t bn = 0, en = 0;  // the next node's row range
    if (gi + ng < n) {
      bn = off[i_nxt];
      en = off[i_nxt + 1];
    }
    i_cur = i_nxt;
    i_nxt = node_of(gi + 2 * ng);
    b_cur = bn;
    e_cur = en;
    Tc u[CH][4], accv[CH][4];
    const Tc mi = Minv[i];
    row_load<LANES, CH>(R + i * ld, ld, lane, u);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        u[c][k] *= mi;
        accv[c][k] = (Tc)0;
      }
    if (eend <= b) records(bn, en, rec, mm);  // no batch of this node prefetches the next
    for (int64_t base = b; base < eend; base += LANES) {
      const int nb = (int)(eend - base < (int64_t)LANES ? eend - base : (int64_t)LANES);
      int2 rec_n;
      IncMeta<Tc> mm_n;
      if (base + LANES < eend)
        records(base + LANES, eend, rec_n, mm_n);
      else
        records(bn, en, rec_n, mm_n);
      for (int j = 0; j < nb; j += NB) {
        Tc v0[NB][CH][4], yh[NB][CH][4];
        Tc cs[NB], mos[NB];
#pragma unroll
        for (int kk = 0; kk < NB; ++kk) {
          const int ex = __shfl_sync(mask, rec.x, j + kk, LANES);
          const int ey = __shfl_sync(mask, rec.y, j + kk, LANES);
          cs[kk] = __shfl_sync(mask, mm.c, j + kk, LANES);
          mos[kk] = __shfl_sync(mask, mm.mo, j + kk, LANES);
          if (j + kk >= nb || !inc_ok(make_int2(ex, ey), B_MATVEC, base + j + kk)) cs[kk] = (Tc)0;
          if (cs[kk] != (Tc)0) {
            row_load<LANES, CH>(R + (int64_t)ey * ld, ld, lane, v0[kk]);
          } else {
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) v0[kk][c][k] = (Tc)0;
          }
          if (cs[kk] < (Tc)0 || cs[kk] > (Tc)1.5) {
            row_load<LANES, CH>(Yh + (int64_t)ex * ld, ld, lane, yh[kk]);
          } else {
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) yh[kk][c][k] = (Tc)0;
          }
        }
#pragma unroll
        for (int kk = 0; kk < NB; ++kk)
          matvec_term<LANES, CH, Tc>(cs[kk], mos[kk], u, v0[kk], yh[kk], accv, mask);
      }
      rec = rec_n;
      mm = mm_n;
    }
    const Tc di = Dg ? Dg[i] : (Tc)1;  // diagonal term (1 for V; cluster sizes for the adjoint)
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        accv[c][k] = di * u[c][k] + sg * accv[c][k];
        dot_acc(dot, dot_e, u[c][k], accv[c][k]);
      }
    row_store<LANES, CH>(W + i * ld, ld, lane, accv);
  }
  double acc[1] = {(double)dot + (double)dot_e};
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_MV], tot) && threadIdx.x == 0)
    cg_set_alpha(ctl, tot[0]);
}

// P = u + beta P, S = W + beta S (u = Minv R; P = u, S = W on the first
// iteration), Dx += alpha P, R -= alpha S; rz = <R, Minv R>, rr = <R,R>;
// beta and the stop test for the next iteration. With the coarse correction
// (Uc non-null) u = Uc = M^-1 R was formed before the operator, and rz and beta
// of the next iteration come from that step (coarse_precondition), not here.
template <typename Tc>
__global__ void __launch_bounds__(256)
k_cg_update(Tc* __restrict__ Dx, Tc* __restrict__ P, Tc* __restrict__ S, Tc* __restrict__ R,
            const Tc* __restrict__ W, const Tc* __restrict__ Minv, int64_t n, int ld,
            double* partials, Ctl* ctl, const Tc* __restrict__ Uc = nullptr) {
  if (!ctl->cg.active) return;
  const Tc al = (Tc)ctl->cg.alpha;
  const Tc be = (Tc)ctl->cg.beta;
  const bool first = ctl->cg.it == 0;
  // a thread's products are summed exactly enough in float-float (two-product and
  // two-sum on the FP32 pipe; plain sums for float64 vectors), then once in
  // float64: float64 arithmetic per element would occupy B300's narrow FP64 pipe
  Tc rz_t = (Tc)0, rz_e = (Tc)0, rr_t = (Tc)0, rr_e = (Tc)0;
  const int64_t total = n * ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; t4 < total;
       t4 += stride * 4) {
    Tc dx[4], p[4], sv[4], r[4], w[4];
    Vec4<Tc>::load(Dx + t4, dx);
    Vec4<Tc>::load(R + t4, r);
    Vec4<Tc>::load(W + t4, w);
    const Tc mi = Minv[t4 / ld];
    Tc u[4];
    if (Uc) {
      Vec4<Tc>::load(Uc + t4, u);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) u[k] = mi * r[k];
    }
    if (first) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        p[k] = u[k];
        sv[k] = w[k];
      }
    } else {
      Vec4<Tc>::load(P + t4, p);
      Vec4<Tc>::load(S + t4, sv);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        p[k] = u[k] + be * p[k];
        sv[k] = w[k] + be * sv[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dx[k] += al * p[k];
      r[k] -= al * sv[k];
      dot_acc(rr_t, rr_e, r[k], r[k]);
      dot_acc(rz_t, rz_e, mi * r[k], r[k]);
    }
    Vec4<Tc>::store(Dx + t4, dx);
    Vec4<Tc>::store(P + t4, p);
    Vec4<Tc>::store(S + t4, sv);
    Vec4<Tc>::store(R + t4, r);
  }
  double acc[2] = {(double)rz_t + (double)rz_e, (double)rr_t + (double)rr_e};
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_UPD], tot) && threadIdx.x == 0) {
    CgCtl& c = ctl->cg;
    c.it += 1;
    if (!Uc) {
      c.beta = (c.rz > 0.0) ? tot[0] / c.rz : 0.0;
      c.rz = tot[0];
    }
    c.rr = tot[1];
    if (!(tot[1] > c.tol2) || c.it >= c.maxit || !isfinite(tot[1]) || (!Uc && !(tot[0] > 0.0)))
      c.active = 0;
  }
}

// ------------------------------------------------------------ line search
// Xt = X + t Dx; gd = <G, Dx>.
template <typename Tc>
__global__ void __launch_bounds__(256)
k_trial(const double* __restrict__ X, const Tc* __restrict__ Dx, const double* __restrict__ G,
        double t, double* __restrict__ Xt, int64_t total, double* partials, Ctl* ctl) {
  double acc[1] = {0.0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    double dx = (double)Dx[q];
    Xt[q] = X[q] + t * dx;
    acc[0] += G[q] * dx;
  }
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_TRIAL], tot) && threadIdx.x == 0)
    ctl->dots[0] = tot[0];
}

// ------------------------------------------------------------ KKT / objectives
// KKT edge pass fused with the next evaluation at the same (X, U): per edge
// bx = x_i - x_j feeds both the primal residual ||BX - prox_p(BX + U)||^2 and
// r_l ||bx|| (for f_p) and y = u + sigma bx with its kind, alpha, yhat, Pi(y)
// and h (as k_edge_eval). With v = u + bx and shrink = max(0, 1 - r/||v||),
// BX - prox_p(BX + U) = bx - shrink v.
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_kkt_edge_eval(const double* __restrict__ X, const double* __restrict__ U,
                const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
                double sigma, double* __restrict__ Ut, Tc* __restrict__ Yh,
                Tc* __restrict__ alpha, uint8_t* __restrict__ kind, int64_t m, int ld,
                double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // ||res||^2, sum r||bx||, sum h, #outside
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = edges[e];
    const double r = gamma * w[e];
    double bx[CH][4], u[CH][4], y[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, bx);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, y);
    row_load<LANES, CH>(U + e * ld, ld, lane, u);
    double sb = 0.0, sv = 0.0, ss = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bx[c][k] -= y[c][k];
        sb = fma(bx[c][k], bx[c][k], sb);
        y[c][k] = fma(sigma, bx[c][k], u[c][k]);
        ss = fma(y[c][k], y[c][k], ss);
        u[c][k] += bx[c][k];  // u now holds v = u + bx
        sv = fma(u[c][k], u[c][k], sv);
      }
    sb = group_sum<LANES>(sb, mask);
    sv = group_sum<LANES>(sv, mask);
    ss = group_sum<LANES>(ss, mask);
    // norms and their inverses from refined inverse square roots (zero rows: 0)
    const double rv = sv > 0.0 ? rsqrt_refined(sv) : 0.0;
    const double nv = sv * rv;
    const double shrink = (nv > r) ? 1.0 - r * rv : 0.0;
    double sres = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double res = fma(-shrink, u[c][k], bx[c][k]);
        sres = fma(res, res, sres);
      }
    acc[0] += sres;
    const double rs = ss > 0.0 ? rsqrt_refined(ss) : 0.0;
    const double ny = ss * rs;
    uint8_t kd;
    double scale, a;
    if (!(r > 0.0)) {
      kd = K_INERT; scale = 0.0; a = 0.0;
    } else if (ny <= r) {
      kd = K_IN; scale = 1.0; a = 1.0;
    } else {
      kd = K_OUT; scale = r * rs; a = scale;
    }
    if (lane == 0) {
      acc[1] += sb > 0.0 ? r * (sb * rsqrt_refined(sb)) : 0.0;
      acc[2] += (ny <= r) ? 0.5 * ss : r * ny - 0.5 * r * r;
      acc[3] += (kd == K_OUT) ? 1.0 : 0.0;
      kind[e] = kd;
      alpha[e] = (Tc)a;
    }
    if (kd == K_IN) {
      row_store<LANES, CH>(Ut + e * ld, ld, lane, y);  // Pi(y) = y inside the ball
    } else {
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) u[c][k] = scale * y[c][k];
      row_store<LANES, CH>(Ut + e * ld, ld, lane, u);
    }
    if (kd == K_OUT) {
      const Tc invc = to_operator<Tc>(rs);
      Tc yh[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) yh[c][k] = to_operator<Tc>(y[c][k]) * invc;
      row_store<LANES, CH>(Yh + e * ld, ld, lane, yh);
    }
  }
  double tot[4];
  if (grid_reduce<4>(acc, partials, &ctl->counter[C_KKT_E], tot) && threadIdx.x == 0) {
    ctl->kkt[0] = tot[0];
    ctl->kkt[1] = tot[1];
    ctl->eval[0] = tot[2];
    ctl->eval[3] = tot[3];
  }
}

// ------------------------------------------------------------ q = 1
// Model CCM with the l1 norm on the differences (Sec. 1 allows any q >= 1): the
// ball of the dual is ||u_l||_inf <= r_l, so Pi clamps each element to
// [-r_l, r_l], h_l(y) = sum_k huber_{r_l}(y_k), and P_l = diag(mask) with mask_k =
// 1 where |y_k| <= r_l. Per edge: Pi(y) -> Ut, the mask row -> Yh (stored only
// when some element is clamped: kind K_MASK, alpha = trace(P_l)/d), kind K_IN when
// no element is clamped, K_INERT when r_l = 0. Returns the number of elements
// still inside, for the caller.
template <int LANES, int CH, typename Tc>
__device__ __forceinline__ void q1_edge_outputs(const double (&y)[CH][4], double r, int d,
                                                int lane, int ld, unsigned mask, int64_t e,
                                                double* __restrict__ Ut, Tc* __restrict__ Yh,
                                                Tc* __restrict__ alpha,
                                                uint8_t* __restrict__ kind, double& hsum,
                                                double& nmask) {
  double pi[CH][4];
  Tc mk[CH][4];
  double h = 0.0;
  int nin = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double v = y[c][k], av = fabs(v);
      const bool in = av <= r;
      pi[c][k] = in ? v : copysign(r, v);
      h += in ? 0.5 * v * v : r * av - 0.5 * r * r;
      const bool real = 4 * (c * LANES + lane) + k < d;
      mk[c][k] = (in && real) ? (Tc)1 : (Tc)0;
      nin += (in && real) ? 1 : 0;
    }
  h = group_sum<LANES>(h, mask);
  nin = (int)group_sum<LANES>((double)nin, mask);
  uint8_t kd;
  if (!(r > 0.0)) kd = K_INERT;
  else if (nin == d) kd = K_IN;
  else kd = K_MASK;
  if (lane == 0) {
    hsum += h;
    nmask += kd == K_MASK ? 1.0 : 0.0;
    kind[e] = kd;
    alpha[e] = (Tc)((double)nin / (double)d);
  }
  row_store<LANES, CH>(Ut + e * ld, ld, lane, pi);
  if (kd == K_MASK) row_store<LANES, CH>(Yh + e * ld, ld, lane, mk);
}

// ------------------------------------------------------------ q = inf
// Model CCM with the max norm on the differences (Sec. 1 allows any q >= 1): the
// ball of the dual is ||u_l||_1 <= r_l. Outside it, Pi(v)_k = sign(v_k)
// max(|v_k| - theta, 0) with theta > 0 fixed by sum_k max(|v_k| - theta, 0) = r_l.
// h_l(y) = (||y||^2 - ||y - Pi(y)||^2)/2 (Moreau envelope; the same identity gives
// the q = 2 and q = 1 forms of h), and prox of r_l||.||_inf = I - Pi.

template <int LANES>
__device__ __forceinline__ double group_max(double x, unsigned mask) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(mask, x, o, LANES));
  return x;
}

// theta of the projection of the row v (d real elements, lanes of one group) onto
// {||u||_1 <= r}, for ||v||_1 = l1 > r > 0. Active-set iteration of Michelot
// (1986): theta = (sum over S of |v_k| - r)/|S|, then S <- {k : |v_k| > theta},
// from S = all d elements. theta never decreases (kept so under rounding by the
// max below), so S only shrinks and the loop ends within d + 1 passes. The
// butterfly sums are bitwise identical on all lanes, so every lane ends with the
// same theta and the same pass count.
template <int LANES, int CH>
__device__ __forceinline__ double l1ball_theta(const double (&v)[CH][4], double l1, double r,
                                               int d, unsigned mask) {
  double theta = (l1 - r) / (double)d;
  int cnt = d;
  for (int pass = 0; pass <= d; ++pass) {
    double sum = 0.0;
    int c = 0;
#pragma unroll
    for (int cc = 0; cc < CH; ++cc)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double av = fabs(v[cc][k]);
        if (av > theta) {
          sum += av;
          ++c;
        }
      }
    sum = group_sum<LANES>(sum, mask);
    c = group_sum<LANES>(c, mask);
    if (c == cnt || c == 0) break;
    cnt = c;
    theta = fmax(theta, (sum - r) / (double)c);
  }
  return theta;
}

// Pi(y) -> Ut, kind, alpha and (kind K_LINF) the unit vector s -> Yh for one edge
// row y; adds h_l to hsum and 1 to nout when y_l is outside the ball.
template <int LANES, int CH, typename Tc>
__device__ __forceinline__ void linf_edge_outputs(const double (&y)[CH][4], double r, int d,
                                                  int lane, int ld, unsigned mask, int64_t e,
                                                  double* __restrict__ Ut, Tc* __restrict__ Yh,
                                                  Tc* __restrict__ alpha,
                                                  uint8_t* __restrict__ kind, double& hsum,
                                                  double& nout) {
  double l1 = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int k = 0; k < 4; ++k) l1 += fabs(y[c][k]);
  l1 = group_sum<LANES>(l1, mask);
  uint8_t kd;
  double theta = 0.0;
  if (!(r > 0.0)) {
    kd = K_INERT;
  } else if (l1 <= r) {
    kd = K_IN;
  } else {
    kd = K_LINF;
    theta = l1ball_theta<LANES, CH>(y, l1, r, d, mask);
  }
  double pi[CH][4];
  double h = 0.0;
  int nsup = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double v = y[c][k];
      double p;
      if (kd == K_IN) p = v;
      else if (kd == K_INERT) p = 0.0;
      else p = copysign(fmax(fabs(v) - theta, 0.0), v);
      pi[c][k] = p;
      const double df = v - p;
      h += v * v - df * df;
      nsup += (p != 0.0) ? 1 : 0;
    }
  h = 0.5 * group_sum<LANES>(h, mask);
  if (kd == K_LINF) nsup = group_sum<LANES>(nsup, mask);
  if (lane == 0) {
    hsum += h;
    nout += kd == K_LINF ? 1.0 : 0.0;
    kind[e] = kd;
    alpha[e] = (Tc)(kd == K_LINF ? (double)max(nsup - 1, 0) / (double)d
                                 : (kd == K_IN ? 1.0 : 0.0));
  }
  row_store<LANES, CH>(Ut + e * ld, ld, lane, pi);
  if (kd == K_LINF) {
    const Tc iv = (Tc)(nsup > 0 ? 1.0 / sqrt((double)nsup) : 0.0);
    Tc sv[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        sv[c][k] = pi[c][k] != 0.0 ? (__double2hiint(y[c][k]) < 0 ? -iv : iv) : (Tc)0;
    row_store<LANES, CH>(Yh + e * ld, ld, lane, sv);
  }
}

// Edge pass of the evaluation for the separable-ball norms: Q = 1 (elementwise
// clamp) or Q = kQInf (l1-ball projection).
template <int Q, int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_edge_eval_qn(const double* __restrict__ X, const double* __restrict__ U,
               const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
               double sigma, double* __restrict__ Ut, Tc* __restrict__ Yh, Tc* __restrict__ alpha,
               uint8_t* __restrict__ kind, int64_t m, int d, int ld, double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  double acc[2] = {0.0, 0.0};
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = edges[e];
    const double r = gamma * w[e];
    double xi[CH][4], xj[CH][4], y[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, xi);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, xj);
    row_load<LANES, CH>(U + e * ld, ld, lane, y);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) y[c][k] = fma(sigma, xi[c][k] - xj[c][k], y[c][k]);
    if constexpr (Q == 1)
      q1_edge_outputs<LANES, CH, Tc>(y, r, d, lane, ld, mask, e, Ut, Yh, alpha, kind, acc[0],
                                     acc[1]);
    else
      linf_edge_outputs<LANES, CH, Tc>(y, r, d, lane, ld, mask, e, Ut, Yh, alpha, kind, acc[0],
                                       acc[1]);
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_EVAL_E], tot) && threadIdx.x == 0) {
    ctl->eval[0] = tot[0];
    ctl->eval[3] = tot[1];
  }
}

// KKT for Q = 1 or Q = kQInf fused with the next evaluation: primal residual
// bx - prox_p(bx + u) and r ||bx||_q for f_p, then the edge outputs. For q = 1 the
// prox is the soft threshold at r; for q = inf, bx - prox_p(v) = Pi(v) - u with
// v = u + bx (Moreau decomposition), and the penalty is r max_k |bx_k|.
template <int Q, int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_kkt_edge_eval_qn(const double* __restrict__ X, const double* __restrict__ U,
                   const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
                   double sigma, double* __restrict__ Ut, Tc* __restrict__ Yh,
                   Tc* __restrict__ alpha, uint8_t* __restrict__ kind, int64_t m, int d, int ld,
                   double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // ||res||^2, sum r||bx||_q, sum h, #outside edges
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = edges[e];
    const double r = gamma * w[e];
    double bx[CH][4], u[CH][4], y[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, bx);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, y);
    row_load<LANES, CH>(U + e * ld, ld, lane, u);
    double sres = 0.0, sq = 0.0;
    if constexpr (Q == 1) {
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          bx[c][k] -= y[c][k];
          sq += fabs(bx[c][k]);
          const double v = u[c][k] + bx[c][k];
          const double soft = copysign(fmax(fabs(v) - r, 0.0), v);
          const double res = bx[c][k] - soft;
          sres = fma(res, res, sres);
          y[c][k] = fma(sigma, bx[c][k], u[c][k]);
        }
      sq = group_sum<LANES>(sq, mask);
    } else {
      double l1 = 0.0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double b = bx[c][k] - y[c][k];
          sq = fmax(sq, fabs(b));
          y[c][k] = fma(sigma, b, u[c][k]);
          bx[c][k] = u[c][k] + b;  // bx now holds v = u + bx
          l1 += fabs(bx[c][k]);
        }
      sq = group_max<LANES>(sq, mask);
      l1 = group_sum<LANES>(l1, mask);
      const bool outside = r > 0.0 && l1 > r;
      const double theta = outside ? l1ball_theta<LANES, CH>(bx, l1, r, d, mask) : 0.0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double v = bx[c][k];
          const double p = outside ? copysign(fmax(fabs(v) - theta, 0.0), v)
                                   : (r > 0.0 ? v : 0.0);
          const double res = p - u[c][k];
          sres = fma(res, res, sres);
        }
    }
    acc[0] += sres;
    if (lane == 0) acc[1] += r * sq;
    if constexpr (Q == 1)
      q1_edge_outputs<LANES, CH, Tc>(y, r, d, lane, ld, mask, e, Ut, Yh, alpha, kind, acc[2],
                                     acc[3]);
    else
      linf_edge_outputs<LANES, CH, Tc>(y, r, d, lane, ld, mask, e, Ut, Yh, alpha, kind, acc[2],
                                       acc[3]);
  }
  double tot[4];
  if (grid_reduce<4>(acc, partials, &ctl->counter[C_KKT_E], tot) && threadIdx.x == 0) {
    ctl->kkt[0] = tot[0];
    ctl->kkt[1] = tot[1];
    ctl->eval[0] = tot[2];
    ctl->eval[3] = tot[3];
  }
}

// Per node: B^T U = G - (X - A); <A, B^T U>, ||B^T U||^2.
__global__ void __launch_bounds__(256)
k_kkt_node(const double* __restrict__ X, const double* __restrict__ Ap,
           const double* __restrict__ G, int64_t total, double* partials, Ctl* ctl);

// ||v||^2 -> ctl->dots[1]
__global__ void k_sumsq(const double* __restrict__ v, int64_t total, double* partials, Ctl* ctl);

// ------------------------------------------------------------ layout
__global__ void k_pad_rows(const double* __restrict__ src, double* __restrict__ dst, int64_t rows,
                           int d, int ld);
__global__ void k_unpad_rows(const double* __restrict__ src, double* __restrict__ dst,
                             int64_t rows, int d, int ld);

static constexpr int kMaxPartBlocksPerSm = 8;  // partial-sum slots per SM

// Register-form operator launch (grid sized to the node groups, at most 4 blocks per SM).
template <int L, int CH, typename Tc>
inline int launch_matvec_reg(Ctx* c, const Tc* R, const Tc* Minv, const Tc* Dg, Tc* W,
                             const Tc* Yh, const IncMeta<Tc>* meta, const int64_t* off,
                             const int2* inc, double sigma, int64_t n, int ld, double* part,
                             Ctl* ctl, cudaStream_t s, const int* ord = nullptr) {
  const int threads = 256;
  using GS = GatherShape<L, CH>;
  const int gpb = threads / GS::L;
  auto fn = k_cg_matvec<GS::L, GS::C, Tc>;
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((n + gpb - 1) / gpb, (int64_t)resident_grid(c, fn, threads)));
  fn<<<blocks, threads, 0, s>>>(R, Minv, Dg, W, Yh, meta, off, inc, sigma, n, ld, part, ctl, ord);
  CCM_COUNT(c);
  return CCM_OK;
}

}  // namespace ccm
