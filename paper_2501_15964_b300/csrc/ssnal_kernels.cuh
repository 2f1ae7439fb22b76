// SSNAL building blocks for model CCM, q = 2 (Sec. 1 names the method).
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
#include "tma.cuh"

namespace ccm {

enum EdgeKind : uint8_t { K_INERT = 0, K_IN = 1, K_OUT = 2 };

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
  unsigned fault;   // nonzero: a bounded device-side wait gave up
};
enum CounterId { C_EVAL_E = 0, C_EVAL_N, C_CGI, C_MV, C_UPD, C_TRIAL, C_KKT_E, C_KKT_N };

struct GridShape {
  int blocks, threads;
};

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
    double h = (ny <= r) ? 0.5 * ss : r * ny - 0.5 * r * r;
    if (lane == 0) {
      acc[0] += h;
      acc[1] += (kd == K_OUT) ? 1.0 : 0.0;
      kind[e] = kd;
      alpha[e] = (Tc)a;
    }
    double o[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) o[c][k] = scale * y[c][k];
    row_store<LANES, CH>(Ut + e * ld, ld, lane, o);
    if (kd == K_OUT) {
      // yhat in the operator's precision: for float32 the scaling runs in
      // float32 (FP64 throughput is the limit of this kernel)
      const double inv = 1.0 / ny;
      const Tc invc = (Tc)inv;
      Tc yh[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) yh[c][k] = (Tc)y[c][k] * invc;
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
// with t_l = 1 (inside) or alpha_l (d-1)/d (outside) = trace(P_l)/d.
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_node_grad(const double* __restrict__ X, const double* __restrict__ Ap,
            const double* __restrict__ Ut, const int64_t* __restrict__ off,
            const int2* __restrict__ inc, const Tc* __restrict__ alpha,
            const uint8_t* __restrict__ kind, double sigma, int d, double* __restrict__ G,
            Tc* __restrict__ Minv, int64_t n, int ld, double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const double tr_out = (double)(d - 1) / (double)d;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = g0; i < n; i += ng) {
    const int64_t b = off[i], eend = off[i + 1];
    // one quad per lane at a time: few registers, many warps in flight; the
    // incidence list is re-read per chunk from L1. Every element still sums
    // its incident edges in increasing edge id (same order as before).
#pragma unroll 1
    for (int c = 0; c < CH; ++c) {
      const int q = c * LANES + lane;
      if (4 * q >= ld) break;
      double g[4], a[4];
      Vec4<double>::load(X + i * ld + 4 * q, g);
      Vec4<double>::load(Ap + i * ld + 4 * q, a);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        g[k] -= a[k];
        acc[1] += 0.5 * g[k] * g[k];
      }
      int64_t t = b;
      for (; t + 1 < eend; t += 2) {  // two incidences in flight
        const int2 e0 = inc[t], e1 = inc[t + 1];
        double u0[4], u1[4];
        Vec4<double>::load(Ut + (int64_t)e0.x * ld + 4 * q, u0);
        Vec4<double>::load(Ut + (int64_t)e1.x * ld + 4 * q, u1);
        const double s0 = (i < e0.y) ? 1.0 : -1.0, s1 = (i < e1.y) ? 1.0 : -1.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] += s0 * u0[k];
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] += s1 * u1[k];
      }
      if (t < eend) {
        const int2 e0 = inc[t];
        double u0[4];
        Vec4<double>::load(Ut + (int64_t)e0.x * ld + 4 * q, u0);
        const double s0 = (i < e0.y) ? 1.0 : -1.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] += s0 * u0[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[0] += g[k] * g[k];
      Vec4<double>::store(G + i * ld + 4 * q, g);
    }
    if (lane == 0) {
      double diag = 0.0;
      for (int64_t t = b; t < eend; ++t) {
        const int e = inc[t].x;
        const uint8_t kd = kind[e];
        diag += kd == K_IN ? 1.0 : (kd == K_OUT ? (double)alpha[e] * tr_out : 0.0);
      }
      Minv[i] = (Tc)(1.0 / (1.0 + sigma * diag));
    }
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_EVAL_N], tot) && threadIdx.x == 0) {
    ctl->eval[2] = tot[0];
    ctl->eval[1] = tot[1];
  }
}

// Node gradient for long rows (LANES = 32): one warp per node over the
// contiguous node ranges of wpart (as the bulk-copy operator). Lane 0 streams
// the Ut row of every non-inert incidence into a per-warp ring of shared-memory
// slots with 1-D bulk copies (one mbarrier per slot); the slot metadata carries
// the other endpoint (for the sign: + when node i is the first endpoint) and
// trace(P_l)/d. Sums run in increasing edge id, as in k_node_grad.
struct GradMeta {
  double t;   // trace(P_l)/d
  int other;  // other endpoint of the incidence
  int live;   // 0: inert edge (no row copied)
};

template <int CH, typename Tc>
__global__ void __launch_bounds__(256, 1)
k_node_grad_tma(const double* __restrict__ X, const double* __restrict__ Ap,
                const double* __restrict__ Ut, const int64_t* __restrict__ off,
                const int2* __restrict__ inc, const Tc* __restrict__ alpha,
                const uint8_t* __restrict__ kind, double sigma, int d, double* __restrict__ G,
                Tc* __restrict__ Minv, const int* __restrict__ wpart, int64_t n, int ld,
                int stages, double* partials, Ctl* ctl) {
  constexpr int LANES = 32;
  extern __shared__ __align__(128) unsigned char smem[];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * nw + warp;
  const uint32_t rowb = (uint32_t)ld * 8u;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + (size_t)warp * stages;
  GradMeta* smeta = reinterpret_cast<GradMeta*>(smem + (size_t)nw * stages * 8) +
                    (size_t)warp * stages;
  double* ring = reinterpret_cast<double*>(smem + tma_ring_header(nw, stages, sizeof(GradMeta))) +
                 (size_t)warp * stages * ld;
  if (lane == 0) {
    for (int q = 0; q < stages; ++q) mbar_init(smem_u32(bars + q), 1);
    fence_mbar_init();
  }
  __syncwarp();
  const double tr_out = (double)(d - 1) / (double)d;
  const int64_t nbeg = wpart[gw], nend = wpart[gw + 1];
  const int64_t kb = off[nbeg], ke = off[nend];

  int2 c_eo, n_eo;
  double c_t, n_t;
  auto fetch = [&](int64_t base, int2& eo, double& t) {
    const int64_t k = base + lane;
    eo = make_int2(0, 0);
    t = -1.0;  // inert
    if (k < ke) {
      eo = inc[k];
      const uint8_t kd = kind[eo.x];
      t = kd == K_IN ? 1.0 : (kd == K_OUT ? (double)alpha[eo.x] * tr_out : -1.0);
    }
  };
  fetch(kb, c_eo, c_t);
  fetch(kb + 32, n_eo, n_t);
  int64_t c_base = kb, pk = kb;
  int pslot = 0;
  auto issue = [&]() {
    if (pk >= ke) return;
    if (pk - c_base >= 32) {
      c_eo = n_eo;
      c_t = n_t;
      c_base += 32;
      fetch(c_base + 32, n_eo, n_t);
    }
    const int src = (int)(pk - c_base);
    const int ex = __shfl_sync(0xffffffffu, c_eo.x, src);
    const int ey = __shfl_sync(0xffffffffu, c_eo.y, src);
    const double t = __shfl_sync(0xffffffffu, c_t, src);
    if (lane == 0) {
      GradMeta gm;
      gm.t = t < 0.0 ? 0.0 : t;
      gm.other = ey;
      gm.live = t < 0.0 ? 0 : 1;
      smeta[pslot] = gm;
      const uint32_t bar = smem_u32(bars + pslot);
      if (!gm.live) {
        mbar_arrive(bar);
      } else {
        mbar_arrive_tx(bar, rowb);
        bulk_g2s(smem_u32(ring + (size_t)pslot * ld), Ut + (int64_t)ex * ld, rowb, bar);
      }
    }
    ++pk;
    if (++pslot == stages) pslot = 0;
  };
  for (int q = 0; q < stages; ++q) issue();
  __syncwarp();

  int cslot = 0;
  uint32_t cpar = 0;
  int64_t ck = kb;
  bool ok = true;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = nbeg; i < nend; ++i) {
    const int64_t eend = off[i + 1];
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
    for (; ck < eend && ok; ++ck) {
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(bars + cslot), cpar))) {
        ok = false;
        if (lane == 0) atomicOr(&ctl->fault, 1u);
        break;
      }
      const GradMeta gm = smeta[cslot];
      if (gm.live) {
        const double* ur = ring + (size_t)cslot * ld;
        const double sg = (i < gm.other) ? 1.0 : -1.0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int q = c * LANES + lane;
          if (4 * q < ld) {
            double u4[4];
            Vec4<double>::load(ur + 4 * q, u4);
#pragma unroll
            for (int k = 0; k < 4; ++k) g[c][k] += sg * u4[k];
          }
        }
        diag += gm.t;
      }
      __syncwarp();
      if (++cslot == stages) {
        cslot = 0;
        cpar ^= 1u;
      }
      issue();
    }
    if (!ok) break;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[0] += g[c][k] * g[c][k];
    row_store<LANES, CH>(G + i * ld, ld, lane, g);
    if (lane == 0) Minv[i] = (Tc)(1.0 / (1.0 + sigma * diag));
  }
  if (!ok) {
    for (; ck < pk; ++ck) {
      mbar_wait(smem_u32(bars + cslot), cpar);
      if (++cslot == stages) {
        cslot = 0;
        cpar ^= 1u;
      }
    }
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
// c = 0 (inert edge); mo = Minv of the incidence's other endpoint.
template <typename Tc>
struct alignas(2 * sizeof(Tc)) IncMeta {
  Tc c, mo;
};

// R = -G, Dx = 0; rr = <R,R>, rz = <R, Minv R>; tol2 = eta^2 rr. Also packs the
// incidence coefficients (meta may be null).
template <typename Tc>
__global__ void __launch_bounds__(256)
k_cg_init(const double* __restrict__ G, const Tc* __restrict__ Minv, Tc* __restrict__ R,
          Tc* __restrict__ Dx, int64_t n, int ld, double eta, int maxit,
          const int2* __restrict__ inc, const uint8_t* __restrict__ kind,
          const Tc* __restrict__ alpha, IncMeta<Tc>* __restrict__ meta, int64_t ninc,
          double* partials, Ctl* ctl) {
  double acc[2] = {0.0, 0.0};
  const int64_t total = n * ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    Tc r = (Tc)(-G[t]);
    R[t] = r;
    Dx[t] = (Tc)0;
    double rd = (double)r;
    acc[0] += rd * rd;
    acc[1] += rd * rd * (double)Minv[t / ld];
  }
  if (meta)
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ninc; t += stride) {
      const int2 eo = inc[t];
      const uint8_t kd = kind[eo.x];
      IncMeta<Tc> mm;
      mm.c = kd == K_IN ? (Tc)1 : (kd == K_OUT ? -alpha[eo.x] : (Tc)0);
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

// W = D u + sigma B^T P B u with u = Minv R (D = I, or the diagonal Dg);
// delta = <W, u>. Node-parallel pull over the CSR of B^T: a group of LANES
// threads owns node i and visits its incidences in increasing edge id,
// gathering the other endpoint's R row (and yhat_l for outside edges) into
// registers. Used for short rows; k_cg_matvec_tma stages long rows through
// shared memory with bulk copies.
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_cg_matvec(const Tc* __restrict__ R, const Tc* __restrict__ Minv, const Tc* __restrict__ Dg,
            Tc* __restrict__ W, const Tc* __restrict__ Yh, const IncMeta<Tc>* __restrict__ meta,
            const int64_t* __restrict__ off, const int2* __restrict__ inc, double sigma,
            int64_t n, int ld, double* partials, Ctl* ctl) {
  if (!ctl->cg.active) return;
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const Tc sg = (Tc)sigma;
  double acc[1] = {0.0};
  for (int64_t i = g0; i < n; i += ng) {
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
    const int64_t b = off[i], eend = off[i + 1];
    // the next incidence and its coefficients are fetched one iteration ahead
    int2 eo_n = make_int2(0, 0);
    IncMeta<Tc> mm_n;
    mm_n.c = (Tc)0;
    mm_n.mo = (Tc)0;
    if (b < eend) {
      eo_n = inc[b];
      mm_n = meta[b];
    }
    for (int64_t t = b; t < eend; ++t) {
      const int2 eo = eo_n;
      const IncMeta<Tc> mm = mm_n;
      if (t + 1 < eend) {
        eo_n = inc[t + 1];
        mm_n = meta[t + 1];
      }
      if (mm.c == (Tc)0) continue;
      Tc v[CH][4];
      row_load<LANES, CH>(R + (int64_t)eo.y * ld, ld, lane, v);
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[c][k] = u[c][k] - mm.mo * v[c][k];
      if (mm.c < (Tc)0) {
        Tc yh[CH][4];
        row_load<LANES, CH>(Yh + (int64_t)eo.x * ld, ld, lane, yh);
        Tc s = (Tc)0;
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) s += yh[c][k] * v[c][k];
        s = group_sum<LANES>(s, mask);
        const Tc a = -mm.c;
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) accv[c][k] += a * (v[c][k] - s * yh[c][k]);
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) accv[c][k] += v[c][k];
      }
    }
    Tc dot = (Tc)0;
    const Tc di = Dg ? Dg[i] : (Tc)1;  // diagonal term (1 for V; cluster sizes for the adjoint)
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        accv[c][k] = di * u[c][k] + sg * accv[c][k];
        dot += u[c][k] * accv[c][k];
      }
    acc[0] += (double)dot;
    row_store<LANES, CH>(W + i * ld, ld, lane, accv);
  }
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_MV], tot) && threadIdx.x == 0)
    cg_set_alpha(ctl, tot[0]);
}

// The operator of k_cg_matvec for long rows (one warp per node, LANES = 32).
// Each warp owns a contiguous node range (balanced by incidences + 2 per node,
// wpart) and so a contiguous run of CSR incidences. Its lane 0 streams the
// other endpoint's R row and, for outside edges, the yhat row of every
// incidence into a per-warp ring of `stages` shared-memory slots with 1-D bulk
// copies, each slot completing on its own mbarrier; the 32 lanes consume the
// slots in order and refill each one as soon as they have read it, so `stages`
// incidences per warp are always in flight and no row is held in registers
// while it is in flight. Incidence records come in lane-parallel batches of 32,
// prefetched one batch ahead. Waits are bounded (ctl->fault records a timeout;
// the warp then drains its own copies, also bounded, and stops computing).
// Shared memory: header of nw*stages (mbarrier + IncMeta), then
// nw*stages*2*ld elements of Tc.

template <int CH, typename Tc>
__global__ void __launch_bounds__(256, 1)
k_cg_matvec_tma(const Tc* __restrict__ R, const Tc* __restrict__ Minv, const Tc* __restrict__ Dg,
                Tc* __restrict__ W, const Tc* __restrict__ Yh,
                const IncMeta<Tc>* __restrict__ meta, const int64_t* __restrict__ off,
                const int2* __restrict__ inc, const int* __restrict__ wpart, double sigma,
                int64_t n, int ld, int stages, double* partials, Ctl* ctl) {
  constexpr int LANES = 32;
  extern __shared__ __align__(128) unsigned char smem[];
  if (!ctl->cg.active) return;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * nw + warp;
  const uint32_t rowb = (uint32_t)ld * (uint32_t)sizeof(Tc);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + (size_t)warp * stages;
  IncMeta<Tc>* smeta = reinterpret_cast<IncMeta<Tc>*>(smem + (size_t)nw * stages * 8) +
                       (size_t)warp * stages;
  Tc* ring = reinterpret_cast<Tc*>(smem + tma_ring_header(nw, stages, sizeof(IncMeta<Tc>))) +
             (size_t)warp * stages * 2 * ld;
  if (lane == 0) {
    for (int q = 0; q < stages; ++q) mbar_init(smem_u32(bars + q), 1);
    fence_mbar_init();
  }
  __syncwarp();

  const int64_t nbeg = wpart[gw], nend = wpart[gw + 1];
  const int64_t kb = off[nbeg], ke = off[nend];

  // ---- producer state (warp-uniform; lane 0 issues)
  int2 c_eo, n_eo;
  IncMeta<Tc> c_m, n_m;
  auto fetch = [&](int64_t base, int2& eo, IncMeta<Tc>& mm) {
    const int64_t k = base + lane;
    if (k < ke) {
      eo = inc[k];
      mm = meta[k];
    } else {
      eo = make_int2(0, 0);
      mm.c = (Tc)0;
      mm.mo = (Tc)0;
    }
  };
  fetch(kb, c_eo, c_m);
  fetch(kb + 32, n_eo, n_m);
  int64_t c_base = kb, pk = kb;
  int pslot = 0;
  // R rows are gathered by every neighbour: keep them in L2; yhat rows stream
  const uint64_t pol_keep = l2_policy_evict_last(), pol_stream = l2_policy_evict_first();
  auto issue = [&]() {
    if (pk >= ke) return;
    if (pk - c_base >= 32) {
      c_eo = n_eo;
      c_m = n_m;
      c_base += 32;
      fetch(c_base + 32, n_eo, n_m);
    }
    const int src = (int)(pk - c_base);
    const int ex = __shfl_sync(0xffffffffu, c_eo.x, src);
    const int ey = __shfl_sync(0xffffffffu, c_eo.y, src);
    const Tc mc = __shfl_sync(0xffffffffu, c_m.c, src);
    const Tc mo = __shfl_sync(0xffffffffu, c_m.mo, src);
    if (lane == 0) {
      smeta[pslot].c = mc;
      smeta[pslot].mo = mo;
      const uint32_t bar = smem_u32(bars + pslot);
      if (mc == (Tc)0) {
        mbar_arrive(bar);
      } else {
        Tc* dst = ring + (size_t)pslot * 2 * ld;
        const bool out = mc < (Tc)0;
        mbar_arrive_tx(bar, out ? 2u * rowb : rowb);
        bulk_g2s_hint(smem_u32(dst), R + (int64_t)ey * ld, rowb, bar, pol_keep);
        if (out) bulk_g2s_hint(smem_u32(dst + ld), Yh + (int64_t)ex * ld, rowb, bar, pol_stream);
      }
    }
    ++pk;
    if (++pslot == stages) pslot = 0;
  };
  for (int q = 0; q < stages; ++q) issue();
  __syncwarp();  // lane 0's slot metadata before any lane reads it

  // ---- consumer
  const Tc sg = (Tc)sigma;
  int cslot = 0;
  uint32_t cpar = 0;
  int64_t ck = kb;
  bool ok = true;
  double acc[1] = {0.0};
  for (int64_t i = nbeg; i < nend; ++i) {
    const int64_t eend = off[i + 1];
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
    for (; ck < eend && ok; ++ck) {
      // the warp agrees on the outcome (a lane that gave up stops all of them)
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(bars + cslot), cpar))) {
        ok = false;
        if (lane == 0) atomicOr(&ctl->fault, 1u);
        break;
      }
      const IncMeta<Tc> mm = smeta[cslot];
      if (mm.c != (Tc)0) {
        const Tc* rr = ring + (size_t)cslot * 2 * ld;
        Tc v[CH][4];
        row_load<LANES, CH>(rr, ld, lane, v);
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) v[c][k] = u[c][k] - mm.mo * v[c][k];
        if (mm.c < (Tc)0) {
          // yhat is read twice from shared memory rather than held in registers
          const Tc* yy = rr + ld;
          Tc s = (Tc)0;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int q = c * LANES + lane;
            if (4 * q < ld) {
              Tc y4[4];
              Vec4<Tc>::load(yy + 4 * q, y4);
#pragma unroll
              for (int k = 0; k < 4; ++k) s += y4[k] * v[c][k];
            }
          }
          s = group_sum<LANES>(s, 0xffffffffu);
          const Tc a = -mm.c;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int q = c * LANES + lane;
            if (4 * q < ld) {
              Tc y4[4];
              Vec4<Tc>::load(yy + 4 * q, y4);
#pragma unroll
              for (int k = 0; k < 4; ++k) accv[c][k] += a * (v[c][k] - s * y4[k]);
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) accv[c][k] += v[c][k];
        }
      }
      __syncwarp();
      if (++cslot == stages) {
        cslot = 0;
        cpar ^= 1u;
      }
      issue();  // refill the slot just read
    }
    if (!ok) break;
    Tc dot = (Tc)0;
    const Tc di = Dg ? Dg[i] : (Tc)1;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        accv[c][k] = di * u[c][k] + sg * accv[c][k];
        dot += u[c][k] * accv[c][k];
      }
    acc[0] += (double)dot;
    row_store<LANES, CH>(W + i * ld, ld, lane, accv);
  }
  if (!ok) {
    // drain this warp's copies still in flight (bounded) before the CTA exits
    for (; ck < pk; ++ck) {
      mbar_wait(smem_u32(bars + cslot), cpar);
      if (++cslot == stages) {
        cslot = 0;
        cpar ^= 1u;
      }
    }
  }
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_MV], tot) && threadIdx.x == 0)
    cg_set_alpha(ctl, tot[0]);
}

// P = u + beta P, S = W + beta S (u = Minv R; P = u, S = W on the first
// iteration), Dx += alpha P, R -= alpha S; rz = <R, Minv R>, rr = <R,R>;
// beta and the stop test for the next iteration.
template <typename Tc>
__global__ void __launch_bounds__(256)
k_cg_update(Tc* __restrict__ Dx, Tc* __restrict__ P, Tc* __restrict__ S, Tc* __restrict__ R,
            const Tc* __restrict__ W, const Tc* __restrict__ Minv, int64_t n, int ld,
            double* partials, Ctl* ctl) {
  if (!ctl->cg.active) return;
  const Tc al = (Tc)ctl->cg.alpha;
  const Tc be = (Tc)ctl->cg.beta;
  const bool first = ctl->cg.it == 0;
  double acc[2] = {0.0, 0.0};
  const int64_t total = n * ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; t4 < total;
       t4 += stride * 4) {
    Tc dx[4], p[4], sv[4], r[4], w[4];
    Vec4<Tc>::load(Dx + t4, dx);
    Vec4<Tc>::load(R + t4, r);
    Vec4<Tc>::load(W + t4, w);
    const Tc mi = Minv[t4 / ld];
    if (first) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        p[k] = mi * r[k];
        sv[k] = w[k];
      }
    } else {
      Vec4<Tc>::load(P + t4, p);
      Vec4<Tc>::load(S + t4, sv);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        p[k] = mi * r[k] + be * p[k];
        sv[k] = w[k] + be * sv[k];
      }
    }
    Tc rr = (Tc)0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dx[k] += al * p[k];
      r[k] -= al * sv[k];
      rr += r[k] * r[k];
    }
    Vec4<Tc>::store(Dx + t4, dx);
    Vec4<Tc>::store(P + t4, p);
    Vec4<Tc>::store(S + t4, sv);
    Vec4<Tc>::store(R + t4, r);
    acc[0] += (double)(mi * rr);
    acc[1] += (double)rr;
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_UPD], tot) && threadIdx.x == 0) {
    CgCtl& c = ctl->cg;
    c.it += 1;
    c.beta = (c.rz > 0.0) ? tot[0] / c.rz : 0.0;
    c.rz = tot[0];
    c.rr = tot[1];
    if (!(tot[1] > c.tol2) || c.it >= c.maxit || !isfinite(tot[1]) || !(tot[0] > 0.0))
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
// Per edge: BX_l, prox residual ||BX - prox_p(BX + U)||^2 and r_l ||BX_l||.
template <int LANES, int CH>
__global__ void __launch_bounds__(256)
k_kkt_edge(const double* __restrict__ X, const double* __restrict__ U,
           const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
           int64_t m, int ld, double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  double acc[2] = {0.0, 0.0};
  for (int64_t e = g0; e < m; e += ng) {
    int2 ij = edges[e];
    double r = gamma * w[e];
    double bx[CH][4], v[CH][4];
    row_load<LANES, CH>(X + (int64_t)ij.x * ld, ld, lane, bx);
    row_load<LANES, CH>(X + (int64_t)ij.y * ld, ld, lane, v);
    double sb = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bx[c][k] -= v[c][k];
        sb += bx[c][k] * bx[c][k];
      }
    row_load<LANES, CH>(U + e * ld, ld, lane, v);
    double sv = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[c][k] += bx[c][k];
        sv += v[c][k] * v[c][k];
      }
    sb = group_sum<LANES>(sb, mask);
    sv = group_sum<LANES>(sv, mask);
    double nv = sqrt(sv);
    double shrink = (nv > r) ? 1.0 - r / nv : 0.0;
    double sres = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double res = bx[c][k] - shrink * v[c][k];
        sres += res * res;
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

// KKT edge pass fused with the next evaluation at the same (X, U): per edge
// bx = x_i - x_j feeds both the prox residual / r||bx|| (as k_kkt_edge) and
// y = u + sigma bx with its kind, alpha, yhat, Pi(y) and h (as k_edge_eval).
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
        const double v = u[c][k] + bx[c][k];
        sv = fma(v, v, sv);
        y[c][k] = fma(sigma, bx[c][k], u[c][k]);
        ss = fma(y[c][k], y[c][k], ss);
      }
    sb = group_sum<LANES>(sb, mask);
    sv = group_sum<LANES>(sv, mask);
    ss = group_sum<LANES>(ss, mask);
    const double nv = sqrt(sv);
    const double shrink = (nv > r) ? 1.0 - r / nv : 0.0;
    double sres = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double res = bx[c][k] - shrink * (u[c][k] + bx[c][k]);
        sres = fma(res, res, sres);
      }
    acc[0] += sres;
    const double ny = sqrt(ss);
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
      acc[1] += r * sqrt(sb);
      acc[2] += (ny <= r) ? 0.5 * ss : r * ny - 0.5 * r * r;
      acc[3] += (kd == K_OUT) ? 1.0 : 0.0;
      kind[e] = kd;
      alpha[e] = (Tc)a;
    }
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) u[c][k] = scale * y[c][k];
    row_store<LANES, CH>(Ut + e * ld, ld, lane, u);
    if (kd == K_OUT) {
      const Tc invc = (Tc)(1.0 / ny);
      Tc yh[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) yh[c][k] = (Tc)y[c][k] * invc;
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

// Per node: B^T U = G - (X - A); <A, B^T U>, ||B^T U||^2.
__global__ void __launch_bounds__(256)
k_kkt_node(const double* __restrict__ X, const double* __restrict__ Ap,
           const double* __restrict__ G, int64_t total, double* partials, Ctl* ctl);

// ------------------------------------------------------------ layout
__global__ void k_pad_rows(const double* __restrict__ src, double* __restrict__ dst, int64_t rows,
                           int d, int ld);
__global__ void k_unpad_rows(const double* __restrict__ src, double* __restrict__ dst,
                             int64_t rows, int d, int ld);

static constexpr int kMaxPartBlocksPerSm = 8;  // partial-sum slots per SM

// Launch shape of the bulk-copy operator: nw warps per CTA, one CTA per SM
// (its shared memory fills most of one SM), `stages` ring slots per warp.
struct TmaShape {
  int nw = 0, stages = 0;
  size_t smem = 0;
};
template <typename Tc>
inline TmaShape tma_shape(int ld) {
  constexpr size_t kBudget = 200 * 1024;
  TmaShape sh;
  const size_t slot = 2 * (size_t)ld * sizeof(Tc);
  for (int nw : {8, 4}) {
    int st = (int)std::min<size_t>(8, kBudget / ((size_t)nw * slot));
    if (st >= 2) {
      sh.nw = nw;
      sh.stages = st;
      sh.smem = tma_ring_header(nw, st, sizeof(IncMeta<Tc>)) + (size_t)nw * st * slot;
      return sh;
    }
  }
  return sh;
}

// Shape of the bulk-copy node gradient with the operator's warps per CTA (so
// both share one node partition): float64 Ut rows, one per slot.
inline TmaShape grad_shape(const TmaShape& op, int ld) {
  constexpr size_t kBudget = 200 * 1024;
  TmaShape sh;
  if (op.nw <= 0) return sh;
  const size_t slot = (size_t)ld * 8;
  const int st = (int)std::min<size_t>(8, kBudget / ((size_t)op.nw * slot));
  if (st < 2) return sh;
  sh.nw = op.nw;
  sh.stages = st;
  sh.smem = tma_ring_header(op.nw, st, sizeof(GradMeta)) + (size_t)op.nw * st * slot;
  return sh;
}

// Node-gradient launch: the bulk-copy form when `wpart` and a shape are given.
template <int L, int CH, typename Tc>
inline int launch_node_grad(Ctx* c, const double* X, const double* Ap, const double* Ut,
                            const int64_t* off, const int2* inc, const Tc* alpha,
                            const uint8_t* kind, double sigma, int d, double* G, Tc* Minv,
                            const int* wpart, const TmaShape& sh, int64_t n, int ld,
                            double* part, Ctl* ctl, cudaStream_t s) {
  if (L == 32 && wpart && sh.nw > 0) {
    static size_t attr_set[64] = {};
    size_t& cur = attr_set[c->device & 63];
    if (cur < sh.smem) {
      CCM_CUDA(cudaFuncSetAttribute(k_node_grad_tma<CH, Tc>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
      cur = sh.smem;
    }
    k_node_grad_tma<CH, Tc><<<c->num_sms, sh.nw * 32, sh.smem, s>>>(
        X, Ap, Ut, off, inc, alpha, kind, sigma, d, G, Minv, wpart, n, ld, sh.stages, part, ctl);
  } else {
    const int threads = 256;
    const int gpb = threads / L;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + gpb - 1) / gpb, (int64_t)c->num_sms * 4));
    k_node_grad<L, CH, Tc><<<blocks, threads, 0, s>>>(X, Ap, Ut, off, inc, alpha, kind, sigma, d,
                                                      G, Minv, n, ld, part, ctl);
  }
  CCM_COUNT(c);
  return CCM_OK;
}

// Node ranges of the nwg warps of the bulk-copy operator, balanced by
// (incidences + 2 per node): part[w] = first node with off[i] + 2i >= w * total / nwg.
__global__ void k_warp_partition(const int64_t* __restrict__ off, int64_t n, int nwg,
                                 int* __restrict__ part);

// Operator launch: the bulk-copy form for rows of at least 32 quads (LANES = 32)
// when `wpart` is given, the register form otherwise.
template <int L, int CH, typename Tc>
inline int launch_matvec(Ctx* c, const Tc* R, const Tc* Minv, const Tc* Dg, Tc* W, const Tc* Yh,
                         const IncMeta<Tc>* meta, const int64_t* off, const int2* inc,
                         const int* wpart, const TmaShape& sh, double sigma, int64_t n, int ld,
                         double* part, Ctl* ctl, cudaStream_t s) {
  if (L == 32 && wpart && sh.nw > 0) {
    static size_t attr_set[64] = {};  // largest dynamic shared memory enabled, per device
    size_t& cur = attr_set[c->device & 63];
    if (cur < sh.smem) {
      CCM_CUDA(cudaFuncSetAttribute(k_cg_matvec_tma<CH, Tc>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
      cur = sh.smem;
    }
    k_cg_matvec_tma<CH, Tc><<<c->num_sms, sh.nw * 32, sh.smem, s>>>(
        R, Minv, Dg, W, Yh, meta, off, inc, wpart, sigma, n, ld, sh.stages, part, ctl);
  } else {
    const int threads = 256;
    const int gpb = threads / L;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + gpb - 1) / gpb, (int64_t)c->num_sms * 4));
    k_cg_matvec<L, CH, Tc><<<blocks, threads, 0, s>>>(R, Minv, Dg, W, Yh, meta, off, inc, sigma,
                                                      n, ld, part, ctl);
  }
  CCM_COUNT(c);
  return CCM_OK;
}

}  // namespace ccm
