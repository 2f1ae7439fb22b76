// Float-float forms of the q = 2 edge passes and of the node gradient (the
// mixed-precision grid engine; ff.cuh has the arithmetic).
//
// Storage in that engine: the multipliers U and the projected rows Pi(y) are
// float-float rows (float2 per element); X keeps its float64 rows (the line
// search, KKT node terms, labels and outputs read them) plus a float-float
// mirror XF written wherever X is written, which the edge passes gather. The
// operator's yhat rows and alpha stay in the operator's precision.
//
// Notation as in ssnal_kernels.cuh: y = u + sigma (x_i - x_j), Pi = projection
// onto {||u_l|| <= r_l}, h = ||y||^2/2 inside, r ||y|| - r^2/2 outside.
#pragma once

#include "ff.cuh"
#include "ring_kernels.cuh"
#include "ssnal_kernels.cuh"

namespace ccm {

// float64 rows (stride d) -> float-float rows (stride ld, zero padding), row r
// taken from source row idx[r] (negated when complemented; idx may be NULL)
__global__ void k_pad_rows_ff(const double* __restrict__ src, float2* __restrict__ dst,
                              int64_t rows, int d, int ld, const int* __restrict__ idx);
// float-float rows (stride ld) -> float64 rows (stride d), row r stored to idx[r]
__global__ void k_unpad_rows_ff(const float2* __restrict__ src, double* __restrict__ dst,
                                int64_t rows, int d, int ld, const int* __restrict__ idx);
// float64 rows (stride ld) -> their float-float mirror (same stride)
__global__ void k_mirror_ff(const double* __restrict__ src, float2* __restrict__ dst,
                            int64_t total);

// Xt = X + t Dx and its float-float mirror; gd = <G, Dx>.
template <typename Tc>
__global__ void __launch_bounds__(256)
k_trial_ff(const double* __restrict__ X, const Tc* __restrict__ Dx, const double* __restrict__ G,
           double t, double* __restrict__ Xt, float2* __restrict__ XFt, int64_t total,
           double* partials, Ctl* ctl) {
  double acc[1] = {0.0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double dx = (double)Dx[q];
    const double v = X[q] + t * dx;
    Xt[q] = v;
    const ff f = d2ff(v);
    XFt[q] = make_float2(f.h, f.l);
    acc[0] += G[q] * dx;
  }
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_TRIAL], tot) && threadIdx.x == 0)
    ctl->dots[0] = tot[0];
}

// Per-edge scalars and outputs shared by both passes, all in float32 /
// float-float (no float64 operation per edge): from ss = ||y||^2 and r = gamma
// w_l, the kind (inert / inside / outside), alpha, Pi(y) (float-float row), yhat
// (operator precision) for outside edges, and h_l added to hacc.
template <int LANES, int CH, typename Tc>
__device__ __forceinline__ uint8_t ff_edge_outputs(const ff (&y)[CH][4], ff r, ff ss, int lane,
                                                   int ld, int64_t e, float2* __restrict__ Ut,
                                                   Tc* __restrict__ Yh, Tc* __restrict__ alpha,
                                                   uint8_t* __restrict__ kind, ff& hacc) {
  const ff rs = ss.h > 0.0f ? ff_rsqrt(ss) : ff{0.0f, 0.0f};  // 1/||y|| (0 for y = 0)
  const ff ny = ff_mul(ss, rs);                                // ||y||
  uint8_t kd;
  ff scale;
  if (!(r.h > 0.0f)) {
    kd = K_INERT;
    scale = ff{0.0f, 0.0f};
  } else if (ff_le(ny, r)) {
    kd = K_IN;
    scale = ff{1.0f, 0.0f};
  } else {
    kd = K_OUT;
    scale = ff_mul(r, rs);
  }
  if (lane == 0) {
    kind[e] = kd;
    alpha[e] = (Tc)scale.h;
    // h = ||y||^2 / 2 inside the ball, r (||y|| - r/2) outside (0 when r = 0)
    hacc = ff_add(hacc, ff_le(ny, r) ? ff_half(ss) : ff_mul(r, ff_sub(ny, ff_half(r))));
  }
  if (kd == K_IN) {
    ff_row_store<LANES, CH>(Ut + e * ld, ld, lane, y);  // Pi(y) = y inside the ball
  } else {
    ff p[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) p[c][k] = kd == K_INERT ? ff{0.0f, 0.0f} : ff_mul(y[c][k], scale);
    ff_row_store<LANES, CH>(Ut + e * ld, ld, lane, p);
  }
  if (kd == K_OUT) {
    Tc yh[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) yh[c][k] = (Tc)(y[c][k].h * rs.h);
    row_store<LANES, CH>(Yh + e * ld, ld, lane, yh);
  }
  return kd;
}

// Evaluation edge pass (as k_edge_eval) in float-float: y, ||y||, kind, Pi(y) ->
// Ut, yhat -> Yh, alpha; accumulates sum_l h_l and the number of outside edges.
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256, CH <= 2 ? 4 : 1)
k_edge_eval_ff(const float2* __restrict__ XF, const float2* __restrict__ U,
               const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
               double sigma, float2* __restrict__ Ut, Tc* __restrict__ Yh, Tc* __restrict__ alpha,
               uint8_t* __restrict__ kind, int64_t m, int ld, double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const ff sg = d2ff(sigma), gm = d2ff(gamma);
  ff hacc = {0.0f, 0.0f};
  int nout = 0;
  // the next edge's endpoints and weight are loaded one edge ahead, so that the
  // row loads of an edge wait on one round trip to memory instead of two
  int2 ij_n = g0 < m ? edges[g0] : make_int2(0, 0);
  double w_n = g0 < m ? w[g0] : 0.0;
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = ij_n;
    const ff r = ff_mul(gm, d2ff(w_n));
    if (e + ng < m) {
      ij_n = edges[e + ng];
      w_n = w[e + ng];
    }
    ff xi[CH][4], xj[CH][4], y[CH][4];
    ff_row_load<LANES, CH>(XF + (int64_t)ij.x * ld, ld, lane, xi);
    ff_row_load<LANES, CH>(XF + (int64_t)ij.y * ld, ld, lane, xj);
    ff_row_load<LANES, CH>(U + e * ld, ld, lane, y);
    ff ss = {0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        y[c][k] = ff_add(y[c][k], ff_mul(ff_sub(xi[c][k], xj[c][k]), sg));
        ff_sqr_acc(ss, y[c][k]);
      }
    ss = ff_group_sum<LANES>(ff_norm(ss), mask);
    const uint8_t kd =
        ff_edge_outputs<LANES, CH, Tc>(y, r, ss, lane, ld, e, Ut, Yh, alpha, kind, hacc);
    if (lane == 0) nout += kd == K_OUT ? 1 : 0;
  }
  double acc[2] = {ff2d(hacc), (double)nout};
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_EVAL_E], tot) && threadIdx.x == 0) {
    ctl->eval[0] = tot[0];
    ctl->eval[3] = tot[1];
  }
}

// KKT edge pass fused with the next evaluation at the same (X, U) (as
// k_kkt_edge_eval) in float-float: bx = x_i - x_j feeds ||BX - prox_p(BX + U)||^2
// (= ||bx - shrink v||^2 with v = u + bx, shrink = max(0, 1 - r/||v||)) and
// r_l ||bx|| for f_p, and y = u + sigma bx the evaluation outputs.
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256, CH <= 4 ? 2 : 1)
k_kkt_edge_eval_ff(const float2* __restrict__ XF, const float2* __restrict__ U,
                   const int2* __restrict__ edges, const double* __restrict__ w, double gamma,
                   double sigma, float2* __restrict__ Ut, Tc* __restrict__ Yh,
                   Tc* __restrict__ alpha, uint8_t* __restrict__ kind, int64_t m, int ld,
                   double* partials, Ctl* ctl) {
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const ff sg = d2ff(sigma), gm = d2ff(gamma);
  ff racc = {0.0f, 0.0f}, pacc = {0.0f, 0.0f}, hacc = {0.0f, 0.0f};  // ||res||^2, sum r||bx||, sum h
  int nout = 0;
  // the next edge's endpoints and weight are loaded one edge ahead, so that the
  // row loads of an edge wait on one round trip to memory instead of two
  int2 ij_n = g0 < m ? edges[g0] : make_int2(0, 0);
  double w_n = g0 < m ? w[g0] : 0.0;
  for (int64_t e = g0; e < m; e += ng) {
    const int2 ij = ij_n;
    const ff r = ff_mul(gm, d2ff(w_n));
    if (e + ng < m) {
      ij_n = edges[e + ng];
      w_n = w[e + ng];
    }
    // u and bx are the edge's rows; v = u + bx and y = u + sigma bx are formed
    // from them where they are needed (by the same operations each time, so
    // with the same values), and the launch bounds ask for two resident blocks
    // per SM where a lane holds at most four quads
    ff bx[CH][4], u[CH][4];
    {
      ff xj[CH][4];
      ff_row_load<LANES, CH>(XF + (int64_t)ij.x * ld, ld, lane, bx);
      ff_row_load<LANES, CH>(XF + (int64_t)ij.y * ld, ld, lane, xj);
      ff_row_load<LANES, CH>(U + e * ld, ld, lane, u);
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) bx[c][k] = ff_sub(bx[c][k], xj[c][k]);
    }
    ff sb = {0.0f, 0.0f}, sv = {0.0f, 0.0f}, ss = {0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ff_sqr_acc(sb, bx[c][k]);
        ff_sqr_acc(ss, ff_add(u[c][k], ff_mul(bx[c][k], sg)));
        ff_sqr_acc(sv, ff_add(u[c][k], bx[c][k]));
      }
    sb = ff_group_sum<LANES>(ff_norm(sb), mask);
    sv = ff_group_sum<LANES>(ff_norm(sv), mask);
    ss = ff_group_sum<LANES>(ff_norm(ss), mask);
    // shrink = 1 - r / ||v|| where ||v|| > r, else 0
    const ff rv = sv.h > 0.0f ? ff_rsqrt(sv) : ff{0.0f, 0.0f};
    const ff nsh = ff_le(ff_mul(sv, rv), r) ? ff{0.0f, 0.0f}
                                            : ff_sub(ff_mul(r, rv), ff{1.0f, 0.0f});  // -shrink
    // residual bx - shrink v: its norm only enters eta_P, so the residual is
    // formed to float32 accuracy: the high words in one fused multiply-add
    // (rounded once, so a residual far below |bx| keeps its relative accuracy)
    // plus the low-word terms in float32 (absolute error about 2^-46 |bx|, the
    // product of the two low words dropped), and its square summed in float32
    float sres = 0.0f;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const ff v = ff_add(u[c][k], bx[c][k]);
        const float lo = bx[c][k].l + fmaf(nsh.h, v.l, nsh.l * v.h);
        const float res = fmaf(nsh.h, v.h, bx[c][k].h) + lo;
        sres = fmaf(res, res, sres);
      }
    racc = ff_add(racc, ff{sres, 0.0f});
    // y = u + sigma bx in place of u
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) u[c][k] = ff_add(u[c][k], ff_mul(bx[c][k], sg));
    const uint8_t kd =
        ff_edge_outputs<LANES, CH, Tc>(u, r, ss, lane, ld, e, Ut, Yh, alpha, kind, hacc);
    if (lane == 0) {
      if (sb.h > 0.0f) pacc = ff_add(pacc, ff_mul(r, ff_mul(sb, ff_rsqrt(sb))));
      nout += kd == K_OUT ? 1 : 0;
    }
  }
  // the residual sums of all lanes join; the per-edge terms were added by lane 0 only
  double acc[4] = {ff2d(racc), ff2d(pacc), ff2d(hacc), (double)nout};
  double tot[4];
  if (grid_reduce<4>(acc, partials, &ctl->counter[C_KKT_E], tot) && threadIdx.x == 0) {
    ctl->kkt[0] = tot[0];
    ctl->kkt[1] = tot[1];
    ctl->eval[0] = tot[2];
    ctl->eval[3] = tot[3];
  }
}

// Node gradient (as k_node_grad, register form) with the incidence sum
// B^T Pi(y) accumulated in float-float; G_i = (x_i - a_i) + that sum in float64.
template <int LANES, int CH, typename Tc>
__global__ void __launch_bounds__(256)
k_node_grad_ff(const double* __restrict__ X, const double* __restrict__ Ap,
               const float2* __restrict__ Ut, const int64_t* __restrict__ off,
               const int2* __restrict__ inc, const Tc* __restrict__ alpha,
               const uint8_t* __restrict__ kind, double sigma, int d, double* __restrict__ G,
               Tc* __restrict__ Minv, int64_t n, int ld, double* partials, Ctl* ctl,
               const int* __restrict__ ord) {
  constexpr int NB = GatherDepth<CH>::v;
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x / LANES;
  const float tr_out = (float)(d - 1) / (float)d;
  double acc[2] = {0.0, 0.0};
  // The chain of dependent scalar loads in front of a node's gathers (its index
  // in the visiting order, then its row range) is pipelined across the group's
  // nodes: the range of the next node and the index of the one after it are
  // loaded while this node is processed. (Loading the record batches one batch
  // ahead as well, as the operator does, needed 6 more registers and took 500
  // against 487 us: at one quad per lane this kernel is bound by the three
  // resident blocks per SM that 80 registers allow.)
  auto node_of = [&](int64_t gi) -> int64_t {
    return gi < n ? (ord ? (int64_t)ord[gi] : gi) : 0;
  };
  int64_t i_cur = node_of(g0);
  int64_t b_cur = g0 < n ? off[i_cur] : 0, e_cur = g0 < n ? off[i_cur + 1] : 0;
  int64_t i_nxt = node_of(g0 + ng);
  for (int64_t gi = g0; gi < n; gi += ng) {
    const int64_t i = i_cur, b = b_cur, eend = e_cur;
    if (gi + ng < n) {
      b_cur = off[i_nxt];
      e_cur = off[i_nxt + 1];
    }
    i_cur = i_nxt;
    i_nxt = node_of(gi + 2 * ng);
    ff g[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) g[c][k] = ff{0.0f, 0.0f};
    float diag = 0.0f;
    for (int64_t base = b; base < eend; base += LANES) {
      const int nb = (int)(eend - base < (int64_t)LANES ? eend - base : (int64_t)LANES);
      int2 rec = make_int2(0, 0);
      float tl = 0.0f;
      if (lane < nb) {
        rec = inc[base + lane];
        const uint8_t kd = kind[rec.x];
        const float al = (float)alpha[rec.x];
        tl = kd == K_IN ? 1.0f : (kd == K_OUT ? al * tr_out : 0.0f);
      }
      diag += group_sum<LANES>(tl, mask);
      for (int j = 0; j < nb; j += NB) {
        ff u[NB][CH][4];
        bool neg[NB];
#pragma unroll
        for (int kk = 0; kk < NB; ++kk) {
          const int ex = __shfl_sync(mask, rec.x, j + kk, LANES);
          const int ey = __shfl_sync(mask, rec.y, j + kk, LANES);
          neg[kk] = i > ey;  // i is the second endpoint: -Pi(y)_l
          if (j + kk < nb) {
            ff_row_load<LANES, CH>(Ut + (int64_t)ex * ld, ld, lane, u[kk]);
          } else {
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) u[kk][c][k] = ff{0.0f, 0.0f};
          }
        }
#pragma unroll
        for (int kk = 0; kk < NB; ++kk)
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k)
              g[c][k] = ff_add(g[c][k], neg[kk] ? ff_neg(u[kk][c][k]) : u[kk][c][k]);
      }
    }
    // the X and A rows are loaded here, after the gathers: loading them first
    // (16 more registers at one quad per lane) cost a resident block per SM and
    // was slower (636 against 481 us on 200,000 nodes of degree 17)
    double gd[CH][4], xa[CH][4], a4[CH][4];
    row_load<LANES, CH>(X + i * ld, ld, lane, xa);
    row_load<LANES, CH>(Ap + i * ld, ld, lane, a4);
    double gg = 0.0, hxa = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        xa[c][k] -= a4[c][k];
        hxa = fma(xa[c][k], xa[c][k], hxa);
        gd[c][k] = xa[c][k] + ff2d(g[c][k]);
        gg = fma(gd[c][k], gd[c][k], gg);
      }
    acc[0] += gg;
    acc[1] += 0.5 * hxa;
    row_store<LANES, CH>(G + i * ld, ld, lane, gd);
    if (lane == 0) Minv[i] = (Tc)(1.0f / fmaf((float)sigma, diag, 1.0f));
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_EVAL_N], tot) && threadIdx.x == 0) {
    ctl->eval[2] = tot[0];
    ctl->eval[1] = tot[1];
  }
}

// Long-row node gradient (as k_node_grad_ring) with float-float Pi(y) rows: the
// ring slots carry the float-float rows (8 bytes per element, as float64), the
// incidence sum is accumulated in float-float, parts of split nodes are stored
// as float-float rows, and the node's G row is formed in float64.
template <int CH, typename Tc, int S>
__global__ void __launch_bounds__(256, 1)
k_node_grad_ring_ff(const double* __restrict__ X, const double* __restrict__ Ap,
                    const float2* __restrict__ Ut, const int64_t* __restrict__ off,
                    const int2* __restrict__ inc, const Tc* __restrict__ alpha,
                    const uint8_t* __restrict__ kind, double sigma, int d,
                    double* __restrict__ G, Tc* __restrict__ Minv,
                    const WarpSpan* __restrict__ spans, float2* __restrict__ parts,
                    double* __restrict__ pdiag, unsigned* __restrict__ cnt, int ld,
                    double* partials, Ctl* ctl) {
  constexpr int LANES = 32;
  extern __shared__ __align__(128) unsigned char smem[];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * nw + warp;
  GradMeta* smeta = reinterpret_cast<GradMeta*>(smem) + (size_t)warp * S;
  float2* ring = reinterpret_cast<float2*>(smem + ring_header(nw, S, sizeof(GradMeta))) +
                 (size_t)warp * S * ld;
  const WarpSpan sp = spans[gw];
  const double tr_out = (double)(d - 1) / (double)d;
  double acc[2] = {0.0, 0.0};  // ||G||^2, 1/2 ||X - A||^2
  split_row_init<2>(sp, gw, lane, partials);
  if (sp.i1 >= sp.i0) {
    const int64_t kb = min(sp.ub - sp.i0, off[sp.i0 + 1]);
    const int64_t ke = min(sp.ue - sp.i1, off[sp.i1 + 1]);
    const uint64_t pol = l2_policy_evict_last();

    int2 c_eo, n_eo;
    double c_t, n_t;
    auto fetch = [&](int64_t base, int2& eo, double& t) {
      const int64_t k = base + lane;
      eo = make_int2(0, 0);
      t = -1.0;
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
      if (pk < ke) {
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
        smeta[pslot].t = t;
        smeta[pslot].other = ey;
        if (t >= 0.0)
          row_copy_async<LANES, CH>(reinterpret_cast<double*>(ring + (size_t)pslot * ld),
                                    reinterpret_cast<const double*>(Ut + (int64_t)ex * ld), ld,
                                    lane, pol);
        ++pk;
      }
      cp_async_commit();
      if (++pslot == S) pslot = 0;
    };
#pragma unroll
    for (int q = 0; q < S; ++q) issue();

    int cslot = 0;
    for (int i = sp.i0; i <= sp.i1; ++i) {
      const int64_t ob = off[i], oe = off[i + 1];
      const int64_t rb = max(ob + i, sp.ub) - i, re = min(oe + i, sp.ue) - i;
      const int np = i == sp.i0 ? sp.np0 : (i == sp.i1 ? sp.np1 : 1);
      ff g[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[c][k] = ff{0.0f, 0.0f};
      double diag = 0.0;
      for (int64_t t = rb; t < re; ++t) {
        cp_async_wait<S - 1>();
        const double tt = smeta[cslot].t;
        if (tt >= 0.0) {
          ff u4[CH][4];
          ff_row_load<LANES, CH>(ring + (size_t)cslot * ld, ld, lane, u4);
          const bool neg = !(i < smeta[cslot].other);
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k)
              g[c][k] = ff_add(g[c][k], neg ? ff_neg(u4[c][k]) : u4[c][k]);
          diag += tt;
        }
        if (++cslot == S) cslot = 0;
        issue();
      }
      if (np > 1) {
        const int wf = i == sp.i0 ? sp.wf0 : sp.wf1, wl = i == sp.i0 ? sp.wl0 : sp.wl1;
        const int64_t row = part_row(spans, gw, i);
        ff_row_store<LANES, CH>(parts + row * ld, ld, lane, g);
        if (lane == 0) pdiag[row] = diag;
        if (!part_arrive(cnt + wf, np, lane)) continue;
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) g[c][k] = ff{0.0f, 0.0f};
        diag = 0.0;
        for (int w = wf; w <= wl; ++w) {
          if (spans[w].i1 < spans[w].i0) continue;  // empty span
          const int64_t pr = part_row(spans, w, i);
          const float2* prow = parts + pr * ld;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int q = c * LANES + lane;
            if (4 * q < ld) {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float2 pv = __ldcg(prow + 4 * q + k);
                g[c][k] = ff_add(g[c][k], ff{pv.x, pv.y});
              }
            }
          }
          diag += __ldcg(pdiag + pr);
        }
      }
      double xa[CH][4], a4[CH][4], gd[CH][4];
      row_load<LANES, CH>(X + (int64_t)i * ld, ld, lane, xa);
      row_load<LANES, CH>(Ap + (int64_t)i * ld, ld, lane, a4);
      double gg = 0.0, hxa = 0.0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          xa[c][k] -= a4[c][k];
          hxa = fma(xa[c][k], xa[c][k], hxa);
          gd[c][k] = xa[c][k] + ff2d(g[c][k]);
          gg = fma(gd[c][k], gd[c][k], gg);
        }
      hxa *= 0.5;
      row_store<LANES, CH>(G + (int64_t)i * ld, ld, lane, gd);
      if (lane == 0) Minv[i] = (Tc)(1.0 / (1.0 + sigma * diag));
      if (np > 1) {  // the split node's own reduction row
        gg = group_sum<LANES>(gg, 0xffffffffu);
        hxa = group_sum<LANES>(hxa, 0xffffffffu);
        const int wf = i == sp.i0 ? sp.wf0 : sp.wf1;
        if (lane == 0) {
          partials[((size_t)gridDim.x + wf) * 2] = gg;
          partials[((size_t)gridDim.x + wf) * 2 + 1] = hxa;
        }
      } else {
        acc[0] += gg;
        acc[1] += hxa;
      }
    }
    cp_async_wait<0>();
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_EVAL_N], tot, gridDim.x * nw) &&
      threadIdx.x == 0) {
    ctl->eval[2] = tot[0];
    ctl->eval[1] = tot[1];
  }
}

// Node gradient over float-float Pi(y) rows: the ring form when a plan is given
// (long rows), the register form otherwise.
template <int L, int CH, typename Tc>
inline int launch_node_grad_ff(Ctx* c, const double* X, const double* Ap, const float2* Ut,
                               const int64_t* off, const int2* inc, const Tc* alpha,
                               const uint8_t* kind, double sigma, int d, double* G, Tc* Minv,
                               const RingPlan& rp, int64_t n, int ld, double* part, Ctl* ctl,
                               cudaStream_t s) {
  if (L == 32 && rp.on()) {
    auto fn = k_node_grad_ring_ff<CH, Tc, kRingStages>;
    CCM_TRY(set_smem_limit(c, (const void*)fn, rp.sh.smem_grad));
    fn<<<c->num_sms, rp.sh.nw * 32, rp.sh.smem_grad, s>>>(X, Ap, Ut, off, inc, alpha, kind, sigma,
                                                          d, G, Minv, rp.spans,
                                                          (float2*)rp.parts, rp.pdiag, rp.cnt, ld,
                                                          part, ctl);
  } else {
    const int threads = 256;
    const int gpb = threads / L;
    auto fn = k_node_grad_ff<L, CH, Tc>;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + gpb - 1) / gpb, (int64_t)resident_grid(c, fn, threads)));
    fn<<<blocks, threads, 0, s>>>(X, Ap, Ut, off, inc, alpha, kind, sigma, d, G, Minv, n, ld,
                                  part, ctl, rp.ord);
  }
  CCM_COUNT(c);
  return CCM_OK;
}

}  // namespace ccm
