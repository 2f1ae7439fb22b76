// Long-row forms (rows of more than 32 quads, one warp per row) of the two
// gather-sums of SSNAL: the Newton-CG operator W = V M R and the node gradient
// G = X - A + B^T Pi(y) with the Jacobi scalars Minv.
//
// Work split. The incidence stream is the CSR of B^T in node order with one
// closing unit after each node: node i owns units [off[i] + i, off[i+1] + i]
// (its incidences, then its close), U = 2m + n units in all. Warp w of nwg
// takes units [w U / nwg, (w+1) U / nwg), so every warp carries the same work
// whatever the degree distribution (kNN graphs of high-dimensional data have
// hubs: the 10,000-point, d = 784 workload has a node of degree 419 against a
// mean of 18). A node whose units straddle warps is split into parts, one per
// warp; each part stores its partial row in a scratch row and counts itself on
// the node's counter, and the part that arrives last sums the parts in part
// order (so the result does not depend on which warp finishes first) and
// finishes the node. The counter is reset by that part.
//
// Gathers. Each warp streams the rows its incidences gather (the other
// endpoint's row; for the operator also yhat of outside edges) into a ring of
// S shared-memory slots with cp.async: every lane copies its own quads and
// later reads only those, so a slot needs no barrier; each slot is one commit
// group and the lane waits for the oldest with cp.async.wait_group. Incidence
// records come in lane-parallel batches of 32, fetched one batch ahead.
#pragma once

#include <algorithm>

#include "async_copy.cuh"
#include "ssnal_kernels.cuh"

namespace ccm {

static constexpr int kRingStages = 4;  // ring slots per warp

// Bytes in front of the per-warp slot rings: nw*stages slot-metadata records,
// rounded up to 128 bytes.
__host__ __device__ inline size_t ring_header(int nw, int stages, size_t meta_bytes) {
  return ((size_t)nw * stages * meta_bytes + 127) / 128 * 128;
}

// One warp's share of the incidence stream.
struct WarpSpan {
  int64_t ub, ue;     // unit range [ub, ue)
  int i0, i1;         // first and last node touched (i1 < i0: empty range)
  int wf0, wl0, np0;  // node i0: first and last warp holding its units, parts (non-empty
                      // spans in [wf0, wl0])
  int wf1, wl1, np1;  // node i1: the same
};

// Builds the nwg spans from the CSR offsets (one thread per warp span).
__global__ void k_span_setup(const int64_t* __restrict__ off, int64_t n, int nwg,
                             WarpSpan* __restrict__ spans);

// Scratch row of warp w's part of node i (its first node: row 2w; its last: 2w+1).
__device__ __forceinline__ int64_t part_row(const WarpSpan* spans, int w, int i) {
  return spans[w].i0 == i ? 2 * (int64_t)w : 2 * (int64_t)w + 1;
}

// Reductions (delta, ||G||^2, ...) must not depend on which warp finishes a split
// node, so a split node's terms go to a reduction row of their own: row
// gridDim.x + wf of the grid_reduce partials, wf the node's first warp. Warp w
// writes zeros there itself when it is the first warp of no split node.
__device__ __forceinline__ bool owns_split(const WarpSpan& sp, int w) {
  return sp.i1 >= sp.i0 && sp.np1 > 1 && sp.wf1 == w;
}
template <int NRED>
__device__ __forceinline__ void split_row_init(const WarpSpan& sp, int w, int lane,
                                               double* partials) {
  if (lane == 0 && !owns_split(sp, w))
#pragma unroll
    for (int k = 0; k < NRED; ++k) partials[((size_t)gridDim.x + w) * NRED + k] = 0.0;
}

// Counts one part of a split node (after its partial row is stored); true for
// the part that arrives last, which then owns the node. Warp-uniform.
__device__ __forceinline__ bool part_arrive(unsigned* cnt, int np, int lane) {
  __threadfence();  // this lane's partial-row stores before the count
  __syncwarp();
  unsigned prev = 0;
  if (lane == 0) prev = atomicAdd(cnt, 1u);
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev + 1 == (unsigned)np) {
    __threadfence();  // the other parts' rows are visible after their counts
    if (lane == 0) *cnt = 0u;
    return true;
  }
  return false;
}

// ------------------------------------------------------------ operator
// W = D u + sigma B^T P B u with u = Minv R; delta = <W, u>; alpha (cg_set_alpha).
// Parts of split nodes are float rows in `parts` (2 nwg rows of ld).
template <int CH, typename Tc, int S>
__global__ void __launch_bounds__(256, 1)
k_cg_matvec_ring(const Tc* __restrict__ R, const Tc* __restrict__ Minv, const Tc* __restrict__ Dg,
                 Tc* __restrict__ W, const Tc* __restrict__ Yh,
                 const IncMeta<Tc>* __restrict__ meta, const int64_t* __restrict__ off,
                 const int2* __restrict__ inc, const WarpSpan* __restrict__ spans,
                 Tc* __restrict__ parts, unsigned* __restrict__ cnt, double sigma, int ld,
                 double* partials, Ctl* ctl) {
  constexpr int LANES = 32;
  extern __shared__ __align__(128) unsigned char smem[];
  if (!ctl->cg.active) return;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * nw + warp;
  IncMeta<Tc>* smeta = reinterpret_cast<IncMeta<Tc>*>(smem) + (size_t)warp * S;
  Tc* ring = reinterpret_cast<Tc*>(smem + ring_header(nw, S, sizeof(IncMeta<Tc>))) +
             (size_t)warp * S * 2 * ld;
  const WarpSpan sp = spans[gw];
  const Tc sg = (Tc)sigma;
  double acc[1] = {0.0};
  split_row_init<1>(sp, gw, lane, partials);
  if (sp.i1 >= sp.i0) {
    const int64_t kb = min(sp.ub - sp.i0, off[sp.i0 + 1]);
    const int64_t ke = min(sp.ue - sp.i1, off[sp.i1 + 1]);
    const uint64_t pol_keep = l2_policy_evict_last(), pol_stream = l2_policy_evict_first();

    // ---- producer: records [kb, ke), this lane's quads of each gathered row
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
    auto issue = [&]() {
      if (pk < ke) {
        if (pk - c_base >= 32) {
          c_eo = n_eo;
          c_m = n_m;
          c_base += 32;
          fetch(c_base + 32, n_eo, n_m);
        }
        const int src = (int)(pk - c_base);
        const int ex = __shfl_sync(0xffffffffu, c_eo.x, src);
        const int ey = __shfl_sync(0xffffffffu, c_eo.y, src);
        const Tc mc_raw = __shfl_sync(0xffffffffu, c_m.c, src);
        const Tc mo = __shfl_sync(0xffffffffu, c_m.mo, src);
        const Tc mc = inc_ok(make_int2(ex, ey), B_MATVEC_RING, pk) ? mc_raw : (Tc)0;
        smeta[pslot].c = mc;  // every lane writes the same value and reads it back itself
        smeta[pslot].mo = mo;
        if (mc != (Tc)0) {
          Tc* dst = ring + (size_t)pslot * 2 * ld;
          row_copy_async<LANES, CH>(dst, R + (int64_t)ey * ld, ld, lane, pol_keep);
          if (mc < (Tc)0 || mc > (Tc)1.5)  // yhat row, the q = 1 mask row or the q = inf s row
            row_copy_async<LANES, CH>(dst + ld, Yh + (int64_t)ex * ld, ld, lane, pol_stream);
        }
        ++pk;
      }
      cp_async_commit();  // one group per slot (empty past the end of the stream)
      if (++pslot == S) pslot = 0;
    };
#pragma unroll
    for (int q = 0; q < S; ++q) issue();

    // ---- consumer: nodes i0..i1, each over its records in this span
    int cslot = 0;
    for (int i = sp.i0; i <= sp.i1; ++i) {
      const int64_t ob = off[i], oe = off[i + 1];
      const int64_t rb = max(ob + i, sp.ub) - i, re = min(oe + i, sp.ue) - i;
      const int np = i == sp.i0 ? sp.np0 : (i == sp.i1 ? sp.np1 : 1);
      Tc u[CH][4], accv[CH][4];
      const Tc mi = Minv[i];
      row_load<LANES, CH>(R + (int64_t)i * ld, ld, lane, u);
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          u[c][k] *= mi;
          accv[c][k] = (Tc)0;
        }
      for (int64_t t = rb; t < re; ++t) {
        cp_async_wait<S - 1>();  // this lane's copies of the oldest slot have landed
        const Tc mc = smeta[cslot].c, mo = smeta[cslot].mo;
        if (mc != (Tc)0) {
          const Tc* rr = ring + (size_t)cslot * 2 * ld;
          Tc v[CH][4];
          row_load<LANES, CH>(rr, ld, lane, v);
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) v[c][k] = u[c][k] - mo * v[c][k];
          if (mc > (Tc)2.5) {  // q = inf: diag(s != 0) - s s^T
            Tc sv[CH][4];
            row_load<LANES, CH>(rr + ld, ld, lane, sv);
            Tc s4[4] = {(Tc)0, (Tc)0, (Tc)0, (Tc)0};
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) s4[k] += sv[c][k] * v[c][k];
            Tc s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
            s = group_sum<LANES>(s, 0xffffffffu);
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k)
                accv[c][k] += (sv[c][k] != (Tc)0 ? v[c][k] : (Tc)0) - s * sv[c][k];
          } else if (mc > (Tc)1.5) {  // q = 1: diagonal mask
            Tc mk[CH][4];
            row_load<LANES, CH>(rr + ld, ld, lane, mk);
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) accv[c][k] += mk[c][k] * v[c][k];
          } else if (mc < (Tc)0) {
            Tc yh[CH][4];
            row_load<LANES, CH>(rr + ld, ld, lane, yh);
            Tc s4[4] = {(Tc)0, (Tc)0, (Tc)0, (Tc)0};  // four independent partial sums
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) s4[k] += yh[c][k] * v[c][k];
            Tc s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
            s = group_sum<LANES>(s, 0xffffffffu);
            const Tc a = -mc;
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
        if (++cslot == S) cslot = 0;
        issue();  // refill the slot just read
      }
      if (np > 1) {
        const int wf = i == sp.i0 ? sp.wf0 : sp.wf1, wl = i == sp.i0 ? sp.wl0 : sp.wl1;
        row_store<LANES, CH>(parts + part_row(spans, gw, i) * ld, ld, lane, accv);
        if (!part_arrive(cnt + wf, np, lane)) continue;
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) accv[c][k] = (Tc)0;
        for (int w = wf; w <= wl; ++w) {
          if (spans[w].i1 < spans[w].i0) continue;  // empty span
          const Tc* pr = parts + part_row(spans, w, i) * ld;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int q = c * LANES + lane;
            if (4 * q < ld) {
#pragma unroll
              for (int k = 0; k < 4; ++k) accv[c][k] += __ldcg(pr + 4 * q + k);
            }
          }
        }
      }
      Tc dot = (Tc)0, dot_e = (Tc)0;  // <W_i, u_i> over this lane's elements, float-float
      const Tc di = Dg ? Dg[i] : (Tc)1;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          accv[c][k] = di * u[c][k] + sg * accv[c][k];
          dot_acc(dot, dot_e, u[c][k], accv[c][k]);
        }
      row_store<LANES, CH>(W + (int64_t)i * ld, ld, lane, accv);
      const double dnode = (double)dot + (double)dot_e;
      if (np > 1) {  // the split node's own reduction row
        const double dsum = group_sum<LANES>(dnode, 0xffffffffu);
        const int wf = i == sp.i0 ? sp.wf0 : sp.wf1;
        if (lane == 0) partials[(size_t)gridDim.x + wf] = dsum;
      } else {
        acc[0] += dnode;
      }
    }
    cp_async_wait<0>();
  }
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_MV], tot, gridDim.x * nw) &&
      threadIdx.x == 0)
    cg_set_alpha(ctl, tot[0]);
}

// ------------------------------------------------------------ node gradient
// G_i = x_i - a_i + sum_l (+-) Ut_l (+ when i is the first endpoint) and
// Minv_i = 1 / (1 + sigma sum_l trace(P_l)/d), sums in increasing edge id within
// each part. Parts of split nodes are float64 rows in `parts` plus one float64
// diagonal partial each in `pdiag`.
struct GradMeta {
  double t;   // trace(P_l)/d; negative: inert edge (no row copied)
  int other;  // other endpoint
  int pad;
};

template <int CH, typename Tc, int S>
__global__ void __launch_bounds__(256, 1)
k_node_grad_ring(const double* __restrict__ X, const double* __restrict__ Ap,
                 const double* __restrict__ Ut, const int64_t* __restrict__ off,
                 const int2* __restrict__ inc, const Tc* __restrict__ alpha,
                 const uint8_t* __restrict__ kind, double sigma, int d, double* __restrict__ G,
                 Tc* __restrict__ Minv, const WarpSpan* __restrict__ spans,
                 double* __restrict__ parts, double* __restrict__ pdiag,
                 unsigned* __restrict__ cnt, int ld, double* partials, Ctl* ctl) {
  constexpr int LANES = 32;
  extern __shared__ __align__(128) unsigned char smem[];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * nw + warp;
  GradMeta* smeta = reinterpret_cast<GradMeta*>(smem) + (size_t)warp * S;
  double* ring = reinterpret_cast<double*>(smem + ring_header(nw, S, sizeof(GradMeta))) +
                 (size_t)warp * S * ld;
  const WarpSpan sp = spans[gw];
  const double tr_out = (double)(d - 1) / (double)d;
  double acc[2] = {0.0, 0.0};  // ||G||^2, 1/2 ||X - A||^2
  split_row_init<2>(sp, gw, lane, partials);
  if (sp.i1 >= sp.i0) {
    const int64_t kb = min(sp.ub - sp.i0, off[sp.i0 + 1]);
    const int64_t ke = min(sp.ue - sp.i1, off[sp.i1 + 1]);
    const uint64_t pol_stream = l2_policy_evict_first();

    int2 c_eo, n_eo;
    double c_t, n_t;
    auto fetch = [&](int64_t base, int2& eo, double& t) {
      const int64_t k = base + lane;
      eo = make_int2(0, 0);
      t = -1.0;
      if (k < ke) {
        eo = inc[k];
        const uint8_t kd = kind[eo.x];
        t = kd == K_IN ? 1.0
            : (kd == K_OUT ? (double)alpha[eo.x] * tr_out
                           : ((kd == K_MASK || kd == K_LINF) ? (double)alpha[eo.x] : -1.0));
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
          row_copy_async<LANES, CH>(ring + (size_t)pslot * ld, Ut + (int64_t)ex * ld, ld, lane,
                                    pol_stream);
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
      double g[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[c][k] = 0.0;
      double diag = 0.0;
      for (int64_t t = rb; t < re; ++t) {
        cp_async_wait<S - 1>();
        const double tt = smeta[cslot].t;
        if (tt >= 0.0) {
          const double* ur = ring + (size_t)cslot * ld;
          double u4[CH][4];
          row_load<LANES, CH>(ur, ld, lane, u4);
          if (i < smeta[cslot].other) {
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) g[c][k] += u4[c][k];
          } else {
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int k = 0; k < 4; ++k) g[c][k] -= u4[c][k];
          }
          diag += tt;
        }
        if (++cslot == S) cslot = 0;
        issue();
      }
      if (np > 1) {
        const int wf = i == sp.i0 ? sp.wf0 : sp.wf1, wl = i == sp.i0 ? sp.wl0 : sp.wl1;
        const int64_t row = part_row(spans, gw, i);
        row_store<LANES, CH>(parts + row * ld, ld, lane, g);
        if (lane == 0) pdiag[row] = diag;
        if (!part_arrive(cnt + wf, np, lane)) continue;
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) g[c][k] = 0.0;
        diag = 0.0;
        for (int w = wf; w <= wl; ++w) {
          if (spans[w].i1 < spans[w].i0) continue;  // empty span
          const int64_t pr = part_row(spans, w, i);
          const double* prow = parts + pr * ld;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int q = c * LANES + lane;
            if (4 * q < ld) {
#pragma unroll
              for (int k = 0; k < 4; ++k) g[c][k] += __ldcg(prow + 4 * q + k);
            }
          }
          diag += __ldcg(pdiag + pr);
        }
      }
      // G_i = (x_i - a_i) + sum of the incidence terms
      double xa[CH][4], a4[CH][4];
      row_load<LANES, CH>(X + (int64_t)i * ld, ld, lane, xa);
      row_load<LANES, CH>(Ap + (int64_t)i * ld, ld, lane, a4);
      double gg = 0.0, hxa = 0.0;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          xa[c][k] -= a4[c][k];
          hxa = fma(xa[c][k], xa[c][k], hxa);
          g[c][k] += xa[c][k];
          gg = fma(g[c][k], g[c][k], gg);
        }
      hxa *= 0.5;
      row_store<LANES, CH>(G + (int64_t)i * ld, ld, lane, g);
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

// ------------------------------------------------------------ shapes and launches
// Ring shape: kRingStages slots per warp, as many warps per CTA (<= 8) as fit
// one CTA per SM. The operator's slot holds two rows of Tc (R and yhat), the
// gradient's one float64 row; both kernels use the operator's warp count so
// they share one span table.
struct RingShape {
  int nw = 0;
  size_t smem_op = 0, smem_grad = 0;
};

template <typename Tc>
inline RingShape ring_shape(int ld) {
  constexpr size_t kBudget = 200 * 1024;
  RingShape sh;
  const size_t slot_op = 2 * (size_t)ld * sizeof(Tc), slot_grad = (size_t)ld * 8;
  const size_t slot = std::max(slot_op, slot_grad);
  const int nw = (int)std::min<size_t>(8, kBudget / ((size_t)kRingStages * slot));
  if (nw < 1) return sh;
  sh.nw = nw;
  sh.smem_op = ring_header(nw, kRingStages, sizeof(IncMeta<Tc>)) + (size_t)nw * kRingStages * slot_op;
  sh.smem_grad = ring_header(nw, kRingStages, sizeof(GradMeta)) + (size_t)nw * kRingStages * slot_grad;
  return sh;
}

// Span table and scratch of the long-row kernels for one CSR (per solve).
struct RingPlan {
  RingShape sh;
  int nwg = 0;                // warps in the grid (num_sms * sh.nw)
  WarpSpan* spans = nullptr;  // nwg
  void* parts = nullptr;      // 2 nwg rows of ld float64 (operator parts use the first half as Tc)
  double* pdiag = nullptr;    // 2 nwg
  unsigned* cnt = nullptr;    // nwg counters (zero between launches)
  const int* ord = nullptr;   // register forms: node visiting order (null: index order)
  bool on() const { return spans != nullptr; }
};

// Span table and scratch for one CSR when rows are long enough for the ring
// kernels (L == 32); otherwise rp stays off and the register forms run.
template <typename Tc>
inline int ring_plan(Ctx* c, int L, int ld, const int64_t* off, int64_t n, RingPlan& rp,
                     cudaStream_t s) {
  if (L != 32) return CCM_OK;
  rp.sh = ring_shape<Tc>(ld);
  if (rp.sh.nw <= 0) return CCM_OK;
  rp.nwg = c->num_sms * rp.sh.nw;
  const size_t b_sp = round_up((int64_t)rp.nwg * sizeof(WarpSpan), 256);
  const size_t b_cnt = round_up((int64_t)rp.nwg * 4, 256);
  const size_t b_pd = round_up((int64_t)rp.nwg * 2 * 8, 256);
  const size_t b_parts = (size_t)rp.nwg * 2 * ld * 8;
  void* p;
  CCM_TRY(ws_get(c, S_WPART, b_sp + b_cnt + b_pd + b_parts, &p));
  char* base = (char*)p;
  rp.spans = (WarpSpan*)base;
  rp.cnt = (unsigned*)(base + b_sp);
  rp.pdiag = (double*)(base + b_sp + b_cnt);
  rp.parts = base + b_sp + b_cnt + b_pd;
  CCM_CUDA(cudaMemsetAsync(rp.cnt, 0, b_cnt, s));
  k_span_setup<<<(rp.nwg + 255) / 256, 256, 0, s>>>(off, n, rp.nwg, rp.spans);
  CCM_COUNT(c);
  return CCM_OK;
}

// Raise the dynamic shared-memory limit of kernel fn to smem on c's device,
// once per (context, kernel instance).
inline int set_smem_limit(Ctx* c, const void* fn, size_t smem) {
  for (auto& e : c->smem_attr) {
    if (e.first != fn) continue;
    if (e.second < smem) {
      CCM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      e.second = smem;
    }
    return CCM_OK;
  }
  CCM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  c->smem_attr.emplace_back(fn, smem);
  return CCM_OK;
}

// Operator: the ring form when a plan is given (long rows), the register form otherwise.
template <int L, int CH, typename Tc>
inline int launch_matvec(Ctx* c, const Tc* R, const Tc* Minv, const Tc* Dg, Tc* W, const Tc* Yh,
                         const IncMeta<Tc>* meta, const int64_t* off, const int2* inc,
                         const RingPlan& rp, double sigma, int64_t n, int ld, double* part,
                         Ctl* ctl, cudaStream_t s) {
  if (L == 32 && rp.on()) {
    auto fn = k_cg_matvec_ring<CH, Tc, kRingStages>;
    CCM_TRY(set_smem_limit(c, (const void*)fn, rp.sh.smem_op));
    fn<<<c->num_sms, rp.sh.nw * 32, rp.sh.smem_op, s>>>(R, Minv, Dg, W, Yh, meta, off, inc,
                                                        rp.spans, (Tc*)rp.parts, rp.cnt, sigma,
                                                        ld, part, ctl);
    CCM_COUNT(c);
    return CCM_OK;
  }
  return launch_matvec_reg<L, CH, Tc>(c, R, Minv, Dg, W, Yh, meta, off, inc, sigma, n, ld, part,
                                      ctl, s, rp.ord);
}

// Node gradient: the ring form when a plan is given, the register form otherwise.
template <int L, int CH, typename Tc>
inline int launch_node_grad(Ctx* c, const double* X, const double* Ap, const double* Ut,
                            const int64_t* off, const int2* inc, const Tc* alpha,
                            const uint8_t* kind, double sigma, int d, double* G, Tc* Minv,
                            const RingPlan& rp, int64_t n, int ld, double* part, Ctl* ctl,
                            cudaStream_t s) {
  if (L == 32 && rp.on()) {
    auto fn = k_node_grad_ring<CH, Tc, kRingStages>;
    CCM_TRY(set_smem_limit(c, (const void*)fn, rp.sh.smem_grad));
    fn<<<c->num_sms, rp.sh.nw * 32, rp.sh.smem_grad, s>>>(X, Ap, Ut, off, inc, alpha, kind, sigma,
                                                          d, G, Minv, rp.spans,
                                                          (double*)rp.parts, rp.pdiag, rp.cnt, ld,
                                                          part, ctl);
  } else {
    const int threads = 256;
    const int gpb = threads / L;
    auto fn = k_node_grad<L, CH, Tc>;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + gpb - 1) / gpb, (int64_t)resident_grid(c, fn, threads)));
    fn<<<blocks, threads, 0, s>>>(X, Ap, Ut, off, inc, alpha, kind, sigma, d, G, Minv, n, ld,
                                  part, ctl);
  }
  CCM_COUNT(c);
  return CCM_OK;
}

}  // namespace ccm
