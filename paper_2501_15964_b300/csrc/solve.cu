// ccm_solve_path: SSNAL for model CCM (q = 2, 1 or inf) along a gamma path, grid engine.
//
// The outer loop (multiplier updates), the semismooth-Newton loop, the
// Armijo line search and the CG loop are driven from the host; every
// reduction and every scalar recurrence of CG runs on the device (grid_reduce
// in the last block of each kernel), and CG kernels skip themselves once the
// device-side stop flag is set, so CG iterations are launched in chunks with
// one host read-back per chunk.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "ccm_internal.cuh"
#include "coarse.cuh"
#include "solve_common.cuh"
#include "ff_kernels.cuh"
#include "ring_kernels.cuh"
#include "ssnal_kernels.cuh"

namespace ccm {

// node count from which ccm_solve_path relabels nodes by graph component
static constexpr int64_t kRelabelMinN = 16384;
// node count from which the register-form gathers visit nodes in degree order
static constexpr int64_t kDegreeOrderMinN = 8192;

// Row gather into the padded layout / scatter back out of it. idx (optional)
// maps a padded row to its source / destination row; a complemented entry (~r)
// marks an edge whose endpoints swapped under the node relabelling, whose row
// changes sign.
__device__ __forceinline__ int64_t idx_row(const int* idx, int64_t r, double& sg) {
  if (!idx) {
    sg = 1.0;
    return r;
  }
  const int v = idx[r];
  sg = v < 0 ? -1.0 : 1.0;
  return v < 0 ? (int64_t)~v : (int64_t)v;
}

__global__ void k_gather_rows(const double* __restrict__ src, double* __restrict__ dst,
                              int64_t rows, int d, int ld, const int* __restrict__ idx) {
  const int64_t total = rows * ld;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / ld;
    const int k = (int)(q - r * ld);
    double sg;
    const int64_t rs = idx_row(idx, r, sg);
    dst[q] = (k < d) ? sg * src[rs * d + k] : 0.0;
  }
}

__global__ void k_scatter_rows(const double* __restrict__ src, double* __restrict__ dst,
                               int64_t rows, int d, int ld, const int* __restrict__ idx) {
  const int64_t total = rows * d;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / d;
    const int k = (int)(q - r * d);
    double sg;
    const int64_t rd = idx_row(idx, r, sg);
    dst[rd * d + k] = sg * src[r * ld + k];
  }
}

__global__ void k_pad_rows_ff(const double* __restrict__ src, float2* __restrict__ dst,
                              int64_t rows, int d, int ld, const int* __restrict__ idx) {
  const int64_t total = rows * ld;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / ld;
    const int k = (int)(q - r * ld);
    double sg;
    const int64_t rs = idx_row(idx, r, sg);
    const ff f = (k < d) ? d2ff(sg * src[rs * d + k]) : ff{0.0f, 0.0f};
    dst[q] = make_float2(f.h, f.l);
  }
}

__global__ void k_unpad_rows_ff(const float2* __restrict__ src, double* __restrict__ dst,
                                int64_t rows, int d, int ld, const int* __restrict__ idx) {
  const int64_t total = rows * d;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / d;
    const int k = (int)(q - r * d);
    double sg;
    const int64_t rd = idx_row(idx, r, sg);
    const float2 v = src[r * ld + k];
    dst[rd * d + k] = sg * ff2d(ff{v.x, v.y});
  }
}

__global__ void k_mirror_ff(const double* __restrict__ src, float2* __restrict__ dst,
                            int64_t total) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const ff f = d2ff(src[q]);
    dst[q] = make_float2(f.h, f.l);
  }
}

__global__ void __launch_bounds__(256)
k_kkt_node(const double* __restrict__ X, const double* __restrict__ Ap,
           const double* __restrict__ G, int64_t total, double* partials, Ctl* ctl) {
  double acc[2] = {0.0, 0.0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    double a = Ap[q];
    double btu = G[q] - (X[q] - a);
    acc[0] += a * btu;
    acc[1] += btu * btu;
  }
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_KKT_N], tot) && threadIdx.x == 0) {
    ctl->kkt[2] = tot[0];
    ctl->kkt[3] = tot[1];
  }
}

// k_kkt_node with the element arithmetic in float-float on the FP32 pipe (the
// float64 form occupies B300's narrow FP64 pipe: four float64 operations per
// element against 24 bytes of loads). Quads of four elements per thread.
__global__ void __launch_bounds__(256)
k_kkt_node_ff(const double* __restrict__ X, const double* __restrict__ Ap,
              const double* __restrict__ G, int64_t total, double* partials, Ctl* ctl) {
  ff s_ab = {0.0f, 0.0f}, s_bb = {0.0f, 0.0f};  // <A, B^T U>, ||B^T U||^2 (bb unnormalised)
  for (int64_t q4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; q4 < total;
       q4 += (int64_t)gridDim.x * blockDim.x * 4) {
    double x[4], a[4], g[4];
    Vec4<double>::load(X + q4, x);
    Vec4<double>::load(Ap + q4, a);
    Vec4<double>::load(G + q4, g);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const ff af = d2ff(a[k]);
      const ff btu = ff_sub(d2ff(g[k]), ff_sub(d2ff(x[k]), af));
      s_ab = ff_add(s_ab, ff_mul(btu, af));
      ff_sqr_acc(s_bb, btu);
    }
  }
  double acc[2] = {ff2d(s_ab), ff2d(ff_norm(s_bb))};
  double tot[2];
  if (grid_reduce<2>(acc, partials, &ctl->counter[C_KKT_N], tot) && threadIdx.x == 0) {
    ctl->kkt[2] = tot[0];
    ctl->kkt[3] = tot[1];
  }
}

__global__ void k_sumsq(const double* __restrict__ v, int64_t total, double* partials,
                        Ctl* ctl) {
  double acc[1] = {0.0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x)
    acc[0] += v[q] * v[q];
  double tot[1];
  if (grid_reduce<1>(acc, partials, &ctl->counter[C_TRIAL], tot) && threadIdx.x == 0)
    ctl->dots[1] = tot[0];
}

__global__ void k_pad_rows(const double* __restrict__ src, double* __restrict__ dst, int64_t rows,
                           int d, int ld) {
  const int64_t total = rows * ld;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = q / ld;
    int k = (int)(q - r * ld);
    dst[q] = (k < d) ? src[r * d + k] : 0.0;
  }
}

__global__ void k_unpad_rows(const double* __restrict__ src, double* __restrict__ dst,
                             int64_t rows, int d, int ld) {
  const int64_t total = rows * d;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = q / d;
    int k = (int)(q - r * d);
    dst[q] = src[r * ld + k];
  }
}

// ---------------------------------------------------------------- edge checks / CSR
__global__ void k_validate_edges(const int2* __restrict__ edges, int64_t m, int64_t n,
                                 const double* __restrict__ w, int* bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int2 ij = edges[e];
    bool ok = ij.x >= 0 && ij.x < ij.y && (int64_t)ij.y < n;
    if (ok && e > 0) {
      int2 p = edges[e - 1];
      ok = (p.x < ij.x) || (p.x == ij.x && p.y < ij.y);
    }
    if (ok && w) ok = w[e] >= 0.0 && isfinite(w[e]);
    if (!ok) atomicExch(bad, 1);
  }
}

__global__ void k_degree(const int2* __restrict__ edges, int64_t m,
                         unsigned long long* __restrict__ deg) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int2 ij = edges[e];
    atomicAdd(deg + ij.x, 1ull);
    atomicAdd(deg + ij.y, 1ull);
  }
}

__global__ void k_fill_inc(const int2* __restrict__ edges, int64_t m,
                           const int64_t* __restrict__ off, unsigned long long* __restrict__ cur,
                           int2* __restrict__ inc) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int2 ij = edges[e];
    unsigned long long a = atomicAdd(cur + ij.x, 1ull);
    unsigned long long b = atomicAdd(cur + ij.y, 1ull);
    inc[off[ij.x] + (int64_t)a] = make_int2((int)e, ij.y);
    inc[off[ij.y] + (int64_t)b] = make_int2((int)e, ij.x);
  }
}

// Sort each node's incidence list by edge id (insertion sort: lists are short;
// the result, and so every reduction order, is deterministic).
__global__ void k_sort_inc(const int64_t* __restrict__ off, int2* __restrict__ inc, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = off[i], e = off[i + 1];
    for (int64_t s = b + 1; s < e; ++s) {
      int2 key = inc[s];
      int64_t t = s - 1;
      while (t >= b && inc[t].x > key.x) {
        inc[t + 1] = inc[t];
        --t;
      }
      inc[t + 1] = key;
    }
  }
}

__global__ void k_span_setup(const int64_t* __restrict__ off, int64_t n, int nwg,
                             WarpSpan* __restrict__ spans) {
  const int64_t U = off[n] + n;
  auto node_of = [&](int64_t u) {  // largest i with off[i] + i <= u
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) / 2;
      if (off[mid] + mid <= u) lo = mid;
      else hi = mid - 1;
    }
    return (int)lo;
  };
  auto warp_of = [&](int64_t u) {  // largest w with U w / nwg <= u
    int lo = 0, hi = nwg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (U * mid / nwg <= u) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwg; w += gridDim.x * blockDim.x) {
    WarpSpan sp;
    sp.ub = U * w / nwg;
    sp.ue = U * (w + 1) / nwg;
    auto parts = [&](int wf, int wl) {  // non-empty spans among warps wf..wl
      int np = 0;
      for (int v = wf; v <= wl; ++v) np += (U * v / nwg < U * (v + 1) / nwg) ? 1 : 0;
      return np;
    };
    if (sp.ub >= sp.ue) {
      sp.i0 = 0;
      sp.i1 = -1;
      sp.wf0 = sp.wl0 = sp.wf1 = sp.wl1 = w;
      sp.np0 = sp.np1 = 1;
    } else {
      sp.i0 = node_of(sp.ub);
      sp.i1 = node_of(sp.ue - 1);
      sp.wf0 = warp_of(off[sp.i0] + sp.i0);
      sp.wl0 = warp_of(off[sp.i0 + 1] + sp.i0);
      sp.np0 = parts(sp.wf0, sp.wl0);
      sp.wf1 = warp_of(off[sp.i1] + sp.i1);
      sp.wl1 = warp_of(off[sp.i1 + 1] + sp.i1);
      sp.np1 = parts(sp.wf1, sp.wl1);
    }
    spans[w] = sp;
  }
}

int check_edges(Ctx* c, const int2* edges, int64_t m, int64_t n, const double* w,
                cudaStream_t s) {
  void* pb;
  CCM_TRY(ws_get(c, S_SCRATCH6, 64, &pb));
  int* bad = (int*)pb;
  CCM_CUDA(cudaMemsetAsync(bad, 0, 4, s));
  if (m > 0) {
    int blocks = (int)std::min<int64_t>((m + 255) / 256, (int64_t)c->num_sms * 8);
    k_validate_edges<<<blocks, 256, 0, s>>>(edges, m, n, w, bad);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
  }
  void* hp;
  CCM_TRY(host_scalars(c, 64, &hp));
  CCM_CUDA(cudaMemcpyAsync(hp, bad, 4, cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  if (*(int*)hp) {
    set_error("edges must satisfy 0 <= i < j < n, be sorted and unique; w finite and >= 0");
    return CCM_ERR_INVALID_ARG;
  }
  return CCM_OK;
}

// CSR of B^T: off[n+1] (int64), inc[2m] {edge id, other endpoint}, per-node
// lists in increasing edge id.
int build_csr(Ctx* c, const int2* edges, int64_t m, int64_t n, int64_t** off_out,
              int2** inc_out, cudaStream_t s) {
  void *p_off, *p_inc, *p_deg;
  CCM_TRY(ws_get(c, S_CSR_OFF, (size_t)(n + 1) * 8, &p_off));
  CCM_TRY(ws_get(c, S_CSR_INC, (size_t)std::max<int64_t>(2 * m, 1) * 8, &p_inc));
  CCM_TRY(ws_get(c, S_BATCH1, (size_t)(n + 1) * 8, &p_deg));
  int64_t* off = (int64_t*)p_off;
  unsigned long long* deg = (unsigned long long*)p_deg;
  CCM_CUDA(cudaMemsetAsync(deg, 0, (size_t)(n + 1) * 8, s));
  int blocks_m = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, c->num_sms * 8));
  int blocks_n = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, c->num_sms * 8));
  if (m > 0) {
    k_degree<<<blocks_m, 256, 0, s>>>(edges, m, deg);
    CCM_COUNT(c);
  }
  CCM_CUDA(cudaGetLastError());
  CCM_TRY(scan_exclusive_i64(c, (const int64_t*)deg, off, n + 1, nullptr, s));
  CCM_CUDA(cudaMemsetAsync(deg, 0, (size_t)(n + 1) * 8, s));
  if (m > 0) {
    k_fill_inc<<<blocks_m, 256, 0, s>>>(edges, m, off, deg, (int2*)p_inc);
    CCM_COUNT(c);
  }
  k_sort_inc<<<blocks_n, 256, 0, s>>>(off, (int2*)p_inc, n);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  *off_out = off;
  *inc_out = (int2*)p_inc;
  return CCM_OK;
}

template <typename Tc>
__global__ void k_fill_one(Tc* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (Tc)1;
}

// Host memory (pinned or pageable) as seen by the CUDA runtime.
static bool is_host_memory(const void* ptr) {
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered;
}

// ---------------------------------------------------------------- engine
template <int L, int CH, typename Tc>
struct GridEngine {
  static int run(Ctx* c, const SolveArgs& a, cudaStream_t s) {
    const int64_t n = a.n, m = a.m;
    const int d = a.d;
    const int ld = (int)round_up(d, 4);
    const int64_t nl = n * ld, ml = m * ld;
    const int threads = 256;
    const int gpb = threads / L;  // groups per block
    const int maxb = c->num_sms * 4;
    auto nb = [&](int64_t work) {
      return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, maxb));
    };
    const int b_edge = (int)std::max<int64_t>(1, std::min<int64_t>((m + gpb - 1) / gpb, maxb));
    // the q = 2 edge passes run in their own (narrower) group shape
    using ES = EdgeShape<L, CH>;
    const int gpb_e = threads / ES::L;
    const int b_edge2 =
        (int)std::max<int64_t>(1, std::min<int64_t>((m + gpb_e - 1) / gpb_e, 2 * maxb));
    using FS = FfEdgeShape<L, CH>;  // the float-float edge passes
    const int gpb_f = threads / FS::L;
    const int b_edge_ff =
        (int)std::max<int64_t>(1, std::min<int64_t>((m + gpb_f - 1) / gpb_f, 2 * maxb));
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
    CCM_TRY(get(S_P0, nl * sizeof(Tc), &p)); Tc* P = (Tc*)p;    // CG search direction
    CCM_TRY(get(S_P1, nl * sizeof(Tc), &p)); Tc* Sv = (Tc*)p;   // S = V P
    CCM_TRY(get(S_Q, nl * sizeof(Tc), &p)); Tc* W = (Tc*)p;     // W = V M R
    CCM_TRY(get(S_META, std::max<int64_t>(2 * m, 1) * sizeof(IncMeta<Tc>), &p));
    IncMeta<Tc>* meta = (IncMeta<Tc>*)p;
    CCM_TRY(get(S_MINV, n * sizeof(Tc), &p)); Tc* Minv = (Tc*)p;
    CCM_TRY(get(S_U, std::max<int64_t>(ml, 1) * 8, &p)); double* Ua = (double*)p;
    CCM_TRY(get(S_UT, std::max<int64_t>(ml, 1) * 8, &p)); double* Ub = (double*)p;
    // q = 2 with the float32 operator: the edge passes and the node gradient run
    // in float-float (ff_kernels.cuh); U / Pi(y) rows are then float-float rows
    // (same 8 bytes per element) and X has a float-float mirror
    const bool FF = a.q == 2 && sizeof(Tc) == 4;
    // two-level preconditioner (q = 2): its vectors are taken at first use
    const bool use_coarse = a.opt.coarse != 0 && a.q == 2;
    Tc* Uco = nullptr;   // U = M^-1 R
    Tc* ones = nullptr;  // unit Jacobi scalars for the operator on U
    float2 *XFa = nullptr, *XFb = nullptr;
    if (FF) {
      CCM_TRY(get(S_XF0, nl * 8, &p)); XFa = (float2*)p;
      CCM_TRY(get(S_XF1, nl * 8, &p)); XFb = (float2*)p;
    }
    CCM_TRY(get(S_YH, std::max<int64_t>(ml, 1) * sizeof(Tc), &p)); Tc* Yh = (Tc*)p;
    CCM_TRY(get(S_ALPHA, std::max<int64_t>(m, 1) * sizeof(Tc), &p)); Tc* alpha = (Tc*)p;
    CCM_TRY(get(S_KIND, std::max<int64_t>(m, 1), &p)); uint8_t* kind = (uint8_t*)p;
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
    // long rows: the shared-memory ring kernels over an even split of the
    // incidence stream (one span per warp)
#ifdef CCM_DEBUG_BOUNDS
    {
      const DebugBounds hb{(long long)n, (long long)m, 0, 0, 0};
      CCM_CUDA(cudaMemcpyToSymbolAsync(g_bounds, &hb, sizeof(hb), 0, cudaMemcpyHostToDevice, s));
      // fault injection for the tests of the bounds-checked library: one incidence
      // record gets an out-of-range endpoint, which the checks must catch before any
      // access
      if (getenv("CCM_DEBUG_CORRUPT") && m > 0) {
        const int bad = (int)n + 3;
        CCM_CUDA(cudaMemcpyAsync(&inc[0].y, &bad, sizeof(int), cudaMemcpyHostToDevice, s));
        CCM_CUDA(cudaStreamSynchronize(s));
      }
    }
#endif
    RingPlan rp;
    CCM_TRY(ring_plan<Tc>(c, L, ld, off, n, rp, s));
    // register forms with several row groups per warp: visit nodes of equal degree
    // together (windows of 4,096 nodes by decreasing degree)
    if (!rp.on() && L < 32 && n >= kDegreeOrderMinN) {
      CCM_TRY(get(S_ORDER, n * 4, &p));
      CCM_TRY(degree_order(c, off, n, (int*)p, s));
      rp.ord = (const int*)p;
    }
    CCM_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    k_gather_rows<<<b_elem, threads, 0, s>>>(a.A, Ap, n, d, ld, a.perm);
    CCM_COUNT(c);
    k_gather_rows<<<b_elem, threads, 0, s>>>(a.X0 ? a.X0 : a.A, Xa, n, d, ld, a.perm);
    CCM_COUNT(c);
    if (FF) {
      k_mirror_ff<<<b_elem, threads, 0, s>>>(Xa, XFa, nl);
      CCM_COUNT(c);
      CCM_CUDA(cudaMemsetAsync(XFb, 0, nl * 8, s));
    }
    if (m > 0) {
      if (a.U0 && FF) {
        k_pad_rows_ff<<<nb(ml), threads, 0, s>>>(a.U0, (float2*)Ua, m, d, ld, a.eperm);
        CCM_COUNT(c);
      } else if (a.U0) {
        k_gather_rows<<<nb(ml), threads, 0, s>>>(a.U0, Ua, m, d, ld, a.eperm);
        CCM_COUNT(c);
      } else {
        CCM_CUDA(cudaMemsetAsync(Ua, 0, ml * 8, s));
      }
    }
    // padding of every other node/edge buffer must be zero once
    CCM_CUDA(cudaMemsetAsync(Ub, 0, std::max<int64_t>(ml, 1) * 8, s));
    CCM_CUDA(cudaMemsetAsync(Xb, 0, nl * 8, s));
    CCM_CUDA(cudaMemsetAsync(Yh, 0, std::max<int64_t>(ml, 1) * sizeof(Tc), s));
    k_sumsq<<<b_elem, threads, 0, s>>>(Ap, nl, part, ctl);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    auto readback = [&]() -> int {
      CCM_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
      CCM_CUDA(cudaStreamSynchronize(s));
#ifdef CCM_DEBUG_BOUNDS
      DebugBounds hb{};
      CCM_CUDA(cudaMemcpyFromSymbol(&hb, g_bounds, sizeof(hb)));
      if (hb.err) {
        static const char* names[] = {"?", "k_cg_init", "k_cg_matvec", "k_cg_matvec_ring"};
        set_error("index check failed in %s at incidence record %lld (bounds-checked build)",
                  names[(hb.where >= 1 && hb.where <= 3) ? hb.where : 0], hb.index);
        const DebugBounds z{0, 0, 0, 0, 0};
        CCM_CUDA(cudaMemcpyToSymbol(g_bounds, &z, sizeof(z)));
        return CCM_ERR_BOUNDS;
      }
#endif
      return CCM_OK;
    };
    CCM_TRY(readback());
    const double nA = std::sqrt(hc->dots[1]);
    const double scale = 1.0 + nA;

    double* X = Xa;    // current iterate
    double* Xt = Xb;   // trial iterate
    double* U = Ua;    // current multipliers
    double* Ut = Ub;   // Pi(U + sigma B X) at the last evaluated point
    float2* XF = XFa;  // float-float mirrors of X and Xt (FF only)
    float2* XFt = XFb;
    double sigma = a.opt.sigma0;
    const bool prof = a.opt.profile != 0;
    ccm_profile profile = {};
    std::vector<cudaEvent_t>& ev = c->ev_pool;
    const int CHUNK = 8;
    if (prof && ev.size() < 2 * CHUNK) {
      while (ev.size() < 2 * CHUNK) {
        cudaEvent_t e;
        CCM_CUDA(cudaEventCreate(&e));
        ev.push_back(e);
      }
    }
    const double tc_floor = sizeof(Tc) == 4 ? 1e-5 : 1e-10;
    double gamma_cur = 0.0;
    int any_fail = 0;

    // evaluate phi, grad phi, Pi(y), yhat, alpha at Xc (one edge pass + one node pass)
    auto evaluate = [&](const double* Xc, const float2* XFc, double* phi, double* gn,
                        double* nout) -> int {
      if (FF) {
        k_edge_eval_ff<FS::L, FS::C, Tc><<<b_edge_ff, threads, 0, s>>>(
            XFc, (const float2*)U, edges, a.w, gamma_cur, sigma, (float2*)Ut, Yh, alpha, kind, m,
            ld, part, ctl);
        CCM_COUNT(c);
        CCM_TRY(launch_node_grad_ff<L, CH, Tc>(c, Xc, Ap, (const float2*)Ut, off, inc, alpha,
                                               kind, sigma, d, G, Minv, rp, n, ld, part, ctl, s));
        CCM_CUDA(cudaGetLastError());
        CCM_TRY(readback());
        *phi = hc->eval[1] + hc->eval[0] / sigma;
        *gn = std::sqrt(hc->eval[2]);
        if (nout) *nout = 0;
        return CCM_OK;
      }
      if (a.q == 1)
        k_edge_eval_qn<1, L, CH, Tc><<<b_edge, threads, 0, s>>>(
            Xc, U, edges, a.w, gamma_cur, sigma, Ut, Yh, alpha, kind, m, d, ld, part, ctl);
      else if (a.q == kQInf)
        k_edge_eval_qn<kQInf, L, CH, Tc><<<b_edge, threads, 0, s>>>(
            Xc, U, edges, a.w, gamma_cur, sigma, Ut, Yh, alpha, kind, m, d, ld, part, ctl);
      else
        k_edge_eval<ES::L, ES::C, Tc><<<b_edge2, threads, 0, s>>>(
            Xc, U, edges, a.w, gamma_cur, sigma, Ut, Yh, alpha, kind, m, ld, part, ctl);
      CCM_COUNT(c);
      CCM_TRY(launch_node_grad<L, CH, Tc>(c, Xc, Ap, Ut, off, inc, alpha, kind, sigma, d, G, Minv,
                                          rp, n, ld, part, ctl, s));
      CCM_CUDA(cudaGetLastError());
      CCM_TRY(readback());
      *phi = hc->eval[1] + hc->eval[0] / sigma;
      *gn = std::sqrt(hc->eval[2]);
      if (nout) *nout = 0;
      return CCM_OK;
    };

    for (int t = 0; t < a.T; ++t) {
      const double gamma = a.gammas[t];
      gamma_cur = gamma;
      ccm_stats st = {};
      double last_kkt = 1.0, last_etap = -1.0;
      sigma = std::min(sigma, a.opt.sigma_max);  // a raised cap lasts one gamma
      double cap = a.opt.sigma_max;
      int at_cap = 0;
      double eps_gap = 1.0;      // inner-tolerance cap from the duality gap (below)
      bool converged = false;
      double gn = 0, phi = 0;
      bool edge_ready = false;   // edge part of the evaluation at (X, U) already done
      double edge_sigma = 0.0;   // ... with this penalty (by k_kkt_edge_eval)
      for (int outer = 0; outer < a.opt.max_outer; ++outer) {
        const double eps_in = std::min(std::max(0.5 * a.tol, 0.1 * last_kkt), eps_gap);
        if (edge_ready && edge_sigma == sigma) {
          if (FF)
            CCM_TRY(launch_node_grad_ff<L, CH, Tc>(c, X, Ap, (const float2*)Ut, off, inc, alpha,
                                                   kind, sigma, d, G, Minv, rp, n, ld, part, ctl,
                                                   s));
          else
            CCM_TRY(launch_node_grad<L, CH, Tc>(c, X, Ap, Ut, off, inc, alpha, kind, sigma, d, G,
                                                Minv, rp, n, ld, part, ctl, s));
          CCM_CUDA(cudaGetLastError());
          CCM_TRY(readback());
          phi = hc->eval[1] + hc->eval[0] / sigma;
          gn = std::sqrt(hc->eval[2]);
        } else {
          CCM_TRY(evaluate(X, XF, &phi, &gn, nullptr));
        }
        edge_ready = false;
        for (int it = 0; it < a.opt.max_newton; ++it) {
          if (gn / scale <= eps_in) break;
          const double gr = gn / scale;
          const double eta = std::min(0.1, std::max(tc_floor, std::sqrt(gr)));
          // two-level preconditioner (options.coarse): when the strong edges form
          // aggregates, the CG runs on U = M^-1 R (coarse.cu) with unit Jacobi scalars
          CoarsePlan<Tc> cp;
          if (use_coarse) {
            CCM_TRY(coarse_build<Tc>(c, edges, kind, alpha, n, m, sigma, d, ld, cp, s));
            if (cp.K > 0) {
              if (!Uco) {
                CCM_TRY(get(S_CO_U, nl * sizeof(Tc), &p)); Uco = (Tc*)p;
                CCM_TRY(get(S_CO_ONES, n * sizeof(Tc), &p)); ones = (Tc*)p;
                k_fill_one<Tc><<<nb(n), threads, 0, s>>>(ones, n);
                CCM_COUNT(c);
              }
              profile.coarse_steps += 1;
              profile.coarse_max_aggregates = std::max(profile.coarse_max_aggregates, cp.K);
            }
          }
          const bool co = cp.K > 0;
          k_cg_init<Tc><<<b_elem, threads, 0, s>>>(G, co ? ones : Minv, R, Dx, n, ld, eta,
                                                   a.opt.max_cg, inc, kind, alpha, meta, 2 * m,
                                                   part, ctl);
          CCM_COUNT(c);
          CCM_CUDA(cudaGetLastError());
          int it_before = 0;
          for (int chunk = 0; chunk * CHUNK < a.opt.max_cg; ++chunk) {
            for (int k = 0; k < CHUNK; ++k) {
              if (co) CCM_TRY(coarse_precondition<Tc>(c, cp, R, Minv, Uco, n, ld, part, ctl, s));
              if (prof) CCM_CUDA(cudaEventRecord(ev[2 * k], s));
              CCM_TRY(launch_matvec<L, CH, Tc>(c, co ? Uco : R, co ? ones : Minv, nullptr, W, Yh,
                                                meta, off, inc, rp, sigma, n, ld, part, ctl, s));
              if (prof) CCM_CUDA(cudaEventRecord(ev[2 * k + 1], s));
              k_cg_update<Tc><<<b_quad, threads, 0, s>>>(Dx, P, Sv, R, W, Minv, n, ld, part, ctl,
                                                         co ? Uco : nullptr);
              CCM_COUNT(c);
            }
            CCM_CUDA(cudaGetLastError());
            CCM_TRY(readback());
            if (prof) {
              int active = hc->cg.it - it_before;
              for (int k = 0; k < active && k < CHUNK; ++k) {
                float ms = 0.f;
                CCM_CUDA(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
                profile.matvec_ms_total += ms;
                profile.matvec_launches += 1;
                profile.matvec_bytes_total += a.matvec_bytes(hc->eval[3], sizeof(Tc));
              }
            }
            it_before = hc->cg.it;
            if (!hc->cg.active) break;
          }
          st.cg += hc->cg.it;
          // Armijo backtracking on phi along Dx
          double tstep = 1.0;
          auto trial = [&]() {
            if (FF)
              k_trial_ff<Tc><<<b_elem, threads, 0, s>>>(X, Dx, G, tstep, Xt, XFt, nl, part, ctl);
            else
              k_trial<Tc><<<b_elem, threads, 0, s>>>(X, Dx, G, tstep, Xt, nl, part, ctl);
            CCM_COUNT(c);
          };
          trial();
          CCM_CUDA(cudaGetLastError());
          CCM_TRY(readback());
          const double gd = hc->dots[0];
          const double slack = 1e-14 * (1.0 + std::fabs(phi));
          double phit = 0, gnt = 0;
          for (;;) {
            CCM_TRY(evaluate(Xt, XFt, &phit, &gnt, nullptr));
            st.line_search += 1;
            if (phit <= phi + 1e-4 * tstep * gd + slack || tstep < 1e-10) break;
            tstep *= 0.5;
            trial();
            CCM_CUDA(cudaGetLastError());
          }
          std::swap(X, Xt);
          std::swap(XF, XFt);
          phi = phit;
          gn = gnt;
          st.newton += 1;
          if (tstep < 1e-10) break;
        }
        // multiplier update: U <- Pi(U + sigma B X) (computed at the last evaluation)
        std::swap(U, Ut);
        // KKT at (X, U) fused with the edge part of the next evaluation at (X, U)
        if (a.q == 1)
          k_kkt_edge_eval_qn<1, L, CH, Tc><<<b_edge, threads, 0, s>>>(
              X, U, edges, a.w, gamma, sigma, Ut, Yh, alpha, kind, m, d, ld, part, ctl);
        else if (a.q == kQInf)
          k_kkt_edge_eval_qn<kQInf, L, CH, Tc><<<b_edge, threads, 0, s>>>(
              X, U, edges, a.w, gamma, sigma, Ut, Yh, alpha, kind, m, d, ld, part, ctl);
        else if (FF)
          k_kkt_edge_eval_ff<FS::L, FS::C, Tc><<<b_edge_ff, threads, 0, s>>>(
              XF, (const float2*)U, edges, a.w, gamma, sigma, (float2*)Ut, Yh, alpha, kind, m, ld,
              part, ctl);
        else
          k_kkt_edge_eval<ES::L, ES::C, Tc><<<b_edge2, threads, 0, s>>>(
              X, U, edges, a.w, gamma, sigma, Ut, Yh, alpha, kind, m, ld, part, ctl);
        CCM_COUNT(c);
        edge_ready = true;
        edge_sigma = sigma;
        if (FF)
          k_kkt_node_ff<<<b_quad, threads, 0, s>>>(X, Ap, G, nl, part, ctl);
        else
          k_kkt_node<<<b_elem, threads, 0, s>>>(X, Ap, G, nl, part, ctl);
        CCM_COUNT(c);
        CCM_CUDA(cudaGetLastError());
        CCM_TRY(readback());
        st.outer += 1;
        const double eta_d = gn / scale;
        const double eta_p = std::sqrt(hc->kkt[0]) / scale;
        const double fp = hc->eval[1] + hc->kkt[1];
        const double fd = hc->kkt[2] - 0.5 * hc->kkt[3];
        const double gap = std::fabs(fp - fd) / (1.0 + std::fabs(fp) + std::fabs(fd));
        st.eta_d = eta_d;
        st.eta_p = eta_p;
        st.kkt = std::max(eta_d, eta_p);
        st.f_p = fp;
        st.f_d = fd;
        st.gap = gap;
        if (st.kkt <= a.tol && gap <= a.tol) {
          converged = true;
          break;
        }
        // f_p - f_d >= 1/2 ||X - A + B^T U||^2 for dual-feasible U, so a gap above
        // tol caps the inner tolerance at half the gradient norm that allows it
        if (gap > a.tol)
          eps_gap = std::min(eps_gap, 0.5 * std::sqrt(2.0 * a.tol * (1.0 + std::fabs(fp) +
                                                                     std::fabs(fd))) / scale);
        // penalty: x3 while eta_p falls by less than 5x per step, up to a cap that
        // starts at sigma_max and rises 10x after 20 outer steps spent at it
        if (last_etap >= 0 && eta_p > 0.2 * last_etap) sigma = std::min(3.0 * sigma, cap);
        if (sigma >= cap) {
          if (++at_cap >= 20) {
            cap = std::min(10.0 * cap, 1e6);
            at_cap = 0;
          }
        } else {
          at_cap = 0;
        }
        last_etap = eta_p;
        last_kkt = st.kkt;
      }
      st.sigma = sigma;
      st.status = converged ? CCM_OK : CCM_ERR_NOT_CONVERGED;
      if (!converged) any_fail = 1;
      k_scatter_rows<<<nb(n * d), threads, 0, s>>>(X, a.Xout + (int64_t)t * n * d, n, d, ld,
                                                   a.perm);
      CCM_COUNT(c);
      if (a.Xhost) {  // this gamma's X goes to the host while the next one solves
        CCM_CUDA(cudaEventRecord(a.copy_event, s));
        CCM_CUDA(cudaStreamWaitEvent(a.copy_stream, a.copy_event, 0));
        CCM_CUDA(cudaMemcpyAsync(a.Xhost + (int64_t)t * n * d, a.Xout + (int64_t)t * n * d,
                                 (size_t)n * d * 8, cudaMemcpyDeviceToHost, a.copy_stream));
      }
      if (a.Uout && m > 0) {
        if (FF)
          k_unpad_rows_ff<<<nb(m * d), threads, 0, s>>>((const float2*)U,
                                                        a.Uout + (int64_t)t * m * d, m, d, ld,
                                                        a.eperm);
        else
          k_scatter_rows<<<nb(m * d), threads, 0, s>>>(U, a.Uout + (int64_t)t * m * d, m, d, ld,
                                                       a.eperm);
        CCM_COUNT(c);
      }
      CCM_CUDA(cudaGetLastError());
      if (a.stats) a.stats[t] = st;
    }
    if (prof) c->last_profile = profile;
    return any_fail ? CCM_ERR_NOT_CONVERGED : CCM_OK;
  }
};

// Dispatch on (lanes per row, quads per lane) from ld/4 and on precision.
template <typename Tc>
static int run_grid(Ctx* c, const SolveArgs& a, cudaStream_t s) {
  const int nq = (int)(round_up(a.d, 4) / 4);
  if (nq <= 1) return GridEngine<1, 1, Tc>::run(c, a, s);
  if (nq <= 2) return GridEngine<2, 1, Tc>::run(c, a, s);
  if (nq <= 4) return GridEngine<4, 1, Tc>::run(c, a, s);
  if (nq <= 8) return GridEngine<8, 1, Tc>::run(c, a, s);
  if (nq <= 16) return GridEngine<16, 1, Tc>::run(c, a, s);
  if (nq <= 32) return GridEngine<32, 1, Tc>::run(c, a, s);
  if (nq <= 64) return GridEngine<32, 2, Tc>::run(c, a, s);
  if (nq <= 96) return GridEngine<32, 3, Tc>::run(c, a, s);
  if (nq <= 128) return GridEngine<32, 4, Tc>::run(c, a, s);
  if (nq <= 160) return GridEngine<32, 5, Tc>::run(c, a, s);
  if (nq <= 192) return GridEngine<32, 6, Tc>::run(c, a, s);
  if (nq <= 224) return GridEngine<32, 7, Tc>::run(c, a, s);
  if (nq <= 256) return GridEngine<32, 8, Tc>::run(c, a, s);
  set_error("d = %d exceeds the compiled maximum %d", a.d, ccm_max_dim());
  return CCM_ERR_UNSUPPORTED;
}

int solve_grid(Ctx* c, const SolveArgs& a, cudaStream_t s) {
  return a.opt.precision == CCM_PREC_FP64 ? run_grid<double>(c, a, s) : run_grid<float>(c, a, s);
}

}  // namespace ccm

using namespace ccm;

extern "C" int ccm_solve_path(ccm_ctx* x, const double* A, int64_t n, int32_t d,
                              const int32_t* edges, const double* w, int64_t m,
                              const double* gammas, int32_t T, int32_t q, double tol,
                              const ccm_options* opt, double* X, int32_t* labels, double* U,
                              ccm_stats* stats, ccm_stream_t stream) {
  Ctx* c = ctx_of(x);
  if (!c || !A || !X || !gammas || n < 1 || d < 1 || m < 0 || T < 1 || (m > 0 && (!edges || !w)) ||
      !(tol > 0) || n > INT32_MAX || m > INT32_MAX) {
    set_error("ccm_solve_path: invalid argument");
    return CCM_ERR_INVALID_ARG;
  }
  if (q != 2 && q != 1 && q != CCM_Q_INF) {
    set_error("ccm_solve_path: q = 1, q = 2 and q = inf (CCM_Q_INF) are implemented (got q = %d)",
              q);
    return CCM_ERR_UNSUPPORTED;
  }
  if (d > ccm_max_dim()) {
    set_error("ccm_solve_path: d = %d exceeds the maximum %d", d, ccm_max_dim());
    return CCM_ERR_UNSUPPORTED;
  }
  for (int t = 0; t < T; ++t) {
    if (!(gammas[t] >= 0) || !std::isfinite(gammas[t]) || (t > 0 && gammas[t] < gammas[t - 1])) {
      set_error("ccm_solve_path: gammas must be finite, >= 0 and non-decreasing");
      return CCM_ERR_INVALID_ARG;
    }
  }
  if (((uintptr_t)edges) % 8 || ((uintptr_t)A) % 8 || ((uintptr_t)X) % 8) {
    set_error("ccm_solve_path: misaligned pointer");
    return CCM_ERR_INVALID_ARG;
  }
  ccm_options o;
  ccm_default_options(&o);
  if (opt) o = *opt;
  o.sigma_max = resolve_sigma_max(o, q);
  if (o.max_outer < 1 || o.max_newton < 1 || o.max_cg < 1 || !(o.sigma0 > 0) ||
      !(o.sigma_max >= o.sigma0)) {
    set_error("ccm_solve_path: invalid options");
    return CCM_ERR_INVALID_ARG;
  }
  CCM_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  // X and labels may be host memory: the path then runs on device staging
  // buffers and the outputs are copied out (X of each gamma while the next one
  // solves, on the context's copy stream); U must be device memory
  const bool x_host = is_host_memory(X), l_host = labels && is_host_memory(labels);
  if (U && is_host_memory(U)) {
    set_error("ccm_solve_path: U must be device memory");
    return CCM_ERR_INVALID_ARG;
  }
  CCM_TRY(check_edges(c, (const int2*)edges, m, n, w, s));
  double* Xd = X;
  int32_t* Ld = labels;
  void* p;
  if (x_host) {
    CCM_TRY(ws_get(c, S_XSTAGE, (size_t)T * n * d * 8, &p));
    Xd = (double*)p;
    if (!c->copy_stream) {
      CCM_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
      CCM_CUDA(cudaEventCreateWithFlags(&c->copy_event, cudaEventDisableTiming));
    }
  }
  if (l_host) {
    CCM_TRY(ws_get(c, S_LSTAGE, (size_t)T * n * 4, &p));
    Ld = (int32_t*)p;
  }
  SolveArgs a;
  a.A = A; a.n = n; a.d = d; a.edges = edges; a.w = w; a.m = m;
  a.gammas = gammas; a.T = T; a.tol = tol; a.opt = o; a.Xout = Xd; a.Uout = U;
  a.stats = stats; a.X0 = o.X0; a.U0 = o.U0; a.q = q;
  c->last_profile = ccm_profile{};
  const int64_t launches0 = c->launches;
  // small problems: one thread block runs the whole path (no host round trips);
  // otherwise the grid engine spreads every phase over the whole GPU
  const int64_t ldd = round_up(d, 4);
  const bool small = n * ldd <= 16384 && m * ldd <= 131072 && d <= 128;
  // the block engine starts every path cold: a warm start (X0 / U0) runs on the grid engine
  const bool warm = o.X0 != nullptr || o.U0 != nullptr;
  const bool use_block =
      o.engine == CCM_ENGINE_BLOCK || (o.engine == CCM_ENGINE_AUTO && small && q == 2 && !warm);
  if (o.engine == CCM_ENGINE_BLOCK && (d > 128 || q != 2 || warm)) {
    set_error("ccm_solve_path: the block engine supports q = 2, d <= 128 and no warm start");
    return CCM_ERR_UNSUPPORTED;
  }
  if (use_block) {
    int st = solve_single_block(c, a, Ld, s);
    if (st == CCM_OK || st == CCM_ERR_NOT_CONVERGED) {
      if (x_host)
        CCM_CUDA(cudaMemcpyAsync(X, Xd, (size_t)T * n * d * 8, cudaMemcpyDeviceToHost, s));
      if (l_host)
        CCM_CUDA(cudaMemcpyAsync(labels, Ld, (size_t)T * n * 4, cudaMemcpyDeviceToHost, s));
      CCM_CUDA(cudaStreamSynchronize(s));
    }
    c->last_profile.kernel_launches = c->launches - launches0;
    if (st == CCM_ERR_NOT_CONVERGED) set_error("ccm_solve_path: some gamma hit an iteration cap");
    return st;
  }
  if (x_host) {
    a.Xhost = X;
    a.copy_stream = c->copy_stream;
    a.copy_event = c->copy_event;
  }
  // large graphs: solve with the nodes grouped by connected component (locality of
  // the gathers); the engine reads and writes the caller's arrays through the maps
  if (o.relabel && n >= kRelabelMinN && m > 0) {
    Relabel r;
    CCM_TRY(locality_relabel(c, (const int2*)edges, w, m, n, r, s));
    a.edges = (const int32_t*)r.edges;
    a.w = r.w;
    a.perm = r.perm;
    a.eperm = r.eperm;
  }
  // no copy into the caller's host memory may outlive the call: the copy stream
  // is drained on every way out (the labels below overlap the last gamma's copy)
  struct CopyDrain {
    cudaStream_t cs;
    ~CopyDrain() {
      if (cs) cudaStreamSynchronize(cs);
    }
  } drain{x_host ? c->copy_stream : nullptr};
  int st = solve_grid(c, a, s);
  if (st != CCM_OK && st != CCM_ERR_NOT_CONVERGED) return st;
  if (labels) {
    for (int t = 0; t < T; ++t) {
      int32_t nc = 0;
      CCM_TRY(labels_device(c, Xd + (int64_t)t * n * d, d, n, d, (const int2*)edges, m,
                            Ld + (int64_t)t * n, stats ? &nc : nullptr, s));
      if (stats) stats[t].n_clusters = nc;
    }
    if (l_host)
      CCM_CUDA(cudaMemcpyAsync(labels, Ld, (size_t)T * n * 4, cudaMemcpyDeviceToHost, s));
  }
  CCM_CUDA(cudaStreamSynchronize(s));
  if (x_host) CCM_CUDA(cudaStreamSynchronize(c->copy_stream));
  c->last_profile.kernel_launches = c->launches - launches0;
  if (st == CCM_ERR_NOT_CONVERGED) set_error("ccm_solve_path: some gamma hit an iteration cap");
  return st;
}
