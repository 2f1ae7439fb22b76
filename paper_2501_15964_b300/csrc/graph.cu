// ccm_build_graph: symmetrized exact kNN graph with Gaussian weights.
//
// The weights of model CCM (Sec. 1; computed by the Data Processor, Sec. 2.2
// item 1) are w_ij = exp(-phi D_ij) on the union of the directed kNN pairs,
// with D the canonical float64 squared distance (ascending features, one
// rounding per operation, no FMA) and ties broken by the smaller index.
//
// Pipeline (all on the device):
//  1. centre A (float64 column means) and round to float32 rows At;
//  2. k_knn_tile: every block owns 64 query rows and sweeps all columns in
//     64-wide tiles, computing float32 sum_k (At_ik - At_jk)^2 in registers
//     (4x4 per thread) and keeping, per row, the K' smallest in shared memory;
//  3. k_rerank: recompute the K' candidates' canonical float64 distances,
//     order by (D, j), keep the first k, and certify the row: with u = 2^-24,
//     |D~ - D| <= E(D~) = 2 [g_d D~/(1-g_d) + 8u'(1+u')(n_i + n_max)],
//     g_d = d u/(1 - d u), u' = u(1+2u), n_i = ||At_i||^2; every column outside
//     the list has D~ >= D~_(K'), so if D~_(K') - E(D~_(K')) > D_(k) (exact)
//     no outside column can enter the top k. Rows that fail are flagged;
//  4. k_exact_row: flagged rows are searched exhaustively in float64;
//  5. bucket the (min, max) pairs by min, sort and deduplicate each bucket,
//     emit edges in lexicographic order;
//  6. canonical D per edge, phi (given, or 1 / lower median by an exact
//     radix select on the float64 bit patterns), w = exp(-(phi * D)).
#include <algorithm>
#include <cmath>

#include "ccm_internal.cuh"

namespace ccm {

static constexpr int TR = 64, TC = 64, TK = 16, KMAX = 64;

__device__ __forceinline__ double canon_sqdist(const double* __restrict__ a,
                                               const double* __restrict__ b, int d) {
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    double dl = __dsub_rn(a[k], b[k]);
    acc = __dadd_rn(acc, __dmul_rn(dl, dl));
  }
  return acc;
}

__device__ __forceinline__ bool key_less(double d1, int j1, double d2, int j2) {
  return d1 < d2 || (d1 == d2 && j1 < j2);
}

__global__ void k_check_finite(const double* __restrict__ A, int64_t total, int* bad) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(A[q])) atomicExch(bad, 1);
}

// column means (one thread per column, rows in order: deterministic)
// Column means in two fixed-order passes: block b sums the rows
// [b R, (b+1) R) of every column (consecutive threads read consecutive columns
// of a row), then one thread per column adds the block partials in block order.
__global__ void k_colsum_part(const double* __restrict__ A, int64_t n, int d, int64_t R,
                              double* __restrict__ part) {
  const int64_t i0 = (int64_t)blockIdx.x * R, i1 = min(n, i0 + R);
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) s += A[i * d + k];
    part[(int64_t)blockIdx.x * d + k] = s;
  }
}

__global__ void k_colmean(const double* __restrict__ part, int nparts, int64_t n, int d,
                          double* __restrict__ mu) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * d + k];
  mu[k] = s / (double)n;
}

// At = float32(A - mu), rows padded to ldf (multiple of TK) with zeros; rows
// n..n_pad-1 zero. nrm[i] = sum_k At_ik^2 (float64).
__global__ void k_center(const double* __restrict__ A, int64_t n, int d, int ldf,
                         const double* __restrict__ mu, float* __restrict__ At,
                         double* __restrict__ nrm, int64_t n_pad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < ldf; ++k) {
      float v = 0.f;
      if (i < n && k < d) v = (float)(A[i * d + k] - mu[k]);
      At[i * ldf + k] = v;
      s += (double)v * (double)v;
    }
    if (i < n) nrm[i] = s;
  }
}

__global__ void k_max_nrm(const double* __restrict__ nrm, int64_t n, double* out) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v = fmax(v, nrm[i]);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

struct TileSmem {
  float As[TK][TR + 4];
  float Bs[TK][TC + 4];
  float listd[TR][KMAX];
  int listj[TR][KMAX];
  float bufd[TR][TC];
  int bufj[TR][TC];
  float thr[TR];
  int cnt[TR];
  int bufn[TR];
};

__global__ void __launch_bounds__(256)
k_knn_tile(const float* __restrict__ At, int ldf, int64_t n, int Kp, int* __restrict__ cand,
           float* __restrict__ cand_thr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t row0 = (int64_t)blockIdx.x * TR;
  if (tid < TR) {
    S.cnt[tid] = 0;
    S.thr[tid] = INFINITY;
    S.bufn[tid] = 0;
  }
  __syncthreads();
  for (int64_t col0 = 0; col0 < n; col0 += TC) {
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int k0 = 0; k0 < ldf; k0 += TK) {
      {  // 64 rows x 16 features for each of As and Bs: one float4 per thread
        const int r = tid / 4, kq = (tid % 4) * 4;
        float4 va = *reinterpret_cast<const float4*>(At + (row0 + r) * ldf + k0 + kq);
        float4 vb = *reinterpret_cast<const float4*>(At + (col0 + r) * ldf + k0 + kq);
        S.As[kq + 0][r] = va.x; S.As[kq + 1][r] = va.y; S.As[kq + 2][r] = va.z; S.As[kq + 3][r] = va.w;
        S.Bs[kq + 0][r] = vb.x; S.Bs[kq + 1][r] = vb.y; S.Bs[kq + 2][r] = vb.z; S.Bs[kq + 3][r] = vb.w;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        float a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = S.As[kk][ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = S.Bs[kk][tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float df = a[r] - b[c];
            acc[r][c] = fmaf(df, df, acc[r][c]);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = ty * 4 + r;
      const int64_t gi = row0 + row;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gj = col0 + tx * 4 + c;
        if (gi < n && gj < n && gj != gi && acc[r][c] < S.thr[row]) {
          int p = atomicAdd(&S.bufn[row], 1);
          S.bufd[row][p] = acc[r][c];
          S.bufj[row][p] = (int)gj;
        }
      }
    }
    __syncthreads();
    if (tid < TR) {
      const int row = tid;
      int cnt = S.cnt[row];
      for (int b = 0; b < S.bufn[row]; ++b) {
        float dv = S.bufd[row][b];
        int jv = S.bufj[row][b];
        if (cnt == Kp && !(dv < S.listd[row][Kp - 1])) continue;
        int pos = (cnt < Kp) ? cnt : Kp - 1;
        while (pos > 0 && S.listd[row][pos - 1] > dv) {
          S.listd[row][pos] = S.listd[row][pos - 1];
          S.listj[row][pos] = S.listj[row][pos - 1];
          --pos;
        }
        S.listd[row][pos] = dv;
        S.listj[row][pos] = jv;
        if (cnt < Kp) ++cnt;
      }
      S.cnt[row] = cnt;
      S.bufn[row] = 0;
      S.thr[row] = (cnt == Kp) ? S.listd[row][Kp - 1] : INFINITY;
    }
    __syncthreads();
  }
  if (tid < TR && row0 + tid < n) {
    const int64_t gi = row0 + tid;
    for (int t = 0; t < Kp; ++t) cand[gi * Kp + t] = (t < S.cnt[tid]) ? S.listj[tid][t] : -1;
    cand_thr[gi] = S.thr[tid];
  }
}

// Canonical rerank of the K' candidates of each row; certify or flag.
// tc_steps = 0: the candidates come from k_knn_tile (float32 direct differences,
// the bound in the header comment). tc_steps > 0: they come from the tensor-core
// Gram form of knn_tc.cu with tc_steps tcgen05.mma accumulation steps along K;
// with b the float32 centred rows, n_i = ||b_i||^2, N = max n_j, u_k = 2^-k:
//   E_G = 4 (u22 + S u22) sqrt(n_i N) + u21 (n_i + N)     (split remainder l l,
//         float32 accumulation, float32 norms and the final combination),
//   delta = u22 (sqrt(n_i) + sqrt(N))                    (|b' - (A - mu)| per row),
//   E_R = 2 (sqrt(D~ + E_G) + delta) delta + delta^2     (from ||b'_i - b'_j|| to ||a_i - a_j||),
//   E = (E_G + E_R)(1 + 1e-6) + d 2^-50 (D~ + E_G + E_R)  (canonical float64 rounding),
// and the row is certified if D~_(K') - E(D~_(K')) > D_(k).
__global__ void k_rerank(const double* __restrict__ A, int64_t n, int d, int k, int Kp,
                         const int* __restrict__ cand, const float* __restrict__ cand_thr,
                         const double* __restrict__ nrm, const double* __restrict__ nmax_p,
                         int tc_steps, int* __restrict__ nbr, int* __restrict__ flag) {
  const double u = 5.9604644775390625e-08;  // 2^-24
  const double up = u * (1.0 + 2.0 * u);
  const double gd = d * u / (1.0 - d * u);
  const double u22 = 2.384185791015625e-07, u21 = 4.76837158203125e-07;  // 2^-22, 2^-21
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double dl[KMAX];
    int jl[KMAX];
    int cnt = 0;
    for (int t = 0; t < Kp; ++t) {
      int j = cand[i * Kp + t];
      if (j < 0) continue;
      double D = canon_sqdist(A + i * d, A + (int64_t)j * d, d);
      int pos = cnt++;
      while (pos > 0 && key_less(D, j, dl[pos - 1], jl[pos - 1])) {
        dl[pos] = dl[pos - 1];
        jl[pos] = jl[pos - 1];
        --pos;
      }
      dl[pos] = D;
      jl[pos] = j;
    }
    bool ok = cnt >= k;
    if (ok && cnt == Kp && (int64_t)Kp < n - 1) {
      const double thr = (double)cand_thr[i];
      double E;
      if (tc_steps > 0) {
        const double ni = nrm[i], N = *nmax_p;
        const double EG = 4.0 * (u22 + tc_steps * u22) * sqrt(ni * N) + u21 * (ni + N);
        const double dl_ = u22 * (sqrt(ni) + sqrt(N));
        const double ER = 2.0 * (sqrt(fmax(thr, 0.0) + EG) + dl_) * dl_ + dl_ * dl_;
        E = (EG + ER) * (1.0 + 1e-6) + d * 8.881784197001252e-16 * (fmax(thr, 0.0) + EG + ER);
      } else {
        E = 2.0 * (gd * thr / (1.0 - gd) +
                   8.0 * up * (1.0 + up) * (nrm[i] + *nmax_p) * (1.0 + 1e-12));
      }
      ok = (thr - E) > dl[k - 1];
    }
    for (int t = 0; t < k; ++t) nbr[i * k + t] = ok ? jl[t] : -1;
    flag[i] = ok ? 0 : 1;
  }
}

__global__ void k_compact_flags(const int* __restrict__ flag, int64_t n, int* __restrict__ rows,
                                int* __restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) rows[atomicAdd(count, 1)] = (int)i;
}

// Exhaustive float64 kNN for one flagged row per block (rows[b]); k rounds of
// a block-wide minimum of (D, j) above the previous key.
__global__ void __launch_bounds__(256)
k_exact_row(const double* __restrict__ A, int64_t n, int d, int k, const int* __restrict__ rows,
            int nrows, double* __restrict__ Dbuf, int* __restrict__ nbr) {
  __shared__ double shd[32];
  __shared__ int shj[32];
  for (int rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
    const int64_t i = rows[rb];
    double* D = Dbuf + (int64_t)blockIdx.x * n;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
      D[j] = (j == i) ? INFINITY : canon_sqdist(A + i * d, A + j * d, d);
    __syncthreads();
    double pd = -1.0;
    int pj = -1;
    for (int t = 0; t < k; ++t) {
      double bd = INFINITY;
      int bj = INT32_MAX;
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        double v = D[j];
        if (key_less(pd, pj, v, (int)j) && key_less(v, (int)j, bd, bj)) {
          bd = v;
          bj = (int)j;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double od = __shfl_xor_sync(0xffffffffu, bd, o);
        int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (key_less(od, oj, bd, bj)) {
          bd = od;
          bj = oj;
        }
      }
      if ((threadIdx.x & 31) == 0) {
        shd[threadIdx.x >> 5] = bd;
        shj[threadIdx.x >> 5] = bj;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
          if (key_less(shd[w], shj[w], shd[0], shj[0])) {
            shd[0] = shd[w];
            shj[0] = shj[w];
          }
        nbr[i * k + t] = shj[0];
      }
      __syncthreads();
      pd = shd[0];
      pj = shj[0];
      __syncthreads();
    }
    __syncthreads();
  }
}

// ---- symmetrize
__global__ void k_bucket_count(const int* __restrict__ nbr, int64_t n, int k,
                               unsigned long long* __restrict__ cnt) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * k;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = q / k;
    int j = nbr[q];
    atomicAdd(cnt + (i < j ? i : j), 1ull);
  }
}

__global__ void k_bucket_fill(const int* __restrict__ nbr, int64_t n, int k,
                              const int64_t* __restrict__ boff,
                              unsigned long long* __restrict__ cur, int* __restrict__ bucket) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * k;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = q / k;
    int j = nbr[q];
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    unsigned long long p = atomicAdd(cur + lo, 1ull);
    bucket[boff[lo] + (int64_t)p] = (int)hi;
  }
}

// sort each bucket ascending, remove duplicates in place, count uniques
__global__ void k_bucket_unique(const int64_t* __restrict__ boff, int* __restrict__ bucket,
                                int64_t n, int64_t* __restrict__ ucnt) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = boff[b], e = boff[b + 1];
    for (int64_t p = s + 1; p < e; ++p) {
      int key = bucket[p];
      int64_t t = p - 1;
      while (t >= s && bucket[t] > key) {
        bucket[t + 1] = bucket[t];
        --t;
      }
      bucket[t + 1] = key;
    }
    int64_t u = 0;
    for (int64_t p = s; p < e; ++p)
      if (p == s || bucket[p] != bucket[p - 1]) bucket[s + u++] = bucket[p];
    ucnt[b] = u;
  }
}

__global__ void k_emit_edges(const int64_t* __restrict__ boff, const int* __restrict__ bucket,
                             const int64_t* __restrict__ ucnt, const int64_t* __restrict__ eoff,
                             int64_t n, int2* __restrict__ edges) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = boff[b], o = eoff[b];
    for (int64_t t = 0; t < ucnt[b]; ++t) edges[o + t] = make_int2((int)b, bucket[s + t]);
  }
}

__global__ void k_edge_dist(const double* __restrict__ A, int d, const int2* __restrict__ edges,
                            int64_t m, double* __restrict__ D) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int2 ij = edges[e];
    D[e] = canon_sqdist(A + (int64_t)ij.x * d, A + (int64_t)ij.y * d, d);
  }
}

// histogram of byte `shift` of the bit patterns whose higher bits equal prefix
__global__ void k_radix_hist(const double* __restrict__ D, int64_t m, int shift,
                             unsigned long long prefix, unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long h[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const unsigned long long hmask = (shift >= 56) ? 0ull : (~0ull << (shift + 8));
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(D[e]);
    if ((b & hmask) == prefix) atomicAdd(&h[(b >> shift) & 255ull], 1ull);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    if (h[t]) atomicAdd(hist + t, h[t]);
}

__global__ void k_weights(const double* __restrict__ D, int64_t m, double phi,
                          double* __restrict__ w) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    w[e] = exp(-__dmul_rn(phi, D[e]));
}

static int sync_read(Ctx* c, const void* dptr, size_t bytes, void** host, cudaStream_t s) {
  CCM_TRY(host_scalars(c, std::max<size_t>(bytes, 64), host));
  CCM_CUDA(cudaMemcpyAsync(*host, dptr, bytes, cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  return CCM_OK;
}

int build_graph_device(Ctx* c, const double* A, int64_t n, int d, int k, double phi,
                       int32_t* edges_out, double* w_out, int64_t cap, int64_t* m_out,
                       double* phi_out, int force_exact, cudaStream_t s) {
  const int threads = 256;
  auto nb = [&](int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads,
                                                       (int64_t)c->num_sms * 8));
  };
  void* p;
  void* hp;
  // 0. finite check
  CCM_TRY(ws_get(c, S_SCRATCH6, 64, &p));
  int* bad = (int*)p;
  CCM_CUDA(cudaMemsetAsync(bad, 0, 4, s));
  k_check_finite<<<nb(n * d), threads, 0, s>>>(A, n * d, bad);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  CCM_TRY(sync_read(c, bad, 4, &hp, s));
  if (*(int*)hp) {
    set_error("ccm_build_graph: A has non-finite entries");
    return CCM_ERR_INVALID_ARG;
  }
  const int Kp = (int)std::min<int64_t>(std::min(k + std::max(8, k), KMAX), n - 1);
  const int ldf = (int)round_up(d, TK);
  const int64_t n_pad = round_up(n, std::max(TR, TC));
  // 1. centre
  CCM_TRY(ws_get(c, S_AP, (size_t)n_pad * ldf * 4 + 16, &p));
  float* At = (float*)p;
  const int64_t rows_per_part = 256;
  const int nparts = (int)((n + rows_per_part - 1) / rows_per_part);
  CCM_TRY(ws_get(c, S_X0, ((size_t)round_up(d, 8) + (size_t)n + 8 + (size_t)nparts * d) * 8, &p));
  double* mu = (double*)p;
  double* nrm = mu + round_up(d, 8);
  double* nmax = nrm + n;
  double* colpart = nmax + 8;
  k_colsum_part<<<nparts, 128, 0, s>>>(A, n, d, rows_per_part, colpart);
  CCM_COUNT(c);
  k_colmean<<<(d + 127) / 128, 128, 0, s>>>(colpart, nparts, n, d, mu);
  CCM_COUNT(c);
  k_center<<<nb(n_pad), threads, 0, s>>>(A, n, d, ldf, mu, At, nrm, n_pad);
  CCM_COUNT(c);
  k_max_nrm<<<1, 256, 0, s>>>(nrm, n, nmax);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  // 2. candidates: tensor cores (d <= 128), else float32 SIMT tiles
  CCM_TRY(ws_get(c, S_X1, (size_t)n * KMAX * 4, &p));
  int* cand = (int*)p;
  CCM_TRY(ws_get(c, S_G, (size_t)n * 4, &p));
  float* cthr = (float*)p;
  int tc_steps = 0;
  int Kc = Kp;  // candidates per row actually produced
  if (knn_tc_supported(d, Kp)) {
    int used = 0;
    const int st = knn_candidates_tc(c, At, ldf, n, d, Kp, cand, cthr, &used, s);
    if (st == CCM_OK) {
      Kc = (int)std::min<int64_t>(used, KMAX);
      tc_steps = 3 * (int)(round_up(d, 32) / 8);
    } else if (st != CCM_ERR_TIMEOUT && st != CCM_ERR_UNSUPPORTED) {
      return st;
    }
  }
  if (tc_steps == 0) {
    size_t smem = sizeof(TileSmem);
    CCM_CUDA(cudaFuncSetAttribute(k_knn_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    k_knn_tile<<<(unsigned)(n_pad / TR), threads, smem, s>>>(At, ldf, n, Kp, cand, cthr);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
  }
  // 3. rerank
  CCM_TRY(ws_get(c, S_DX, (size_t)n * k * 4, &p));
  int* nbr = (int*)p;
  CCM_TRY(ws_get(c, S_R, (size_t)n * 4 * 2 + 64, &p));
  int* flag = (int*)p;
  int* rows = flag + n;
  int* nflag = rows + n;
  k_rerank<<<nb(n), 128, 0, s>>>(A, n, d, k, Kc, cand, cthr, nrm, nmax, tc_steps, nbr, flag);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  if (force_exact)  // every row exhaustively (exercises the fallback path)
    CCM_CUDA(cudaMemsetAsync(flag, 0xff, (size_t)n * 4, s));
  CCM_CUDA(cudaMemsetAsync(nflag, 0, 4, s));
  k_compact_flags<<<nb(n), threads, 0, s>>>(flag, n, rows, nflag);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  CCM_TRY(sync_read(c, nflag, 4, &hp, s));
  const int nrows = *(int*)hp;
  c->last_graph.candidates = tc_steps > 0 ? 1 : 0;
  c->last_graph.per_row = Kc;
  c->last_graph.rows_exhaustive = nrows;
  if (nrows > 0) {
    const int fb = (int)std::min<int64_t>(nrows, std::max<int64_t>(1, ((int64_t)1 << 28) / (n * 8) ));
    const int blocks = std::max(1, std::min(fb, c->num_sms * 4));
    CCM_TRY(ws_get(c, S_P0, (size_t)blocks * n * 8, &p));
    k_exact_row<<<blocks, 256, 0, s>>>(A, n, d, k, rows, nrows, (double*)p, nbr);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
  }
  // 4. symmetrize
  CCM_TRY(ws_get(c, S_P1, (size_t)(n + 1) * 8, &p));
  unsigned long long* bcnt = (unsigned long long*)p;
  CCM_TRY(ws_get(c, S_Q, (size_t)(n + 1) * 8, &p));
  int64_t* boff = (int64_t*)p;
  CCM_TRY(ws_get(c, S_U, (size_t)n * k * 4 + 16, &p));
  int* bucket = (int*)p;
  CCM_TRY(ws_get(c, S_UT, (size_t)(n + 1) * 8 * 2, &p));
  int64_t* ucnt = (int64_t*)p;
  int64_t* eoff = ucnt + (n + 1);
  CCM_CUDA(cudaMemsetAsync(bcnt, 0, (size_t)(n + 1) * 8, s));
  k_bucket_count<<<nb(n * k), threads, 0, s>>>(nbr, n, k, bcnt);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  CCM_TRY(scan_exclusive_i64(c, (const int64_t*)bcnt, boff, n + 1, nullptr, s));
  CCM_CUDA(cudaMemsetAsync(bcnt, 0, (size_t)(n + 1) * 8, s));
  k_bucket_fill<<<nb(n * k), threads, 0, s>>>(nbr, n, k, boff, bcnt, bucket);
  CCM_COUNT(c);
  k_bucket_unique<<<nb(n), threads, 0, s>>>(boff, bucket, n, ucnt);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  int64_t m = 0;
  CCM_TRY(scan_exclusive_i64(c, ucnt, eoff, n, &m, s));
  *m_out = m;
  if (m > cap) {
    set_error("ccm_build_graph: %lld edges exceed capacity %lld", (long long)m, (long long)cap);
    return CCM_ERR_BUFFER_TOO_SMALL;
  }
  k_emit_edges<<<nb(n), threads, 0, s>>>(boff, bucket, ucnt, eoff, n, (int2*)edges_out);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  // 5. weights
  CCM_TRY(ws_get(c, S_YH, (size_t)std::max<int64_t>(m, 1) * 8, &p));
  double* D = (double*)p;
  k_edge_dist<<<nb(m), threads, 0, s>>>(A, d, (const int2*)edges_out, m, D);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  double ph = phi;
  if (!(phi > 0)) {
    if (m == 0) {
      set_error("ccm_build_graph: no edges, cannot take a median");
      return CCM_ERR_INVALID_ARG;
    }
    CCM_TRY(ws_get(c, S_ALPHA, 256 * 8, &p));
    unsigned long long* hist = (unsigned long long*)p;
    unsigned long long prefix = 0;
    int64_t rank = (m - 1) / 2;
    for (int shift = 56; shift >= 0; shift -= 8) {
      CCM_CUDA(cudaMemsetAsync(hist, 0, 256 * 8, s));
      k_radix_hist<<<nb(m), threads, 0, s>>>(D, m, shift, prefix, hist);
      CCM_COUNT(c);
      CCM_CUDA(cudaGetLastError());
      CCM_TRY(sync_read(c, hist, 256 * 8, &hp, s));
      const unsigned long long* h = (const unsigned long long*)hp;
      int bin = 0;
      for (; bin < 256; ++bin) {
        if ((int64_t)h[bin] > rank) break;
        rank -= (int64_t)h[bin];
      }
      if (bin == 256) {
        set_error("ccm_build_graph: median selection failed");
        return CCM_ERR_CUDA;
      }
      prefix |= ((unsigned long long)bin) << shift;
    }
    double med;
    memcpy(&med, &prefix, 8);
    if (!(med > 0)) {
      set_error("ccm_build_graph: lower median of edge distances is zero");
      return CCM_ERR_INVALID_ARG;
    }
    ph = 1.0 / med;
  }
  k_weights<<<nb(m), threads, 0, s>>>(D, m, ph, w_out);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  CCM_CUDA(cudaStreamSynchronize(s));
  *phi_out = ph;
  return CCM_OK;
}

}  // namespace ccm

using namespace ccm;

extern "C" int ccm_build_graph(ccm_ctx* x, const double* A, int64_t n, int32_t d, int32_t k,
                               double phi, int32_t* edges, double* w, int64_t cap,
                               int64_t* m_out, double* phi_out, ccm_stream_t stream) {
  Ctx* c = ctx_of(x);
  if (!c || !A || !edges || !w || !m_out || !phi_out || n < 2 || d < 1 || k < 1 || k >= n ||
      n > INT32_MAX || cap < 0 || !std::isfinite(phi)) {
    set_error("ccm_build_graph: invalid argument");
    return CCM_ERR_INVALID_ARG;
  }
  if (k > 32) {
    set_error("ccm_build_graph: k = %d exceeds the supported maximum 32", k);
    return CCM_ERR_UNSUPPORTED;
  }
  if (((uintptr_t)edges) % 8 || ((uintptr_t)A) % 8) {
    set_error("ccm_build_graph: misaligned pointer");
    return CCM_ERR_INVALID_ARG;
  }
  CCM_CUDA(cudaSetDevice(c->device));
  const char* fe = getenv("CCM_KNN_FORCE_EXACT");
  return build_graph_device(c, A, n, d, k, phi, edges, w, cap, m_out, phi_out,
                            fe && fe[0] == '1', (cudaStream_t)stream);
}
