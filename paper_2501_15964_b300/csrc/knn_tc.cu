// kNN candidate distances on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The Data Processor's weights (Sec. 2.2 item 1; model CCM, Sec. 1) need the k
// nearest neighbours of every point. Candidates come from approximate squared
// distances in the Gram form
//     D~_ij = n_i + n_j - 2 <b_i, b_j>,   b = float32(A - column mean),
// with the inner products on the tensor cores in TF32 and a three-product
// split for float32-level accuracy: b = h + l with h = tf32(b), l = tf32(b - h)
// (both rounded to nearest), and <b_i, b_j> ~ <h_i, h_j> + <h_i, l_j> + <l_i, h_j>
// accumulated in float32 in tensor memory. Every candidate is then re-ranked in
// float64 (k_rerank in graph.cu) with a rigorous bound on |D~ - D| for this
// form, so the edge set is the exact one of the definition.
//
// One CTA owns 128 query rows and sweeps all columns in tiles of 128:
//   warp 0     TMA producer: the CTA's A rows (h and l, every K-block) once,
//              then the B tile of each (column tile, K-block) into a ring of
//              shared-memory stages (128-byte swizzled, K-major);
//   warp 1     allocates all 512 TMEM columns (four 128 x 128 float32 accumulators)
//              and one elected lane issues tcgen05.mma kind::tf32, M = N = 128,
//              K = 8 per instruction, three per K-step;
//   warps 2-9  epilogue: tcgen05.ld of the finished accumulator, two threads per
//              query row (TMEM lane; each takes half of the tile's columns), D~
//              per column, and a running list of the K' smallest (D~, j) per
//              thread in registers, merged per row at the end.
// Stages and accumulators are handed over with mbarriers (TMA complete_tx,
// tcgen05.commit). Every wait is bounded: on timeout the kernel records an
// error, drains what it has in flight, frees its TMEM and returns, and the host
// falls back to the SIMT kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "ccm_internal.cuh"

namespace ccm {
namespace {

constexpr int kBM = 128;            // query rows per CTA (MMA M)
constexpr int kBN = 128;            // columns per tile (MMA N)
constexpr int kKB = 32;             // floats per K-block: one 128-byte swizzled row
constexpr int kTileFloats = 128 * kKB;  // 16 KB: one operand block of 128 rows
constexpr int kThreads = 320;       // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kAccBufs = 4;          // accumulators in flight (4 x 128 columns = all of TMEM)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kWaitCap = 1u << 24;  // try_wait polls before a wait gives up

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t sptr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(sptr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; !mbar_try(b, parity); ++it)
    if (it > kWaitCap || *abort_flag) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(sptr(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(sptr(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          sptr(bar))
      : "memory");
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 32 consecutive float32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld_32cols(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor of a K-major operand block in the 128-byte
// swizzled layout written by TMA (rows of 128 bytes, eight-row atoms of 1024
// bytes, atoms 1024 bytes apart): start address >> 4 (bits 0-13), leading-
// dimension offset (bits 16-29, unused for this layout: 1), stride-dimension
// offset 1024 >> 4 (bits 32-45), descriptor version 1 (bits 46-47), base offset
// 0 (atoms are 1024-byte aligned), swizzle mode 2 = 128 bytes (bits 61-63).
// A K-step of 8 TF32 elements inside the 128-byte row advances the start
// address by 32 bytes.
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  const uint64_t a = (uint64_t)(sptr(p) >> 4) & 0x3FFFull;
  return a | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::tf32: float32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Bh / Bl (n_pad x Kp): h = tf32(b), l = tf32(b - h) for b = At (zero past d and n).
__global__ void k_tf32_split(const float* __restrict__ At, int ldf, int64_t n, int64_t n_pad,
                             int d, int Kp, float* __restrict__ Bh, float* __restrict__ Bl) {
  const int64_t total = n_pad * Kp;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / Kp;
    const int k = (int)(q - i * Kp);
    const float v = (i < n && k < d) ? At[i * ldf + k] : 0.0f;
    const float h = tf32_rn(v);
    Bh[q] = h;
    Bl[q] = tf32_rn(v - h);
  }
}

// nbf_i = float32(||h_i + l_i||^2) (sums in float64); padding rows get +inf so
// their distances never enter a list.
__global__ void k_tf32_norms(const float* __restrict__ Bh, const float* __restrict__ Bl,
                             int64_t n, int64_t n_pad, int Kp, float* __restrict__ nbf) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < n_pad; i += nw) {
    double s = 0.0;
    for (int k = lane; k < Kp; k += 32) {
      const double v = (double)Bh[i * Kp + k] + (double)Bl[i * Kp + k];
      s += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nbf[i] = i < n ? (float)s : INFINITY;
  }
}

template <int KP>
__device__ __forceinline__ void list_insert(float (&ld)[KP], int (&lj)[KP], float& thr,
                                            float dt, int j) {
  // replace the current maximum, then find the new maximum (static indices only)
  bool done = false;
#pragma unroll
  for (int p = 0; p < KP; ++p) {
    const bool hit = !done && ld[p] == thr;
    ld[p] = hit ? dt : ld[p];
    lj[p] = hit ? j : lj[p];
    done = done || hit;
  }
  thr = ld[0];
#pragma unroll
  for (int p = 1; p < KP; ++p) thr = fmaxf(thr, ld[p]);
}

template <int KP>
__global__ void __launch_bounds__(kThreads, 1)
k_knn_tc(const __grid_constant__ CUtensorMap tm_h, const __grid_constant__ CUtensorMap tm_l,
         const float* __restrict__ nbf, int64_t n, int nkb, int nstages, int ntiles,
         int* __restrict__ cand, float* __restrict__ cand_thr, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* sA = reinterpret_cast<float*>(base);               // [nkb][2][128 x 32]
  float* sB = sA + (size_t)nkb * 2 * kTileFloats;          // [nstages][2][128 x 32]
  float* snorm = sB + (size_t)nstages * 2 * kTileFloats;    // [2][128] column norms
  float* sdist = snorm + 2 * kBN;                             // [32][256] one chunk per thread
  uint64_t* full = reinterpret_cast<uint64_t*>(sdist + 256 * 32 + 4);
  uint64_t* empty = full + nstages;
  uint64_t* tfull = empty + nstages;        // [kAccBufs]
  uint64_t* tempty = tfull + kAccBufs;      // [kAccBufs]
  uint64_t* afull = tempty + kAccBufs;      // [1]
  uint64_t* drain = afull + 1;              // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);  // [2]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kBM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, 8);
    }
    mbar_init(afull, 1);
    mbar_init(drain, 1);
    abort_flag[0] = 0;
    abort_flag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sptr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(err, 1);
  };

  if (warp == 0) {
    // ---------------- producer
    if (lane == 0) {
      const uint32_t abytes = (uint32_t)nkb * 2 * kTileFloats * 4;
      mbar_expect_tx(afull, abytes);
      for (int kb = 0; kb < nkb; ++kb) {
        tma_load_2d(sA + (size_t)(2 * kb) * kTileFloats, &tm_h, kb * kKB, (int)row0, afull);
        tma_load_2d(sA + (size_t)(2 * kb + 1) * kTileFloats, &tm_l, kb * kKB, (int)row0, afull);
      }
      const int64_t total = (int64_t)ntiles * nkb;
      int64_t it = 0;
      for (; it < total; ++it) {
        const int s = (int)(it % nstages);
        const uint32_t round = (uint32_t)(it / nstages);
        if (round > 0 && !mbar_wait(empty + s, (round - 1) & 1u, abort_flag)) {
          fail();
          break;
        }
        const int t = (int)(it / nkb), kb = (int)(it % nkb);
        mbar_expect_tx(full + s, 2u * kTileFloats * 4);
        tma_load_2d(sB + (size_t)(2 * s) * kTileFloats, &tm_h, kb * kKB, t * kBN, full + s);
        tma_load_2d(sB + (size_t)(2 * s + 1) * kTileFloats, &tm_l, kb * kKB, t * kBN, full + s);
      }
      // every issued copy lands before the CTA's shared memory is released (the
      // copies complete on their own; these waits are bounded as well)
      for (uint32_t k2 = 0; !mbar_try(afull, 0) && k2 < kWaitCap; ++k2) {
      }
      for (int64_t q = std::max<int64_t>(0, it - nstages); q < it; ++q) {
        const int s = (int)(q % nstages);
        const uint32_t par = (uint32_t)(q / nstages) & 1u;
        for (uint32_t k2 = 0; !mbar_try(full + s, par) && k2 < kWaitCap; ++k2) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      bool ok = mbar_wait(afull, 0, abort_flag);
      if (!ok) fail();
      for (int t = 0; ok && t < ntiles; ++t) {
        const int b = t % kAccBufs;
        if (t >= kAccBufs &&
            !mbar_wait(tempty + b, (uint32_t)(t / kAccBufs - 1) & 1u, abort_flag)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(b * kBN);
        for (int kb = 0; kb < nkb; ++kb) {
          const int64_t it = (int64_t)t * nkb + kb;
          const int s = (int)(it % nstages);
          if (!mbar_wait(full + s, (uint32_t)(it / nstages) & 1u, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const float* ah = sA + (size_t)(2 * kb) * kTileFloats;
          const float* al = ah + kTileFloats;
          const float* bh = sB + (size_t)(2 * s) * kTileFloats;
          const float* bl = bh + kTileFloats;
#pragma unroll
          for (int k8 = 0; k8 < kKB / 8; ++k8) {
            const uint64_t dah = sw128_desc(ah + 8 * k8), dal = sw128_desc(al + 8 * k8);
            const uint64_t dbh = sw128_desc(bh + 8 * k8), dbl = sw128_desc(bl + 8 * k8);
            tc_mma_tf32(dt, dah, dbh, kIdesc, (kb | k8) != 0 ? 1u : 0u);
            tc_mma_tf32(dt, dah, dbl, kIdesc, 1u);
            tc_mma_tf32(dt, dal, dbh, kIdesc, 1u);
          }
          tc_commit(empty + s);  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        tc_commit(tfull + b);
      }
      // every issued MMA has completed before TMEM is freed
      tc_commit(drain);
      for (uint32_t k2 = 0; !mbar_try(drain, 0) && k2 < kWaitCap; ++k2) {
      }
    }
  } else {
    // ---------------- epilogue: eight warps, two per TMEM lane quarter
    // Warp w reads TMEM lanes 32 (w % 4) .. + 31 (its query rows); the two warps
    // of a quarter take the two halves of each tile's columns, each keeping its
    // own list for its row, and the lists are merged at the end. The column norms
    // of tile t + 1 are loaded while tile t is processed and published to the
    // other half of a double buffer; a named barrier of the epilogue warps orders
    // the buffers.
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int et = threadIdx.x - 64;  // 0..255
    const int r = quarter * 32 + lane;
    const int gi = (int)(row0 + r);
    const float ni = (int64_t)gi < n ? nbf[gi] : INFINITY;
    float ld[KP];
    int lj[KP];
#pragma unroll
    for (int p = 0; p < KP; ++p) {
      ld[p] = INFINITY;
      lj[p] = -1;
    }
    float thr = INFINITY;
    volatile int* stop = abort_flag + 1;  // the epilogue's common decision to stop
    if (et < kBN) snorm[et] = nbf[et];    // tile 0
    asm volatile("bar.sync 1, 256;" ::: "memory");
    float* sdc = sdist + et;  // this thread's staging column ([32][256] layout)
    for (int t = 0; t < ntiles; ++t) {
      const int b = t % kAccBufs;
      const float pf = (t + 1 < ntiles && et < kBN) ? nbf[(int64_t)(t + 1) * kBN + et] : 0.0f;
      const bool ok = mbar_wait(tfull + b, (uint32_t)(t / kAccBufs) & 1u, abort_flag);
      if (!ok) {
        fail();
      } else {
        tc_fence_after();
        const float* sn = snorm + (t & 1) * kBN;
        const int col0 = t * kBN;
#pragma unroll 1
        for (int c = 2 * half; c < 2 * half + 2; ++c) {
          float v[32];
          tc_ld_32cols(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kBN + c * 32),
                       v);
          // D~ for the 32 columns in registers and their minimum; only when that
          // minimum is below the current threshold (rare once the list holds
          // near neighbours) are the distances staged in shared memory (column
          // j of this thread at sdc[256 j]: fixed offsets, no bank conflicts)
          // and the insertions run from one copy of the insertion code, which
          // keeps the loop small enough for the instruction cache and costs the
          // warp only as many passes as its busiest lane has insertions
          const float4* sn4 = reinterpret_cast<const float4*>(sn + c * 32);
          float mn = INFINITY;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 s4 = sn4[q];
            const float sv4[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int jj = 4 * q + e;
              v[jj] = fmaf(-2.0f, v[jj], ni + sv4[e]);
              mn = fminf(mn, v[jj]);
            }
          }
          if (mn < thr) {
            uint32_t msk = 0u;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              sdc[jj * 256] = v[jj];
              msk |= (v[jj] < thr ? 1u : 0u) << jj;
            }
            const int cb = col0 + c * 32;
            if (gi >= cb && gi < cb + 32) msk &= ~(1u << (gi - cb));
            while (msk) {
              const int jj = __ffs(msk) - 1;
              msk &= msk - 1u;
              const float dt = sdc[jj * 256];
              if (dt < thr) list_insert<KP>(ld, lj, thr, dt, cb + jj);
            }
          }
        }
        tc_fence_before();
      }
      __syncwarp();
      if (lane == 0 && ok) mbar_arrive(tempty + b);
      if (et < kBN) snorm[((t + 1) & 1) * kBN + et] = pf;
      if (et == 0) *stop = *abort_flag;  // read once, before the barrier, for all
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (*stop) break;  // the same value in every epilogue thread
    }
    // merge: the second half's list of each row joins the first half's. Every
    // tile has been loaded and consumed, so the stage ring is free for this.
    float* mdist = sB;
    int* mcol = reinterpret_cast<int*>(sB + kBM * KP);
    if (half == 1) {
#pragma unroll
      for (int p = 0; p < KP; ++p) {
        mdist[r * KP + p] = ld[p];
        mcol[r * KP + p] = lj[p];
      }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (half == 0) {
      for (int p = 0; p < KP; ++p) {
        const float dt = mdist[r * KP + p];
        if (dt < thr) list_insert<KP>(ld, lj, thr, dt, mcol[r * KP + p]);
      }
      if ((int64_t)gi < n) {
#pragma unroll
        for (int p = 0; p < KP; ++p)
          cand[(int64_t)gi * KP + p] = ld[p] < INFINITY ? lj[p] : -1;
        cand_thr[gi] = thr;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------- host
using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

int encoder(EncodeFn* out) {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    CCM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                              cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return CCM_ERR_CUDA;
    }
    fn = (EncodeFn)p;
  }
  *out = fn;
  return CCM_OK;
}

int make_map(const float* base, int64_t rows, int Kp, CUtensorMap* tm) {
  EncodeFn enc;
  CCM_TRY(encoder(&enc));
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kKB, 128u};
  const cuuint32_t estr[2] = {1u, 1u};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return CCM_ERR_CUDA;
  }
  return CCM_OK;
}

}  // namespace

int knn_tc_supported(int d, int Kp) { return d >= 1 && d <= 128 && Kp <= 64; }

int knn_candidates_tc(Ctx* c, const float* At, int ldf, int64_t n, int d, int Kp, int* cand,
                      float* cand_thr, int* used_kp, cudaStream_t s) {
  const int KPT = Kp <= 32 ? 32 : 64;  // list length of the kernel (>= Kp)
  const int Kpad = (int)round_up(d, kKB);
  const int nkb = Kpad / kKB;
  const int64_t n_pad = round_up(n, 128);
  const int ntiles = (int)(n_pad / kBN);
  const size_t abytes = (size_t)nkb * 2 * kTileFloats * 4;
  const size_t stage = (size_t)2 * kTileFloats * 4;
  // shared memory: alignment slack, A (resident), the B stage ring, column norms,
  // the epilogue's staging buffer and the barriers; as many stages (2..4) as fit
  int optin = 0;
  CCM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  const size_t fixed = 1024 + (2 * kBN + 256 * 32 + 4) * 4 + 256;
  if ((size_t)optin < fixed + abytes + 2 * stage) {
    set_error("tensor-core kNN: not enough shared memory for d = %d", d);
    return CCM_ERR_UNSUPPORTED;
  }
  const int nstages = (int)std::min<size_t>(4, ((size_t)optin - fixed - abytes) / stage);
  const size_t smem = fixed + abytes + (size_t)nstages * stage;
  void* p;
  const size_t mat = (size_t)n_pad * Kpad * 4;
  CCM_TRY(ws_get(c, S_KNN, 2 * mat + (size_t)n_pad * 4 + 256, &p));
  float* Bh = (float*)p;
  float* Bl = (float*)((char*)p + mat);
  float* nbf = (float*)((char*)p + 2 * mat);
  int* err = (int*)((char*)nbf + round_up(n_pad * 4, 64));
  const int blocks = (int)std::min<int64_t>((n_pad * Kpad + 255) / 256, (int64_t)c->num_sms * 8);
  k_tf32_split<<<blocks, 256, 0, s>>>(At, ldf, n, n_pad, d, Kpad, Bh, Bl);
  CCM_COUNT(c);
  k_tf32_norms<<<(int)std::min<int64_t>((n_pad * 32 + 255) / 256, (int64_t)c->num_sms * 8), 256,
                 0, s>>>(Bh, Bl, n, n_pad, Kpad, nbf);
  CCM_COUNT(c);
  CCM_CUDA(cudaMemsetAsync(err, 0, 4, s));
  CUtensorMap th, tl;
  CCM_TRY(make_map(Bh, n_pad, Kpad, &th));
  CCM_TRY(make_map(Bl, n_pad, Kpad, &tl));
  auto launch = [&](auto kern) -> int {
    CCM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)(n_pad / kBM), kThreads, smem, s>>>(th, tl, nbf, n, nkb, nstages, ntiles,
                                                         cand, cand_thr, err);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    return CCM_OK;
  };
  if (KPT == 32)
    CCM_TRY(launch(k_knn_tc<32>));
  else
    CCM_TRY(launch(k_knn_tc<64>));
  int herr = 0;
  CCM_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
  CCM_CUDA(cudaStreamSynchronize(s));
  *used_kp = KPT;
  if (herr) {
    set_error("tensor-core kNN: a bounded wait gave up");
    return CCM_ERR_TIMEOUT;
  }
  return CCM_OK;
}

}  // namespace ccm
