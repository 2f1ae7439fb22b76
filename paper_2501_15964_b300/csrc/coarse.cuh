// Two-level (coarse-corrected) preconditioner of the Newton-CG; coarse.cu.
#pragma once

#include "ssnal_kernels.cuh"

namespace ccm {

constexpr int kCoarseMinSize = 16;  // nodes in an aggregate (component of inside edges)
constexpr int kCoarseMaxAgg = 224;  // aggregates (the inverse is formed in shared memory)
constexpr double kCoarseStrong = 0.5;  // t_l = tr(P_l) / d of an edge that joins aggregates

// Aggregates and the inverted coarse matrix of one Newton step (device
// pointers into the context's workspace); K = 0: no coarse correction.
template <typename Tc>
struct CoarsePlan {
  int K = 0;
  const int* agg = nullptr;      // n: aggregate of each node, -1 for none
  const int* mem_off = nullptr;  // K + 1
  const int* mem = nullptr;      // members of each aggregate, increasing node index
  const float* Ainv = nullptr;   // K x K
  Tc* y = nullptr;               // K x ld: P^T R
  Tc* z = nullptr;               // K x ld: A_c^-1 P^T R
};

// Aggregates from the inside edges of the current edge kinds, and A_c^-1
// (synchronises the stream: the aggregate selection runs on the host).
template <typename Tc>
int coarse_build(Ctx* c, const int2* edges, const uint8_t* kind, const Tc* alpha, int64_t n,
                 int64_t m, double sigma, int d, int ld, CoarsePlan<Tc>& cp, cudaStream_t s);

// U = M^-1 R = Minv R + P A_c^-1 P^T R; sets the CG scalars rz = <R, U> and beta.
template <typename Tc>
int coarse_precondition(Ctx* c, const CoarsePlan<Tc>& cp, const Tc* R, const Tc* Minv, Tc* U,
                        int64_t n, int ld, double* part, Ctl* ctl, cudaStream_t s);

}  // namespace ccm
