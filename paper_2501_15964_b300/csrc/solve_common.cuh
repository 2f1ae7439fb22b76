// Arguments of one path solve, shared by the solver engines.
#pragma once

#include "ccm_internal.cuh"

namespace ccm {

struct SolveArgs {
  const double* A = nullptr;
  int64_t n = 0;
  int d = 0;
  const int32_t* edges = nullptr;
  const double* w = nullptr;
  int64_t m = 0;
  const double* gammas = nullptr;  // host
  int T = 0;
  double tol = 1e-6;
  ccm_options opt{};
  double* Xout = nullptr;
  double* Uout = nullptr;
  ccm_stats* stats = nullptr;      // host
  const double* X0 = nullptr;
  const double* U0 = nullptr;
  int q = 2;  // norm of the differences: 2 (group lasso), 1 (elementwise) or CCM_Q_INF (max)
  // node relabelling (grid engine; both NULL = identity): A, X0 rows are read
  // through perm (new -> old) and X rows written back through it; U0 / U rows
  // through eperm (new -> old edge, ~id = endpoints swapped: the row's sign flips)
  const int* perm = nullptr;
  const int* eperm = nullptr;
  // host destination of X (caller's host memory; Xout is then a device staging
  // buffer): each gamma's rows are copied on copy_stream while the next solves
  double* Xhost = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_event = nullptr;

  // Algorithmic bytes of one Newton-CG operator launch (each datum once):
  // R read and W written (n x ld each), Minv (n), the yhat rows of the m_out
  // outside edges, the packed incidence coefficients (2m x 2 elements), the
  // CSR incidences (2m int2) and offsets (n+1 int64).
  double matvec_bytes(double m_out, size_t tcb) const {
    const double ld = (double)((d + 3) / 4 * 4);
    return 2.0 * (double)n * ld * (double)tcb + (double)n * tcb + m_out * ld * tcb +
           2.0 * (double)m * (8.0 + 2.0 * tcb) + 8.0 * (double)(n + 1);
  }
};

int solve_grid(Ctx* c, const SolveArgs& a, cudaStream_t s);
int solve_single_block(Ctx* c, const SolveArgs& a, int32_t* labels, cudaStream_t s);
int check_edges(Ctx* c, const int2* edges, int64_t m, int64_t n, const double* w, cudaStream_t s);
int build_csr(Ctx* c, const int2* edges, int64_t m, int64_t n, int64_t** off_out, int2** inc_out,
              cudaStream_t s);

}  // namespace ccm
