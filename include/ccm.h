/*
 * ccm.h - C ABI of libccm: convex clustering (model CCM; q = 2, 1 or inf) along a
 * gamma path on one NVIDIA B300 (sm_103a).
 *
 * Model (Sec. 1, model CCM): given points a_1..a_n in R^d, weights
 * w_ij = w_ji >= 0 and gamma >= 0,
 *     X*(gamma) = argmin_X 1/2 sum_i ||x_i - a_i||^2 + gamma sum_{i<j} w_ij ||x_i - x_j||_q ,
 * q = 2 (default), 1 or inf (ccm_solve_path only), solved for a non-decreasing
 * sequence gamma_1 <= ... <= gamma_T (the clustering path); a_i and a_j share a
 * cluster when x_i* = x_j*.
 *
 * Conventions for every function below:
 *   - Arrays are DEVICE pointers unless marked "host", row-major, owned and
 *     allocated by the caller, and must not alias each other unless stated.
 *   - A and X are n x d float64 with row stride d (no padding).
 *   - An edge list is m rows of (i, j) int32 with 0 <= i < j < n, sorted
 *     lexicographically and without duplicates; the row index is the edge id.
 *   - Work is issued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream). Functions that return sizes or statistics to the host
 *     synchronise that stream before returning.
 *   - Every function returns a ccm_status; nothing throws across the ABI and
 *     no kernel traps. On error, ccm_last_error() describes the failure.
 *   - A ccm_ctx owns all scratch memory (grown on demand, freed by
 *     ccm_destroy). A context is not thread-safe: use one per host thread.
 */
#ifndef CCM_H
#define CCM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ccm_stream_t; /* ABI-compatible with cudaStream_t */
typedef struct ccm_ctx ccm_ctx;

typedef enum {
  CCM_OK = 0,
  CCM_ERR_INVALID_ARG = 1,      /* bad size, pointer, or value; nothing was launched */
  CCM_ERR_UNSUPPORTED = 2,      /* e.g. q not 1, 2 or CCM_Q_INF; d above the compiled maximum */
  CCM_ERR_CUDA = 3,             /* a CUDA runtime call failed */
  CCM_ERR_OOM = 4,              /* scratch allocation failed */
  CCM_ERR_NOT_CONVERGED = 5,    /* an iteration cap was hit; outputs are still written */
  CCM_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up */
  CCM_ERR_BUFFER_TOO_SMALL = 7, /* an output capacity is too small; *m_out says how much */
  CCM_ERR_BOUNDS = 8            /* bounds-checked build only (CCM_DEBUG_BOUNDS): a kernel met
                                   an out-of-range index, skipped the access and recorded it */
} ccm_status;

/* The value of the int32 argument q that selects q = inf (the max norm). */
#define CCM_Q_INF 2147483647

typedef enum { CCM_PREC_FP64 = 0, CCM_PREC_MIXED = 1 } ccm_precision;
typedef enum { CCM_ENGINE_AUTO = 0, CCM_ENGINE_GRID = 1, CCM_ENGINE_BLOCK = 2 } ccm_engine;

/* Solver options; fill with ccm_default_options() and override fields. */
typedef struct {
  double sigma0;          /* initial augmented-Lagrangian penalty (default 1) */
  double sigma_max;       /* cap on the penalty; <= 0 (the default) selects 10 for
                             q = 2 and 1 for q = 1 and q = inf (at least sigma0) */
  int32_t max_outer;      /* multiplier updates per gamma (default 200) */
  int32_t max_newton;     /* semismooth-Newton steps per multiplier update (default 50) */
  int32_t max_cg;         /* CG iterations per Newton step (default 500) */
  int32_t precision;      /* ccm_precision. MIXED (default): CG vectors and the Newton
                             operator in float32, with float64 accumulation of every
                             CG dot product; gradient, line search, multiplier update,
                             KKT and gap in float64. FP64: everything float64. */
  int32_t engine;         /* ccm_engine. GRID: one problem across the whole GPU;
                             BLOCK: one thread block runs the whole path (small n; q = 2,
                             d <= 128, no warm start: X0 / U0 make AUTO pick GRID and
                             BLOCK return CCM_ERR_UNSUPPORTED). */
  int32_t profile;        /* 1: time every Newton-CG operator launch with CUDA events
                             (read back with ccm_last_profile) */
  int32_t relabel;        /* 1 (default): the grid engine solves n >= 16384 with the
                             nodes relabelled by connected component of the graph
                             (better cache reuse of gathered rows; inputs and outputs
                             keep the caller's order); 0: never */
  int32_t autotune;       /* 1 (default): ccm_solve_path_batched measures its group
                             shapes (lanes x quads per row) on a sample of a batch of
                             >= 8 problems and caches the fastest per context, d,
                             precision and mean degree; 0: default shape unless cached */
  int32_t coarse;         /* 1: q = 2 grid-engine Newton steps add a coarse correction to
                             the Jacobi preconditioner, one unknown per component of
                             >= 16 nodes of the strong edges (inside, or outside with
                             tr(P_l)/d >= 1/2; the 224 largest); 0 (default): Jacobi only */
  const double* X0;       /* optional device n x d warm start for the first gamma, or NULL */
  const double* U0;       /* optional device m x d multipliers for the first gamma (must
                             satisfy ||u_l|| <= gamma_1 w_l), or NULL */
} ccm_options;

/* Per-gamma solve statistics (host). */
typedef struct {
  int32_t status;         /* CCM_OK or CCM_ERR_NOT_CONVERGED */
  int32_t outer, newton, cg, line_search;
  int32_t n_clusters;     /* number of distinct labels at this gamma */
  double kkt;             /* max(eta_d, eta_p) */
  double eta_d;           /* ||X - A + B^T U||_F / (1 + ||A||_F) */
  double eta_p;           /* ||BX - prox_p(BX + U)||_F / (1 + ||A||_F), p = sum_l gamma w_l ||.|| */
  double gap;             /* |f_p - f_d| / (1 + |f_p| + |f_d|)  (Sec. 4) */
  double f_p, f_d;        /* primal and dual objective values */
  double sigma;           /* penalty at exit */
} ccm_stats;

/* Timing of the Newton-CG operator launches of the last ccm_solve_path call
 * made with options.profile = 1 (CUDA events on the launch stream). */
typedef struct {
  int64_t matvec_launches;
  double matvec_ms_total;
  double matvec_bytes_total; /* algorithmic bytes moved by those launches */
  int64_t kernel_launches;   /* all kernels the last ccm_solve_path call launched */
  int32_t block_lanes;       /* block engine (last block-engine call): lanes per row group */
  int32_t block_quads;       /* ... and quads per lane (the autotuned or cached shape) */
  int32_t coarse_steps;      /* Newton steps that used the coarse correction */
  int32_t coarse_max_aggregates; /* largest number of coarse unknowns of those steps */
} ccm_profile;

/* Total number of kernels launched through this context since ccm_create. */
int64_t ccm_launch_count(ccm_ctx* ctx);

void ccm_default_options(ccm_options* opt);

/* Create a context on CUDA device `device`. */
int ccm_create(ccm_ctx** ctx, int device);
/* Free a context and all its scratch memory (NULL is ignored). */
void ccm_destroy(ccm_ctx* ctx);
/* Thread-local description of the last failure (never NULL). */
const char* ccm_last_error(void);
/* Largest d that ccm_solve_path / ccm_path_vjp accept. */
int32_t ccm_max_dim(void);

/*
 * ccm_build_graph - symmetrized kNN graph with Gaussian weights (the weights
 * w_ij of model CCM, Sec. 1; computed by the Data Processor, Sec. 2.2 item 1).
 *
 *   D_ij  = sum_k (a_ik - a_jk)^2 in float64, one rounding per operation,
 *           features in ascending order, no fused multiply-add;
 *   N(i)  = the k points j != i with the smallest (D_ij, j);
 *   edges = { (min(i,j), max(i,j)) : j in N(i) }, sorted, unique;
 *   w_l   = exp(-phi * D_l), phi = `phi` if phi > 0, else 1 / D_(floor((m-1)/2)),
 *           the lower median of the edge distances.
 * A: device n x d float64. 1 <= k < n, n < 2^31. edges: device capacity
 * `cap` rows of 2 int32; w: device capacity `cap` float64 (cap >= n*k always
 * suffices). On success *m_out (host) is the edge count and *phi_out (host) the
 * phi used. CCM_ERR_BUFFER_TOO_SMALL if m > cap (then *m_out = m).
 * Approximate float32 distances select candidates; every candidate within a
 * rigorous error bound of the k-th distance is re-ranked in float64, and rows
 * where the bound cannot separate the k-th neighbour are searched exhaustively
 * in float64, so the edge set equals the definition above exactly.
 */
int ccm_build_graph(ccm_ctx* ctx, const double* A, int64_t n, int32_t d, int32_t k,
                    double phi, int32_t* edges, double* w, int64_t cap, int64_t* m_out,
                    double* phi_out, ccm_stream_t stream);

/*
 * ccm_solve_path - X*(gamma_t) and cluster labels for t = 0..T-1 by a
 * semismooth-Newton augmented Lagrangian method (SSNAL, Sec. 1), warm-started
 * along the path (Sec. 1: 0 <= gamma_1 < ... < gamma_T).
 *
 * A: n x d; edges: m x 2 (see conventions); w: m float64 >= 0;
 * gammas: HOST array of T non-decreasing values >= 0; q = 2 (the Euclidean norm
 * of x_i - x_j), q = 1 (its l1 norm: the dual ball becomes ||u_l||_inf <= r_l,
 * the Newton Jacobian a 0/1 diagonal per edge) or q = CCM_Q_INF (its max norm:
 * the dual ball becomes ||u_l||_1 <= r_l, projected onto by an active-set
 * threshold search per edge, the Jacobian diag(mask) - s s^T on the support of
 * the projection); q = 1 and q = inf run on the grid engine only; other q give
 * CCM_ERR_UNSUPPORTED; tol > 0: stop each gamma when max(eta_d, eta_p) <= tol
 * and the relative duality gap of Sec. 4 is <= tol (definitions in ccm_stats).
 * Outputs: X: T x n x d float64; labels: T x n int32 or NULL (label = rank of the
 * cluster's smallest node index; an edge is fused when the float64 squared
 * distance of its endpoints, summed in feature order without FMA, is <= 1e-12);
 * U: T x m x d float64 or NULL (final multipliers); stats: HOST array of T or NULL.
 * X and labels may be device or host memory (pinned host memory recommended):
 * for host X the path runs on a device staging buffer held by the context, and
 * each gamma's X is copied to the host on the context's copy stream while the
 * next gamma solves; host labels are copied after the path. The call returns
 * after every copy has landed. U must be device memory (CCM_ERR_INVALID_ARG).
 * For q = 1, eta_p uses prox of r_l ||.||_1 (soft threshold) and f_p r_l ||.||_1;
 * for q = inf, prox of r_l ||.||_inf (identity minus the l1-ball projection) and
 * r_l ||.||_inf.
 * Returns CCM_ERR_NOT_CONVERGED if any gamma hit an iteration cap (all outputs
 * are still written; stats[t].status says which).
 */
int ccm_solve_path(ccm_ctx* ctx, const double* A, int64_t n, int32_t d,
                   const int32_t* edges, const double* w, int64_t m,
                   const double* gammas, int32_t T, int32_t q, double tol,
                   const ccm_options* opt, double* X, int32_t* labels, double* U,
                   ccm_stats* stats, ccm_stream_t stream);

/*
 * ccm_solve_path_admm - the same path, outputs and stopping rule as
 * ccm_solve_path, solved by ADMM (the paper's second solver, Sec. 1, Table 3)
 * instead of SSNAL: split z_l = (BX)_l with multiplier U and the fixed penalty
 * options.sigma0;
 *   X <- (I + sigma B^T B)^{-1} (A + B^T (sigma Z - U))   (CG correction, relative 1e-2),
 *   Z <- prox_{p/sigma}(B X + U / sigma),   U <- U + sigma (B X - Z);
 * KKT residuals and gap (definitions in ccm_stats) every 10 iterations; at most
 * options.max_outer * options.max_newton iterations per gamma (stats[t].outer
 * counts them, stats[t].cg the CG iterations of the X-steps). Warm-started along
 * the path from (X, Z, U); options.precision selects the X-step CG precision.
 * Grid engine only (options.engine is ignored).
 */
int ccm_solve_path_admm(ccm_ctx* ctx, const double* A, int64_t n, int32_t d,
                        const int32_t* edges, const double* w, int64_t m,
                        const double* gammas, int32_t T, int32_t q, double tol,
                        const ccm_options* opt, double* X, int32_t* labels, double* U,
                        ccm_stats* stats, ccm_stream_t stream);

/*
 * ccm_solve_path_ama - the same path, outputs and stopping rule as
 * ccm_solve_path, solved by fast AMA (the paper's third solver, Sec. 1, Table 3):
 * projected gradient ascent on the dual with Nesterov momentum and gradient
 * restart, X(U) = A - B^T U,
 *   U <- Pi(Uh + nu B X(Uh)),  Uh = U + momentum,  nu = 1 / max_l (deg_i + deg_j);
 * KKT residuals and gap every 10 iterations (eta_d is 0 by construction); at most
 * 10 * options.max_outer * options.max_newton iterations per gamma (stats[t].outer
 * counts them; stats[t].sigma reports nu). Warm-started along the path from U.
 * Grid engine only; options.precision and options.engine are ignored (float64).
 */
int ccm_solve_path_ama(ccm_ctx* ctx, const double* A, int64_t n, int32_t d,
                       const int32_t* edges, const double* w, int64_t m,
                       const double* gammas, int32_t T, int32_t q, double tol,
                       const ccm_options* opt, double* X, int32_t* labels, double* U,
                       ccm_stats* stats, ccm_stream_t stream);

/* Profile of the last ccm_solve_path run with options.profile = 1 (host out). */
int ccm_last_profile(ccm_ctx* ctx, ccm_profile* out);

/* How the last ccm_build_graph on this context found its candidates. */
typedef struct {
  int32_t candidates;       /* 1: tensor-core TF32 Gram form (d <= 128), 0: float32
                               direct-difference tiles on the CUDA cores */
  int32_t per_row;          /* candidates kept per row before the float64 re-rank */
  int64_t rows_exhaustive;  /* rows the error bound could not certify, searched
                               exhaustively in float64 */
} ccm_graph_info;
int ccm_last_graph_info(ccm_ctx* ctx, ccm_graph_info* out);

/*
 * ccm_labels - cluster labels of one solution X (n x d) on an edge list, with
 * the fusion rule of ccm_solve_path. labels: device n int32. *n_clusters (host)
 * receives the number of clusters (may be NULL).
 */
int ccm_labels(ccm_ctx* ctx, const double* X, int64_t n, int32_t d, const int32_t* edges,
               int64_t m, int32_t* labels, int32_t* n_clusters, ccm_stream_t stream);

/*
 * ccm_labels_noalloc - ccm_labels for callers that cannot allocate device
 * memory. The paper has no counterpart; this is a deployment variant.
 *
 * Some callers must not call cudaMalloc or cudaFree: code running under a
 * memory pool or allocator that owns all device memory, hosts that reserve the
 * device memory up front, or callers that cannot afford the implicit
 * synchronisation an allocation may bring. This entry point needs no context and
 * allocates nothing: its scratch is a fixed static device array of 262,144
 * nodes (about 2 MB, kept by every GPU that loads libccm until the process exits).
 * The caller still passes X (n x d), the edges (m x 2) and labels (n int32), all
 * device pointers; *n_clusters (host, may be NULL) receives the cluster count.
 * n above 262,144 returns CCM_ERR_INVALID_ARG with a message naming the limit.
 * Every call looks up the scratch address of the current device with
 * cudaGetSymbolAddress (so the address stays valid across cudaDeviceReset);
 * the first call on a device also loads the module, so make that first call
 * before any stream capture. All calls share the one scratch array, so calls
 * that can overlap on the GPU (different streams or host threads) race:
 * serialise them. The call synchronises `stream` before returning, so `stream`
 * must not be under capture, and must not be the legacy NULL stream while
 * another stream of the device captures in global mode.
 */
int ccm_labels_noalloc(const double* X, int64_t n, int32_t d, const int32_t* edges, int64_t m,
                       int32_t* labels, int32_t* n_clusters, ccm_stream_t stream);

/*
 * ccm_path_vjp - vector-Jacobian product of the path (not in the paper):
 * given G_t = dL/dX*(gamma_t) (T x n x d), returns
 *     dLdA = sum_t dL_t/dA  (n x d)   and   dLdw = sum_t dL_t/dw  (m),
 * by implicit differentiation of the optimality conditions away from fusion
 * events: clusters are the components of fused edges (rule of ccm_labels);
 * with s_l = (x_i-x_j)/||x_i-x_j|| and c_l = gamma w_l/||x_i-x_j|| on edges
 * joining two clusters, lambda solves (M + sum_l c_l B_l^T (I - s_l s_l^T) B_l) lambda = Q^T G
 * in the cluster space (M = cluster sizes) by iterative refinement: float64
 * residuals, float32 conjugate-gradient corrections with the Newton-CG operator,
 * until ||residual|| <= 1e-11 ||Q^T G|| (or a correction stops halving it);
 * dL/da_i = lambda_c(i), dL/dw_l = -gamma s_l^T (lambda_c(i) - lambda_c(j))
 * (0 for fused edges). X: T x n x d from ccm_solve_path. U is accepted for
 * interface symmetry and may be NULL (the gradient depends on X only).
 * gammas: HOST. Both outputs are overwritten (not accumulated into).
 */
int ccm_path_vjp(ccm_ctx* ctx, const double* A, int64_t n, int32_t d,
                 const int32_t* edges, const double* w, int64_t m,
                 const double* gammas, int32_t T, const double* X, const double* U,
                 const double* dLdX, double* dLdA, double* dLdw, ccm_stream_t stream);

/* One independent problem of a batch (device pointers, host struct). */
typedef struct {
  const double* A;        /* n x d */
  const int32_t* edges;   /* m x 2 */
  const double* w;        /* m */
  int64_t n, m;
  double* X;              /* T x n x d out */
  int32_t* labels;        /* T x n out, or NULL */
} ccm_problem;

/*
 * ccm_solve_path_batched - P independent path problems that share d, the
 * gamma grid (HOST, T values) and tol, solved in one persistent launch: each
 * thread block takes the next problem from a device work queue (largest
 * first) and runs its whole path. stats: HOST P x T or NULL. Same fusion rule
 * and stopping rule as ccm_solve_path.
 */
int ccm_solve_path_batched(ccm_ctx* ctx, int32_t P, const ccm_problem* probs, int32_t d,
                           const double* gammas, int32_t T, double tol,
                           const ccm_options* opt, ccm_stats* stats, ccm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CCM_H */
