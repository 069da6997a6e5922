/*
 * proxsdp_gpu.h — C ABI of the GB300 (sm_103a) low-rank primal-dual SDP solver.
 *
 * The library implements the low-rank primal-dual hybrid gradient iteration
 * "LR-PD-SDP" (Alg. 2 of Souto, Garcia & Veiga, "Exploiting Low-Rank
 * Structure in Semidefinite Programming by Approximate Operator Splitting")
 * and its full-projection special case "PD-SDP" (Alg. 1) for the general SDP
 *
 *     minimize tr(C X)  s.t.  tr(A_i X) = b_i (i < m_eq),
 *                             tr(G_j X) <= h_j (the remaining rows),  X psd
 *
 * of Sec. 1.3 (Eq. sdp_general).  Every step of the iteration runs in the
 * library's own CUDA kernels: the truncated psd projection of Sec. 3.1
 * (Eq. trunc_eig) by a restarted block Lanczos solver, the rank update of
 * Sec. 3.2, the rebuild X = V diag(max(lambda,0)) V^T fused with the primal
 * update of Alg. 1 / Alg. 2, the sparse constraint operator M(X) and its
 * adjoint M*(y), the dual step with the equality / inequality split of
 * Sec. 2.3.1 (Eq. resolvent_1), and the residual / gap reductions of Sec. 2.2
 * (Eq. comb_residual).  There is no CPU fallback: without a usable sm_103a
 * device every entry point returns PROXSDP_ERR_CUDA.
 *
 * Conventions
 * -----------
 * - Symmetric matrices are passed as packed upper-triangle ("svec") entries
 *   without sqrt(2) scaling: entry (i, j), 0 <= i <= j < n, has index
 *   j*(j+1)/2 + i, and a value a there means A[i][j] = A[j][i] = a, so
 *   tr(A X) = sum_i A_ii X_ii + 2 sum_{i<j} A_ij X_ij.
 * - The constraint operator M = [A; G] (Sec. 2) is a CSR matrix whose row i
 *   lists the svec entries of A_i (rows 0..m_eq-1) or G_{i-m_eq}.  A row whose
 *   only entry has column index -1 is the structured dense matrix a * 11^T
 *   (e.g. the equipartition constraint tr(11^T X) = 0 of Sec. 5.1).
 * - The dual vector returned is the paper's y of the dual problem of Sec. 1.3
 *   (maximise [b; h]^T y s.t. M*(y) <= C, y_ineq <= 0).  Internally the
 *   iteration carries its negation (non-negative on inequality rows).
 * - Every function returns an int status: 0 = OK, < 0 = error (codes below).
 *   Non-convergence is not an error; it is reported in proxsdp_gpu_info.status.
 *
 * Ownership and threading
 * -----------------------
 * The caller owns every host array; set_problem copies what it needs.  A
 * handle owns all device memory it allocates and frees it in destroy.  One
 * handle is bound to one device and one CUDA stream and is not thread safe.
 * Device-pointer entry points (proxsdp_gpu_aproj, _block_matvec, _sym_eig)
 * read and write caller-owned device memory on the given stream and allocate
 * their own scratch (released before they return).
 */
#ifndef PROXSDP_GPU_H
#define PROXSDP_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define PROXSDP_OK 0
#define PROXSDP_ERR_INVALID_ARG (-1) /* bad sizes, malformed CSR, NaN/Inf, NULL where required */
#define PROXSDP_ERR_CUDA (-2)        /* CUDA runtime error, or no usable device */
#define PROXSDP_ERR_OOM (-3)         /* device allocation failed */
#define PROXSDP_ERR_BAD_STATE (-4)   /* e.g. solve before set_problem */
#define PROXSDP_ERR_UNSUPPORTED (-5) /* size beyond a compiled limit */
#define PROXSDP_ERR_TIMEOUT (-6)     /* a bounded device wait ran out */

/* proxsdp_gpu_info.status */
#define PROXSDP_CONVERGED 0           /* residuals and gap <= tol with a sufficient rank */
#define PROXSDP_MAX_ITER 1            /* max_iter reached */
#define PROXSDP_TIME_LIMIT 2          /* time_limit_s reached */
#define PROXSDP_STALLED_AT_MAX_RANK 3 /* the rank rule asked for r > max_rank */
#define PROXSDP_NUMERIC_ERROR 4       /* NaN/Inf in the iteration */

/* precision of the S * V products and the rebuild */
#define PROXSDP_PREC_FP32 0

/* proxsdp_gpu_settings.operator_form: how the projection applies
 * S^k = X^k - alpha (C + M*(y^k)) (Alg. 2 primal step) to its Krylov blocks.
 * EXPLICIT writes S^k (n*n FP32) to device memory every iteration and
 * multiplies it; FACTORED never forms it and applies
 * V Lambda_+ V^T Q - alpha (C + M*(y^k)) Q from the factors of X^k (Sec. 3)
 * and the union sparsity pattern of C and the A_i, O(n r w + nnz w) per
 * product; AUTO takes FACTORED when that pattern holds at most n*n/8 entries.
 * Problems with n <= 128 and Alg. 1 (full_eig) always use the explicit S. */
#define PROXSDP_OP_EXPLICIT 0
#define PROXSDP_OP_FACTORED 1
#define PROXSDP_OP_AUTO 2

typedef struct proxsdp_gpu_ctx* proxsdp_gpu_t;

/* Settings; proxsdp_gpu_settings_default fills the defaults listed here. */
typedef struct {
  double tol;             /* stop when max(rel_primal, rel_dual, rel_gap) <= tol      [1e-4] */
  int64_t max_iter;       /* iteration cap                                              [1e6]  */
  double time_limit_s;    /* wall-clock cap of one solve call (Sec. 5 uses 1200 s)      [1200] */
  int full_eig;           /* 1: PD-SDP (Alg. 1, exact projection), 0: LR-PD-SDP (Alg. 2) [0]   */
  int rank_init;          /* initial target rank r (Alg. 2 starts at 1)                  [8]   */
  int block_size;         /* Lanczos block granularity b; block width = b*ceil((r+g)/b)  [16]  */
  int window;             /* stall window l of Sec. 3.2 (<= 1024)                        [100] */
  double eps_lambda;      /* rank test threshold of Alg. 2; <= 0 means tol               [0]   */
  double alpha_frac;      /* step alpha = alpha_frac / ||M||_2 (Sec. 2.2: alpha<1/||M||) [0.95]*/
  int precision;          /* PROXSDP_PREC_FP32                                           [0]   */
  int normalize_rows;     /* scale each (A_i, rhs_i) to ||A_i||_F = 1                    [1]   */
  uint64_t seed;          /* Lanczos start block                                         [1]   */
  int max_rank;           /* cap on the target rank; the Lanczos path (n > 128) holds
                             at most 64, or 60 with the factored operator                [64]  */
  int lanczos_steps;      /* block Krylov steps per restart cycle (0: automatic)         [0]   */
  int lanczos_max_cycles; /* restart cycles per projection                               [8]   */
  double lanczos_tol;     /* Ritz residual tolerance relative to |theta_1| (0: adaptive) [0]   */
  int guard;              /* extra Ritz vectors kept beyond r (0: automatic)             [0]   */
  int check_every;        /* iterations between host checks of the stop status           [50]  */
  int use_graphs;         /* run the iteration as a CUDA graph with conditional nodes    [1]   */
  int operator_form;      /* PROXSDP_OP_EXPLICIT / _FACTORED / _AUTO                     [0]   */
  int64_t memory_limit_bytes; /* cap on the device memory one handle allocates; set_problem
                                 returns PROXSDP_ERR_OOM beyond it (0: no cap)        [0]   */
  int at_max_rank;        /* when Alg. 2's rank rule asks for r > max_rank: 0 stops with
                             PROXSDP_STALLED_AT_MAX_RANK; 1 keeps iterating at max_rank,
                             and there the stop test accepts residuals and gap within
                             tol without the rank test (the pair is then certified by
                             its residuals and gap only)                             [0]   */
} proxsdp_gpu_settings;

typedef struct {
  int status;                /* PROXSDP_CONVERGED, ... */
  int final_rank;            /* target rank r at exit */
  int64_t iters;             /* PDHG iterations */
  int rank_changes;          /* number of rank doublings */
  double primal_obj;         /* tr(C X) */
  double dual_obj;           /* [b; h]^T y (paper's dual sign) */
  double rel_primal_res;     /* eps_primal / (1 + ||C||_F) on the row-scaled problem */
  double rel_dual_res;       /* eps_dual / (1 + ||rhs||_2) on the row-scaled problem */
  double rel_gap;            /* |pobj - dobj| / (1 + |pobj| + |dobj|) */
  double eps_primal;         /* Sec. 2.2 primal residual (row-scaled problem) */
  double eps_dual;           /* Sec. 2.2 dual residual (row-scaled problem) */
  double lambda_r;           /* r-th largest eigenvalue of the last projected matrix */
  double solve_seconds;      /* device time of the solve call */
  int64_t matvecs;           /* block products S * V (each reads S once) */
  int64_t lanczos_cycles;    /* restart cycles over all projections */
  int64_t lanczos_unconverged; /* projections that hit lanczos_max_cycles */
  double alpha;              /* step size used */
  double norm_M;             /* ||M||_2 of the row-scaled operator */
  int64_t kernel_launches;   /* library kernels executed by the iterations of this call sequence */
} proxsdp_gpu_info;

/* Fill *s with the defaults above. */
int proxsdp_gpu_settings_default(proxsdp_gpu_settings* s);

/* Create a solver bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL: the library creates its own).  `settings` may be NULL
 * (defaults).  Returns PROXSDP_ERR_CUDA when the device is not usable. */
int proxsdp_gpu_create(const proxsdp_gpu_settings* settings, int device, void* cuda_stream,
                       proxsdp_gpu_t* out);

/* Load a problem (Sec. 1.3).  C is dense (n*n doubles, symmetric; row and
 * column major coincide) when C_dense != NULL, else sparse svec entries
 * (c_nnz, c_idx, c_val; duplicates are summed).  A_rowptr has m_total+1
 * entries, A_col/A_val A_rowptr[m_total] entries (svec indices, or a lone -1
 * for a dense a*11^T row).  rhs = [b; h] (m_total).  Validates everything
 * (sorted-or-not, in-range indices, finite values) and returns
 * PROXSDP_ERR_INVALID_ARG on malformed input; copies the data to the device,
 * scales rows (settings.normalize_rows) and computes ||M||_2 and alpha.
 * Device memory: O(n*128 + nnz) for the Krylov basis, the factors and the
 * sparse data, plus n * ceil(n/32)*32 floats for S unless the factored
 * operator form applies (operator_form); PROXSDP_ERR_OOM when it does not fit. */
int proxsdp_gpu_set_problem(proxsdp_gpu_t h, int64_t n, const double* C_dense, int64_t c_nnz,
                            const int64_t* c_idx, const double* c_val, int64_t m_total,
                            int64_t m_eq, const int64_t* A_rowptr, const int64_t* A_col,
                            const double* A_val, const double* rhs);

/* Host-only analysis of a problem (no device needed): validates the data
 * exactly as set_problem does and reports the row-scaled operator norm
 * ||M||_2 (power iteration on the Gram operator v -> M(M*(v))), the step
 * alpha = alpha_frac/||M||_2 (Sec. 2.2 requires alpha < 1/||M||_2), the
 * size of the union sparsity pattern of C and the A_i, and ||C||_F.  Any
 * output pointer may be NULL.  Returns PROXSDP_ERR_INVALID_ARG on malformed
 * input (same checks as set_problem). */
int proxsdp_gpu_analyze_problem(const proxsdp_gpu_settings* settings, int64_t n, const double* C_dense,
                                int64_t c_nnz, const int64_t* c_idx, const double* c_val,
                                int64_t m_total, int64_t m_eq, const int64_t* A_rowptr,
                                const int64_t* A_col, const double* A_val, const double* rhs,
                                double* norm_M, double* alpha, int64_t* n_union, double* norm_C);

/* Run Alg. 2 (or Alg. 1 with full_eig) from X = 0, y = 0 until convergence or a
 * cap.  `info` may be NULL. */
int proxsdp_gpu_solve(proxsdp_gpu_t h, proxsdp_gpu_info* info);

/* Solve `count` independent problems concurrently on one GPU (many small
 * instances of uneven size).  handles[i] is a handle created with its own
 * stream (cuda_stream = NULL at create) and loaded with set_problem; all
 * handles must be distinct.  `host_threads` host threads (<= 0: 16, at most
 * `count`) each take the next unsolved handle, largest n first, and run
 * proxsdp_gpu_solve on it, so the kernels and graphs of different handles run
 * concurrently on their streams.  infos[i] (infos may be NULL) receives
 * handle i's result.  Every handle is attempted; the return value is the
 * first nonzero code in handle order (its message is on that handle), or
 * PROXSDP_ERR_INVALID_ARG for a NULL/repeated handle (message on NULL).
 * The CUDA_DEVICE_MAX_CONNECTIONS environment variable (set before the first
 * CUDA call of the process) bounds how many streams run without false
 * dependencies. */
int proxsdp_gpu_solve_batch(proxsdp_gpu_t* handles, int count, proxsdp_gpu_info* infos, int host_threads);

/* Copy the last iterate to the host.  Any pointer may be NULL.
 *   X      n*n doubles (dense V diag(max(lambda,0)) V^T),
 *   y      m_total doubles, the paper's dual sign, original row scaling,
 *   V      n*r doubles, column-major Ritz vectors (r = *r_out),
 *   lambda r doubles, the Ritz values (unclamped),
 *   r_out  the number of factors. */
int proxsdp_gpu_get_primal_dual(proxsdp_gpu_t h, double* X, double* y, double* V,
                                double* lambda, int64_t* r_out);

/* Add the element-wise box -u <= X_ij <= u for all i != j (the bounds of the
 * MIMO relaxation, Sec. 5.3) to the loaded problem as a structured class of
 * n (n - 1) inequality rows, X_ij <= u and -X_ij <= u for i < j, without
 * passing them as CSR rows: their duals are two dense n x n arrays on the
 * device (8 n^2 bytes) and their dual step runs element-wise beside the
 * rebuild of S^k.  The rows take part in everything the CSR rows do (the
 * step alpha = alpha_frac / ||M||_2 of the extended operator, the residuals,
 * rhs^T y), with the same row scaling (sqrt(2) when normalize_rows).  Call it
 * after set_problem and before solve; a new set_problem removes it.
 * Supported when every CSR row acts on the diagonal only (diag(X) = b type
 * rows, as in Sec. 5.3) and the operator form is explicit: otherwise
 * PROXSDP_ERR_UNSUPPORTED (pass the bounds as CSR rows instead).
 * PROXSDP_ERR_INVALID_ARG unless 0 < u < inf; PROXSDP_ERR_BAD_STATE before
 * set_problem. */
int proxsdp_gpu_set_box(proxsdp_gpu_t h, double u);

/* Copy the duals of the element-wise box rows of the current iterate: n x n
 * row-major, Y_upper for X_ij <= u and Y_lower for -X_ij <= u (i != j; zero
 * diagonal), the paper's sign (<= 0) and original scaling, symmetric.
 * Either pointer may be NULL.  PROXSDP_ERR_BAD_STATE without a box or an
 * iterate.  proxsdp_gpu_set_iterate (and so a resume from a saved pair)
 * starts the box duals from zero. */
int proxsdp_gpu_get_box_dual(proxsdp_gpu_t h, double* Y_upper, double* Y_lower);

/* Copy the feasible pair (X_[r], y_[r]) that Alg. 2 saves ("save feasible
 * solution", Sec. 3.2): the last iterate of the most recent solve / iterate
 * call at which the relative residuals met tol while the rank test found the
 * rank r insufficient (so r was doubled, or the solve stopped at max_rank).
 * Same outputs and layouts as proxsdp_gpu_get_primal_dual, plus iter_out, the
 * iteration at which it was saved.  Any pointer may be NULL.  Returns
 * PROXSDP_ERR_BAD_STATE when no pair was saved since the iteration started
 * (solve, or set_iterate followed by iterate). */
int proxsdp_gpu_get_saved_pair(proxsdp_gpu_t h, double* X, double* y, double* V, double* lambda,
                               int64_t* r_out, int64_t* iter_out);

/* Set the iterate (X = V diag(max(lambda,0)) V^T with V n*r column-major,
 * orthonormal columns, and y in the paper's dual sign / original scaling) and
 * the target rank, so that proxsdp_gpu_iterate continues from it (one-step
 * parity against Alg. 1 / Alg. 2, or resuming from a saved pair).  On the
 * block Lanczos path (n > 128) r <= 64, or r <= 60 with the factored
 * operator; larger r returns PROXSDP_ERR_UNSUPPORTED. */
int proxsdp_gpu_set_iterate(proxsdp_gpu_t h, int r, const double* V, const double* lambda,
                            const double* y);

/* Run exactly `iters` iterations of Alg. 2 from the current iterate (rank
 * rule active), then fill `info` with the residuals of the last one. */
int proxsdp_gpu_iterate(proxsdp_gpu_t h, int64_t iters, proxsdp_gpu_info* info);

/* Continue Alg. 2 from the current iterate until its stop test holds (Sec. 3.2:
 * residuals within the tolerance at a sufficient rank, gap within the
 * tolerance), for at most `max_iters` further iterations (< 0: up to
 * settings.max_iter in total) and settings.time_limit_s for this call.  The
 * current iterate is where the last solve, iterate or resume call stopped,
 * or the one given to proxsdp_gpu_set_iterate (for instance a saved feasible
 * pair (X_[r], y_[r]) from proxsdp_gpu_get_saved_pair); without one the run
 * starts from X = 0, y = 0 like proxsdp_gpu_solve.  Iteration counts in
 * `info` are cumulative.  A solve interrupted by a cap and resumed goes
 * through the same iterates as one run without interruption.  Returns
 * PROXSDP_ERR_BAD_STATE before set_problem. */
int proxsdp_gpu_resume(proxsdp_gpu_t h, int64_t max_iters, proxsdp_gpu_info* info);

/* Destroy the handle and free its device memory. */
void proxsdp_gpu_destroy(proxsdp_gpu_t h);

/* Last error message of the handle (or of the last failed create when h is
 * NULL).  Valid until the next call on the handle. */
const char* proxsdp_gpu_last_error(proxsdp_gpu_t h);

/* ---------------------------------------------------------------------------
 * Building blocks on caller-owned device memory (all pointers are device
 * pointers; `cuda_stream` is a cudaStream_t or NULL for the legacy stream).
 * ------------------------------------------------------------------------- */

/* Truncated psd projection aproj(S, r) of Sec. 3.1 (Eq. trunc_eig):
 * P = sum_{t<r} max(lambda_t, 0) v_t v_t^T over the r algebraically largest
 * eigenpairs of the symmetric S (n x n FP32, row stride lds >= n).  Computed
 * with the library's restarted block Lanczos (n > 128) or the one-block dense
 * eigensolver of proxsdp_gpu_sym_eig (n <= 128).  Outputs (each may be NULL): P (n x n FP32, stride ldp), V
 * (n x r FP32 column-major, stride n), lambda (r FP64, descending,
 * unclamped).  `settings` may be NULL.  `info` (may be NULL) receives
 * matvecs / lanczos_cycles / lanczos_unconverged / lambda_r. */
int proxsdp_gpu_aproj(const float* S, int64_t n, int64_t lds, int r, float* P, int64_t ldp,
                      float* V, double* lambda, const proxsdp_gpu_settings* settings,
                      void* cuda_stream, proxsdp_gpu_info* info);

/* aproj(S, r) for callers that cannot allocate device memory.  The paper has
 * no counterpart; this entry point exists for callers such as applications
 * whose own pool allocator owns all GPU memory and forbids other allocations,
 * plugins running inside such hosts, and embedded or real-time hosts that
 * must not allocate (or risk an allocation failure) while they run.  Same
 * arguments, results, defaults and errors as proxsdp_gpu_aproj (settings are
 * validated the same way; an unsupported device gives PROXSDP_ERR_CUDA), but
 * the work buffers live in one file-scope static device array of about
 * 6.7 MB, which every GPU that loads the library holds until the process
 * exits; nothing is allocated per call (no cudaMalloc/cudaFree, no allocating
 * library routine).
 * Limits: n <= 2048 (larger n returns PROXSDP_ERR_UNSUPPORTED with a message
 * for proxsdp_gpu_last_error(NULL)); r as for proxsdp_gpu_aproj.
 * The first call on a device looks up the array's device address on that
 * device with cudaGetSymbolAddress and keeps it for later calls.  The kept address
 * belongs to the device's primary context: after cudaDeviceReset (or any
 * other end of that context) the process must not call this entry point
 * again on that device.  All calls share the one array, which keeps the
 * previous call's contents, so calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller; each call
 * clears the parts that must start at zero and synchronises its stream
 * before returning. */
int proxsdp_gpu_aproj_noalloc(const float* S, int64_t n, int64_t lds, int r, float* P, int64_t ldp,
                              float* V, double* lambda, const proxsdp_gpu_settings* settings,
                              void* cuda_stream, proxsdp_gpu_info* info);

/* Symmetric block product W = S * Q (the Lanczos matvec of Sec. 3.1): S
 * n x n FP32 with row stride lds, Q n x k FP32 column-major (stride
 * ldq >= n), W likewise (stride ldw).  k <= 256.  For n >= 1024, when S
 * starts on a 16-byte boundary and lds is a multiple of 4, the product runs
 * on the tensor cores (S streamed by TMA, 3xTF32 with FP32 sums, FP32-grade
 * accuracy, relative bias about -9e-8); otherwise on the SIMT FP32 kernel
 * (below n = 1024 S stays in L2, where it is as fast, with a bias about
 * -1e-9).  Scratch (2 * ceil(n/32)*32 * k floats for the
 * TF32 parts of Q) comes from a library-owned stream-ordered pool that keeps
 * its largest block until the process exits.  Asynchronous on cuda_stream;
 * a tensor-core CTA whose bounded waits run out writes NaN to its rows of W. */
int proxsdp_gpu_block_matvec(const float* S, int64_t n, int64_t lds, const float* Q, int64_t ldq,
                             int k, float* W, int64_t ldw, void* cuda_stream);

/* Eigendecomposition of a small symmetric matrix T (K x K FP64 row-major,
 * K <= 128) in one thread block (the Rayleigh-Ritz step of the Lanczos
 * solver): Householder reduction to tridiagonal form, Sturm-count bisection,
 * inverse iteration (groups of close eigenvalues orthogonalised together),
 * back-transformation, and one correction of every vector from residuals
 * accumulated in FP32 pairs.  Outputs theta (K FP64, descending, Rayleigh
 * quotients) and Y (K x K FP32 column-major eigenvectors, column t for
 * theta[t]). */
int proxsdp_gpu_sym_eig(const double* T, int K, double* theta, float* Y, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PROXSDP_GPU_H */
