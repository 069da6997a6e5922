// psdp.cuh — internal types and kernel launchers of the GB300 LR-PD-SDP library.
//
// Device state of one solver handle.  The iteration of Alg. 2 is split into
// kernels that read their dynamic sizes (rank, block width, parity of the
// ping-pong buffers, convergence flags) from a device control block `Ctl`, so
// that one iteration can be captured once as a CUDA graph and replayed under a
// conditional WHILE node without host round trips.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace psdp {

constexpr int kMaxWindow = 1024;  // longest stall window l (Sec. 3.2)
constexpr int kMaxK = 128;        // largest Rayleigh-Ritz basis (one-block eigensolver)
constexpr int kMaxW = 64;         // largest Krylov block width (products, orthogonalisation pieces)
constexpr int kMaxP = 112;        // largest kept Ritz block the kernels hold (the restart vectors, r + guard)
// Largest target rank on the Lanczos path: a kept block of r + 16 = 80 and an
// expansion of 48 fill the 128-wide Rayleigh-Ritz basis.  Measured on
// cold-start projections (100 restart cycles, tolerance 1e-6): r = 72 with
// 8 guard vectors stays 2.4e-4 off, r = 80 with an expansion of 32 1.5e-3,
// r >= 96 with 16 about 4e-2.
constexpr int kMaxRankLanczos = 64;
constexpr int kMaxRankFactored = 60;  // the factored operator holds at most 63 factors
constexpr int kFullEigMax = 128;  // n up to which the projection uses the dense eigensolver
constexpr int kTile = 64;         // rebuild tile edge
constexpr int kRedSlots = 16;     // scalar reductions per kernel
constexpr int kMaxR = 128;        // largest factor rank held (full projection up to n = 128)

enum Status : int {
  ST_CONVERGED = 0,
  ST_MAX_ITER = 1,
  ST_TIME_LIMIT = 2,
  ST_STALLED_MAX_RANK = 3,
  ST_NUMERIC = 4,
  ST_RUNNING = 5,
  ST_RANK_CHANGE = 6,  // the controller asked for r <- 2r; the host regrows the basis
  ST_PAUSE = 7,        // reached the host-set iteration bound
};

// Device control block (one per handle).
struct Ctl {
  int it;            // completed PDHG iterations
  int par;           // buffer index holding the current iterate X^k
  int r;             // target rank
  int w;             // Lanczos block width
  int K;             // Rayleigh-Ritz basis size
  int status;
  int lz_done;       // projection of the current iteration converged
  int lz_cycle;      // restart cycles run in the current iteration
  int k_change;      // iteration of the last rank change
  int it_stop;       // pause after this many iterations
  int r_old;         // rank of X^k (differs from r right after a rank change)
  int rank_changes;
  int saved;         // feasible (X_[r], y_[r]) pairs seen (Alg. 2)
  int full_eig;      // 1: exact projection (Alg. 1)
  int window;
  int max_rank;
  int max_cycles;
  int fixed_rank;    // 1: never change r (building-block use)
  int full_eig_path; // projection by the dense eigensolver (n <= 128 or Alg. 1)
  int at_max_rank;   // 1: keep iterating at max_rank instead of stopping (settings.at_max_rank)
  long long matvecs;
  long long lz_cycles_total;
  long long lz_unconverged;
  long long launches;   // kernels launched by the iteration (graph nodes executed)
  double tol, eps_lambda, lz_tol_fixed, lz_tol;
  double eps_p, eps_d, rel_p, rel_d, rel_gap, pobj, dobj, lam_r, normX, lz_res;
  double red_dual[kRedSlots];
  double red_dvals[kRedSlots];
  double hist[kMaxWindow];
};

// Problem data on the device (row-scaled).  Constraint rows 0..m-1 plus the
// objective C as row m ("extended" operator) so tr(CX) comes out of M(X).
struct DevProblem {
  int n, m, m_eq;
  int nnz_ext;                 // entries of the extended rows
  const int* dense_of_row;     // m: index into dense_row / dense_a, or -1
  const int* ent_p;            // entry row index p (p <= q)
  const int* ent_q;
  const double* ent_a;         // a, times 2 off the diagonal: tr(A X) = sum a_eff X_pq
  int n_chunks;                // work chunks of <= kChunk entries of one row
  const int* chunk_beg;
  const int* chunk_end;
  const int* row_chunk;        // m + 2: chunks of row i are [row_chunk[i], row_chunk[i+1]) (>= 1 each)
  const int* chunk_row;        // row of each chunk
  int n_multi;                 // constraint rows with more than one chunk
  const int* multi_rows;
  const double* rhs;           // m (scaled)
  int n_dense;                 // structured rows a * 11^T
  const int* dense_row;
  const double* dense_a;
  // union pattern of C and all A_i (upper triangle), for D = C + M*(y)
  int nU;
  const int* u_p;
  const int* u_q;
  const double* u_c;           // C entry (0 where C has none)
  const int* u_ptr;            // nU + 1
  const int* u_row;            // constraint row of each contribution
  const double* u_a;           // its (scaled) matrix entry value
  // rebuild tiles: entries of the (full, both triangles) pattern per 64x64 tile
  int ntile;                   // tiles per dimension
  const int* tile_ptr;         // ntile*ntile + 1
  const int* tile_loc;         // local offset lr*64 + lc
  const int* tile_u;           // union entry index
  double alpha;
  double normC, normRhs;       // ||C||_F, ||rhs||_2 (scaled problem)
  // element-wise box -u <= X_pq <= u for all p != q as a structured row
  // class (duals in DevWork::ybp / ybm): rows +-box_s (E_pq + E_qp) / 2 with
  // rhs box_s * u; box = 0 when absent
  int box;
  float box_s, box_u;
  const double* C_dense;       // dense C (row-major n x n) or nullptr
  // rows of the full (both triangles) union pattern, for the factored
  // operator: row i holds entries [sym_ptr[i], sym_ptr[i+1]) at columns
  // sym_col; union entry u sits at u_pos[2u] (row u_p) and, off the diagonal,
  // at u_pos[2u+1] (row u_q; -1 on the diagonal)
  int nsym;
  const int* sym_ptr;          // n + 1
  const int* sym_col;
  const int* u_pos;            // 2 nU
};

// Work buffers.
struct DevWork {
  float* S;  int lds;          // n x n row-major, row stride lds
  float* Q;  float* W;  int ldq;  // n x kMaxK column-major Lanczos basis and S*Q
  float* Vrm[2];  int ldv;     // X factors, n x ldv row-major (ping-pong by Ctl::par), ldv = kMaxR
  double* lam[2];              // their eigenvalues (unclamped), ldv each
  double* colsum[2];           // column sums of Vrm (structured dense rows)
  double* y;                   // current dual (scaled problem, algorithm sign)
  double* dy;                  // last dual change
  double* mx[2];               // M_ext(X) for both buffers (m + 1)
  double* chunk_part;          // per-chunk partial sums
  double* D;                   // D = C + M*(y) on the union pattern
  double* dshift;              // [0]: sum over dense rows a*y, [1]: same with dy
  double* part;                // generic per-CTA partials
  double* H;                   // small dense FP64 results (Gram, T)
  float* Hf;                   // FP32 copy / R^{-1}
  int* flags;                  // deficient-column flags
  float* Y;  double* theta;    // Ritz solve output (kMaxK x kMaxK), values
  double* ritz_part;           // partials of the Ritz kernel
  unsigned* counters;          // last-block counters (512 per kernel kind)
  float* Vcm;                  // column-major factor slots [slot 0 | slot 1], kMaxR columns each
  double* Hx;                  // Gram of the factor slots (2 kMaxR)^2
  float* mv_part;              // split-K partials of the block product
  unsigned* mv_cnt;            // its per-tile counters
  // factored operator (S never formed; all three nullptr on the explicit path)
  float* Dsym;                 // (float)(alpha * D) on the full pattern, CSR order of sym_col
  float* Qr;                   // row-major copy of the block being multiplied (n x w)
  float* lrP;                  // its coefficient block [Lambda_+ V^T Q ; -alpha s0 1^T Q]
  // duals of the box rows X_pq <= u (ybp) and -X_pq <= u (ybm), algorithm
  // sign (>= 0), scaled problem: n x n symmetric, row stride lds (nullptr
  // without a box)
  float* ybp;
  float* ybm;
  Ctl* ctl;
};

enum CounterId { CNT_GRAM = 0, CNT_RITZ, CNT_DUAL, CNT_DVALS, CNT_CTL, CNT_BOX, CNT_NUM };

// Ctl::red_dvals slots written by the box kernel: its rows' shares of
// eps_dual^2, <dy, M(dX)>, rhs^T y and ||M*(dy)||_F^2
constexpr int kRedBox = 4;

// ---------------------------------------------------------------------------
// launchers (k_lanczos.cu)
// ---------------------------------------------------------------------------
// W = S Q (S n x n symmetric, row stride lds; Q, W column-major).  With
// `part` (block_matvec_scratch_floats(n, k) floats: the TF32 high / low parts
// of Q) and S meeting the TMA alignment rules (16-byte base, lds a multiple
// of 4) the product runs on the tensor cores (k_mv_tc.cu); otherwise on the
// SIMT kernel (inner dimension split over a thread-block cluster).
void launch_block_matvec(const float* S, int lds, int n, const float* Q, int ldq, float* W, int ldw,
                         int k, const int* skip, cudaStream_t st, float* part = nullptr,
                         unsigned* counters = nullptr, cudaGraphConditionalHandle cond = 0,
                         int set_cond = 0);
size_t block_matvec_scratch_floats(int n, int k);
size_t block_matvec_counters(int n, int k);
void launch_random_block(float* Q, int ldq, int n, int col0, int k, unsigned long long seed,
                         cudaStream_t st);
// Z (n x b, stride ldz) = columns (off + j) mod w of W (n x w, stride ldw),
// off = (restart cycles so far) * b mod w, read from the control block.
void launch_compress_block(const float* W, int ldw, int w, float* Z, int ldz, int b, int n, const Ctl* ctl,
                           const int* skip, cudaStream_t st);
// launchers (k_mv_tc.cu): the tensor-core block product; false (nothing
// launched) when it does not apply
bool launch_block_matvec_tc(const float* S, int lds, int n, const float* Q, int ldq, float* W, int ldw, int k,
                            const int* skip, cudaStream_t st, float* scratch, cudaGraphConditionalHandle cond,
                            int set_cond);
size_t block_matvec_tc_scratch_floats(int n, int k);
// The tensor-core product runs from kTcMinN up.  Below it S (<= 4 MB) stays
// in L2, where the SIMT kernel takes the same time (measured at n = 2000:
// 28 us each), and the SIMT product's bias is about 100x smaller (-1e-9
// against -9e-8 relative): on MIMO relaxations at n = 284..511 that bias
// left the duality gap at 2e-4..4e-4 with residuals near 1e-6 (45 of 256
// instances of the batch workload), and the same instances converge with the
// SIMT product.
constexpr int kTcMinN = 1024;
bool block_matvec_tc_applies(const float* S, int lds, int n, const float* scratch);
// kernels one launch_block_matvec enqueues (the tensor-core path splits Q first)
inline int block_matvec_kernels(const float* S, int lds, int n, const float* scratch) {
  return block_matvec_tc_applies(S, lds, n, scratch) ? 2 : 1;
}
bool block_matvec_tc_enabled();
void init_mv_tc_attributes();
// H = A^T B (ka x kb, FP64 row-major) with deterministic block reduction.
// With act > 0 only output tiles whose row and column offsets modulo `slot`
// fall below `act` are computed (Gram of a few columns of each factor slot).
void launch_gram(const float* A, int lda, int ka, const float* B, int ldb, int kb, int n,
                 double* H, double* part, unsigned* counter, const int* skip, cudaStream_t st,
                 int act = 0, int slot = 0);
// Z -= A * H
void launch_block_update(float* Z, int ldz, int kb, const float* A, int lda, int ka, const double* H,
                         int n, const int* skip, cudaStream_t st);
// Cholesky of G (w x w), writes R^{-1} (FP32) and deficient flags.
void launch_chol_inv(const double* G, int w, float* Rinv, int* flags, const int* skip, cudaStream_t st);
// Z <- Z * R^{-1}; deficient columns replaced by pseudo-random vectors.
void launch_apply_rinv(float* Z, int ldz, int w, const float* Rinv, const int* flags, int n,
                       unsigned long long seed, const int* skip, cudaStream_t st);
// Eigenpairs of the symmetric K x K T (FP64 row-major, K <= 128): the nout
// algebraically largest, descending, to theta / Y (columns, stride ldy).
// refine = 1 corrects the wanted vectors once from residuals accumulated in
// FP32 pairs and returns FP64 Rayleigh quotients; refine = 0 returns the FP32
// eigenpairs of the tridiagonal method as they are.  With adapt_tol (a device
// pointer) the kernel refines only when *adapt_tol is below 5e-6.
void launch_sym_eig(const double* T, int K, double* theta, float* Y, int ldy, int nout,
                    const int* skip, cudaStream_t st, int refine = 1, const double* adapt_tol = nullptr);
void init_lanczos_attributes();
void init_orth_attributes();
bool orth_cluster_applies(int n, int c0, int w);
void launch_orth_cluster(float* Q, int ldq, const float* src, int n, int c0, int w, int passes,
                         int chol_first, unsigned long long seed, const int* skip, cudaStream_t st);

// ---------------------------------------------------------------------------
// launchers (k_pdhg.cu)
// ---------------------------------------------------------------------------
void launch_ritz(const DevWork& wk, int n, int K, int w, int r, int s_steps, int cycle_launches,
                 cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st);
// M(X^{k+1}) from the factors fused with the dual step and its reductions.
void launch_mxdual(const DevProblem& pb, const DevWork& wk, int r, cudaStream_t st);
void launch_dvals(const DevProblem& pb, const DevWork& wk, cudaStream_t st);
// Gram of the factor slots (columns < act of each slot) fused with the controller.
void launch_gram_control(const DevProblem& pb, const DevWork& wk, int act, int iter_launches,
                         cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st);
// sel = 0: factors of the current iterate (Ctl::par); sel = 1: the other buffer.
void launch_rebuild(const DevProblem& pb, const DevWork& wk, int r, int sel, cudaStream_t st);
// Dual step of the element-wise box rows and their residual / objective
// shares (after launch_dvals, before launch_gram_control).
void launch_box_dual(const DevProblem& pb, const DevWork& wk, int r, cudaStream_t st);
// Streaming multiprocessors of the current device (launch heuristics).
int num_sms();

// ---------------------------------------------------------------------------
// launchers (k_factored.cu)
// ---------------------------------------------------------------------------
// W = S^k Q for the w <= 64 columns of Q without S: S^k = V Lambda_+ V^T -
// alpha (D_sym + s0 11^T) with the factors of the current iterate (Ctl::par,
// Ctl::r_old columns) and Dsym / dshift[0] as written by the last launch_dvals.
// Two kernels; the second sets the graph conditional `cond` to 1 when set_cond.
void launch_factored_matvec(const DevProblem& pb, const DevWork& wk, const float* Q, int ldq, float* W,
                            int ldw, int w, const int* skip, cudaStream_t st,
                            cudaGraphConditionalHandle cond = 0, int set_cond = 0);
constexpr int kFactoredLaunches = 2;  // kernels per factored product
void init_factored_attributes();
void launch_copy_cols(const float* src, int lds, float* dst, int ldd, int n, int k, const int* skip,
                      cudaStream_t st);
void launch_full_eig_factors(const DevWork& wk, int n, cudaStream_t st);
void launch_s_to_t(const float* S, int lds, int n, double* T, cudaStream_t st);
void launch_ctl_set(Ctl* ctl, int status, int it_stop, int r, int w, int K, int k_change,
                    cudaStream_t st);
void init_pdhg_attributes();
void launch_count_nonfinite_f(const float* p, size_t count, unsigned* out, cudaStream_t st);
void launch_count_nonfinite_d(const double* p, size_t count, unsigned* out, cudaStream_t st);

}  // namespace psdp
