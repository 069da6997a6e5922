// solver.cu — device memory, kernel sequencing and CUDA-graph capture of the
// LR-PD-SDP iteration (Alg. 2; Alg. 1 when every eigenpair is kept).
//
// One iteration is:
//   warm-start product  W[:, :w] = S^k Q[:, :w]        (Q[:, :w]: Ritz vectors of S^{k-1})
//   restart cycles       block Krylov steps + Rayleigh-Ritz until the r wanted
//                        Ritz pairs have converged                  (aproj, Sec. 3.1)
//   M(X^{k+1})           from the factors                           (dual step part 1)
//   dual step            equality / inequality split                (Eq. resolvent_1)
//   D = C + M*(y^{k+1})  and ||M*(dy)||
//   controller           residuals (Sec. 2.2), stop test, rank rule (Sec. 3.2)
//   rebuild              S^{k+1} = X^{k+1} - alpha D                (primal step input)
// Inside a CUDA graph the restart cycles sit under a conditional WHILE node
// (set by the Ritz kernel) and the iterations under an outer WHILE node (set
// by the controller), so a whole batch of iterations runs without the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <mutex>

#include "solver.h"

namespace psdp {

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return fail(PROXSDP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Debugging aid (environment variable PSDP_DEBUG=1, direct launches only):
// after every kernel, synchronise and report the first buffer that holds a
// non-finite value, with the name of the kernel that ran last.
static bool g_debug = getenv("PSDP_DEBUG") != nullptr;
static bool g_debug_reported = false;
static unsigned* g_debug_cnt = nullptr;
static int g_debug_n = 0;

static void dbg(const DevWork& wk, const char* tag, cudaStream_t st) {
  if (!g_debug || g_debug_reported) return;
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (!g_debug_cnt) cudaMallocManaged(&g_debug_cnt, 16 * sizeof(unsigned));
  const int n = g_debug_n;
  struct B {
    const char* name;
    const void* p;
    size_t count;
    bool dbl;
  } bufs[] = {{"S", wk.S, (size_t)n * wk.lds, false}, {"Q", wk.Q, (size_t)wk.ldq * kMaxK, false},
              {"W", wk.W, (size_t)wk.ldq * kMaxK, false}, {"Vrm0", wk.Vrm[0], (size_t)n * kMaxR, false},
              {"Vrm1", wk.Vrm[1], (size_t)n * kMaxR, false}, {"lam0", wk.lam[0], kMaxR, true},
              {"lam1", wk.lam[1], kMaxR, true}, {"H", wk.H, (size_t)kMaxK * kMaxK, true},
              {"Y", wk.Y, (size_t)kMaxK * kMaxK, false}, {"theta", wk.theta, kMaxK, true},
              {"Hf", wk.Hf, (size_t)kMaxW * kMaxW, false}};
  const int nb = sizeof(bufs) / sizeof(bufs[0]);
  cudaStreamSynchronize(st);
  for (int b = 0; b < nb; ++b) g_debug_cnt[b] = 0;
  for (int b = 0; b < nb; ++b) {
    if (!bufs[b].p) continue;
    if (bufs[b].dbl) launch_count_nonfinite_d((const double*)bufs[b].p, bufs[b].count, g_debug_cnt + b, st);
    else launch_count_nonfinite_f((const float*)bufs[b].p, bufs[b].count, g_debug_cnt + b, st);
  }
  cudaStreamSynchronize(st);
  for (int b = 0; b < nb; ++b) {
    if (g_debug_cnt[b]) {
      fprintf(stderr, "[psdp debug] after %s: %u non-finite values in %s\n", tag, g_debug_cnt[b], bufs[b].name);
      g_debug_reported = true;
    }
  }
}

// Function attributes are per device: set them once on each device, under a
// lock (solves of a batch start from several host threads).
void init_kernel_attributes() {
  static std::mutex mu;
  static bool done[256] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 256 || done[dev]) return;
  init_pdhg_attributes();
  init_lanczos_attributes();
  init_factored_attributes();
  init_mv_tc_attributes();
  done[dev] = true;
}

Solver::~Solver() { free_all(); }

void Solver::free_all() {
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  graphs.clear();
  for (void* p : allocs) cudaFree(p);
  allocs.clear();
  dev_bytes = 0;
  if (ctl_host) cudaFreeHost(ctl_host);
  ctl_host = nullptr;
  if (st_aux) cudaStreamDestroy(st_aux);
  st_aux = nullptr;
  if (own_stream && st) cudaStreamDestroy(st);
  st = nullptr;
  own_stream = false;
}

// Device allocation owned by the handle.  With settings.memory_limit_bytes > 0
// the handle's allocations are capped at that many bytes in total (an
// allocation beyond the cap fails as if the device were out of memory).
template <class T>
static cudaError_t dalloc(Solver& sv, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (sv.set.memory_limit_bytes > 0 && (int64_t)(sv.dev_bytes + bytes) > sv.set.memory_limit_bytes)
    return cudaErrorMemoryAllocation;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return e;
  sv.allocs.push_back(q);
  sv.dev_bytes += bytes;
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

template <class T>
static cudaError_t dupload(Solver& sv, const T** p, const std::vector<T>& v, cudaStream_t st) {
  T* q = nullptr;
  cudaError_t e = dalloc(sv, &q, v.size());
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpyAsync(q, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
  *p = q;
  return e;
}

#define CKA(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ == cudaErrorMemoryAllocation) return fail(PROXSDP_ERR_OOM, "device allocation failed"); \
    if (e_ != cudaSuccess) return fail(PROXSDP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int Solver::upload(const HostProblem& h, bool alloc_S) {
  // release a previous problem
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  graphs.clear();
  for (void* p : allocs) cudaFree(p);
  allocs.clear();
  dev_bytes = 0;
  has_problem = false;
  has_iterate = false;
  hp = h;
  box_u = 0.0;
  const int n = h.n;
  DevProblem& P = pb;
  P = DevProblem{};
  P.n = n;
  P.m = h.m;
  P.m_eq = h.m_eq;
  P.nnz_ext = (int)h.ent_p.size();
  CKA(dupload(*this, &P.ent_p, h.ent_p, st));
  CKA(dupload(*this, &P.ent_q, h.ent_q, st));
  CKA(dupload(*this, &P.ent_a, h.ent_a, st));
  P.n_chunks = (int)h.chunk_beg.size();
  CKA(dupload(*this, &P.chunk_beg, h.chunk_beg, st));
  CKA(dupload(*this, &P.chunk_end, h.chunk_end, st));
  CKA(dupload(*this, &P.row_chunk, h.row_chunk, st));
  CKA(dupload(*this, &P.chunk_row, h.chunk_row, st));
  P.n_multi = (int)h.multi_rows.size();
  CKA(dupload(*this, &P.multi_rows, h.multi_rows, st));
  CKA(dupload(*this, &P.rhs, h.rhs, st));
  P.n_dense = (int)h.dense_row.size();
  CKA(dupload(*this, &P.dense_row, h.dense_row, st));
  CKA(dupload(*this, &P.dense_a, h.dense_a, st));
  CKA(dupload(*this, &P.dense_of_row, h.dense_of_row, st));
  P.nU = (int)h.u_p.size();
  CKA(dupload(*this, &P.u_p, h.u_p, st));
  CKA(dupload(*this, &P.u_q, h.u_q, st));
  CKA(dupload(*this, &P.u_c, h.u_c, st));
  CKA(dupload(*this, &P.u_ptr, h.u_ptr, st));
  CKA(dupload(*this, &P.u_row, h.u_row, st));
  CKA(dupload(*this, &P.u_a, h.u_a, st));
  P.ntile = h.ntile;
  CKA(dupload(*this, &P.tile_ptr, h.tile_ptr, st));
  CKA(dupload(*this, &P.tile_loc, h.tile_loc, st));
  CKA(dupload(*this, &P.tile_u, h.tile_u, st));
  P.alpha = h.alpha;
  P.normC = h.normC;
  P.normRhs = h.normRhs;
  P.C_dense = nullptr;
  // operator form of S^k: the factored one needs the Lanczos path and the
  // row structure of the union pattern
  const bool lanczos_path = !(n <= kFullEigMax || set.full_eig);
  const int64_t nsym = (int64_t)h.sym_col.size();
  factored = lanczos_path && !h.sym_ptr.empty() &&
             (set.operator_form == PROXSDP_OP_FACTORED ||
              (set.operator_form == PROXSDP_OP_AUTO && 8 * nsym <= (int64_t)n * n));
  if (factored) {
    alloc_S = false;
    P.nsym = (int)nsym;
    CKA(dupload(*this, &P.sym_ptr, h.sym_ptr, st));
    CKA(dupload(*this, &P.sym_col, h.sym_col, st));
    CKA(dupload(*this, &P.u_pos, h.u_pos, st));
  }

  DevWork& Wk = wk;
  Wk = DevWork{};
  const int ld = (n + 31) / 32 * 32;
  Wk.lds = ld;
  Wk.ldq = ld;
  Wk.ldv = kMaxR;
  if (alloc_S) CKA(dalloc(*this, &Wk.S, (size_t)n * ld));
  CKA(dalloc(*this, &Wk.Q, (size_t)ld * kMaxK));
  CKA(dalloc(*this, &Wk.W, (size_t)ld * kMaxK));
  for (int b = 0; b < 2; ++b) {
    CKA(dalloc(*this, &Wk.Vrm[b], (size_t)n * kMaxR));
    CKA(dalloc(*this, &Wk.lam[b], kMaxR));
    CKA(dalloc(*this, &Wk.colsum[b], kMaxR));
    CKA(dalloc(*this, &Wk.mx[b], (size_t)h.m + 1));
  }
  CKA(dalloc(*this, &Wk.y, (size_t)h.m));
  CKA(dalloc(*this, &Wk.dy, (size_t)h.m));
  CKA(dalloc(*this, &Wk.chunk_part, std::max<size_t>(h.chunk_beg.size(), 1)));
  CKA(dalloc(*this, &Wk.D, std::max<size_t>(h.u_p.size(), 1)));
  CKA(dalloc(*this, &Wk.dshift, 4));
  CKA(dalloc(*this, &Wk.part, (size_t)1 << 20));
  CKA(dalloc(*this, &Wk.H, (size_t)kMaxK * kMaxK));
  CKA(dalloc(*this, &Wk.Hf, (size_t)kMaxW * kMaxW));
  CKA(dalloc(*this, &Wk.flags, kMaxW));
  CKA(dalloc(*this, &Wk.Y, (size_t)kMaxK * kMaxK));
  CKA(dalloc(*this, &Wk.theta, kMaxK));
  CKA(dalloc(*this, &Wk.ritz_part, ((size_t)(n + 31) / 32 + 1) * 4 * kMaxP));
  CKA(dalloc(*this, &Wk.counters, (size_t)CNT_NUM * 512));
  CKA(dalloc(*this, &Wk.ctl, 1));
  CKA(dalloc(*this, &Vcm, (size_t)ld * 2 * kMaxR));
  CKA(dalloc(*this, &Hx, (size_t)4 * kMaxR * kMaxR));
  Wk.Vcm = Vcm;
  Wk.Hx = Hx;
  if (factored) {
    CKA(dalloc(*this, &Wk.Dsym, (size_t)nsym));
    CKA(dalloc(*this, &Wk.Qr, (size_t)n * kMaxW));
    CKA(dalloc(*this, &Wk.lrP, (size_t)64 * kMaxW));
    CK(cudaMemsetAsync(Wk.Dsym, 0, sizeof(float) * std::max<size_t>((size_t)nsym, 1), st));
  }
  CKA(dalloc(*this, &saved_V, (size_t)n * kMaxR));
  CKA(dalloc(*this, &saved_lam, kMaxR));
  CKA(dalloc(*this, &saved_y, (size_t)h.m));
  saved_r = 0;
  saved_it = -1;
  saved_seen = 0;
  CKA(dalloc(*this, &Wk.mv_part, block_matvec_scratch_floats(n, kMaxP)));  // the warm product has up to kMaxP columns
  CKA(dalloc(*this, &Wk.mv_cnt, block_matvec_counters(n, kMaxW)));
  CK(cudaMemsetAsync(Wk.mv_cnt, 0, sizeof(unsigned) * block_matvec_counters(n, kMaxW), st));
  CK(cudaMemsetAsync(Wk.counters, 0, sizeof(unsigned) * CNT_NUM * 512, st));
  CK(cudaMemsetAsync(Wk.Q, 0, sizeof(float) * (size_t)ld * kMaxK, st));
  CK(cudaMemsetAsync(Wk.W, 0, sizeof(float) * (size_t)ld * kMaxK, st));
  CK(cudaMemsetAsync(Vcm, 0, sizeof(float) * (size_t)ld * 2 * kMaxR, st));
  if (alloc_S) CK(cudaMemsetAsync(Wk.S, 0, sizeof(float) * (size_t)n * ld, st));
  CK(cudaStreamSynchronize(st));
  has_problem = true;
  return PROXSDP_OK;
}

void lanczos_dims(int rr, const proxsdp_gpu_settings& set, int k_target, int wmax, int& w, int& K, int& s) {
  const int b = std::max(1, set.block_size);
  const int g = set.guard > 0 ? set.guard : std::max(8, rr / 4);
  w = ((rr + g + b - 1) / b) * b;
  if (w > kMaxW && wmax > kMaxW) {
    // wide kept block: r + 8 vectors (or r + guard when set), at most kMaxP,
    // leaving the largest expansion of K - w <= kMaxW directions per cycle
    const int gw = set.guard > 0 ? set.guard : 8;
    w = std::min(((rr + gw + b - 1) / b) * b, kMaxP);
    s = 1;
    K = std::min(kMaxK, w + kMaxW);
    return;
  }
  w = std::min(w, kMaxW);
  if (set.lanczos_steps > 0) s = set.lanczos_steps;
  else s = std::max(1, k_target / w - 1);
  while ((s + 1) * w > kMaxK && s > 1) --s;
  K = (s + 1) * w;
}

int Solver::rank_cap() const {
  const int n = hp.n;
  if (set.full_eig) return n;
  if (n <= kFullEigMax) return std::min(set.max_rank, n);
  return std::min(std::min(set.max_rank, n), factored ? kMaxRankFactored : kMaxRankLanczos);
}

// Krylov block width w, Rayleigh-Ritz basis K = (s+1) w and steps s for rank r.
void Solver::dims(int rr, int& w, int& K, int& s) const {
  const int n = hp.n;
  if (n <= kFullEigMax || set.full_eig) {
    w = n;
    K = n;
    s = 0;
    return;
  }
  lanczos_dims(rr, set, k_target, factored ? kMaxW : kMaxP, w, K, s);
}

int Solver::set_ctl_fields(int status, int it_stop, int rr, int w, int K, int k_change) {
  launch_ctl_set(wk.ctl, status, it_stop, rr, w, K, k_change, st);
  CK(cudaGetLastError());
  return PROXSDP_OK;
}

// Orthonormalise Z = Q[:, c0:c0+w] against Q[:, :c0] and within itself:
// two passes of (classical Gram-Schmidt, Cholesky QR); columns found
// dependent in the first pass are refilled with pseudo-random vectors.
void enqueue_orth(const DevWork& wk, int n, int c0, int w, unsigned long long seed,
                  const int* skip, cudaStream_t st, const float* src) {
  float* Z = wk.Q + (size_t)c0 * wk.ldq;
  if (orth_cluster_applies(n, c0, w)) {  // the whole orthogonalisation in one cluster launch
    launch_orth_cluster(wk.Q, wk.ldq, src ? src : Z, n, c0, w, 2, 1, seed, skip, st);
    dbg(wk, "orth cluster", st);
    return;
  }
  if (src) launch_copy_cols(src, wk.ldq, Z, wk.ldq, n, w, skip, st);
  unsigned* cnt = wk.counters + CNT_GRAM * 512;
  for (int pass = 0; pass < 2; ++pass) {
    if (c0 > 0) {
      launch_gram(wk.Q, wk.ldq, c0, Z, wk.ldq, w, n, wk.H, wk.part, cnt, skip, st);
      dbg(wk, "orth gram QtZ", st);
      launch_block_update(Z, wk.ldq, w, wk.Q, wk.ldq, c0, wk.H, n, skip, st);
      dbg(wk, "orth update", st);
    }
    launch_gram(Z, wk.ldq, w, Z, wk.ldq, w, n, wk.H, wk.part, cnt, skip, st);
    dbg(wk, "orth gram ZtZ", st);
    launch_chol_inv(wk.H, w, wk.Hf, wk.flags, skip, st);
    dbg(wk, "orth chol", st);
    launch_apply_rinv(Z, wk.ldq, w, wk.Hf, wk.flags, n, seed * 131ULL + (unsigned long long)(pass * 7 + c0),
                      skip, st);
    dbg(wk, "orth apply", st);
  }
}

// Kernels enqueue_orth launches for Q[:, c0:c0+w] (with a source to copy from or not).
static int orth_kernel_count(int n, int c0, int w, bool src) {
  if (orth_cluster_applies(n, c0, w)) return 1;
  return (src ? 1 : 0) + 2 * ((c0 > 0 ? 2 : 0) + 3);
}

// enqueue_orth for blocks wider than kMaxW: pieces of at most kMaxW columns,
// each orthogonalised against everything before it.
static void enqueue_orth_wide(const DevWork& wk, int n, int c0, int w, unsigned long long seed, const int* skip,
                              cudaStream_t st) {
  for (int off = 0; off < w; off += kMaxW)
    enqueue_orth(wk, n, c0 + off, std::min(kMaxW, w - off), seed + (unsigned long long)off, skip, st);
}

static int cholqr_kernel_count(int n, int w);

// One Cholesky-QR pass on Q[:, c0:c0+w] (re-orthonormalises the kept Ritz
// block); a block wider than kMaxW is re-orthonormalised piece by piece.
static void enqueue_cholqr(const DevWork& wk, int n, int c0, int w, unsigned long long seed, cudaStream_t st) {
  if (w > kMaxW) {
    enqueue_cholqr(wk, n, c0, kMaxW, seed, st);
    for (int off = kMaxW; off < w; off += kMaxW)
      enqueue_orth(wk, n, c0 + off, std::min(kMaxW, w - off), seed + (unsigned long long)off, nullptr, st);
    return;
  }
  float* Z = wk.Q + (size_t)c0 * wk.ldq;
  if (orth_cluster_applies(n, c0, w)) {
    launch_orth_cluster(wk.Q, wk.ldq, Z, n, c0, w, 1, 0, seed, nullptr, st);
    return;
  }
  unsigned* cnt = wk.counters + CNT_GRAM * 512;
  launch_gram(Z, wk.ldq, w, Z, wk.ldq, w, n, wk.H, wk.part, cnt, nullptr, st);
  launch_chol_inv(wk.H, w, wk.Hf, wk.flags, nullptr, st);
  launch_apply_rinv(Z, wk.ldq, w, wk.Hf, wk.flags, n, seed, nullptr, st);
}

static int cholqr_kernel_count(int n, int w) {
  if (w <= kMaxW) return orth_cluster_applies(n, 0, w) ? 1 : 3;
  int c = cholqr_kernel_count(n, kMaxW);
  for (int off = kMaxW; off < w; off += kMaxW) c += orth_kernel_count(n, off, std::min(kMaxW, w - off), false);
  return c;
}

void enqueue_cycle(const DevWork& wk, int n, int w, int K, int s, int r,
                   unsigned long long seed, cudaGraphConditionalHandle cond, int use_cond,
                   cudaStream_t st, const DevProblem* fac) {
  const int* skip = &wk.ctl->lz_done;
  if (w > kMaxW) {
    // wide kept block: one expansion by bx = K - w residual directions of a
    // window of the kept vectors that rotates with the cycles
    // (k_compress_block), orthogonalised in place
    const int bx = K - w;
    float* Z = wk.Q + (size_t)w * wk.ldq;
    float* W1 = wk.W + (size_t)w * wk.ldq;
    launch_compress_block(wk.W, wk.ldq, w, Z, wk.ldq, bx, n, wk.ctl, skip, st);
    enqueue_orth(wk, n, w, bx, seed + 1ULL, skip, st);
    if (fac) launch_factored_matvec(*fac, wk, Z, wk.ldq, W1, wk.ldq, bx, skip, st);
    else launch_block_matvec(wk.S, wk.lds, n, Z, wk.ldq, W1, wk.ldq, bx, skip, st, wk.mv_part, wk.mv_cnt);
    dbg(wk, "wide cycle matvec", st);
    launch_gram(wk.Q, wk.ldq, K, wk.W, wk.ldq, K, n, wk.H, wk.part, wk.counters + CNT_GRAM * 512, skip, st);
    launch_sym_eig(wk.H, K, wk.theta, wk.Y, kMaxK, w, skip, st, 1, &wk.ctl->lz_tol);
    const int launches = 4 + orth_kernel_count(n, w, bx, false) +
                         (fac ? kFactoredLaunches : block_matvec_kernels(wk.S, wk.lds, n, wk.mv_part));
    launch_ritz(wk, n, K, w, r, 1, launches, cond, use_cond, st);
    dbg(wk, "ritz", st);
    return;
  }
  for (int j = 1; j <= s; ++j) {
    enqueue_orth(wk, n, j * w, w, seed + (unsigned long long)j, skip, st, wk.W + (size_t)(j - 1) * w * wk.ldq);
    const float* Qj = wk.Q + (size_t)j * w * wk.ldq;
    float* Wj = wk.W + (size_t)j * w * wk.ldq;
    if (fac) launch_factored_matvec(*fac, wk, Qj, wk.ldq, Wj, wk.ldq, w, skip, st);
    else launch_block_matvec(wk.S, wk.lds, n, Qj, wk.ldq, Wj, wk.ldq, w, skip, st, wk.mv_part, wk.mv_cnt);
    dbg(wk, "cycle matvec", st);
  }
  launch_gram(wk.Q, wk.ldq, K, wk.W, wk.ldq, K, n, wk.H, wk.part, wk.counters + CNT_GRAM * 512, skip, st);
  dbg(wk, "rr gram T", st);
  launch_sym_eig(wk.H, K, wk.theta, wk.Y, kMaxK, w, skip, st, 1, &wk.ctl->lz_tol);
  dbg(wk, "rr eig", st);
  // Gram of T, eigensolver, Ritz; the products
  int cycle_launches = 3 + s * (fac ? kFactoredLaunches : block_matvec_kernels(wk.S, wk.lds, n, wk.mv_part));
  for (int j = 1; j <= s; ++j) cycle_launches += orth_kernel_count(n, j * w, w, true);
  launch_ritz(wk, n, K, w, r, s, cycle_launches, cond, use_cond, st);
  dbg(wk, "ritz", st);
}

// Enqueue one iteration on `st` (direct launches or inside a capture).
int Solver::enqueue_iteration(const GraphKey& k, bool in_graph, cudaGraphConditionalHandle outer,
                              cudaGraphConditionalHandle inner) {
  const int n = hp.n;
  const int use = in_graph ? 1 : 0;
  if (k.full) {
    launch_s_to_t(wk.S, wk.lds, n, wk.H, st);
    launch_sym_eig(wk.H, n, wk.theta, wk.Y, kMaxK, n, nullptr, st, 1, &wk.ctl->lz_tol);
    launch_full_eig_factors(wk, n, st);
  } else {
    if (g_debug) g_debug_n = n;
    enqueue_cholqr(wk, n, 0, k.w, seed + 17, st);
    if (factored)  // the factored form keeps w <= kMaxW (rank cap)
      launch_factored_matvec(pb, wk, wk.Q, wk.ldq, wk.W, wk.ldq, k.w, nullptr, st, inner, use);
    else
      launch_block_matvec(wk.S, wk.lds, n, wk.Q, wk.ldq, wk.W, wk.ldq, k.w, nullptr, st, wk.mv_part, wk.mv_cnt,
                          inner, use);
    dbg(wk, "warm matvec", st);
    if (in_graph) {
      cudaStreamCaptureStatus cs;
      cudaGraph_t g;
      const cudaGraphNode_t* deps = nullptr;
      const cudaGraphEdgeData* ed = nullptr;
      size_t nd = 0;
      CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
      cudaGraphNodeParams p = {};
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = inner;
      p.conditional.type = cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      cudaGraphNode_t node;
      CK(cudaGraphAddNode(&node, g, deps, ed, nd, &p));
      CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
      cudaGraph_t body = p.conditional.phGraph_out[0];
      CK(cudaStreamBeginCaptureToGraph(st_aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      enqueue_cycle(wk, n, k.w, k.K, k.s, k.r, seed, inner, 1, st_aux, factored ? &pb : nullptr);
      CK(cudaStreamEndCapture(st_aux, &body));
    } else {
      // direct launches: the same kernels as the graph body, with the host
      // reading the projection's convergence flag after every restart cycle
      for (int c = 0; c < std::max(1, set.lanczos_max_cycles); ++c) {
        enqueue_cycle(wk, n, k.w, k.K, k.s, k.r, seed, inner, 0, st, factored ? &pb : nullptr);
        int done = 0;
        CK(cudaMemcpyAsync(&ctl_host->lz_done, &wk.ctl->lz_done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        done = ctl_host->lz_done;
        if (done) break;
      }
    }
  }
  dbg(wk, "projection", st);
  launch_mxdual(pb, wk, k.r, st);
  launch_dvals(pb, wk, st);
  if (pb.box) launch_box_dual(pb, wk, k.r, st);
  dbg(wk, "mxdual/dvals", st);
  const int act = std::min(kMaxR, ((k.r + 15) / 16) * 16);
  // kernels per iteration outside the restart cycles: Cholesky-QR, the warm
  // product, M(X)/dual step, D values, Gram + controller, the rebuild of S
  const int iter_launches = (k.full ? 7
                                    : cholqr_kernel_count(n, k.w) +
                                          (factored ? kFactoredLaunches + 3
                                                    : 4 + block_matvec_kernels(wk.S, wk.lds, n, wk.mv_part))) +
                            (pb.box ? 1 : 0);
  launch_gram_control(pb, wk, act, iter_launches, outer, use, st);
  dbg(wk, "gram+control", st);
  if (!factored) {
    launch_rebuild(pb, wk, k.r, 0, st);
    dbg(wk, "rebuild", st);
  }
  CK(cudaGetLastError());
  return PROXSDP_OK;
}

int Solver::get_graph(const GraphKey& k, cudaGraphExec_t* out) {
  auto it = graphs.find(k);
  if (it != graphs.end()) {
    *out = it->second;
    return PROXSDP_OK;
  }
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle outer, inner = 0;
  CK(cudaGraphConditionalHandleCreate(&outer, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = outer;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  if (!k.full) CK(cudaGraphConditionalHandleCreate(&inner, body, 1, cudaGraphCondAssignDefault));
  CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int rc = enqueue_iteration(k, true, outer, inner);
  cudaGraph_t body2;
  cudaError_t ce = cudaStreamEndCapture(st, &body2);
  if (rc != PROXSDP_OK) {
    cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(PROXSDP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  }
  cudaGraphExec_t ex;
  cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return fail(PROXSDP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
  graphs[k] = ex;
  *out = ex;
  return PROXSDP_OK;
}

int Solver::read_ctl() {
  CK(cudaMemcpyAsync(ctl_host, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PROXSDP_OK;
}

// X = 0, y = 0: S^0 = -alpha C; random orthonormal start block.
int Solver::init_iterate_zero() {
  const int n = hp.n;
  CK(cudaMemsetAsync(wk.y, 0, sizeof(double) * std::max(hp.m, 1), st));
  if (pb.box) {
    CK(cudaMemsetAsync(wk.ybp, 0, sizeof(float) * (size_t)n * wk.lds, st));
    CK(cudaMemsetAsync(wk.ybm, 0, sizeof(float) * (size_t)n * wk.lds, st));
  }
  CK(cudaMemsetAsync(wk.dy, 0, sizeof(double) * std::max(hp.m, 1), st));
  for (int b = 0; b < 2; ++b) {
    CK(cudaMemsetAsync(wk.Vrm[b], 0, sizeof(float) * (size_t)n * kMaxR, st));
    CK(cudaMemsetAsync(wk.lam[b], 0, sizeof(double) * kMaxR, st));
    CK(cudaMemsetAsync(wk.colsum[b], 0, sizeof(double) * kMaxR, st));
    CK(cudaMemsetAsync(wk.mx[b], 0, sizeof(double) * (hp.m + 1), st));
  }
  CK(cudaMemsetAsync(Vcm, 0, sizeof(float) * (size_t)wk.ldq * 2 * kMaxR, st));
  rank_changes = 0;
  saved_r = 0;
  saved_it = -1;
  saved_seen = 0;
  r = std::max(1, std::min(set.full_eig ? n : set.rank_init, n));
  if (!set.full_eig) r = std::min(r, rank_cap());
  int w, K, s;
  dims(r, w, K, s);
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.par = 0;
  c.r = r;
  c.r_old = r;
  c.w = w;
  c.K = K;
  c.status = ST_RUNNING;
  c.full_eig = set.full_eig ? 1 : 0;
  c.full_eig_path = (n <= kFullEigMax || set.full_eig) ? 1 : 0;
  c.window = std::max(1, std::min(set.window, kMaxWindow));
  c.max_rank = rank_cap();
  c.at_max_rank = set.at_max_rank ? 1 : 0;
  c.max_cycles = std::max(1, set.lanczos_max_cycles);
  c.tol = set.tol;
  c.eps_lambda = set.eps_lambda > 0 ? set.eps_lambda : set.tol;
  c.lz_tol_fixed = set.lanczos_tol;
  c.lz_tol = set.lanczos_tol > 0 ? set.lanczos_tol : 1e-3;
  for (int i = 0; i < kMaxWindow; ++i) c.hist[i] = INFINITY;
  std::memcpy(ctl_host, &c, sizeof(Ctl));
  CK(cudaMemcpyAsync(wk.ctl, ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, st));
  // D = C (y = 0), S^0 = -alpha C
  launch_dvals(pb, wk, st);
  if (!factored) launch_rebuild(pb, wk, 1, 0, st);
  if (!(n <= kFullEigMax || set.full_eig)) {
    launch_random_block(wk.Q, wk.ldq, n, 0, w, seed, st);
    enqueue_orth_wide(wk, n, 0, w, seed, nullptr, st);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  has_iterate = true;
  return PROXSDP_OK;
}

// Element-wise box -u <= X_pq <= u for all p != q (Sec. 5.3) as a structured
// class of n (n - 1) inequality rows: A = +-(E_pq + E_qp) / 2, rhs u, scaled
// by s = sqrt(2) to unit Frobenius norm when rows are normalised.  Supported
// when every other row acts on the diagonal only: the two parts of M*M then
// act on orthogonal subspaces (diagonal / off-diagonal), so
// ||M||^2 = max(||M_rows||^2, s^2), and the box part of M*(y) never meets
// the other rows' part.
int Solver::set_box(double u) {
  if (!has_problem) return fail(PROXSDP_ERR_BAD_STATE, "set_box before set_problem");
  if (!(u > 0.0) || !std::isfinite(u)) return fail(PROXSDP_ERR_INVALID_ARG, "box bound must be positive and finite");
  if (factored) return fail(PROXSDP_ERR_UNSUPPORTED, "the element-wise box needs the explicit operator form");
  if (!hp.dense_row.empty()) return fail(PROXSDP_ERR_UNSUPPORTED, "the element-wise box with a dense (11^T) row");
  for (int row = 0; row < hp.m; ++row)
    for (int c = hp.row_chunk[row]; c < hp.row_chunk[row + 1]; ++c)
      for (int e = hp.chunk_beg[c]; e < hp.chunk_end[c]; ++e)
        if (hp.ent_p[e] != hp.ent_q[e])
          return fail(PROXSDP_ERR_UNSUPPORTED, "the element-wise box with rows off the diagonal (give them as rows)");
  const int n = hp.n;
  if (!pb.box) {
    CKA(dalloc(*this, &wk.ybp, (size_t)n * wk.lds));
    CKA(dalloc(*this, &wk.ybm, (size_t)n * wk.lds));
  }
  const double s = set.normalize_rows ? std::sqrt(2.0) : 1.0;
  // row-only norms are kept in hp; the box adds its n (n - 1) rows
  const double nr2 = hp.normRhs * hp.normRhs + (double)n * (double)(n - 1) * (s * u) * (s * u);
  const double nm = std::max(hp.normM, s);
  pb.box = 1;
  pb.box_s = (float)s;
  pb.box_u = (float)u;
  pb.normRhs = std::sqrt(nr2);
  pb.alpha = (set.alpha_frac > 0.0 ? set.alpha_frac : 0.95) / nm;
  box_u = u;
  box_normM = nm;
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);  // they hold the problem by value
  graphs.clear();
  has_iterate = false;
  CK(cudaMemsetAsync(wk.ybp, 0, sizeof(float) * (size_t)n * wk.lds, st));
  CK(cudaMemsetAsync(wk.ybm, 0, sizeof(float) * (size_t)n * wk.lds, st));
  CK(cudaStreamSynchronize(st));
  return PROXSDP_OK;
}

// Grow the Krylov block from w_old to w_new columns: new columns are random
// vectors orthogonalised against the current Ritz vectors.
int Solver::grow_basis(int w_old, int w_new) {
  if (w_new <= w_old || hp.n <= kFullEigMax || set.full_eig) return PROXSDP_OK;
  launch_random_block(wk.Q, wk.ldq, hp.n, w_old, w_new - w_old, seed + 31ULL * (unsigned long long)w_new, st);
  enqueue_orth_wide(wk, hp.n, w_old, w_new - w_old, seed + 7ULL * (unsigned long long)w_new, nullptr, st);
  CK(cudaGetLastError());
  return PROXSDP_OK;
}

// Alg. 2 saves the feasible pair (X_[r], y_[r]) when the inner loop has
// converged at a rank the rank test finds insufficient; the controller counts
// such iterations in Ctl::saved and ends the graph there (the rank change or
// the stall at the rank cap goes back to the host), so the current iterate
// (Ctl::par, rank Ctl::r_old) is the pair to keep.
int Solver::keep_saved_pair() {
  const Ctl& c = *ctl_host;
  if (c.saved <= saved_seen || !saved_V) return PROXSDP_OK;
  saved_seen = c.saved;
  const int n = hp.n;
  CK(cudaMemcpyAsync(saved_V, wk.Vrm[c.par], sizeof(float) * (size_t)n * kMaxR, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(saved_lam, wk.lam[c.par], sizeof(double) * kMaxR, cudaMemcpyDeviceToDevice, st));
  if (hp.m > 0) CK(cudaMemcpyAsync(saved_y, wk.y, sizeof(double) * hp.m, cudaMemcpyDeviceToDevice, st));
  saved_r = c.r_old;
  saved_it = c.it;
  return PROXSDP_OK;
}

// Run iterations until convergence / a cap.  iters_cap < 0: no cap beyond
// max_iter.  With stop_on_converge == false exactly iters_cap iterations run
// (the rank rule still acts).
int Solver::run(int64_t iters_cap, bool stop_on_converge, proxsdp_gpu_info* info) {
  if (!has_problem) return fail(PROXSDP_ERR_BAD_STATE, "no problem loaded");
  const int n = hp.n;
  const auto t0 = std::chrono::steady_clock::now();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  CK(cudaMemcpyAsync(ctl_host, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int it0 = ctl_host->it;
  int64_t limit = set.max_iter;
  if (iters_cap >= 0) limit = std::min<int64_t>(limit, it0 + iters_cap);
  int final_status = ST_MAX_ITER;
  const bool graphs_on = set.use_graphs != 0;
  for (;;) {
    int it = ctl_host->it;
    if (it >= limit) {
      final_status = ST_MAX_ITER;
      break;
    }
    double elapsed = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (set.time_limit_s > 0 && elapsed > set.time_limit_s) {
      final_status = ST_TIME_LIMIT;
      break;
    }
    int w, K, s;
    dims(r, w, K, s);
    GraphKey key{r, w, K, s, (n <= kFullEigMax || set.full_eig) ? 1 : 0};
    int chunk = std::max(1, set.check_every);
    int it_stop = (int)std::min<int64_t>(limit, (int64_t)it + chunk);
    int rc = set_ctl_fields(ST_RUNNING, it_stop, r, w, K, -1);
    if (rc) return rc;
    if (graphs_on) {
      cudaGraphExec_t ex;
      rc = get_graph(key, &ex);
      if (rc) return rc;
      CK(cudaGraphLaunch(ex, st));
      rc = read_ctl();
      if (rc) return rc;
    } else {
      for (int i = it; i < it_stop; ++i) {
        rc = enqueue_iteration(key, false, 0, 0);
        if (rc) return rc;
        rc = read_ctl();
        if (rc) return rc;
        if (ctl_host->status != ST_RUNNING) break;
      }
    }
    const int status = ctl_host->status;
    if (status == ST_RUNNING || status == ST_PAUSE) continue;
    if (status == ST_RANK_CHANGE || status == ST_STALLED_MAX_RANK) {
      rc = keep_saved_pair();
      if (rc) return rc;
    }
    if (status == ST_CONVERGED) {
      final_status = ST_CONVERGED;
      if (stop_on_converge) break;
      continue;
    }
    if (status == ST_RANK_CHANGE) {
      int r_new = std::min(2 * r, std::max(rank_cap(), 1));
      int w_old = w;
      r = r_new;
      int w2, K2, s2;
      dims(r, w2, K2, s2);
      rc = grow_basis(w_old, w2);
      if (rc) return rc;
      rc = set_ctl_fields(ST_RUNNING, it_stop, r, w2, K2, ctl_host->it);
      if (rc) return rc;
      rank_changes += 1;
      continue;
    }
    final_status = status;  // STALLED_AT_MAX_RANK / NUMERIC
    break;
  }
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc = read_ctl();
  if (rc) return rc;
  if (info) {
    const Ctl& c = *ctl_host;
    std::memset(info, 0, sizeof(*info));
    info->status = final_status;
    info->final_rank = r;
    info->iters = c.it;
    info->rank_changes = rank_changes;
    info->primal_obj = c.pobj;
    info->dual_obj = c.dobj;
    info->rel_primal_res = c.rel_p;
    info->rel_dual_res = c.rel_d;
    info->rel_gap = c.rel_gap;
    info->eps_primal = c.eps_p;
    info->eps_dual = c.eps_d;
    info->lambda_r = c.lam_r;
    info->solve_seconds = ms * 1e-3;
    info->matvecs = c.matvecs;
    info->lanczos_cycles = c.lz_cycles_total;
    info->lanczos_unconverged = c.lz_unconverged;
    info->alpha = pb.alpha;  // with a box: the step of the extended operator
    info->norm_M = pb.box ? box_normM : hp.normM;
    info->kernel_launches = c.launches;
  }
  return PROXSDP_OK;
}

// Start the iteration from X = V diag(max(lambda,0)) V^T, y (paper's sign,
// original row scaling).
int Solver::set_iterate(int rr, const double* V, const double* lam, const double* y) {
  const int n = hp.n, m = hp.m;
  int rc = init_iterate_zero();
  if (rc) return rc;
  r = rr;
  int w, K, s;
  dims(r, w, K, s);
  std::vector<float> vrm((size_t)n * kMaxR, 0.f), vcm((size_t)wk.ldq * kMaxR, 0.f);
  std::vector<double> l(kMaxR, 0.0), cs(kMaxR, 0.0);
  for (int t = 0; t < rr; ++t) {
    l[t] = lam[t];
    for (int i = 0; i < n; ++i) {
      float v = (float)V[(size_t)t * n + i];
      vrm[(size_t)i * kMaxR + t] = v;
      vcm[(size_t)t * wk.ldq + i] = v;
      cs[t] += (double)v;
    }
  }
  // M_ext(X) of the given iterate, from the stored (FP32) factors
  std::vector<double> mx(m + 1, 0.0);
  for (int row = 0; row <= m; ++row) {
    for (int c = hp.row_chunk[row]; c < hp.row_chunk[row + 1]; ++c)
      for (int e = hp.chunk_beg[c]; e < hp.chunk_end[c]; ++e) {
        const int p = hp.ent_p[e], q = hp.ent_q[e];
        double x = 0.0;
        for (int t = 0; t < rr; ++t)
          x += std::max(l[t], 0.0) * (double)vrm[(size_t)p * kMaxR + t] * (double)vrm[(size_t)q * kMaxR + t];
        mx[row] += hp.ent_a[e] * x;
      }
    if (row < m && hp.dense_of_row[row] >= 0) {
      double sacc = 0.0;
      for (int t = 0; t < rr; ++t) sacc += std::max(l[t], 0.0) * cs[t] * cs[t];
      mx[row] += hp.dense_a[hp.dense_of_row[row]] * sacc;
    }
  }
  std::vector<double> ya(std::max(m, 1), 0.0);
  if (y)
    for (int i = 0; i < m; ++i) ya[i] = -y[i] / hp.scale[i];
  CK(cudaMemcpyAsync(wk.Vrm[0], vrm.data(), sizeof(float) * vrm.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(wk.lam[0], l.data(), sizeof(double) * kMaxR, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(wk.colsum[0], cs.data(), sizeof(double) * kMaxR, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(wk.mx[0], mx.data(), sizeof(double) * (m + 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(Vcm, vcm.data(), sizeof(float) * vcm.size(), cudaMemcpyHostToDevice, st));
  if (m > 0) CK(cudaMemcpyAsync(wk.y, ya.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(wk.dy, 0, sizeof(double) * std::max(m, 1), st));
  CK(cudaStreamSynchronize(st));
  // control block: current iterate in buffer 0 with rank rr
  Ctl* c = ctl_host;
  CK(cudaMemcpyAsync(c, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  c->par = 0;
  c->r = rr;
  c->r_old = rr;
  c->w = w;
  c->K = K;
  c->it = 0;
  c->k_change = 0;
  c->status = ST_RUNNING;
  c->max_rank = std::max(rank_cap(), rr);
  CK(cudaMemcpyAsync(wk.ctl, c, sizeof(Ctl), cudaMemcpyHostToDevice, st));
  // S^k = X^k - alpha (C + M*(y^k)), Lanczos warm start = the given factors
  launch_dvals(pb, wk, st);
  if (!factored) launch_rebuild(pb, wk, rr, 0, st);
  if (!(n <= kFullEigMax || set.full_eig)) {
    CK(cudaMemcpyAsync(wk.Q, vcm.data(), sizeof(float) * (size_t)wk.ldq * std::min(rr, w),
                       cudaMemcpyHostToDevice, st));
    if (w > rr) {
      launch_random_block(wk.Q, wk.ldq, n, rr, w - rr, seed + 5, st);
      enqueue_orth_wide(wk, n, rr, w - rr, seed + 9, nullptr, st);
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  has_iterate = true;
  return PROXSDP_OK;
}

// aproj(S, r) on caller memory: Lanczos (or the dense eigensolver for n <= 128) on S,
// then P = V diag(max(lambda,0)) V^T through the rebuild kernel.
int aproj_device(const float* S, int n, int lds, int r, float* P, int ldp, float* V, double* lambda,
                 const proxsdp_gpu_settings& set, cudaStream_t st_in, proxsdp_gpu_info* info,
                 std::string& err) {
  Solver sv;
  sv.k_target = kMaxK;  // cold start: the largest Rayleigh-Ritz basis
  sv.set = set;
  sv.set.full_eig = 0;
  sv.seed = set.seed ? set.seed : 1;
  sv.st = st_in;
  sv.own_stream = false;
  if (cudaStreamCreateWithFlags(&sv.st_aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&sv.ctl_host, sizeof(Ctl)) != cudaSuccess) {
    err = "stream / host allocation failed";
    return PROXSDP_ERR_CUDA;
  }
  HostProblem h;
  h.n = n;
  h.m = 0;
  h.m_eq = 0;
  h.row_chunk.assign(2, 0);
  h.dense_of_row.assign(1, -1);
  h.ntile = (n + kTile - 1) / kTile;
  h.tile_ptr.assign((size_t)h.ntile * h.ntile + 1, 0);
  h.u_ptr.assign(1, 0);
  h.alpha = 0.0;
  int rc = sv.upload(h, false);
  if (rc) {
    err = sv.err;
    return rc;
  }
  DevWork& wk = sv.wk;
  wk.S = const_cast<float*>(S);
  wk.lds = lds;
  const bool full = n <= kFullEigMax;
  sv.r = r;
  int w, K, s;
  sv.dims(r, w, K, s);
  if (!full && r > std::min(w - 4, kMaxRankLanczos)) {
    err = "rank too large for the Lanczos block (r <= 64)";
    return PROXSDP_ERR_UNSUPPORTED;
  }
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.par = 0;
  c.r = r;
  c.r_old = r;
  c.w = w;
  c.K = K;
  c.status = ST_RUNNING;
  c.max_cycles = std::max(1, set.lanczos_max_cycles);
  c.lz_tol_fixed = set.lanczos_tol > 0 ? set.lanczos_tol : 1e-6;
  c.lz_tol = c.lz_tol_fixed;
  std::memcpy(sv.ctl_host, &c, sizeof(Ctl));
  cudaError_t e = cudaMemcpyAsync(wk.ctl, sv.ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, sv.st);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  cudaMemsetAsync(wk.dshift, 0, 4 * sizeof(double), sv.st);
  if (full) {
    launch_s_to_t(S, lds, n, wk.H, sv.st);
    launch_sym_eig(wk.H, n, wk.theta, wk.Y, kMaxK, n, nullptr, sv.st);
    launch_full_eig_factors(wk, n, sv.st);
  } else {
    launch_random_block(wk.Q, wk.ldq, n, 0, w, sv.seed, sv.st);
    enqueue_orth_wide(wk, n, 0, w, sv.seed, nullptr, sv.st);
    launch_block_matvec(S, lds, n, wk.Q, wk.ldq, wk.W, wk.ldq, w, nullptr, sv.st, wk.mv_part, wk.mv_cnt);
    for (int cyc = 0; cyc < c.max_cycles; ++cyc)
      enqueue_cycle(wk, n, w, K, s, r, sv.seed + 1000ULL * (unsigned long long)(cyc + 1), 0, 0, sv.st);
  }
  if (P) {
    DevWork out = wk;
    out.S = P;
    out.lds = ldp;
    launch_rebuild(sv.pb, out, r, 1, sv.st);
  }
  if (V) {
    if (full) {
      e = cudaMemcpy2DAsync(V, sizeof(float) * n, wk.Y, sizeof(float) * kMaxK, sizeof(float) * n, r,
                            cudaMemcpyDeviceToDevice, sv.st);
    } else {
      e = cudaMemcpy2DAsync(V, sizeof(float) * n, wk.Q, sizeof(float) * wk.ldq, sizeof(float) * n, r,
                            cudaMemcpyDeviceToDevice, sv.st);
    }
    if (e != cudaSuccess) {
      err = cudaGetErrorString(e);
      return PROXSDP_ERR_CUDA;
    }
  }
  if (lambda) {
    e = cudaMemcpyAsync(lambda, wk.lam[1], sizeof(double) * r, cudaMemcpyDeviceToDevice, sv.st);
    if (e != cudaSuccess) {
      err = cudaGetErrorString(e);
      return PROXSDP_ERR_CUDA;
    }
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(sv.ctl_host, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, sv.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sv.st);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->final_rank = r;
    info->matvecs = full ? 0 : 1 + (int64_t)sv.ctl_host->lz_cycles_total * s;
    info->lanczos_cycles = sv.ctl_host->lz_cycles_total;
    info->lanczos_unconverged = sv.ctl_host->lz_unconverged;
    info->eps_primal = sv.ctl_host->lz_res;
    info->status = (sv.ctl_host->lz_done && sv.ctl_host->lz_unconverged == 0) ? PROXSDP_CONVERGED : PROXSDP_MAX_ITER;
  }
  sv.st = nullptr;  // caller's stream
  return PROXSDP_OK;
}

int sym_eig_device(const double* T, int K, double* theta, float* Y, cudaStream_t st) {
  launch_sym_eig(T, K, theta, Y, K, K, nullptr, st, 1);
  return cudaGetLastError() == cudaSuccess ? PROXSDP_OK : PROXSDP_ERR_CUDA;
}

}  // namespace psdp
