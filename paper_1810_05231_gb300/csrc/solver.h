// solver.h — host-side state of a proxsdp_gpu handle.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/proxsdp_gpu.h"
#include "psdp.cuh"

namespace psdp {

constexpr int kChunk = 128; // entries per M(X) work chunk

// Problem after validation, row scaling and the layout passes (host copy).
struct HostProblem {
  int n = 0, m = 0, m_eq = 0;
  std::vector<int> ent_p, ent_q;
  std::vector<double> ent_a;  // extended rows: constraints then the objective row
  std::vector<int> chunk_beg, chunk_end, row_chunk, chunk_row, multi_rows;
  std::vector<double> rhs, scale;
  std::vector<int> dense_row, dense_of_row;
  std::vector<double> dense_a;
  std::vector<int> u_p, u_q, u_ptr, u_row;
  std::vector<double> u_c, u_a;
  int ntile = 0;
  std::vector<int> tile_ptr, tile_loc, tile_u;
  std::vector<int> sym_ptr, sym_col, u_pos;
  double normM = 1.0, alpha = 0.0, normC = 0.0, normRhs = 0.0;
};

struct GraphKey {
  int r, w, K, s, full;
  bool operator<(const GraphKey& o) const {
    return std::tie(r, w, K, s, full) < std::tie(o.r, o.w, o.K, o.s, o.full);
  }
};

struct Solver {
  proxsdp_gpu_settings set{};
  int device = 0;
  cudaStream_t st = nullptr, st_aux = nullptr;
  bool own_stream = false;
  std::string err;
  bool has_problem = false;
  bool has_iterate = false;
  HostProblem hp;
  DevProblem pb{};
  DevWork wk{};
  float* Vcm = nullptr;  // column-major factor slots (2 * kMaxR columns)
  double* Hx = nullptr;  // Gram of the factor slots
  std::vector<void*> allocs;
  size_t dev_bytes = 0;  // bytes held in `allocs`
  Ctl* ctl_host = nullptr;  // pinned mirror
  std::map<GraphKey, cudaGraphExec_t> graphs;
  bool factored = false;  // S^k applied from the factors (never formed)
  int r = 8;
  int rank_changes = 0;
  // Alg. 2 "save feasible solution": the iterate at which the residuals met
  // tol while the rank test asked for r <- 2r (the last such pair of a solve)
  float* saved_V = nullptr;     // n x kMaxR row-major factors
  double* saved_lam = nullptr;  // kMaxR eigenvalues
  double* saved_y = nullptr;    // m dual (scaled problem, algorithm sign)
  int saved_r = 0;              // rank of the saved pair (0: none)
  int64_t saved_it = -1;        // its iteration
  int saved_seen = 0;           // Ctl::saved already copied
  int k_target = 32;  // Rayleigh-Ritz basis size aimed at by dims() (one Krylov step per cycle)
  unsigned long long seed = 1;

  ~Solver();
  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  int upload(const HostProblem& h, bool alloc_S = true);
  // element-wise box -u <= X_pq <= u (p != q) as a structured row class
  int set_box(double u);
  double box_u = 0.0;  // 0: no box
  double box_normM = 0.0;  // ||M||_2 of the rows with the box
  int init_iterate_zero();
  int set_iterate(int r, const double* V, const double* lam, const double* y);
  int run(int64_t iters_cap, bool stop_on_converge, proxsdp_gpu_info* info);
  int read_ctl();
  void dims(int r, int& w, int& K, int& s) const;
  // largest target rank of this handle: max_rank, n, and on the Lanczos path
  // kMaxRankLanczos (kMaxRankFactored with the factored operator)
  int rank_cap() const;
  int grow_basis(int w_old, int w_new);
  int enqueue_iteration(const GraphKey& k, bool in_graph, cudaGraphConditionalHandle outer,
                        cudaGraphConditionalHandle inner);
  int get_graph(const GraphKey& k, cudaGraphExec_t* out);
  int set_ctl_fields(int status, int it_stop, int r, int w, int K, int k_change);
  int keep_saved_pair();
  void free_all();
};

// Settings and device checks shared by the entry points (api.cpp):
// PROXSDP_ERR_INVALID_ARG / PROXSDP_ERR_CUDA with a message in `err`.
int check_settings(const proxsdp_gpu_settings& s, std::string& err);
int check_device(int device, std::string& err);

// Kept Ritz block w, Rayleigh-Ritz basis K and Krylov steps s per restart
// cycle for target rank r on the block Lanczos path (n > kFullEigMax):
// w = the smallest multiple of block_size holding r + guard vectors.  Up to
// kMaxW the kept block is also the Krylov block: s = k_target / w - 1 steps
// unless lanczos_steps fixes it, K = (s + 1) w <= kMaxK.  Beyond kMaxW (when
// wmax allows it) the kept block holds up to kMaxP vectors (at least r + 8)
// and one cycle expands it by K - w <= kMaxW directions, K <= kMaxK.
void lanczos_dims(int r, const proxsdp_gpu_settings& set, int k_target, int wmax, int& w, int& K, int& s);

// device helpers used by the API (solver.cu)
int aproj_device(const float* S, int n, int lds, int r, float* P, int ldp, float* V, double* lambda,
                 const proxsdp_gpu_settings& set, cudaStream_t st, proxsdp_gpu_info* info,
                 std::string& err);
int sym_eig_device(const double* T, int K, double* theta, float* Y, cudaStream_t st);
void init_kernel_attributes();
// Orthonormalise Q[:, c0:c0+w] (read from `src` when given) against Q[:, :c0]
// and within itself; one restart cycle of the block Krylov projection.
void enqueue_orth(const DevWork& wk, int n, int c0, int w, unsigned long long seed, const int* skip,
                  cudaStream_t st, const float* src = nullptr);
// With `fac` (the problem of a factored-operator solve) the block products
// apply S^k from the factors instead of reading wk.S.
void enqueue_cycle(const DevWork& wk, int n, int w, int K, int s, int r, unsigned long long seed,
                   cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st,
                   const DevProblem* fac = nullptr);

}  // namespace psdp
