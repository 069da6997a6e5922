// api.cpp — the extern "C" boundary (include/proxsdp_gpu.h): argument
// validation, the host-side layout passes of set_problem, and result export.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_set>
#include <vector>

#include "solver.h"

using psdp::HostProblem;
using psdp::Solver;

struct proxsdp_gpu_ctx {
  Solver s;
};

static std::string g_last_create_error;

namespace psdp {
// Error text for entry points that have no handle (read with proxsdp_gpu_last_error(NULL)).
void set_global_error(const std::string& msg) { g_last_create_error = msg; }
}  // namespace psdp

namespace {

bool finite(double v) { return std::isfinite(v); }

// (i, j), i <= j, of the packed upper-triangle index j(j+1)/2 + i.
void svec_unpack(int64_t idx, int* i, int* j) {
  int64_t jj = (int64_t)((std::sqrt(8.0 * (double)idx + 1.0) - 1.0) / 2.0);
  while (jj * (jj + 1) / 2 > idx) --jj;
  while ((jj + 1) * (jj + 2) / 2 <= idx) ++jj;
  *j = (int)jj;
  *i = (int)(idx - jj * (jj + 1) / 2);
}

struct Entry {
  int64_t key;  // svec index
  double a;
};

// Build the device layout of the problem (Sec. 1.3 data; rows scaled to unit
// Frobenius norm when requested).
int preprocess(const proxsdp_gpu_settings& set, int64_t n64, const double* C_dense, int64_t c_nnz,
               const int64_t* c_idx, const double* c_val, int64_t m64, int64_t meq64,
               const int64_t* A_rowptr, const int64_t* A_col, const double* A_val, const double* rhs,
               HostProblem& h, std::string& err) {
  if (n64 < 1 || n64 > 46340) {
    err = "n must be in [1, 46340]";
    return PROXSDP_ERR_INVALID_ARG;
  }
  if (m64 < 0 || meq64 < 0 || meq64 > m64 || m64 > (int64_t)1 << 30) {
    err = "need 0 <= m_eq <= m_total";
    return PROXSDP_ERR_INVALID_ARG;
  }
  const int n = (int)n64, m = (int)m64;
  const int64_t ntri = n64 * (n64 + 1) / 2;
  if (m > 0 && (!A_rowptr || !rhs)) {
    err = "A_rowptr and rhs are required when m_total > 0";
    return PROXSDP_ERR_INVALID_ARG;
  }
  if (m > 0 && A_rowptr[0] != 0) {
    err = "A_rowptr[0] must be 0";
    return PROXSDP_ERR_INVALID_ARG;
  }
  for (int i = 0; i < m; ++i)
    if (A_rowptr[i + 1] < A_rowptr[i]) {
      err = "A_rowptr must be non-decreasing";
      return PROXSDP_ERR_INVALID_ARG;
    }
  const int64_t nnz = m > 0 ? A_rowptr[m] : 0;
  if (nnz > 0 && (!A_col || !A_val)) {
    err = "A_col and A_val are required";
    return PROXSDP_ERR_INVALID_ARG;
  }
  if (nnz > ((int64_t)1 << 31) - 2) {
    err = "too many constraint entries";
    return PROXSDP_ERR_UNSUPPORTED;
  }
  for (int i = 0; i < m; ++i)
    if (!finite(rhs[i])) {
      err = "rhs has a non-finite value";
      return PROXSDP_ERR_INVALID_ARG;
    }
  h = HostProblem{};
  h.n = n;
  h.m = m;
  h.m_eq = (int)meq64;
  h.rhs.assign(m, 0.0);
  h.scale.assign(m, 1.0);
  h.dense_of_row.assign(std::max(m, 1), -1);
  // rows: sort, merge duplicates, classify
  std::vector<std::vector<Entry>> rows(m);
  for (int i = 0; i < m; ++i) {
    const int64_t b = A_rowptr[i], e = A_rowptr[i + 1];
    bool dense = false;
    for (int64_t k = b; k < e; ++k) {
      if (!finite(A_val[k])) {
        err = "A_val has a non-finite value";
        return PROXSDP_ERR_INVALID_ARG;
      }
      if (A_col[k] == -1) {
        if (e - b != 1) {
          err = "a dense row (column -1) must have exactly one entry";
          return PROXSDP_ERR_INVALID_ARG;
        }
        dense = true;
      } else if (A_col[k] < 0 || A_col[k] >= ntri) {
        err = "A_col index out of range (row " + std::to_string(i) + ")";
        return PROXSDP_ERR_INVALID_ARG;
      }
    }
    if (dense) {
      h.dense_of_row[i] = (int)h.dense_row.size();
      h.dense_row.push_back(i);
      h.dense_a.push_back(A_val[b]);
      continue;
    }
    std::vector<Entry> v;
    v.reserve(e - b);
    for (int64_t k = b; k < e; ++k) v.push_back({A_col[k], A_val[k]});
    std::sort(v.begin(), v.end(), [](const Entry& x, const Entry& y) { return x.key < y.key; });
    std::vector<Entry> u;
    for (const Entry& x : v) {
      if (!u.empty() && u.back().key == x.key) u.back().a += x.a;
      else u.push_back(x);
    }
    rows[i] = std::move(u);
  }
  // C entries
  std::vector<Entry> centries;
  if (C_dense) {
    for (int j = 0; j < n; ++j)
      for (int i = 0; i <= j; ++i) {
        double v = C_dense[(size_t)i * n + j];
        double v2 = C_dense[(size_t)j * n + i];
        if (!finite(v) || !finite(v2)) {
          err = "C has a non-finite value";
          return PROXSDP_ERR_INVALID_ARG;
        }
        if (v != v2) {
          err = "dense C must be symmetric";
          return PROXSDP_ERR_INVALID_ARG;
        }
        if (v != 0.0) centries.push_back({(int64_t)j * (j + 1) / 2 + i, v});
      }
  } else if (c_nnz > 0) {
    if (!c_idx || !c_val) {
      err = "c_idx and c_val are required when c_nnz > 0";
      return PROXSDP_ERR_INVALID_ARG;
    }
    std::vector<Entry> v;
    for (int64_t k = 0; k < c_nnz; ++k) {
      if (c_idx[k] < 0 || c_idx[k] >= ntri) {
        err = "c_idx out of range";
        return PROXSDP_ERR_INVALID_ARG;
      }
      if (!finite(c_val[k])) {
        err = "c_val has a non-finite value";
        return PROXSDP_ERR_INVALID_ARG;
      }
      v.push_back({c_idx[k], c_val[k]});
    }
    std::sort(v.begin(), v.end(), [](const Entry& x, const Entry& y) { return x.key < y.key; });
    for (const Entry& x : v) {
      if (!centries.empty() && centries.back().key == x.key) centries.back().a += x.a;
      else centries.push_back(x);
    }
  } else if (c_nnz < 0) {
    err = "c_nnz must be >= 0";
    return PROXSDP_ERR_INVALID_ARG;
  }
  // row scaling: ||A_i||_F = sqrt(sum_diag a^2 + 2 sum_off a^2), dense row |a| n
  for (int i = 0; i < m; ++i) {
    double sq = 0.0;
    if (h.dense_of_row[i] >= 0) {
      double a = h.dense_a[h.dense_of_row[i]];
      sq = a * a * (double)n * (double)n;
    } else {
      for (const Entry& x : rows[i]) {
        int p, q;
        svec_unpack(x.key, &p, &q);
        sq += (p == q ? 1.0 : 2.0) * x.a * x.a;
      }
    }
    double s = (set.normalize_rows && sq > 0.0) ? 1.0 / std::sqrt(sq) : 1.0;
    h.scale[i] = s;
    h.rhs[i] = rhs[i] * s;
  }
  for (size_t d = 0; d < h.dense_row.size(); ++d) h.dense_a[d] *= h.scale[h.dense_row[d]];
  // extended rows (constraints, then the objective) and their chunks
  h.row_chunk.assign(m + 2, 0);
  auto push_row = [&](const std::vector<Entry>& v, double s, int row) {
    int64_t b = (int64_t)h.ent_p.size();
    for (const Entry& x : v) {
      int p, q;
      svec_unpack(x.key, &p, &q);
      h.ent_p.push_back(p);
      h.ent_q.push_back(q);
      h.ent_a.push_back(x.a * s * (p == q ? 1.0 : 2.0));
    }
    int64_t e = (int64_t)h.ent_p.size();
    int64_t c = b;
    do {  // every row owns at least one (possibly empty) chunk
      h.chunk_beg.push_back((int)c);
      h.chunk_end.push_back((int)std::min<int64_t>(e, c + psdp::kChunk));
      h.chunk_row.push_back(row);
      c += psdp::kChunk;
    } while (c < e);
  };
  for (int i = 0; i < m; ++i) {
    h.row_chunk[i] = (int)h.chunk_beg.size();
    push_row(rows[i], h.scale[i], i);
    if ((int)h.chunk_beg.size() - h.row_chunk[i] > 1) h.multi_rows.push_back(i);
  }
  h.row_chunk[m] = (int)h.chunk_beg.size();
  push_row(centries, 1.0, m);
  h.row_chunk[m + 1] = (int)h.chunk_beg.size();
  // union pattern of C and the constraint entries
  struct Contrib {
    int64_t key;
    int row;
    double a;
  };
  std::vector<Contrib> contrib;
  for (int i = 0; i < m; ++i)
    for (const Entry& x : rows[i]) contrib.push_back({x.key, i, x.a * h.scale[i]});
  std::vector<int64_t> keys;
  keys.reserve(contrib.size() + centries.size());
  for (const auto& c : contrib) keys.push_back(c.key);
  for (const auto& c : centries) keys.push_back(c.key);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  const int nU = (int)keys.size();
  auto uidx = [&](int64_t key) { return (int)(std::lower_bound(keys.begin(), keys.end(), key) - keys.begin()); };
  h.u_p.resize(nU);
  h.u_q.resize(nU);
  h.u_c.assign(nU, 0.0);
  for (int u = 0; u < nU; ++u) svec_unpack(keys[u], &h.u_p[u], &h.u_q[u]);
  for (const auto& c : centries) h.u_c[uidx(c.key)] += c.a;
  std::stable_sort(contrib.begin(), contrib.end(), [](const Contrib& x, const Contrib& y) { return x.key < y.key; });
  h.u_ptr.assign(nU + 1, 0);
  for (const auto& c : contrib) h.u_ptr[uidx(c.key) + 1] += 1;
  for (int u = 0; u < nU; ++u) h.u_ptr[u + 1] += h.u_ptr[u];
  h.u_row.resize(contrib.size());
  h.u_a.resize(contrib.size());
  for (size_t k = 0; k < contrib.size(); ++k) {
    h.u_row[k] = contrib[k].row;
    h.u_a[k] = contrib[k].a;
  }
  // rebuild tiles (both triangles)
  const int T = psdp::kTile;
  h.ntile = (n + T - 1) / T;
  const size_t nt2 = (size_t)h.ntile * h.ntile;
  std::vector<int> cnt(nt2 + 1, 0);
  for (int u = 0; u < nU; ++u) {
    int p = h.u_p[u], q = h.u_q[u];
    cnt[(size_t)(p / T) * h.ntile + q / T + 1] += 1;
    if (p != q) cnt[(size_t)(q / T) * h.ntile + p / T + 1] += 1;
  }
  for (size_t t = 0; t < nt2; ++t) cnt[t + 1] += cnt[t];
  h.tile_ptr = cnt;
  h.tile_loc.resize(cnt[nt2]);
  h.tile_u.resize(cnt[nt2]);
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int u = 0; u < nU; ++u) {
    int p = h.u_p[u], q = h.u_q[u];
    size_t t = (size_t)(p / T) * h.ntile + q / T;
    h.tile_loc[fill[t]] = (p % T) * T + q % T;
    h.tile_u[fill[t]++] = u;
    if (p != q) {
      t = (size_t)(q / T) * h.ntile + p / T;
      h.tile_loc[fill[t]] = (q % T) * T + p % T;
      h.tile_u[fill[t]++] = u;
    }
  }
  // rows of the full pattern (the factored operator's sparse part; left empty
  // when the pattern has more entries than an int indexes)
  if (2 * (int64_t)nU < (int64_t)INT32_MAX) {
    h.sym_ptr.assign((size_t)n + 1, 0);
    for (int u = 0; u < nU; ++u) {
      h.sym_ptr[(size_t)h.u_p[u] + 1] += 1;
      if (h.u_p[u] != h.u_q[u]) h.sym_ptr[(size_t)h.u_q[u] + 1] += 1;
    }
    for (int i = 0; i < n; ++i) h.sym_ptr[(size_t)i + 1] += h.sym_ptr[i];
    h.sym_col.resize(h.sym_ptr[n]);
    h.u_pos.assign(2 * (size_t)nU, -1);
    {
      std::vector<int> at(h.sym_ptr.begin(), h.sym_ptr.end() - 1);
      for (int u = 0; u < nU; ++u) {
        const int p = h.u_p[u], q = h.u_q[u];
        h.u_pos[2 * (size_t)u] = at[p];
        h.sym_col[at[p]++] = q;
        if (p != q) {
          h.u_pos[2 * (size_t)u + 1] = at[q];
          h.sym_col[at[q]++] = p;
        }
      }
    }
  }
  // norms for the relative residuals
  double c2 = 0.0;
  for (int u = 0; u < nU; ++u) c2 += (h.u_p[u] == h.u_q[u] ? 1.0 : 2.0) * h.u_c[u] * h.u_c[u];
  h.normC = std::sqrt(c2);
  double r2 = 0.0;
  for (int i = 0; i < m; ++i) r2 += h.rhs[i] * h.rhs[i];
  h.normRhs = std::sqrt(r2);
  // ||M||_2: power iteration on the Gram operator v -> M(M*(v)) (FP64, host)
  double lam = 0.0;
  if (m > 0) {
    std::vector<int> ent_u;
    ent_u.reserve(h.ent_p.size());
    std::vector<int> ent_row;
    for (int i = 0; i < m; ++i)
      for (const Entry& x : rows[i]) {
        ent_u.push_back(uidx(x.key));
        ent_row.push_back(i);
      }
    std::vector<double> wu(nU);
    for (int u = 0; u < nU; ++u) wu[u] = (h.u_p[u] == h.u_q[u]) ? 1.0 : 2.0;
    double wsum_all = (double)n * (double)n;
    std::vector<double> v(m), gv(m), z(nU);
    for (int i = 0; i < m; ++i) v[i] = 1.0 + 0.01 * std::sin(1.0 + i);
    double nv = std::sqrt(std::inner_product(v.begin(), v.end(), v.begin(), 0.0));
    for (double& x : v) x /= nv;
    double prev = -1.0;
    for (int itp = 0; itp < 20000; ++itp) {
      // z = sparse part of M*(v) on the union pattern; cshift = dense part
      std::fill(z.begin(), z.end(), 0.0);
      for (size_t k = 0; k < ent_u.size(); ++k) {
        int i = ent_row[k];
        const double a = h.ent_a[k] / (h.ent_p[k] == h.ent_q[k] ? 1.0 : 2.0);
        z[ent_u[k]] += v[i] * a;
      }
      double cshift = 0.0;
      for (size_t d = 0; d < h.dense_row.size(); ++d) cshift += v[h.dense_row[d]] * h.dense_a[d];
      double zsum = 0.0;
      for (int u = 0; u < nU; ++u) zsum += wu[u] * z[u];
      // gv = M(z + cshift 11^T)
      std::fill(gv.begin(), gv.end(), 0.0);
      for (size_t k = 0; k < ent_u.size(); ++k) gv[ent_row[k]] += h.ent_a[k] * (z[ent_u[k]] + cshift);
      for (size_t d = 0; d < h.dense_row.size(); ++d)
        gv[h.dense_row[d]] += h.dense_a[d] * (zsum + cshift * wsum_all);
      lam = std::inner_product(v.begin(), v.end(), gv.begin(), 0.0);
      double ng = std::sqrt(std::inner_product(gv.begin(), gv.end(), gv.begin(), 0.0));
      if (ng == 0.0) break;
      for (int i = 0; i < m; ++i) v[i] = gv[i] / ng;
      if (std::fabs(lam - prev) <= 1e-13 * std::fabs(lam)) break;
      prev = lam;
    }
  }
  h.normM = lam > 0.0 ? std::sqrt(lam) : 1.0;
  h.alpha = (set.alpha_frac > 0.0 ? set.alpha_frac : 0.95) / h.normM;
  return PROXSDP_OK;
}

}  // namespace

namespace psdp {

int check_settings(const proxsdp_gpu_settings& s, std::string& err) {
  if (!(s.tol > 0.0) || s.max_iter < 0 || s.rank_init < 1 || s.block_size < 1 || s.window < 1 ||
      s.window > psdp::kMaxWindow || !(s.alpha_frac > 0.0 && s.alpha_frac < 1.0) || s.max_rank < 1 ||
      s.lanczos_max_cycles < 1 || s.lanczos_steps < 0 || s.lanczos_tol < 0.0 || s.guard < 0 ||
      s.check_every < 1 || s.precision != PROXSDP_PREC_FP32 || s.operator_form < PROXSDP_OP_EXPLICIT ||
      s.operator_form > PROXSDP_OP_AUTO || s.memory_limit_bytes < 0 || s.at_max_rank < 0 || s.at_max_rank > 1) {
    err = "invalid settings";
    return PROXSDP_ERR_INVALID_ARG;
  }
  return PROXSDP_OK;
}

int check_device(int device, std::string& err) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    err = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  if (device < 0 || device >= count) {
    err = "device index out of range";
    return PROXSDP_ERR_CUDA;
  }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  if (!(prop.major == 10 && prop.minor == 3)) {
    err = "this library is built for sm_103a (GB300); device is sm_" + std::to_string(prop.major) +
          std::to_string(prop.minor);
    return PROXSDP_ERR_CUDA;
  }
  e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  return PROXSDP_OK;
}

}  // namespace psdp

using psdp::check_device;
using psdp::check_settings;

namespace {

// Stream-ordered scratch of the device-pointer entry points comes from a
// library-owned memory pool per device whose release threshold keeps freed
// blocks mapped (the default pool unmaps them at every synchronisation, and
// mapping device memory again costs about 0.1 ms per call).  The pool keeps
// the largest scratch in use so far until the process exits.
cudaMemPool_t scratch_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[256] = {};
  if (dev < 0 || dev >= 256) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

}  // namespace

extern "C" {

int proxsdp_gpu_settings_default(proxsdp_gpu_settings* s) {
  if (!s) return PROXSDP_ERR_INVALID_ARG;
  std::memset(s, 0, sizeof(*s));
  s->tol = 1e-4;
  s->max_iter = 1000000;
  s->time_limit_s = 1200.0;
  s->full_eig = 0;
  s->rank_init = 8;
  s->block_size = 16;
  s->window = 100;
  s->eps_lambda = 0.0;
  s->alpha_frac = 0.95;
  s->precision = PROXSDP_PREC_FP32;
  s->normalize_rows = 1;
  s->seed = 1;
  s->max_rank = 64;
  s->lanczos_steps = 0;
  s->lanczos_max_cycles = 8;
  s->lanczos_tol = 0.0;
  s->guard = 0;
  s->check_every = 50;
  s->use_graphs = 1;
  s->operator_form = PROXSDP_OP_EXPLICIT;
  s->memory_limit_bytes = 0;
  s->at_max_rank = 0;
  return PROXSDP_OK;
}

int proxsdp_gpu_create(const proxsdp_gpu_settings* settings, int device, void* cuda_stream,
                       proxsdp_gpu_t* out) {
  if (!out) return PROXSDP_ERR_INVALID_ARG;
  *out = nullptr;
  proxsdp_gpu_settings s;
  if (settings) s = *settings;
  else proxsdp_gpu_settings_default(&s);
  std::string err;
  int rc = check_settings(s, err);
  if (rc) {
    g_last_create_error = err;
    return rc;
  }
  rc = check_device(device, err);
  if (rc) {
    g_last_create_error = err;
    return rc;
  }
  proxsdp_gpu_ctx* h = new proxsdp_gpu_ctx();
  Solver& S = h->s;
  S.set = s;
  S.device = device;
  S.seed = s.seed ? s.seed : 1;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    S.st = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking);
    S.own_stream = true;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S.st_aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&S.ctl_host, sizeof(psdp::Ctl));
  if (e != cudaSuccess) {
    g_last_create_error = cudaGetErrorString(e);
    delete h;
    return PROXSDP_ERR_CUDA;
  }
  psdp::init_kernel_attributes();
  *out = h;
  return PROXSDP_OK;
}

int proxsdp_gpu_set_problem(proxsdp_gpu_t h, int64_t n, const double* C_dense, int64_t c_nnz,
                            const int64_t* c_idx, const double* c_val, int64_t m_total, int64_t m_eq,
                            const int64_t* A_rowptr, const int64_t* A_col, const double* A_val,
                            const double* rhs) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  cudaSetDevice(S.device);
  HostProblem hp;
  int rc = preprocess(S.set, n, C_dense, c_nnz, c_idx, c_val, m_total, m_eq, A_rowptr, A_col, A_val, rhs,
                      hp, S.err);
  if (rc) return rc;
  if (S.set.full_eig && n > psdp::kFullEigMax)
    return S.fail(PROXSDP_ERR_UNSUPPORTED, "full_eig (Alg. 1) is limited to n <= 128");
  return S.upload(hp);
}

int proxsdp_gpu_analyze_problem(const proxsdp_gpu_settings* settings, int64_t n, const double* C_dense,
                                int64_t c_nnz, const int64_t* c_idx, const double* c_val, int64_t m_total,
                                int64_t m_eq, const int64_t* A_rowptr, const int64_t* A_col,
                                const double* A_val, const double* rhs, double* norm_M, double* alpha,
                                int64_t* n_union, double* norm_C) {
  proxsdp_gpu_settings s;
  if (settings) s = *settings;
  else proxsdp_gpu_settings_default(&s);
  std::string err;
  int rc = check_settings(s, err);
  if (rc) {
    g_last_create_error = err;
    return rc;
  }
  HostProblem hp;
  rc = preprocess(s, n, C_dense, c_nnz, c_idx, c_val, m_total, m_eq, A_rowptr, A_col, A_val, rhs, hp, err);
  if (rc) {
    g_last_create_error = err;
    return rc;
  }
  if (norm_M) *norm_M = hp.normM;
  if (alpha) *alpha = hp.alpha;
  if (n_union) *n_union = (int64_t)hp.u_p.size();
  if (norm_C) *norm_C = hp.normC;
  return PROXSDP_OK;
}

int proxsdp_gpu_solve(proxsdp_gpu_t h, proxsdp_gpu_info* info) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  if (!S.has_problem) return S.fail(PROXSDP_ERR_BAD_STATE, "solve before set_problem");
  cudaSetDevice(S.device);
  int rc = S.init_iterate_zero();
  if (rc) return rc;
  return S.run(-1, true, info);
}

int proxsdp_gpu_iterate(proxsdp_gpu_t h, int64_t iters, proxsdp_gpu_info* info) {
  if (!h || iters < 0) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  if (!S.has_problem) return S.fail(PROXSDP_ERR_BAD_STATE, "iterate before set_problem");
  cudaSetDevice(S.device);
  if (!S.has_iterate) {
    int rc = S.init_iterate_zero();
    if (rc) return rc;
  }
  return S.run(iters, false, info);
}

int proxsdp_gpu_resume(proxsdp_gpu_t h, int64_t max_iters, proxsdp_gpu_info* info) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  if (!S.has_problem) return S.fail(PROXSDP_ERR_BAD_STATE, "resume before set_problem");
  cudaSetDevice(S.device);
  if (!S.has_iterate) {
    int rc = S.init_iterate_zero();
    if (rc) return rc;
  }
  return S.run(max_iters < 0 ? -1 : max_iters, true, info);
}

int proxsdp_gpu_set_iterate(proxsdp_gpu_t h, int r, const double* V, const double* lambda,
                            const double* y) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  if (!S.has_problem) return S.fail(PROXSDP_ERR_BAD_STATE, "set_iterate before set_problem");
  if (r < 1 || r > std::min(S.hp.n, psdp::kMaxR) || (!V && r > 0) || !lambda)
    return S.fail(PROXSDP_ERR_INVALID_ARG, "bad rank or NULL factors");
  if (S.hp.n > psdp::kFullEigMax && !S.set.full_eig &&
      r > (S.factored ? psdp::kMaxRankFactored : psdp::kMaxRankLanczos))
    return S.fail(PROXSDP_ERR_UNSUPPORTED, S.factored ? "rank above 60 with the factored operator"
                                                      : "rank above 64 on the block Lanczos path");
  cudaSetDevice(S.device);
  return S.set_iterate(r, V, lambda, y);
}

}  // extern "C"

namespace {

// Copy factors (n x kMaxR row-major FP32), eigenvalues and the scaled dual
// (algorithm sign) from the device and export them in the ABI's form.
int export_pair(Solver& S, const float* dV, const double* dlam, const double* dy, int r, double* X, double* y,
                double* V, double* lambda) {
  const int n = S.hp.n, m = S.hp.m;
  std::vector<float> Vr((size_t)n * psdp::kMaxR);
  std::vector<double> lam(psdp::kMaxR), yy(std::max(m, 1));
  cudaError_t e = cudaMemcpyAsync(Vr.data(), dV, sizeof(float) * Vr.size(), cudaMemcpyDeviceToHost, S.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lam.data(), dlam, sizeof(double) * psdp::kMaxR, cudaMemcpyDeviceToHost, S.st);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(yy.data(), dy, sizeof(double) * m, cudaMemcpyDeviceToHost, S.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S.st);
  if (e != cudaSuccess) return S.fail(PROXSDP_ERR_CUDA, cudaGetErrorString(e));
  if (X) {
    std::fill(X, X + (size_t)n * n, 0.0);
    for (int t = 0; t < r; ++t) {
      double l = std::max(lam[t], 0.0);
      if (l == 0.0) continue;
      for (int i = 0; i < n; ++i) {
        double vi = l * (double)Vr[(size_t)i * psdp::kMaxR + t];
        if (vi == 0.0) continue;
        double* row = X + (size_t)i * n;
        for (int j = 0; j < n; ++j) row[j] += vi * (double)Vr[(size_t)j * psdp::kMaxR + t];
      }
    }
  }
  if (y)
    for (int i = 0; i < m; ++i) y[i] = -yy[i] * S.hp.scale[i];  // paper's dual sign, original rows
  if (V)
    for (int t = 0; t < r; ++t)
      for (int i = 0; i < n; ++i) V[(size_t)t * n + i] = (double)Vr[(size_t)i * psdp::kMaxR + t];
  if (lambda)
    for (int t = 0; t < r; ++t) lambda[t] = lam[t];
  return PROXSDP_OK;
}

}  // namespace

extern "C" {

int proxsdp_gpu_get_primal_dual(proxsdp_gpu_t h, double* X, double* y, double* V, double* lambda,
                                int64_t* r_out) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  if (!S.has_problem || !S.has_iterate) return S.fail(PROXSDP_ERR_BAD_STATE, "no iterate yet");
  cudaSetDevice(S.device);
  int rc = S.read_ctl();
  if (rc) return rc;
  const int par = S.ctl_host->par;
  const int r = S.ctl_host->r_old;  // rank of the current iterate
  rc = export_pair(S, S.wk.Vrm[par], S.wk.lam[par], S.wk.y, r, X, y, V, lambda);
  if (rc) return rc;
  if (r_out) *r_out = r;
  return PROXSDP_OK;
}

int proxsdp_gpu_set_box(proxsdp_gpu_t h, double u) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  cudaSetDevice(S.device);
  return S.set_box(u);
}

int proxsdp_gpu_get_box_dual(proxsdp_gpu_t h, double* Y_upper, double* Y_lower) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  if (!S.has_problem || !S.has_iterate) return S.fail(PROXSDP_ERR_BAD_STATE, "no iterate yet");
  if (!S.pb.box) return S.fail(PROXSDP_ERR_BAD_STATE, "no element-wise box was set");
  cudaSetDevice(S.device);
  const int n = S.hp.n, ld = S.wk.lds;
  std::vector<float> buf((size_t)n * ld);
  // paper's sign (<= 0), original scaling: y = -s y_scaled
  const double sc = -(double)S.pb.box_s;
  float* src[2] = {S.wk.ybp, S.wk.ybm};
  double* dst[2] = {Y_upper, Y_lower};
  for (int k = 0; k < 2; ++k) {
    if (!dst[k]) continue;
    if (cudaMemcpyAsync(buf.data(), src[k], sizeof(float) * buf.size(), cudaMemcpyDeviceToHost, S.st) !=
            cudaSuccess ||
        cudaStreamSynchronize(S.st) != cudaSuccess)
      return S.fail(PROXSDP_ERR_CUDA, "copy of the box duals failed");
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) dst[k][(size_t)i * n + j] = (i == j) ? 0.0 : sc * (double)buf[(size_t)i * ld + j];
  }
  return PROXSDP_OK;
}

int proxsdp_gpu_get_saved_pair(proxsdp_gpu_t h, double* X, double* y, double* V, double* lambda,
                               int64_t* r_out, int64_t* iter_out) {
  if (!h) return PROXSDP_ERR_INVALID_ARG;
  Solver& S = h->s;
  if (!S.has_problem || S.saved_r <= 0)
    return S.fail(PROXSDP_ERR_BAD_STATE, "no feasible pair was saved by the last solve");
  cudaSetDevice(S.device);
  int rc = export_pair(S, S.saved_V, S.saved_lam, S.saved_y, S.saved_r, X, y, V, lambda);
  if (rc) return rc;
  if (r_out) *r_out = S.saved_r;
  if (iter_out) *iter_out = S.saved_it;
  return PROXSDP_OK;
}

int proxsdp_gpu_solve_batch(proxsdp_gpu_t* handles, int count, proxsdp_gpu_info* infos, int host_threads) {
  if (count < 0 || (count > 0 && !handles)) return PROXSDP_ERR_INVALID_ARG;
  std::unordered_set<proxsdp_gpu_t> seen;
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || !seen.insert(handles[i]).second) {
      psdp::set_global_error("solve_batch: NULL or repeated handle");
      return PROXSDP_ERR_INVALID_ARG;
    }
  }
  // largest problems first (n^2 bounds the work of an iteration), so that the
  // long solves start early and the short ones fill in behind them
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return handles[a]->s.hp.n > handles[b]->s.hp.n; });
  std::vector<int> rc(count, PROXSDP_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int i = order[k];
      rc[i] = proxsdp_gpu_solve(handles[i], infos ? &infos[i] : nullptr);
    }
  };
  int nt = host_threads > 0 ? host_threads : 16;
  nt = std::max(1, std::min(nt, count));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  for (int i = 0; i < count; ++i)
    if (rc[i] != PROXSDP_OK) return rc[i];
  return PROXSDP_OK;
}

void proxsdp_gpu_destroy(proxsdp_gpu_t h) {
  if (!h) return;
  cudaSetDevice(h->s.device);
  if (h->s.st) cudaStreamSynchronize(h->s.st);
  delete h;
}

const char* proxsdp_gpu_last_error(proxsdp_gpu_t h) {
  if (!h) return g_last_create_error.c_str();
  return h->s.err.c_str();
}

int proxsdp_gpu_aproj(const float* S, int64_t n, int64_t lds, int r, float* P, int64_t ldp, float* V,
                      double* lambda, const proxsdp_gpu_settings* settings, void* cuda_stream,
                      proxsdp_gpu_info* info) {
  if (!S || n < 1 || n > 46340 || lds < n || r < 1 || r > n || (P && ldp < n))
    return PROXSDP_ERR_INVALID_ARG;
  proxsdp_gpu_settings s;
  if (settings) s = *settings;
  else {
    proxsdp_gpu_settings_default(&s);
    s.lanczos_max_cycles = 100;
    s.lanczos_tol = 1e-6;
  }
  std::string err;
  int rc = check_settings(s, err);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PROXSDP_ERR_CUDA;
  rc = check_device(dev, err);
  if (rc) return rc;
  psdp::init_kernel_attributes();
  return psdp::aproj_device(S, (int)n, (int)lds, r, P, (int)ldp, V, lambda, s, (cudaStream_t)cuda_stream,
                            info, err);
}

int proxsdp_gpu_block_matvec(const float* S, int64_t n, int64_t lds, const float* Q, int64_t ldq, int k,
                             float* W, int64_t ldw, void* cuda_stream) {
  if (!S || !Q || !W || n < 1 || lds < n || ldq < n || ldw < n || k < 1 || k > 256)
    return PROXSDP_ERR_INVALID_ARG;
  int dev = 0;
  std::string err;
  if (cudaGetDevice(&dev) != cudaSuccess) return PROXSDP_ERR_CUDA;
  int rc = check_device(dev, err);
  if (rc) return rc;
  psdp::init_kernel_attributes();
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float* part = nullptr;
  const size_t np = psdp::block_matvec_scratch_floats((int)n, k);
  cudaMemPool_t pool = scratch_pool(dev);
  if (!pool) return PROXSDP_ERR_CUDA;
  if (cudaMallocFromPoolAsync((void**)&part, np * sizeof(float), pool, st) != cudaSuccess) {
    cudaGetLastError();
    return PROXSDP_ERR_OOM;
  }
  psdp::launch_block_matvec(S, (int)lds, (int)n, Q, (int)ldq, W, (int)ldw, k, nullptr, st, part, nullptr);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, st);
  if (e != cudaSuccess) {
    psdp::set_global_error(std::string("block product launch: ") + cudaGetErrorString(e));
    return PROXSDP_ERR_CUDA;
  }
  return PROXSDP_OK;
}

int proxsdp_gpu_sym_eig(const double* T, int K, double* theta, float* Y, void* cuda_stream) {
  if (!T || !theta || !Y || K < 1 || K > psdp::kMaxK) return PROXSDP_ERR_INVALID_ARG;
  int dev = 0;
  std::string err;
  if (cudaGetDevice(&dev) != cudaSuccess) return PROXSDP_ERR_CUDA;
  int rc = check_device(dev, err);
  if (rc) return rc;
  psdp::init_kernel_attributes();
  return psdp::sym_eig_device(T, K, theta, Y, (cudaStream_t)cuda_stream);
}

}  // extern "C"
