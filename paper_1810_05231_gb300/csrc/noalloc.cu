// noalloc.cu — the truncated psd projection aproj(S, r) for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: applications that hand all of the GPU's
// memory to their own pool allocator and forbid anything else from
// allocating, plugins that run inside such a host, and embedded or real-time
// hosts that must not take the allocator's locks or risk an out-of-memory
// failure in the middle of a run.  For them this file provides
// proxsdp_gpu_aproj_noalloc: the same computation as proxsdp_gpu_aproj, but
// every work buffer lives in one file-scope static __device__ array of fixed
// size (about 6.7 MB, held by every GPU that loads the library until the
// process exits), so the call allocates nothing.  The price is a size limit,
// n <= kNoAllocMaxN, and the fact that all calls share the one array.
#include <cstring>
#include <mutex>
#include <string>

#include "solver.h"

namespace psdp {

void set_global_error(const std::string& msg);

namespace {

constexpr int kNoAllocMaxN = 2048;
constexpr size_t kLd = kNoAllocMaxN;  // row stride of the basis (a multiple of 32)
constexpr int kNt = kNoAllocMaxN / kTile;

// Layout of the scratch array (byte offsets, 256-byte aligned pieces).
constexpr size_t al(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffQ = 0;
constexpr size_t kOffW = kOffQ + al(kLd * kMaxK * sizeof(float));
constexpr size_t kOffV0 = kOffW + al(kLd * kMaxK * sizeof(float));
constexpr size_t kOffV1 = kOffV0 + al(kLd * kMaxR * sizeof(float));
constexpr size_t kOffVcm = kOffV1 + al(kLd * kMaxR * sizeof(float));
constexpr size_t kOffY = kOffVcm + al(kLd * 2 * kMaxR * sizeof(float));
constexpr size_t kOffHf = kOffY + al((size_t)kMaxK * kMaxK * sizeof(float));
constexpr size_t kOffLam = kOffHf + al((size_t)kMaxW * kMaxW * sizeof(float));   // lam0, lam1, colsum0, colsum1
constexpr size_t kOffH = kOffLam + al(4 * kMaxR * sizeof(double));
constexpr size_t kOffTheta = kOffH + al((size_t)kMaxK * kMaxK * sizeof(double));
constexpr size_t kOffRitz = kOffTheta + al(kMaxK * sizeof(double));
constexpr size_t kOffSmall = kOffRitz + al(((size_t)kNoAllocMaxN / 32 + 1) * 4 * kMaxW * sizeof(double));  // dshift, D
constexpr size_t kOffFlags = kOffSmall + al(8 * sizeof(double));
constexpr size_t kOffCnt = kOffFlags + al(kMaxW * sizeof(int));
constexpr size_t kOffTile = kOffCnt + al((size_t)CNT_NUM * 512 * sizeof(unsigned));
constexpr size_t kOffCtl = kOffTile + al(((size_t)kNt * kNt + 1) * sizeof(int));
constexpr size_t kScratchBytes = kOffCtl + al(sizeof(Ctl));

// The scratch.  In host code this name is only a host-side stand-in for the
// device array (never dereference it or pass it to a kernel); its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_aproj_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[256];
bool g_have[256];

// Device address of the scratch on the current device (looked up on the
// first call per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_have[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_aproj_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
    g_have[dev] = true;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return cudaSuccess;
}

}  // namespace

int aproj_noalloc_device(const float* S, int n, int lds, int r, float* P, int ldp, float* V, double* lambda,
                         const proxsdp_gpu_settings& set, cudaStream_t st, proxsdp_gpu_info* info,
                         std::string& err) {
  if (n > kNoAllocMaxN) {
    err = "proxsdp_gpu_aproj_noalloc supports n <= " + std::to_string(kNoAllocMaxN) + " (got " +
          std::to_string(n) + "); use proxsdp_gpu_aproj for larger matrices";
    return PROXSDP_ERR_UNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  unsigned char* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    err = std::string("scratch address: ") + cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  // block width / basis size exactly as the allocating entry point chooses
  // them (a cold start: the largest Rayleigh-Ritz basis)
  const bool full = n <= kFullEigMax;
  int w, K, s;
  if (full) {
    w = n;
    K = n;
    s = 0;
  } else {
    lanczos_dims(r, set, kMaxK, kMaxW, w, K, s);  // this scratch layout holds blocks of up to kMaxW
    if (r > w - 4) {
      err = "rank too large for the Lanczos block (r <= 60)";
      return PROXSDP_ERR_UNSUPPORTED;
    }
  }
  DevProblem pb = {};
  pb.n = n;
  pb.ntile = (n + kTile - 1) / kTile;
  pb.tile_ptr = reinterpret_cast<const int*>(base + kOffTile);
  DevWork wk = {};
  wk.S = const_cast<float*>(S);
  wk.lds = lds;
  wk.ldq = (int)kLd;
  wk.ldv = kMaxR;
  wk.Q = reinterpret_cast<float*>(base + kOffQ);
  wk.W = reinterpret_cast<float*>(base + kOffW);
  wk.Vrm[0] = reinterpret_cast<float*>(base + kOffV0);
  wk.Vrm[1] = reinterpret_cast<float*>(base + kOffV1);
  wk.Vcm = reinterpret_cast<float*>(base + kOffVcm);
  wk.Y = reinterpret_cast<float*>(base + kOffY);
  wk.Hf = reinterpret_cast<float*>(base + kOffHf);
  double* lam = reinterpret_cast<double*>(base + kOffLam);
  wk.lam[0] = lam;
  wk.lam[1] = lam + kMaxR;
  wk.colsum[0] = lam + 2 * kMaxR;
  wk.colsum[1] = lam + 3 * kMaxR;
  wk.H = reinterpret_cast<double*>(base + kOffH);
  wk.theta = reinterpret_cast<double*>(base + kOffTheta);
  wk.ritz_part = reinterpret_cast<double*>(base + kOffRitz);
  wk.dshift = reinterpret_cast<double*>(base + kOffSmall);
  wk.D = wk.dshift + 4;
  wk.flags = reinterpret_cast<int*>(base + kOffFlags);
  wk.counters = reinterpret_cast<unsigned*>(base + kOffCnt);
  wk.ctl = reinterpret_cast<Ctl*>(base + kOffCtl);
  // The array keeps the previous call's contents: clear what must start at
  // zero (last-block counters, the empty sparse pattern of the rebuild, the
  // dense shift) and write a fresh control block.
  e = cudaMemsetAsync(base + kOffSmall, 0, kOffTile + al(((size_t)kNt * kNt + 1) * sizeof(int)) - kOffSmall, st);
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.par = 0;
  c.r = r;
  c.r_old = r;
  c.w = w;
  c.K = K;
  c.status = ST_RUNNING;
  c.max_cycles = set.lanczos_max_cycles > 0 ? set.lanczos_max_cycles : 1;
  c.lz_tol_fixed = set.lanczos_tol > 0 ? set.lanczos_tol : 1e-6;
  c.lz_tol = c.lz_tol_fixed;
  if (e == cudaSuccess) e = cudaMemcpyAsync(wk.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  const unsigned long long seed = set.seed ? set.seed : 1;
  if (full) {
    launch_s_to_t(S, lds, n, wk.H, st);
    launch_sym_eig(wk.H, n, wk.theta, wk.Y, kMaxK, n, nullptr, st);
    launch_full_eig_factors(wk, n, st);
  } else {
    launch_random_block(wk.Q, wk.ldq, n, 0, w, seed, st);
    enqueue_orth(wk, n, 0, w, seed, nullptr, st);
    launch_block_matvec(S, lds, n, wk.Q, wk.ldq, wk.W, wk.ldq, w, nullptr, st);
    for (int cyc = 0; cyc < c.max_cycles; ++cyc)
      enqueue_cycle(wk, n, w, K, s, r, seed + 1000ULL * (unsigned long long)(cyc + 1), 0, 0, st);
  }
  if (P) {
    DevWork out = wk;
    out.S = P;
    out.lds = ldp;
    launch_rebuild(pb, out, r, 1, st);
  }
  if (V) {
    e = full ? cudaMemcpy2DAsync(V, sizeof(float) * n, wk.Y, sizeof(float) * kMaxK, sizeof(float) * n, r,
                                 cudaMemcpyDeviceToDevice, st)
             : cudaMemcpy2DAsync(V, sizeof(float) * n, wk.Q, sizeof(float) * wk.ldq, sizeof(float) * n, r,
                                 cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess && lambda)
    e = cudaMemcpyAsync(lambda, wk.lam[1], sizeof(double) * r, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  Ctl done;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&done, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PROXSDP_ERR_CUDA;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->final_rank = r;
    info->matvecs = full ? 0 : 1 + (int64_t)done.lz_cycles_total * s;
    info->lanczos_cycles = done.lz_cycles_total;
    info->lanczos_unconverged = done.lz_unconverged;
    info->eps_primal = done.lz_res;
    info->status = (done.lz_done && done.lz_unconverged == 0) ? PROXSDP_CONVERGED : PROXSDP_MAX_ITER;
  }
  return PROXSDP_OK;
}

}  // namespace psdp

extern "C" int proxsdp_gpu_aproj_noalloc(const float* S, int64_t n, int64_t lds, int r, float* P, int64_t ldp,
                                         float* V, double* lambda, const proxsdp_gpu_settings* settings,
                                         void* cuda_stream, proxsdp_gpu_info* info) {
  if (!S || n < 1 || lds < n || r < 1 || r > n || (P && ldp < n)) return PROXSDP_ERR_INVALID_ARG;
  proxsdp_gpu_settings s;
  if (settings) s = *settings;
  else {
    proxsdp_gpu_settings_default(&s);
    s.lanczos_max_cycles = 100;
    s.lanczos_tol = 1e-6;
  }
  std::string err;
  int rc = psdp::check_settings(s, err);
  int dev = 0;
  if (rc == PROXSDP_OK && cudaGetDevice(&dev) != cudaSuccess) {
    err = "no current CUDA device";
    rc = PROXSDP_ERR_CUDA;
  }
  if (rc == PROXSDP_OK) rc = psdp::check_device(dev, err);
  if (rc) {
    psdp::set_global_error(err);
    return rc;
  }
  psdp::init_kernel_attributes();
  rc = psdp::aproj_noalloc_device(S, (int)std::min<int64_t>(n, 1 << 30), (int)lds, r, P, (int)ldp, V, lambda,
                                      s, (cudaStream_t)cuda_stream, info, err);
  if (rc) psdp::set_global_error(err);
  return rc;
}
