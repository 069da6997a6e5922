// k_mv_tc.cu — the block Krylov product W = S Q of the truncated projection
// (Sec. 3.1, Eq. trunc_eig) on the fifth-generation tensor cores.
//
// S (n x n FP32, symmetric, row stride lds) is streamed from HBM once per
// product by TMA in 128-row x 32-column tiles (128-byte swizzle); Q (n x k)
// is split once per product into TF32 high and low parts (hi = Q with the low
// 13 mantissa bits cleared, lo = Q - hi, both exact in FP32) and streamed by
// TMA too.  Each CTA owns 128 rows of S and up to 64 columns of Q over one
// slice of the inner dimension.  Its four warps read their rows of each S
// tile from shared memory, split them the same way and store S_hi and S_lo
// into tensor memory (TMEM), and one thread issues
//     D += S_lo Q_hi + S_hi Q_lo + S_hi Q_hi
// as tcgen05.mma kind::tf32 with A read from TMEM and B from shared memory,
// accumulating in FP32 in TMEM ("3xTF32": the dropped term S_lo Q_lo and the
// TF32 rounding of S_lo are O(2^-22) relative, FP32-grade).  Slices of one
// row block form a thread-block cluster whose partial tiles are summed in a
// fixed CTA order through distributed shared memory (deterministic).
//
// Every wait on an mbarrier is bounded (kWaitCycles); a CTA that gives up
// drains its own copies in flight (bounded again), frees its TMEM and writes
// NaN to its output rows, so the iteration using the product reports a
// numeric error instead of hanging.
#include <cuda.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "psdp.cuh"

namespace psdp {

namespace {

constexpr int TC_M = 128;        // rows of S per CTA = the MMA's M
constexpr int TC_KC = 32;        // inner-dimension chunk: one 128-byte swizzle row of FP32
constexpr int TC_NS = 3;         // shared-memory stages
constexpr int TC_NMAX = 64;      // columns of Q per CTA
constexpr int TC_THREADS = 128;  // four warps: one TMEM lane quarter each
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kAccCol = 0;  // accumulator: columns [0, 64)
constexpr uint32_t kABase = 64;  // A buffers b = 0, 1: hi at 64 + 64 b, lo at 96 + 64 b
constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at 2 GHz
constexpr int kSmemFloor = 80 * 1024;  // at most two CTAs per SM, so two TMEM allocations always fit

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait until the phase with the given parity has completed; false after
// `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem descriptor], kind::tf32, FP32 accumulator.
__device__ __forceinline__ void tc_mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n"
      "}\n" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

#define PSDP_R8(a, o) "r"(a[o]), "r"(a[o + 1]), "r"(a[o + 2]), "r"(a[o + 3]), "r"(a[o + 4]), "r"(a[o + 5]), "r"(a[o + 6]), "r"(a[o + 7])

// 32 consecutive TMEM columns of this thread's lane <- v[0..31]
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      PSDP_R8(v, 0), PSDP_R8(v, 8), PSDP_R8(v, 16), PSDP_R8(v, 24)
      : "memory");
}
#undef PSDP_R8

// v[0..15] <- 16 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows in the
// 128-byte swizzle (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1 << 16;                   // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride between 8-row groups
  d |= (uint64_t)1 << 46;                   // descriptor version of sm_100-family targets
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  const uint32_t h = __float_as_uint(x) & 0xFFFFE000u;
  hi = h;
  lo = __float_as_uint(x - __uint_as_float(h));
}

}  // namespace

// Q (n x k, column stride ldq) -> Qhi, Qlo (column stride ld2): hi keeps the
// 10 explicit mantissa bits of TF32 (the other 13 cleared), lo = Q - hi.
__global__ void k_split_tf32(const float* __restrict__ Q, int ldq, int n, int k, float* __restrict__ Qhi,
                             float* __restrict__ Qlo, int ld2, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const size_t total = (size_t)n * k;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / n), i = (int)(idx % n);
    uint32_t h, l;
    split_tf32(Q[(size_t)j * ldq + i], h, l);
    Qhi[(size_t)j * ld2 + i] = __uint_as_float(h);
    Qlo[(size_t)j * ld2 + i] = __uint_as_float(l);
  }
}

// Shared memory: [stage s: S tile 16 KB | Qhi tile nt*128 B | Qlo tile nt*128 B] x TC_NS,
// then the mbarriers and the TMEM address slot; the base is aligned to 1024 B.
__global__ void __launch_bounds__(TC_THREADS) k_block_matvec_tc(const __grid_constant__ CUtensorMap tmS,
                                                                const __grid_constant__ CUtensorMap tmQh,
                                                                const __grid_constant__ CUtensorMap tmQl, int n,
                                                                int k, float* __restrict__ W, int ldw, int nt,
                                                                int kslice, const int* skip,
                                                                cudaGraphConditionalHandle cond, int set_cond) {
  namespace cg = cooperative_groups;
  if (skip && *(volatile const int*)skip) return;  // uniform over the grid
  if (set_cond && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    cudaGraphSetConditional(cond, 1u);
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  unsigned char* dsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ns = gridDim.x;
  const int r0 = blockIdx.y * TC_M;
  const int c0 = blockIdx.z * TC_NMAX;
  const int kc_cols = min(TC_NMAX, k - c0);  // output columns of this CTA
  const int kb = blockIdx.x * kslice, ke = min(n, kb + kslice);
  const int nk = ke > kb ? (ke - kb + TC_KC - 1) / TC_KC : 0;  // chunks of this slice
  const uint32_t tileS = TC_M * TC_KC * 4;                      // 16 KB
  const uint32_t tileQ = (uint32_t)nt * TC_KC * 4;
  const uint32_t stage = tileS + 2 * tileQ;
  uint64_t* full = reinterpret_cast<uint64_t*>(dsm + TC_NS * stage);
  uint64_t* mma_done = full + TC_NS;  // [2]: the MMAs of chunks with parity b have completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 2);
  __shared__ int s_fail;
  if (tid == 0) {
    for (int s = 0; s < TC_NS; ++s) mbar_init(&full[s], 1);
    mbar_init(&mma_done[0], 1);
    mbar_init(&mma_done[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;  // this warp's TMEM lane quarter
  const uint32_t idesc = idesc_tf32(TC_M, nt);
  auto issue_load = [&](int j) {  // chunk j of the slice into stage j % TC_NS
    unsigned char* st = dsm + (j % TC_NS) * stage;
    uint64_t* bar = &full[j % TC_NS];
    mbar_expect_tx(bar, stage);
    const int x = kb + j * TC_KC;
    tma_load_2d(st, &tmS, bar, x, r0);
    tma_load_2d(st + tileS, &tmQh, bar, x, c0);
    tma_load_2d(st + tileS + tileQ, &tmQl, bar, x, c0);
  };
  int issued = 0;    // chunks whose loads were issued (thread 0)
  int committed = -1;  // last chunk whose MMAs were committed (thread 0)
  if (tid == 0) {
    for (; issued < min(TC_NS, nk); ++issued) issue_load(issued);
  }
  bool fail = false;
  for (int c = 0; c < nk; ++c) {
    const int s = c % TC_NS, b = c & 1;
    unsigned char* st = dsm + s * stage;
    bool ok = mbar_wait(&full[s], (uint32_t)((c / TC_NS) & 1), kWaitCycles);
    if (ok && c >= 2) ok = mbar_wait(&mma_done[b], (uint32_t)(((c - 2) >> 1) & 1), kWaitCycles);
    tc_fence_after();
    if (!ok) s_fail = 1;
    // this thread's row of the S tile: 16-byte chunk q of row tid sits at chunk q ^ (tid & 7)
    uint32_t hi[32], lo[32];
    const unsigned char* srow = st + tid * 128;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(srow + ((q ^ (tid & 7)) << 4));
      split_tf32(v.x, hi[4 * q], lo[4 * q]);
      split_tf32(v.y, hi[4 * q + 1], lo[4 * q + 1]);
      split_tf32(v.z, hi[4 * q + 2], lo[4 * q + 2]);
      split_tf32(v.w, hi[4 * q + 3], lo[4 * q + 3]);
    }
    const uint32_t abuf = tmem + kABase + 64u * (uint32_t)b;
    if (ok) {
      tmem_st32(abuf + lane_off, hi);
      tmem_st32(abuf + 32u + lane_off, lo);
    }
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    if (s_fail) {
      fail = true;
      break;
    }
    if (tid == 0) {
      tc_fence_after();
      const uint64_t dh = sdesc_k_sw128(smem_u32(st + tileS));
      const uint64_t dl = sdesc_k_sw128(smem_u32(st + tileS + tileQ));
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk) {
        const uint32_t ah = abuf + 8u * kk, al = ah + 32u;
        const uint64_t step = (uint64_t)(kk * 32 >> 4);  // 8 TF32 = 32 bytes along K
        tc_mma_ts(tmem + kAccCol, al, dh + step, idesc, (c > 0 || kk > 0) ? 1u : 0u);
        tc_mma_ts(tmem + kAccCol, ah, dl + step, idesc, 1u);
        tc_mma_ts(tmem + kAccCol, ah, dh + step, idesc, 1u);
      }
      tc_commit(&mma_done[b]);
      committed = c;
      // refill the stage of chunk c - 1 once its MMAs (which read its Q tiles) are done
      if (c >= 1 && issued < nk) {
        if (mbar_wait(&mma_done[(c - 1) & 1], (uint32_t)(((c - 1) >> 1) & 1), kWaitCycles)) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_load(issued);
          ++issued;
        } else {
          s_fail = 1;
        }
      }
    }
  }
  // accumulator -> registers (row tid of the tile, columns [0, nt))
  float acc[TC_NMAX];
#pragma unroll
  for (int j = 0; j < TC_NMAX; ++j) acc[j] = 0.f;
  if (!fail && nk > 0) {
    const int last = nk - 1;
    if (!mbar_wait(&mma_done[last & 1], (uint32_t)((last >> 1) & 1), kWaitCycles)) fail = true;
    tc_fence_after();
    if (!fail) {
#pragma unroll
      for (int g = 0; g < TC_NMAX / 16; ++g) {
        if (g * 16 < nt) {
          uint32_t v[16];
          tmem_ld16(tmem + kAccCol + 16u * g + lane_off, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[16 * g + j] = __uint_as_float(v[j]);
        }
      }
    }
  }
  if (__syncthreads_or(fail ? 1 : 0)) {
    // give up: drain this CTA's own copies and MMAs in flight (bounded), NaN output
    fail = true;
    if (tid == 0) {
      for (int j = max(0, issued - TC_NS); j < issued; ++j)
        mbar_wait(&full[j % TC_NS], (uint32_t)((j / TC_NS) & 1), kWaitCycles / 8);
      if (committed >= 0) mbar_wait(&mma_done[committed & 1], (uint32_t)((committed >> 1) & 1), kWaitCycles / 8);
    }
#pragma unroll
    for (int j = 0; j < TC_NMAX; ++j) acc[j] = __int_as_float(0x7fc00000);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (ns == 1) {
    const int row = r0 + tid;
    if (row < n)
#pragma unroll
      for (int j = 0; j < TC_NMAX; ++j)
        if (j < kc_cols) W[(size_t)(c0 + j) * ldw + row] = acc[j];
    return;
  }
  // split inner dimension: partial tiles in shared memory (the stages are idle
  // now), summed in slice order through distributed shared memory
  const int ldp = TC_NMAX + 1;
  float* Ps = reinterpret_cast<float*>(dsm);
#pragma unroll
  for (int j = 0; j < TC_NMAX; ++j) Ps[tid * ldp + j] = acc[j];
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();
  const int rank = (int)cluster.block_rank();
  const int rows_per = TC_M / ns;
  for (int idx = tid; idx < kc_cols * rows_per; idx += TC_THREADS) {
    const int col = idx / rows_per, rr = rank * rows_per + idx % rows_per;
    float v[16];
#pragma unroll
    for (int sl = 0; sl < 16; ++sl) v[sl] = (sl < ns) ? cluster.map_shared_rank(Ps, sl)[rr * ldp + col] : 0.f;
    float sum = 0.f;
#pragma unroll
    for (int sl = 0; sl < 16; ++sl) sum += v[sl];
    const int row = r0 + rr;
    if (row < n) W[(size_t)(c0 + col) * ldw + row] = sum;
  }
  cluster.sync();  // keep every CTA's shared memory alive until all reads are done
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D FP32 tensor map: inner dimension `inner` (contiguous), `outer` rows of
// stride `ld` floats, box `box_inner` x `box_outer`, 128-byte swizzle, zero
// fill outside the tensor.
bool make_map(CUtensorMap* m, const float* base, int inner, int outer, int ld, int box_inner, int box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_tc_cluster_max = 8;  // 16 where the device co-schedules 16-CTA clusters of this kernel

size_t tc_smem_bytes(int nt) {
  const size_t stage = (size_t)TC_M * TC_KC * 4 + 2 * (size_t)nt * TC_KC * 4;
  const size_t need = 1024 + TC_NS * stage + (TC_NS + 2) * sizeof(uint64_t) + 16;
  return need < (size_t)kSmemFloor ? (size_t)kSmemFloor : need;
}

}  // namespace

void init_mv_tc_attributes() {
  cudaFuncSetAttribute(k_block_matvec_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(TC_NMAX));
  if (cudaFuncSetAttribute(k_block_matvec_tc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = tc_smem_bytes(TC_NMAX);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_block_matvec_tc, &cfg) == cudaSuccess && clusters > 0)
      g_tc_cluster_max = 16;
  }
  cudaGetLastError();
}

bool block_matvec_tc_enabled() {
  static const bool off = [] {
    const char* v = getenv("PSDP_BLOCK_PRODUCT");
    return v && std::strcmp(v, "simt") == 0;
  }();
  return !off && encode_fn() != nullptr;
}

bool block_matvec_tc_applies(const float* S, int lds, const float* scratch) {
  return scratch && block_matvec_tc_enabled() && !(lds & 3) && !(reinterpret_cast<uintptr_t>(S) & 15) &&
         !(reinterpret_cast<uintptr_t>(scratch) & 15);
}

size_t block_matvec_tc_scratch_floats(int n, int k) { return 2 * (size_t)((n + 31) / 32 * 32) * (size_t)k; }

// Slices of the inner dimension (= cluster size): the largest power of two
// whose CTAs (two resident per SM) still run in one wave, keeping at least
// two chunks per slice.
static int tc_slices(int n, int tiles, int sms) {
  int ns = 1;
  while (ns < g_tc_cluster_max && tiles * (2 * ns) <= 2 * sms && n >= (2 * ns) * 2 * TC_KC) ns *= 2;
  return ns;
}

bool launch_block_matvec_tc(const float* S, int lds, int n, const float* Q, int ldq, float* W, int ldw, int k,
                            const int* skip, cudaStream_t st, float* scratch, cudaGraphConditionalHandle cond,
                            int set_cond) {
  if (!block_matvec_tc_applies(S, lds, scratch) || n < 1 || k < 1) return false;
  const int ld2 = (n + 31) / 32 * 32;
  float* Qhi = scratch;
  float* Qlo = scratch + (size_t)ld2 * k;
  const int nt = ((std::min(k, TC_NMAX) + 15) / 16) * 16;  // MMA N (multiple of 16) and Q box rows
  CUtensorMap mS, mQh, mQl;
  if (!make_map(&mS, S, n, n, lds, TC_KC, TC_M) || !make_map(&mQh, Qhi, n, k, ld2, TC_KC, nt) ||
      !make_map(&mQl, Qlo, n, k, ld2, TC_KC, nt))
    return false;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  {
    const size_t total = (size_t)n * k;
    int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)sms * 8);
    k_split_tf32<<<blocks, 256, 0, st>>>(Q, ldq, n, k, Qhi, Qlo, ld2, skip);
  }
  const int rb = (n + TC_M - 1) / TC_M, ztiles = (k + TC_NMAX - 1) / TC_NMAX;
  const int ns = tc_slices(n, rb * ztiles, sms);
  const int kslice = ((n + ns - 1) / ns + TC_KC - 1) / TC_KC * TC_KC;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ns, rb, ztiles);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = tc_smem_bytes(nt);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ns;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_block_matvec_tc, mS, mQh, mQl, n, k, W, ldw, nt, kslice, skip, cond, set_cond);
  return true;
}

}  // namespace psdp
