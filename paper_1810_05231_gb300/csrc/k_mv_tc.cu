// k_mv_tc.cu — the block Krylov product W = S Q of the truncated projection
// (Sec. 3.1, Eq. trunc_eig) on the fifth-generation tensor cores.
//
// S (n x n FP32, symmetric, row stride lds) is streamed from HBM once per
// product by TMA in 128-row x 32-column tiles (128-byte swizzle).  Q (n x k)
// is split once per product into TF32 high and low parts (hi = tf32(Q),
// lo = tf32(Q - hi), both rounded to nearest) that TMA streams too.  Each CTA
// owns 128 rows of S and up to 64 columns of Q over one slice of the inner
// dimension; its converter warps split S the same way into tensor memory
// (TMEM) and one thread issues
//     D = S_hi [Q_hi | Q_lo] (+) S_lo Q_hi
// as tcgen05.mma kind::tf32 with A read from TMEM and B from shared memory
// ("3xTF32": the dropped term S_lo Q_lo and the TF32 rounding of the parts are
// O(2^-22) relative, FP32-grade).  Two properties of the tensor cores shape
// the design (both measured on GB300):
//   - they read an FP32 operand as TF32 by truncation, so parts that are not
//     TF32 values already pick up a systematic error (splitting by
//     truncation gave a -3e-7 relative bias in S Q, which raised the PDHG
//     residual floor from 2e-6 to 1.5e-5 on a bipartite MaxCut instance);
//     both parts are therefore rounded to nearest before the MMA;
//   - their FP32 accumulation truncates too (an error growing linearly with
//     the number of accumulations: 5.8e-5 relative over 8192 inner indices),
//     so each 32-wide chunk writes a fresh accumulator that the converter
//     threads add into FP32 registers, rounded to nearest.
// Measured: relative error 1.5e-7 (random data, n = 2000) with a bias of
// -9e-8; the SIMT kernel gives 2e-7 and -1e-9.  Slices of one row block form a
// thread-block cluster whose partial tiles are summed in a fixed CTA order
// through distributed shared memory (deterministic).
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
constexpr int TC_NMAX = 64;      // columns of Q per CTA
constexpr int TC_CONV_WARPS = 8;  // converter warps: two per TMEM lane quarter (one per column half)
constexpr int TC_THREADS = 32 * (TC_CONV_WARPS + 2);  // plus the control and producer warps
constexpr int TC_HALF = TC_NMAX / 2;                  // accumulator columns per converter thread
constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at 2 GHz
constexpr int kSmemTwoPerSm = 80 * 1024;   // floor that keeps at most two CTAs on an SM

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


// 16 consecutive TMEM columns of this thread's lane <- v[0..15]
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// v[0..7] <- 8 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
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

// x (FP32) rounded to the nearest TF32 value (10 explicit mantissa bits;
// halfway cases away from zero), as an FP32 bit pattern whose 13 low bits are
// zero, so the tensor cores read it exactly.
__device__ __forceinline__ uint32_t tf32_rn(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// x = hi + lo + e with hi = tf32(x), lo = tf32(x - hi) (both rounded to
// nearest, so neither part is biased toward zero) and |e| <= 2^-22 |x|.
// Truncating instead leaves every lo with the sign of x and lets the tensor
// cores' own conversion of lo truncate it again: a systematic -3e-7 relative
// error in S Q (measured), which raises the PDHG residual floor.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  const uint32_t h = tf32_rn(x);
  hi = h;
  lo = tf32_rn(x - __uint_as_float(h));
}

}  // namespace

// Q (n x k, column stride ldq) -> Qhi, Qlo (column stride ld2): hi = tf32(Q),
// lo = tf32(Q - hi), both rounded to nearest (split_tf32).
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Converter thread (row_t, column half) results -> W: directly when the
// inner dimension is not split (ns == 1); otherwise the partial tiles of the
// ns CTAs of the cluster (in shared memory, the rings being idle) are summed
// in slice order through distributed shared memory.  Called by every thread.
__device__ __forceinline__ void tc_store_result(const float* acc, unsigned char* dsm, float* __restrict__ W, int ldw,
                                                int n, int r0, int c0, int kc_cols, int hcols, int half, int row_t,
                                                bool conv_thread, int ns, int tid) {
  namespace cg = cooperative_groups;
  if (ns == 1) {
    const int row = r0 + row_t;
    if (conv_thread && row < n)
#pragma unroll
      for (int j = 0; j < TC_HALF; ++j) {
        const int col = half * hcols + j;
        if (j < hcols && col < kc_cols) W[(size_t)(c0 + col) * ldw + row] = acc[j];
      }
    return;
  }
  const int ldp = TC_NMAX + 1;
  float* Ps = reinterpret_cast<float*>(dsm);
  if (conv_thread)
#pragma unroll
    for (int j = 0; j < TC_HALF; ++j)
      if (j < hcols) Ps[row_t * ldp + half * hcols + j] = acc[j];
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

// Warp roles: warps 0-7 ("converters", two per TMEM lane quarter, one per
// half of the columns) read their part of each S tile from shared memory,
// split it and store S_hi | S_lo into an A buffer in TMEM, and add the
// chunk's accumulators into FP32 registers once its MMAs have completed;
// warp 8 ("control", one thread) issues the MMAs; warp 9 ("producer", one
// thread) issues the S tile loads; converter warp 0 also refills the Q ring.
// S tiles and Q tiles live in separate rings: an S stage is free as soon as
// the converters have read it, a Q stage once the MMAs reading it have
// completed, so S can be fetched further ahead.
// Two MMAs per k-step: S_hi [Q_hi | Q_lo] as one MMA of width 2 nt (the Q
// stage holds the two tiles back to back, so they form one K-major operand),
// then S_lo Q_hi into the second half.  An accumulator is 2 nt TMEM columns:
// the first nt sum S_hi Q_hi over the chunk's four k-steps, the next nt the
// two small terms (which therefore never meet the large partial in a
// truncating addition); the converters add both halves into FP32 registers.
// Buffers (two CTAs per SM, 256 TMEM columns each): `nd` accumulators from
// column 0 and `na` A buffers of 64 columns from column 2 nt nd.
//   na = 1, nd = 2 (widths <= 48): the converters store chunk c's S_hi | S_lo
//     once the MMAs of chunk c - 1 have completed and drain chunk c - 1's
//     accumulator while the MMAs of chunk c run;
//   na = 2, nd = 1 (width 64): they store chunk c while the MMAs of chunk c - 1
//     run, then drain chunk c - 1's accumulator before the MMAs of chunk c.
// Handoffs through mbarriers only:
//   fullS[i] / fullQ[j]  TMA -> consumers: the stage holds its tile(s)
//   emptyS[i]            converters -> producer (8 arrivals): S stage read
//   conv[b]              converters -> control (8 arrivals): the A buffer of
//                        chunk c holds it (barrier c & 1, phase c >> 1)
//   done[b]              control (tcgen05.commit) -> converters: the MMAs of
//                        the chunk with parity b have completed
//   drained[b]           converters -> control (nd = 1): the accumulator of
//                        chunk c has been read (barrier c & 1)
// One barrier per chunk parity wherever the other side can be two chunks
// ahead, so that no phase parity aliases.
// Shared memory (base aligned to 1024 B): nss S stages of 16 KB, nqs Q stages
// of [Qhi tile nt*128 B | Qlo tile nt*128 B], the mbarriers, the TMEM address
// slot.
__global__ void __launch_bounds__(TC_THREADS, 2) k_block_matvec_tc(const __grid_constant__ CUtensorMap tmS,
                                                                    const __grid_constant__ CUtensorMap tmQh,
                                                                    const __grid_constant__ CUtensorMap tmQl, int n,
                                                                    int k, float* __restrict__ W, int ldw, int nt,
                                                                    int kslice, int nss, int nqs, int na, int nd,
                                                                    uint32_t tmem_cols, const int* skip,
                                                                    cudaGraphConditionalHandle cond, int set_cond) {
  if (skip && *(volatile const int*)skip) return;  // uniform over the grid
  if (set_cond && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    cudaGraphSetConditional(cond, 1u);
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  unsigned char* dsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ns = gridDim.x;
  const int r0 = blockIdx.y * TC_M;
  const int c0 = blockIdx.z * TC_NMAX;
  const int kc_cols = min(TC_NMAX, k - c0);
  const int kb = blockIdx.x * kslice, ke = min(n, kb + kslice);
  const int nk = ke > kb ? (ke - kb + TC_KC - 1) / TC_KC : 0;
  const uint32_t tileS = TC_M * TC_KC * 4;
  const uint32_t tileQ = (uint32_t)nt * TC_KC * 4;
  unsigned char* ringS = dsm;
  unsigned char* ringQ = dsm + (size_t)nss * tileS;
  uint64_t* fullS = reinterpret_cast<uint64_t*>(ringQ + (size_t)nqs * 2 * tileQ);
  uint64_t* emptyS = fullS + nss;
  uint64_t* fullQ = emptyS + nss;
  // [2]: the A buffer of chunk c holds it (barrier c & 1, phase c >> 1; one
  // barrier per parity, since with two A buffers the converters may run two
  // chunks ahead of the MMAs and a single barrier's phase parity would alias)
  uint64_t* conv = fullQ + nqs;
  uint64_t* done = conv + 2;     // [2]: the MMAs of the chunk with parity b have completed
  uint64_t* drained = done + 2;  // [2]: (one accumulator) the converters have read chunk c's (barrier c & 1)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 2);
  __shared__ int s_fail;
  if (tid == 0) {
    for (int i = 0; i < nss; ++i) {
      mbar_init(&fullS[i], 1);
      mbar_init(&emptyS[i], TC_CONV_WARPS);
    }
    for (int j = 0; j < nqs; ++j) mbar_init(&fullQ[j], 1);
    mbar_init(&conv[0], TC_CONV_WARPS);
    mbar_init(&conv[1], TC_CONV_WARPS);
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    mbar_init(&drained[0], TC_CONV_WARPS);
    mbar_init(&drained[1], TC_CONV_WARPS);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_col = 2u * (uint32_t)nt * (uint32_t)nd;  // the A buffers (na of them, 64 columns each)
  auto issue_q = [&](int j) {                // Q tiles of chunk j into Q stage j % nqs
    unsigned char* st = ringQ + (size_t)(j % nqs) * 2 * tileQ;
    uint64_t* bar = &fullQ[j % nqs];
    mbar_expect_tx(bar, 2 * tileQ);
    const int x = kb + j * TC_KC;
    tma_load_2d(st, &tmQh, bar, x, c0);
    tma_load_2d(st + tileQ, &tmQl, bar, x, c0);
  };
  const int row_t = 32 * (warp & 3) + lane, half = (warp >> 2) & 1;
  const int hcols = nt / 2;
  float acc[TC_HALF];
#pragma unroll
  for (int j = 0; j < TC_HALF; ++j) acc[j] = 0.f;
  int issuedS = 0, issuedQ = 0, committed = -1;
  bool fail = false;
  if (warp < TC_CONV_WARPS) {
    // ------------------------------------------------------------ converters
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    // acc += main + small-term halves of the accumulator of chunk parity b (columns of my half)
    auto drain = [&](int b) {
      const uint32_t col = tmem + 2u * (uint32_t)nt * (uint32_t)(b & (nd - 1)) + (uint32_t)(half * hcols) + lane_off;
#pragma unroll
      for (int h = 0; h < TC_HALF / 8; ++h) {
        if (h * 8 < hcols) {
          uint32_t vm[8], vc[8];
          tmem_ld8(col + 8u * h, vm);
          tmem_ld8(col + (uint32_t)nt + 8u * h, vc);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[8 * h + j] += __uint_as_float(vm[j]) + __uint_as_float(vc[j]);
        }
      }
    };
    if (warp == 0 && lane == 0) issuedQ = min(nqs, nk);  // the control thread issued those
    for (int c = 0; c < nk; ++c) {
      const int si = c % nss;
      bool ok = mbar_wait(&fullS[si], (uint32_t)((c / nss) & 1), kWaitCycles);
      float4 sv[4];
      const unsigned char* srow = ringS + (size_t)si * tileS + row_t * 128;
      if (ok) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          sv[q] = *reinterpret_cast<const float4*>(srow + (((4 * half + q) ^ (row_t & 7)) << 4));
      }
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&emptyS[si]);
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split_tf32(sv[q].x, hi[4 * q], lo[4 * q]);
        split_tf32(sv[q].y, hi[4 * q + 1], lo[4 * q + 1]);
        split_tf32(sv[q].z, hi[4 * q + 2], lo[4 * q + 2]);
        split_tf32(sv[q].w, hi[4 * q + 3], lo[4 * q + 3]);
      }
      // the A buffer of chunk c is free once the MMAs of chunk c - na have
      // completed (with two A buffers, chunk c - 2 also frees the accumulators
      // chunk c will write: drained here, before the store)
      const int cw = c - na;
      if (ok && cw >= 0) ok = mbar_wait(&done[cw & 1], (uint32_t)((cw >> 1) & 1), kWaitCycles);
      ok = __all_sync(0xffffffffu, ok && !*(volatile int*)&s_fail);
      if (!ok) {
        s_fail = 1;
        fail = true;
        break;
      }
      tc_fence_after();
      if (warp == 0 && lane == 0 && cw >= 0 && issuedQ < nk) {  // chunk c - na's Q stage is free
        issue_q(issuedQ);
        ++issuedQ;
      }
      if (nd == 2 && na == 2 && cw >= 0) drain(cw & 1);
      const uint32_t abuf = tmem + a_col + 64u * (uint32_t)(c & (na - 1)) + 16u * (uint32_t)half + lane_off;
      tmem_st16(abuf, hi);
      tmem_st16(abuf + 32u, lo);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[c & 1]);
      if (nd == 2 && na == 1 && c >= 1) drain((c - 1) & 1);  // while the MMAs of chunk c run
      if (nd == 1 && c >= 1) {  // one accumulator: read chunk c - 1's before the MMAs of chunk c start
        const int cp = c - 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&done[cp & 1], (uint32_t)((cp >> 1) & 1), kWaitCycles) &&
                                         !*(volatile int*)&s_fail)) {
          s_fail = 1;
          fail = true;
          break;
        }
        tc_fence_after();
        drain(0);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&drained[cp & 1]);
      }
    }
    if (!fail) {  // the accumulators not drained yet: the last na chunks (one with a single accumulator)
      for (int j = max(0, nk - (nd == 1 ? 1 : na)); j < nk; ++j) {
        if (!__all_sync(0xffffffffu, mbar_wait(&done[j & 1], (uint32_t)((j >> 1) & 1), kWaitCycles))) {
          s_fail = 1;
          fail = true;
          break;
        }
        tc_fence_after();
        drain(j & 1);
      }
    }
  } else if (warp == TC_CONV_WARPS && lane == 0) {
    // ------------------------------------------------------------ control: MMAs
    const uint32_t idesc2 = idesc_tf32(TC_M, 2 * nt), idesc1 = idesc_tf32(TC_M, nt);
    for (; issuedQ < min(nqs, nk); ++issuedQ) issue_q(issuedQ);
    for (int c = 0; c < nk; ++c) {
      const int qj = c % nqs, b = c & 1;
      unsigned char* st = ringQ + (size_t)qj * 2 * tileQ;
      if (!mbar_wait(&fullQ[qj], (uint32_t)((c / nqs) & 1), kWaitCycles) ||
          !mbar_wait(&conv[b], (uint32_t)((c >> 1) & 1), kWaitCycles) ||
          (nd == 1 && c >= 1 && !mbar_wait(&drained[(c - 1) & 1], (uint32_t)(((c - 1) >> 1) & 1), kWaitCycles)) ||
          *(volatile int*)&s_fail) {
        s_fail = 1;
        fail = true;
        break;
      }
      tc_fence_after();
      const uint64_t dq = sdesc_k_sw128(smem_u32(st));  // [Q_hi | Q_lo], 2 nt rows
      const uint32_t dmain = tmem + 2u * (uint32_t)nt * (uint32_t)(b & (nd - 1)), dsmall = dmain + (uint32_t)nt;
      const uint32_t abuf = tmem + a_col + 64u * (uint32_t)(c & (na - 1));
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk)  // S_hi [Q_hi | Q_lo]
        tc_mma_ts(dmain, abuf + 8u * kk, dq + (uint64_t)(kk * 32 >> 4), idesc2, kk > 0 ? 1u : 0u);
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk)  // + S_lo Q_hi into the small half
        tc_mma_ts(dsmall, abuf + 32u + 8u * kk, dq + (uint64_t)(kk * 32 >> 4), idesc1, 1u);
      tc_commit(&done[b]);
      committed = c;
    }
  } else if (warp == TC_CONV_WARPS + 1 && lane == 0) {
    // ------------------------------------------------------------ producer: S tiles
    for (; issuedS < nk; ++issuedS) {
      const int j = issuedS, si = j % nss;
      if (j >= nss && (!mbar_wait(&emptyS[si], (uint32_t)(((j / nss) - 1) & 1), kWaitCycles) ||
                       *(volatile int*)&s_fail)) {
        s_fail = 1;
        fail = true;
        break;
      }
      mbar_expect_tx(&fullS[si], tileS);
      tma_load_2d(ringS + (size_t)si * tileS, &tmS, &fullS[si], kb + j * TC_KC, r0);
    }
  }
  if (__syncthreads_or(fail ? 1 : 0)) {
    fail = true;
    if (warp == 0 && lane == 0) {  // Q loads (issued by the control thread and this one)
      for (int j = max(0, issuedQ - nqs); j < issuedQ; ++j)
        mbar_wait(&fullQ[j % nqs], (uint32_t)((j / nqs) & 1), kWaitCycles / 8);
    }
    if (warp == TC_CONV_WARPS && lane == 0 && committed >= 0)
      mbar_wait(&done[committed & 1], (uint32_t)((committed >> 1) & 1), kWaitCycles / 8);
    if (warp == TC_CONV_WARPS + 1 && lane == 0) {
      for (int j = max(0, issuedS - nss); j < issuedS; ++j)
        mbar_wait(&fullS[j % nss], (uint32_t)((j / nss) & 1), kWaitCycles / 8);
    }
#pragma unroll
    for (int j = 0; j < TC_HALF; ++j) acc[j] = __int_as_float(0x7fc00000);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
  tc_store_result(acc, dsm, W, ldw, n, r0, c0, kc_cols, hcols, half, row_t, warp < TC_CONV_WARPS, ns, tid);
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

int g_smem_max = 227 * 1024 - 1024;  // dynamic shared memory a CTA may use (set from the device at init)

struct TcShape {
  int nss, nqs, na, nd;
  uint32_t tmem_cols;
  size_t smem;
};

// Shared memory of a shape: 1024 B alignment slack, the rings, the barriers.
size_t tc_smem_need(int nt, int nss, int nqs) {
  return 1024 + (size_t)nss * TC_M * TC_KC * 4 + (size_t)nqs * 2 * nt * TC_KC * 4 +
         (size_t)(2 * nss + 2 * nqs + 6) * sizeof(uint64_t) + 16;
}

// Launch shape for a CTA width of nt columns (two CTAs per SM): na / nd as
// described at the kernel (PSDP_TC_NA / PSDP_TC_ND override them for
// measurements), as many S stages as fit beside two Q stages, then up to
// four Q stages.
TcShape tc_shape(int nt, int want_na, int want_nd) {
  TcShape t;
  int na = want_na > 0 ? want_na : (nt <= 48 ? 1 : 2);
  int nd = want_nd > 0 ? want_nd : (nt <= 48 ? 2 : 1);
  if (2 * nt * nd + 64 * na > 256) {  // what fits in 256 columns
    na = 2;
    nd = 1;
  }
  t.na = na;
  t.nd = nd;
  t.tmem_cols = 256;
  const size_t cap = (size_t)(228 * 1024 / 2 - 1024);  // two CTAs per SM
  int nss = 2, nqs = 2;
  while (nss < 8 && tc_smem_need(nt, nss + 1, nqs) <= cap) ++nss;
  while (nqs < 4 && tc_smem_need(nt, nss, nqs + 1) <= cap) ++nqs;
  t.nss = nss;
  t.nqs = nqs;
  const size_t need = tc_smem_need(nt, nss, nqs);
  t.smem = need < (size_t)kSmemTwoPerSm ? (size_t)kSmemTwoPerSm : need;
  return t;
}

int g_tc_na = 0;  // A buffers (0: by width; PSDP_TC_NA overrides: 1 or 2)
int g_tc_nd = 0;  // accumulators (0: by width; PSDP_TC_ND overrides: 1 or 2)
int g_tc_cluster_max = 8;  // 16 where the device co-schedules 16-CTA clusters of this kernel

}  // namespace

void init_mv_tc_attributes() {
  if (const char* v = getenv("PSDP_TC_NA")) g_tc_na = atoi(v) == 1 ? 1 : 2;
  if (const char* v = getenv("PSDP_TC_ND")) g_tc_nd = atoi(v) == 2 ? 2 : 1;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
      cudaFuncGetAttributes(&fa, k_block_matvec_tc) == cudaSuccess)
    g_smem_max = optin - (int)fa.sharedSizeBytes;
  cudaFuncSetAttribute(k_block_matvec_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, g_smem_max);
  if (cudaFuncSetAttribute(k_block_matvec_tc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    const TcShape t = tc_shape(TC_NMAX, g_tc_na, g_tc_nd);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = t.smem;
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

bool block_matvec_tc_applies(const float* S, int lds, int n, const float* scratch) {
  return scratch && n >= kTcMinN && block_matvec_tc_enabled() && !(lds & 3) && !(reinterpret_cast<uintptr_t>(S) & 15) &&
         !(reinterpret_cast<uintptr_t>(scratch) & 15);
}

size_t block_matvec_tc_scratch_floats(int n, int k) { return 2 * (size_t)((n + 31) / 32 * 32) * (size_t)k; }

// Slices of the inner dimension (= cluster size): the largest power of two
// whose CTAs (`per_sm` resident per SM) still run in one wave, keeping at
// least two chunks per slice.
static int tc_slices(int n, int tiles, int sms, int per_sm) {
  int ns = 1;
  while (ns < g_tc_cluster_max && tiles * (2 * ns) <= per_sm * sms && n >= (2 * ns) * 2 * TC_KC) ns *= 2;
  return ns;
}

bool launch_block_matvec_tc(const float* S, int lds, int n, const float* Q, int ldq, float* W, int ldw, int k,
                            const int* skip, cudaStream_t st, float* scratch, cudaGraphConditionalHandle cond,
                            int set_cond) {
  if (!block_matvec_tc_applies(S, lds, n, scratch) || k < 1) return false;
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
  const TcShape shape = tc_shape(nt, g_tc_na, g_tc_nd);
  const int rb = (n + TC_M - 1) / TC_M, ztiles = (k + TC_NMAX - 1) / TC_NMAX;
  const int ns = tc_slices(n, rb * ztiles, sms, 2);
  const int kslice = ((n + ns - 1) / ns + TC_KC - 1) / TC_KC * TC_KC;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ns, rb, ztiles);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = shape.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ns;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_block_matvec_tc, mS, mQh, mQl, n, k, W, ldw, nt, kslice, shape.nss, shape.nqs, shape.na,
                     shape.nd, shape.tmem_cols, skip, cond, set_cond);
  return true;
}

}  // namespace psdp
