// k_lanczos.cu — kernels of the restarted block Lanczos solver behind the
// truncated psd projection aproj(S, r) of Sec. 3.1 (Eq. trunc_eig).
//
// The paper computes the r largest eigenpairs with a Krylov method (ARPACK on
// a CPU, Sec. 3.1 / Sec. 4); here the Krylov basis lives in HBM as FP32
// column blocks, inner products are accumulated exactly-rounded in a pair of
// FP32 numbers (Knuth's TwoSum with the FMA-based TwoProduct of Ogita, Rump &
// Oishi, "Accurate sum and dot product", 2005) and combined across blocks in
// FP64, and the small Rayleigh-Ritz eigenproblem is solved in one thread
// block (Householder tridiagonalisation, bisection, inverse iteration and a
// residual correction).
#include "psdp.cuh"

#include <math.h>

#include <algorithm>

#include <cooperative_groups.h>

namespace psdp {

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 148;
    }
    cached[dev] = v;
  }
  return cached[dev];
}


// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// Pseudo-random uniform in [-1, 1) from (seed, i, j): the splitmix64 finaliser
// (Steele, Lea & Flood 2014) applied to a mixed counter.
__device__ __forceinline__ float hash_uniform(unsigned long long seed, unsigned long long i,
                                              unsigned long long j) {
  unsigned long long x = seed + 0x9E3779B97F4A7C15ULL * (i + 1) + 0xC2B2AE3D27D4EB4FULL * (j + 7);
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ULL;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (float)(x >> 40) * (2.0f / 16777216.0f) - 1.0f;
}

// Accumulator of a sum of exact FP32 products in two FP32 words.
struct DF {
  float hi, lo;
  __device__ __forceinline__ DF() : hi(0.f), lo(0.f) {}
  // s += a * b : the product is split exactly (p + e = a*b) with one FMA and
  // p is added to hi with TwoSum; the rounding errors go to lo.
  __device__ __forceinline__ void fma_acc(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = fmaf(a, b, -p);
    float s = __fadd_rn(hi, p);
    float bb = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------------------
// S * Q block product (SIMT, inner dimension split across a thread-block cluster)
// ---------------------------------------------------------------------------
// CTA tile: 128 rows of S x up to 64 columns of Q over one slice of the inner
// dimension, in chunks of 32.  The S chunk is staged transposed (Ss[k][row],
// the 4-row groups of row k permuted by XOR with k & 28 against bank
// conflicts) so a thread reads its 8 rows as two float4 broadcasts; each thread holds
// 8 rows x G columns (G = column groups of 16).  The `ns` slices of a row
// block form one cluster: their partial tiles stay in shared memory and, after
// a cluster barrier, CTA c of the cluster sums rows [c*128/ns, (c+1)*128/ns)
// over the ns partials through distributed shared memory, in slice order
// (deterministic, no global partials).  S is symmetric, so its row blocks are
// also column blocks.
constexpr int MV_RB = 128, MV_KC = 32, MV_LDS = 132;

template <int G>
__global__ void __launch_bounds__(256) k_block_matvec(const float* __restrict__ S, int lds, int n,
                                                      const float* __restrict__ Q, int ldq,
                                                      float* __restrict__ W, int ldw, int k,
                                                      int kslice, const int* skip,
                                                      cudaGraphConditionalHandle cond, int set_cond) {
  namespace cg = cooperative_groups;
  if (skip && *(volatile const int*)skip) return;  // uniform over the grid: no CTA reaches a barrier
  if (set_cond && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    cudaGraphSetConditional(cond, 1u);
  // staging (S chunk, Q chunk) and, after the main loop, this CTA's partial
  // tile (row-major, 128 x 16G, row stride 16G + 2: the two rows a warp
  // stores per column group land 16 banks apart, so the stores are
  // conflict-free) share one buffer
  constexpr int kStage = MV_KC * MV_LDS + MV_KC * (16 * G + 1);
  constexpr int kLdp = 16 * G + 2;
  constexpr int kPart = MV_RB * kLdp;
  __shared__ __align__(16) float smbuf[kStage > kPart ? kStage : kPart];
  float(*Ss)[MV_LDS] = reinterpret_cast<float(*)[MV_LDS]>(smbuf);
  float(*Qs)[16 * G + 1] = reinterpret_cast<float(*)[16 * G + 1]>(smbuf + MV_KC * MV_LDS);
  float(*Ps)[kLdp] = reinterpret_cast<float(*)[kLdp]>(smbuf);
  const int tid = threadIdx.x;
  const int tc = tid & 15, tr = tid >> 4;  // column within group, row group (8 rows)
  const int ns = gridDim.x;                // slices = cluster size
  const int r0 = blockIdx.y * MV_RB;
  const int c0 = blockIdx.z * 64;
  const int kc = min(16 * G, k - c0);
  const int kb = blockIdx.x * kslice, ke = min(n, kb + kslice);
  float acc[8][G];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int g = 0; g < G; ++g) acc[a][g] = 0.f;
  // Register staging: each thread loads 4 float4 of the S chunk (128 rows x 32
  // columns) and G/2 (rounded up) float4 of the Q chunk, all issued before any
  // is used, and the next chunk's loads are issued before the current chunk
  // is consumed (software pipelining).  Rows of S and columns of Q are read
  // with the inner index contiguous (coalesced 128-byte rows).
  const bool vec = ((lds & 3) == 0) && ((ldq & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(S) & 15) == 0) && ((reinterpret_cast<uintptr_t>(Q) & 15) == 0);
  constexpr int QV = (16 * G * MV_KC / 4 + 255) / 256;  // float4 of Q per thread
  float4 sreg[4], qreg[QV];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int idx = tid + 256 * v;  // 1024 float4 = 128 rows x 8
      const int rr = idx >> 3, kq = (idx & 7) * 4;
      const int gr = r0 + rr, gk = k0 + kq;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < n) {
        const float* src = S + (size_t)gr * lds + gk;
        if (vec && gk + 3 < ke) x = __ldg(reinterpret_cast<const float4*>(src));
        else {
          if (gk < ke) x.x = __ldg(src);
          if (gk + 1 < ke) x.y = __ldg(src + 1);
          if (gk + 2 < ke) x.z = __ldg(src + 2);
          if (gk + 3 < ke) x.w = __ldg(src + 3);
        }
      }
      sreg[v] = x;
    }
#pragma unroll
    for (int v = 0; v < QV; ++v) {
      const int idx = tid + 256 * v;  // 16G columns x 8 float4
      const int cc = idx >> 3, kq = (idx & 7) * 4;
      const int gk = k0 + kq;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (cc < kc) {
        const float* src = Q + (size_t)(c0 + cc) * ldq + gk;
        if (vec && gk + 3 < ke) x = __ldg(reinterpret_cast<const float4*>(src));
        else {
          if (gk < ke) x.x = __ldg(src);
          if (gk + 1 < ke) x.y = __ldg(src + 1);
          if (gk + 2 < ke) x.z = __ldg(src + 2);
          if (gk + 3 < ke) x.w = __ldg(src + 3);
        }
      }
      qreg[v] = x;
    }
  };
  auto store_chunk = [&]() {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int idx = tid + 256 * v;
      // row k of the transposed chunk holds S row rr at column rr ^ (k & 28)
      // (4-float groups permuted by the row: conflict-free transposed stores,
      // float4 reads stay aligned)
      const int rr = idx >> 3, kq = (idx & 7) * 4;
      const int cs = rr ^ kq;
      Ss[kq][cs] = sreg[v].x;
      Ss[kq + 1][cs] = sreg[v].y;
      Ss[kq + 2][cs] = sreg[v].z;
      Ss[kq + 3][cs] = sreg[v].w;
    }
#pragma unroll
    for (int v = 0; v < QV; ++v) {
      const int idx = tid + 256 * v;
      const int cc = idx >> 3, kq = (idx & 7) * 4;
      if (cc < 16 * G) {
        Qs[kq][cc] = qreg[v].x;
        Qs[kq + 1][cc] = qreg[v].y;
        Qs[kq + 2][cc] = qreg[v].z;
        Qs[kq + 3][cc] = qreg[v].w;
      }
    }
  };
  if (kb < ke) load_chunk(kb);
  for (int k0 = kb; k0 < ke; k0 += MV_KC) {
    store_chunk();
    __syncthreads();
    if (k0 + MV_KC < ke) load_chunk(k0 + MV_KC);  // in flight during the compute below
#pragma unroll 4
    for (int kk = 0; kk < MV_KC; ++kk) {
      const float4 s0 = *reinterpret_cast<const float4*>(&Ss[kk][(tr * 8) ^ (kk & 28)]);
      const float4 s1 = *reinterpret_cast<const float4*>(&Ss[kk][(tr * 8 + 4) ^ (kk & 28)]);
      const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const float q = Qs[kk][tc + 16 * g];
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[a][g] = fmaf(sv[a], q, acc[a][g]);
      }
    }
    __syncthreads();
  }
  if (ns == 1) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int col = tc + 16 * g;
      if (col < kc)
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int row = r0 + tr * 8 + a;
          if (row < n) W[(size_t)(c0 + col) * ldw + row] = acc[a][g];
        }
    }
    return;
  }
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int a = 0; a < 8; ++a) Ps[tr * 8 + a][tc + 16 * g] = acc[a][g];
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();
  const int rank = (int)cluster.block_rank();
  const int rows_per = MV_RB / ns;
  for (int idx = tid; idx < kc * rows_per; idx += 256) {
    const int col = idx / rows_per, rr = rank * rows_per + idx % rows_per;
    // all remote loads issued before the additions (slice order kept)
    float v[16];
#pragma unroll
    for (int sl = 0; sl < 16; ++sl) v[sl] = (sl < ns) ? cluster.map_shared_rank(&Ps[0][0], sl)[rr * kLdp + col] : 0.f;
    float sum = 0.f;
#pragma unroll
    for (int sl = 0; sl < 16; ++sl) sum += v[sl];
    const int row = r0 + rr;
    if (row < n) W[(size_t)(c0 + col) * ldw + row] = sum;
  }
  cluster.sync();  // keep every CTA's shared memory alive until all reads are done
}

// Inner-dimension slices per 128-row block: a power of two <= 8 (the cluster
// size), about two CTAs per SM, at least four 32-wide chunks per slice.
static int g_mv_cluster_max = 8;  // 16 where the device co-schedules 16-CTA clusters of this kernel

// Slices of the inner dimension (= cluster size): split until about two CTAs
// per SM, keeping at least two 32-column chunks per slice.
static int matvec_slices(int n, int k) {
  const int tiles = ((n + MV_RB - 1) / MV_RB) * ((k + 63) / 64);
  int ns = 1;
  const int slots = 2 * num_sms();  // two CTAs per SM
  while (ns < g_mv_cluster_max && tiles * (2 * ns) <= slots && n >= (2 * ns) * 2 * MV_KC) ns *= 2;
  return ns;
}

size_t block_matvec_scratch_floats(int n, int k) { return block_matvec_tc_scratch_floats(n, k); }
size_t block_matvec_counters(int, int) { return 0; }

template <int G>
static void launch_mv(dim3 grid, int ns, cudaStream_t st, const float* S, int lds, int n, const float* Q,
                      int ldq, float* W, int ldw, int k, int kslice, const int* skip,
                      cudaGraphConditionalHandle cond, int set_cond) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ns;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_block_matvec<G>, S, lds, n, Q, ldq, W, ldw, k, kslice, skip, cond, set_cond);
}

void launch_block_matvec(const float* S, int lds, int n, const float* Q, int ldq, float* W, int ldw,
                         int k, const int* skip, cudaStream_t st, float* part, unsigned*,
                         cudaGraphConditionalHandle cond, int set_cond) {
  // tensor cores (3xTF32, TMA-staged S) when the scratch for the split Q is
  // given and S meets the TMA alignment rules; the SIMT kernel otherwise
  if (launch_block_matvec_tc(S, lds, n, Q, ldq, W, ldw, k, skip, st, part, cond, set_cond)) return;
  const int ns = matvec_slices(n, k);
  const int kslice = ((n + ns - 1) / ns + MV_KC - 1) / MV_KC * MV_KC;
  dim3 grid(ns, (n + MV_RB - 1) / MV_RB, (k + 63) / 64);
  const int kmax = std::min(k, 64);
  if (kmax <= 16) launch_mv<1>(grid, ns, st, S, lds, n, Q, ldq, W, ldw, k, kslice, skip, cond, set_cond);
  else if (kmax <= 32) launch_mv<2>(grid, ns, st, S, lds, n, Q, ldq, W, ldw, k, kslice, skip, cond, set_cond);
  else if (kmax <= 48) launch_mv<3>(grid, ns, st, S, lds, n, Q, ldq, W, ldw, k, kslice, skip, cond, set_cond);
  else launch_mv<4>(grid, ns, st, S, lds, n, Q, ldq, W, ldw, k, kslice, skip, cond, set_cond);
}

// ---------------------------------------------------------------------------
// random start block
// ---------------------------------------------------------------------------
__global__ void k_random_block(float* Q, int ldq, int n, int col0, int k, unsigned long long seed) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)n * k;
  if (idx >= total) return;
  int c = (int)(idx / n), i = (int)(idx % n);
  Q[(size_t)(col0 + c) * ldq + i] = hash_uniform(seed, (unsigned long long)i, (unsigned long long)(col0 + c));
}

void launch_random_block(float* Q, int ldq, int n, int col0, int k, unsigned long long seed,
                         cudaStream_t st) {
  size_t total = (size_t)n * k;
  int blocks = (int)((total + 255) / 256);
  k_random_block<<<blocks, 256, 0, st>>>(Q, ldq, n, col0, k, seed);
}

// ---------------------------------------------------------------------------
// expansion block of a wide kept block
// ---------------------------------------------------------------------------
// When the kept Ritz block is wider than the Krylov block (w > kMaxW), one
// restart cycle expands the basis by b < w directions: the columns
// (off + j) mod w, j < b, of W = S Q_kept, with the offset advancing by b
// with every restart cycle (the cycle count comes from the control block).
// Orthogonalised against Q_kept they are the residual directions of those b
// Ritz pairs, i.e. one block Lanczos step for them, and over w / b
// successive cycles every kept pair gets one.
__global__ void __launch_bounds__(256) k_compress_block(const float* __restrict__ W, int ldw, int w,
                                                        float* __restrict__ Z, int ldz, int b, int n,
                                                        const Ctl* ctl, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const int off = (int)(((long long)ctl->lz_cycles_total * b) % w);
  const size_t total = (size_t)n * b;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / n), i = (int)(idx % n);
    Z[(size_t)j * ldz + i] = W[(size_t)((off + j) % w) * ldw + i];
  }
}

void launch_compress_block(const float* W, int ldw, int w, float* Z, int ldz, int b, int n, const Ctl* ctl,
                           const int* skip, cudaStream_t st) {
  const size_t total = (size_t)n * b;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  k_compress_block<<<blocks, 256, 0, st>>>(W, ldw, w, Z, ldz, b, n, ctl, skip);
}

// ---------------------------------------------------------------------------
// Gram H = A^T B with exact-product accumulation
// ---------------------------------------------------------------------------
// Grid (output tiles, row splits); the row splits of one 16 x 16 output tile
// form a thread-block cluster.  Each CTA accumulates its rows in FP32 pairs,
// keeps its partial tile in shared memory, and after a cluster barrier CTA c
// adds the partials of its share of the tile over the splits in split order
// through distributed shared memory (deterministic).
constexpr int GR_T = 16, GR_RC = 128;

__global__ void __launch_bounds__(256) k_gram(const float* __restrict__ A, int lda, int ka,
                                              const float* __restrict__ B, int ldb, int kb, int n,
                                              int rows_per_split, double* __restrict__ H, const int* skip,
                                              int act, int slot) {
  namespace cg = cooperative_groups;
  if (skip && *(volatile const int*)skip) return;  // uniform over the grid
  __shared__ float As[GR_RC][GR_T + 1];
  __shared__ float Bs[GR_RC][GR_T + 1];
  __shared__ double Pt[GR_T * GR_T];
  const int tid = threadIdx.x;
  int a0, b0;
  if (act > 0) {
    // only the first `act` columns of every `slot`-wide column group
    const int per = (act + GR_T - 1) / GR_T;
    const int tiles_b = per * (kb / slot);
    const int ta = blockIdx.x / tiles_b, tb = blockIdx.x % tiles_b;
    a0 = (ta / per) * slot + (ta % per) * GR_T;
    b0 = (tb / per) * slot + (tb % per) * GR_T;
  } else {
    const int tiles_b = (kb + GR_T - 1) / GR_T;
    a0 = (blockIdx.x / tiles_b) * GR_T;
    b0 = (blockIdx.x % tiles_b) * GR_T;
  }
  const int ty = tid / GR_T, tx = tid % GR_T;
  const int rbeg = blockIdx.y * rows_per_split;
  const int rend = min(n, rbeg + rows_per_split);
  DF acc;
  // register staging with one chunk of prefetch: each thread issues its
  // GR_RC * 16 / 256 loads of A and of B before the previous chunk is consumed
  constexpr int NL = GR_RC * GR_T / 256;
  float ra[NL], rb[NL];
  auto load_chunk = [&](int i0) {
#pragma unroll
    for (int v = 0; v < NL; ++v) {
      const int idx = tid + 256 * v;
      const int c = idx / GR_RC, i = idx % GR_RC;
      const int gi = i0 + i;
      ra[v] = (gi < rend && a0 + c < ka) ? __ldg(&A[(size_t)(a0 + c) * lda + gi]) : 0.f;
      rb[v] = (gi < rend && b0 + c < kb) ? __ldg(&B[(size_t)(b0 + c) * ldb + gi]) : 0.f;
    }
  };
  if (rbeg < rend) load_chunk(rbeg);
  for (int i0 = rbeg; i0 < rend; i0 += GR_RC) {
#pragma unroll
    for (int v = 0; v < NL; ++v) {
      const int idx = tid + 256 * v;
      const int c = idx / GR_RC, i = idx % GR_RC;
      As[i][c] = ra[v];
      Bs[i][c] = rb[v];
    }
    __syncthreads();
    if (i0 + GR_RC < rend) load_chunk(i0 + GR_RC);
#pragma unroll 8
    for (int i = 0; i < GR_RC; ++i) acc.fma_acc(As[i][ty], Bs[i][tx]);
    __syncthreads();
  }
  const int ns = gridDim.y;
  if (ns == 1) {
    if (a0 + ty < ka && b0 + tx < kb) H[(size_t)(a0 + ty) * kb + b0 + tx] = acc.value();
    return;
  }
  Pt[tid] = acc.value();
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();
  const int rank = (int)cluster.block_rank();
  const int per_rank = (GR_T * GR_T) / ns;
  for (int o = rank * per_rank + tid; o < (rank + 1) * per_rank && tid < per_rank; o += 256) {
    double sum = 0.0;
    for (int sp = 0; sp < ns; ++sp) sum += cluster.map_shared_rank(Pt, sp)[o];
    const int a = a0 + o / GR_T, b = b0 + o % GR_T;
    if (a < ka && b < kb) H[(size_t)a * kb + b] = sum;
  }
  cluster.sync();
}

void launch_gram(const float* A, int lda, int ka, const float* B, int ldb, int kb, int n, double* H,
                 double*, unsigned*, const int* skip, cudaStream_t st, int act, int slot) {
  int tiles = ((ka + GR_T - 1) / GR_T) * ((kb + GR_T - 1) / GR_T);
  if (act > 0) {
    int per = (act + GR_T - 1) / GR_T;
    tiles = per * (ka / slot) * per * (kb / slot);
  }
  // row splits: a power of two <= 8, >= 256 rows each, about one CTA per SM in all
  int ns = 1;
  const int sms = num_sms();
  while (ns < 8 && tiles * ns * 2 <= sms && n >= 2 * ns * 256) ns *= 2;
  const int rows = (n + ns - 1) / ns;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles, ns, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = ns;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_gram, A, lda, ka, B, ldb, kb, n, rows, H, skip, act, slot > 0 ? slot : 1);
}

// ---------------------------------------------------------------------------
// Z -= A * H  (classical Gram-Schmidt update)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_block_update(float* __restrict__ Z, int ldz, int kb,
                                                      const float* __restrict__ A, int lda, int ka,
                                                      const double* __restrict__ H, int n,
                                                      const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ float Hs[];  // ka x kb
  for (int idx = threadIdx.x; idx < ka * kb; idx += blockDim.x) Hs[idx] = (float)H[idx];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= n) return;
  float acc = 0.f;
#pragma unroll 8
  for (int a = 0; a < ka; ++a) acc = fmaf(__ldg(&A[(size_t)a * lda + i]), Hs[a * kb + b], acc);
  Z[(size_t)b * ldz + i] -= acc;
}

void launch_block_update(float* Z, int ldz, int kb, const float* A, int lda, int ka, const double* H,
                         int n, const int* skip, cudaStream_t st) {
  if (ka == 0) return;
  dim3 grid((n + 255) / 256, kb);
  k_block_update<<<grid, 256, (size_t)ka * kb * sizeof(float), st>>>(Z, ldz, kb, A, lda, ka, H, n, skip);
}

// ---------------------------------------------------------------------------
// Cholesky of the w x w Gram (FP64, one CTA) with deficient-column detection
// ---------------------------------------------------------------------------
// G = R^T R with R upper triangular; writes R^{-1} (FP32, w x w row-major,
// upper triangular) and flags[j] = 1 for columns whose remaining norm fell
// below 1e-10 of their original norm (numerically dependent; their row of R
// is taken as e_j).  One barrier per elimination step: the factor is written
// to a separate array so the trailing update reads stay race-free.
__global__ void __launch_bounds__(256) k_chol(const double* __restrict__ G, int w,
                                              float* __restrict__ Rinv_out, int* __restrict__ flags,
                                              const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ double chs[];
  double(*Gs)[kMaxW + 1] = reinterpret_cast<double(*)[kMaxW + 1]>(chs);
  double(*Rs)[kMaxW + 1] = reinterpret_cast<double(*)[kMaxW + 1]>(chs + kMaxW * (kMaxW + 1));
  __shared__ double d0[kMaxW];
  __shared__ int fl[kMaxW];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < w * w; idx += blockDim.x) {
    int i = idx / w, j = idx % w;
    Gs[i][j] = 0.5 * (G[i * w + j] + G[j * w + i]);
    Rs[i][j] = 0.0;
  }
  __syncthreads();
  for (int j = tid; j < w; j += blockDim.x) d0[j] = Gs[j][j];
  __syncthreads();
  __shared__ double s_inv;
  __shared__ int s_def;
  __shared__ double rdiag[kMaxW];
  for (int j = 0; j < w; ++j) {
    if (tid == 0) {  // one FP64 square root / division per step (FP64 specials are slow)
      const double piv = Gs[j][j];
      const bool def = !(piv > 1e-10 * d0[j]) || !(d0[j] > 0.0);
      const double djj = def ? 1.0 : sqrt(piv);
      s_inv = 1.0 / djj;
      s_def = def ? 1 : 0;
      Rs[j][j] = djj;
      rdiag[j] = s_inv;
      fl[j] = s_def;
    }
    __syncthreads();
    const double inv = s_inv;
    const int def = s_def;
    const int rem = w - j - 1;
    for (int l = j + 1 + tid; l < w; l += blockDim.x) Rs[j][l] = def ? 0.0 : Gs[j][l] * inv;
    if (!def)
      for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
        int k = j + 1 + idx / rem, l = j + 1 + idx % rem;
        if (l >= k) Gs[k][l] -= (Gs[j][k] * inv) * (Gs[j][l] * inv);
      }
    __syncthreads();
  }
  for (int j = tid; j < w; j += blockDim.x) flags[j] = fl[j];
  // R^{-1} by columns (thread j solves R x = e_j), staged in the upper part of Gs (free now)
  for (int j = tid; j < w; j += blockDim.x) {
    for (int i = j; i >= 0; --i) {
      double sacc = (i == j) ? 1.0 : 0.0;
      for (int k = i + 1; k <= j; ++k) sacc -= Rs[i][k] * Gs[k][j];
      Gs[i][j] = sacc * rdiag[i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < w * w; idx += blockDim.x) {
    int i = idx / w, j = idx % w;
    Rinv_out[idx] = (j >= i) ? (float)Gs[i][j] : 0.f;
  }
}

constexpr size_t kCholSmem = 2 * (size_t)kMaxW * (kMaxW + 1) * sizeof(double);

void launch_chol_inv(const double* G, int w, float* Rinv, int* flags, const int* skip, cudaStream_t st) {
  k_chol<<<1, 256, kCholSmem, st>>>(G, w, Rinv, flags, skip);
}

// Z <- Z R^{-1} row by row (R^{-1} upper triangular); flagged columns are
// replaced by pseudo-random entries (re-orthogonalised by the caller).
template <int WMAX>
__global__ void __launch_bounds__(128) k_apply_rinv(float* __restrict__ Z, int ldz, int w,
                                                    const float* __restrict__ Ri, const int* flags,
                                                    int n, unsigned long long seed, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  __shared__ float Rs[WMAX * WMAX];
  __shared__ int fl[WMAX];
  for (int idx = threadIdx.x; idx < WMAX * WMAX; idx += blockDim.x) {
    int i = idx / WMAX, j = idx % WMAX;
    Rs[idx] = (i < w && j < w) ? Ri[i * w + j] : 0.f;
  }
  for (int j = threadIdx.x; j < WMAX; j += blockDim.x) fl[j] = (j < w) ? flags[j] : 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float z[WMAX];
#pragma unroll
  for (int k = 0; k < WMAX; ++k) z[k] = (k < w) ? Z[(size_t)k * ldz + i] : 0.f;
#pragma unroll
  for (int j = 0; j < WMAX; ++j) {
    if (j < w) {
      float x = 0.f;
#pragma unroll
      for (int k = 0; k <= j; ++k) x = fmaf(z[k], Rs[k * WMAX + j], x);
      if (fl[j]) x = hash_uniform(seed, (unsigned long long)i, (unsigned long long)(1000 + j));
      Z[(size_t)j * ldz + i] = x;
    }
  }
}

void launch_apply_rinv(float* Z, int ldz, int w, const float* Rinv, const int* flags, int n,
                       unsigned long long seed, const int* skip, cudaStream_t st) {
  const int blocks = (n + 127) / 128;
  if (w <= 16) k_apply_rinv<16><<<blocks, 128, 0, st>>>(Z, ldz, w, Rinv, flags, n, seed, skip);
  else if (w <= 32) k_apply_rinv<32><<<blocks, 128, 0, st>>>(Z, ldz, w, Rinv, flags, n, seed, skip);
  else k_apply_rinv<64><<<blocks, 128, 0, st>>>(Z, ldz, w, Rinv, flags, n, seed, skip);
}

// ---------------------------------------------------------------------------
// Symmetric eigensolver for the Rayleigh-Ritz matrix (one CTA, K <= 128)
// ---------------------------------------------------------------------------
// (1) Householder reduction of T (FP32) to tridiagonal form: for k = 0..K-3
//     the reflector H_k = I - tau_k v_k v_k^T (v_k(0) = 1, acting on rows
//     k+1..K-1) annihilates column k below the subdiagonal, and the trailing
//     block becomes A22 - v w^T - w v^T with p = tau A22 v and
//     w = p - (tau/2)(p^T v) v.
// (2) Eigenvalues of the tridiagonal matrix (scaled to unit infinity norm) by
//     Sturm counts (the number of negative pivots of the LDL^T factorisation
//     of T - x I): one count per thread at evenly spaced points of the
//     Gershgorin interval brackets every eigenvalue, then G threads per
//     eigenvalue narrow its bracket by multisection.
// (3) Eigenvectors of the tridiagonal matrix by inverse iteration: two
//     solves with the partially pivoted LU factorisation of T - lambda I from
//     a pseudo-random start, one thread per isolated eigenvalue.  Eigenvalues
//     closer than kSeGroupTol ||T|| form a group that one warp handles (a lane
//     per member), orthogonalising each member against the previous ones after
//     every solve (modified Gram-Schmidt).
// (4) Back-transformation Y = H_0 H_1 ... H_{K-3} Z.
// (5) One refinement step for the `nout` wanted eigenvectors (Ogita & Aishima,
//     "Iterative refinement for symmetric eigenvalue decomposition", 2018):
//     with Y the eigenvectors, S = Y^T T Y and R = I - Y^T Y accumulated in
//     FP32 pairs against the FP64 input T, lambda_j = S_jj / (1 - R_jj) and
//     y_j <- y_j + sum_i y_i E_ij,  E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)
//     (E_ij = R_ij / 2 for i = j or nearly equal eigenvalues), followed by a
//     symmetric orthonormality correction.
constexpr int JB = 32;  // wanted columns refined per pass
constexpr int SE_THREADS = 512;
constexpr float kSePivmin = 1e-30f;   // Sturm pivots below this (unit-norm matrix) count as negative
constexpr float kSeGroupTol = 2e-5f;  // inverse-iteration groups (unit-norm matrix)
constexpr double kRefineBelow = 5e-6;  // adaptive refinement: Ritz residual tolerances below this

// Number of eigenvalues of the tridiagonal (d, e2 = squared off-diagonal) below x.
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int K, float x) {
  float q = d[0] - x;
  if (fabsf(q) < kSePivmin) q = -kSePivmin;
  int c = (q < 0.f);
  for (int i = 1; i < K; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < kSePivmin) q = -kSePivmin;
    c += (q < 0.f);
  }
  return c;
}

// Numbers of eigenvalues of the tridiagonal (d, e2 = squared off-diagonal)
// below x0 and below x1 (two interleaved Sturm sequences).
__device__ __forceinline__ void sturm_count2(const float* d, const float* e2, int K, float x0, float x1,
                                             int& c0, int& c1) {
  float q0 = d[0] - x0, q1 = d[0] - x1;
  if (fabsf(q0) < kSePivmin) q0 = -kSePivmin;
  if (fabsf(q1) < kSePivmin) q1 = -kSePivmin;
  int n0 = (q0 < 0.f), n1 = (q1 < 0.f);
  for (int i = 1; i < K; ++i) {
    const float di = d[i], ei = e2[i - 1];
    q0 = (di - x0) - __fdividef(ei, q0);
    q1 = (di - x1) - __fdividef(ei, q1);
    if (fabsf(q0) < kSePivmin) q0 = -kSePivmin;
    if (fabsf(q1) < kSePivmin) q1 = -kSePivmin;
    n0 += (q0 < 0.f);
    n1 += (q1 < 0.f);
  }
  c0 = n0;
  c1 = n1;
}

// Partially pivoted LU factorisation of the tridiagonal T - lam I (diagonal
// d, off-diagonal e), rows eliminated top-down: U has two superdiagonals;
// u0 holds the reciprocals of the pivots.
struct TriLU {
  float u0[kMaxK], u1[kMaxK], u2[kMaxK], l[kMaxK];
  unsigned sw[kMaxK / 32];
};

__device__ void tri_lu(const float* d, const float* e, int K, float lam, float tiny, TriLU& f) {
  float p0 = d[0] - lam, p1 = (K > 1) ? e[0] : 0.f;
  for (int w = 0; w < kMaxK / 32; ++w) f.sw[w] = 0u;
  for (int i = 0; i < K - 1; ++i) {
    const float s0 = e[i], s1 = d[i + 1] - lam, s2 = (i + 2 < K) ? e[i + 1] : 0.f;
    if (fabsf(p0) >= fabsf(s0)) {  // the current row is the pivot row
      if (p0 == 0.f) p0 = tiny;
      const float l = s0 / p0;
      f.u0[i] = 1.f / p0;
      f.u1[i] = p1;
      f.u2[i] = 0.f;
      f.l[i] = l;
      p0 = s1 - l * p1;
      p1 = s2;
    } else {  // rows i and i+1 swap
      const float l = p0 / s0;
      f.u0[i] = 1.f / s0;
      f.u1[i] = s1;
      f.u2[i] = s2;
      f.l[i] = l;
      f.sw[i >> 5] |= 1u << (i & 31);
      p0 = p1 - l * s1;
      p1 = -l * s2;
    }
  }
  f.u0[K - 1] = 1.f / ((p0 == 0.f) ? tiny : p0);
}

// x <- (T - lam I)^{-1} x for the factorisation above; x has stride ld > 0
// (loads of x issued one step ahead of the store before them).
__device__ void tri_solve(const TriLU& f, int K, float* x, int ld) {
  float a = x[0];  // the current row's entry, carried in a register
  float bn = (K > 1) ? x[ld] : 0.f;
  for (int i = 0; i < K - 1; ++i) {
    float b = bn;
    if (i + 2 < K) bn = x[(i + 2) * ld];
    if ((f.sw[i >> 5] >> (i & 31)) & 1u) {
      const float t = a;
      a = b;
      b = t;
    }
    x[i * ld] = a;
    a = fmaf(-f.l[i], a, b);
  }
  float x2 = 0.f, x1 = a * f.u0[K - 1];
  float xn = (K > 1) ? x[(K - 2) * ld] : 0.f;
  x[(K - 1) * ld] = x1;
  for (int i = K - 2; i >= 0; --i) {
    const float xv = xn;
    if (i > 0) xn = x[(i - 1) * ld];
    const float xi = (xv - f.u1[i] * x1 - f.u2[i] * x2) * f.u0[i];
    x[i * ld] = xi;
    x2 = x1;
    x1 = xi;
  }
}

// The same factorisation stored compactly in shared memory, one slot per
// thread (slot-interleaved arrays: entry i of slot s at i * ns + s): the
// multiplier l_i, the reciprocal pivot of row i and the swap bit.  The rest
// of U is rebuilt from d, e and lam during the solve: a swapped row i is
// (e_i, d_{i+1} - lam, e_{i+1}); an unswapped row is (p0_i, p1_i, 0) with
// p1_i = e_i after an unswapped row (or at i = 0) and -l_{i-1} e_i after a
// swapped one.
__device__ void tri_lu_slot(const float* __restrict__ d, const float* __restrict__ e, int K, float lam, float tiny,
                            float* __restrict__ lm, float* __restrict__ rp, unsigned* __restrict__ sw, int ns,
                            int s) {
  float p0 = d[0] - lam, p1 = (K > 1) ? e[0] : 0.f;
  for (int w = 0; w < (K + 31) / 32; ++w) sw[w * ns + s] = 0u;
  unsigned bits = 0u;
  for (int i = 0; i < K - 1; ++i) {
    const float s0 = e[i], s1 = d[i + 1] - lam, s2 = (i + 2 < K) ? e[i + 1] : 0.f;
    float l;
    if (fabsf(p0) >= fabsf(s0)) {
      if (p0 == 0.f) p0 = tiny;
      const float rcp = __frcp_rn(p0);  // one reciprocal per step, shared by l and the pivot
      l = s0 * rcp;
      rp[i * ns + s] = rcp;
      p0 = s1 - l * p1;
      p1 = s2;
    } else {
      const float rcp = __frcp_rn(s0);
      l = p0 * rcp;
      rp[i * ns + s] = rcp;
      bits |= 1u << (i & 31);
      p0 = p1 - l * s1;
      p1 = -l * s2;
    }
    lm[i * ns + s] = l;
    if ((i & 31) == 31 || i == K - 2) {  // flush a full word, or the last one
      sw[(i >> 5) * ns + s] = bits;
      bits = 0u;
    }
  }
  rp[(K - 1) * ns + s] = __frcp_rn((p0 == 0.f) ? tiny : p0);
}

// x holds the right-hand side on entry (stride ld > 0) and the solution on
// exit.  Every load of x is issued one step ahead of the store before it (the
// entries differ), which keeps the memory latency off the recurrence.
__device__ void tri_solve_slot(const float* __restrict__ d, const float* __restrict__ e, int K, float lam,
                               const float* __restrict__ lm, const float* __restrict__ rp,
                               const unsigned* __restrict__ sw, int ns, int s, float* x, int ld) {
  float a = x[0];
  float bn = (K > 1) ? x[ld] : 0.f;
  for (int i = 0; i < K - 1; ++i) {
    float b = bn;
    if (i + 2 < K) bn = x[(i + 2) * ld];
    if ((sw[(i >> 5) * ns + s] >> (i & 31)) & 1u) {
      const float t = a;
      a = b;
      b = t;
    }
    x[i * ld] = a;
    a = fmaf(-lm[i * ns + s], a, b);
  }
  float x2 = 0.f, x1 = a * rp[(K - 1) * ns + s];
  float xn = (K > 1) ? x[(K - 2) * ld] : 0.f;
  x[(K - 1) * ld] = x1;
  for (int i = K - 2; i >= 0; --i) {
    const float xv = xn;
    if (i > 0) xn = x[(i - 1) * ld];
    const bool swp = (sw[(i >> 5) * ns + s] >> (i & 31)) & 1u;
    float u1, u2;
    if (swp) {
      u1 = d[i + 1] - lam;
      u2 = (i + 2 < K) ? e[i + 1] : 0.f;
    } else {
      const bool prev_swp = (i > 0) && ((sw[((i - 1) >> 5) * ns + s] >> ((i - 1) & 31)) & 1u);
      u1 = prev_swp ? -lm[(i - 1) * ns + s] * e[i] : e[i];
      u2 = 0.f;
    }
    const float xi = (xv - u1 * x1 - u2 * x2) * rp[i * ns + s];
    x[i * ld] = xi;
    x2 = x1;
    x1 = xi;
  }
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Normalise column q of V (K entries, stride ld) with the whole warp; a zero
// or non-finite column is refilled with pseudo-random entries first.
__device__ void warp_normalise(float* V, int ld, int K, int q, int lane, unsigned long long salt) {
  float mx = 0.f;
  for (int i = lane; i < K; i += 32) mx = fmaxf(mx, fabsf(V[i * ld + q]));
  mx = warp_max_f(mx);
  if (!(mx > 0.f) || !(mx < 3e38f)) {
    for (int i = lane; i < K; i += 32) V[i * ld + q] = hash_uniform(0xBADULL + salt, (unsigned long long)i, 78ULL);
    mx = 1.f;
  }
  const float im = 1.f / mx;
  float ss = 0.f;
  for (int i = lane; i < K; i += 32) {
    const float v = V[i * ld + q] * im;
    ss = fmaf(v, v, ss);
  }
  ss = warp_sum_f(ss);
  const float sc = im * rsqrtf(ss);
  for (int i = lane; i < K; i += 32) V[i * ld + q] *= sc;
  __syncwarp();
}

__global__ void __launch_bounds__(SE_THREADS) k_sym_eig(const double* __restrict__ Tin, int K, int Kp,
                                                        double* __restrict__ theta, float* __restrict__ Yout,
                                                        int ldy, int nout, int refine, const double* adapt_tol,
                                                        const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  // adaptive mode: refine only when the projection's tolerance is below what
  // the FP32 eigenpairs reach by themselves
  if (adapt_tol) refine = (*(volatile const double*)adapt_tol < kRefineBelow) ? 1 : 0;
  extern __shared__ float smj[];
  const int ld = Kp + 1;
  float* A = smj;                      // Kp x (Kp+1): T, then the Householder vectors
  float* V = A + (size_t)Kp * ld;      // Kp x (Kp+1): eigenvectors (columns)
  float* td = V + (size_t)Kp * ld;     // Kp: tridiagonal diagonal (scaled)
  float* te = td + Kp;                 // Kp: off-diagonal (scaled)
  float* te2 = te + Kp;                // Kp: squared off-diagonal
  float* tau = te2 + Kp;               // Kp
  float* vb = tau + Kp;                // 2 Kp: Householder vectors of steps k and k+1
  float* pb = vb + 2 * Kp;             // Kp: p = tau A22 v
  float* blo = pb + Kp;                // Kp: eigenvalue brackets, then scaled eigenvalues
  float* bhi = blo + Kp;               // Kp
  float* dg = bhi + Kp;                // Kp: eigenvalue estimates (unscaled)
  int* slice = reinterpret_cast<int*>(dg + Kp);  // 2 SE_THREADS: Sturm counts of the slicing pass
  int* flg = slice + 2 * SE_THREADS;   // 2 x 2 SE_THREADS: multisection flags (double-buffered)
  int* rank = flg + 4 * SE_THREADS;    // Kp
  int* wanted = rank + Kp;             // JB
  int* gsz = wanted + JB;              // Kp: size of the group starting at a (0 inside a group)
  int* glist = gsz + Kp;               // Kp: starts of the groups with two or more members
  double* red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(glist + Kp) + 7) & ~uintptr_t(7));
  double* lamj = red + 64;             // JB
  float* scr = reinterpret_cast<float*>(lamj + JB);  // refinement scratch: Tl, Zh, Zl
  __shared__ float s_norm, s_gl, s_gu;
  __shared__ int s_ng;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;

  for (int idx = tid; idx < K * K; idx += nth) {
    const int i = idx / K, j = idx % K;
    A[i * ld + j] = (float)(0.5 * (Tin[i * K + j] + Tin[j * K + i]));
  }
  __syncthreads();

  // ---- (1) tridiagonalisation
  // Householder vector of column k below the diagonal (warp 0): v (v(0) = 1,
  // also stored in A's column k), tau[k], te[k] = beta, td[k] = A_kk
  auto householder = [&](int k, float* v) {
    const int m = K - k - 1;
    float ss = 0.f;
    for (int i = 1 + lane; i < m; i += 32) {
      const float x = A[(k + 1 + i) * ld + k];
      ss = fmaf(x, x, ss);
    }
    ss = warp_sum_f(ss);
    const float x0 = A[(k + 1) * ld + k];
    float t = 0.f, beta = x0, scal = 0.f;
    if (ss > 0.f) {
      beta = -copysignf(sqrtf(x0 * x0 + ss), x0);
      t = (beta - x0) / beta;
      scal = 1.f / (x0 - beta);
    }
    for (int i = lane; i < m; i += 32) {
      const float vv = (i == 0) ? 1.f : A[(k + 1 + i) * ld + k] * scal;
      v[i] = vv;
      A[(k + 1 + i) * ld + k] = vv;
    }
    if (lane == 0) {
      tau[k] = t;
      te[k] = beta;
      td[k] = A[k * ld + k];
    }
  };
  if (K >= 3 && warp == 0) householder(0, vb);
  __syncthreads();
  for (int k = 0; k + 2 < K; ++k) {
    const int m = K - k - 1;
    const float* v = vb + (k & 1) * Kp;
    float* vn = vb + ((k + 1) & 1) * Kp;
    const float tk = tau[k];
    if (tk != 0.f) {  // uniform
      {  // p = tau A22 v: four threads per row
        const int i = tid >> 2, part = tid & 3;
        float acc = 0.f, acc1 = 0.f;
        if (i < m) {
          // blocks of 8 columns, 32 apart: the 32 lanes (8 rows x 4 parts)
          // then touch 32 different banks
          const float* row = A + (size_t)(k + 1 + i) * ld + (k + 1);
          for (int jb = 8 * part; jb < m; jb += 32) {
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
              if (jb + u < m) acc = fmaf(row[jb + u], v[jb + u], acc);
              if (jb + u + 1 < m) acc1 = fmaf(row[jb + u + 1], v[jb + u + 1], acc1);
            }
          }
        }
        acc += acc1;
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (i < m && part == 0) pb[i] = tk * acc;
      }
      __syncthreads();
      // w = p - (tau/2)(p^T v) v, with (p^T v) reduced by every warp itself
      float pv = 0.f;
      for (int i = lane; i < m; i += 32) pv = fmaf(pb[i], v[i], pv);
      const float kk = 0.5f * tk * warp_sum_f(pv);
      if (warp == 0) {
        // column k+1 (local column 0), kept in registers (m <= 127: four rows
        // per lane), and from it the next Householder vector in the same pass
        const float v0 = v[0], w0 = pb[0] - kk * v0;
        float nv[4];
        float ss = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = lane + 32 * q;
          nv[q] = 0.f;
          if (i < m) {
            const float wi = pb[i] - kk * v[i];
            nv[q] = fmaf(-v[i], w0, fmaf(-wi, v0, A[(k + 1 + i) * ld + (k + 1)]));
            if (i >= 2) ss = fmaf(nv[q], nv[q], ss);
          }
        }
        if (k + 3 < K) {
          ss = warp_sum_f(ss);
          const float x0 = __shfl_sync(0xffffffffu, nv[0], 1);  // local row 1
          float t = 0.f, beta = x0, scal = 0.f;
          if (ss > 0.f) {
            beta = -copysignf(sqrtf(x0 * x0 + ss), x0);
            t = __fdividef(beta - x0, beta);
            scal = __frcp_rn(x0 - beta);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            if (i == 0) {
              A[(k + 1) * ld + (k + 1)] = nv[q];
            } else if (i < m) {
              const float vv = (i == 1) ? 1.f : nv[q] * scal;
              vn[i - 1] = vv;
              A[(k + 1 + i) * ld + (k + 1)] = vv;
            }
          }
          if (lane == 0) {
            tau[k + 1] = t;
            te[k + 1] = beta;
            td[k + 1] = nv[0];
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            if (i < m) A[(k + 1 + i) * ld + (k + 1)] = nv[q];
          }
        }
      } else {
        // the next trailing block (local rows and columns 1..m-1); local row 0
        // (the upper part of row k+1) is never read again
        for (int i = warp; i < m; i += nwarps - 1) {  // warps 1.. take rows 1, 2, ...
          const float vi = v[i], wi = pb[i] - kk * vi;
          float* arow = &A[(k + 1 + i) * ld + (k + 1)];
#pragma unroll 2
          for (int j = 1 + lane; j < m; j += 32) {
            const float vj = v[j], wj = pb[j] - kk * vj;
            arow[j] = fmaf(-vi, wj, fmaf(-wi, vj, arow[j]));
          }
        }
      }
      __syncthreads();
    } else {
      if (warp == 0 && k + 3 < K) householder(k + 1, vn);
      __syncthreads();
    }
  }
  if (tid == 0) {
    if (K >= 2) {
      td[K - 2] = A[(K - 2) * ld + (K - 2)];
      te[K - 2] = A[(K - 1) * ld + (K - 2)];
      tau[K - 2] = 0.f;
    }
    td[K - 1] = A[(K - 1) * ld + (K - 1)];
    tau[K - 1] = 0.f;
    float nrm = 0.f;
    for (int i = 0; i < K; ++i) {
      float r = fabsf(td[i]);
      if (i > 0) r += fabsf(te[i - 1]);
      if (i + 1 < K) r += fabsf(te[i]);
      nrm = fmaxf(nrm, r);
    }
    s_norm = (nrm > 0.f) ? nrm : 1.f;
  }
  __syncthreads();
  // scale to unit infinity norm
  const float tn = s_norm, itn = 1.f / s_norm;
  for (int i = tid; i < K; i += nth) {
    td[i] *= itn;
    const float ei = (i + 1 < K) ? te[i] * itn : 0.f;
    te[i] = ei;
    te2[i] = ei * ei;
  }
  __syncthreads();
  if (tid == 0) {
    float gl = 0.f, gu = 0.f;
    for (int i = 0; i < K; ++i) {
      float r = 0.f;
      if (i > 0) r += fabsf(te[i - 1]);
      if (i + 1 < K) r += fabsf(te[i]);
      gl = (i == 0) ? td[i] - r : fminf(gl, td[i] - r);
      gu = (i == 0) ? td[i] + r : fmaxf(gu, td[i] + r);
    }
    const float pad = 4e-6f * fmaxf(fabsf(gl), fabsf(gu)) + 1e-20f;
    s_gl = gl - pad;
    s_gu = gu + pad;
  }
  __syncthreads();

  // ---- (2) eigenvalues: slicing pass (one point per thread), then
  // multisection of the wanted eigenvalues only (a >= a_need: the nout
  // largest, or all of them when the vectors are refined)
  const int a_need = refine ? 0 : max(0, K - nout);
  const float gl = s_gl, gu = s_gu;
  const int P = nth;
  {
    const float x0 = gl + (gu - gl) * (float)(tid + 1) / (float)(P + 1);
    const float x1 = gl + (gu - gl) * (float)(((tid + nth / 2) % nth) + 1) / (float)(P + 1);
    int c0, c1;
    if (tid < nth / 2) {  // two interleaved sequences per thread of the lower half
      sturm_count2(td, te2, K, x0, x1, c0, c1);
      slice[tid] = c0;
      slice[tid + nth / 2] = c1;
    }
  }
  __syncthreads();
  for (int a = tid; a < K; a += nth) {  // bracket of the a-th smallest eigenvalue
    // last slice point with count <= a (binary search; counts are non-decreasing)
    int lo = -1, hi = P;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (slice[mid] <= a) lo = mid;
      else hi = mid;
    }
    blo[a] = (lo < 0) ? gl : gl + (gu - gl) * (float)(lo + 1) / (float)(P + 1);
    bhi[a] = (hi >= P) ? gu : gl + (gu - gl) * (float)(hi + 1) / (float)(P + 1);
    if (bhi[a] < blo[a]) bhi[a] = blo[a];
  }
  __syncthreads();
  {
    const int nw = K - a_need;
    const int G = nth / nw;  // threads (= points) per wanted eigenvalue, >= 4
    const int a = a_need + tid / G, g = tid % G;
    const bool act = a < K;
    float lo = act ? blo[a] : 0.f, hi = act ? bhi[a] : 0.f;
    int steps = 0;
    for (long span = 1; span < 32768; span *= (G + 1)) ++steps;
    for (int st = 0; st < steps; ++st) {
      int* f = flg + (st & 1) * 2 * SE_THREADS;
      if (act) {
        const float x = lo + (hi - lo) * (float)(g + 1) / (float)(G + 1);
        f[(a - a_need) * G + g] = (sturm_count(td, te2, K, x) <= a) ? 1 : 0;
      }
      __syncthreads();
      if (act) {
        float nlo = lo, nhi = hi;
        for (int q = 0; q < G; ++q) {
          const float x = lo + (hi - lo) * (float)(q + 1) / (float)(G + 1);
          if (f[(a - a_need) * G + q]) nlo = fmaxf(nlo, x);
          else nhi = fminf(nhi, x);
        }
        lo = nlo;
        hi = fmaxf(nhi, nlo);
      }
    }
    if (act && g == 0) {
      blo[a] = 0.5f * (lo + hi);  // scaled eigenvalue
      dg[a] = 0.5f * (lo + hi) * tn;
    }
    for (int b = tid; b < a_need; b += nth) {  // unwanted: the bracket's midpoint
      blo[b] = 0.5f * (blo[b] + bhi[b]);
      dg[b] = blo[b] * tn;
    }
  }
  __syncthreads();

  // ---- (3) eigenvectors of the tridiagonal matrix by inverse iteration
  // Only the eigenvalues a >= a_need are wanted (all with refinement); groups
  // of eigenvalues closer than kSeGroupTol are handled by one warp each.
  const float* lam = blo;
  if (tid == 0) {
    int ng = 0;
    for (int a = 0; a < a_need; ++a) gsz[a] = 0;
    for (int a = a_need; a < K;) {
      int last = a;
      while (last + 1 < K && lam[last + 1] - lam[last] <= kSeGroupTol) ++last;
      gsz[a] = last - a + 1;
      for (int b = a + 1; b <= last; ++b) gsz[b] = 0;
      if (last > a) glist[ng++] = a;
      a = last + 1;
    }
    s_ng = ng;
  }
  __syncthreads();
  // isolated eigenvalues: one thread each, two solves (each multiplies the
  // wanted component by at least gap / |lambda error| > 100 against any
  // other: eigenvalues closer than kSeGroupTol go to the group path); LU
  // factors in shared-memory slots (the refinement scratch), in batches of ns.
  // The groups go to the warps that hold no isolated slot.
  const int nwords = (K + 31) / 32;
  const int ns = min(nth, (int)((Kp * (Kp + 1) / 2 + 2 * Kp * JB) / (2 * K + nwords)));
  const int wbusy = min(nwarps - 1, (min(ns, K - a_need) + 31) / 32);
  {
    float* lm = scr;
    float* rp = lm + (size_t)K * ns;
    unsigned* swb = reinterpret_cast<unsigned*>(rp + (size_t)K * ns);
    for (int b0 = a_need; b0 < K; b0 += ns) {
      const int b = b0 + tid;
      if (tid < ns && b < K && gsz[b] == 1) {
        tri_lu_slot(td, te, K, lam[b], 1.2e-7f, lm, rp, swb, ns, tid);
        float* x = V + b;  // column b, stride ld
        for (int i = 0; i < K; ++i)
          x[i * ld] = hash_uniform(0x5EEDULL + (unsigned long long)b, (unsigned long long)i, 77ULL);
        for (int it = 0; it < 2; ++it) {
          tri_solve_slot(td, te, K, lam[b], lm, rp, swb, ns, tid, x, ld);
          float mx = 0.f;
          for (int i = 0; i < K; ++i) mx = fmaxf(mx, fabsf(x[i * ld]));
          if (!(mx > 0.f) || !(mx < 3e38f)) {
            for (int i = 0; i < K; ++i)
              x[i * ld] = hash_uniform(0xBADULL + (unsigned long long)(b * 8 + it), (unsigned long long)i, 78ULL);
            continue;
          }
          float ss = 0.f;
          const float im = 1.f / mx;
#pragma unroll 4
          for (int i = 0; i < K; ++i) {
            const float v = x[i * ld] * im;
            ss = fmaf(v, v, ss);
          }
          const float is = rsqrtf(ss);
          float xn = x[0];
          for (int i = 0; i < K; ++i) {
            const float xv = xn;
            if (i + 1 < K) xn = x[(i + 1) * ld];
            x[i * ld] = (xv * im) * is;
          }
        }
      }
    }
  }
  for (int gi = warp - wbusy; warp >= wbusy && gi < s_ng; gi += nwarps - wbusy) {  // groups: lane = member, MGS in member order
    const int a0 = glist[gi], c = gsz[a0];
    for (int base = a0; base < a0 + c; base += 32) {
      const int cc = min(32, a0 + c - base);
      const int b = base + lane;
      const bool act = lane < cc;
      TriLU f;
      if (act) {
        tri_lu(td, te, K, lam[b], 1.2e-7f, f);
        for (int i = 0; i < K; ++i)
          V[i * ld + b] = hash_uniform(0x5EEDULL + (unsigned long long)b, (unsigned long long)i, 77ULL);
      }
      for (int it = 0; it < 2; ++it) {
        if (act) tri_solve(f, K, V + b, ld);
        __syncwarp();
        for (int q = a0; q < base + cc; ++q) {
          if (q >= base) warp_normalise(V, ld, K, q, lane, (unsigned long long)(q * 8 + it));
          if (act && b > q) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            int i = 0;
#pragma unroll 2
            for (; i + 3 < K; i += 4) {
#pragma unroll
              for (int u = 0; u < 4; ++u) d[u] = fmaf(V[(i + u) * ld + b], V[(i + u) * ld + q], d[u]);
            }
            for (; i < K; ++i) d[0] = fmaf(V[i * ld + b], V[i * ld + q], d[0]);
            const float dot = (d[0] + d[1]) + (d[2] + d[3]);
#pragma unroll 8
            for (int r = 0; r < K; ++r) V[r * ld + b] = fmaf(-dot, V[r * ld + q], V[r * ld + b]);
          }
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();

  // ---- (4) back-transformation V <- H_0 ... H_{K-3} V: each warp applies all
  // reflectors (last first) to its own columns, four at a time, two
  // reflectors per reduction round: with a = v_b^T y, b = v_a^T y and
  // c = v_a^T v_b, H_a H_b y = y - tau_b a v_b - tau_a (b - tau_b a c) v_a
  {
    float* pc = pb;  // c for the pair (k - 1, k), at index k - 1
    for (int k0 = warp; k0 + 1 <= K - 3; k0 += nwarps) {
      float c = 0.f;
      for (int i = k0 + 2 + lane; i < K; i += 32) c = fmaf(A[i * ld + k0], A[i * ld + k0 + 1], c);
      c = warp_sum_f(c);
      if (lane == 0) pc[k0] = c;
    }
    __syncthreads();
    const int ncols = K - a_need;
    for (int c0 = warp; c0 < ncols; c0 += 4 * nwarps) {
      int col[4];
      bool use[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = c0 + u * nwarps;
        use[u] = j < ncols;
        col[u] = use[u] ? a_need + j : a_need + c0;
      }
      for (int k = K - 3; k >= 0; k -= 2) {
        const int kb = k, ka = k - 1;  // H_kb first, then H_ka
        const float tb = tau[kb], ta = (ka >= 0) ? tau[ka] : 0.f;
        if (tb == 0.f && ta == 0.f) continue;
        const int i0 = (ka >= 0) ? ka + 1 : kb + 1;
        float av[4] = {0.f, 0.f, 0.f, 0.f}, bv[4] = {0.f, 0.f, 0.f, 0.f};
        for (int i = i0 + lane; i < K; i += 32) {
          const float v1 = (i >= kb + 1) ? A[i * ld + kb] : 0.f;
          const float v0 = (ka >= 0) ? A[i * ld + ka] : 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float yv = V[i * ld + col[u]];
            av[u] = fmaf(v1, yv, av[u]);
            bv[u] = fmaf(v0, yv, bv[u]);
          }
        }
        const float cc = (ka >= 0) ? pc[ka] : 0.f;
        float s1[4], s0[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float a = warp_sum_f(av[u]), bb = warp_sum_f(bv[u]);
          s1[u] = tb * a;
          s0[u] = ta * (bb - tb * a * cc);
        }
        for (int i = i0 + lane; i < K; i += 32) {
          const float v1 = (i >= kb + 1) ? A[i * ld + kb] : 0.f;
          const float v0 = (ka >= 0) ? A[i * ld + ka] : 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (use[u]) V[i * ld + col[u]] = fmaf(-s1[u], v1, fmaf(-s0[u], v0, V[i * ld + col[u]]));
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  if (!refine) {
    // the FP32 eigenpairs in descending order, with one symmetric
    // orthonormality correction Y <- Y (3I - G)/2, G = Y^T Y (inverse
    // iteration leaves eigenvectors of eigenvalues closer than ~1e-3 ||T||
    // apart non-orthogonal to O(eps ||T|| / gap); mixing inside such pairs
    // changes V diag(lambda) V^T only by O(eps ||T||))
    float* Yr = A;    // Yr[row * nout + j] (A is free after the back-transformation)
    float* IG = scr;  // (I - G)[i * nout + j]
    for (int o = tid; o < K * nout; o += nth) {
      const int j = o % nout, row = o / nout;
      Yr[row * nout + j] = V[row * ld + (K - 1 - j)];
    }
    __syncthreads();
    for (int o = tid; o < nout * nout; o += nth) {
      const int i = o / nout, j = o % nout;
      if (j < i) continue;
      float g[4] = {0.f, 0.f, 0.f, 0.f};
      int k = 0;
#pragma unroll 2
      for (; k + 3 < K; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) g[u] = fmaf(Yr[(k + u) * nout + i], Yr[(k + u) * nout + j], g[u]);
      }
      for (; k < K; ++k) g[0] = fmaf(Yr[k * nout + i], Yr[k * nout + j], g[0]);
      const float v = (i == j ? 1.f : 0.f) - ((g[0] + g[1]) + (g[2] + g[3]));
      IG[i * nout + j] = v;
      IG[j * nout + i] = v;
    }
    __syncthreads();
    for (int o = tid; o < K * nout; o += nth) {  // consecutive threads: consecutive j (no bank conflicts)
      const int row = o / nout, j = o % nout;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      int i = 0;
#pragma unroll 2
      for (; i + 3 < nout; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = fmaf(Yr[row * nout + i + u], IG[(i + u) * nout + j], c[u]);
      }
      for (; i < nout; ++i) c[0] = fmaf(Yr[row * nout + i], IG[i * nout + j], c[0]);
      V[row * ld + j] = Yr[row * nout + j] + 0.5f * ((c[0] + c[1]) + (c[2] + c[3]));
    }
    __syncthreads();
    for (int o = tid; o < K * nout; o += nth) {
      const int j = o / K, row = o % K;
      Yout[(size_t)j * ldy + row] = V[row * ld + j];
    }
    for (int j = tid; j < nout; j += nth) theta[j] = (double)dg[K - 1 - j];
    return;
  }

  // ---- (5) refinement of the wanted vectors: one first-order correction
  // from accurately computed residuals.  With y_j the estimate of the j-th
  // largest eigenvector, z = T y_j is accumulated in FP32 pairs against
  // T = Th + Tl (T rounded to FP32 plus its rounding remainder),
  // theta_j = y_j^T z / y_j^T y_j in FP64, r_j = z - theta_j y_j, and
  //   y_j <- y_j + sum_{i : |theta_j - lambda_i| > delta} y_i (y_i^T r_j) / (theta_j - lambda_i)
  // (the first-order eigenvector perturbation; once r_j is formed, FP32
  // suffices); eigenvalues closer than delta are left to the orthonormality
  // correction below.
  float scale = 0.f;
  for (int i = 0; i < K; ++i) scale = fmaxf(scale, fabsf(dg[i]));
  const float delta = 1e-3f * fmaxf(scale, 1e-30f);
  float* Th = A;                             // K x K, stride ld (A is free now)
  float* Tl = scr;                           // packed upper triangle, K (K+1) / 2
  float* Zh = Tl + Kp * (Kp + 1) / 2;        // K x JB
  float* Zl = Zh + Kp * JB;                  // K x JB
  for (int idx = tid; idx < K * K; idx += nth) {
    const int i = idx / K, j = idx % K;
    const double t = 0.5 * (Tin[i * K + j] + Tin[j * K + i]);
    const float hi = (float)t;
    Th[i * ld + j] = hi;
    if (i <= j) Tl[j * (j + 1) / 2 + i] = (float)(t - (double)hi);
  }
  __syncthreads();
  for (int j0 = 0; j0 < nout; j0 += JB) {
    const int nb = min(JB, nout - j0);
    for (int o = tid; o < K * nb; o += nth) {  // z = T y_j
      const int k = o / nb, jj = o % nb;
      const int col = K - 1 - (j0 + jj);
      DF acc0, acc1;  // two interleaved halves of the sum
      float lo0 = 0.f, lo1 = 0.f;
      const float* th = Th + k * ld;
      int l = 0;
#pragma unroll 2
      for (; l + 1 < K; l += 2) {
        acc0.fma_acc(th[l], V[l * ld + col]);
        acc1.fma_acc(th[l + 1], V[(l + 1) * ld + col]);
      }
      if (l < K) acc0.fma_acc(th[l], V[l * ld + col]);
      const int pk = k * (k + 1) / 2;  // Tl(k, l) for l < k, then Tl(l, k) for l >= k
#pragma unroll 4
      for (int q = 0; q < k; ++q) lo0 = fmaf(Tl[pk + q], V[q * ld + col], lo0);
      int pl = pk + k;
      for (int q = k; q < K; ++q) {
        lo1 = fmaf(Tl[pl], V[q * ld + col], lo1);
        pl += q + 1;
      }
      // (hi0 + hi1) exactly as a pair, then the low parts
      const float sh = acc0.hi + acc1.hi;
      const float bb = sh - acc0.hi;
      const float eh = (acc0.hi - (sh - bb)) + (acc1.hi - bb);
      Zh[k * JB + jj] = sh;
      Zl[k * JB + jj] = eh + acc0.lo + acc1.lo + lo0 + lo1;
    }
    __syncthreads();
    for (int jj = warp; jj < nb; jj += nwarps) {  // theta_j: FP64 Rayleigh quotient
      const int col = K - 1 - (j0 + jj);
      double num = 0.0, den = 0.0;
      for (int k = lane; k < K; k += 32) {
        const double y = (double)V[k * ld + col];
        num += y * ((double)Zh[k * JB + jj] + (double)Zl[k * JB + jj]);
        den += y * y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
      }
      if (lane == 0) lamj[jj] = (den > 0.0) ? num / den : 0.0;
    }
    __syncthreads();
    for (int o = tid; o < K * nb; o += nth) {  // r = z - theta y (into Zh)
      const int k = o / nb, jj = o % nb;
      const int col = K - 1 - (j0 + jj);
      const double th = lamj[jj];
      const float thh = (float)th, thl = (float)(th - (double)thh);
      const float y = V[k * ld + col];
      Zh[k * JB + jj] = fmaf(-thh, y, Zh[k * JB + jj]) + fmaf(-thl, y, Zl[k * JB + jj]);
    }
    __syncthreads();
    for (int o = tid; o < K * nb; o += nth) {  // e_ij = y_i^T r_j / (theta_j - lambda_i) (into Zl)
      const int i = o / nb, jj = o % nb;
      const int col = K - 1 - (j0 + jj);
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      int k = 0;
#pragma unroll 2
      for (; k + 3 < K; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) d[u] = fmaf(V[(k + u) * ld + i], Zh[(k + u) * JB + jj], d[u]);
      }
      for (; k < K; ++k) d[0] = fmaf(V[k * ld + i], Zh[k * JB + jj], d[0]);
      const float gap = (float)lamj[jj] - dg[i];
      Zl[i * JB + jj] = (i == col || fabsf(gap) <= delta) ? 0.f : ((d[0] + d[1]) + (d[2] + d[3])) / gap;
    }
    __syncthreads();
    for (int o = tid; o < K * nb; o += nth) {  // y_j + Y e_j
      const int row = o / nb, jj = o % nb;
      const int col = K - 1 - (j0 + jj);
      float a[4] = {V[row * ld + col], 0.f, 0.f, 0.f};
      int i = 0;
#pragma unroll 2
      for (; i + 3 < K; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = fmaf(V[row * ld + i + u], Zl[(i + u) * JB + jj], a[u]);
      }
      for (; i < K; ++i) a[0] = fmaf(V[row * ld + i], Zl[i * JB + jj], a[0]);
      Yout[(size_t)(j0 + jj) * ldy + row] = (a[0] + a[1]) + (a[2] + a[3]);
    }
    for (int jj = tid; jj < nb; jj += nth) theta[j0 + jj] = lamj[jj];
    __syncthreads();
  }
  // Symmetric orthonormality correction of the refined vectors (the first-
  // order correction leaves O(E^2) non-orthogonality): with G = Y^T Y from
  // FP32-pair sums, Y <- Y (3I - G) / 2, which maps G to I + O((G - I)^2).
  // The refined vectors are staged in A (K x nout), I - G in the refinement
  // scratch (nout x nout), the corrected vectors in V.
  float* Yr = A;    // Yr[row * nout + j]
  float* IG = scr;  // (I - G)[i * nout + j]
  for (int o = tid; o < K * nout; o += nth) {
    const int row = o / nout, j = o % nout;
    Yr[row * nout + j] = __ldcg(&Yout[(size_t)j * ldy + row]);
  }
  __syncthreads();
  for (int o = tid; o < nout * nout; o += nth) {
    const int i = o / nout, j = o % nout;
    if (j < i) continue;
    DF g0, g1;
    int k = 0;
#pragma unroll 2
    for (; k + 1 < K; k += 2) {
      g0.fma_acc(Yr[k * nout + i], Yr[k * nout + j]);
      g1.fma_acc(Yr[(k + 1) * nout + i], Yr[(k + 1) * nout + j]);
    }
    if (k < K) g0.fma_acc(Yr[k * nout + i], Yr[k * nout + j]);
    const float v = (float)((i == j ? 1.0 : 0.0) - (g0.value() + g1.value()));
    IG[i * nout + j] = v;
    IG[j * nout + i] = v;
  }
  __syncthreads();
  for (int o = tid; o < K * nout; o += nth) {
    const int row = o / nout, j = o % nout;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    int i = 0;
#pragma unroll 2
    for (; i + 3 < nout; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] = fmaf(Yr[row * nout + i + u], IG[(i + u) * nout + j], c[u]);
    }
    for (; i < nout; ++i) c[0] = fmaf(Yr[row * nout + i], IG[i * nout + j], c[0]);
    V[row * ld + j] = Yr[row * nout + j] + 0.5f * ((c[0] + c[1]) + (c[2] + c[3]));
  }
  __syncthreads();
  for (int o = tid; o < K * nout; o += nth) {
    const int j = o / K, row = o % K;
    Yout[(size_t)j * ldy + row] = V[row * ld + j];
  }
}

static size_t sym_eig_smem(int Kp) {
  const size_t ld = Kp + 1;
  const size_t f = 2 * (size_t)Kp * ld + 10 * (size_t)Kp;          // A, V, ten vectors
  const size_t ints = 6 * (size_t)SE_THREADS + 3 * (size_t)Kp + JB;  // slice, flags, rank, gsz, glist, wanted
  const size_t scr = (size_t)Kp * (Kp + 1) / 2 + 2 * (size_t)Kp * JB;  // Tl, Zh, Zl
  return f * sizeof(float) + ints * sizeof(int) + 8 + (64 + JB) * sizeof(double) + scr * sizeof(float);
}

void init_lanczos_attributes() {
  init_orth_attributes();
  {
    cudaFuncSetAttribute(k_block_matvec<1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_block_matvec<2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_block_matvec<3>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_block_matvec<4>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    g_mv_cluster_max = (cudaOccupancyMaxActiveClusters(&nc, k_block_matvec<4>, &cfg) == cudaSuccess && nc > 0) ? 16 : 8;
    cudaGetLastError();
  }
  cudaFuncSetAttribute(k_sym_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sym_eig_smem(kMaxK));
  cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmem);
}

void launch_sym_eig(const double* T, int K, double* theta, float* Y, int ldy, int nout,
                    const int* skip, cudaStream_t st, int refine, const double* adapt_tol) {
  const int Kp = (K + 1) & ~1;
  k_sym_eig<<<1, SE_THREADS, sym_eig_smem(Kp), st>>>(T, K, Kp, theta, Y, ldy, nout, refine, adapt_tol, skip);
}

}  // namespace psdp

namespace psdp {

// ---------------------------------------------------------------------------
// Block orthogonalisation in one thread-block cluster
// ---------------------------------------------------------------------------
// Z (n x W, column stride ldq, read from `src`) is orthogonalised against the
// orthonormal basis Q[:, :c0] and within itself by `passes` rounds of
//   H = Q^T Z,  Z <- Z - Q H,  G = Z^T Z,  then either
//   (Cholesky-QR)   D = diag(G), D^{-1/2} G D^{-1/2} = R^T R, Z <- Z D^{-1/2} R^{-1}
//   (Newton-Schulz) Z <- Z (3I - G) / 2, which maps G = I + E to I + O(E^2),
// and written to Q[:, c0:c0+W].  The first pass of a call with chol_first
// uses Cholesky-QR; every other pass uses the Newton-Schulz step when
// max |G - I| <= 0.1 and Cholesky-QR otherwise.  The C CTAs of one cluster
// each keep a slice of rows of Z and of Q[:, :c0] in shared memory for the
// whole call.  H and G are per-CTA partial sums, combined through
// distributed shared memory: CTA c adds slice c of the entries over the C
// partials in CTA order (deterministic), then every CTA gathers the full
// matrix, so every CTA takes the same decisions.  The Cholesky factor of the
// unit-diagonal Gram matrix is computed in FP32 by one warp with the matrix in
// registers; a pivot below kOrthDefTol marks its
// column as dependent, and that column is replaced by pseudo-random entries
// which the next pass orthogonalises.
constexpr float kOrthDefTol = 1e-5f;
constexpr float kOrthNsTol = 0.1f;

struct OrthLayout {
  int rows, ldr, ldqs, c0;
  size_t zs, qs, tmp, ph, pg, hf, gd, rf, total;  // byte offsets
};

__host__ __device__ inline OrthLayout orth_layout(int rows, int c0, int W) {
  OrthLayout L;
  L.rows = rows;
  L.c0 = c0;
  L.ldr = ((rows + 3) / 4) * 4 + 1;  // column-major Z: odd stride, row-per-thread access conflict-free
  L.ldqs = ((rows + 3) / 4) * 4 + 4;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += (bytes + 15) & ~size_t(15);
    return at;
  };
  L.zs = take((size_t)W * L.ldr * 4);
  L.qs = take((size_t)(c0 > 0 ? c0 : 1) * L.ldqs * 4);
  L.tmp = take(8192 * 4);  // split-row partial tiles: <= max(c0*W, 3*48*48, 7*32*32, 25*16*16) floats
  L.ph = take((size_t)(c0 > 0 ? c0 : 1) * W * 4);
  L.pg = take((size_t)W * W * 8);
  L.hf = take((size_t)(c0 > 0 ? c0 : 1) * W * 4);
  L.gd = take((size_t)W * W * 4);
  L.rf = take((size_t)W * W * 4);
  L.total = o;
  return L;
}

// Sum over the C CTAs of a cluster of entry o of `part` (in CTA order); the
// C remote loads are issued before the additions.
template <typename T>
__device__ __forceinline__ T cluster_sum(cooperative_groups::cluster_group& cl, T* part, int C, int o) {
  T v[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = (c < C) ? cl.map_shared_rank(part, c)[o] : T(0);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 16; ++c) s += v[c];
  return s;
}

// One elimination step J of the warp Cholesky below (a template so that every
// register index is a compile-time constant: the matrix never leaves registers).
template <int W, int NC, int J>
__device__ __forceinline__ void chol_warp_step(float (&g)[NC][W], float* R, float* rd, int* fl,
                                               const double* d0s, int lane) {
  if constexpr (J < W) {
    const float piv = __shfl_sync(0xffffffffu, g[J / 32][J], J % 32);
    const bool def = !(piv > kOrthDefTol);
    const float inv = def ? 0.f : rsqrtf(piv);
    float rj[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int l = lane + 32 * c;
      rj[c] = (l > J) ? g[c][J] * inv : 0.f;
      if (l < W) R[J * W + l] = (l == J) ? (def ? 1.f : piv * inv) : rj[c];
    }
    if (lane == 0) {
      rd[J] = def ? 1.f : inv;
      fl[J] = (def || d0s[J] <= 0.0) ? 1 : 0;
    }
#pragma unroll
    for (int k = J + 1; k < W; ++k) {
      const float rjk = __shfl_sync(0xffffffffu, rj[k / 32], k % 32);
#pragma unroll
      for (int c = 0; c < NC; ++c) g[c][k] = fmaf(-rjk, rj[c], g[c][k]);
    }
    chol_warp_step<W, NC, J + 1>(g, R, rd, fl, d0s, lane);
  }
}

// Cholesky of the unit-diagonal W x W matrix in G (upper triangle read) by one
// warp, lane l holding columns l and l + 32 in registers; R (upper, row-major)
// overwrites G, 1/R_jj goes to rd, dependency flags to fl.
template <int W>
__device__ __forceinline__ void chol_warp(float* G, float* rd, int* fl, const double* d0s, int lane) {
  constexpr int NC = (W + 31) / 32;
  float g[NC][W];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int l = lane + 32 * c;
#pragma unroll
    for (int k = 0; k < W; ++k) g[c][k] = (l < W && k <= l) ? G[k * W + l] : 0.f;
  }
  __syncwarp();
  chol_warp_step<W, NC, 0>(g, G, rd, fl, d0s, lane);
}

template <int W>
__global__ void __launch_bounds__(256, 1) k_orth_cluster(float* __restrict__ Q, int ldq, const float* src, int n,
                                                      int c0, int rows, int passes, int chol_first,
                                                      unsigned long long seed, const int* skip) {
  namespace cg = cooperative_groups;
  if (skip && *(volatile const int*)skip) return;  // uniform over the grid
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const OrthLayout L = orth_layout(rows, c0, W);
  extern __shared__ __align__(16) unsigned char osm[];
  float* Zs = reinterpret_cast<float*>(osm + L.zs);
  float* Qs = reinterpret_cast<float*>(osm + L.qs);
  float* Tmp = reinterpret_cast<float*>(osm + L.tmp);
  float* PartH = reinterpret_cast<float*>(osm + L.ph);
  double* PartG = reinterpret_cast<double*>(osm + L.pg);
  float* Hf = reinterpret_cast<float*>(osm + L.hf);
  float* Gh = reinterpret_cast<float*>(osm + L.gd);  // scaled Gram (upper), then R
  float* X = reinterpret_cast<float*>(osm + L.rf);   // Newton-Schulz factor
  __shared__ float sc[W], rd[W];
  __shared__ double d0s[W];
  __shared__ int fl[W];
  __shared__ unsigned s_dev;  // max |G - I| as float bits (non-negative)
  const int tid = threadIdx.x;
  const int ldr = L.ldr, ldqs = L.ldqs;
  const int i0 = rank * rows;
  const int nr = max(0, min(rows, n - i0));
  const int rows4 = ((rows + 3) / 4) * 4;
  // stage my rows of Z (row-major) and of Q[:, :c0] (column-major); padding rows are zero
#pragma unroll 4
  for (int idx = tid; idx < rows4 * W; idx += 256) {
    const int b = idx / rows4, i = idx % rows4;
    Zs[b * ldr + i] = (i < nr) ? __ldg(&src[(size_t)b * ldq + i0 + i]) : 0.f;
  }
#pragma unroll 4
  for (int idx = tid; idx < rows4 * c0; idx += 256) {
    const int a = idx / rows4, i = idx % rows4;
    Qs[a * ldqs + i] = (i < nr) ? __ldg(&Q[(size_t)a * ldq + i0 + i]) : 0.f;
  }
  __syncthreads();
  constexpr int nTb = W / 4;
  for (int pass = 0; pass < passes; ++pass) {
    // without the H phase, no cluster barrier separates the previous pass's
    // gather of PartG from this pass's partial writes
    if (c0 == 0 && pass > 0) cluster.sync();
    if (c0 > 0) {
      // ---- partial H = Qs^T Zs: 4x4 register tiles, rows split over idle threads
      const int nT = (c0 / 4) * nTb;
      const int rs = max(1, 256 / nT);
      const int rlen = (rows4 + rs - 1) / rs;
      const int cw = c0 * W;
      if (tid < nT * rs) {
        const int t = tid % nT, p = tid / nT;
        const int ta = t / nTb, tb = t % nTb;
        float acc[4][4] = {};
        const int ib = p * rlen, ie = min(rows4, ib + rlen);
#pragma unroll 4
        for (int i = ib; i < ie; ++i) {
          const float4 z = make_float4(Zs[(4 * tb) * ldr + i], Zs[(4 * tb + 1) * ldr + i],
                                       Zs[(4 * tb + 2) * ldr + i], Zs[(4 * tb + 3) * ldr + i]);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float q = Qs[(4 * ta + k) * ldqs + i];
            acc[k][0] = fmaf(q, z.x, acc[k][0]);
            acc[k][1] = fmaf(q, z.y, acc[k][1]);
            acc[k][2] = fmaf(q, z.z, acc[k][2]);
            acc[k][3] = fmaf(q, z.w, acc[k][3]);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          *reinterpret_cast<float4*>(&Tmp[p * cw + (4 * ta + k) * W + 4 * tb]) =
              make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
      }
      __syncthreads();
      for (int o = tid; o < cw; o += 256) {
        float s = 0.f;
        for (int p = 0; p < rs; ++p) s += Tmp[p * cw + o];
        PartH[o] = s;
      }
      cluster.sync();
      // reduce-scatter (slice `rank` of the entries, summed in CTA order), then all-gather
      const int chunk = (cw + C - 1) / C;
      for (int o = rank * chunk + tid; o < min(cw, (rank + 1) * chunk); o += 256)
        PartH[o] = cluster_sum(cluster, PartH, C, o);  // only this CTA touches slice `rank` now
      cluster.sync();
      for (int o0 = tid; o0 < cw; o0 += 4 * 256) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int o = o0 + 256 * u;
          v[u] = (o < cw) ? cluster.map_shared_rank(PartH, o / chunk)[o] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (o0 + 256 * u < cw) Hf[o0 + 256 * u] = v[u];
      }
      __syncthreads();
      // ---- Zs <- Zs - Qs Hf on my rows (4x4 tiles)
      const int nU = (rows4 / 4) * nTb;
      for (int t = tid; t < nU; t += 256) {
        const int ti = t / nTb, tb = t % nTb;
        float acc[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[k][u] = Zs[(4 * tb + u) * ldr + 4 * ti + k];
        }
#pragma unroll 4
        for (int a = 0; a < c0; ++a) {
          const float4 q = *reinterpret_cast<const float4*>(&Qs[a * ldqs + 4 * ti]);
          const float4 h = *reinterpret_cast<const float4*>(&Hf[a * W + 4 * tb]);
          const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[k][0] = fmaf(-qv[k], h.x, acc[k][0]);
            acc[k][1] = fmaf(-qv[k], h.y, acc[k][1]);
            acc[k][2] = fmaf(-qv[k], h.z, acc[k][2]);
            acc[k][3] = fmaf(-qv[k], h.w, acc[k][3]);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int u = 0; u < 4; ++u) Zs[(4 * tb + u) * ldr + 4 * ti + k] = acc[k][u];
      }
      __syncthreads();
    }
    // ---- partial G = Zs^T Zs on the upper 4x4 tiles
    {
      const int nT = nTb * (nTb + 1) / 2;
      const int rs = max(1, 256 / nT);
      const int rlen = (rows4 + rs - 1) / rs;
      const int ww = W * W;
      if (tid < nT * rs) {
        int t = tid % nT;
        const int p = tid / nT;
        int ta = 0;
        while (t >= nTb - ta) {
          t -= nTb - ta;
          ++ta;
        }
        const int tb = ta + t;
        float acc[4][4] = {};
        const int ib = p * rlen, ie = min(rows4, ib + rlen);
#pragma unroll 4
        for (int i = ib; i < ie; ++i) {
          const float4 za = make_float4(Zs[(4 * ta) * ldr + i], Zs[(4 * ta + 1) * ldr + i],
                                        Zs[(4 * ta + 2) * ldr + i], Zs[(4 * ta + 3) * ldr + i]);
          const float4 zb = make_float4(Zs[(4 * tb) * ldr + i], Zs[(4 * tb + 1) * ldr + i],
                                        Zs[(4 * tb + 2) * ldr + i], Zs[(4 * tb + 3) * ldr + i]);
          const float av[4] = {za.x, za.y, za.z, za.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[k][0] = fmaf(av[k], zb.x, acc[k][0]);
            acc[k][1] = fmaf(av[k], zb.y, acc[k][1]);
            acc[k][2] = fmaf(av[k], zb.z, acc[k][2]);
            acc[k][3] = fmaf(av[k], zb.w, acc[k][3]);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          *reinterpret_cast<float4*>(&Tmp[p * ww + (4 * ta + k) * W + 4 * tb]) =
              make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
      }
      __syncthreads();
      for (int o = tid; o < ww; o += 256) {
        const int a = o / W, b = o % W;
        double s = 0.0;
        if (a / 4 <= b / 4)
          for (int p = 0; p < rs; ++p) s += (double)Tmp[p * ww + o];
        PartG[o] = s;
      }
      if (tid == 0) s_dev = 0u;
      cluster.sync();
      const int chunk = (ww + C - 1) / C;
      for (int o = rank * chunk + tid; o < min(ww, (rank + 1) * chunk); o += 256)
        PartG[o] = cluster_sum(cluster, PartG, C, o);
      cluster.sync();
      // gather the diagonal first (for the scaling), then the upper triangle:
      // scaled into Gh, and max |G - I| for the choice of the orthonormalisation
      for (int j = tid; j < W; j += 256) {
        const int o = j * W + j;
        const double d = cluster.map_shared_rank(PartG, o / chunk)[o];
        d0s[j] = d;
        sc[j] = (d > 0.0) ? (float)(1.0 / sqrt(d)) : 0.f;
      }
      __syncthreads();
      float dev = 0.f;
      for (int o0 = tid; o0 < ww; o0 += 4 * 256) {
        float v[4];  // the reduced entries are FP64; the scaled Gram is FP32 (FP64 is 1/64 rate here)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int o = o0 + 256 * u;
          v[u] = (o < ww && (o / W) <= (o % W)) ? (float)cluster.map_shared_rank(PartG, o / chunk)[o] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int o = o0 + 256 * u;
          if (o < ww) {
            const int a = o / W, b = o % W;
            Gh[o] = (a <= b) ? v[u] * sc[a] * sc[b] : 0.f;
            if (a <= b) dev = fmaxf(dev, fabsf(v[u] - (a == b ? 1.f : 0.f)));
          }
        }
      }
      if (!(dev == dev)) dev = 3e38f;
      atomicMax(&s_dev, __float_as_uint(dev));
      __syncthreads();
    }
    const bool newton = !(pass == 0 && chol_first) && (__uint_as_float(s_dev) <= kOrthNsTol);  // CTA-uniform
    const unsigned long long pseed = seed * 131ULL + (unsigned long long)(pass * 7 + c0);
    if (newton) {
      // ---- Z <- Z (3I - G)/2, one row per thread; G from the unscaled upper triangle
      for (int o = tid; o < W * W; o += 256) {
        const int a = o / W, b = o % W;
        const int lo = min(a, b), hi = max(a, b);
        const float g = (sc[lo] > 0.f && sc[hi] > 0.f) ? Gh[lo * W + hi] / (sc[lo] * sc[hi]) : 0.f;
        X[o] = (a == b ? 1.5f : 0.f) - 0.5f * g;
      }
      __syncthreads();
      for (int i = tid; i < nr; i += 256) {
        float y[W];
#pragma unroll
        for (int l = 0; l < W; ++l) y[l] = 0.f;
        for (int k = 0; k < W; ++k) {
          const float zk = Zs[k * ldr + i];
#pragma unroll
          for (int m = 0; m < W / 4; ++m) {
            const float4 x = *reinterpret_cast<const float4*>(&X[k * W + 4 * m]);
            y[4 * m + 0] = fmaf(zk, x.x, y[4 * m + 0]);
            y[4 * m + 1] = fmaf(zk, x.y, y[4 * m + 1]);
            y[4 * m + 2] = fmaf(zk, x.z, y[4 * m + 2]);
            y[4 * m + 3] = fmaf(zk, x.w, y[4 * m + 3]);
          }
        }
#pragma unroll
        for (int m = 0; m < W / 4; ++m)
#pragma unroll
          for (int u = 0; u < 4; ++u) Zs[(4 * m + u) * ldr + i] = y[4 * m + u];
      }
    } else {
      // ---- Cholesky of the unit-diagonal Gram matrix by warp 0, the matrix
      // in registers (R written over Gh's upper triangle)
      if (tid < 32) chol_warp<W>(Gh, rd, fl, d0s, tid);
      __syncthreads();
      // ---- Z <- Z D^{-1/2} R^{-1} by forward substitution, one row per thread
      // (x_j = (z_j - sum_{k<j} x_k R_kj) / R_jj; dependent columns get pseudo-random entries)
      for (int i = tid; i < nr; i += 256) {
        float* zr = Zs + i;  // column-major: entry k of this row at zr[k * ldr]
        for (int j = 0; j < W; ++j) {
          float sa[4] = {zr[j * ldr] * sc[j], 0.f, 0.f, 0.f};
          int k = 0;
#pragma unroll 2
          for (; k + 3 < j; k += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) sa[u] = fmaf(-zr[(k + u) * ldr], Gh[(k + u) * W + j], sa[u]);
          }
          for (; k < j; ++k) sa[0] = fmaf(-zr[k * ldr], Gh[k * W + j], sa[0]);
          float x = ((sa[0] + sa[1]) + (sa[2] + sa[3])) * rd[j];
          if (fl[j]) x = hash_uniform(pseed, (unsigned long long)(i0 + i), (unsigned long long)(1000 + j));
          zr[j * ldr] = x;
        }
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nr * W; idx += 256) {
    const int b = idx / nr, i = idx % nr;
    Q[(size_t)(c0 + b) * ldq + i0 + i] = Zs[b * ldr + i];
  }
  cluster.sync();  // no CTA exits while another may still read its shared memory
}

constexpr size_t kOrthSmemMax = 200 * 1024;
static int g_orth_cluster_max = 8;  // largest cluster size the device can co-schedule

template <int W>
static void orth_attr() {
  cudaFuncSetAttribute(k_orth_cluster<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOrthSmemMax);
  cudaFuncSetAttribute(k_orth_cluster<W>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

void init_orth_attributes() {
  orth_attr<16>();
  orth_attr<32>();
  orth_attr<48>();
  orth_attr<64>();
  // can a 16-CTA cluster with the largest footprint be scheduled?
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = kOrthSmemMax;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_orth_cluster<64>, &cfg) == cudaSuccess && nclusters > 0)
    g_orth_cluster_max = 16;
  else
    g_orth_cluster_max = 8;
  cudaGetLastError();
}

// Cluster size and rows per CTA for the fused kernel, or 0 if it does not apply.
static int orth_plan(int n, int c0, int w, int* csize) {
  if (w % 16 != 0 || w > kMaxW || c0 % 16 != 0 || c0 + w > kMaxK) return 0;
  for (int C = 8; C <= g_orth_cluster_max; C *= 2) {
    const int rows = (n + C - 1) / C;
    if (C < g_orth_cluster_max && rows > 128) continue;  // prefer more CTAs for long blocks
    if (orth_layout(rows, c0, w).total <= kOrthSmemMax) {
      *csize = C;
      return rows;
    }
  }
  return 0;
}

bool orth_cluster_applies(int n, int c0, int w) {
  int C = 0;
  return orth_plan(n, c0, w, &C) > 0;
}

void launch_orth_cluster(float* Q, int ldq, const float* src, int n, int c0, int w, int passes,
                         int chol_first, unsigned long long seed, const int* skip, cudaStream_t st) {
  int C = 0;
  const int rows = orth_plan(n, c0, w, &C);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = orth_layout(rows, c0, w).total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (w) {
    case 16: cudaLaunchKernelEx(&cfg, k_orth_cluster<16>, Q, ldq, src, n, c0, rows, passes, chol_first, seed, skip); break;
    case 32: cudaLaunchKernelEx(&cfg, k_orth_cluster<32>, Q, ldq, src, n, c0, rows, passes, chol_first, seed, skip); break;
    case 48: cudaLaunchKernelEx(&cfg, k_orth_cluster<48>, Q, ldq, src, n, c0, rows, passes, chol_first, seed, skip); break;
    default: cudaLaunchKernelEx(&cfg, k_orth_cluster<64>, Q, ldq, src, n, c0, rows, passes, chol_first, seed, skip); break;
  }
}

}  // namespace psdp
