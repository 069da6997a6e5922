// k_lanczos.cu — kernels of the restarted block Lanczos solver behind the
// truncated psd projection aproj(S, r) of Sec. 3.1 (Eq. trunc_eig).
//
// The paper computes the r largest eigenpairs with a Krylov method (ARPACK on
// a CPU, Sec. 3.1 / Sec. 4); here the Krylov basis lives in HBM as FP32
// column blocks, inner products are accumulated exactly-rounded in a pair of
// FP32 numbers (Knuth's TwoSum with the FMA-based TwoProduct of Ogita, Rump &
// Oishi, "Accurate sum and dot product", 2005) and combined across blocks in
// FP64, and the small Rayleigh-Ritz eigenproblem is solved by cyclic Jacobi
// rotations in one thread block.
#include "psdp.cuh"

#include <math.h>

#include <algorithm>

#include <cooperative_groups.h>

namespace psdp {

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
// dimension, in chunks of 32.  The S chunk is staged transposed (Ss[k][row])
// so a thread reads its 8 rows as two float4 broadcasts; each thread holds
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
  // tile (column-major, 16G x 128) share one buffer
  constexpr int kStage = MV_KC * MV_LDS + MV_KC * (16 * G + 1);
  constexpr int kPart = 16 * G * MV_RB;
  __shared__ __align__(16) float smbuf[kStage > kPart ? kStage : kPart];
  float(*Ss)[MV_LDS] = reinterpret_cast<float(*)[MV_LDS]>(smbuf);
  float(*Qs)[16 * G + 1] = reinterpret_cast<float(*)[16 * G + 1]>(smbuf + MV_KC * MV_LDS);
  float(*Ps)[MV_RB] = reinterpret_cast<float(*)[MV_RB]>(smbuf);
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
      const int rr = idx >> 3, kq = (idx & 7) * 4;
      Ss[kq][rr] = sreg[v].x;
      Ss[kq + 1][rr] = sreg[v].y;
      Ss[kq + 2][rr] = sreg[v].z;
      Ss[kq + 3][rr] = sreg[v].w;
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
      const float4 s0 = *reinterpret_cast<const float4*>(&Ss[kk][tr * 8]);
      const float4 s1 = *reinterpret_cast<const float4*>(&Ss[kk][tr * 8 + 4]);
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
    for (int a = 0; a < 8; ++a) Ps[tc + 16 * g][tr * 8 + a] = acc[a][g];
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();
  const int rank = (int)cluster.block_rank();
  const int rows_per = MV_RB / ns;
  for (int idx = tid; idx < kc * rows_per; idx += 256) {
    const int col = idx / rows_per, rr = rank * rows_per + idx % rows_per;
    float sum = 0.f;
    for (int sl = 0; sl < ns; ++sl) {
      const float* rp = cluster.map_shared_rank(&Ps[0][0], sl);
      sum += rp[col * MV_RB + rr];
    }
    const int row = r0 + rr;
    if (row < n) W[(size_t)(c0 + col) * ldw + row] = sum;
  }
  cluster.sync();  // keep every CTA's shared memory alive until all reads are done
}

// Inner-dimension slices per 128-row block: a power of two <= 8 (the cluster
// size), about two CTAs per SM, at least four 32-wide chunks per slice.
static int matvec_slices(int n, int k) {
  const int tiles = ((n + MV_RB - 1) / MV_RB) * ((k + 63) / 64);
  int ns = 1;
  while (ns < 8 && tiles * ns * 2 <= 2 * 148 && (n + 2 * ns * 4 * MV_KC - 1) / (2 * ns * 4 * MV_KC) >= 1 &&
         n >= 2 * ns * 4 * MV_KC)
    ns *= 2;
  return ns;
}

size_t block_matvec_scratch_floats(int, int) { return 0; }
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
                         int k, const int* skip, cudaStream_t st, float*, unsigned*,
                         cudaGraphConditionalHandle cond, int set_cond) {
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
  // row splits: a power of two <= 8, >= 256 rows each, about 148 CTAs in all
  int ns = 1;
  while (ns < 8 && tiles * ns * 2 <= 148 && n >= 2 * ns * 256) ns *= 2;
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
// Symmetric eigensolver: parallel cyclic Jacobi in one CTA + refinement
// ---------------------------------------------------------------------------
// (1) Cyclic Jacobi in FP32.  Round-robin ordering: in round s (0..K-2)
//     position K-1 meets s and, for t = 1..K/2-1, (s+t) mod (K-1) meets
//     (s-t) mod (K-1); the K/2 rotations of a round act on disjoint pairs.
//     Each rotation J (c, s in the (p,q) plane) zeroes A_pq
//     (tan 2 theta = 2 A_pq / (A_qq - A_pp)); A <- J^T A J, V <- V J.
//     Pairs with |A_pq| below 1e-7 sqrt(|A_pp A_qq|) are not rotated.  Sweeps
//     stop when off(A) <= 1e-6 ||A||_F.
// (2) One refinement step for the `nout` wanted eigenvectors (Ogita & Aishima,
//     "Iterative refinement for symmetric eigenvalue decomposition", 2018):
//     with Y the Jacobi vectors, S = Y^T T Y and R = I - Y^T Y accumulated in
//     FP32 pairs against the FP64 input T, lambda_j = S_jj / (1 - R_jj) and
//     y_j <- y_j + sum_i y_i E_ij,  E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)
//     (E_ij = R_ij / 2 for i = j or nearly equal eigenvalues).  The refined
//     eigenvalues are FP64-accurate; the vectors are FP32-rounded.
constexpr int JB = 32;  // wanted columns refined per pass

__global__ void __launch_bounds__(512) k_jacobi(const double* __restrict__ Tin, int K, int Kp,
                                                double* __restrict__ theta, float* __restrict__ Yout,
                                                int ldy, int nout, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ float smj[];
  const int ld = Kp + 1;
  float* A = smj;                      // Kp x (Kp+1)
  float* V = A + (size_t)Kp * ld;      // Kp x (Kp+1)
  float* cs = V + (size_t)Kp * ld;     // Kp/2
  float* sn = cs + Kp / 2;             // Kp/2
  float* dg = sn + Kp / 2;             // Kp: eigenvalue estimates
  int* pp = reinterpret_cast<int*>(dg + Kp);
  int* qq = pp + Kp / 2;
  int* rank = qq + Kp / 2;             // Kp
  int* wanted = rank + Kp;             // JB
  double* red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(wanted + JB) + 7) & ~uintptr_t(7));
  double* lamj = red + 64;             // JB
  float* scr = reinterpret_cast<float*>(lamj + JB);  // 4 * Kp * JB refinement scratch
  __shared__ int s_stop;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int half = Kp / 2;

  for (int idx = tid; idx < Kp * Kp; idx += nth) {
    int i = idx / Kp, j = idx % Kp;
    double v = 0.0;
    if (i < K && j < K) v = 0.5 * (Tin[i * K + j] + Tin[j * K + i]);
    A[i * ld + j] = (float)v;
    V[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  if (Kp > K && tid == 0) {  // isolated padding index, below every eigenvalue
    float s = 0.f;
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < K; ++j) s = fmaxf(s, fabsf(A[i * ld + j]));
    A[K * ld + K] = -4.f * (s + 1.f) * (float)K;
  }
  __syncthreads();

  for (int sweep = 0; sweep < 15; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < K * K; idx += nth) {
      int i = idx / K, j = idx % K;
      double v = (double)A[i * ld + j];
      tot += v * v;
      if (i != j) off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5] = off;
      red[32 + (tid >> 5)] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      double o2 = 0.0, t2 = 0.0;
      for (int k = 0; k < (nth >> 5); ++k) {
        o2 += red[k];
        t2 += red[32 + k];
      }
      // the refinement below restores full accuracy, so the sweeps stop at
      // off(A) <= 1e-5 ||A||_F (above the FP32 rounding floor of ~K eps ||A||)
      s_stop = (o2 <= 1e-10 * t2) || (t2 == 0.0);
    }
    __syncthreads();
    if (s_stop) break;
    for (int round = 0; round < Kp - 1; ++round) {
      if (tid < half) {
        int p, q;
        if (tid == 0) {
          p = round;
          q = Kp - 1;
        } else {
          p = (round + tid) % (Kp - 1);
          q = (round - tid + (Kp - 1)) % (Kp - 1);
        }
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        float apq = A[p * ld + q];
        float app = A[p * ld + p], aqq = A[q * ld + q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > 1e-7f * sqrtf(fabsf(app * aqq)) && apq != 0.f) {
          float tau = (aqq - app) / (2.f * apq);
          float t;
          if (fabsf(tau) > 1e15f) t = 0.5f / tau;
          else t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = 1.f / sqrtf(1.f + t * t);
          s = t * c;
        }
        cs[tid] = c;
        sn[tid] = s;
        pp[tid] = p;
        qq[tid] = q;
      }
      __syncthreads();
      // A <- J^T A J: every 2x2 block (pair t rows, pair u columns) transforms
      // independently, B <- J_t^T B J_u; blocks t <= u, mirrored.
      for (int idx = tid; idx < half * half; idx += nth) {
        const int t = idx / half, u = idx % half;
        if (u > t) continue;
        const float ct = cs[t], st = sn[t], cu = cs[u], su = sn[u];
        if (st == 0.f && su == 0.f) continue;
        const int pt = pp[t], qt = qq[t], pu = pp[u], qu = qq[u];
        float b00 = A[pt * ld + pu], b01 = A[pt * ld + qu], b10 = A[qt * ld + pu], b11 = A[qt * ld + qu];
        float m00 = ct * b00 - st * b10, m01 = ct * b01 - st * b11;
        float m10 = st * b00 + ct * b10, m11 = st * b01 + ct * b11;
        float n00 = cu * m00 - su * m01, n01 = su * m00 + cu * m01;
        float n10 = cu * m10 - su * m11, n11 = su * m10 + cu * m11;
        if (t == u) {  // the rotation annihilates the pair's off-diagonal entry
          n01 = 0.f;
          n10 = 0.f;
        }
        A[pt * ld + pu] = n00;
        A[pt * ld + qu] = n01;
        A[qt * ld + pu] = n10;
        A[qt * ld + qu] = n11;
        if (t != u) {
          A[pu * ld + pt] = n00;
          A[qu * ld + pt] = n01;
          A[pu * ld + qt] = n10;
          A[qu * ld + qt] = n11;
        }
      }
      for (int idx = tid; idx < half * Kp; idx += nth) {  // V <- V J
        int u = idx / Kp, i = idx % Kp;
        float c = cs[u], s = sn[u];
        if (s == 0.f) continue;
        int p = pp[u], q = qq[u];
        float vp = V[i * ld + p], vq = V[i * ld + q];
        V[i * ld + p] = c * vp - s * vq;
        V[i * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // eigenvalue estimates and their descending order (ties by index)
  for (int i = tid; i < Kp; i += nth) dg[i] = A[i * ld + i];
  __syncthreads();
  float scale = 0.f;
  for (int i = 0; i < K; ++i) scale = fmaxf(scale, fabsf(dg[i]));
  const float delta = 1e-3f * fmaxf(scale, 1e-30f);  // eigenvalues closer than this form a cluster
  for (int i = tid; i < K; i += nth) {
    float di = dg[i];
    int rk = 0;
    for (int j = 0; j < K; ++j) {
      float dj = dg[j];
      rk += (dj > di) || (dj == di && j < i);
    }
    rank[i] = rk;
  }
  __syncthreads();
  // T (symmetrised) as a packed upper triangle in the freed A region, split
  // once into FP32 hi + lo parts (Kp (Kp+1)/2 entries each = Kp (Kp+1) floats);
  // hi + lo carries ~48 bits, enough for the FP32-pair products below
  float* Th = A;
  float* Tl = A + Kp * (Kp + 1) / 2;
  for (int idx = tid; idx < K * K; idx += nth) {
    int i = idx / K, j = idx % K;
    if (i <= j) {
      const double t = 0.5 * (Tin[i * K + j] + Tin[j * K + i]);
      const float hi = (float)t;
      Th[j * (j + 1) / 2 + i] = hi;
      Tl[j * (j + 1) / 2 + i] = (float)(t - (double)hi);
    }
  }
  __syncthreads();
  // refinement scratch, per pass: Ph | Pl | Sm | Rm  (each Kp x jb floats)
  const int jb = JB;
  float* Ph = scr;
  float* Pl = Ph + Kp * jb;
  float* Sm = Pl + Kp * jb;
  float* Rm = Sm + Kp * jb;
  for (int j0 = 0; j0 < nout; j0 += jb) {
    const int nb = min(jb, nout - j0);
    for (int i = tid; i < K; i += nth) {
      int rk = rank[i];
      if (rk >= j0 && rk < j0 + nb) wanted[rk - j0] = i;
    }
    __syncthreads();
    // P = T Y_wanted  (FP32-pair accumulation, T split into hi + lo)
    for (int o = tid; o < K * nb; o += nth) {
      int k = o / nb, jj = o % nb;
      const int j = wanted[jj];
      DF acc;
      for (int l = 0; l < K; ++l) {
        const int pi = (k <= l) ? l * (l + 1) / 2 + k : k * (k + 1) / 2 + l;
        const float y = V[l * ld + j];
        acc.fma_acc(Th[pi], y);
        acc.fma_acc(Tl[pi], y);
      }
      Ph[k * jb + jj] = acc.hi;
      Pl[k * jb + jj] = acc.lo;
    }
    __syncthreads();
    // S = Y^T P, R = I - Y^T Y_wanted
    for (int o = tid; o < K * nb; o += nth) {
      int i = o / nb, jj = o % nb;
      const int j = wanted[jj];
      DF s_acc, r_acc;
      for (int k = 0; k < K; ++k) {
        float yi = V[k * ld + i];
        s_acc.fma_acc(yi, Ph[k * jb + jj]);
        s_acc.fma_acc(yi, Pl[k * jb + jj]);
        r_acc.fma_acc(yi, V[k * ld + j]);
      }
      double rv = (i == j ? 1.0 : 0.0) - r_acc.value();
      if (i == j) lamj[jj] = s_acc.value() / (1.0 - rv);
      Sm[i * jb + jj] = (float)s_acc.value();
      Rm[i * jb + jj] = (float)rv;
    }
    __syncthreads();
    // E (in place of S)
    for (int o = tid; o < K * nb; o += nth) {
      int i = o / nb, jj = o % nb;
      const int j = wanted[jj];
      float r = Rm[i * jb + jj];
      float e;
      float lj = (float)lamj[jj];
      float gap = lj - dg[i];
      if (i == j || fabsf(gap) <= delta) e = 0.5f * r;
      else e = (Sm[i * jb + jj] + lj * r) / gap;
      Sm[i * jb + jj] = e;
    }
    __syncthreads();
    // y_j <- y_j + Y E_j
    for (int o = tid; o < K * nb; o += nth) {
      int row = o / nb, jj = o % nb;
      const int j = wanted[jj];
      float acc = V[row * ld + j];
      for (int i = 0; i < K; ++i) acc = fmaf(V[row * ld + i], Sm[i * jb + jj], acc);
      Yout[(size_t)(j0 + jj) * ldy + row] = acc;
    }
    for (int jj = tid; jj < nb; jj += nth) theta[j0 + jj] = lamj[jj];
    __syncthreads();
  }
  // Symmetric orthonormality correction of the refined vectors (the first-
  // order refinement leaves O(E^2) non-orthogonality): with G = Y^T Y from
  // FP32-pair sums, Y <- Y (3I - G) / 2, which maps G to I + O((G - I)^2).
  // A (now free) holds I - G, V (now free) the corrected columns.
  for (int o = tid; o < nout * nout; o += nth) {
    int i = o / nout, j = o % nout;
    if (j < i) continue;
    DF g;
#pragma unroll 8
    for (int k = 0; k < K; ++k) g.fma_acc(__ldcg(&Yout[(size_t)i * ldy + k]), __ldcg(&Yout[(size_t)j * ldy + k]));
    float v = (float)((i == j ? 1.0 : 0.0) - g.value());
    A[i * nout + j] = v;
    A[j * nout + i] = v;
  }
  __syncthreads();
  for (int o = tid; o < K * nout; o += nth) {
    int row = o / nout, j = o % nout;
    float corr = 0.f;
#pragma unroll 8
    for (int i = 0; i < nout; ++i) corr = fmaf(__ldcg(&Yout[(size_t)i * ldy + row]), A[i * nout + j], corr);
    V[row * ld + j] = __ldcg(&Yout[(size_t)j * ldy + row]) + 0.5f * corr;
  }
  __syncthreads();
  for (int o = tid; o < K * nout; o += nth) {
    int row = o / nout, j = o % nout;
    Yout[(size_t)j * ldy + row] = V[row * ld + j];
  }
}

static size_t jacobi_smem(int Kp) {
  size_t ld = Kp + 1;
  size_t f = 2 * (size_t)Kp * ld + (size_t)Kp + (size_t)Kp;  // A, V, cs+sn, dg
  size_t ints = (size_t)Kp + (size_t)Kp + JB;                // pp+qq, rank, wanted
  return f * sizeof(float) + ints * sizeof(int) + 8 + (64 + JB) * sizeof(double) +
         4 * (size_t)Kp * JB * sizeof(float);
}

void init_lanczos_attributes() {
  cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jacobi_smem(kMaxK));
  cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmem);
}

void launch_sym_eig(const double* T, int K, double* theta, float* Y, int ldy, int nout,
                    const int* skip, cudaStream_t st) {
  int Kp = (K + 1) & ~1;
  // fewer warps for small K: the rotation rounds are barrier-bound
  const int threads = Kp <= 32 ? 128 : (Kp <= 64 ? 256 : 512);
  k_jacobi<<<1, threads, jacobi_smem(Kp), st>>>(T, K, Kp, theta, Y, ldy, nout, skip);
}

}  // namespace psdp
