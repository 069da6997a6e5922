// k_factored.cu — the primal-step input of Alg. 2 applied as an operator,
// without the n x n matrix.
//
// Alg. 2 keeps X^k = V diag(lambda) V^T in factored form (Sec. 3), so the
// projection input S^k = X^k - alpha (C + M*(y^k)) (Alg. 2 primal step) acts
// on a block Q as
//
//   S^k Q = V (Lambda_+ (V^T Q)) - alpha D_sym Q - alpha s0 1 (1^T Q),
//
// with D_sym = C + M*(y^k) on the union sparsity pattern of C and the A_i
// (both triangles) and s0 the summed coefficient of the structured rows
// a 11^T.  Appending a column of ones to V folds the last term into the
// low-rank one: S^k Q = [V | 1] P - alpha D_sym Q with
// P = [Lambda_+ V^T Q ; -alpha s0 1^T Q] ((r+1) x w).  In exact arithmetic
// this is the product with the S that the explicit path writes to HBM; the
// cost drops from O(n^2 w) to O(n (r+1) w + nnz w) per product and the n^2
// buffer is never allocated.
//
//   k_lr_coeff  one thread-block cluster: each CTA takes a slice of the rows,
//               stages [V | 1] and Q for 64 rows at a time, accumulates its
//               partial P, and writes the row-major copy Qr of Q that the
//               gathers below read; the partials are summed in CTA order
//               through distributed shared memory (deterministic) and scaled.
//   k_lr_apply  16 rows per CTA: the low-rank part from P in shared memory,
//               then the sparse part as row gathers of Qr (one 4-byte load per
//               lane per entry, coalesced over the columns of the row).
#include "psdp.cuh"

#include <cooperative_groups.h>

namespace psdp {

constexpr int LC_THREADS = 512;  // k_lr_coeff: 16 warps
constexpr int LC_RC = 64;        // rows staged per chunk
constexpr int LC_LDV = 68;       // [V | 1] chunk row stride (16-byte rows for float4 reads)
constexpr int LC_LDQ = 65;       // Q chunk row stride (odd: conflict-free transposed stores)
constexpr int LC_LDP = 64;       // partial P row stride
constexpr int LA_THREADS = 256;  // k_lr_apply: 8 warps, two rows each
constexpr int LA_RB = 16;        // rows per CTA

static int g_lc_cluster = 8;  // 16 where the device co-schedules 16-CTA clusters of k_lr_coeff

// Factor count of the current iterate, capped at 63 so [V | 1] fits 64 columns
// (the Lanczos path holds at most 60 factors).
__device__ __forceinline__ int factor_count(const Ctl* ctl) { return min(max(ctl->r_old, 0), 63); }

__global__ void __launch_bounds__(LC_THREADS) k_lr_coeff(DevProblem pb, DevWork wk, const float* __restrict__ Q,
                                                         int ldq, int w, const int* skip) {
  namespace cg = cooperative_groups;
  if (skip && *(volatile const int*)skip) return;  // uniform over the grid: no CTA reaches a barrier
  __shared__ __align__(16) float Vs[LC_RC * LC_LDV];  // [V | 1] chunk; after the loop the partial P
  __shared__ __align__(16) float Qs[LC_RC * LC_LDQ];
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const Ctl* ctl = wk.ctl;
  const int par = ctl->par;
  const int rf = factor_count(ctl);
  const int R1 = rf + 1;
  const int ntg = (R1 + 7) / 8;  // groups of 8 coefficient rows
  const int tw = 8 * ntg;        // staged columns of [V | 1] (zero beyond R1)
  const float* V = wk.Vrm[par];
  const int n = pb.n;
  const int nr = (n + CS - 1) / CS;
  const int rb = min(n, rank * nr), re = min(n, rb + nr);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tg = wid & 7, half = wid >> 3;  // warp: coefficient rows 8 tg..8 tg+7, chunk rows of parity `half`
  const bool active = tg < ntg;
  float acc[8][2];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a][0] = acc[a][1] = 0.f;
  // staging through registers: every load of a chunk is issued before the
  // first store, and the next chunk's loads fly during this chunk's products
  constexpr int kPer = LC_RC * 64 / LC_THREADS;
  float vreg[kPer], qreg[kPer];
  auto load_chunk = [&](int c0) {
    const int rows = min(LC_RC, re - c0);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int idx = tid + k * LC_THREADS;
      const int ii = idx / tw, t = idx - ii * tw;
      vreg[k] = 0.f;
      if (ii < rows) vreg[k] = (t < rf) ? V[(size_t)(c0 + ii) * wk.ldv + t] : (t == rf ? 1.f : 0.f);
      const int c = idx / LC_RC, jj = idx % LC_RC;  // rows fastest: coalesced column reads
      qreg[k] = (c < w && jj < rows) ? Q[(size_t)c * ldq + c0 + jj] : 0.f;
    }
  };
  if (rb < re) load_chunk(rb);
  for (int c0 = rb; c0 < re; c0 += LC_RC) {
    const int rows = min(LC_RC, re - c0);
    __syncthreads();  // the previous chunk's readers are done
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int idx = tid + k * LC_THREADS;
      const int ii = idx / tw, t = idx - ii * tw;
      if (ii < LC_RC) Vs[ii * LC_LDV + t] = vreg[k];
      const int c = idx / LC_RC, jj = idx % LC_RC;
      if (c < w) Qs[jj * LC_LDQ + c] = qreg[k];
    }
    __syncthreads();
    if (c0 + LC_RC < re) load_chunk(c0 + LC_RC);
    for (int idx = tid; idx < rows * w; idx += LC_THREADS) {  // columns fastest: coalesced row writes
      const int ii = idx / w, c = idx % w;
      wk.Qr[(size_t)(c0 + ii) * w + c] = Qs[ii * LC_LDQ + c];
    }
    if (active) {
      for (int ii = half; ii < rows; ii += 2) {
        const float4 a0 = *reinterpret_cast<const float4*>(&Vs[ii * LC_LDV + 8 * tg]);
        const float4 a1 = *reinterpret_cast<const float4*>(&Vs[ii * LC_LDV + 8 * tg + 4]);
        const float q0 = Qs[ii * LC_LDQ + lane];
        const float q1 = Qs[ii * LC_LDQ + lane + 32];  // columns >= w: never stored
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          acc[a][0] = fmaf(av[a], q0, acc[a][0]);
          acc[a][1] = fmaf(av[a], q1, acc[a][1]);
        }
      }
    }
  }
  // partial P of this CTA (rows of both parities added) in Vs
  __syncthreads();
  float* Gp = Vs;
  if (active && half == 1)
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      Gp[(8 * tg + a) * LC_LDP + lane] = acc[a][0];
      Gp[(8 * tg + a) * LC_LDP + lane + 32] = acc[a][1];
    }
  __syncthreads();
  if (active && half == 0)
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      Gp[(8 * tg + a) * LC_LDP + lane] += acc[a][0];
      Gp[(8 * tg + a) * LC_LDP + lane + 32] += acc[a][1];
    }
  cluster.sync();
  // CTA `rank` sums its share of the R1 x w coefficients over the cluster in
  // CTA order (all remote loads issued before the additions) and scales them.
  const int E = R1 * w;
  const int share = (E + CS - 1) / CS;
  const float ash = (float)(pb.alpha * wk.dshift[0]);
  for (int o = rank * share + tid; o < min(E, (rank + 1) * share); o += LC_THREADS) {
    const int t = o / w, c = o % w;
    float v[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) v[b] = (b < CS) ? cluster.map_shared_rank(Gp, b)[t * LC_LDP + c] : 0.f;
    float s = 0.f;
#pragma unroll
    for (int b = 0; b < 16; ++b) s += v[b];
    const float scale = (t < rf) ? (float)fmax(wk.lam[par][t], 0.0) : -ash;
    wk.lrP[o] = s * scale;
  }
  cluster.sync();  // keep every CTA's shared memory alive until all remote reads are done
}

__global__ void __launch_bounds__(LA_THREADS) k_lr_apply(DevProblem pb, DevWork wk, float* __restrict__ W, int ldw,
                                                         int w, const int* skip, cudaGraphConditionalHandle cond,
                                                         int set_cond) {
  if (skip && *(volatile const int*)skip) return;
  if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 1u);
  __shared__ __align__(16) float Ps[64 * 64];              // P, row stride 64
  __shared__ __align__(16) float Vs[LA_RB * LC_LDV];       // [V | 1] rows of this CTA
  __shared__ float Ws[kMaxW * (LA_RB + 1)];                // output, column-major
  const Ctl* ctl = wk.ctl;
  const int par = ctl->par;
  const int rf = factor_count(ctl);
  const int R1 = rf + 1;
  const int R1p = (R1 + 3) & ~3;
  const int n = pb.n;
  const int r0 = blockIdx.x * LA_RB;
  const int rows = min(LA_RB, n - r0);
  const float* V = wk.Vrm[par];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int i0 = 2 * wid;  // this warp's rows i0, i0 + 1 of the CTA; lanes: columns lane, lane + 32
  // first batch of the sparse entries of both rows, loaded before the staging
  int pe0[2], pe1[2], pj[2];
  float pa[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = r0 + i0 + h;
    pe0[h] = pe1[h] = 0;
    pj[h] = 0;
    pa[h] = 0.f;
    if (i0 + h < rows) {
      pe0[h] = pb.sym_ptr[i];
      pe1[h] = pb.sym_ptr[i + 1];
      if (lane < pe1[h] - pe0[h]) {
        pj[h] = pb.sym_col[pe0[h] + lane];
        pa[h] = wk.Dsym[pe0[h] + lane];
      }
    }
  }
  {  // P and the [V | 1] rows: all loads in flight before the stores
    constexpr int kP = 64 * 64 / LA_THREADS, kV = LA_RB * 64 / LA_THREADS;
    float preg[kP], vreg[kV];
    const int E = R1p * w;
#pragma unroll
    for (int k = 0; k < kP; ++k) {
      const int o = tid + k * LA_THREADS;
      preg[k] = (o < R1 * w) ? wk.lrP[o] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kV; ++k) {
      const int idx = tid + k * LA_THREADS;
      const int ii = idx / R1p, t = idx - ii * R1p;
      vreg[k] = 0.f;
      if (ii < rows) vreg[k] = (t < rf) ? V[(size_t)(r0 + ii) * wk.ldv + t] : (t == rf ? 1.f : 0.f);
    }
#pragma unroll
    for (int k = 0; k < kP; ++k) {
      const int o = tid + k * LA_THREADS;
      if (o < E) {
        const int t = o / w;
        Ps[t * 64 + o - t * w] = preg[k];
      }
    }
#pragma unroll
    for (int k = 0; k < kV; ++k) {
      const int idx = tid + k * LA_THREADS;
      const int ii = idx / R1p;
      if (ii < LA_RB) Vs[ii * LC_LDV + idx - ii * R1p] = vreg[k];
    }
  }
  __syncthreads();
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int t = 0; t < R1p; t += 4) {
    const float4 va = *reinterpret_cast<const float4*>(&Vs[i0 * LC_LDV + t]);
    const float4 vb = *reinterpret_cast<const float4*>(&Vs[(i0 + 1) * LC_LDV + t]);
    const float xa[4] = {va.x, va.y, va.z, va.w}, xb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float p0 = Ps[(t + u) * 64 + lane], p1 = Ps[(t + u) * 64 + lane + 32];  // columns >= w unused
      acc[0][0] = fmaf(xa[u], p0, acc[0][0]);
      acc[0][1] = fmaf(xa[u], p1, acc[0][1]);
      acc[1][0] = fmaf(xb[u], p0, acc[1][0]);
      acc[1][1] = fmaf(xb[u], p1, acc[1][1]);
    }
  }
  // - alpha D_sym Q: the entries of a row in batches of 32 (one per lane),
  // broadcast by shuffles, eight row gathers of Qr in flight per step
  const bool c0ok = lane < w, c1ok = lane + 32 < w;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (i0 + h >= rows) break;  // warp-uniform
    for (int eb = pe0[h]; eb < pe1[h]; eb += 32) {
      const int cnt = min(32, pe1[h] - eb);
      int j = pj[h];
      float a = pa[h];
      if (eb != pe0[h]) {
        j = 0;
        a = 0.f;
        if (lane < cnt) {
          j = pb.sym_col[eb + lane];
          a = wk.Dsym[eb + lane];
        }
      }
      for (int k = 0; k < cnt; k += 8) {
        float g0[8], g1[8], aa[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {  // lanes >= cnt hold j = 0, a = 0
          const int jj = __shfl_sync(0xffffffffu, j, k + u);
          aa[u] = __shfl_sync(0xffffffffu, a, k + u);
          const float* qr = wk.Qr + (size_t)jj * w;
          g0[u] = c0ok ? __ldcg(qr + lane) : 0.f;
          g1[u] = c1ok ? __ldcg(qr + lane + 32) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          acc[h][0] = fmaf(-aa[u], g0[u], acc[h][0]);
          acc[h][1] = fmaf(-aa[u], g1[u], acc[h][1]);
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (c0ok) Ws[lane * (LA_RB + 1) + i0 + h] = acc[h][0];
    if (c1ok) Ws[(lane + 32) * (LA_RB + 1) + i0 + h] = acc[h][1];
  }
  __syncthreads();
  for (int idx = tid; idx < w * LA_RB; idx += LA_THREADS) {  // rows fastest: 64-byte column segments
    const int c = idx / LA_RB, ii = idx % LA_RB;
    if (ii < rows) W[(size_t)c * ldw + r0 + ii] = Ws[c * (LA_RB + 1) + ii];
  }
}

void init_factored_attributes() {
  cudaFuncSetAttribute(k_lr_coeff, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(LC_THREADS, 1, 1);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  g_lc_cluster = (cudaOccupancyMaxActiveClusters(&nc, k_lr_coeff, &cfg) == cudaSuccess && nc > 0) ? 16 : 8;
  cudaGetLastError();
}

void launch_factored_matvec(const DevProblem& pb, const DevWork& wk, const float* Q, int ldq, float* W, int ldw,
                            int w, const int* skip, cudaStream_t st, cudaGraphConditionalHandle cond,
                            int set_cond) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g_lc_cluster, 1, 1);
  cfg.blockDim = dim3(LC_THREADS, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = g_lc_cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_lr_coeff, pb, wk, Q, ldq, w, skip);
  const int blocks = (pb.n + LA_RB - 1) / LA_RB;
  k_lr_apply<<<blocks, LA_THREADS, 0, st>>>(pb, wk, W, ldw, w, skip, cond, set_cond);
}

}  // namespace psdp
