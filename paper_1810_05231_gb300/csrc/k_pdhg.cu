// k_pdhg.cu — the primal-dual part of one LR-PD-SDP iteration (Alg. 2):
// Ritz-vector assembly and the projection's convergence test, the constraint
// operator M(X) evaluated from the factors of X, the dual step with the
// equality / inequality split (Sec. 2.3.1, Eq. resolvent_1), the adjoint
// D = C + M*(y), the residuals of Sec. 2.2 (Eq. comb_residual), the rank
// rule of Sec. 3.2, and the rebuild of the next primal-step input
// S = V diag(max(lambda,0)) V^T - alpha (C + M*(y)) (Alg. 2 primal step).
#include "psdp.cuh"

#include <math.h>

#include <cooperative_groups.h>

namespace psdp {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of `nv` doubles per thread into out[0..nv) (thread 0 holds
// the result).  `sh` needs 32 * nv doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int q = 0; q < nw; ++q) s += sh[k * 32 + q];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Returns true in every thread of the last block to arrive (after all blocks
// stored their partials and fenced).
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}


// out[i] = sum_{b < P} part[b * stride + i] for i < L, by all threads of the
// block: groups of g threads (g a power of two, g <= 32, g * L <= blockDim)
// share one output, thread j of a group adding blocks j, j+g, ... in order,
// the group combining with a fixed shuffle tree (deterministic).
__device__ void reduce_partials(const double* part, int P, int stride, int L, double* out) {
  // g threads per entry (power of two <= 32), each summing every g-th
  // partial; more than one pass over the entries when L * g > blockDim
  int g = 1;
  while (g < 32 && 4 * g <= P && g * L < 4 * (int)blockDim.x) g *= 2;
  const int per_pass = blockDim.x / g;
  for (int i0 = 0; i0 < L; i0 += per_pass) {
    const int i = i0 + (int)threadIdx.x / g, j = threadIdx.x % g;
    double s = 0.0;
    if (i < L) {
#pragma unroll 4
      for (int b = j; b < P; b += g) s += __ldcg(&part[(size_t)b * stride + i]);
    }
    for (int o = g / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, g);
    if (i < L && j == 0) out[i] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Ritz vectors V = Q Y, S V = W Y, residuals and the projection's stop test
// ---------------------------------------------------------------------------
struct DFc {
  float hi, lo;
  __device__ __forceinline__ DFc() : hi(0.f), lo(0.f) {}
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

constexpr int RZ_RB = 32;

__global__ void __launch_bounds__(256) k_ritz(DevWork wk, int n, int K, int w, int r, int s_steps, int cycle_launches,
                                              cudaGraphConditionalHandle cond, int use_cond) {
  Ctl* ctl = wk.ctl;
  if (*(volatile int*)&ctl->lz_done) return;
  extern __shared__ float sm[];
  const int ldk = K + 1;
  float* Qs = sm;                      // RB x (K+1)
  float* Ws = Qs + RZ_RB * ldk;        // RB x (K+1)
  float* Ys = Ws + RZ_RB * ldk;        // K x w
  float* Vs = Ys + K * w;              // RB x (w+1)
  float* WVs = Vs + RZ_RB * (w + 1);   // RB x (w+1)
  __shared__ double th[kMaxP];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * RZ_RB;
  const int rows = min(RZ_RB, n - r0);
  const int nw = 1 - ctl->par;  // buffer of the new iterate
#pragma unroll 4
  for (int idx = tid; idx < RZ_RB * K; idx += blockDim.x) {
    int k = idx / RZ_RB, i = idx % RZ_RB;
    float q = 0.f, ww = 0.f;
    if (i < rows) {
      q = wk.Q[(size_t)k * wk.ldq + r0 + i];
      ww = wk.W[(size_t)k * wk.ldq + r0 + i];
    }
    Qs[i * ldk + k] = q;
    Ws[i * ldk + k] = ww;
  }
#pragma unroll 4
  for (int idx = tid; idx < K * w; idx += blockDim.x) {
    int t = idx / K, k = idx % K;
    Ys[k * w + t] = wk.Y[(size_t)t * kMaxK + k];
  }
  for (int t = tid; t < w; t += blockDim.x) th[t] = wk.theta[t];
  __syncthreads();
  {  // V = Q Y and W Y on this CTA's rows: 2 rows x (w/16) columns per thread
    const int ti = tid >> 4, tt = tid & 15;  // rows ti, ti + 16; columns tt + 16 j
    const int wg = (w + 15) / 16;            // <= kMaxP / 16 = 7
    float v[2][kMaxP / 16] = {}, u[2][kMaxP / 16] = {};
    const float* q0 = Qs + ti * ldk;
    const float* q1 = Qs + (ti + 16) * ldk;
    const float* w0 = Ws + ti * ldk;
    const float* w1 = Ws + (ti + 16) * ldk;
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
      const float a0 = q0[k], a1 = q1[k], b0 = w0[k], b1 = w1[k];
#pragma unroll
      for (int j = 0; j < kMaxP / 16; ++j) {
        if (j < wg) {
          const float y = Ys[k * w + min(tt + 16 * j, w - 1)];
          v[0][j] = fmaf(a0, y, v[0][j]);
          v[1][j] = fmaf(a1, y, v[1][j]);
          u[0][j] = fmaf(b0, y, u[0][j]);
          u[1][j] = fmaf(b1, y, u[1][j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxP / 16; ++j) {
      const int t = tt + 16 * j;
      if (j < wg && t < w) {
        Vs[ti * (w + 1) + t] = v[0][j];
        Vs[(ti + 16) * (w + 1) + t] = v[1][j];
        WVs[ti * (w + 1) + t] = u[0][j];
        WVs[(ti + 16) * (w + 1) + t] = u[1][j];
      }
    }
  }
  __syncthreads();
  // in-place write-back (each CTA owns its rows), row-major copy of V
  for (int o = tid; o < RZ_RB * w; o += blockDim.x) {
    int t = o / RZ_RB, i = o % RZ_RB;
    if (i < rows) {
      wk.Q[(size_t)t * wk.ldq + r0 + i] = Vs[i * (w + 1) + t];
      wk.W[(size_t)t * wk.ldq + r0 + i] = WVs[i * (w + 1) + t];
    }
  }
  for (int o = tid; o < RZ_RB * w; o += blockDim.x) {
    int i = o / w, t = o % w;
    if (i < rows) wk.Vrm[nw][(size_t)(r0 + i) * wk.ldv + t] = Vs[i * (w + 1) + t];
  }
  for (int o = tid; o < RZ_RB * w; o += blockDim.x) {  // column-major slot of the new factors
    int t = o / RZ_RB, i = o % RZ_RB;
    if (i < rows) wk.Vcm[(size_t)(nw * kMaxR + t) * wk.ldq + r0 + i] = Vs[i * (w + 1) + t];
  }
  // partial sums per Ritz column: ||wv - theta v||^2, v.wv, v.v, sum v
  double* part = wk.ritz_part + (size_t)blockIdx.x * 4 * w;
  for (int t = tid; t < w; t += blockDim.x) {  // FP32 pairs over this CTA's rows
    DFc b, c, d;
    float a = 0.f;
    float tht = (float)th[t];
    for (int i = 0; i < rows; ++i) {
      float v = Vs[i * (w + 1) + t], u = WVs[i * (w + 1) + t];
      float res = fmaf(-tht, v, u);
      a = fmaf(res, res, a);
      b.fma_acc(v, u);
      c.fma_acc(v, v);
      d.fma_acc(v, 1.f);  // column sums enter (1^T v)^2 of structured rows: keep them exact
    }
    part[t] = (double)a;
    part[w + t] = b.value();
    part[2 * w + t] = c.value();
    part[3 * w + t] = d.value();
  }
  if (!last_block(&wk.counters[CNT_RITZ * 512])) return;
  // final reduction in block order
  __shared__ double fin4[4 * kMaxP];
  reduce_partials(wk.ritz_part, gridDim.x, 4 * w, 4 * w, fin4);
  __shared__ double fin[4 * kMaxP];
  for (int t = tid; t < w; t += blockDim.x) {
    fin[t] = fin4[t];
    fin[kMaxP + t] = fin4[w + t];
    fin[2 * kMaxP + t] = fin4[2 * w + t];
    fin[3 * kMaxP + t] = fin4[3 * w + t];
  }
  __syncthreads();
  __shared__ double rres[kMaxP];
  for (int t = tid; t < w; t += blockDim.x) {  // one column per thread
    double vv = fin[2 * kMaxP + t];
    double lam = vv > 0.0 ? fin[kMaxP + t] / vv : th[t];  // Rayleigh quotient (FP64 sums)
    wk.lam[nw][t] = lam;
    wk.colsum[nw][t] = fin[3 * kMaxP + t];
    rres[t] = sqrt(fin[t] / (vv > 0.0 ? vv : 1.0));
  }
  for (int t = w + tid; t < wk.ldv; t += blockDim.x) {
    wk.lam[nw][t] = 0.0;
    wk.colsum[nw][t] = 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double scale = 0.0;
    for (int t = 0; t < w; ++t) scale = fmax(scale, fabs(th[t]));
    if (scale == 0.0) scale = 1.0;
    double worst = 0.0;
    for (int t = 0; t < r; ++t) worst = fmax(worst, rres[t] / scale);
    ctl->lz_res = worst;
    ctl->lz_cycle += 1;
    ctl->lz_cycles_total += 1;
    ctl->matvecs += s_steps;
    ctl->launches += cycle_launches;  // kernels of one restart cycle, counted by the host at enqueue time
    bool ok = worst <= ctl->lz_tol || !(worst == worst);
    if (ok || ctl->lz_cycle >= ctl->max_cycles) {
      if (!ok) ctl->lz_unconverged += 1;
      ctl->lz_done = 1;
    }
    if (use_cond) cudaGraphSetConditional(cond, ctl->lz_done ? 0u : 1u);
    wk.counters[CNT_RITZ * 512] = 0u;
  }
}

// ---------------------------------------------------------------------------
// M(X^{k+1}) from the factors, fused with the dual step (Alg. 2 dual step
// parts 1 and 2) and its reductions
// ---------------------------------------------------------------------------
// X = sum_{t<r} max(lambda_t,0) v_t v_t^T; one warp per chunk of <= kChunk
// entries of one extended row.  A row with one chunk is updated by that warp:
//   y_half = y + alpha (2 M(X+) - M(X));  equality rows y+ = y_half - alpha b,
//   inequality rows y+ = max(y_half - alpha h, 0)  (= y_half - alpha proj(y_half/alpha)).
// Rows with several chunks and the objective row m are finished by the last block.
__device__ __forceinline__ void dual_row(const DevProblem& pb, const DevWork& wk, int nw, int od, int row,
                                         double mxn, int r, const float* lp, double (&v)[4]) {
  const int d = pb.n_dense ? pb.dense_of_row[row] : -1;
  if (d >= 0) {  // tr(a 11^T X) = a sum_t max(lambda_t,0) (1^T v_t)^2
    double s = 0.0;
    for (int t = 0; t < r; ++t) {
      double cs = wk.colsum[nw][t];
      s += (double)lp[t] * cs * cs;
    }
    mxn += pb.dense_a[d] * s;
  }
  const double alpha = pb.alpha;
  const double mxo = wk.mx[od][row];
  const double yo = wk.y[row];
  const double yh = yo + alpha * (2.0 * mxn - mxo);
  const double yn = (row < pb.m_eq) ? yh - alpha * pb.rhs[row] : fmax(yh - alpha * pb.rhs[row], 0.0);
  const double dyv = yn - yo;
  wk.y[row] = yn;
  wk.dy[row] = dyv;
  wk.mx[nw][row] = mxn;
  const double dmx = mxn - mxo;
  const double ed = dyv / alpha - dmx;
  v[0] += ed * ed;          // eps_dual^2
  v[1] += dyv * dmx;        // <dy, M(dX)> = <M*(dy), dX>
  v[2] += pb.rhs[row] * yn; // rhs^T y
}

__global__ void __launch_bounds__(256) k_mxdual(DevProblem pb, DevWork wk, int r) {
  __shared__ float lp[kMaxR];
  __shared__ double sh[32 * 4];
  Ctl* ctl = wk.ctl;
  const int nw = 1 - ctl->par, od = ctl->par;
  for (int t = threadIdx.x; t < kMaxR; t += blockDim.x) lp[t] = (t < r) ? (float)fmax(wk.lam[nw][t], 0.0) : 0.f;
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (warp < pb.n_chunks) {
    const float* V = wk.Vrm[nw];
    double acc = 0.0;
    for (int e = pb.chunk_beg[warp] + lane; e < pb.chunk_end[warp]; e += 32) {
      const float* vp = V + (size_t)pb.ent_p[e] * wk.ldv;
      const float* vq = V + (size_t)pb.ent_q[e] * wk.ldv;
      float x = 0.f;
#pragma unroll 8
      for (int t = 0; t < r; ++t) x = fmaf(lp[t] * vp[t], vq[t], x);
      acc += pb.ent_a[e] * (double)x;
    }
    acc = warp_sum(acc);
    const int row = pb.chunk_row[warp];
    const bool single = row < pb.m && (pb.row_chunk[row + 1] - pb.row_chunk[row] == 1);
    if (lane == 0) {
      if (single) dual_row(pb, wk, nw, od, row, acc, r, lp, v);
      else wk.chunk_part[warp] = acc;
    }
  }
  block_sum<4>(v, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) wk.part[(size_t)blockIdx.x * 4 + k] = v[k];
  if (!last_block(&wk.counters[CNT_DUAL * 512])) return;
  // rows spread over several chunks
  double u[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < pb.n_multi; k += blockDim.x) {
    const int row = pb.multi_rows[k];
    double mxn = 0.0;
    for (int c = pb.row_chunk[row]; c < pb.row_chunk[row + 1]; ++c) mxn += __ldcg(&wk.chunk_part[c]);
    dual_row(pb, wk, nw, od, row, mxn, r, lp, u);
  }
  block_sum<4>(u, sh);
  __shared__ double tot[4];
  __shared__ double pobj_s[1];
  reduce_partials(wk.part, gridDim.x, 4, 3, tot);
  // objective row m: tr(C X+)
  reduce_partials(wk.chunk_part + pb.row_chunk[pb.m], pb.row_chunk[pb.m + 1] - pb.row_chunk[pb.m], 1, 1, pobj_s);
  if (threadIdx.x == 0) {
    double s[3] = {u[0] + tot[0], u[1] + tot[1], u[2] + tot[2]};
    const double pobj = pobj_s[0];
    wk.mx[nw][pb.m] = pobj;
    ctl->red_dual[0] = s[0];
    ctl->red_dual[1] = s[1];
    ctl->red_dual[2] = s[2];
    ctl->red_dual[3] = pobj;
    wk.counters[CNT_DUAL * 512] = 0u;
  }
}

// ---------------------------------------------------------------------------
// D = C + M*(y) on the union pattern, and ||M*(dy)||_F^2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dvals(DevProblem pb, DevWork wk) {
  __shared__ double sh[32 * 2];
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (u < pb.nU) {
    double d = pb.u_c[u], md = 0.0;
    for (int j = pb.u_ptr[u]; j < pb.u_ptr[u + 1]; ++j) {
      d += wk.y[pb.u_row[j]] * pb.u_a[j];
      md += wk.dy[pb.u_row[j]] * pb.u_a[j];
    }
    wk.D[u] = d;
    if (wk.Dsym) {  // factored operator: alpha D on both triangles, as the rebuild subtracts it
      const float ad = (float)(pb.alpha * d);
      wk.Dsym[pb.u_pos[2 * (size_t)u]] = ad;
      const int p2 = pb.u_pos[2 * (size_t)u + 1];
      if (p2 >= 0) wk.Dsym[p2] = ad;
    }
    const double wgt = (pb.u_p[u] == pb.u_q[u]) ? 1.0 : 2.0;
    v[0] = wgt * md * md;
    v[1] = wgt * md;
  }
  block_sum<2>(v, sh);
  double* part = wk.part + (size_t)blockIdx.x * 2;
  if (threadIdx.x == 0) {
    part[0] = v[0];
    part[1] = v[1];
  }
  if (!last_block(&wk.counters[CNT_DVALS * 512])) return;
  __shared__ double tot2[2];
  reduce_partials(wk.part, gridDim.x, 2, 2, tot2);
  if (threadIdx.x == 0) {
    const double s0 = tot2[0], s1 = tot2[1];
    double sh0 = 0.0, sh1 = 0.0;
    for (int d = 0; d < pb.n_dense; ++d) {
      sh0 += pb.dense_a[d] * wk.y[pb.dense_row[d]];
      sh1 += pb.dense_a[d] * wk.dy[pb.dense_row[d]];
    }
    wk.dshift[0] = sh0;
    wk.dshift[1] = sh1;
    // ||sparse + sh1 11^T||_F^2
    wk.ctl->red_dvals[0] = s0 + 2.0 * sh1 * s1 + sh1 * sh1 * (double)pb.n * (double)pb.n;
    wk.counters[CNT_DVALS * 512] = 0u;
  }
}

// ---------------------------------------------------------------------------
// controller: residuals (Sec. 2.2), stop test, rank rule (Sec. 3.2)
// ---------------------------------------------------------------------------
// G is the Gram of the column-major factor slots [slot0 | slot1] (2*kMaxR
// columns); X = V_s Lambda_+ V_s^T for slot s, so
// ||X1 - X0||_F^2 = sum lam1 lam1 G11^2 + sum lam0 lam0 G00^2 - 2 sum lam1 lam0 G10^2.
__device__ void control_tail(const DevProblem& pb, const DevWork& wk, const double* G, int iter_launches,
                             cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sh[32 * 3];
  Ctl* ctl = wk.ctl;
  const int nw = 1 - ctl->par, od = ctl->par;
  const int r = ctl->r, ro = ctl->r_old;
  const int ldg = 2 * kMaxR;
  const int on = nw * kMaxR, oo = od * kMaxR;
  double v[3] = {0.0, 0.0, 0.0};
  const int rm = max(r, ro);
  for (int idx = threadIdx.x; idx < rm * rm; idx += blockDim.x) {
    int s = idx / rm, t = idx % rm;
    if (s < r && t < r) {
      double g = G[(size_t)(on + s) * ldg + on + t];
      v[0] += fmax(wk.lam[nw][s], 0.0) * fmax(wk.lam[nw][t], 0.0) * g * g;
    }
    if (s < ro && t < ro) {
      double g = G[(size_t)(oo + s) * ldg + oo + t];
      v[1] += fmax(wk.lam[od][s], 0.0) * fmax(wk.lam[od][t], 0.0) * g * g;
    }
    if (s < r && t < ro) {
      double g = G[(size_t)(on + s) * ldg + oo + t];
      v[2] += fmax(wk.lam[nw][s], 0.0) * fmax(wk.lam[od][t], 0.0) * g * g;
    }
  }
  block_sum<3>(v, sh);
  if (threadIdx.x != 0) return;
  const double alpha = pb.alpha;
  const double x1 = v[0], x0 = v[1], x10 = v[2];
  const double dX2 = fmax(x1 + x0 - 2.0 * x10, 0.0);
  // CSR rows plus the element-wise box rows (zero slots without a box)
  const double ed2 = ctl->red_dual[0] + ctl->red_dvals[kRedBox];
  const double cross = ctl->red_dual[1] + ctl->red_dvals[kRedBox + 1];
  const double ms2 = ctl->red_dvals[0] + ctl->red_dvals[kRedBox + 3];
  // ||dX/alpha - M*(dy)||^2 = ||dX||^2/alpha^2 - 2/alpha <dX, M*(dy)> + ||M*(dy)||^2
  const double ep2 = dX2 / (alpha * alpha) - 2.0 * cross / alpha + ms2;
  const double eps_p = sqrt(fmax(ep2, 0.0));
  const double eps_d = sqrt(fmax(ed2, 0.0));
  const double pobj = ctl->red_dual[3];
  const double dobj = -(ctl->red_dual[2] + ctl->red_dvals[kRedBox + 2]);
  const double rel_p = eps_p / (1.0 + pb.normC);
  const double rel_d = eps_d / (1.0 + pb.normRhs);
  const double rel_gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
  const double normX = sqrt(fmax(x1, 0.0));
  const double lam_r = wk.lam[nw][r - 1];
  const int n = pb.n;
  const int it = ctl->it + 1;
  ctl->it = it;
  ctl->eps_p = eps_p;
  ctl->eps_d = eps_d;
  ctl->rel_p = rel_p;
  ctl->rel_d = rel_d;
  ctl->rel_gap = rel_gap;
  ctl->pobj = pobj;
  ctl->dobj = dobj;
  ctl->lam_r = lam_r;
  ctl->normX = normX;
  ctl->matvecs += 1;  // warm-start product of the next iteration
  ctl->launches += iter_launches;  // per-iteration kernels outside the restart cycles (host count)
  const double comb = eps_p + eps_d;
  const int win = ctl->window;
  const double old = ctl->hist[it % win];
  ctl->hist[it % win] = comb;
  // projection tolerance for the next iteration: tighter as the residuals fall
  if (ctl->lz_tol_fixed > 0.0) ctl->lz_tol = ctl->lz_tol_fixed;
  else ctl->lz_tol = fmin(1e-3, fmax(2e-6, 0.05 * fmax(rel_p, rel_d)));
  int status = ST_RUNNING;
  if (!(ep2 == ep2) || !(ed2 == ed2) || !(pobj == pobj) || !(dobj == dobj) || !(x1 == x1) ||
      !(lam_r == lam_r) || fabs(pobj) > 1e300) {
    status = ST_NUMERIC;
  } else {
    // inner-loop test of Alg. 2 on the relative residuals; the final stop also
    // needs a sufficient rank and a small relative gap
    const bool conv = fmax(rel_p, rel_d) <= ctl->tol;
    const bool rank_ok = (r >= n) || ctl->full_eig ||
                         (sqrt((double)(n - r)) * fmax(lam_r, 0.0) <= ctl->eps_lambda * fmax(1.0, normX));
    // at the rank cap with settings.at_max_rank, the residuals and the gap
    // alone decide (r cannot grow)
    const bool cap_ok = ctl->at_max_rank && r >= ctl->max_rank;
    bool grow = false;
    if (conv && (rank_ok || cap_ok)) {
      if (rel_gap <= ctl->tol) status = ST_CONVERGED;
    } else if (conv) {
      ctl->saved += 1;  // feasible (X_[r], y_[r]) of Alg. 2
      grow = true;
    } else if (it - ctl->k_change >= win && comb >= old) {
      grow = !rank_ok;
    }
    if (grow && !ctl->fixed_rank) {
      if (r >= ctl->max_rank || r >= n) status = ctl->at_max_rank ? ST_RUNNING : ST_STALLED_MAX_RANK;
      else status = ST_RANK_CHANGE;
    }
    if (status == ST_RUNNING && it >= ctl->it_stop) status = ST_PAUSE;
  }
  ctl->status = status;
  ctl->r_old = r;
  ctl->par = nw;       // X^{k+1} becomes the current iterate
  ctl->lz_done = 0;    // next projection starts
  ctl->lz_cycle = 0;
  if (use_cond) cudaGraphSetConditional(cond, status == ST_RUNNING ? 1u : 0u);
}


// Gram of the factor slots (only the first `act` columns of each slot; the
// deterministic split-row reduction of the Lanczos Gram kernel) followed, in
// the last block to finish, by the controller.
constexpr int GC_T = 16, GC_RC = 128;


__global__ void __launch_bounds__(256) k_gram_control(DevProblem pb, DevWork wk, int act, int rows_per_split,
                                                      int iter_launches, cudaGraphConditionalHandle cond,
                                                      int use_cond) {
  namespace cg = cooperative_groups;
  __shared__ float As[GC_RC][GC_T + 1];
  __shared__ float Bs[GC_RC][GC_T + 1];
  __shared__ double Pt[GC_T * GC_T];
  __shared__ unsigned s_last;
  const int tid = threadIdx.x;
  const int n = pb.n;
  const int slot = kMaxR, ka = 2 * kMaxR;
  const int per = (act + GC_T - 1) / GC_T;
  const int tiles_b = per * 2;
  const int ta = blockIdx.x / tiles_b, tb = blockIdx.x % tiles_b;
  const int a0 = (ta / per) * slot + (ta % per) * GC_T;
  const int b0 = (tb / per) * slot + (tb % per) * GC_T;
  const int ty = tid / GC_T, tx = tid % GC_T;
  const int rbeg = blockIdx.y * rows_per_split;
  const int rend = min(n, rbeg + rows_per_split);
  const float* A = wk.Vcm;
  const int lda = wk.ldq;
  DFc acc;
  constexpr int NL = GC_RC * GC_T / 256;
  float ra[NL], rb[NL];
  auto load_chunk = [&](int i0) {
#pragma unroll
    for (int v = 0; v < NL; ++v) {
      const int idx = tid + 256 * v;
      const int c = idx / GC_RC, i = idx % GC_RC;
      const int gi = i0 + i;
      ra[v] = (gi < rend) ? __ldg(&A[(size_t)(a0 + c) * lda + gi]) : 0.f;
      rb[v] = (gi < rend) ? __ldg(&A[(size_t)(b0 + c) * lda + gi]) : 0.f;
    }
  };
  if (rbeg < rend) load_chunk(rbeg);
  for (int i0 = rbeg; i0 < rend; i0 += GC_RC) {
#pragma unroll
    for (int v = 0; v < NL; ++v) {
      const int idx = tid + 256 * v;
      const int c = idx / GC_RC, i = idx % GC_RC;
      As[i][c] = ra[v];
      Bs[i][c] = rb[v];
    }
    __syncthreads();
    if (i0 + GC_RC < rend) load_chunk(i0 + GC_RC);
#pragma unroll 8
    for (int i = 0; i < GC_RC; ++i) acc.fma_acc(As[i][ty], Bs[i][tx]);
    __syncthreads();
  }
  // reduce the row splits of this tile across the cluster (split order)
  Pt[tid] = acc.value();
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();
  const int ns = gridDim.y;
  const int rank = (int)cluster.block_rank();
  const int per_rank = (GC_T * GC_T) / ns;
  if (tid < per_rank) {
    const int o = rank * per_rank + tid;
    double sum = 0.0;
    for (int sp = 0; sp < ns; ++sp) sum += cluster.map_shared_rank(Pt, sp)[o];
    wk.Hx[(size_t)(a0 + o / GC_T) * ka + b0 + o % GC_T] = sum;
  }
  cluster.sync();
  // the last CTA to finish runs the controller
  unsigned* cnt = wk.counters + CNT_CTL * 512;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&cnt[0], 1u) == gridDim.x * gridDim.y - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) cnt[0] = 0u;
  control_tail(pb, wk, wk.Hx, iter_launches, cond, use_cond);
}

// ---------------------------------------------------------------------------
// rebuild: S = V Lambda_+ V^T - alpha (D + shift 11^T)   (64 x 64 tiles)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rebuild(DevProblem pb, DevWork wk, int r, int sel) {
  extern __shared__ float smr[];
  const int ldr = r + 1;
  float* Ap = smr;                    // kTile x (r+1): lambda_+ scaled rows of V
  float* Bq = Ap + kTile * ldr;       // kTile x (r+1)
  float* Tl = Bq + kTile * ldr;       // kTile x (kTile+1)
  const int cur = sel ? 1 - wk.ctl->par : wk.ctl->par;
  const float* V = wk.Vrm[cur];
  const double* lam = wk.lam[cur];
  const int tid = threadIdx.x;
  const int bi = blockIdx.y, bj = blockIdx.x;
  const int p0 = bi * kTile, q0 = bj * kTile;
  const int n = pb.n;
#pragma unroll 4
  for (int idx = tid; idx < kTile * r; idx += blockDim.x) {
    int i = idx / r, t = idx % r;
    float lp = (float)fmax(lam[t], 0.0);
    Ap[i * ldr + t] = (p0 + i < n) ? lp * V[(size_t)(p0 + i) * wk.ldv + t] : 0.f;
    Bq[i * ldr + t] = (q0 + i < n) ? V[(size_t)(q0 + i) * wk.ldv + t] : 0.f;
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int t = 0; t < r; ++t) {
    float av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = Ap[(ty + 16 * a) * ldr + t];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bq[(tx + 16 * b) * ldr + t];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
  }
  const float ash = (float)(pb.alpha * wk.dshift[0]);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) Tl[(ty + 16 * a) * (kTile + 1) + tx + 16 * b] = acc[a][b] - ash;
  __syncthreads();
  const int tile = bi * pb.ntile + bj;
  for (int e = pb.tile_ptr[tile] + tid; e < pb.tile_ptr[tile + 1]; e += blockDim.x) {
    int loc = pb.tile_loc[e];
    Tl[(loc / kTile) * (kTile + 1) + loc % kTile] -= (float)(pb.alpha * wk.D[pb.tile_u[e]]);
  }
  __syncthreads();
  // element-wise box rows: M*(y) holds box_s (y_up - y_lo) / 2 off the diagonal
  const float abox = (float)(pb.alpha * 0.5 * (double)pb.box_s);
  for (int idx = tid; idx < kTile * kTile; idx += blockDim.x) {
    int i = idx / kTile, j = idx % kTile;
    if (p0 + i < n && q0 + j < n) {
      const size_t o = (size_t)(p0 + i) * wk.lds + q0 + j;
      float sv = Tl[i * (kTile + 1) + j];
      if (pb.box && p0 + i != q0 + j) sv -= abox * (wk.ybp[o] - wk.ybm[o]);
      wk.S[o] = sv;
    }
  }
}

// ---------------------------------------------------------------------------
// Element-wise box -u <= X_pq <= u (p != q) as a structured row class (the
// bounds of the MIMO relaxation, Sec. 5.3): per pair p < q the rows
// X_pq <= u and -X_pq <= u, i.e. A = +-s (E_pq + E_qp) / 2 with rhs s u
// (s = sqrt(2) when the rows are scaled to unit Frobenius norm), so that
// M(Z) = +-s Z_pq on them and M*(y) = s (y_up - y_lo) / 2 off the diagonal.
// The dual step of Sec. 2.2, y_half = y + alpha M(2 X+ - X) followed by
// y+ = y_half - alpha proj_{v <= rhs}(y_half / alpha), becomes per entry,
// with z = (2 X^{k+1} - X^k)_pq formed from the factors of both iterates,
//   y_up+ = max(0, y_up + alpha s (z - u)),   y_lo+ = max(0, y_lo - alpha s (z + u)).
// The kernel also sums the rows' shares of eps_dual^2, <dy, M(dX)>, rhs^T y
// and ||M*(dy)||_F^2 into Ctl::red_dvals[kRedBox..].  One CTA per tile pair
// bi <= bj; it writes (p, q) and, through shared memory, (q, p).
constexpr int BX_C = 32;  // factor columns staged per pass

__global__ void __launch_bounds__(256) k_box_dual(DevProblem pb, DevWork wk, int r) {
  __shared__ float smb[4 * kTile * (BX_C + 1)];
  __shared__ double sh[32 * 4];
  float* An = smb;                        // kTile x (BX_C+1): lambda_+ V rows p, new iterate
  float* Bn = An + kTile * (BX_C + 1);    // V rows q, new iterate
  float* Ao = Bn + kTile * (BX_C + 1);    // the same for the previous iterate
  float* Bo = Ao + kTile * (BX_C + 1);
  Ctl* ctl = wk.ctl;
  const int nw = 1 - ctl->par, od = ctl->par;
  const int ro = ctl->r_old;
  const int T = pb.ntile;
  int b = blockIdx.x, bi = 0;
  while (bi < T && b >= T - bi) {  // row bi of the upper tile triangle holds T - bi tiles
    b -= T - bi;
    ++bi;
  }
  const int bj = bi + b;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int n = pb.n;
  const int p0 = bi * kTile, q0 = bj * kTile;
  float xn[4][4], xo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      xn[a][c] = 0.f;
      xo[a][c] = 0.f;
    }
  const int rm = max(r, ro);
  for (int t0 = 0; t0 < rm; t0 += BX_C) {
    for (int idx = tid; idx < kTile * BX_C; idx += blockDim.x) {
      const int i = idx / BX_C, tt = idx % BX_C, t = t0 + tt;
      const bool okp = p0 + i < n, okq = q0 + i < n;
      const float ln = (t < r) ? (float)fmax(wk.lam[nw][t], 0.0) : 0.f;
      const float lo = (t < ro) ? (float)fmax(wk.lam[od][t], 0.0) : 0.f;
      An[i * (BX_C + 1) + tt] = (okp && t < r) ? ln * wk.Vrm[nw][(size_t)(p0 + i) * wk.ldv + t] : 0.f;
      Bn[i * (BX_C + 1) + tt] = (okq && t < r) ? wk.Vrm[nw][(size_t)(q0 + i) * wk.ldv + t] : 0.f;
      Ao[i * (BX_C + 1) + tt] = (okp && t < ro) ? lo * wk.Vrm[od][(size_t)(p0 + i) * wk.ldv + t] : 0.f;
      Bo[i * (BX_C + 1) + tt] = (okq && t < ro) ? wk.Vrm[od][(size_t)(q0 + i) * wk.ldv + t] : 0.f;
    }
    __syncthreads();
    const int tn = min(BX_C, rm - t0);
    for (int t = 0; t < tn; ++t) {
      float an[4], ao[4], bn[4], bo[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        an[a] = An[(ty + 16 * a) * (BX_C + 1) + t];
        ao[a] = Ao[(ty + 16 * a) * (BX_C + 1) + t];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        bn[c] = Bn[(tx + 16 * c) * (BX_C + 1) + t];
        bo[c] = Bo[(tx + 16 * c) * (BX_C + 1) + t];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          xn[a][c] = fmaf(an[a], bn[c], xn[a][c]);
          xo[a][c] = fmaf(ao[a], bo[c], xo[a][c]);
        }
    }
    __syncthreads();
  }
  float* Ut = smb;                        // kTile x (kTile+1): new y_up of the tile, then transposed out
  float* Lt = smb + kTile * (kTile + 1);  // new y_lo
  const double alpha = pb.alpha;
  const float as = (float)(alpha * (double)pb.box_s), u = pb.box_u;
  const double s = pb.box_s, su = (double)pb.box_s * (double)pb.box_u;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = ty + 16 * a, j = tx + 16 * c;
      const int p = p0 + i, q = q0 + j;
      if (p < q && q < n) {
        const size_t o = (size_t)p * wk.lds + q;
        const float z = 2.f * xn[a][c] - xo[a][c], dx = xn[a][c] - xo[a][c];
        const float yu = wk.ybp[o], yl = wk.ybm[o];
        const float yun = fmaxf(0.f, yu + as * (z - u));
        const float yln = fmaxf(0.f, yl - as * (z + u));
        wk.ybp[o] = yun;
        wk.ybm[o] = yln;
        Ut[i * (kTile + 1) + j] = yun;
        Lt[i * (kTile + 1) + j] = yln;
        const double du = (double)yun - (double)yu, dl = (double)yln - (double)yl;
        const double mdx = s * (double)dx;  // M(X+ - X) on the upper row; its negative on the lower
        const double e1 = du / alpha - mdx, e2 = dl / alpha + mdx;
        v[0] += e1 * e1 + e2 * e2;
        v[1] += mdx * (du - dl);
        v[2] += su * ((double)yun + (double)yln);
        v[3] += 0.5 * s * s * (du - dl) * (du - dl);
      }
    }
  __syncthreads();
  for (int idx = tid; idx < kTile * kTile; idx += blockDim.x) {  // (q, p): consecutive threads, consecutive p
    const int j = idx / kTile, i = idx % kTile;
    const int p = p0 + i, q = q0 + j;
    if (p < q && q < n) {
      const size_t o = (size_t)q * wk.lds + p;
      wk.ybp[o] = Ut[i * (kTile + 1) + j];
      wk.ybm[o] = Lt[i * (kTile + 1) + j];
    }
  }
  block_sum<4>(v, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) wk.part[(size_t)blockIdx.x * 4 + k] = v[k];
  if (!last_block(&wk.counters[CNT_BOX * 512])) return;
  __shared__ double tot[4];
  reduce_partials(wk.part, gridDim.x, 4, 4, tot);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) ctl->red_dvals[kRedBox + k] = tot[k];
    wk.counters[CNT_BOX * 512] = 0u;
  }
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__global__ void k_copy_cols(const float* src, int lds_, float* dst, int ldd, int n, int k,
                            const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * k) return;
  int c = (int)(idx / n), i = (int)(idx % n);
  dst[(size_t)c * ldd + i] = src[(size_t)c * lds_ + i];
}

// Full projection (n <= 128): eigenvectors of S from the dense one-block eigensolver
// become the factors of the new iterate (all n of them).
__global__ void k_full_eig_factors(DevWork wk, int n) {
  Ctl* ctl = wk.ctl;
  const int nw = 1 - ctl->par;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * kMaxR; idx += gridDim.x * blockDim.x) {
    int i = idx / kMaxR, t = idx % kMaxR;
    float v = (t < n) ? wk.Y[(size_t)t * kMaxK + i] : 0.f;
    wk.Vrm[nw][(size_t)i * wk.ldv + t] = v;
    if (t < n) {
      wk.Q[(size_t)t * wk.ldq + i] = v;
      wk.Vcm[(size_t)(nw * kMaxR + t) * wk.ldq + i] = v;
    }
  }
  if (blockIdx.x == 0) {
    for (int t = threadIdx.x; t < kMaxR; t += blockDim.x) {
      double cs = 0.0;
      if (t < n)
        for (int i = 0; i < n; ++i) cs += (double)wk.Y[(size_t)t * kMaxK + i];
      wk.lam[nw][t] = (t < n) ? wk.theta[t] : 0.0;
      wk.colsum[nw][t] = cs;
    }
    if (threadIdx.x == 0) {
      ctl->lz_done = 1;
      ctl->lz_res = 0.0;
    }
  }
}

__global__ void k_s_to_t(const float* S, int lds, int n, double* T) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int i = idx / n, j = idx % n;
  T[idx] = (double)S[(size_t)i * lds + j];
}

__global__ void k_ctl_set(Ctl* ctl, int status, int it_stop, int r, int w, int K, int k_change) {
  ctl->status = status;
  ctl->it_stop = it_stop;
  ctl->r = r;
  ctl->w = w;
  ctl->K = K;
  if (k_change >= 0) ctl->k_change = k_change;
}

// debugging aid: count non-finite entries of a buffer
template <typename T>
__global__ void k_count_nonfinite(const T* p, size_t count, unsigned* out) {
  unsigned c = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    c += !isfinite((double)p[i]);
  if (c) atomicAdd(out, c);
}

void launch_count_nonfinite_f(const float* p, size_t count, unsigned* out, cudaStream_t st) {
  k_count_nonfinite<float><<<64, 256, 0, st>>>(p, count, out);
}
void launch_count_nonfinite_d(const double* p, size_t count, unsigned* out, cudaStream_t st) {
  k_count_nonfinite<double><<<64, 256, 0, st>>>(p, count, out);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t ritz_smem(int K, int w) {
  return ((size_t)2 * RZ_RB * (K + 1) + (size_t)K * w + (size_t)2 * RZ_RB * (w + 1)) * sizeof(float);
}
static size_t rebuild_smem(int r) {
  return ((size_t)2 * kTile * (r + 1) + (size_t)kTile * (kTile + 1)) * sizeof(float);
}

void init_pdhg_attributes() {
  cudaFuncSetAttribute(k_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ritz_smem(kMaxK, kMaxP));
  cudaFuncSetAttribute(k_rebuild, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rebuild_smem(kMaxR));
}

void launch_ritz(const DevWork& wk, int n, int K, int w, int r, int s_steps, int cycle_launches,
                 cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st) {
  int blocks = (n + RZ_RB - 1) / RZ_RB;
  k_ritz<<<blocks, 256, ritz_smem(K, w), st>>>(wk, n, K, w, r, s_steps, cycle_launches, cond, use_cond);
}

void launch_mxdual(const DevProblem& pb, const DevWork& wk, int r, cudaStream_t st) {
  int blocks = (pb.n_chunks * 32 + 255) / 256;
  if (blocks < 1) blocks = 1;
  k_mxdual<<<blocks, 256, 0, st>>>(pb, wk, r);
}

void launch_dvals(const DevProblem& pb, const DevWork& wk, cudaStream_t st) {
  int blocks = (pb.nU + 255) / 256;
  if (blocks < 1) blocks = 1;
  k_dvals<<<blocks, 256, 0, st>>>(pb, wk);
}

void launch_gram_control(const DevProblem& pb, const DevWork& wk, int act, int iter_launches,
                         cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st) {
  const int per = (act + GC_T - 1) / GC_T;
  const int tiles = per * 2 * per * 2;
  int ns = 1;
  const int sms = num_sms();
  while (ns < 8 && tiles * ns * 2 <= sms && pb.n >= 2 * ns * 256) ns *= 2;
  const int rows = (pb.n + ns - 1) / ns;
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
  cudaLaunchKernelEx(&cfg, k_gram_control, pb, wk, act, rows, iter_launches, cond, use_cond);
}

void launch_box_dual(const DevProblem& pb, const DevWork& wk, int r, cudaStream_t st) {
  const int T = pb.ntile;
  k_box_dual<<<T * (T + 1) / 2, 256, 0, st>>>(pb, wk, r);
}

void launch_rebuild(const DevProblem& pb, const DevWork& wk, int r, int sel, cudaStream_t st) {
  dim3 grid(pb.ntile, pb.ntile);
  int rr = r < 1 ? 1 : r;
  k_rebuild<<<grid, 256, rebuild_smem(rr), st>>>(pb, wk, r, sel);
}

void launch_copy_cols(const float* src, int lds, float* dst, int ldd, int n, int k, const int* skip,
                      cudaStream_t st) {
  size_t total = (size_t)n * k;
  k_copy_cols<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(src, lds, dst, ldd, n, k, skip);
}

void launch_full_eig_factors(const DevWork& wk, int n, cudaStream_t st) {
  k_full_eig_factors<<<32, 256, 0, st>>>(wk, n);
}

void launch_s_to_t(const float* S, int lds, int n, double* T, cudaStream_t st) {
  k_s_to_t<<<(n * n + 255) / 256, 256, 0, st>>>(S, lds, n, T);
}

void launch_ctl_set(Ctl* ctl, int status, int it_stop, int r, int w, int K, int k_change,
                    cudaStream_t st) {
  k_ctl_set<<<1, 1, 0, st>>>(ctl, status, it_stop, r, w, K, k_change);
}

}  // namespace psdp
