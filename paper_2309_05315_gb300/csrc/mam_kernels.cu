// libmam device code: the per-iteration kernels of the Method of Averaged
// Marginals (arXiv 2309.05315, Algorithm 1) for sm_103a.
//
//   column_kernel   (mam_column.cuh; the dense-plan instances are launched
//                   from here) Step 2 of Algorithm 1 for every column of the
//                   index set M^k, fused with the row sums of Step 3
//                   (order-independent fixed-point accumulation) and with the
//                   diagnostics (W-hat, lower bound, fixed-point residual).
//   average_kernel  Step 3 completion (64-bit fixed point), Step 1 (p = sum_m a_m p^(m),
//                   eq. pr) and the factor t^k.
//
// Plans theta and costs c are stored column-contiguous with a padded stride
// ld (a multiple of 8 elements), so that one column is one contiguous run of
// 4*ld (theta) and ld*sizeof(cost) bytes: each column is brought into shared
// memory by two bulk-async copies (cp.async.bulk, completion on an mbarrier)
// while the CTA works on the previous column.
#include "mam_column.cuh"

#include <cfloat>
#include <cmath>
#include <type_traits>

namespace mam {
namespace {

// ------------------------------------------------------ average kernel

// Step 3 completion and Step 1 of Algorithm 1:
//   p^(m)_r = sum_s pihat_rs - S_m d_r   (row sums of theta' = pihat - d)
//   p = sum_m a_m p^(m)                  (eq. pr)
//   delta^(m) = (p - p^(m)) / S_m        (the next column step uses t delta)
// and the block sums of sum_m ||p - p^(m)||^2 / S_m (dist_L(theta)^2, which
// fixes t^k), of the same for the pi-hat marginals (diagnostics) and of
// ||p_new - p_old||^2.  p^(m) and p are 64-bit fixed point (scale F = 2^e):
// sum_s pihat arrives as an integer, d is an FP32 value whose product with F
// is rounded to an integer, S_m d and the differences are exact, and
// a_m p^(m) is a 64 x 64-bit product with a_m held to 2^-62; no per-(m, r)
// step uses the FP64 pipe.  Only the measures of the index set just
// processed get new p^(m); the others keep theirs (Remark 2).
// Block (kAvgThreads / SL rows) x (SL measure slices): threadIdx.x picks the
// row, threadIdx.y a slice of the measures (m = m0 + y + k SL), so each
// thread walks several measures with independent loads; slices are combined
// in shared memory.  Grid (ceil(R / rows), P).
template <int SL, bool DIAG>
__global__ void __launch_bounds__(kAvgThreads) average_kernel(const AvgArgs A) {
  constexpr int RX = kAvgThreads / SL;
  constexpr int NW = kAvgThreads / 32;
  __shared__ long long sp[SL][RX];
  __shared__ double sq[SL][RX];
  __shared__ float se[NW];
  __shared__ double sr[NW][2];
  __shared__ float t_sh;
  pdl_wait();         // the column step's row sums and t are complete
  pdl_launch_next();  // the next column step may start copying its columns
  const int pr = blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int flat = ty * RX + tx;
  const int r = blockIdx.x * RX + tx;
  const int m0 = A.prob_meas[pr], m1 = A.prob_meas[pr + 1];
  if (flat == 0) t_sh = float(A.t_used[pr]);
  const Sched sc = A.sched[draw_index_set(A.draw, *A.iter - 1)];
  const bool row = r < A.R;
  constexpr bool diag = DIAG;  // compile-time: no FP64 per (m, r) without diagnostics
  __syncthreads();
  const float t_old = t_sh;
  // pass 1: new marginals of this slice's measures, partial sums of a_m p^(m).
  // Measures go in groups of kAvgGroup whose loads are all issued before any
  // store (the stores could alias later loads, which would serialise the L2
  // round trips); the first kAvgKeep marginals stay in registers for pass 2.
  const bool upd_all = A.reduce != 0;
  long long ps = 0;
  double phs = 0.0;
  long long pmr[kAvgKeep];
  const int mb = m0 + ty;
  const int nk = row && mb < m1 ? (m1 - mb + SL - 1) / SL : 0;  // this thread's measures
#pragma unroll
  for (int k0 = 0; k0 < kAvgKeep; k0 += kAvgGroup) {
    if (k0 >= nk) break;
    long long av[kAvgGroup];
    float dlv[kAvgGroup];
#pragma unroll
    for (int u = 0; u < kAvgGroup; ++u) {
      const int m = mb + (k0 + u) * SL;
      av[u] = 0;
      dlv[u] = 0.f;
      if (k0 + u < nk) {
        const size_t o = size_t(m) * A.R + r;
        const bool upd = upd_all && m >= sc.meas_begin && m < sc.meas_end;
        av[u] = upd ? (long long)A.acc[o] : A.pm[o];
        if (upd) dlv[u] = A.delta32[size_t(m) * A.ld + r];
      }
    }
#pragma unroll
    for (int u = 0; u < kAvgGroup; ++u) {
      const int m = mb + (k0 + u) * SL;
      if (k0 + u < nk) {
        const size_t o = size_t(m) * A.R + r;
        const bool upd = upd_all && m >= sc.meas_begin && m < sc.meas_end;
        long long pmv = av[u];
        if (upd) {
          A.acc[o] = 0ull;
          // the column kernel subtracted d = float(t delta) from every entry
          const float d_used = __fmul_rn(t_old, dlv[u]);
          if (A.d_last) A.d_last[size_t(m) * A.ld + r] = d_used;  // sparse plans
          const long long d_fx = f32_to_i64_rn(d_used * A.fx_f);  // F = 2^e: exact scaling
          if (diag) A.phat[o] = double(av[u]) * A.fx_inv_scale;
          pmv = av[u] - (long long)__ldg(A.S + m) * d_fx;
          A.pm[o] = pmv;
        }
        pmr[k0 + u] = pmv;
        ps += mul_q62(pmv, __ldg(A.a_q + m));
        if (diag) phs += A.a[m] * A.phat[o];
      }
    }
  }
  for (int k = kAvgKeep; k < nk; ++k) {  // more measures than registers: plain loop
    const int m = mb + k * SL;
    const size_t o = size_t(m) * A.R + r;
    long long pmv;
    if (upd_all && m >= sc.meas_begin && m < sc.meas_end) {
      const long long sum_pihat = (long long)A.acc[o];
      A.acc[o] = 0ull;
      const float d_used = __fmul_rn(t_old, A.delta32[size_t(m) * A.ld + r]);
      if (A.d_last) A.d_last[size_t(m) * A.ld + r] = d_used;
      const long long d_fx = f32_to_i64_rn(d_used * A.fx_f);
      if (diag) A.phat[o] = double(sum_pihat) * A.fx_inv_scale;
      pmv = sum_pihat - (long long)A.S[m] * d_fx;
      A.pm[o] = pmv;
    } else {
      pmv = A.pm[o];
    }
    ps += mul_q62(pmv, A.a_q[m]);
    if (diag) phs += A.a[m] * A.phat[o];
  }
  long long p_fx = ps;
  double ph = phs;
  if (SL > 1) {
    sp[ty][tx] = ps;
    if (diag) sq[ty][tx] = phs;
    __syncthreads();
    p_fx = 0;
    ph = 0.0;
#pragma unroll
    for (int y = 0; y < SL; ++y) p_fx += sp[y][tx];
    if (diag)
      for (int y = 0; y < SL; ++y) ph += sq[y][tx];
  }
  // pass 2: shifts and the distance terms
  float e = 0.f;
  double eh = 0.0, dp2 = 0.0;
  if (row) {
#pragma unroll
    for (int k = 0; k < kAvgKeep; ++k) {
      if (k >= nk) break;
      const int m = mb + k * SL;
      const long long dfx = p_fx - pmr[k];  // (p - p^(m)) F, exact
      A.delta32[size_t(m) * A.ld + r] = shift_f32(dfx, __ldg(A.inv_SFd + m));
      const float dv = i64_to_f32(dfx) * A.fx_inv_f;
      e = fmaf(dv * dv, __ldg(A.inv_S + m), e);
      if (diag) {
        const double dh = ph - A.phat[size_t(m) * A.R + r];
        eh += dh * dh * A.inv_Sd[m];
      }
    }
    for (int k = kAvgKeep; k < nk; ++k) {
      const int m = mb + k * SL;
      const size_t o = size_t(m) * A.R + r;
      const long long dfx = p_fx - A.pm[o];
      A.delta32[size_t(m) * A.ld + r] = shift_f32(dfx, A.inv_SFd[m]);
      const float dv = i64_to_f32(dfx) * A.fx_inv_f;
      e = fmaf(dv * dv, A.inv_S[m], e);
      if (diag) {
        const double dh = ph - A.phat[o];
        eh += dh * dh * A.inv_Sd[m];
      }
    }
    if (ty == 0) {
      double* pp = A.p + size_t(pr) * A.R + r;
      const double p_new = double(p_fx) * A.fx_inv_scale;
      const double dd = p_new - *pp;
      dp2 = dd * dd;
      *pp = p_new;
    }
  }
  const int warp = flat >> 5, lane = flat & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if (diag) eh = warp_sum_d(eh);
  if (warp < (RX + 31) / 32) dp2 = warp_sum_d(dp2);  // only slice-0 rows carry dp2
  if (lane == 0) {
    se[warp] = e;
    sr[warp][0] = eh;
    sr[warp][1] = dp2;
  }
  __syncthreads();
  if (flat == 0) {
    double b0 = 0, b1 = 0, b2 = 0;
    for (int i = 0; i < NW; ++i) {
      b0 += double(se[i]);
      b1 += sr[i][0];
      b2 += sr[i][1];
    }
    double* blk = A.blk + (size_t(pr) * gridDim.x + blockIdx.x) * 4;
    blk[0] = b0;
    blk[1] = b1;
    blk[2] = b2;
  }
}

// --------------------------------------------------------- other kernels

// Sums of the per-column diagnostics of problem blockIdx.x, FP64, fixed
// order: out[3*i] = sum wc, out[3*i+1] = sum lb, out[3*i+2] = sum res over
// the columns of the last index set.
__global__ void __launch_bounds__(256) diag_reduce_kernel(
    const float* wc, const float* lb, const float* res,
    const long long* prob_cols, const Sched* sched, Draw draw,
    const long long* iter, double* out) {
  __shared__ double sh[8][3];
  const int i = blockIdx.x;
  const long long c0 = prob_cols[i], c1 = prob_cols[i + 1];
  long long r0 = c0, r1 = c1;
  if (draw.nb > 1) {
    const Sched sc = sched[draw_index_set(draw, *iter - 1)];
    r0 = sc.col_begin > c0 ? sc.col_begin : c0;
    r1 = sc.col_end < c1 ? sc.col_end : c1;
  }
  double a = 0, b = 0, c = 0;
  for (long long k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
    a += double(wc[k]);
    b += double(lb[k]);
    if (k >= r0 && k < r1) c += double(res[k]);
  }
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  c = warp_sum_d(c);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[warp][0] = a;
    sh[warp][1] = b;
    sh[warp][2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0, z = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      x += sh[w][0];
      y += sh[w][1];
      z += sh[w][2];
    }
    out[3 * i] = x;
    out[3 * i + 1] = y;
    out[3 * i + 2] = z;
  }
}

// Lower bound only (randomized runs, where the fused value would mix index
// sets): diag_lb[col] = q_s * min_r (c_rs - rho_m t (p_r - p^(m)_r) / S_m).
// One warp per column.
template <typename CT>
__global__ void __launch_bounds__(256) lb_kernel(
    const CT* cost, const int* cost_col, const float* cmul, const float* gen_xi,
    const float4* gen_zeta, const float* q, const float* delta32, const double* t_used,
    const int* meas_prob, const float* rho, const int* col_meas, long long T,
    int R, int ld, float lb_cap, float* diag_lb) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long col = w0; col < T; col += nwarp) {
    const int m = col_meas[col];
    const float tt = float(t_used[meas_prob[m]]);
    const float rh = rho[m];
    const float* dl = delta32 + size_t(m) * ld;
    const CT* cc = gen_xi ? nullptr
                          : cost + size_t(cost_col ? (long long)cost_col[col] : col) * ld;
    const float cm = cmul[m];
    const float* xg = gen_xi ? gen_xi + size_t(meas_prob[m]) * 3 * ld : nullptr;
    const float4 zg = gen_xi ? gen_zeta[col] : make_float4(0.f, 0.f, 0.f, 0.f);
    float mn = INFINITY;
    for (int r = lane; r < R; r += 32) {
      float c;
      if (gen_xi) c = gen_cost(xg, ld, r, zg);
      else if constexpr (sizeof(CT) == 4) c = float(cc[r]);
      else if constexpr (std::is_same<CT, __half>::value) c = __half2float(cc[r]);
      else c = __bfloat162float(cc[r]);
      mn = fminf(mn, cm * c - rh * __fmul_rn(tt, dl[r]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if (lane == 0) diag_lb[col] = q[col] * fminf(mn, lb_cap);
  }
}


}  // namespace

int column_max_threads(int nv) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return MaxThreads<N>::value;
    MAM_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return 0;
  }
}

cudaError_t launch_column(int nv, int cost_dtype, bool diag, int grid,
                          int threads, size_t smem, cudaStream_t st,
                          const ColArgs& a) {
  return col_op_any<false>(nv, cost_dtype, 0, diag, grid, threads, smem, st, &a, nullptr);
}

cudaError_t set_column_smem(int nv, int cost_dtype, bool diag, size_t smem) {
  return col_op_any<false>(nv, cost_dtype, 1, diag, 0, 0, smem, nullptr, nullptr, nullptr);
}

cudaError_t column_occupancy(int nv, int cost_dtype, bool diag, int threads,
                             size_t smem, int* blocks_per_sm) {
  return col_op_any<false>(nv, cost_dtype, 2, diag, 0, threads, smem, nullptr, nullptr,
                    blocks_per_sm);
}

cudaError_t launch_average(const AvgArgs& a, int nblk, cudaStream_t st) {
  const dim3 grid(nblk, a.P);
  const bool dg = a.diag != 0;
  switch (a.slices) {
    case 1:
      return dg ? launch_pdl(average_kernel<1, true>, grid, dim3(kAvgThreads, 1), 0, st, a)
                : launch_pdl(average_kernel<1, false>, grid, dim3(kAvgThreads, 1), 0, st, a);
    case 2:
      return dg ? launch_pdl(average_kernel<2, true>, grid, dim3(kAvgThreads / 2, 2), 0, st, a)
                : launch_pdl(average_kernel<2, false>, grid, dim3(kAvgThreads / 2, 2), 0, st, a);
    case 4:
      return dg ? launch_pdl(average_kernel<4, true>, grid, dim3(kAvgThreads / 4, 4), 0, st, a)
                : launch_pdl(average_kernel<4, false>, grid, dim3(kAvgThreads / 4, 4), 0, st, a);
    case 8:
      return dg ? launch_pdl(average_kernel<8, true>, grid, dim3(kAvgThreads / 8, 8), 0, st, a)
                : launch_pdl(average_kernel<8, false>, grid, dim3(kAvgThreads / 8, 8), 0, st, a);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_lb(int cost_dtype, const void* cost, const int* cost_col,
                      const float* cmul, const float* gen_xi, const float4* gen_zeta,
                      const float* q,
                      const float* delta32, const double* t_used,
                      const int* meas_prob, const float* rho,
                      const int* col_meas, long long T, int R, int ld,
                      float lb_cap, float* diag_lb, cudaStream_t st) {
  long long g = (T * 32 + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  switch (cost_dtype) {
    case 0:
      lb_kernel<float><<<int(g), 256, 0, st>>>(static_cast<const float*>(cost), cost_col, cmul, gen_xi, gen_zeta, q, delta32, t_used, meas_prob, rho, col_meas, T, R, ld, lb_cap, diag_lb);
      break;
    case 1:
      lb_kernel<__nv_bfloat16><<<int(g), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(cost), cost_col, cmul, gen_xi, gen_zeta, q, delta32, t_used, meas_prob, rho, col_meas, T, R, ld, lb_cap, diag_lb);
      break;
    case 2:
      lb_kernel<__half><<<int(g), 256, 0, st>>>(static_cast<const __half*>(cost), cost_col, cmul, gen_xi, gen_zeta, q, delta32, t_used, meas_prob, rho, col_meas, T, R, ld, lb_cap, diag_lb);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_diag_reduce(const float* wc, const float* lb,
                               const float* res, const long long* prob_cols,
                               const Sched* sched, Draw draw,
                               const long long* iter, int P, double* out,
                               cudaStream_t st) {
  diag_reduce_kernel<<<P, 256, 0, st>>>(wc, lb, res, prob_cols, sched, draw,
                                        iter, out);
  return cudaGetLastError();
}

}  // namespace mam
