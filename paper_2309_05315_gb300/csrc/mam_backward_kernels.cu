// libmam: reverse mode through unrolled MAM iterations (balanced,
// deterministic, t = 1).
//
// One forward iteration (Algorithm 1) maps theta to theta' by
//   d^(m) = (p - p^(m)) / S_m,  p^(m) = row sums of theta^(m),  p = sum a_m p^(m)
//   w = theta + 2 d - c / rho,  pihat = max(w - lambda, 0) with
//   sum_r pihat = q_s,  theta' = pihat - d.
// Where the active sets A_s = {r : w_r > lambda_s} do not change, pihat is
// affine in (w, q): d pihat / d w = I_A - 1_A 1_A^T / |A| and
// d pihat / d q_s = 1_A / |A|.  Given thetabar' (the gradient w.r.t. theta')
// the reverse step is
//   wbar = [A] (thetabar' - mean_A thetabar'),   qbar_s += mean_A thetabar',
//   cbar = -wbar / rho,   dbar^(m)_r = sum_s (2 wbar_rs - thetabar'_rs),
//   pbar = sum_m dbar^(m) / S_m,   pbarm^(m) = -dbar^(m) / S_m + a_m pbar,
//   thetabar = wbar + pbarm^(m) broadcast along each column,
// and the cost c^(m)_rs = alpha_m ||xi_r - zeta_s||^2 gives
//   zetabar_s += (2 alpha_m / rho) sum_r wbar_rs (xi_r - zeta_s),
//   xibar_r   -= (2 alpha_m / rho) sum_s wbar_rs (xi_r - zeta_s).
// thetabar is kept as a column-sparse part ("stored": wbar, zero off the
// active set) plus a per-(measure,row) part ("pend": pbarm).  Since the stored
// part entering step k is the wbar of step k+1, sum_s thetabar'_rs =
// (sum_s wbar^(k+1)_rs) + S_m pend_r: the row sums of one step are reused by
// the next and no column is read twice.
//
// Layout of the work: a CTA owns a chunk of consecutive columns of one
// measure and a thread owns fixed rows r = tid + i * blockDim.x of every
// column of its chunk, so the per-row sums over the chunk (sum_s wbar_rs and
// sum_s wbar_rs zeta_s) stay in registers.  Each chunk writes them once; the
// row kernel adds the chunks of a measure in a fixed order.  No atomics, and
// the result does not depend on scheduling.
#include "mam_device.cuh"
#include "mam_internal.h"

namespace mam {
namespace {

template <int N, typename V>
__device__ __forceinline__ void block_sum_n(V (&v)[N], V (*sh)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  __syncthreads();  // the previous call's readers are done
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < N; ++j) sh[warp][j] = v[j];
  }
  __syncthreads();
  const int nw = int(blockDim.x >> 5);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    V t = V(0);
    for (int w = 0; w < nw; ++w) t += sh[w][j];
    v[j] = t;
  }
}

// One reverse step over the columns of chunk blockIdx.x.  Per-entry
// arithmetic is FP32 (the FP64 pipe of this GPU is a small fraction of its
// FP32 rate); per-column and per-row results are accumulated in FP64.
template <int NVB, typename CT, int DIM>
__global__ void __launch_bounds__(kBwdMaxThreads) bwd_column_kernel(const BwdArgs A) {
  __shared__ float sh[kBwdMaxThreads / 32][4];
  constexpr int DZ = DIM > 0 ? DIM : 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long c0 = A.chunk_begin[blockIdx.x], c1 = A.chunk_begin[blockIdx.x + 1];
  const int m = A.col_meas[c0];
  const int R = A.R, ld = A.ld;
  const float irho = A.irho[m];
  const double coef = 2.0 * A.alpha[m] / A.rho;
  float d[NVB], pd[NVB], accW[NVB], accZ[NVB][DZ], xr[NVB][DZ];
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    const int r = tid + i * nt;
    d[i] = r < R ? A.delta32[size_t(m) * ld + r] : 0.f;  // t = 1: d = delta32
    pd[i] = r < R ? float(A.pend[size_t(m) * R + r]) : 0.f;
    accW[i] = 0.f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      accZ[i][k] = 0.f;
      xr[i][k] = r < R ? float(A.xi[size_t(r) * DIM + k]) : 0.f;
    }
  }
  for (long long col = c0; col < c1; ++col) {
    const float* th = A.theta + size_t(col) * ld;
    const CT* c = static_cast<const CT*>(A.cost) + size_t(col) * ld;
    float* st = A.stored + size_t(col) * ld;
    const float lam = A.lam[col];
    float tb[NVB];
    bool act[NVB];
    float v2[2] = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NVB; ++i) {
      const int r = tid + i * nt;
      act[i] = false;
      tb[i] = 0.f;
      if (r < R) {
        // w exactly as the forward column step formed it
        const float w = fmaf(-float(c[r]), irho, fmaf(2.f, d[i], th[r]));
        act[i] = w > lam;
        tb[i] = st[r] + pd[i];
        if (act[i]) {
          v2[0] += tb[i];
          v2[1] += 1.f;
        }
      }
    }
    block_sum_n<2, float>(v2, sh);
    const float mean = v2[1] > 0.f ? v2[0] / v2[1] : 0.f;
    float zs[DZ], zx[DZ];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      zs[k] = float(A.zeta[size_t(col) * DIM + k]);
      zx[k] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < NVB; ++i) {
      const int r = tid + i * nt;
      if (r >= R) continue;
      const float wb = act[i] ? tb[i] - mean : 0.f;
      st[r] = wb;
      if (act[i]) {
        accW[i] += wb;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          accZ[i][k] = fmaf(wb, zs[k], accZ[i][k]);
          zx[k] = fmaf(wb, xr[i][k] - zs[k], zx[k]);
        }
      }
    }
    if (DIM > 0) block_sum_n<DZ, float>(zx, sh);
    if (tid == 0) {
      A.qbar[col] += double(mean);
#pragma unroll
      for (int k = 0; k < DIM; ++k) A.zetabar[size_t(col) * DIM + k] += coef * double(zx[k]);
    }
  }
  // chunk partials, [chunk][1 + DIM][R]
  double* part = A.part + size_t(blockIdx.x) * (1 + DIM) * R;
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    const int r = tid + i * nt;
    if (r >= R) continue;
    part[r] = double(accW[i]);
#pragma unroll
    for (int k = 0; k < DIM; ++k) part[size_t(1 + k) * R + r] = double(accZ[i][k]);
  }
}

// Per row r: dbar, pbar, the new broadcast part of thetabar and xibar.
// acc_prev holds sum_s wbar^(k+1)_rs (the stored part entering this step).
__global__ void bwd_row_kernel(const BwdArgs A) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.R) return;
  const int dim = A.dim, R = A.R;
  double pbar = 0.0;
  for (int m = 0; m < A.Mtot; ++m) {
    double w = 0.0;
    for (int j = A.meas_chunk[m]; j < A.meas_chunk[m + 1]; ++j)
      w += A.part[size_t(j) * (1 + dim) * R + r];
    const size_t o = size_t(m) * R + r;
    const double dbar = 2.0 * w - (A.acc_prev[o] + A.Sd[m] * A.pend[o]);
    A.acc_w[o] = w;
    pbar += dbar / A.Sd[m];
  }
  for (int m = 0; m < A.Mtot; ++m) {
    const size_t o = size_t(m) * R + r;
    const double w = A.acc_w[o];
    const double dbar = 2.0 * w - (A.acc_prev[o] + A.Sd[m] * A.pend[o]);
    const double coef = 2.0 * A.alpha[m] / A.rho;
    for (int k = 0; k < dim; ++k) {
      double wz = 0.0;
      for (int j = A.meas_chunk[m]; j < A.meas_chunk[m + 1]; ++j)
        wz += A.part[(size_t(j) * (1 + dim) + 1 + k) * R + r];
      A.xibar[size_t(r) * dim + k] -= coef * (A.xi[size_t(r) * dim + k] * w - wz);
    }
    A.pend[o] = -dbar / A.Sd[m] + A.a[m] * pbar;
    A.acc_prev[o] = w;
  }
}

// theta^0_rs = q_s / R: qbar_s += sum_r thetabar^0_rs / R.
__global__ void __launch_bounds__(256) bwd_theta0_kernel(const BwdArgs A) {
  __shared__ double sh[8][4];
  const long long col = blockIdx.x;
  const int m = A.col_meas[col];
  double s[1] = {0.0};
  for (int r = threadIdx.x; r < A.R; r += blockDim.x)
    s[0] += double(A.stored[size_t(col) * A.ld + r]) + A.pend[size_t(m) * A.R + r];
  block_sum_n<1, double>(s, sh);
  if (threadIdx.x == 0) A.qbar[col] += s[0] / double(A.R);
}

template <int NVB, int DIM>
cudaError_t bwd_col_dt(int dt, int nchunks, int nt, cudaStream_t st, const BwdArgs& a) {
  switch (dt) {
    case 0: bwd_column_kernel<NVB, float, DIM><<<nchunks, nt, 0, st>>>(a); break;
    case 1: bwd_column_kernel<NVB, __nv_bfloat16, DIM><<<nchunks, nt, 0, st>>>(a); break;
    case 2: bwd_column_kernel<NVB, __half, DIM><<<nchunks, nt, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NVB>
cudaError_t bwd_col_nv(int dt, int dim, int nchunks, int nt, cudaStream_t st, const BwdArgs& a) {
  switch (dim) {
    case 0: return bwd_col_dt<NVB, 0>(dt, nchunks, nt, st, a);
    case 1: return bwd_col_dt<NVB, 1>(dt, nchunks, nt, st, a);
    case 2: return bwd_col_dt<NVB, 2>(dt, nchunks, nt, st, a);
    case 3: return bwd_col_dt<NVB, 3>(dt, nchunks, nt, st, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int bwd_max_rows() { return 8 * kBwdMaxThreads; }

static int bwd_threads(int R) { return R <= 4 * 256 ? 256 : kBwdMaxThreads; }

cudaError_t launch_bwd_step(int cost_dtype, int nchunks, cudaStream_t st, const BwdArgs& a) {
  const int nt = bwd_threads(a.R);
  const int need = (a.R + nt - 1) / nt;
  cudaError_t e;
  if (need <= 1) e = bwd_col_nv<1>(cost_dtype, a.dim, nchunks, nt, st, a);
  else if (need <= 2) e = bwd_col_nv<2>(cost_dtype, a.dim, nchunks, nt, st, a);
  else if (need <= 4) e = bwd_col_nv<4>(cost_dtype, a.dim, nchunks, nt, st, a);
  else if (need <= 6) e = bwd_col_nv<6>(cost_dtype, a.dim, nchunks, nt, st, a);
  else if (need <= 8) e = bwd_col_nv<8>(cost_dtype, a.dim, nchunks, nt, st, a);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  bwd_row_kernel<<<(a.R + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bwd_theta0(long long T, cudaStream_t st, const BwdArgs& a) {
  bwd_theta0_kernel<<<unsigned(T), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mam
