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
// active set) plus a per-(measure,row) part ("pend": pbarm), which keeps every
// row accumulation sparse.
#include "mam_device.cuh"
#include "mam_internal.h"

namespace mam {

namespace {

constexpr int kBwdThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

template <int NVB, typename CT>
__global__ void __launch_bounds__(kBwdThreads) bwd_column_kernel(const BwdArgs A) {
  __shared__ double sh[32];
  const long long col = blockIdx.x;
  const int tid = threadIdx.x;
  const int m = A.col_meas[col];
  const int R = A.R, ld = A.ld, dim = A.dim;
  const float* th = A.theta + size_t(col) * ld;
  const CT* c = static_cast<const CT*>(A.cost) + size_t(col) * ld;
  const float* dl = A.delta32 + size_t(m) * ld;
  float* st = A.stored + size_t(col) * ld;
  const double* pd = A.pend + size_t(m) * R;
  const float lam = A.lam[col];
  const float irho = A.irho[m];
  double tb[NVB];
  float so[NVB];
  bool act[NVB];
  double s1 = 0.0, na = 0.0;
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    const int r = tid + i * kBwdThreads;
    act[i] = false;
    tb[i] = 0.0;
    so[i] = 0.f;
    if (r < R) {
      const float d = dl[r];  // t = 1: d = delta32 exactly
      const float w = fmaf(-float(c[r]), irho, fmaf(2.f, d, th[r]));
      act[i] = w > lam;
      so[i] = st[r];
      tb[i] = double(so[i]) + pd[r];
      if (act[i]) {
        s1 += tb[i];
        na += 1.0;
      }
    }
  }
  s1 = block_sum_d(s1, sh);
  na = block_sum_d(na, sh);
  const double mean = na > 0 ? s1 / na : 0.0;
  const double* zs = A.zeta + size_t(col) * dim;
  double zx[3] = {0.0, 0.0, 0.0}, zw = 0.0;
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    const int r = tid + i * kBwdThreads;
    if (r >= R) continue;
    const double wb = act[i] ? tb[i] - mean : 0.0;
    st[r] = float(wb);
    const size_t o = size_t(m) * R + r;
    if (so[i] != 0.f) atomicAdd(A.acc_t + o, double(so[i]));
    if (act[i]) {
      atomicAdd(A.acc_w + o, wb);
      for (int k = 0; k < dim; ++k) {
        atomicAdd(A.acc_wz + o * dim + k, wb * zs[k]);
        zx[k] += wb * A.xi[size_t(r) * dim + k];
      }
      zw += wb;
    }
  }
  const double coef = 2.0 * A.alpha[m] / A.rho;
  double tot[3];
  for (int k = 0; k < 3; ++k) tot[k] = (k < dim) ? block_sum_d(zx[k], sh) : 0.0;
  const double zwt = block_sum_d(zw, sh);
  if (tid == 0) {
    A.qbar[col] += mean;
    for (int k = 0; k < dim; ++k) A.zetabar[size_t(col) * dim + k] += coef * (tot[k] - zs[k] * zwt);
  }
}

// Per row r: dbar, pbar, the new broadcast part of thetabar and xibar.
__global__ void bwd_row_kernel(const BwdArgs A) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.R) return;
  double pbar = 0.0;
  for (int m = 0; m < A.Mtot; ++m) {
    const size_t o = size_t(m) * A.R + r;
    const double dbar = 2.0 * A.acc_w[o] - (A.acc_t[o] + A.Sd[m] * A.pend[o]);
    pbar += dbar / A.Sd[m];
  }
  for (int m = 0; m < A.Mtot; ++m) {
    const size_t o = size_t(m) * A.R + r;
    const double dbar = 2.0 * A.acc_w[o] - (A.acc_t[o] + A.Sd[m] * A.pend[o]);
    const double coef = 2.0 * A.alpha[m] / A.rho;
    for (int k = 0; k < A.dim; ++k)
      A.xibar[size_t(r) * A.dim + k] -=
          coef * (A.xi[size_t(r) * A.dim + k] * A.acc_w[o] - A.acc_wz[o * A.dim + k]);
    A.pend[o] = -dbar / A.Sd[m] + A.a[m] * pbar;
    A.acc_w[o] = 0.0;
    A.acc_t[o] = 0.0;
    for (int k = 0; k < A.dim; ++k) A.acc_wz[o * A.dim + k] = 0.0;
  }
}

// theta^0_rs = q_s / R: qbar_s += sum_r thetabar^0_rs / R.
__global__ void __launch_bounds__(kBwdThreads) bwd_theta0_kernel(const BwdArgs A) {
  __shared__ double sh[32];
  const long long col = blockIdx.x;
  const int m = A.col_meas[col];
  double s = 0.0;
  for (int r = threadIdx.x; r < A.R; r += blockDim.x)
    s += double(A.stored[size_t(col) * A.ld + r]) + A.pend[size_t(m) * A.R + r];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) A.qbar[col] += s / double(A.R);
}

template <int NVB>
cudaError_t bwd_col_nv(int dt, long long T, cudaStream_t st, const BwdArgs& a) {
  switch (dt) {
    case 0: bwd_column_kernel<NVB, float><<<unsigned(T), kBwdThreads, 0, st>>>(a); break;
    case 1: bwd_column_kernel<NVB, __nv_bfloat16><<<unsigned(T), kBwdThreads, 0, st>>>(a); break;
    case 2: bwd_column_kernel<NVB, __half><<<unsigned(T), kBwdThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

int bwd_max_rows() { return 16 * kBwdThreads; }

cudaError_t launch_bwd_step(int cost_dtype, long long T, cudaStream_t st, const BwdArgs& a) {
  const int need = (a.R + kBwdThreads - 1) / kBwdThreads;
  cudaError_t e;
  if (need <= 1) e = bwd_col_nv<1>(cost_dtype, T, st, a);
  else if (need <= 2) e = bwd_col_nv<2>(cost_dtype, T, st, a);
  else if (need <= 4) e = bwd_col_nv<4>(cost_dtype, T, st, a);
  else if (need <= 8) e = bwd_col_nv<8>(cost_dtype, T, st, a);
  else if (need <= 16) e = bwd_col_nv<16>(cost_dtype, T, st, a);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  bwd_row_kernel<<<(a.R + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bwd_theta0(long long T, cudaStream_t st, const BwdArgs& a) {
  bwd_theta0_kernel<<<unsigned(T), kBwdThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mam
