// libmam: the free-support step of Algorithm 2 (Prop. 4).
//
// Algorithm 2 alternates MAM on a fixed support with a support step: given
// the plans pi, the support minimising
//   Psi(xi) = sum_m alpha_m sum_{r,s} ||xi_r - zeta_s||^2 pi_rs / 2
// is the weighted mean
//   xi_r = sum_m alpha_m sum_s zeta_s pi_rs / sum_m alpha_m sum_s pi_rs   (Prop. 4).
// The plans used are the pi-hat the next column step would compute from the
// current state (Step 1 and the projection of Step 2, Algorithm 1), found
// here without touching theta: one warp per column recomputes
// w = theta + 2 t d - c / rho from memory on every pass of an exact threshold
// search, then adds alpha_m zeta_s pi-hat_rs and alpha_m pi-hat_rs to per-row
// 64-bit fixed-point sums (integer atomics: the result does not depend on
// the order of the adds).  A second kernel forms the ratios.  This is a
// rare operation, kept apart from the per-iteration kernels.
#include "mam_device.cuh"
#include "mam_support.h"

#include <type_traits>

namespace mam {
namespace {

template <typename CT>
__device__ __forceinline__ float cost_at(const CT* c, int r) {
  if constexpr (std::is_same<CT, float>::value) return c[r];
  else if constexpr (std::is_same<CT, __half>::value) return __half2float(c[r]);
  else return __bfloat162float(c[r]);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per column (grid-stride).  The threshold search is the method of
// the column kernels: Newton (Michelot) steps from the column's last
// threshold, or from max w - q_s (a point at or below the threshold); it
// ends when two successive active sets have the same size, which makes the
// threshold exact.  A step that leaves no active row restarts from
// max w - q_s.
template <typename CT>
__global__ void __launch_bounds__(256) support_accumulate_kernel(const SupportArgs A) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  const int R = A.R, dim = A.dim;
  for (long long col = w0; col < A.T; col += nwarp) {
    const float tau = A.q[col];
    if (!(tau > 0.f)) continue;  // Delta(0) = {0}: no mass
    const int m = A.col_meas[col];
    const float irho = A.inv_rho[m];
    const float* th = A.theta + size_t(col) * A.ld;
    const CT* cc = A.gen_xi ? nullptr
                            : static_cast<const CT*>(A.cost) +
                                  size_t(A.cost_col ? (long long)A.cost_col[col] : col) * A.ld;
    const float4 zg = A.gen_xi ? A.gen_zeta[col] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float* dl = A.delta32 + size_t(m) * A.ld;
    auto w_at = [&](int r) {
      const float c = A.gen_xi ? gen_cost(A.gen_xi, A.ld, r, zg) : cost_at(cc, r);
      return fmaf(-c, irho, fmaf(2.f, __fmul_rn(A.t, dl[r]), th[r]));
    };
    float mx = -INFINITY;
    for (int r = lane; r < R; r += 32) mx = fmaxf(mx, w_at(r));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float lo = mx - tau;
    const float lp = A.lam[col];
    float lam = (lp == lp && lp > -INFINITY && lp < INFINITY) ? lp : lo;
    float nprev = -1.f;
    for (int it = 0; it < 256; ++it) {
      float f = 0.f, n = 0.f;
      for (int r = lane; r < R; r += 32) {
        const float x = w_at(r) - lam;
        if (x > 0.f) {
          f += x;
          n += 1.f;
        }
      }
      f = warp_sum_f(f);
      n = warp_sum_f(n);
      if (n == nprev) break;  // same active set twice: lam is the threshold
      if (n == 0.f) {         // at or above max w: restart below the threshold
        lam = lo;
        nprev = -1.f;
        continue;
      }
      nprev = n;
      lam = lam + (f - tau) / n;
    }
    const float lu = fmaxf(lam, A.lam_floor);  // capped columns: max(lambda, 0)
    const double al = A.alpha[m];
    const double* z = A.zeta + size_t(col) * dim;
    double zw[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < dim; ++k) zw[k] = al * z[k];
    for (int r = lane; r < R; r += 32) {
      const float x = w_at(r) - lu;
      if (x > 0.f) {
        unsigned long long* a = A.acc + size_t(r) * (dim + 1);
        for (int k = 0; k < dim; ++k)
          atomicAdd(a + k, (unsigned long long)__double2ll_rn(zw[k] * double(x) * A.fx));
        atomicAdd(a + dim, (unsigned long long)__double2ll_rn(al * double(x) * A.fx));
      }
    }
  }
}

// xi_r = (sum alpha zeta pi-hat) / (sum alpha pi-hat) for rows with mass; the
// fixed-point scale cancels in the ratio.  Clears the sums.
__global__ void support_finish_kernel(unsigned long long* acc, double* xi, int R, int dim) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  unsigned long long* a = acc + size_t(r) * (dim + 1);
  const long long den = (long long)a[dim];
  if (den > 0)
    for (int k = 0; k < dim; ++k) xi[size_t(r) * dim + k] = double((long long)a[k]) / double(den);
  for (int k = 0; k <= dim; ++k) a[k] = 0ull;
}

}  // namespace

cudaError_t launch_support_step(int cost_dtype, const SupportArgs& a, double* xi,
                                cudaStream_t st) {
  long long g = (a.T * 32 + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  switch (cost_dtype) {
    case 0: support_accumulate_kernel<float><<<int(g), 256, 0, st>>>(a); break;
    case 1: support_accumulate_kernel<__nv_bfloat16><<<int(g), 256, 0, st>>>(a); break;
    case 2: support_accumulate_kernel<__half><<<int(g), 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  support_finish_kernel<<<(a.R + 127) / 128, 128, 0, st>>>(a.acc, xi, a.R, a.dim);
  return cudaGetLastError();
}

}  // namespace mam
