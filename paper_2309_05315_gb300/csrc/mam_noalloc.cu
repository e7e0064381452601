// libmam: an entry point that performs no device allocation.
//
// mam_column_update_noalloc runs Step 2 of Algorithm 1 (projection of every
// column of one measure's plan onto Delta_R(q_s) and the theta update) and
// the Step 3 row sums on buffers the caller owns.  The row sums need a
// scratch accumulator; instead of allocating it, this file keeps it in a
// file-scope __device__ array of kNoAllocMaxR entries (96 KB), which every
// GPU that loads the library holds until the process exits.  The entry point
// is meant for callers that cannot call cudaMalloc: code running inside a
// framework that owns the device memory through its own pool (a raw
// cudaMalloc bypasses the pool and can fail once the pool has reserved the
// GPU), and latency-critical loops where cudaMalloc's implicit device-wide
// synchronisation is not acceptable.
#include "mam.h"
#include "mam_device.cuh"
#include "mam_handle.h"

#include <cmath>
#include <string>

namespace mam {

constexpr int kNoAllocMaxR = 12288;

// Fixed-point row sums of pi-hat (order-independent integer adds) in entries
// 0..kNoAllocMaxR-1, and one status word after them (0: ok; bit 0: a
// column's threshold search ended with an empty active set; bit 1: a row sum
// overflowed the accumulator because mass_bound was below the column masses).
// Shared by every call on this device: calls whose work overlaps on the GPU
// race.
constexpr int kNoAllocStatus = kNoAllocMaxR;
static __device__ __align__(256) unsigned long long g_noalloc_acc[kNoAllocMaxR + 1];

namespace {

constexpr int kNaThreads = 256;

__global__ void noalloc_clear(unsigned long long* acc, int R) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
    acc[r] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0) acc[kNoAllocStatus] = 0ull;
}

// One CTA per column; w lives in shared memory.  Cold start every call:
// bracket [max w - tau, max w), then Newton/Michelot steps from the lower
// end until two successive active sets agree (exact threshold).
__global__ void __launch_bounds__(kNaThreads)
    noalloc_column(float* theta, const float* cost, const float* q, const float* d,
                   int R, int ld, float rho, float fx, unsigned long long* acc) {
  extern __shared__ float w[];
  __shared__ float4 red[2 * kRedSlots];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nw = nt >> 5;
  const long long col = blockIdx.x;
  float* th = theta + col * ld;
  const float* c = cost + col * ld;
  const float tau = q[col];
  const float irho = 1.f / rho;
  float mx = -INFINITY;
  for (int r = tid; r < R; r += nt) {
    const float v = fmaf(-c[r], irho, fmaf(2.f, d[r], th[r]));
    w[r] = v;
    mx = fmaxf(mx, v);
  }
  int rb = 0;
  float lam = INFINITY;
  if (tau > 0.f) {
    float z0 = 0.f, z1 = 0.f;
    reduce3<false>(z0, z1, mx, red, rb, lane, warp, nw);
    lam = mx - tau;
    float nprev = -1.f;
    for (int it = 0; it < kMaxNewton; ++it) {
      float f = 0.f, n = 0.f, z = 0.f;
      for (int r = tid; r < R; r += nt) {
        const float x = w[r] - lam;
        f += fmaxf(x, 0.f);
        n += x > 0.f ? 1.f : 0.f;
      }
      reduce3<false>(f, n, z, red, rb, lane, warp, nw);
      if (n == 0.f) {
        // An empty active set: lambda rounded to or above max w, which
        // happens only when tau is below the FP32 resolution of w.  The
        // column would carry no mass, so the call reports a failure.
        if (tid == 0) atomicOr(acc + kNoAllocStatus, 1ull);
        break;
      }
      if (n == nprev) break;
      nprev = n;
      lam = lam + (f - tau) / n;
    }
  }
  for (int r = tid; r < R; r += nt) {
    const float pv = fmaxf(w[r] - lam, 0.f);
    th[r] = pv - d[r];
    if (pv > 0.f) atomicAdd(acc + r, (unsigned long long)__float2ll_rn(pv * fx));
  }
}

// rowsum_r = sum_s pihat_rs - S d_r (row sums of theta' = pihat - d).  One
// CTA: every pi-hat entry is >= 0, so a negative signed accumulator means the
// sum overflowed (mass_bound below the mass of the columns).  A failed column
// search or an overflow makes every output row NaN, so the caller sees the
// failure in the one result the call returns.
constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads)
    noalloc_finish(unsigned long long* acc, const float* d, int R, int S, double inv_fx,
                   double* out) {
  bool ovf = false;
  for (int r = threadIdx.x; r < R; r += blockDim.x) ovf |= (long long)acc[r] < 0;
  ovf = __syncthreads_or(ovf) != 0;
  if (ovf && threadIdx.x == 0) atomicOr(acc + kNoAllocStatus, 2ull);
  __syncthreads();
  const bool bad = *(volatile unsigned long long*)(acc + kNoAllocStatus) != 0ull;
  for (int r = threadIdx.x; r < R; r += blockDim.x)
    out[r] = bad ? __longlong_as_double(0x7ff8000000000000ll)
                 : double((long long)acc[r]) * inv_fx - double(S) * double(d[r]);
}

}  // namespace
}  // namespace mam

using namespace mam;

extern "C" mam_status mam_column_update_noalloc(float* theta, const float* cost,
                                                const float* q, const float* d,
                                                int32_t R, int32_t ld, int32_t S,
                                                double rho, double mass_bound,
                                                double* rowsum_out, void* stream) {
  if (!theta || !cost || !q || !d || !rowsum_out)
    return fail(nullptr, MAM_ERR_INVALID_ARG, "noalloc: null buffer");
  if (R < 1 || R > kNoAllocMaxR)
    return fail(nullptr, MAM_ERR_INVALID_ARG,
                "noalloc: R must be in 1.." + std::to_string(kNoAllocMaxR) +
                    " (the size of the static scratch accumulator)");
  if (ld < R || S < 1)
    return fail(nullptr, MAM_ERR_INVALID_ARG, "noalloc: need ld >= R and S >= 1");
  if (!(rho > 0) || !std::isfinite(rho) || !(mass_bound > 0) || !std::isfinite(mass_bound))
    return fail(nullptr, MAM_ERR_INVALID_ARG, "noalloc: rho and mass_bound must be finite and > 0");
  if (size_t(R) * sizeof(float) > 227 * 1024)
    return fail(nullptr, MAM_ERR_INVALID_ARG, "noalloc: column too long");
  // Set-up, on every call, with the caller's device current: the host-side
  // name of the array is not a device address, so ask the runtime for the
  // real one.  Both calls are host-side lookups; repeating them keeps the
  // address right if the device's context was reset and the module loaded
  // again.  The first call on a device also loads the module (lazy loading),
  // which is why that first call must come before any stream capture.
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_acc);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
  e = cudaFuncSetAttribute(noalloc_column, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(kNoAllocMaxR * sizeof(float)));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaFuncSetAttribute");
  unsigned long long* acc = static_cast<unsigned long long*>(p);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int e2 = 61 - int(std::ceil(std::log2(mass_bound * 1.0001)));
  const int ex = e2 < 0 ? 0 : (e2 > 100 ? 100 : e2);
  const double fx = std::ldexp(1.0, ex);
  const int gb = (R + 255) / 256;
  noalloc_clear<<<gb, 256, 0, st>>>(acc, R);
  noalloc_column<<<S, kNaThreads, size_t(R) * sizeof(float), st>>>(
      theta, cost, q, d, R, ld, float(rho), float(fx), acc);
  noalloc_finish<<<1, kFinThreads, 0, st>>>(acc, d, R, S, 1.0 / fx, rowsum_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "noalloc launch");
  return MAM_OK;
}
