// Device helpers shared by libmam's kernel translation units: PTX wrappers
// (mbarrier, bulk-async copies, global timer), cost-type loads, CTA and warp
// reductions, Remark 2 draws and t^k of Algorithm 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdint>

#include "mam_internal.h"

namespace mam {
namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait
constexpr int kMaxNewton = 64;  // bound on threshold-search passes / column

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// Orders this thread's view of earlier generic-proxy shared-memory accesses
// (made visible to it by a barrier) before its later async-proxy copies.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One bulk copy global -> shared (sizes and addresses multiples of 16 B);
// completion is reported as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src,
                                          uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar`, giving up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar,
                                                  uint32_t parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Programmatic dependent launch: wait until the preceding kernel in the
// stream has finished and its writes are visible / let the next kernel start
// its prologue.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------ cost types

template <typename CT>
struct CostIO;

template <>
struct CostIO<float> {
  static __device__ __forceinline__ float4 load4(const float* base, int idx) {
    return reinterpret_cast<const float4*>(base)[idx];
  }
};

template <>
struct CostIO<__nv_bfloat16> {
  // bf16 -> fp32 is exact: the bf16 pattern is the top half of the fp32 one.
  static __device__ __forceinline__ float4 load4(const __nv_bfloat16* base,
                                                 int idx) {
    const uint2 u = reinterpret_cast<const uint2*>(base)[idx];
    return make_float4(__uint_as_float(u.x << 16),
                       __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
  }
};

template <>
struct CostIO<__half> {
  static __device__ __forceinline__ float4 load4(const __half* base, int idx) {
    const uint2 u = reinterpret_cast<const uint2*>(base)[idx];
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
};

// ------------------------------------------------------------ reductions

// CTA-wide reduction of (sum a, sum b, min-or-max c).  The xor butterfly
// leaves identical values in every lane, and every thread then combines the
// per-warp values in the same order, so all threads obtain bit-identical
// results (the search below relies on that for uniform control flow).
// `red` is double-buffered ([2][32]); alternating buffers makes one
// __syncthreads per reduction sufficient.
template <bool kMin>
__device__ __forceinline__ void reduce3(float& a, float& b, float& c,
                                        float4* red, int& rb, int lane,
                                        int warp, int nw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    const float cc = __shfl_xor_sync(0xffffffffu, c, o);
    c = kMin ? fminf(c, cc) : fmaxf(c, cc);
  }
  if (nw == 1) return;
  if (lane == 0) red[rb * kRedSlots + warp] = make_float4(a, b, c, 0.f);
  __syncthreads();
  const float ident = kMin ? INFINITY : -INFINITY;
  float4 r = lane < nw ? red[rb * kRedSlots + lane] : make_float4(0.f, 0.f, ident, 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
    r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
    const float cc = __shfl_xor_sync(0xffffffffu, r.z, o);
    r.z = kMin ? fminf(r.z, cc) : fmaxf(r.z, cc);
  }
  a = r.x;
  b = r.y;
  c = r.z;
  rb ^= 1;
}

// Certificate for one warm Newton step l1 = l0 + dl from the threshold search:
// gap0 = min_r |fl(w_r - l0)|.  When gap0 exceeds |dl| by more than the
// rounding of w_r - l0 (at most 2^-24 |w_r - l0| relative) and of l0 + dl
// (at most 2^-24 (|l0| + |dl|)), every w_r lies on the same side of l1 as of
// l0, so the active set, and with it the exact threshold, is the one at l0's
// Newton point: l1.  A w_r equal to l0 gives gap0 = 0 and no certificate.
__device__ __forceinline__ bool newton_certified(float gap0, float dl, float l0) {
  const float adl = fabsf(dl);
  return gap0 * (1.f - 0x1p-20f) > adl + 0x1p-20f * (fabsf(l0) + adl);
}

template <int NV>
struct MaxThreads {
  static constexpr int value = NV == 1 ? 1024 : NV == 2 ? 768
                               : NV <= 4 ? 512 : NV <= 6 ? 192 : 384;
};
// Resident CTAs per SM the register allocation is sized for.  The 5- and
// 6-group shapes (columns of up to 3840 / 4608 rows) are held to 4 CTAs of
// 192 threads, the 8-group shape (up to 12288 rows) to 2 CTAs of 384: with
// the shift d in shared memory this spills at most a few bytes, and
// with a one-stage pipeline the extra resident columns hide the copies
// (R = 3600: 54 vs 56 us per step; R = 10000 unbalanced: 0.69 vs 0.82 ms).
template <int NV>
struct MinCtas {
  static constexpr int value = (NV == 5 || NV == 6) ? 4 : NV == 8 ? 2 : 1;
};

// ------------------------------------------------------------ helpers

// Conversions between FP32 and 64-bit integers with integer instructions
// only (the hardware conversions run on the FP64 pipe, a small fraction of
// the FP32 rate on this GPU).
// f32_to_i64_rn: round to nearest, ties to even, for finite |x| < 2^63.
__device__ __forceinline__ long long f32_to_i64_rn(float x) {
  const unsigned u = __float_as_uint(x);
  const int ex = int((u >> 23) & 0xffu);
  if (ex < 126) return 0;  // |x| < 0.5, zero and subnormals included
  const unsigned long long mant = (u & 0x7fffffu) | 0x800000u;
  const int sh = ex - 150;  // |x| = mant * 2^sh
  unsigned long long mag;
  if (sh >= 0) {
    mag = mant << sh;
  } else {
    const int r = -sh;  // 1..24
    const unsigned long long q = mant >> r;
    const unsigned long long rem = mant & ((1ull << r) - 1ull);
    const unsigned long long half = 1ull << (r - 1);
    mag = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  }
  return (u >> 31) ? -(long long)mag : (long long)mag;
}

// i64_to_f32: v = hi 2^32 + lo, each half converted, then one fused
// multiply-add (within about one unit in the last place).
__device__ __forceinline__ float i64_to_f32(long long v) {
  const int hi = int(v >> 32);
  const unsigned lo = unsigned(v & 0xffffffffll);
  return fmaf(float(hi), 4294967296.f, float(lo));
}

// Generated cost ||xi_r - zeta_s||^2 - eta in FP32: xi from coordinate
// planes [3][ld] (x, y, z), zeta as (x, y, z, eta); coordinates past dim are
// 0 in both.
__device__ __forceinline__ float gen_cost(const float* planes, int ld, int r, float4 zeta) {
  const float dx = planes[r] - zeta.x, dy = planes[ld + r] - zeta.y,
              dz = planes[2 * ld + r] - zeta.z;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx)) - zeta.w;
}

// floor(x * a / 2^62) for |x| < 2^63, 0 <= a <= 2^62 (exact): the product of
// a fixed-point marginal and an averaging weight a_m held as round(a_m 2^62).
__device__ __forceinline__ long long mul_q62(long long x, long long a) {
  const long long hi = __mul64hi(x, a);
  const unsigned long long lo = (unsigned long long)x * (unsigned long long)a;
  return (long long)(((unsigned long long)hi << 2) | (lo >> 62));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Index set of column step k (Remark 2): bundle i is drawn with probability
// beta_i from u_k = (SplitMix64(seed + (k+1) * 0x9E3779B97F4A7C15) >> 11)
// * 2^-53.  Deterministic MAM (nb <= 1) always uses index set 0.  Also called
// on the host (with a host copy of the cumulative probabilities) to count
// the work of each step.
__host__ __device__ __forceinline__ int draw_index_set(const Draw& d, long long k) {
  if (d.nb <= 1) return 0;
  unsigned long long z = d.seed + (unsigned long long)k * 0x9E3779B97F4A7C15ull;
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double u = double(z >> 11) * (1.0 / 9007199254740992.0);
  int i = 0;
  while (i < d.nb - 1 && !(u < d.cum[i])) ++i;
  return i;
}

// t^k of Algorithm 1 from the averaging kernel's block sums of
// sum_m ||p - p^(m)||^2 / S_m:  D = sqrt(sum), t = 1 if gamma = inf or
// rho D <= gamma, else gamma / (rho D).  Every CTA of the column kernel
// evaluates it with the same thread count and the same summation order, so
// all of them obtain the same t.  Uses dred[0..31]; all threads must call.
__device__ double t_from_blocks(const double* blk, int nblk, double rho,
                                double gamma, double* dred, int tid, int nt) {
  if (isinf(gamma)) return 1.0;  // balanced: t = 1 (uniform over the CTA)
  double acc = 0.0;
  for (int i = tid; i < nblk; i += nt) acc += blk[4 * i];
  acc = warp_sum_d(acc);
  if ((tid & 31) == 0) dred[tid >> 5] = acc;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (nt >> 5); ++w) tot += dred[w];
  __syncthreads();
  // sqrt and quotient in FP32 (the FP64 ones are long sequences on the slow
  // FP64 pipe); t carries about 1e-7 relative error, the same in every CTA.
  const float D = sqrtf(float(tot));
  const float rD = float(rho) * D;
  if (rD <= float(gamma)) return 1.0;
  return double(__fdiv_rn(float(gamma), rD));
}

// The shift delta_r = (p_r - p^(m)_r) / S_m in FP32 from the exact
// fixed-point difference (p - p^(m)) F and 1 / (S_m F) in FP64: one FP64
// product, then one rounding to FP32.  (Rounding 1 / (S_m F) to FP32 instead
// would give every row of measure m the same relative error in every
// iteration, a bias that the iterates accumulate.)
__device__ __forceinline__ float shift_f32(long long dfx, double inv_SFd) {
  return __double2float_rn(double(dfx) * inv_SFd);
}

// ------------------------------------------------------- packed FP32 pairs

// Blackwell executes two FP32 lanes per instruction for add/sub/fma on
// register pairs (PTX .f32x2).  Pairs are plain 64-bit registers here.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t pk(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float lo(f2_t r) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
  return a;
}
__device__ __forceinline__ float hi(f2_t r) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
  return b;
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
  f2_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
  f2_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
  f2_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// (max(x.lo, 0), max(x.hi, 0)) and the number of positive lanes.
__device__ __forceinline__ f2_t relu2(f2_t x, float& cnt) {
  const float a = lo(x), b = hi(x);
  cnt += (a > 0.f ? 1.f : 0.f) + (b > 0.f ? 1.f : 0.f);
  return pk(fmaxf(a, 0.f), fmaxf(b, 0.f));
}


// Launch `kernel` with programmatic stream serialization (see pdl_wait).
template <typename... Args>
cudaError_t launch_pdl(void (*kernel)(Args...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace
}  // namespace mam
