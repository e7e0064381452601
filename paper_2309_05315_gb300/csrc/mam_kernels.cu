// libmam device code: the per-iteration kernels of the Method of Averaged
// Marginals (arXiv 2309.05315, Algorithm 1) for sm_103a.
//
//   column_kernel   Step 2 of Algorithm 1 for every column of the index set
//                   M^k, fused with the partial row sums of Step 3 and with
//                   the diagnostics (W-hat, lower bound, fixed-point residual).
//   average_kernel  Step 3 reduction of those partials (deterministic, FP64),
//                   Step 1 (p = sum_m a_m p^(m), eq. pr) and the factor t^k.
//
// Plans theta and costs c are stored column-contiguous with a padded stride
// ld (a multiple of 8 elements), so that one column is one contiguous run of
// 4*ld (theta) and ld*sizeof(cost) bytes: each column is brought into shared
// memory by two bulk-async copies (cp.async.bulk, completion on an mbarrier)
// while the CTA works on the previous column.
#include "mam_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cfloat>
#include <cmath>
#include <type_traits>

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
  if (lane == 0) red[rb * kRedSlots + warp] = make_float4(a, b, c, 0.f);
  __syncthreads();
  float4 r = red[rb * kRedSlots];
  for (int i = 1; i < nw; ++i) {
    const float4 x = red[rb * kRedSlots + i];
    r.x += x.x;
    r.y += x.y;
    r.z = kMin ? fminf(r.z, x.z) : fmaxf(r.z, x.z);
  }
  a = r.x;
  b = r.y;
  c = r.z;
  rb ^= 1;
}

template <int NV>
struct MaxThreads {
  static constexpr int value = NV == 1 ? 1024 : NV == 2 ? 768
                               : NV <= 6 ? 512 : 384;
};

// ------------------------------------------------------- column kernel

// Step 2 of Algorithm 1 for one CTA's slice of the index set, one column at
// a time.  Thread `tid` owns the float4 groups idx = v*nt + tid (v < NV) of
// every column, i.e. rows r = 4*idx .. 4*idx+3; its shift d^(m)_r and its
// partial row sums stay in registers for all columns of a measure.
//
// Per column s of measure m (tau = q_s):
//   w_r     = theta_rs + 2 d_r - c_rs / rho        (Alg. 1, w)
//   lambda  : sum_r max(w_r - lambda, 0) = tau     (Prop. 3, Remark 1)
//   pihat_r = max(w_r - lambda, 0)                 (Alg. 1, projection)
//   theta'  = pihat_r - d_r                        (Alg. 1, update)
// with d_r = t^k (p_r - p^(m)_r) / S_m.
//
// Threshold search (exact).  f(l) = sum_r max(w_r - l, 0) is convex,
// piecewise linear and decreasing; n(l) = #{w_r > l} = -f'(l).  The Newton
// step l <- l + (f(l) - tau) / n(l) equals Michelot's update
// (sum_{w>l} w - tau) / n(l): from any l > lambda* it lands in
// [lambda_prev_set, lambda*], and from below it increases monotonically.  The
// active sets {w > l} of two successive iterates are nested, so equal counts
// mean equal sets, and then the iterate is exactly lambda*.  The search
// starts from the column's previous threshold (warm start); without one it
// brackets lambda* in [max w - tau, max w), bisects bisect_depth times and
// continues from the lower end.
template <int NV, typename CT, bool DIAG>
__global__ void __launch_bounds__(MaxThreads<NV>::value)
    column_kernel(const ColArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nw = nt >> 5;
  const int ld = A.ld;
  const int R = A.R;
  const int ld4 = ld >> 2;
  const int stages = A.stages;

  float* th_s = reinterpret_cast<float*>(smem);
  CT* c_s = reinterpret_cast<CT*>(smem + size_t(stages) * ld * sizeof(float));
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      smem + size_t(stages) * ld * (sizeof(float) + sizeof(CT)));
  float4* red = reinterpret_cast<float4*>(bar + 4);

  const int bundle = A.bundle_cur ? *A.bundle_cur : 0;
  const Sched sc = A.sched[bundle];
  const int sb = sc.cta_seg_begin[blockIdx.x];
  const int se = sc.cta_seg_begin[blockIdx.x + 1];
  if (sb >= se) return;  // uniform over the CTA
  int4 sg = sc.segs[sb];
  const long long col0 = sg.y;
  const long long ncol = (long long)sc.segs[se - 1].z - col0;

  const uint32_t bytes_th = uint32_t(ld) * sizeof(float);
  const uint32_t bytes_c = uint32_t(ld) * sizeof(CT);
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  long long issued = 0;  // meaningful in thread 0 only
  auto issue = [&](long long j) {
    const int s = int(j % stages);
    const long long col = col0 + j;
    mbar_expect_tx(&bar[s], bytes_th + bytes_c);
    bulk_load(th_s + size_t(s) * ld, A.theta + size_t(col) * ld, bytes_th,
              &bar[s]);
    bulk_load(c_s + size_t(s) * ld,
              static_cast<const CT*>(A.cost) + size_t(col) * ld, bytes_c,
              &bar[s]);
  };
  if (tid == 0) {
    const long long n0 = ncol < stages ? ncol : stages;
    for (long long j = 0; j < n0; ++j) issue(j);
    issued = n0;
  }

  float d[NV][4];
  float part[NV][4];
  float rho_m = 0.f, irho_m = 0.f;
  auto setup = [&](int m) {
    const double tt = A.t[A.meas_prob[m]];
    rho_m = A.rho[m];
    irho_m = A.inv_rho[m];
    const double* dl = A.delta + size_t(m) * R;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int idx = v * nt + tid;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 4 * idx + e;
        d[v][e] = (idx < ld4 && r < R) ? float(tt * dl[r]) : 0.f;
        part[v][e] = 0.f;
      }
    }
  };
  auto flush = [&](int slot) {
    float4* dst = reinterpret_cast<float4*>(A.partials + size_t(slot) * ld);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int idx = v * nt + tid;
      if (idx < ld4)
        dst[idx] = make_float4(part[v][0], part[v][1], part[v][2], part[v][3]);
    }
  };
  setup(sg.x);

  int rb = 0;
  unsigned long long my_passes = 0;
  bool failed = false;
  bool any_fail = false;
  int seg = sb;
  for (long long j = 0; j < ncol; ++j) {
    const long long col = col0 + j;
    if (col >= sg.z) {  // next measure inside this CTA's slice
      flush(sg.w);
      ++seg;
      sg = sc.segs[seg];
      setup(sg.x);
    }
    const int s = int(j % stages);
    if (!mbar_wait_bounded(&bar[s], uint32_t((j / stages) & 1), kWaitLimitNs))
      failed = true;  // keep control flow uniform; checked below

    const float tau = A.q[col];
    float lam = A.lam[col];
    const float* ths = th_s + size_t(s) * ld;
    const CT* cs = c_s + size_t(s) * ld;

    float w[NV][4];
    float lbmin = INFINITY;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int idx = v * nt + tid;
      if (idx < ld4) {
        const float4 th = reinterpret_cast<const float4*>(ths)[idx];
        const float4 c = CostIO<CT>::load4(cs, idx);
        const float thv[4] = {th.x, th.y, th.z, th.w};
        const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool ok = 4 * idx + e < R;
          w[v][e] = ok ? (thv[e] + 2.f * d[v][e]) - cv[e] * irho_m : -INFINITY;
          if (DIAG && ok) lbmin = fminf(lbmin, cv[e] - rho_m * d[v][e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) w[v][e] = -INFINITY;
      }
    }

    int np = 0;
    if (!(tau > 0.f)) {
      lam = INFINITY;  // Remark 1: the projection onto Delta_R(0) is 0
    } else {
      float nprev = -1.f;
      bool need_max = true;
      if (!(lam == lam)) {  // no previous threshold: bracket and bisect
        float mx = -INFINITY;
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int e = 0; e < 4; ++e) mx = fmaxf(mx, w[v][e]);
        float z0 = 0.f, z1 = 0.f;
        reduce3<false>(z0, z1, mx, red, rb, lane, warp, nw);
        ++np;
        float lo = mx - tau, hi = mx;
        for (int b = 0; b < A.bisect_depth; ++b) {
          const float mid = 0.5f * (lo + hi);
          float f = 0.f, n = 0.f, z = 0.f;
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int e = 0; e < 4; ++e) f += fmaxf(w[v][e] - mid, 0.f);
          reduce3<false>(f, n, z, red, rb, lane, warp, nw);
          ++np;
          if (f >= tau) lo = mid; else hi = mid;
        }
        lam = lo;
        need_max = false;
      }
      for (int it = 0; it < kMaxNewton; ++it) {
        float f = 0.f, n = 0.f, mx = -INFINITY;
        if (need_max) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x = w[v][e] - lam;
              f += fmaxf(x, 0.f);
              n += x > 0.f ? 1.f : 0.f;
              mx = fmaxf(mx, w[v][e]);
            }
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x = w[v][e] - lam;
              f += fmaxf(x, 0.f);
              n += x > 0.f ? 1.f : 0.f;
            }
        }
        reduce3<false>(f, n, mx, red, rb, lane, warp, nw);
        ++np;
        if (n == nprev) {  // same active set twice: lam is the threshold
          lam = lam + (f - tau) / n;
          break;
        }
        if (n == 0.f) {  // warm start above max w: restart from below
          lam = mx - tau;
          nprev = -1.f;
          need_max = false;
          continue;
        }
        lam = lam + (f - tau) / n;
        nprev = n;
        need_max = false;
      }
    }

    // Projection, theta update, partial row sums (+ diagnostics).
    float wc = 0.f, res = 0.f;
    float4* gth = reinterpret_cast<float4*>(A.theta + size_t(col) * ld);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int idx = v * nt + tid;
      if (idx < ld4) {
        float o[4];
        float pv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          pv[e] = fmaxf(w[v][e] - lam, 0.f);
          o[e] = pv[e] - d[v][e];
          part[v][e] += o[e];
        }
        if (DIAG) {
          const float4 th = reinterpret_cast<const float4*>(ths)[idx];
          const float4 c = CostIO<CT>::load4(cs, idx);
          const float thv[4] = {th.x, th.y, th.z, th.w};
          const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (4 * idx + e < R) {
              wc += cv[e] * pv[e];
              const float dd = o[e] - thv[e];
              res += dd * dd;
            }
          }
        }
        gth[idx] = make_float4(o[0], o[1], o[2], o[3]);
      }
    }
    if (DIAG) {
      reduce3<true>(wc, res, lbmin, red, rb, lane, warp, nw);
      if (tid == 0) {
        A.diag_wc[col] = wc;
        A.diag_res[col] = res;
        A.diag_lb[col] = tau * lbmin;
      }
    }
    if (tid == 0) A.lam[col] = lam;
    my_passes += np;

    any_fail = __syncthreads_or(failed) != 0;  // stage s is free after this
    if (any_fail) break;
    if (tid == 0 && j + stages < ncol) {
      issue(j + stages);
      ++issued;
    }
  }
  if (!any_fail) {
    flush(sg.w);
  } else if (tid == 0) {
    atomicCAS(A.err, 0, 1);
    // Drain the copies still in flight (bounded) before leaving.
    for (long long j = 0; j < issued; ++j)
      mbar_wait_bounded(&bar[j % stages], uint32_t((j / stages) & 1),
                        kWaitLimitNs / 20);
  }
  if (tid == 0) atomicAdd(A.passes, my_passes);
}

// ------------------------------------------------------ average kernel

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Step 3 (reduction of the partial row sums into p^(m), FP64, fixed order),
// Step 1 (p = sum_m a_m p^(m)) and the factor t^k of Algorithm 1:
//   D = sqrt(sum_m ||p - p^(m)||^2 / S_m) = dist_L(theta)   (text after Alg. 1)
//   t = 1 if gamma = inf or rho D <= gamma, else gamma / (rho D).
// Grid (ceil(R/256), P).  The last block of each problem to finish combines
// the block sums (arrival counter, fixed order) and publishes t, the
// statistics and, for Remark 2, the next bundle.
__global__ void __launch_bounds__(256) average_kernel(const AvgArgs A) {
  __shared__ double sred[8][4];
  __shared__ bool is_last;
  const int pr = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int m0 = A.prob_meas[pr], m1 = A.prob_meas[pr + 1];
  const double t_old = A.t[pr];
  const int bundle = A.bundle_cur ? *A.bundle_cur : 0;
  const Sched sc = A.sched[bundle];
  double e = 0.0, eh = 0.0, dp2 = 0.0;
  if (r < A.R) {
    double p_new = 0.0;
    for (int m = m0; m < m1; ++m) {
      const size_t o = size_t(m) * A.R + r;
      if (A.reduce) {
        const int s0 = sc.slot_begin[m], s1 = sc.slot_end[m];
        if (s1 > s0) {
          double acc = 0.0;
          for (int s = s0; s < s1; ++s) acc += double(A.partials[size_t(s) * A.ld + r]);
          if (A.diag) A.phat[o] = acc + double(A.S[m]) * t_old * A.delta[o];
          A.pm[o] = acc;
        }
      }
      p_new += A.a[m] * A.pm[o];
    }
    double ph = 0.0;
    for (int m = m0; m < m1; ++m) {
      const size_t o = size_t(m) * A.R + r;
      const double df = p_new - A.pm[o];
      const double sm = double(A.S[m]);
      e += df * df / sm;
      A.delta[o] = df / sm;
      if (A.diag) ph += A.a[m] * A.phat[o];
    }
    if (A.diag) {
      for (int m = m0; m < m1; ++m) {
        const double df = ph - A.phat[size_t(m) * A.R + r];
        eh += df * df / double(A.S[m]);
      }
    }
    double* pp = A.p + size_t(pr) * A.R + r;
    const double dd = p_new - *pp;
    dp2 = dd * dd;
    *pp = p_new;
  }
  e = warp_sum_d(e);
  eh = warp_sum_d(eh);
  dp2 = warp_sum_d(dp2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sred[warp][0] = e;
    sred[warp][1] = eh;
    sred[warp][2] = dp2;
  }
  __syncthreads();
  const int nblk = gridDim.x;
  if (threadIdx.x == 0) {
    double b0 = 0, b1 = 0, b2 = 0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) {
      b0 += sred[i][0];
      b1 += sred[i][1];
      b2 += sred[i][2];
    }
    double* blk = A.blk + (size_t(pr) * nblk + blockIdx.x) * 4;
    blk[0] = b0;
    blk[1] = b1;
    blk[2] = b2;
    __threadfence();
    const unsigned prev = atomicAdd(A.counter + pr, 1u);
    is_last = (prev == unsigned(nblk - 1));
  }
  __syncthreads();
  if (!is_last || threadIdx.x != 0) return;
  __threadfence();
  double s0 = 0, s1 = 0, s2 = 0;
  for (int i = 0; i < nblk; ++i) {
    const volatile double* blk = A.blk + (size_t(pr) * nblk + i) * 4;
    s0 += blk[0];
    s1 += blk[1];
    s2 += blk[2];
  }
  const double D = sqrt(s0);
  const double rho = A.rho[pr], gamma = A.gamma[pr];
  double t_new = 1.0;
  if (!isinf(gamma) && !(rho * D <= gamma)) t_new = gamma / (rho * D);
  double* st = A.stat + size_t(pr) * 4;
  st[0] = D;
  if (A.diag) st[1] = sqrt(s1);
  st[2] = sqrt(s2);
  st[3] = t_old;
  A.t[pr] = t_new;
  A.counter[pr] = 0u;
  if (pr == 0 && A.iter) {
    if (A.bundle_prev) *A.bundle_prev = bundle;
    long long k = *A.iter;
    if (A.reduce) k += 1;
    *A.iter = k;
    if (A.nb > 1) {
      // Remark 2 draw for column step k (counter-based SplitMix64).
      unsigned long long z = A.seed + (unsigned long long)k * 0x9E3779B97F4A7C15ull;
      z += 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double u = double(z >> 11) * (1.0 / 9007199254740992.0);
      int i = 0;
      while (i < A.nb - 1 && !(u < A.bundle_cum[i])) ++i;
      *A.bundle_next = i;
    }
  }
}

// --------------------------------------------------------- other kernels

// c_rs = alpha_m * ||xi_r - zeta_s||^2 (eq. HugeLP) or alpha_m * C_rs,
// computed in FP64 without contraction, rounded to FP32, then to the storage
// type (round to nearest even).  Padding rows get 0.  zeta and gen hold the
// columns col0 .. col0+ncols-1 only.
template <typename CT>
__device__ __forceinline__ CT to_cost(float x);
template <>
__device__ __forceinline__ float to_cost<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_cost<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half to_cost<__half>(float x) {
  return __float2half_rn(x);
}

template <typename CT>
__global__ void build_cost_kernel(CT* cost, const double* xi,
                                  const double* zeta, const double* gen,
                                  const int* col_meas, const double* alpha,
                                  long long col0, long long ncols, int R,
                                  int ld, int dim) {
  const long long n = ncols * ld;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long jc = i / ld;
    const int r = int(i - jc * ld);
    const long long col = col0 + jc;
    double c = 0.0;
    if (r < R) {
      const double al = alpha[col_meas[col]];
      if (gen) {
        c = __dmul_rn(al, gen[jc * R + r]);
      } else {
        double acc = 0.0;
        for (int k = 0; k < dim; ++k) {
          const double df = __dadd_rn(zeta[jc * dim + k], -xi[size_t(r) * dim + k]);
          acc = __dadd_rn(acc, __dmul_rn(df, df));
        }
        c = __dmul_rn(al, acc);
      }
    }
    cost[size_t(col) * ld + r] = to_cost<CT>(__double2float_rn(c));
  }
}

// theta^0 (Alg. 1 Step 0; "Initialization" leaves it arbitrary):
// mode 0: theta_rs = q_s / R, mode 1: 0.  Padding rows are 0 and every
// threshold starts unknown (NaN).
__global__ void init_theta_kernel(float* theta, float* lam, const double* q,
                                  long long T, int R, int ld, int mode) {
  const long long n = T * ld;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long col = i / ld;
    const int r = int(i - col * ld);
    float v = 0.f;
    if (mode == 0 && r < R) v = float(q[col] / double(R));
    theta[i] = v;
    if (r == 0) lam[col] = __int_as_float(0x7fc00000);
  }
}

// p^(m)_r = sum_s theta^(m)_rs in FP64 (Alg. 1 Step 0 and checkpoint restore).
__global__ void rowsum_kernel(const float* theta, const long long* col_off,
                              int R, int ld, double* pm) {
  const int m = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double acc = 0.0;
  for (long long c = col_off[m]; c < col_off[m + 1]; ++c)
    acc += double(theta[size_t(c) * ld + r]);
  pm[size_t(m) * R + r] = acc;
}

// Sums of the per-column diagnostics of problem blockIdx.x, FP64, fixed
// order: out[3*i] = sum wc, out[3*i+1] = sum lb, out[3*i+2] = sum res over
// the columns of the last index set.
__global__ void __launch_bounds__(256) diag_reduce_kernel(
    const float* wc, const float* lb, const float* res,
    const long long* prob_cols, const Sched* sched, const int* bundle_prev,
    double* out) {
  __shared__ double sh[8][3];
  const int i = blockIdx.x;
  const long long c0 = prob_cols[i], c1 = prob_cols[i + 1];
  long long r0 = c0, r1 = c1;
  if (bundle_prev) {
    const Sched sc = sched[*bundle_prev];
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
    const CT* cost, const float* q, const double* delta, const double* t,
    const int* meas_prob, const float* rho, const int* col_meas, long long T,
    int R, int ld, float* diag_lb) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long col = w0; col < T; col += nwarp) {
    const int m = col_meas[col];
    const float tt = float(t[meas_prob[m]]);
    const float rh = rho[m];
    const double* dl = delta + size_t(m) * R;
    const CT* cc = cost + size_t(col) * ld;
    float mn = INFINITY;
    for (int r = lane; r < R; r += 32) {
      float c;
      if constexpr (sizeof(CT) == 4) c = float(cc[r]);
      else if constexpr (std::is_same<CT, __half>::value) c = __half2float(cc[r]);
      else c = __bfloat162float(cc[r]);
      mn = fminf(mn, c - rh * (tt * float(dl[r])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if (lane == 0) diag_lb[col] = q[col] * mn;
  }
}

template <int NV, typename CT, bool DIAG>
cudaError_t launch_col_t(int grid, int threads, size_t smem, cudaStream_t st,
                         const ColArgs& a) {
  column_kernel<NV, CT, DIAG><<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int NV, typename CT, bool DIAG>
cudaError_t smem_col_t(size_t smem) {
  return cudaFuncSetAttribute(column_kernel<NV, CT, DIAG>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(smem));
}

template <int NV, typename CT, bool DIAG>
cudaError_t occ_col_t(int threads, size_t smem, int* n) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      n, column_kernel<NV, CT, DIAG>, threads, smem);
}

// Dispatch over the compile-time (NV, cost type, DIAG) variants.
#define MAM_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(8)

template <int NV, typename CT>
cudaError_t col_op(int op, bool diag, int grid, int threads, size_t smem,
                   cudaStream_t st, const ColArgs* a, int* occ) {
  if (op == 0)
    return diag ? launch_col_t<NV, CT, true>(grid, threads, smem, st, *a)
                : launch_col_t<NV, CT, false>(grid, threads, smem, st, *a);
  if (op == 1)
    return diag ? smem_col_t<NV, CT, true>(smem) : smem_col_t<NV, CT, false>(smem);
  return diag ? occ_col_t<NV, CT, true>(threads, smem, occ)
              : occ_col_t<NV, CT, false>(threads, smem, occ);
}

template <typename CT>
cudaError_t col_op_nv(int nv, int op, bool diag, int grid, int threads,
                      size_t smem, cudaStream_t st, const ColArgs* a, int* occ) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return col_op<N, CT>(op, diag, grid, threads, smem, st, a, occ);
    MAM_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t col_op_any(int nv, int dt, int op, bool diag, int grid,
                       int threads, size_t smem, cudaStream_t st,
                       const ColArgs* a, int* occ) {
  switch (dt) {
    case 0: return col_op_nv<float>(nv, op, diag, grid, threads, smem, st, a, occ);
    case 1: return col_op_nv<__nv_bfloat16>(nv, op, diag, grid, threads, smem, st, a, occ);
    case 2: return col_op_nv<__half>(nv, op, diag, grid, threads, smem, st, a, occ);
    default: return cudaErrorInvalidValue;
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
  return col_op_any(nv, cost_dtype, 0, diag, grid, threads, smem, st, &a, nullptr);
}

cudaError_t set_column_smem(int nv, int cost_dtype, bool diag, size_t smem) {
  return col_op_any(nv, cost_dtype, 1, diag, 0, 0, smem, nullptr, nullptr, nullptr);
}

cudaError_t column_occupancy(int nv, int cost_dtype, bool diag, int threads,
                             size_t smem, int* blocks_per_sm) {
  return col_op_any(nv, cost_dtype, 2, diag, 0, threads, smem, nullptr, nullptr,
                    blocks_per_sm);
}

cudaError_t launch_average(const AvgArgs& a, int nblk, cudaStream_t st) {
  average_kernel<<<dim3(nblk, a.P), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_build_cost(int cost_dtype, void* cost, const double* xi,
                              const double* zeta, const double* gen_cost,
                              const int* col_meas, const double* alpha,
                              long long col0, long long ncols, int R, int ld,
                              int dim, cudaStream_t st) {
  const long long n = ncols * ld;
  long long g = (n + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  switch (cost_dtype) {
    case 0:
      build_cost_kernel<float><<<int(g), 256, 0, st>>>(
          static_cast<float*>(cost), xi, zeta, gen_cost, col_meas, alpha, col0,
          ncols, R, ld, dim);
      break;
    case 1:
      build_cost_kernel<__nv_bfloat16><<<int(g), 256, 0, st>>>(
          static_cast<__nv_bfloat16*>(cost), xi, zeta, gen_cost, col_meas,
          alpha, col0, ncols, R, ld, dim);
      break;
    case 2:
      build_cost_kernel<__half><<<int(g), 256, 0, st>>>(
          static_cast<__half*>(cost), xi, zeta, gen_cost, col_meas, alpha, col0,
          ncols, R, ld, dim);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_init_theta(float* theta, float* lam, const double* q,
                              long long T, int R, int ld, int mode,
                              cudaStream_t st) {
  const long long n = T * ld;
  long long g = (n + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  init_theta_kernel<<<int(g), 256, 0, st>>>(theta, lam, q, T, R, ld, mode);
  return cudaGetLastError();
}

cudaError_t launch_rowsum(const float* theta, const long long* col_off,
                          int Mtot, int R, int ld, double* pm,
                          cudaStream_t st) {
  rowsum_kernel<<<dim3((R + 127) / 128, Mtot), 128, 0, st>>>(theta, col_off, R,
                                                             ld, pm);
  return cudaGetLastError();
}

cudaError_t launch_lb(int cost_dtype, const void* cost, const float* q,
                      const double* delta, const double* t,
                      const int* meas_prob, const float* rho,
                      const int* col_meas, long long T, int R, int ld,
                      float* diag_lb, cudaStream_t st) {
  long long g = (T * 32 + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  switch (cost_dtype) {
    case 0:
      lb_kernel<float><<<int(g), 256, 0, st>>>(static_cast<const float*>(cost), q, delta, t, meas_prob, rho, col_meas, T, R, ld, diag_lb);
      break;
    case 1:
      lb_kernel<__nv_bfloat16><<<int(g), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(cost), q, delta, t, meas_prob, rho, col_meas, T, R, ld, diag_lb);
      break;
    case 2:
      lb_kernel<__half><<<int(g), 256, 0, st>>>(static_cast<const __half*>(cost), q, delta, t, meas_prob, rho, col_meas, T, R, ld, diag_lb);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_diag_reduce(const float* wc, const float* lb,
                               const float* res, const long long* prob_cols,
                               const Sched* sched, const int* bundle_prev,
                               int P, double* out, cudaStream_t st) {
  diag_reduce_kernel<<<P, 256, 0, st>>>(wc, lb, res, prob_cols, sched,
                                        bundle_prev, out);
  return cudaGetLastError();
}

}  // namespace mam
