// libmam: the column step with one warp per plan column (R up to 32*4*32).
//
// Same mathematics as column_kernel in mam_kernels.cu (Algorithm 1, Step 2,
// with the Step 3 row sums and the diagnostics), organised for columns short
// enough to live in one warp's registers: lane l holds the float4 groups
// g = v*32 + l (v < NV) of the column, the threshold search reduces with warp
// shuffles only (no CTA barrier per column), and the shift d^(m) sits once in
// shared memory for all warps of the CTA, which work on the columns of one
// measure at a time.  Columns are read straight from global memory into
// registers (streaming loads), the new plan column is written back with
// streaming stores.
#include "mam_device.cuh"

namespace mam {
namespace {

constexpr int kWarpThreads = 128;  // CTA size of the warp kernel

// Registers per thread allowed by the occupancy target of each width.
template <int NV>
struct WarpMinBlocks {
  static constexpr int value = NV >= 24 ? 3 : NV >= 13 ? 4 : NV >= 8 ? 6 : 8;
};

__device__ __forceinline__ void warp_sum2(float& a, float& b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

__device__ __forceinline__ float warp_max(float a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
  return a;
}

__device__ __forceinline__ float warp_min(float a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
  return a;
}

template <typename CT>
__device__ __forceinline__ float4 load_cost_global(const CT* base, int g);
template <>
__device__ __forceinline__ float4 load_cost_global<float>(const float* base, int g) {
  return __ldcs(reinterpret_cast<const float4*>(base) + g);
}
template <>
__device__ __forceinline__ float4 load_cost_global<__nv_bfloat16>(const __nv_bfloat16* base,
                                                                  int g) {
  const uint2 u = __ldcs(reinterpret_cast<const uint2*>(base) + g);
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
template <>
__device__ __forceinline__ float4 load_cost_global<__half>(const __half* base, int g) {
  const uint2 u = __ldcs(reinterpret_cast<const uint2*>(base) + g);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

// Sum of max(w - l, 0) and #{w > l} over this lane's rows (independent
// accumulators per group keep the dependency chains short).
template <int NV>
__device__ __forceinline__ void lane_fn(const float (&w)[NV][4], float l, float& f,
                                        float& n) {
  float fs[4] = {0.f, 0.f, 0.f, 0.f}, ns[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x = w[v][e] - l;
      fs[e] += fmaxf(x, 0.f);
      ns[e] += x > 0.f ? 1.f : 0.f;
    }
  f = (fs[0] + fs[1]) + (fs[2] + fs[3]);
  n = (ns[0] + ns[1]) + (ns[2] + ns[3]);
}

// One plan column by one warp: Step 2 of Algorithm 1 (see column_kernel for
// the threshold search), Step 3 fixed-point row sums, diagnostics.  Returns
// the number of search passes.
template <int NV, typename CT, bool DIAG>
__device__ __forceinline__ int warp_column(const ColArgs& A, long long col,
                                           const float* d_s, float irho,
                                           float rho_m,
                                           unsigned long long* acc_m, int lane) {
  const int ld4 = A.ld >> 2;
  const float tau = A.q[col];
  const float lam_prev = A.lam[col];
  const float4* thg = reinterpret_cast<const float4*>(A.theta + size_t(col) * A.ld);
  const CT* cg = static_cast<const CT*>(A.cost) + size_t(col) * A.ld;
  const float4* d4 = reinterpret_cast<const float4*>(d_s);

  // w = theta + 2 d - c / rho; rows past the column read as theta = 0,
  // c = +inf, d = 0, i.e. w = -inf.
  float w[NV][4];
  float lbmin = INFINITY;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int g = v * 32 + lane;
    float4 th = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 c = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    if (g < ld4) {
      th = __ldcs(thg + g);
      c = load_cost_global<CT>(cg, g);
    }
    const float4 d = d4[g];
    w[v][0] = fmaf(-c.x, irho, fmaf(2.f, d.x, th.x));
    w[v][1] = fmaf(-c.y, irho, fmaf(2.f, d.y, th.y));
    w[v][2] = fmaf(-c.z, irho, fmaf(2.f, d.z, th.z));
    w[v][3] = fmaf(-c.w, irho, fmaf(2.f, d.w, th.w));
    if (DIAG)
      lbmin = fminf(fminf(fminf(lbmin, c.x - rho_m * d.x), fminf(c.y - rho_m * d.y, c.z - rho_m * d.z)),
                    c.w - rho_m * d.w);
  }

  int np = 0;
  float lam_fin = INFINITY;
  if (tau > 0.f) {
    const bool warm = lam_prev == lam_prev;
    float lam = warm ? lam_prev : 0.f;
    float nprev = -1.f;
    bool bracket = !warm;
    for (int it = 0; it < kMaxNewton; ++it) {
      if (bracket) {  // lambda* lies in [max w - tau, max w)
        float mx = -INFINITY;
#pragma unroll
        for (int v = 0; v < NV; ++v)
          mx = fmaxf(mx, fmaxf(fmaxf(w[v][0], w[v][1]), fmaxf(w[v][2], w[v][3])));
        mx = warp_max(mx);
        ++np;
        float lo_b = mx - tau, hi_b = mx;
        for (int b = 0; b < A.bisect_depth; ++b) {
          const float mid = 0.5f * (lo_b + hi_b);
          float f, n;
          lane_fn<NV>(w, mid, f, n);
          warp_sum2(f, n);
          ++np;
          if (f >= tau) lo_b = mid; else hi_b = mid;
        }
        lam = lo_b;
        nprev = -1.f;
        bracket = false;
      }
      float f, n;
      lane_fn<NV>(w, lam, f, n);
      warp_sum2(f, n);
      ++np;
      if (n == nprev) {  // same active set twice: lam is the threshold
        lam_fin = lam;
        break;
      }
      if (n == 0.f) {  // at or above max w: restart from the bracket
        bracket = true;
        continue;
      }
      nprev = n;
      lam = lam + (f - tau) / n;
      lam_fin = lam;  // used if the pass budget runs out (not expected)
    }
  }

  // Commit: theta' = pihat - d (streaming stores), Step 3 row sums.
  float4* tho = reinterpret_cast<float4*>(A.theta + size_t(col) * A.ld);
  float wc = 0.f, res = 0.f;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int g = v * 32 + lane;
    const float4 d = d4[g];
    const float pv[4] = {fmaxf(w[v][0] - lam_fin, 0.f), fmaxf(w[v][1] - lam_fin, 0.f),
                         fmaxf(w[v][2] - lam_fin, 0.f), fmaxf(w[v][3] - lam_fin, 0.f)};
    const float4 o = make_float4(pv[0] - d.x, pv[1] - d.y, pv[2] - d.z, pv[3] - d.w);
    const bool act = fmaxf(fmaxf(pv[0], pv[1]), fmaxf(pv[2], pv[3])) > 0.f;
    if (__any_sync(0xffffffffu, act) && act) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (pv[e] > 0.f)
          atomicAdd(acc_m + 4 * g + e,
                    (unsigned long long)__float2ll_rn(pv[e] * A.fx_scale));
    }
    if (g < ld4) {
      if (DIAG) {
        const float4 c = load_cost_global<CT>(cg, g);
        const float4 th = thg[g];  // still the old column: stored below
        const float cv[4] = {c.x, c.y, c.z, c.w};
        const float ov[4] = {o.x, o.y, o.z, o.w};
        const float tv[4] = {th.x, th.y, th.z, th.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (pv[e] > 0.f) wc += cv[e] * pv[e];
          const float dd = ov[e] - tv[e];
          res += dd * dd;
        }
      }
      __stcs(tho + g, o);
    }
  }
  if (DIAG) {
    warp_sum2(wc, res);
    lbmin = warp_min(lbmin);
    if (lane == 0) {
      A.diag_wc[col] = wc;
      A.diag_res[col] = res;
      A.diag_lb[col] = tau * lbmin;
    }
  }
  if (lane == 0) A.lam[col] = lam_fin;
  return np;
}

template <int NV, typename CT, bool DIAG>
__global__ void __launch_bounds__(kWarpThreads, WarpMinBlocks<NV>::value)
    column_warp_kernel(const ColArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kTile = NV * 32 * 4;  // rows covered by one warp
  float* d_s = reinterpret_cast<float*>(smem);
  double* dred = reinterpret_cast<double*>(d_s + kTile);
  int* next_s = reinterpret_cast<int*>(dred + kRedSlots);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  const int R = A.R;

  const long long k_iter = *A.iter;
  const Sched sc = A.sched[draw_index_set(A.draw, k_iter)];
  const long long n_all = sc.col_end - sc.col_begin;
  const long long G = gridDim.x;
  const long long c0 = sc.col_begin + n_all * blockIdx.x / G;
  const long long c1 = sc.col_begin + n_all * (blockIdx.x + 1) / G;
  unsigned long long my_passes = 0;

  int p_cur = -1;
  double t_cur = 1.0;
  for (long long seg = c0; seg < c1;) {  // one measure at a time
    const int m = A.col_meas[seg];
    const long long seg_end = A.col_off[m + 1] < c1 ? A.col_off[m + 1] : c1;
    const int pr = A.meas_prob[m];
    if (pr != p_cur) {  // uniform: all threads call
      p_cur = pr;
      t_cur = t_from_blocks(A.blk + size_t(pr) * A.nblk * 4, A.nblk, A.rho_p[pr],
                            A.gamma_p[pr], dred, tid, nt);
      if (tid == 0) A.t_used[pr] = t_cur;
    }
    __syncthreads();  // every warp is done with the previous measure's d
    const double* dl = A.delta + size_t(m) * R;
    for (int i = tid; i < kTile; i += nt) d_s[i] = i < R ? float(t_cur * dl[i]) : 0.f;
    if (tid == 0) *next_s = 0;
    __syncthreads();
    const float irho = A.inv_rho[m];
    const float rho_m = A.rho[m];
    unsigned long long* acc_m = A.acc + size_t(m) * R;
    // Columns go to whichever warp is free (results do not depend on it).
    while (true) {
      int j = 0;
      if (lane == 0) j = atomicAdd(next_s, 1);
      j = __shfl_sync(0xffffffffu, j, 0);
      const long long col = seg + j;
      if (col >= seg_end) break;
      my_passes += warp_column<NV, CT, DIAG>(A, col, d_s, irho, rho_m, acc_m, lane);
    }
    seg = seg_end;
  }
  // Pass count and the iteration counter (the last CTA advances it).
  if (lane == 0) atomicAdd(A.passes, my_passes);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(A.done, 1u) == gridDim.x - 1) {
      *A.iter = k_iter + 1;
      *A.done = 0u;
    }
  }
}

#define MAM_WARP_NV_CASES(X) X(1) X(2) X(4) X(7) X(8) X(13) X(16) X(24) X(29) X(32)

template <int NV, typename CT>
cudaError_t warp_op(int op, bool diag, int grid, size_t smem, cudaStream_t st,
                    const ColArgs* a, int* occ) {
  if (op == 0) {
    if (diag) column_warp_kernel<NV, CT, true><<<grid, kWarpThreads, smem, st>>>(*a);
    else column_warp_kernel<NV, CT, false><<<grid, kWarpThreads, smem, st>>>(*a);
    return cudaGetLastError();
  }
  if (op == 1)
    return diag ? cudaFuncSetAttribute(column_warp_kernel<NV, CT, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))
                : cudaFuncSetAttribute(column_warp_kernel<NV, CT, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  return diag ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    occ, column_warp_kernel<NV, CT, true>, kWarpThreads, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    occ, column_warp_kernel<NV, CT, false>, kWarpThreads, smem);
}

template <typename CT>
cudaError_t warp_op_nv(int nv, int op, bool diag, int grid, size_t smem,
                       cudaStream_t st, const ColArgs* a, int* occ) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return warp_op<N, CT>(op, diag, grid, smem, st, a, occ);
    MAM_WARP_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t warp_op_any(int nv, int dt, int op, bool diag, int grid, size_t smem,
                        cudaStream_t st, const ColArgs* a, int* occ) {
  switch (dt) {
    case 0: return warp_op_nv<float>(nv, op, diag, grid, smem, st, a, occ);
    case 1: return warp_op_nv<__nv_bfloat16>(nv, op, diag, grid, smem, st, a, occ);
    case 2: return warp_op_nv<__half>(nv, op, diag, grid, smem, st, a, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool warp_kernel_has(int nv) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return true;
    MAM_WARP_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return false;
  }
}

int warp_kernel_threads() { return kWarpThreads; }

size_t warp_kernel_smem(int nv) {
  return size_t(nv) * 32 * 4 * sizeof(float) + kRedSlots * sizeof(double) + 16;
}

cudaError_t launch_column_warp(int nv, int cost_dtype, bool diag, int grid,
                               size_t smem, cudaStream_t st, const ColArgs& a) {
  return warp_op_any(nv, cost_dtype, 0, diag, grid, smem, st, &a, nullptr);
}

cudaError_t set_column_warp_smem(int nv, int cost_dtype, bool diag, size_t smem) {
  return warp_op_any(nv, cost_dtype, 1, diag, 0, smem, nullptr, nullptr, nullptr);
}

cudaError_t column_warp_occupancy(int nv, int cost_dtype, bool diag, size_t smem,
                                  int* blocks_per_sm) {
  return warp_op_any(nv, cost_dtype, 2, diag, 0, smem, nullptr, nullptr, blocks_per_sm);
}

}  // namespace mam
