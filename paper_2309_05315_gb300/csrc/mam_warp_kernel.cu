// libmam: the column step with one warp per plan column (R up to 2048).
//
// Same mathematics as column_kernel in mam_kernels.cu (Algorithm 1, Step 2,
// with the Step 3 row sums and the diagnostics), organised so that no CTA
// barrier sits on the per-column path:
//  * lane l of a warp holds the float4 groups g = v*32 + l (v < NV) of one
//    column in registers, and the threshold search reduces with warp
//    shuffles only;
//  * columns arrive through a ring of K shared-memory slots filled by
//    bulk-async copies (cp.async.bulk, completion counted on one mbarrier per
//    slot).  Warps claim columns in increasing order j; column j uses slot
//    j mod K and is phase j / K of that slot's mbarrier.  The warp that
//    consumed column j refills the slot with column j + K as soon as it has
//    read it, and counts the refill in the slot's issue counter.  A warp that
//    claims column j first waits until the counter shows that column j was
//    issued: the warp holding column j - K may still be waiting for its data
//    while other warps run ahead, and a parity wait started before phase
//    j / K - 1 completed would pass on that older phase.  Every issued copy
//    is therefore consumed before the CTA exits;
//  * the shift d^(m) = t (p - p^(m)) / S_m is read through L1 from an FP32
//    copy of (p - p^(m)) / S_m, so warps on different measures need no
//    shared state.
#include "mam_device.cuh"

namespace mam {
namespace {

// Threads per CTA allowed by the register budget of each width.
template <int NV>
struct RingMaxThreads {
  static constexpr int value = NV >= 24 ? 384 : NV >= 13 ? 512 : NV >= 7 ? 768 : 1024;
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

// t^k of Algorithm 1 for problem pr, evaluated by one warp from the
// averaging kernel's block sums (fixed order: every warp gets the same t).
__device__ __forceinline__ double warp_t(const ColArgs& A, int pr, int lane) {
  if (isinf(A.gamma_p[pr])) return 1.0;  // balanced: t = 1
  const double* b = A.blk + size_t(pr) * A.nblk * 4;
  double acc = 0.0;
  for (int i = lane; i < A.nblk; i += 32) acc += b[4 * i];
  acc = warp_sum_d(acc);
  // as t_from_blocks: sqrt and quotient in FP32, identical in every warp
  const float D = sqrtf(float(acc));
  const float rD = float(A.rho_p[pr]) * D;
  const float gamma = float(A.gamma_p[pr]);
  if (rD <= gamma) return 1.0;
  return double(__fdiv_rn(gamma, rD));
}

// Sum of max(w - l, 0) and #{w > l} over this lane's rows (independent
// accumulators keep the dependency chains short).
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

// The shift of rows 4g..4g+3: t * (p - p^(m)) / S_m (zero past the column).
__device__ __forceinline__ float4 shift4(const float* dm, int g, int ld4, float tf) {
  if (g >= ld4) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 v = __ldg(reinterpret_cast<const float4*>(dm) + g);
  return make_float4(__fmul_rn(tf, v.x), __fmul_rn(tf, v.y), __fmul_rn(tf, v.z),
                     __fmul_rn(tf, v.w));
}

// Threshold search on one warp's column (see column_kernel for the method):
// warm start from lam_prev, otherwise bracket [max w - tau, max w) and
// bisect.  Returns the threshold; np counts the passes.
template <int NV>
__device__ __forceinline__ float warp_search(const float (&w)[NV][4], float tau,
                                             float lam_prev, int bisect_depth, int& np) {
  if (!(tau > 0.f)) return INFINITY;  // Remark 1: Delta_R(0) = {0}
  const bool warm = lam_prev == lam_prev;
  float lam = warm ? lam_prev : 0.f;
  float lam_fin = lam;
  float nprev = -1.f;
  bool bracket = !warm;
  int it0 = 0;
  if (warm) {  // first pass at the warm start, with the Newton-step certificate
    float fs[4] = {0.f, 0.f, 0.f, 0.f}, ns[4] = {0.f, 0.f, 0.f, 0.f}, g = INFINITY;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float x = w[v][e] - lam;
        fs[e] += fmaxf(x, 0.f);
        ns[e] += x > 0.f ? 1.f : 0.f;
        g = fminf(g, fabsf(x));
      }
    float f = (fs[0] + fs[1]) + (fs[2] + fs[3]);
    float n = (ns[0] + ns[1]) + (ns[2] + ns[3]);
    warp_sum2(f, n);
    g = warp_min(g);
    ++np;
    it0 = 1;
    if (n == 0.f) {
      bracket = true;  // warm start at or above max w
    } else {
      const float dl = (f - tau) / n;
      const float l0 = lam;
      lam = lam + dl;
      if (newton_certified(g, dl, l0)) return lam;  // same active set: exact
      nprev = n;
      lam_fin = lam;
    }
  }
  for (int it = it0; it < kMaxNewton; ++it) {
    if (bracket) {
      float mx = -INFINITY;
#pragma unroll
      for (int v = 0; v < NV; ++v)
        mx = fmaxf(mx, fmaxf(fmaxf(w[v][0], w[v][1]), fmaxf(w[v][2], w[v][3])));
      mx = warp_max(mx);
      ++np;
      float lo_b = mx - tau, hi_b = mx;
      for (int b = 0; b < bisect_depth; ++b) {
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
    if (n == nprev) return lam;  // same active set twice: lam is the threshold
    if (n == 0.f) {              // at or above max w: restart from the bracket
      bracket = true;
      continue;
    }
    nprev = n;
    lam = lam + (f - tau) / n;
    lam_fin = lam;  // used if the pass budget runs out (not expected)
  }
  return lam_fin;
}

// Waits (bounded) until the shared counter *cnt reaches target.
__device__ __forceinline__ bool wait_count_bounded(const int* cnt, int target,
                                                   unsigned long long limit_ns) {
  const volatile int* v = cnt;
  if (*v >= target) return true;
  const unsigned long long t0 = global_ns();
  while (*v < target) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

template <int NV, typename CT, bool DIAG>
__global__ void __launch_bounds__(RingMaxThreads<NV>::value)
    column_ring_kernel(const ColArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int kSlot = NV * 128;  // elements per slot: what one warp covers
  const int K = A.stages;          // ring slots (>= warps per CTA)
  const int tid = threadIdx.x, lane = tid & 31;
  const int ld = A.ld, ld4 = ld >> 2, R = A.R;
  float* th_s = reinterpret_cast<float*>(smem);
  CT* c_s = reinterpret_cast<CT*>(smem + size_t(K) * kSlot * sizeof(float));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(K) * kSlot *
                                               (sizeof(float) + sizeof(CT)));
  int* issued_cnt = reinterpret_cast<int*>(full + K);
  int* next = issued_cnt + K;

  const long long k_iter = *A.iter;
  const Sched sc = A.sched[draw_index_set(A.draw, k_iter)];
  const long long n_all = sc.col_end - sc.col_begin;
  const long long G = gridDim.x;
  const long long c0 = sc.col_begin + n_all * blockIdx.x / G;
  const long long ncol = sc.col_begin + n_all * (blockIdx.x + 1) / G - c0;
  unsigned long long my_passes = 0;
  bool failed = false;

  if (ncol > 0) {  // uniform over the CTA
    const uint32_t bytes_th = uint32_t(ld) * sizeof(float);
    const uint32_t bytes_c = uint32_t(ld) * sizeof(CT);
    // Slot tails past the column (never written by the copies): theta = 0,
    // c = +inf, so those rows have w = -inf.
    for (int i = ld + tid; i < kSlot; i += blockDim.x)
      for (int s = 0; s < K; ++s) {
        th_s[size_t(s) * kSlot + i] = 0.f;
        c_s[size_t(s) * kSlot + i] = CT(INFINITY);
      }
    if (tid == 0) {
      for (int s = 0; s < K; ++s) {
        mbar_init(&full[s], 1);
        issued_cnt[s] = 0;
      }
      *next = 0;
      fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int j, int s) {  // column j into slot s = j mod K; one thread
      const long long col = c0 + j;
      mbar_expect_tx(&full[s], bytes_th + bytes_c);
      bulk_load(th_s + size_t(s) * kSlot, A.theta + size_t(col) * ld, bytes_th, &full[s]);
      const long long ccol = A.cost_col ? (long long)A.cost_col[col] : col;
      bulk_load(c_s + size_t(s) * kSlot, static_cast<const CT*>(A.cost) + size_t(ccol) * ld,
                bytes_c, &full[s]);
      __threadfence_block();  // the arrive and the copies precede the count
      atomicAdd(&issued_cnt[s], 1);
    };
    if (tid == 0)
      for (int j = 0; j < ncol && j < K; ++j) issue(j, j);

    pdl_wait();  // the averaging kernel's outputs are used from here on
    int p_cur = -1;
    float tf = 1.f;
    int m_cur = -1;
    float irho = 0.f, rho_m = 0.f, cm = 1.f;  // cm: factor of the stored cost (diagnostics)
    while (true) {
      int jj = 0;
      if (lane == 0) jj = atomicAdd(next, 1);
      const int j = __shfl_sync(0xffffffffu, jj, 0);
      if (j >= ncol) break;
      const int jq = j / K;  // 32-bit: a CTA holds fewer than 2^31 columns
      const int s = j - jq * K;
      bool ok = true;
      if (lane == 0) ok = wait_count_bounded(&issued_cnt[s], jq + 1, kWaitLimitNs);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (ok) ok = mbar_wait_bounded(&full[s], uint32_t(jq & 1), kWaitLimitNs);
      if (!__all_sync(0xffffffffu, ok)) {
        failed = true;
        break;
      }
      const long long col = c0 + j;
      const int m = A.col_meas[col];
      if (m != m_cur) {
        m_cur = m;
        const int pr = A.meas_prob[m];
        if (pr != p_cur) {
          p_cur = pr;
          const double t = warp_t(A, pr, lane);
          tf = float(t);
          if (lane == 0) A.t_used[pr] = t;
        }
        irho = A.inv_rho[m];
        rho_m = A.rho[m];
        if (DIAG) cm = A.cmul[m];
      }
      const float* dm = A.delta32 + size_t(m) * ld;
      const float* ths = th_s + size_t(s) * kSlot;
      const CT* cs = c_s + size_t(s) * kSlot;
      const float tau = A.q[col];
      const float lam_prev = A.lam[col];

      float w[NV][4];
      float lbmin = INFINITY;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int g = v * 32 + lane;
        const float4 th = reinterpret_cast<const float4*>(ths)[g];
        const float4 c = CostIO<CT>::load4(cs, g);
        const float4 d = shift4(dm, g, ld4, tf);
        w[v][0] = fmaf(-c.x, irho, fmaf(2.f, d.x, th.x));
        w[v][1] = fmaf(-c.y, irho, fmaf(2.f, d.y, th.y));
        w[v][2] = fmaf(-c.z, irho, fmaf(2.f, d.z, th.z));
        w[v][3] = fmaf(-c.w, irho, fmaf(2.f, d.w, th.w));
        if (DIAG)
          lbmin = fminf(fminf(fminf(lbmin, cm * c.x - rho_m * d.x),
                              fminf(cm * c.y - rho_m * d.y, cm * c.z - rho_m * d.z)),
                        cm * c.w - rho_m * d.w);
      }
      if (!DIAG) {
        __syncwarp();  // every lane has read the slot
        if (lane == 0 && j + K < ncol) issue(j + K, s);
      }
      int np = 0;
      const float lam_s = warp_search<NV>(w, tau, lam_prev, A.bisect_depth, np);
      // capped columns apply max(lambda, 0) (lam_floor = 0; -inf otherwise)
      const float lam = fmaxf(lam_s, A.lam_floor);
      my_passes += np;

      // Commit: theta' = pihat - d (streaming stores), Step 3 row sums.
      unsigned long long* acc_m = A.acc + size_t(m) * R;
      float4* tho = reinterpret_cast<float4*>(A.theta + size_t(col) * ld);
      float wc = 0.f, res = 0.f;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int g = v * 32 + lane;
        const float4 d = shift4(dm, g, ld4, tf);
        const float pv[4] = {fmaxf(w[v][0] - lam, 0.f), fmaxf(w[v][1] - lam, 0.f),
                             fmaxf(w[v][2] - lam, 0.f), fmaxf(w[v][3] - lam, 0.f)};
        const float4 o = make_float4(pv[0] - d.x, pv[1] - d.y, pv[2] - d.z, pv[3] - d.w);
        const bool act = fmaxf(fmaxf(pv[0], pv[1]), fmaxf(pv[2], pv[3])) > 0.f;
        if (__any_sync(0xffffffffu, act) && act) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (pv[e] > 0.f)
              atomicAdd(acc_m + 4 * g + e,
                        (unsigned long long)f32_to_i64_rn(pv[e] * A.fx_scale));
        }
        if (A.amask) {  // active-set bits of this column (reverse sweep)
          unsigned word = ((pv[0] > 0.f ? 1u : 0u) | (pv[1] > 0.f ? 2u : 0u) |
                           (pv[2] > 0.f ? 4u : 0u) | (pv[3] > 0.f ? 8u : 0u))
                          << (4 * (lane & 7));
          word |= __shfl_xor_sync(0xffffffffu, word, 1);
          word |= __shfl_xor_sync(0xffffffffu, word, 2);
          word |= __shfl_xor_sync(0xffffffffu, word, 4);
          if ((lane & 7) == 0 && 4 * g < ld) A.amask[size_t(col) * A.mw + g / 8] = word;
        }
        if (g < ld4) {
          if (DIAG) {
            const float4 c = CostIO<CT>::load4(cs, g);
            const float4 th = reinterpret_cast<const float4*>(ths)[g];
            const float cv[4] = {cm * c.x, cm * c.y, cm * c.z, cm * c.w};
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
          A.diag_lb[col] = tau * fminf(lbmin, A.lb_cap);
        }
        __syncwarp();
        if (lane == 0 && j + K < ncol) issue(j + K, s);
      }
      if (lane == 0) A.lam[col] = lam_s;
    }
    if (lane == 0 && my_passes) atomicAdd(A.passes, my_passes);
    if (failed && lane == 0) atomicCAS(A.err, 0, 1);
    __syncthreads();
    if (tid == 0 && atomicOr(A.err, 0) != 0) {
      // Drain the copies still in flight (bounded) before leaving.
      for (int s = 0; s < K; ++s)
        if (issued_cnt[s] > 0)
          mbar_wait_bounded(&full[s], uint32_t((issued_cnt[s] - 1) & 1), kWaitLimitNs / 20);
    }
  }
  pdl_wait();
  // The last CTA to finish advances the iteration counter (every CTA has
  // read it by then).
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(A.done, 1u) == gridDim.x - 1) {
      *A.iter = k_iter + 1;
      *A.done = 0u;
    }
  }
}

#define MAM_RING_NV_CASES(X) X(1) X(2) X(4) X(7) X(8) X(13) X(16)

template <int NV, typename CT>
cudaError_t ring_op(int op, bool diag, int grid, int threads, size_t smem,
                    cudaStream_t st, const ColArgs* a, int* occ) {
  if (op == 0) {
    return diag ? launch_pdl(column_ring_kernel<NV, CT, true>, dim3(grid), dim3(threads), smem, st, *a)
                : launch_pdl(column_ring_kernel<NV, CT, false>, dim3(grid), dim3(threads), smem, st, *a);
  }
  if (op == 1)
    return diag ? cudaFuncSetAttribute(column_ring_kernel<NV, CT, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))
                : cudaFuncSetAttribute(column_ring_kernel<NV, CT, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  return diag ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    occ, column_ring_kernel<NV, CT, true>, threads, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    occ, column_ring_kernel<NV, CT, false>, threads, smem);
}

template <typename CT>
cudaError_t ring_op_nv(int nv, int op, bool diag, int grid, int threads, size_t smem,
                       cudaStream_t st, const ColArgs* a, int* occ) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return ring_op<N, CT>(op, diag, grid, threads, smem, st, a, occ);
    MAM_RING_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t ring_op_any(int nv, int dt, int op, bool diag, int grid, int threads,
                        size_t smem, cudaStream_t st, const ColArgs* a, int* occ) {
  switch (dt) {
    case 0: return ring_op_nv<float>(nv, op, diag, grid, threads, smem, st, a, occ);
    case 1: return ring_op_nv<__nv_bfloat16>(nv, op, diag, grid, threads, smem, st, a, occ);
    case 2: return ring_op_nv<__half>(nv, op, diag, grid, threads, smem, st, a, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool ring_kernel_has(int nv) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return true;
    MAM_RING_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return false;
  }
}

int ring_kernel_max_threads(int nv) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return RingMaxThreads<N>::value;
    MAM_RING_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return 0;
  }
}

size_t ring_kernel_smem(int nv, int slots, int cost_bytes) {
  return size_t(slots) * nv * 128 * (sizeof(float) + cost_bytes) +
         size_t(slots) * (sizeof(uint64_t) + sizeof(int)) + 16;
}

cudaError_t launch_column_ring(int nv, int cost_dtype, bool diag, int grid, int threads,
                               size_t smem, cudaStream_t st, const ColArgs& a) {
  return ring_op_any(nv, cost_dtype, 0, diag, grid, threads, smem, st, &a, nullptr);
}

cudaError_t set_column_ring_smem(int nv, int cost_dtype, bool diag, size_t smem) {
  return ring_op_any(nv, cost_dtype, 1, diag, 0, 0, smem, nullptr, nullptr, nullptr);
}

cudaError_t column_ring_occupancy(int nv, int cost_dtype, bool diag, int threads,
                                  size_t smem, int* blocks_per_sm) {
  return ring_op_any(nv, cost_dtype, 2, diag, 0, threads, smem, nullptr, nullptr, blocks_per_sm);
}

}  // namespace mam
