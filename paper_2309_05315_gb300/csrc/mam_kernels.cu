// libmam device code: the per-iteration kernels of the Method of Averaged
// Marginals (arXiv 2309.05315, Algorithm 1) for sm_103a.
//
//   column_kernel   Step 2 of Algorithm 1 for every column of the index set
//                   M^k, fused with the row sums of Step 3 (order-independent
//                   fixed-point accumulation) and with the diagnostics
//                   (W-hat, lower bound, fixed-point residual).
//   average_kernel  Step 3 completion (64-bit fixed point), Step 1 (p = sum_m a_m p^(m),
//                   eq. pr) and the factor t^k.
//
// Plans theta and costs c are stored column-contiguous with a padded stride
// ld (a multiple of 8 elements), so that one column is one contiguous run of
// 4*ld (theta) and ld*sizeof(cost) bytes: each column is brought into shared
// memory by two bulk-async copies (cp.async.bulk, completion on an mbarrier)
// while the CTA works on the previous column.
#include "mam_device.cuh"

#include <cfloat>
#include <cmath>
#include <type_traits>

namespace mam {
namespace {

// ------------------------------------------------------- column kernel

// Step 2 of Algorithm 1 for one CTA's slice of the index set, one column at
// a time.  Thread `tid` owns the float4 groups idx = v*nt + tid (v < NV) of
// every column, i.e. rows r = 4*idx .. 4*idx+3, held as two FP32 pairs; its
// shift d^(m)_r is written once per measure to a thread-private shared-memory
// tile and read from there by every column of that measure.
//
// Per column s of measure m (tau = q_s):
//   w_r     = theta_rs + 2 d_r - c_rs / rho        (Alg. 1, w)
//   lambda  : sum_r max(w_r - lambda, 0) = tau     (Prop. 3, Remark 1)
//   pihat_r = max(w_r - lambda, 0)                 (Alg. 1, projection)
//   theta'  = pihat_r - d_r                        (Alg. 1, update)
// with d_r = t^k (p_r - p^(m)_r) / S_m.  Step 3 needs the row sums of
// theta', i.e. sum_s pihat_rs - S_m d_r; the kernel accumulates the sparse
// part sum_s pihat_rs as 64-bit fixed-point integers (pihat * 2^e, added with
// integer atomics, so the result does not depend on the order of the adds).
//
// Threshold search (exact).  f(l) = sum_r max(w_r - l, 0) is convex,
// piecewise linear and decreasing; n(l) = #{w_r > l} = -f'(l).  The Newton
// step l <- l + (f(l) - tau) / n(l) equals Michelot's update
// (sum_{w>l} w - tau) / n(l): from any l > lambda* it lands at or below
// lambda*, and from below it increases monotonically.  The active sets
// {w > l} of two successive iterates are nested, so equal counts mean equal
// sets, and then the later iterate is exactly lambda*.  The search starts
// from the column's previous threshold (warm start, usually one Newton step
// and one confirming pass); without one it brackets lambda* in
// [max w - tau, max w), bisects bisect_depth times and continues from the
// lower end.
//
// Rows beyond R need no masks: the shared-memory tiles are threads*vec*4
// long, their tails past the column hold theta = 0 and c = +inf (written
// once per CTA), and the cost's padding rows R..ld-1 are +inf in memory, so
// every such row has w = -inf and never enters the active set.
template <int NV, typename CT, bool DIAG>
__global__ void __launch_bounds__(MaxThreads<NV>::value, MinCtas<NV>::value)
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
  const int tile = nt * NV * 4;  // elements per shared-memory stage
  const int stages = A.stages;

  float* th_s = reinterpret_cast<float*>(smem);
  CT* c_s = reinterpret_cast<CT*>(smem + size_t(stages) * tile * sizeof(float));
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      smem + size_t(stages) * tile * (sizeof(float) + sizeof(CT)));
  float4* red = reinterpret_cast<float4*>(bar + 4);
  double* dred = reinterpret_cast<double*>(red + 2 * kRedSlots);
  // d of this thread's rows for the current measure: thread-private (a thread
  // reads only the rows it wrote), so it needs no barrier, and it frees the
  // registers that would hold it across the column loop.
  float4* d_s = reinterpret_cast<float4*>(dred + kRedSlots);

  const long long k_iter = *A.iter;
  const Sched sc = A.sched[draw_index_set(A.draw, k_iter)];
  const long long n_all = sc.col_end - sc.col_begin;
  const long long G = gridDim.x;
  const long long col0 = sc.col_begin + n_all * blockIdx.x / G;
  const long long ncol = sc.col_begin + n_all * (blockIdx.x + 1) / G - col0;
  bool any_fail = false;
  unsigned long long my_passes = 0;

  if (ncol > 0) {  // uniform over the CTA
    const uint32_t bytes_th = uint32_t(ld) * sizeof(float);
    const uint32_t bytes_c = uint32_t(ld) * sizeof(CT);
    // Tails of every stage (never written by the copies).
    for (int i = ld + tid; i < tile; i += nt)
      for (int s = 0; s < stages; ++s) {
        th_s[size_t(s) * tile + i] = 0.f;
        c_s[size_t(s) * tile + i] = CT(INFINITY);
      }
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
      bulk_load(th_s + size_t(s) * tile, A.theta + size_t(col) * ld, bytes_th,
                &bar[s]);
      const long long ccol = A.cost_col ? (long long)A.cost_col[col] : col;
      bulk_load(c_s + size_t(s) * tile,
                static_cast<const CT*>(A.cost) + size_t(ccol) * ld, bytes_c,
                &bar[s]);
    };
    if (tid == 0) {
      const long long n0 = ncol < stages ? ncol : stages;
      for (long long j = 0; j < n0; ++j) issue(j);
      issued = n0;
    }
    // Thread 0 refills the stage of column j with column j + stages, once
    // every thread is past its last read of that stage.
    auto refill = [&](long long j) {
      if (tid == 0 && j + stages < ncol) {
        issue(j + stages);
        ++issued;
      }
    };

    float rho_m = 0.f, cm = 1.f;  // cm: factor of the stored cost (diagnostics)
    f2_t nirho2 = 0ull;
    const f2_t two2 = pk(2.f, 2.f);
    int m_cur = -1, p_cur = -1;
    double t_cur = 1.0;
    unsigned long long* acc_m = nullptr;
    const float fx = A.fx_scale;
    int rb = 0;

    // Per-column scalars are loaded one column ahead.
    // Everything above only touched this kernel's own inputs (plans and costs
    // written by the previous column step); from here on the averaging
    // kernel's outputs (shifts, block sums, cleared accumulators) are used.
    pdl_wait();
    int m_nx = A.col_meas[col0];
    float tau_nx = A.q[col0];
    float lam_nx = A.lam[col0];
    for (long long j = 0; j < ncol; ++j) {
      const long long col = col0 + j;
      const int m = m_nx;
      const float tau = tau_nx;
      const float lam_prev = lam_nx;
      if (j + 1 < ncol) {
        m_nx = A.col_meas[col + 1];
        tau_nx = A.q[col + 1];
        lam_nx = A.lam[col + 1];
      }
      if (m != m_cur) {  // first column of a measure in this slice
        m_cur = m;
        const int pr = A.meas_prob[m];
        if (pr != p_cur) {
          p_cur = pr;
          t_cur = t_from_blocks(A.blk + size_t(pr) * A.nblk * 4, A.nblk,
                                A.rho_p[pr], A.gamma_p[pr], dred, tid, nt);
          if (tid == 0) A.t_used[pr] = t_cur;
        }
        rho_m = A.rho[m];
        if (DIAG) cm = A.cmul[m];
        nirho2 = pk(-A.inv_rho[m], -A.inv_rho[m]);
        acc_m = A.acc + size_t(m) * R;
        const float* dl = A.delta32 + size_t(m) * ld;
        const float tf = float(t_cur);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int idx = v * nt + tid;
          float dv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int r = 4 * idx + e;
            dv[e] = r < R ? __fmul_rn(tf, dl[r]) : 0.f;
          }
          d_s[idx] = make_float4(dv[0], dv[1], dv[2], dv[3]);
        }
      }
      const int s = int(j % stages);
      const bool failed =
          !mbar_wait_bounded(&bar[s], uint32_t((j / stages) & 1), kWaitLimitNs);
      const float* ths = th_s + size_t(s) * tile;
      const CT* cs = c_s + size_t(s) * tile;
      const bool pos = tau > 0.f;
      const bool warm = pos && (lam_prev == lam_prev);
      const float l0 = warm ? lam_prev : 0.f;
      const f2_t l02 = pk(l0, l0);

      // Pass 1: w, and (f, n) at l0.
      f2_t w2[NV][2];
      float lbmin = INFINITY;
      f2_t fa = 0ull, fb = 0ull;  // two packed accumulators
      float n = 0.f;
      float gap0 = INFINITY;  // min_r |w_r - l0|: certificate of the warm Newton step
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int idx = v * nt + tid;
        const float4 th = reinterpret_cast<const float4*>(ths)[idx];
        const float4 c = CostIO<CT>::load4(cs, idx);
        const f2_t c01 = pk(c.x, c.y), c23 = pk(c.z, c.w);
        const float4 dd = d_s[idx];
        const f2_t d01 = pk(dd.x, dd.y), d23 = pk(dd.z, dd.w);
        w2[v][0] = fma2(c01, nirho2, fma2(two2, d01, pk(th.x, th.y)));
        w2[v][1] = fma2(c23, nirho2, fma2(two2, d23, pk(th.z, th.w)));
        const f2_t x0 = sub2(w2[v][0], l02), x1 = sub2(w2[v][1], l02);
        gap0 = fminf(gap0, fminf(fminf(fabsf(lo(x0)), fabsf(hi(x0))),
                                 fminf(fabsf(lo(x1)), fabsf(hi(x1)))));
        fa = add2(fa, relu2(x0, n));
        fb = add2(fb, relu2(x1, n));
        if (DIAG) {
          lbmin = fminf(lbmin, fminf(fminf(cm * c.x - rho_m * dd.x, cm * c.y - rho_m * dd.y),
                                     fminf(cm * c.z - rho_m * dd.z, cm * c.w - rho_m * dd.w)));
        }
      }
      // The failure flag rides in the first reduction (f < 0 marks it).
      {
        const f2_t fs = add2(fa, fb);
        float f = lo(fs) + hi(fs);
        if (failed) f = -INFINITY;
        reduce3<true>(f, n, gap0, red, rb, lane, warp, nw);
        if (!DIAG) refill(j);
        any_fail = !(f >= 0.f);
        fa = pk(f, 0.f);  // keep f (lo) for the search below
      }
      int np = 1;
      float lam_fin = INFINITY;
      if (pos) {
        float f = lo(fa);
        float nprev = -1.f;
        bool bracket = !warm;
        float lam = l0;
        bool done = false;
        if (warm) {
          if (n == 0.f) bracket = true;  // warm start at or above max w
          else {
            const float dl = (f - tau) / n;
            lam = l0 + dl;
            nprev = n;
            // No w_r between l0 and the Newton point (with a margin for the
            // rounding of w - l0 and of l0 + dl): the active set at lam is the
            // one at l0, so lam is the threshold -- the value the confirming
            // pass below would return.
            if (newton_certified(gap0, dl, l0)) {
              lam_fin = lam;
              done = true;
            }
          }
        }
        for (int it = 0; it < kMaxNewton && !done; ++it) {
          if (bracket) {  // lambda* lies in [max w - tau, max w)
            float mx = -INFINITY, z0 = 0.f, z1 = 0.f;
#pragma unroll
            for (int v = 0; v < NV; ++v)
              mx = fmaxf(mx, fmaxf(fmaxf(lo(w2[v][0]), hi(w2[v][0])),
                                   fmaxf(lo(w2[v][1]), hi(w2[v][1]))));
            reduce3<false>(z0, z1, mx, red, rb, lane, warp, nw);
            ++np;
            float lo_b = mx - tau, hi_b = mx;
            for (int b = 0; b < A.bisect_depth; ++b) {
              const float mid = 0.5f * (lo_b + hi_b);
              const f2_t mid2 = pk(mid, mid);
              f2_t ga = 0ull;
              float cnt = 0.f, zz = 0.f;
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                ga = add2(ga, relu2(sub2(w2[v][0], mid2), cnt));
                ga = add2(ga, relu2(sub2(w2[v][1], mid2), cnt));
              }
              float fm = lo(ga) + hi(ga);
              reduce3<false>(fm, cnt, zz, red, rb, lane, warp, nw);
              ++np;
              if (fm >= tau) lo_b = mid; else hi_b = mid;
            }
            lam = lo_b;
            nprev = -1.f;
            bracket = false;
          }
          // (f, n) at lam.
          const f2_t lam2 = pk(lam, lam);
          f2_t ga = 0ull, gb = 0ull;
          float cnt = 0.f;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            ga = add2(ga, relu2(sub2(w2[v][0], lam2), cnt));
            gb = add2(gb, relu2(sub2(w2[v][1], lam2), cnt));
          }
          const f2_t gs = add2(ga, gb);
          f = lo(gs) + hi(gs);
          float z = 0.f;
          reduce3<false>(f, cnt, z, red, rb, lane, warp, nw);
          ++np;
          if (cnt == nprev) {  // same active set twice: lam is the threshold
            lam_fin = lam;
            break;
          }
          if (cnt == 0.f) {  // not expected from below; restart from the bracket
            bracket = true;
            continue;
          }
          nprev = cnt;
          lam = lam + (f - tau) / cnt;
          lam_fin = lam;  // used if the pass budget runs out (not expected)
        }
      }

      // Commit: theta' = pihat - d, Step 3 row sums (+ diagnostics).  With
      // capped columns (Delta_<=(q_s)) the threshold applied is
      // max(lambda, 0): a simplex threshold at or below 0 means the clipped
      // column already carries at most q_s.  lam_floor is -inf otherwise.
      const float lam_use = fmaxf(lam_fin, A.lam_floor);
      const f2_t lf2 = pk(lam_use, lam_use);
      float wc = 0.f, res = 0.f;
      float4* gth = reinterpret_cast<float4*>(A.theta + size_t(col) * ld);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int idx = v * nt + tid;
        float dummy = 0.f;
        const f2_t p01 = relu2(sub2(w2[v][0], lf2), dummy);
        const f2_t p23 = relu2(sub2(w2[v][1], lf2), dummy);
        const float4 dd = d_s[idx];
        const f2_t o01 = sub2(p01, pk(dd.x, dd.y));
        const f2_t o23 = sub2(p23, pk(dd.z, dd.w));
        const float pv[4] = {lo(p01), hi(p01), lo(p23), hi(p23)};
        // pihat is sparse: convert and add only where some lane of the warp
        // has an active row in this group.
        const bool act = fmaxf(fmaxf(pv[0], pv[1]), fmaxf(pv[2], pv[3])) > 0.f;
        if (__any_sync(0xffffffffu, act) && act) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (pv[e] > 0.f)
              atomicAdd(acc_m + 4 * idx + e,
                        (unsigned long long)f32_to_i64_rn(pv[e] * fx));
        }
        if (A.amask) {  // active-set bits of this column (reverse sweep)
          unsigned word = ((pv[0] > 0.f ? 1u : 0u) | (pv[1] > 0.f ? 2u : 0u) |
                           (pv[2] > 0.f ? 4u : 0u) | (pv[3] > 0.f ? 8u : 0u))
                          << (4 * (tid & 7));
          word |= __shfl_xor_sync(0xffffffffu, word, 1);
          word |= __shfl_xor_sync(0xffffffffu, word, 2);
          word |= __shfl_xor_sync(0xffffffffu, word, 4);
          if ((tid & 7) == 0 && 4 * idx < ld) A.amask[size_t(col) * A.mw + idx / 8] = word;
        }
        if (idx < ld4) {
          const float4 ov = make_float4(lo(o01), hi(o01), lo(o23), hi(o23));
          if (DIAG) {
            const float4 th = reinterpret_cast<const float4*>(ths)[idx];
            const float4 c = CostIO<CT>::load4(cs, idx);
            const float thv[4] = {th.x, th.y, th.z, th.w};
            const float cv[4] = {cm * c.x, cm * c.y, cm * c.z, cm * c.w};
            const float ovv[4] = {ov.x, ov.y, ov.z, ov.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (pv[e] > 0.f) wc += cv[e] * pv[e];
              const float dd = ovv[e] - thv[e];
              res += dd * dd;
            }
          }
          gth[idx] = ov;
        }
      }
      if (DIAG) {
        reduce3<true>(wc, res, lbmin, red, rb, lane, warp, nw);
        if (tid == 0) {
          A.diag_wc[col] = wc;
          A.diag_res[col] = res;
          A.diag_lb[col] = tau * fminf(lbmin, A.lb_cap);
        }
        refill(j);  // the reduction's barrier ended every read of stage s
      }
      if (tid == 0) A.lam[col] = lam_fin;
      my_passes += np;
      if (any_fail) break;  // uniform: the flag went through a reduction
    }
    if (any_fail && tid == 0) {
      atomicCAS(A.err, 0, 1);
      // Drain the copies still in flight (bounded) before leaving.
      for (long long j = 0; j < issued; ++j)
        mbar_wait_bounded(&bar[j % stages], uint32_t((j / stages) & 1),
                          kWaitLimitNs / 20);
    }
  }
  if (tid == 0) {
    atomicAdd(A.passes, my_passes);
    pdl_wait();  // (CTAs with no columns reach this point directly)
    // The last CTA to finish advances the iteration counter (every CTA has
    // read it by then).
    __threadfence();
    if (atomicAdd(A.done, 1u) == gridDim.x - 1) {
      *A.iter = k_iter + 1;
      *A.done = 0u;
    }
  }
}

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

template <int NV, typename CT, bool DIAG>
cudaError_t col_op_k(int op, int grid, int threads, size_t smem, cudaStream_t st,
                     const ColArgs* a, int* occ) {
  auto kern = column_kernel<NV, CT, DIAG>;
  if (op == 0) return launch_pdl(kern, dim3(grid), dim3(threads), smem, st, *a);
  if (op == 1)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, threads, smem);
}

// Dispatch over the compile-time (NV, cost type, DIAG) variants.
#define MAM_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(8)

template <int NV, typename CT>
cudaError_t col_op(int op, bool diag, int grid, int threads, size_t smem,
                   cudaStream_t st, const ColArgs* a, int* occ) {
  return diag ? col_op_k<NV, CT, true>(op, grid, threads, smem, st, a, occ)
              : col_op_k<NV, CT, false>(op, grid, threads, smem, st, a, occ);
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
