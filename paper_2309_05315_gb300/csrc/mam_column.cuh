// libmam device code: the fused column kernel of the Method of Averaged
// Marginals (arXiv 2309.05315, Algorithm 1, Step 2 with the Step 3 row sums),
// one CTA per column, for sm_103a, with its launch dispatch.  Included by
// mam_kernels.cu (dense plans) and mam_sparse.cu (sparse plans), each of
// which instantiates one layout.
#pragma once

#include "mam_device.cuh"

#include <cfloat>
#include <cmath>
#include <type_traits>

namespace mam {
namespace {

// Sparse plans, one float4 group of rows r0 .. r0 + 3 with an active row:
// the Step 3 row sums of its active rows and their (row, pihat) pairs, a slot
// each from the column's shared-memory counter (the order of the pairs is
// immaterial; slots past K are counted, not written).  Not inlined: active
// groups are few, and the column kernel's loop stays small enough for the
// instruction cache.
__device__ __noinline__ void sparse_commit_group(const float (&pv)[4], int r0,
                                                 unsigned long long* acc, float fx,
                                                 int* counter, int2* dst, int K) {
  int slot = atomicAdd(counter, int(pv[0] > 0.f) + int(pv[1] > 0.f) + int(pv[2] > 0.f) +
                                    int(pv[3] > 0.f));
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (pv[e] > 0.f) {
      atomicAdd(acc + r0 + e, (unsigned long long)f32_to_i64_rn(pv[e] * fx));
      if (slot < K) dst[slot] = make_int2(r0 + e, __float_as_int(pv[e]));
      ++slot;
    }
}

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
// sets, and then the later iterate is exactly lambda*.  A pass that finds no
// w_r between its point and its Newton point (up to rounding) certifies that
// point without the confirming pass.  The search starts from the column's
// previous threshold (warm start, usually one pass); without one it brackets
// lambda* in [max w - tau, max w), bisects bisect_depth times and continues
// from the lower end.
//
// Rows beyond R need no masks: the shared-memory tiles are threads*vec*4
// long, their tails past the column hold theta = 0 and c = +inf (written
// once per CTA), and the cost's padding rows R..ld-1 are +inf in memory, so
// every such row has w = -inf and never enters the active set.
//
// SP: the sparse plan layout.  Every step sets theta' = pihat - d with pihat
// zero off the active set, so a column is stored as the (row, value) pairs
// of its pihat and each measure keeps the d of its last visit (d_last,
// written by the averaging kernel).  One theta tile per CTA holds 0 - d_last
// of the current measure; a column's pairs arrive with its cost (one bulk
// copy of round_up(count, 2) pairs), are scattered into the tile as
// value + (0 - d_last_r) -- the FP32 value the dense layout stores -- before
// pass 1 and restored after it, so pass 1 reads the column's theta from the
// tile.  A column never visited (count -1) fills the tile with theta^0
// (q_s / R, or 0) and refills it with 0 - d_last afterwards.  The commit
// skips groups without an active row and writes a pair per active row
// (sparse_commit_group) instead of theta; the count is stored once the next
// barrier has passed.  Stages must be 1.
template <int NV, typename CT, bool DIAG, bool SP>
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

  // Dense: [stages][tile] theta, [stages][tile] c.  Sparse: one theta tile
  // (-d_last with the column's pihat scattered in), [stages][tile] c,
  // [stages][K] pairs.  Then 4 barriers, the reduction slots, (sparse: 4
  // counters,) the d tile.
  const int nth = SP ? 1 : stages;
  const int K = SP ? A.sp_k : 0;
  float* th_s = reinterpret_cast<float*>(smem);
  CT* c_s = reinterpret_cast<CT*>(smem + size_t(nth) * tile * sizeof(float));
  int2* pr_s = reinterpret_cast<int2*>(reinterpret_cast<unsigned char*>(c_s) +
                                       size_t(stages) * tile * sizeof(CT));
  uint64_t* bar = reinterpret_cast<uint64_t*>(pr_s + size_t(stages) * K);
  float4* red = reinterpret_cast<float4*>(bar + 4);
  double* dred = reinterpret_cast<double*>(red + 2 * kRedSlots);
  int* cnt_s = reinterpret_cast<int*>(dred + kRedSlots);  // sparse: pairs written, by column parity
  // d of this thread's rows for the current measure: thread-private (a thread
  // reads only the rows it wrote), so it needs no barrier, and it frees the
  // registers that would hold it across the column loop.
  float4* d_s = reinterpret_cast<float4*>(cnt_s + (SP ? 4 : 0));

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
    for (int i = ld + tid; i < tile; i += nt) {
      for (int s = 0; s < nth; ++s) th_s[size_t(s) * tile + i] = 0.f;
      for (int s = 0; s < stages; ++s) c_s[size_t(s) * tile + i] = CT(INFINITY);
    }
    if (SP && tid < 4) cnt_s[tid] = 0;
    if (tid == 0) {
      for (int s = 0; s < stages; ++s) mbar_init(&bar[s], 1);
      fence_mbar_init();
    }
    __syncthreads();
    long long issued = 0;  // meaningful in thread 0 only
    // Sparse: cnt is the column's number of stored pairs (-1: theta^0).
    auto issue = [&](long long j, int cnt) {
      const int s = int(j % stages);
      const long long col = col0 + j;
      const long long ccol = A.cost_col ? (long long)A.cost_col[col] : col;
      if (SP) {
        // the slots were last written by the scatter (generic proxy), and
        // every thread has passed a barrier since
        fence_proxy_async_smem();
        const uint32_t bytes_p = cnt > 0 ? uint32_t((cnt + 1) & ~1) * uint32_t(sizeof(int2)) : 0u;
        mbar_expect_tx(&bar[s], bytes_c + bytes_p);
        if (bytes_p)
          bulk_load(pr_s + size_t(s) * K, A.sp_pairs + size_t(col) * K, bytes_p, &bar[s]);
      } else {
        mbar_expect_tx(&bar[s], bytes_th + bytes_c);
        bulk_load(th_s + size_t(s) * tile, A.theta + size_t(col) * ld, bytes_th,
                  &bar[s]);
      }
      bulk_load(c_s + size_t(s) * tile,
                static_cast<const CT*>(A.cost) + size_t(ccol) * ld, bytes_c,
                &bar[s]);
    };
    if (tid == 0) {
      const long long n0 = ncol < stages ? ncol : stages;
      for (long long j = 0; j < n0; ++j) issue(j, SP ? min(A.sp_cnt[col0 + j], K) : 0);
      issued = n0;
    }
    // Thread 0 refills the stage of column j with column j + stages, once
    // every thread is past its last read of that stage (sparse: cnt_next is
    // the count of column j + 1 = j + stages).
    auto refill = [&](long long j, int cnt_next) {
      if (tid == 0 && j + stages < ncol) {
        issue(j + stages, cnt_next);
        ++issued;
      }
    };
    // Sparse: store the number of pairs column j wrote (every thread has
    // passed a barrier since its commit); a count above K fails the step.
    auto finalize = [&](long long j) {
      int* c = cnt_s + (j & 1);
      const int n = *c;
      *c = 0;
      A.sp_cnt[col0 + j] = n < K ? n : K;
      if (n > K) atomicCAS(A.err, 0, 2);
    };

    // Sparse: the theta tile of measure m, 0 - d_last_r on every row (the
    // value the dense commit stores on an inactive row).
    auto fill_tile = [&](int m) {
      const float4* dla = reinterpret_cast<const float4*>(A.d_last + size_t(m) * ld);
#pragma unroll 1
      for (int idx = tid; idx < ld4; idx += nt) {
        const float4 x = dla[idx];
        reinterpret_cast<float4*>(th_s)[idx] =
            make_float4(0.f - x.x, 0.f - x.y, 0.f - x.z, 0.f - x.w);
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
    // (counts above K, possible only in a foreign state blob, are clamped:
    // the copies never pass the slots)
    int cnt_nx = SP ? min(A.sp_cnt[col0], K) : 0;
    for (long long j = 0; j < ncol; ++j) {
      const long long col = col0 + j;
      const int m = m_nx;
      const float tau = tau_nx;
      const float lam_prev = lam_nx;
      const int npairs = cnt_nx;   // sparse: pairs of this column (-1: theta^0)
      // sparse: theta^0 of a column never visited (read only then)
      const float th0v = (SP && npairs < 0) ? __ldg(A.th0 + col) : 0.f;
      if (j + 1 < ncol) {
        m_nx = A.col_meas[col + 1];
        tau_nx = A.q[col + 1];
        lam_nx = A.lam[col + 1];
        if (SP) {
          cnt_nx = min(A.sp_cnt[col + 1], K);
        }
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
        if (SP) {
          // (shared: the scatters below write any row, hence the barrier)
          fill_tile(m);
          __syncthreads();
        }
      }
      if (SP && npairs < 0) {
        // a column never visited: theta^0 on rows < R (the copies do not
        // touch the tile, and every read of it by the previous column ended
        // at a barrier)
#pragma unroll 1
        for (int idx = tid; idx < ld4; idx += nt) {
          const int r = 4 * idx;
          reinterpret_cast<float4*>(th_s)[idx] =
              make_float4(r < R ? th0v : 0.f, r + 1 < R ? th0v : 0.f, r + 2 < R ? th0v : 0.f,
                          r + 3 < R ? th0v : 0.f);
        }
        __syncthreads();
      }
      const int s = int(j % stages);
      const bool failed =
          !mbar_wait_bounded(&bar[s], uint32_t((j / stages) & 1), kWaitLimitNs);
      const float* ths = SP ? th_s : th_s + size_t(s) * tile;
      const CT* cs = c_s + size_t(s) * tile;
      if (SP && npairs > 0) {
        // scatter the column's pihat: theta_r = pihat_r + (-d_last_r); the
        // slot keeps the tile's value for the restore
        int2* prs = pr_s + size_t(s) * K;
#pragma unroll 1
        for (int i = tid; i < npairs; i += nt) {
          const int2 e = prs[i];
          if ((unsigned)e.x < (unsigned)ld) {
            const float orig = th_s[e.x];
            th_s[e.x] = __int_as_float(e.y) + orig;
            prs[i].y = __float_as_int(orig);
          }
        }
        __syncthreads();
      }
      // restore the measure's tile after the column's last read of it
      auto restore = [&]() {
        if (SP && npairs > 0) {
          const int2* prs = pr_s + size_t(s) * K;
#pragma unroll 1
          for (int i = tid; i < npairs; i += nt) {
            const int2 e = prs[i];
            if ((unsigned)e.x < (unsigned)ld) th_s[e.x] = __int_as_float(e.y);
          }
        }
        if (SP && npairs < 0) fill_tile(m);
      };
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
        if (SP && j > 0) {
          // every commit of column j - 1 is ordered before this point: by the
          // reduction's barrier, or (one warp, where it has none) here
          if (nw == 1) __syncwarp();
          if (tid == 0) finalize(j - 1);
        }
        if (!DIAG) {
          if (SP && npairs != 0) {
            restore();
            __syncthreads();
          }
          refill(j, cnt_nx);
        }
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
          // (f, n) at lam, and (columns of 6 or more groups per thread)
          // min_r |w_r - lam| for the certificate of the Newton step from lam,
          // as in pass 1.  Shorter columns confirm with one more pass, which
          // costs them less than the extra work of every pass (R = 1600:
          // 49.2 against 48.7 us per step; R = 10000 in its first 25 steps:
          // 0.87 against 0.94 ms).
          constexpr bool kCert = NV >= 6;
          const f2_t lam2 = pk(lam, lam);
          f2_t ga = 0ull, gb = 0ull;
          float cnt = 0.f;
          float gap = INFINITY;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const f2_t x0 = sub2(w2[v][0], lam2), x1 = sub2(w2[v][1], lam2);
            if (kCert)
              gap = fminf(gap, fminf(fminf(fabsf(lo(x0)), fabsf(hi(x0))),
                                     fminf(fabsf(lo(x1)), fabsf(hi(x1)))));
            ga = add2(ga, relu2(x0, cnt));
            gb = add2(gb, relu2(x1, cnt));
          }
          const f2_t gs = add2(ga, gb);
          f = lo(gs) + hi(gs);
          reduce3<true>(f, cnt, gap, red, rb, lane, warp, nw);
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
          const float dl = (f - tau) / cnt;
          const float lam_from = lam;
          lam = lam + dl;
          lam_fin = lam;  // used if the pass budget runs out (not expected)
          // No w_r between lam_from and the Newton point: the active set
          // there is this pass's, so the next pass would only confirm lam.
          if (kCert && newton_certified(gap, dl, lam_from)) break;
        }
      }

      // Commit: theta' = pihat - d, Step 3 row sums (+ diagnostics).  With
      // capped columns (Delta_<=(q_s)) the threshold applied is
      // max(lambda, 0): a simplex threshold at or below 0 means the clipped
      // column already carries at most q_s.  lam_floor is -inf otherwise.
      const float lam_use = fmaxf(lam_fin, A.lam_floor);
      const f2_t lf2 = pk(lam_use, lam_use);
      float wc = 0.f, res = 0.f;
      float4* gth = SP ? nullptr : reinterpret_cast<float4*>(A.theta + size_t(col) * ld);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int idx = v * nt + tid;
        if constexpr (SP && !DIAG) {
          // Sparse plans keep pihat only.  fl(w_r - lam) > 0 implies w_r >
          // lam, so a group none of whose rows exceeds lam has no pihat and
          // is skipped without forming it.
          const bool act = fmaxf(fmaxf(lo(w2[v][0]), hi(w2[v][0])),
                                 fmaxf(lo(w2[v][1]), hi(w2[v][1]))) > lam_use;
          if (A.amask) {  // active-set bits of this column (reverse sweep)
            float dummy = 0.f;
            const f2_t p01 = relu2(sub2(w2[v][0], lf2), dummy);
            const f2_t p23 = relu2(sub2(w2[v][1], lf2), dummy);
            unsigned word = ((lo(p01) > 0.f ? 1u : 0u) | (hi(p01) > 0.f ? 2u : 0u) |
                             (lo(p23) > 0.f ? 4u : 0u) | (hi(p23) > 0.f ? 8u : 0u))
                            << (4 * (tid & 7));
            word |= __shfl_xor_sync(0xffffffffu, word, 1);
            word |= __shfl_xor_sync(0xffffffffu, word, 2);
            word |= __shfl_xor_sync(0xffffffffu, word, 4);
            if ((tid & 7) == 0 && 4 * idx < ld) A.amask[size_t(col) * A.mw + idx / 8] = word;
          }
          if (__any_sync(0xffffffffu, act) && act) {
            float dummy = 0.f;
            const f2_t p01 = relu2(sub2(w2[v][0], lf2), dummy);
            const f2_t p23 = relu2(sub2(w2[v][1], lf2), dummy);
            const float pv[4] = {lo(p01), hi(p01), lo(p23), hi(p23)};
            sparse_commit_group(pv, 4 * idx, acc_m, fx, cnt_s + (j & 1),
                                A.sp_pairs + size_t(col) * K, K);
          }
        } else {
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
            if (SP) {
              sparse_commit_group(pv, 4 * idx, acc_m, fx, cnt_s + (j & 1),
                                  A.sp_pairs + size_t(col) * K, K);
            } else {
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (pv[e] > 0.f)
                  atomicAdd(acc_m + 4 * idx + e,
                            (unsigned long long)f32_to_i64_rn(pv[e] * fx));
            }
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
            if (!SP) gth[idx] = ov;
          }
        }
      }
      if (DIAG) {
        reduce3<true>(wc, res, lbmin, red, rb, lane, warp, nw);
        if (tid == 0) {
          A.diag_wc[col] = wc;
          A.diag_res[col] = res;
          A.diag_lb[col] = tau * fminf(lbmin, A.lb_cap);
        }
        // the reduction's barrier ended every read of stage s (and, sparse,
        // of the tile: the restore and its barrier precede the refill)
        if (SP && npairs != 0) {
          restore();
          __syncthreads();
        }
        refill(j, cnt_nx);
      }
      if (tid == 0) A.lam[col] = lam_fin;
      my_passes += np;
      if (any_fail) break;  // uniform: the flag went through a reduction
    }
    if (SP) {  // the last column's count (all commits done at the barrier)
      __syncthreads();
      if (tid == 0 && !any_fail) finalize(ncol - 1);
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

template <int NV, typename CT, bool DIAG, bool SP>
cudaError_t col_op_k(int op, int grid, int threads, size_t smem, cudaStream_t st,
                     const ColArgs* a, int* occ) {
  auto kern = column_kernel<NV, CT, DIAG, SP>;
  if (op == 0) return launch_pdl(kern, dim3(grid), dim3(threads), smem, st, *a);
  if (op == 1)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, threads, smem);
}

// Dispatch over the compile-time (NV, cost type, DIAG) variants of one
// plan layout.
#define MAM_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(8)

template <int NV, typename CT, bool SP>
cudaError_t col_op(int op, bool diag, int grid, int threads, size_t smem,
                   cudaStream_t st, const ColArgs* a, int* occ) {
  return diag ? col_op_k<NV, CT, true, SP>(op, grid, threads, smem, st, a, occ)
              : col_op_k<NV, CT, false, SP>(op, grid, threads, smem, st, a, occ);
}

template <typename CT, bool SP>
cudaError_t col_op_nv(int nv, int op, bool diag, int grid, int threads,
                      size_t smem, cudaStream_t st, const ColArgs* a, int* occ) {
  switch (nv) {
#define MAM_CASE(N) \
  case N:           \
    return col_op<N, CT, SP>(op, diag, grid, threads, smem, st, a, occ);
    MAM_NV_CASES(MAM_CASE)
#undef MAM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <bool SP>
cudaError_t col_op_any(int nv, int dt, int op, bool diag, int grid,
                       int threads, size_t smem, cudaStream_t st,
                       const ColArgs* a, int* occ) {
  switch (dt) {
    case 0: return col_op_nv<float, SP>(nv, op, diag, grid, threads, smem, st, a, occ);
    case 1: return col_op_nv<__nv_bfloat16, SP>(nv, op, diag, grid, threads, smem, st, a, occ);
    case 2: return col_op_nv<__half, SP>(nv, op, diag, grid, threads, smem, st, a, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace mam
