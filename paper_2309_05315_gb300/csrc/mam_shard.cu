// libmam: Step 1 / Step 3 of Algorithm 1 for a measure-sharded problem.
//
// A rank holds measures m_begin .. m_end - 1 of the problem.  Step 3 and
// Step 1 split around one exchange:
//   phase A (shard_partial_kernel): the new marginals p^(m) of the rank's
//     measures of the index set just processed, p^(m)_r = sum_s pihat_rs -
//     S_m d_r (64-bit fixed point, as in the unsharded averaging kernel),
//     and the rank's partial sum of a_m p^(m) (eq. pr) over ALL its measures,
//     as an integer R-vector;
//   exchange: the caller's callback sums the R integers over the ranks
//     (exact: p is bit for bit the unsharded p);
//   phase B (shard_finish_kernel): p, the shifts (p - p^(m)) / S_m of the
//     rank's measures, and block sums of the distance terms;
//   when t^k is needed (gamma finite) or diagnostics are taken, the block
//     sums are collapsed to four values (shard_collapse_kernel) and summed
//     over the ranks by a second exchange; the column kernel takes t^k from
//     that single global block.
// Every per-(m, r) formula is the one of the unsharded averaging kernel, so
// the marginals and shifts of a measure are the same numbers whichever rank
// holds it.
#include "mam.h"
#include "mam_device.cuh"
#include "mam_handle.h"

#include <cmath>
#include <string>

namespace mam {
namespace {

constexpr int kShardThreads = 128;

__global__ void __launch_bounds__(kShardThreads)
    shard_partial_kernel(const AvgArgs A, long long* part, double* part_hat) {
  pdl_wait();
  pdl_launch_next();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.R) return;
  const int Mloc = A.prob_meas[1];
  const Sched sc = A.sched[draw_index_set(A.draw, *A.iter - 1)];
  const float t_old = float(A.t_used[0]);
  long long ps = 0;
  double phs = 0.0;
  for (int m = 0; m < Mloc; ++m) {
    const size_t o = size_t(m) * A.R + r;
    long long pmv;
    if (A.reduce && m >= sc.meas_begin && m < sc.meas_end) {
      const long long sum_pihat = (long long)A.acc[o];
      A.acc[o] = 0ull;
      // the column kernel subtracted d = float(t delta) from every entry
      const float d_used = __fmul_rn(t_old, A.delta32[size_t(m) * A.ld + r]);
      if (A.d_last) A.d_last[size_t(m) * A.ld + r] = d_used;  // sparse plans
      const long long d_fx = f32_to_i64_rn(d_used * A.fx_f);  // F = 2^e: exact scaling
      if (A.diag) A.phat[o] = double(sum_pihat) * A.fx_inv_scale;
      pmv = sum_pihat - (long long)A.S[m] * d_fx;
      A.pm[o] = pmv;
    } else {
      pmv = A.pm[o];
    }
    ps += mul_q62(pmv, A.a_q[m]);
    if (A.diag) phs += A.a[m] * A.phat[o];
  }
  part[r] = ps;
  if (A.diag) part_hat[r] = phs;
}

// count_dp: this rank adds the |p_new - p_old|^2 terms (one rank does, since
// every rank holds the same p).
__global__ void __launch_bounds__(kShardThreads)
    shard_finish_kernel(const AvgArgs A, const long long* p_sum, const double* phat_sum,
                        int count_dp) {
  __shared__ float se[kShardThreads / 32];
  __shared__ double sr[kShardThreads / 32][2];
  pdl_wait();
  pdl_launch_next();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int Mloc = A.prob_meas[1];
  float e = 0.f;
  double eh = 0.0, dp2 = 0.0;
  if (r < A.R) {
    const long long p_fx = p_sum[r];
    const double ph = A.diag ? phat_sum[r] : 0.0;
    for (int m = 0; m < Mloc; ++m) {
      const size_t o = size_t(m) * A.R + r;
      const long long dfx = p_fx - A.pm[o];  // (p - p^(m)) F, exact
      A.delta32[size_t(m) * A.ld + r] = shift_f32(dfx, A.inv_SFd[m]);
      const float dv = i64_to_f32(dfx) * A.fx_inv_f;
      e = fmaf(dv * dv, A.inv_S[m], e);
      if (A.diag) {
        const double dh = ph - A.phat[o];
        eh += dh * dh * A.inv_Sd[m];
      }
    }
    const double p_new = double(p_fx) * A.fx_inv_scale;
    const double dd = p_new - A.p[r];
    dp2 = count_dp ? dd * dd : 0.0;
    A.p[r] = p_new;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  eh = warp_sum_d(eh);
  dp2 = warp_sum_d(dp2);
  if (lane == 0) {
    se[warp] = e;
    sr[warp][0] = eh;
    sr[warp][1] = dp2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = 0, b1 = 0, b2 = 0;
    for (int i = 0; i < kShardThreads / 32; ++i) {
      b0 += double(se[i]);
      b1 += sr[i][0];
      b2 += sr[i][1];
    }
    double* blk = A.blk + size_t(blockIdx.x) * 4;
    blk[0] = b0;
    blk[1] = b1;
    blk[2] = b2;
    blk[3] = 0.0;
  }
}

// out[0..3] = sums of the rank's block sums (fixed order), before the exchange.
__global__ void __launch_bounds__(32) shard_collapse_kernel(const double* blk, int nblk,
                                                            double* out) {
  pdl_wait();
  double s[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < nblk; i += 32)
    for (int k = 0; k < 4; ++k) s[k] += blk[4 * i + k];
  for (int k = 0; k < 4; ++k) s[k] = warp_sum_d(s[k]);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) out[k] = s[k];
}

}  // namespace

int shard_blocks(const mam_problem* h) { return (h->R + kShardThreads - 1) / kShardThreads; }

// Calls the caller's exchange on a device buffer of the handle.
mam_status shard_exchange(mam_problem* h, void* buf, long long count, int dtype) {
  const int32_t rc = h->allreduce(buf, count, dtype, h->stream, h->ar_user);
  if (rc != 0)
    return fail(h, MAM_ERR_COMM,
                "the exchange callback of the sharded problem returned " + std::to_string(rc));
  return MAM_OK;
}

// Global block sums of the distance terms (t^k, diagnostics) into blk_glob.
mam_status shard_block_sums(mam_problem* h) {
  shard_collapse_kernel<<<1, 32, 0, h->stream>>>(h->blk, shard_blocks(h), h->blk_glob);
  MAM_CUDA(cudaGetLastError(), "sharded collapse kernel");
  return shard_exchange(h, h->blk_glob, 4, MAM_SUM_F64);
}

// Step 3 completion and Step 1 of a sharded problem (reduce = 0: the
// marginals are given, as after the Step 0 row sums).
mam_status shard_average(mam_problem* h, int reduce, bool diag) {
  AvgArgs a = avg_args(h, reduce, diag ? 1 : 0);
  const int nb = shard_blocks(h);
  MAM_CUDA(launch_pdl(shard_partial_kernel, dim3(nb), dim3(kShardThreads), 0, h->stream, a,
                      h->exch_i64, h->exch_f64),
           "sharded partial kernel");
  MAM_TRY(shard_exchange(h, h->exch_i64, h->R, MAM_SUM_I64));
  if (diag) MAM_TRY(shard_exchange(h, h->exch_f64, h->R, MAM_SUM_F64));
  MAM_CUDA(launch_pdl(shard_finish_kernel, dim3(nb), dim3(kShardThreads), 0, h->stream, a,
                      (const long long*)h->exch_i64, (const double*)h->exch_f64,
                      h->m_begin == 0 ? 1 : 0),
           "sharded finish kernel");
  if (diag || !std::isinf(h->gamma[0])) MAM_TRY(shard_block_sums(h));
  return MAM_OK;
}

}  // namespace mam
