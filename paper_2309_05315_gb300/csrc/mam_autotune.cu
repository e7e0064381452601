// libmam: the launch-shape autotuner of the column step.
//
// mam_autotune times candidate kernel configurations on the handle's own
// problem and keeps the fastest.  The state is saved first and restored
// before every candidate and at the end, so tuning changes nothing but the
// configuration.  Two searches:
//  1. launch shapes at the current bisection depth, timed from the current
//     (warm) state: for the one-CTA-per-column kernel the threads x float4
//     groups that cover a column, the copy-pipeline depth and the resident
//     CTAs per SM (which fixes the columns each CTA of the persistent grid
//     takes); for the cluster kernel the CTAs per cluster and their width;
//     for the warp-per-column kernel the width, the ring slots, the
//     warps per CTA and the CTAs per SM;
//  2. the bisection depth of a cold threshold search (Algorithm 1, Step 2:
//     the search brackets lambda in [max w - q_s, max w), bisects, then
//     takes Newton/Michelot steps), on the best shape, timed from the same
//     state with every stored threshold cleared, so that every column takes
//     the cold path on the first of the timed iterations.  A warm search
//     never bisects; the depth only pays on cold starts (the first
//     iterations from theta^0, a restored state without thresholds).
// Any failure restores the starting configuration and state before the
// status is returned.
#include "mam.h"
#include "mam_handle.h"
#include "mam_internal.h"

#include <algorithm>
#include <vector>

namespace mam {
namespace {

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Time `iters` iterations of configuration c from the saved state (after two
// untimed ones); cold: clear every stored threshold first.
mam_status time_config(mam_problem* h, const mam_kernel_config& c,
                       const std::vector<char>& snap, int iters, bool cold, Timer& tm,
                       float* ms) {
  MAM_TRY(apply_config(h, c));
  MAM_TRY(mam_set_state(h, snap.data(), snap.size()));
  if (!cold) MAM_TRY(run_iterations(h, 2, false));
  else  // all-ones bits are a NaN: "no threshold", the cold path of the search
    MAM_CUDA(cudaMemsetAsync(h->lam, 0xFF, sizeof(float) * size_t(h->T), h->stream),
             "threshold reset");
  MAM_CUDA(cudaEventRecord(tm.e0, h->stream), "cudaEventRecord");
  MAM_TRY(run_iterations(h, iters, false));
  MAM_CUDA(cudaEventRecord(tm.e1, h->stream), "cudaEventRecord");
  MAM_TRY(sync(h));
  MAM_CUDA(cudaEventElapsedTime(ms, tm.e0, tm.e1), "cudaEventElapsedTime");
  return MAM_OK;
}

std::vector<mam_kernel_config> shape_candidates(const mam_problem* h, int depth) {
  std::vector<mam_kernel_config> out;
  const int ld4 = h->ld / 4;
  for (int nv : {1, 2, 3, 4, 5, 6, 8}) {
    int nt = std::max(32, (ld4 + nv - 1) / nv);
    nt = (nt + 31) / 32 * 32;
    for (int extra = 0; extra < 2; ++extra) {
      const int t = nt + 32 * extra;
      if (t > column_max_threads(nv)) continue;
      for (int stg = 1; stg <= 3; ++stg)
        for (int cps : {0, 1, 2}) {
          mam_kernel_config c{t, nv, stg, cps, depth, 0};
          if (check_config(h, c) == MAM_OK) out.push_back(c);
        }
    }
  }
  for (int cs : {2, 4, 8, 16})
    for (int t : {128, 256}) {
      mam_kernel_config c{t, cs, 1, 0, depth, 2};
      if (h->ld > kMaxCtaR && check_config(h, c) == MAM_OK) out.push_back(c);
    }
  for (int nv : {1, 2, 4, 7, 8, 13, 16}) {
    if (32 * nv * 4 < h->ld || 32 * nv * 4 > 2 * h->ld + 512) continue;
    for (int K : {2, 4, 7, 8, 12, 16, 24, 32})
      for (int W : {2, 4, 7, 8, 12, 16})
        for (int cps : {1, 2}) {
          if (W > K) continue;
          mam_kernel_config c{32 * W, nv, K, cps, depth, 1};
          if (check_config(h, c) == MAM_OK) out.push_back(c);
        }
  }
  return out;
}

}  // namespace
}  // namespace mam

using namespace mam;

extern "C" mam_status mam_autotune(mam_problem* h, int32_t iters, mam_kernel_config* best) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  if (h->failed) return MAM_ERR_STATE;
  if (iters < 1) return fail(h, MAM_ERR_INVALID_ARG, "iters must be >= 1");
  if (h->sharded)  // every timing run would be a collective with its own outcome per rank
    return fail(h, MAM_ERR_INVALID_ARG, "autotuning is not offered for sharded problems");
  size_t bytes = 0;
  mam_status s = mam_get_state(h, nullptr, &bytes);
  if (s != MAM_OK) return s;
  std::vector<char> snap(bytes);
  if ((s = mam_get_state(h, snap.data(), &bytes)) != MAM_OK) return s;
  const mam_kernel_config start = h->cfg;
  // Restores the starting configuration and state; keeps the first error.
  auto restore = [&](mam_status st) {
    if (h->failed) return st;
    const std::string msg = h->err;
    mam_status r = apply_config(h, start);
    if (r == MAM_OK) r = mam_set_state(h, snap.data(), bytes);
    if (st != MAM_OK) h->err = msg;
    return st != MAM_OK ? st : r;
  };
  Timer tm;
  if (cudaEventCreate(&tm.e0) != cudaSuccess || cudaEventCreate(&tm.e1) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MAM_ERR_CUDA, "cudaEventCreate failed");
  }
  float best_ms = 1e30f;
  mam_kernel_config best_cfg = start;
  for (const auto& c : shape_candidates(h, start.bisect_depth)) {
    float ms = 0.f;
    s = time_config(h, c, snap, iters, false, tm, &ms);
    if (s == MAM_ERR_INVALID_ARG && !h->failed) {  // not resident on an SM: skip it
      h->err.clear();
      continue;
    }
    if (s != MAM_OK) return restore(s);
    if (ms < best_ms) {
      best_ms = ms;
      best_cfg = c;
    }
  }
  // Bisection depth on the best shape, from cold thresholds.
  float best_cold = 1e30f;
  mam_kernel_config depth_cfg = best_cfg;
  for (int depth : {0, 2, 4, 6, 8, 12, 16, 24}) {
    mam_kernel_config c = best_cfg;
    c.bisect_depth = depth;
    float ms = 0.f;
    s = time_config(h, c, snap, iters, true, tm, &ms);
    if (s != MAM_OK) return restore(s);
    if (ms < best_cold) {
      best_cold = ms;
      depth_cfg = c;
    }
  }
  best_cfg = depth_cfg;
  if ((s = apply_config(h, best_cfg)) != MAM_OK) return restore(s);
  if ((s = mam_set_state(h, snap.data(), bytes)) != MAM_OK) return restore(s);
  if (best) *best = best_cfg;
  return MAM_OK;
}
