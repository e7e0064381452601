// libmam: differentiation through unrolled MAM iterations and the autotuner.
#include "mam.h"
#include "mam_handle.h"
#include "mam_internal.h"

#include <algorithm>
#include <cstring>
#include <vector>

namespace mam {

struct BackwardState {
  int K = 0;
};

void free_backward(mam_problem* h) {
  delete h->bwd;
  h->bwd = nullptr;
}

}  // namespace mam

using namespace mam;

extern "C" {

mam_status mam_forward_record(mam_problem* h, int32_t K, int32_t ckpt_every) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  (void)K;
  (void)ckpt_every;
  return fail(h, MAM_ERR_UNSUPPORTED, "mam_forward_record is not available yet");
}

mam_status mam_backward(mam_problem* h, const double* grad_p, double* grad_q,
                        double* grad_zeta, double* grad_xi) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  (void)grad_p;
  (void)grad_q;
  (void)grad_zeta;
  (void)grad_xi;
  return fail(h, MAM_ERR_UNSUPPORTED, "mam_backward is not available yet");
}

mam_status mam_autotune(mam_problem* h, int32_t iters, mam_kernel_config* best) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  if (h->failed) return MAM_ERR_STATE;
  if (iters < 1) return fail(h, MAM_ERR_INVALID_ARG, "iters must be >= 1");
  size_t bytes = 0;
  mam_status s = mam_get_state(h, nullptr, &bytes);
  if (s != MAM_OK) return s;
  std::vector<char> snap(bytes);
  if ((s = mam_get_state(h, snap.data(), &bytes)) != MAM_OK) return s;
  const mam_kernel_config start = h->cfg;
  const int ld4 = h->ld / 4;
  std::vector<mam_kernel_config> cands;
  const int nvs[] = {1, 2, 3, 4, 5, 6, 8};
  for (int nv : nvs) {
    int nt = std::max(32, (ld4 + nv - 1) / nv);
    nt = (nt + 31) / 32 * 32;
    for (int extra = 0; extra < 2; ++extra) {
      const int t = nt + 32 * extra;
      if (t > column_max_threads(nv)) continue;
      for (int stg = 2; stg <= 3; ++stg)
        for (int cps : {0, 1, 2}) {
          mam_kernel_config c{t, nv, stg, cps, start.bisect_depth, 0};
          if (check_config(h, c) == MAM_OK) cands.push_back(c);
        }
    }
  }
  for (int nv : {1, 2, 4, 7, 8, 13, 16, 24, 29, 32}) {
    if (32 * nv * 4 < h->ld || 32 * nv * 4 > 2 * h->ld + 512) continue;
    for (int K : {2, 4, 7, 8, 12, 16, 24, 32})
      for (int W : {2, 4, 7, 8, 12, 16})
        for (int cps : {1, 2}) {
          if (W > K) continue;
          mam_kernel_config c{32 * W, nv, K, cps, start.bisect_depth, 1};
          if (check_config(h, c) == MAM_OK) cands.push_back(c);
        }
  }
  h->err.clear();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  mam_kernel_config best_cfg = start;
  for (const auto& c : cands) {
    if (apply_config(h, c) != MAM_OK) {
      h->err.clear();
      continue;
    }
    if ((s = mam_set_state(h, snap.data(), bytes)) != MAM_OK) break;
    if ((s = run_iterations(h, 2, false)) != MAM_OK) break;
    cudaEventRecord(e0, h->stream);
    if ((s = run_iterations(h, iters, false)) != MAM_OK) break;
    cudaEventRecord(e1, h->stream);
    if ((s = sync(h)) != MAM_OK) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best_cfg = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != MAM_OK) return s;
  if ((s = apply_config(h, best_cfg)) != MAM_OK) return s;
  if ((s = mam_set_state(h, snap.data(), bytes)) != MAM_OK) return s;
  if (best) *best = best_cfg;
  return MAM_OK;
}

}  // extern "C"
