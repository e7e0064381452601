// libmam host side: the C ABI of include/mam.h.
//
// Responsibilities: argument validation, pruning of zero-weight columns
// (Section 4.3 "Storage complexity"), the device layout (plans and costs
// column-contiguous with a padded stride), the persistent-grid work
// schedules, the iteration driver (Algorithm 1 replayed from a captured CUDA
// graph), diagnostics, checkpoints and kernel configuration.
#include "mam.h"
#include "mam_internal.h"
#include "mam_support.h"
#include "mam_handle.h"
#include "mam_device.cuh"

#include <algorithm>
#include <limits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace mam;

namespace mam {

thread_local std::string g_last_error;

mam_status fail(mam_problem* h, mam_status code, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (code == MAM_ERR_CUDA || code == MAM_ERR_TIMEOUT || code == MAM_ERR_COMM ||
        code == MAM_ERR_CAPACITY)
      h->failed = true;
  } else {
    g_last_error = msg;
  }
  return code;
}

mam_status cuda_fail(mam_problem* h, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return fail(h, MAM_ERR_OOM, msg);
  }
  return fail(h, MAM_ERR_CUDA, msg);
}

template <typename T>
mam_status upload(mam_problem* h, T* dst, const T* src, size_t count) {
  if (count == 0) return MAM_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(T),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "upload");
  return MAM_OK;
}

size_t cost_elem_size(int dt) { return dt == MAM_F32 ? 4 : 2; }

}  // namespace mam

namespace {

bool finite_all(const double* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

mam_status validate(const mam_desc* d, int idx) {
  const std::string p = "desc[" + std::to_string(idx) + "]: ";
  if (!d) return fail(nullptr, MAM_ERR_INVALID_ARG, p + "null descriptor");
  if (d->M < 1) return fail(nullptr, MAM_ERR_INVALID_ARG, p + "M must be >= 1");
  if (d->R < 1) return fail(nullptr, MAM_ERR_INVALID_ARG, p + "R must be >= 1");
  if (d->R > kMaxR)
    return fail(nullptr, MAM_ERR_INVALID_ARG,
                p + "R must be <= " + std::to_string(kMaxR) +
                    " (a cluster of 16 CTAs holds a whole column in shared memory)");
  if (d->dim < 1 || d->dim > 3)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "dim must be 1..3");
  if (!d->S || !d->q || !d->alpha || !d->xi)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "S, q, alpha and xi are required");
  if (!d->zeta && !d->cost)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "zeta is required without a cost matrix");
  if (!(d->rho > 0) || !std::isfinite(d->rho))
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "rho must be finite and > 0");
  // the kernels use rho and 1/rho in FP32
  if (d->rho < 1e-30 || d->rho > 1e30)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "rho must lie in [1e-30, 1e30]");
  if (std::isnan(d->gamma) || d->gamma < 0)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "gamma must be >= 0 (or INFINITY)");
  if (d->cost_dtype < 0 || d->cost_dtype > 2)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "unknown cost_dtype");
  if (d->theta0_mode < 0 || d->theta0_mode > 1)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "theta0_mode must be 0 or 1");
  if (d->diag_mode < 0 || d->diag_mode > 2)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "unknown diag_mode");
  if (d->n_bundles < 0 || d->n_bundles > d->M)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "n_bundles must be in 0..M");
  if (d->capped != 0 && d->capped != 1)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "capped must be 0 or 1");
  if (!std::isfinite(d->eta) || d->eta < 0 || (!d->capped && d->eta != 0))
    return fail(nullptr, MAM_ERR_INVALID_ARG,
                p + "eta must be finite and >= 0, and 0 unless capped is set");
  if (d->cost_layout != MAM_COST_PER_COLUMN && d->cost_layout != MAM_COST_SHARED &&
      d->cost_layout != MAM_COST_GENERATED)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "unknown cost_layout");
  if (d->cost_layout != MAM_COST_PER_COLUMN) {
    // alpha_m multiplies the unscaled distance inside the kernels, where the
    // padding rows carry an infinite distance
    for (int m = 0; m < d->M; ++m)
      if (!(d->alpha[m] > 0))
        return fail(nullptr, MAM_ERR_INVALID_ARG,
                    p + "the shared and generated cost layouts need alpha_m > 0");
  }
  if (d->plan_layout != MAM_PLAN_DENSE && d->plan_layout != MAM_PLAN_SPARSE)
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "unknown plan_layout");
  if (d->plan_layout == MAM_PLAN_SPARSE) {
    if (d->cost_layout == MAM_COST_GENERATED)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  p + "the sparse plan layout does not run with the generated cost layout");
    if ((d->R + 7) / 8 * 8 > kMaxCtaR)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  p + "the sparse plan layout needs R <= " + std::to_string(kMaxCtaR) +
                      " (one CTA per column)");
    if (d->sparse_slots != 0 &&
        (d->sparse_slots < 2 || d->sparse_slots % 2 || d->sparse_slots > (d->R + 7) / 8 * 8))
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  p + "sparse_slots must be 0 or even in 2..round_up(R, 8)");
  } else if (d->sparse_slots != 0) {
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "sparse_slots needs the sparse plan layout");
  }
  if (d->cost_layout == MAM_COST_GENERATED && (d->cost || !d->zeta))
    return fail(nullptr, MAM_ERR_INVALID_ARG,
                p + "the generated cost layout needs support points and the squared "
                    "Euclidean cost (cost = NULL)");
  long long tot = 0;
  for (int m = 0; m < d->M; ++m) {
    if (d->S[m] < 1)
      return fail(nullptr, MAM_ERR_INVALID_ARG, p + "every S_m must be >= 1");
    tot += d->S[m];
  }
  if (d->cost_layout == MAM_COST_SHARED) {
    // one support for every measure: the same S_m and the same points
    if (d->cost || !d->zeta)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  p + "the shared cost layout needs support points and the squared "
                      "Euclidean cost (cost = NULL)");
    for (int m = 1; m < d->M; ++m) {
      if (d->S[m] != d->S[0])
        return fail(nullptr, MAM_ERR_INVALID_ARG,
                    p + "the shared cost layout needs the same support for every measure");
      const size_t n = size_t(d->S[0]) * d->dim;
      if (std::memcmp(d->zeta, d->zeta + size_t(m) * n, n * sizeof(double)) != 0)
        return fail(nullptr, MAM_ERR_INVALID_ARG,
                    p + "the shared cost layout needs the same support points for every "
                        "measure");
    }
  }
  if (!finite_all(d->q, size_t(tot)) || !finite_all(d->alpha, size_t(d->M)) ||
      !finite_all(d->xi, size_t(d->R) * d->dim) ||
      (d->zeta && !finite_all(d->zeta, size_t(tot) * d->dim)))
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "non-finite input");
  if (d->cost && !finite_all(d->cost, size_t(tot) * d->R))
    return fail(nullptr, MAM_ERR_INVALID_ARG, p + "non-finite cost");
  for (int m = 0; m < d->M; ++m)
    if (d->alpha[m] < 0)
      return fail(nullptr, MAM_ERR_INVALID_ARG, p + "alpha must be >= 0");
  long long off = 0;
  double Q0 = 0;
  for (int m = 0; m < d->M; ++m) {
    double Q = 0;
    int pos = 0;
    for (int s = 0; s < d->S[m]; ++s) {
      const double v = d->q[off + s];
      if (v < 0) return fail(nullptr, MAM_ERR_INVALID_ARG, p + "negative weight");
      if (v > 0) {
        ++pos;
        Q += v;
      }
    }
    if (pos == 0)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  p + "measure " + std::to_string(m) + " has no positive weight");
    if (m == 0) Q0 = Q;
    if (std::isinf(d->gamma) && !d->capped && std::fabs(Q - Q0) > 1e-9 * Q0)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  p + "balanced problems (gamma = inf) need equal total masses; "
                      "use a finite gamma or capped columns for the unbalanced variants");
    off += d->S[m];
  }
  return MAM_OK;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

namespace mam {

// ----------------------------------------------------------- schedules

static void free_sched(mam_problem* h) {
  for (void* p : h->sched_allocs) cudaFree(p);
  h->sched_allocs.clear();
  h->sched_d = nullptr;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
}

static mam_status sched_alloc(mam_problem* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MAM_ERR_OOM, "cudaMalloc failed for the work schedule");
  }
  h->sched_allocs.push_back(*p);
  return MAM_OK;
}

size_t column_smem_bytes(const mam_problem* h, const mam_kernel_config& c) {
  // Each stage holds one column padded to threads * vec * 4 elements.
  // Sparse plans: one theta tile, and per stage the cost and the pair slots.
  const size_t tile = size_t(c.threads) * c.vec * 4;
  const size_t fixed = 4 * sizeof(uint64_t) + 2 * kRedSlots * sizeof(float4) +
                       kRedSlots * sizeof(double) + tile * sizeof(float);
  if (h->sparse)
    return tile * sizeof(float) + size_t(c.stages) * tile * cost_elem_size(h->cost_dtype) +
           size_t(c.stages) * h->sp_k * sizeof(int2) + fixed + 4 * sizeof(int);
  return size_t(c.stages) * tile * (sizeof(float) + cost_elem_size(h->cost_dtype)) + fixed;
}

mam_status check_config(const mam_problem* h, const mam_kernel_config& c) {
  if (h->gen_cost && c.kind != 2)
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                "the generated cost layout runs on the cluster kernel (kind 2)");
  if (h->sparse && (c.kind != 0 || c.stages != 1))
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                "the sparse plan layout runs on the one-CTA-per-column kernel (kind 0) "
                "with 1 stage");
  if (c.kind == 2) {  // one column per thread-block cluster
    if (c.vec != 2 && c.vec != 4 && c.vec != 8 && c.vec != 16)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 2: vec (CTAs per cluster) must be 2, 4, 8 or 16");
    if (c.threads < 64 || c.threads % 32 || c.threads > 256)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 2: threads must be a multiple of 32 in 64..256");
    if (c.stages != 1)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG, "kind 2: stages must be 1");
    if (cluster_kernel_smem(h->ld, c.vec) > 196608)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 2: a CTA's slice of the column exceeds 192 KB; use more CTAs per "
                  "cluster");
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 32 || c.bisect_depth < 0 || c.bisect_depth > 30)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG, "bad ctas_per_sm or bisect_depth");
    return MAM_OK;
  }
  if (c.kind == 1) {  // one warp per column, shared-memory ring
    if (!ring_kernel_has(c.vec))
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 1: vec must be one of 1,2,4,7,8,13,16");
    if (c.threads < 32 || c.threads % 32 || c.threads > ring_kernel_max_threads(c.vec))
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 1: threads must be a multiple of 32 up to " +
                      std::to_string(ring_kernel_max_threads(c.vec)));
    if ((long long)32 * c.vec * 4 < h->ld)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 1: 32 * vec * 4 must cover the padded column (" +
                      std::to_string(h->ld) + ")");
    if (c.stages < c.threads / 32 || c.stages > 64)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 1: stages (ring slots) must be >= warps per CTA and <= 64");
    if (ring_kernel_smem(c.vec, c.stages, int(cost_elem_size(h->cost_dtype))) > 232448)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                  "kind 1: ring does not fit in shared memory; use fewer slots");
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 32 || c.bisect_depth < 0 || c.bisect_depth > 30)
      return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG, "bad ctas_per_sm or bisect_depth");
    return MAM_OK;
  }
  if (c.kind != 0)
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG, "kind must be 0, 1 or 2");
  const int nvs[] = {1, 2, 3, 4, 5, 6, 8};
  if (std::find(std::begin(nvs), std::end(nvs), c.vec) == std::end(nvs))
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                "vec must be one of 1,2,3,4,5,6,8");
  if (c.threads < 32 || c.threads % 32 || c.threads > column_max_threads(c.vec))
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                "threads must be a multiple of 32 within the variant's limit (" +
                    std::to_string(column_max_threads(c.vec)) + ")");
  if ((long long)c.threads * c.vec * 4 < h->ld)
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                "threads * vec * 4 must cover the padded column (" +
                    std::to_string(h->ld) + ")");
  if (c.stages < 1 || c.stages > 4)
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                "stages must be 1..4");
  if (c.ctas_per_sm < 0 || c.ctas_per_sm > 32)
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG, "ctas_per_sm must be 0..32");
  if (c.bisect_depth < 0 || c.bisect_depth > 30)
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG, "bisect_depth must be 0..30");
  if (column_smem_bytes(h, c) > 232448)
    return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG,
                "pipeline does not fit in shared memory; use fewer stages");
  return MAM_OK;
}

// Default launch shape.  Columns of up to 1024 rows go to the
// warp-per-column ring kernel (measured at R = 784 x 256 problems: 0.84 ms
// per step against 0.96 ms for the best CTA shape); longer columns to the
// one-CTA-per-column kernel (R = 1600: 49 us per step with 96 x 5, 52 us
// for the ring kernel; R = 3600: 54 us against 81 us).
mam_kernel_config default_config(const mam_problem* h) {
  const int ld4 = h->ld / 4;
  if (h->ld > kMaxCtaR || h->gen_cost) {
    // Longer than one CTA holds: a cluster per column, the fewest CTAs whose
    // slices stay within 64 KB of w (several resident CTAs per SM), else 16.
    mam_kernel_config c{};
    c.kind = 2;
    c.vec = 16;
    for (int cs : {2, 4, 8, 16})
      if (cluster_kernel_smem(h->ld, cs) <= 65536) {
        c.vec = cs;
        break;
      }
    c.threads = 256;
    c.stages = 1;
    c.ctas_per_sm = 0;
    c.bisect_depth = 4;
    return c;
  }
  if (h->ld <= 1024 && !h->sparse) {
    // The narrowest compiled width that covers the column, up to 12 ring
    // slots (as many as fit in shared memory) and one warp per slot.
    const int need = (ld4 + 31) / 32;
    for (int nv : {1, 2, 4, 7, 8, 13, 16})
      if (nv >= need) {
        mam_kernel_config c{};
        c.kind = 1;
        c.vec = nv;
        const size_t slot = ring_kernel_smem(nv, 1, int(cost_elem_size(h->cost_dtype)));
        const int K = std::min(12, int((232448 - 64) / slot));
        const int W = std::min(K, ring_kernel_max_threads(nv) / 32);
        c.stages = K;
        c.threads = 32 * W;
        c.ctas_per_sm = 2;
        c.bisect_depth = 4;
        if (W >= 1 && check_config(h, c) == MAM_OK) return c;
        break;
      }
  }
  const int nvs[] = {4, 5, 3, 6, 2, 8, 1};
  mam_kernel_config best{};
  double best_score = -1;
  for (int nv : nvs) {
    const int nt = std::max(32, round_up((ld4 + nv - 1) / nv, 32));
    if (nt > column_max_threads(nv)) continue;
    const double util = double(ld4) / (double(nt) * nv);
    // Prefer covering the column with few warps: every threshold-search pass
    // ends in a CTA-wide reduction whose latency grows with the warp count
    // (R = 1600, one stage: 48-51 us per step with 3 warps x 5 groups,
    // 51-54 with 4 x 4, 57-62 with 5 x 3, 59-62 with 7 x 2).
    const double score = util - 0.03 * (nt / 32);
    if (score > best_score + 1e-12) {
      best_score = score;
      best.threads = nt;
      best.vec = nv;
    }
  }
  best.ctas_per_sm = 0;
  // Cold starts (no stored threshold) go straight to Newton from the
  // bracket's lower end: measured on the 100-measure unbalanced workload from
  // a fresh state, the first 5 steps take 8.1 ms with no bisection against
  // 9.3 ms with 4 steps, the next 20 steps 19.5 against 20.0 ms, and the same
  // afterwards (R = 3600: no difference).
  best.bisect_depth = 0;
  best.kind = 0;
  // Two stages overlap the next column's copy with this one's search; one
  // stage frees the shared memory for more resident CTAs, whose columns hide
  // the copy instead (measured at R = 3600, 160 x 6: 54 us per step with one
  // stage at 4 CTAs/SM, 60-64 us with two at 2 CTAs/SM).  Take one stage
  // when it admits more CTAs per SM.
  int occ_by_stages[3] = {0, 0, 0};
  for (int st = 1; st <= (h->sparse ? 1 : 2); ++st) {
    best.stages = st;
    const size_t smem = column_smem_bytes(h, best);
    int occ = 1 << 30;
    for (int dg = 0; dg < 2; ++dg) {
      int o = 0;
      if (smem > 232448 ||
          (h->sparse ? set_column_sparse_smem(best.vec, h->cost_dtype, dg != 0, smem)
                     : set_column_smem(best.vec, h->cost_dtype, dg != 0, smem)) !=
              cudaSuccess ||
          (h->sparse ? column_sparse_occupancy(best.vec, h->cost_dtype, dg != 0, best.threads,
                                               smem, &o)
                     : column_occupancy(best.vec, h->cost_dtype, dg != 0, best.threads, smem,
                                        &o)) != cudaSuccess)
        o = 0;
      occ = std::min(occ, o);
    }
    occ_by_stages[st] = occ;
  }
  best.stages = occ_by_stages[1] > occ_by_stages[2] ? 1 : 2;
  return best;
}

mam_status apply_config(mam_problem* h, const mam_kernel_config& c) {
  MAM_TRY(check_config(h, c));
  if (c.kind == 2) {
    const size_t smem = cluster_kernel_smem(h->ld, c.vec);
    int clusters = 1 << 30;
    const int dt = h->gen_cost ? -1 : h->cost_dtype;  // -1: costs generated in the kernel
    for (int dg = 0; dg < 2; ++dg) {
      MAM_CUDA(set_column_cluster_smem(dt, dg != 0, smem), "cudaFuncSetAttribute");
      int n = 0;
      MAM_CUDA(column_cluster_occupancy(dt, dg != 0, c.vec, c.threads, smem, &n),
               "cluster occupancy");
      clusters = std::min(clusters, n);
    }
    if (clusters < 1)
      return fail(h, MAM_ERR_INVALID_ARG, "cluster configuration cannot be resident");
    if (c.ctas_per_sm > 0)  // at most ctas_per_sm CTAs of this kernel per SM
      clusters = std::min<long long>(clusters, (long long)c.ctas_per_sm * h->num_sms / c.vec);
    long long max_cols = 0;
    for (auto& r : h->index_sets) max_cols = std::max(max_cols, r.second - r.first);
    const long long G = std::max(1LL, std::min<long long>(clusters, max_cols));
    free_sched(h);
    std::vector<Sched> sd(h->index_sets.size());
    for (size_t i = 0; i < sd.size(); ++i) {
      sd[i].col_begin = h->index_sets[i].first;
      sd[i].col_end = h->index_sets[i].second;
      sd[i].meas_begin = h->index_meas[i].first;
      sd[i].meas_end = h->index_meas[i].second;
    }
    void* sp;
    MAM_TRY(sched_alloc(h, &sp, sd.size() * sizeof(Sched)));
    MAM_CUDA(cudaMemcpyAsync(sp, sd.data(), sd.size() * sizeof(Sched), cudaMemcpyHostToDevice,
                             h->stream),
             "sched upload");
    h->sched_d = static_cast<Sched*>(sp);
    h->cfg = c;
    h->grid = int(G * c.vec);
    h->smem = smem;
    MAM_CUDA(cudaStreamSynchronize(h->stream), "schedule upload");
    return MAM_OK;
  }
  const bool wk = c.kind == 1;
  const size_t smem = wk ? ring_kernel_smem(c.vec, c.stages, int(cost_elem_size(h->cost_dtype)))
                         : column_smem_bytes(h, c);
  const bool sparse = h->sparse;
  for (int dg = 0; dg < 2; ++dg)
    MAM_CUDA(wk ? set_column_ring_smem(c.vec, h->cost_dtype, dg != 0, smem)
             : sparse ? set_column_sparse_smem(c.vec, h->cost_dtype, dg != 0, smem)
                  : set_column_smem(c.vec, h->cost_dtype, dg != 0, smem),
             "cudaFuncSetAttribute");
  int occ = 0;
  MAM_CUDA(wk ? column_ring_occupancy(c.vec, h->cost_dtype, true, c.threads, smem, &occ)
           : sparse ? column_sparse_occupancy(c.vec, h->cost_dtype, true, c.threads, smem, &occ)
                : column_occupancy(c.vec, h->cost_dtype, true, c.threads, smem, &occ),
           "occupancy");
  int occ2 = 0;
  MAM_CUDA(wk ? column_ring_occupancy(c.vec, h->cost_dtype, false, c.threads, smem, &occ2)
           : sparse ? column_sparse_occupancy(c.vec, h->cost_dtype, false, c.threads, smem, &occ2)
                : column_occupancy(c.vec, h->cost_dtype, false, c.threads, smem, &occ2),
           "occupancy");
  occ = std::min(occ, occ2);
  if (occ < 1)
    return fail(h, MAM_ERR_INVALID_ARG, "kernel configuration cannot be resident on an SM");
  const int per_sm = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, occ) : occ;
  long long max_cols = 0;
  for (auto& r : h->index_sets) max_cols = std::max(max_cols, r.second - r.first);
  long long G = (long long)per_sm * h->num_sms;
  G = std::max(1LL, std::min(G, max_cols));

  free_sched(h);
  std::vector<Sched> sd(h->index_sets.size());
  for (size_t i = 0; i < sd.size(); ++i) {
    sd[i].col_begin = h->index_sets[i].first;
    sd[i].col_end = h->index_sets[i].second;
    sd[i].meas_begin = h->index_meas[i].first;
    sd[i].meas_end = h->index_meas[i].second;
  }
  void* sp;
  MAM_TRY(sched_alloc(h, &sp, sd.size() * sizeof(Sched)));
  MAM_CUDA(cudaMemcpyAsync(sp, sd.data(), sd.size() * sizeof(Sched), cudaMemcpyHostToDevice, h->stream), "sched upload");
  h->sched_d = static_cast<Sched*>(sp);
  h->cfg = c;
  h->grid = int(G);
  h->smem = smem;
  MAM_CUDA(cudaStreamSynchronize(h->stream), "schedule upload");
  return MAM_OK;
}

// ------------------------------------------------------------ iteration

Draw draw_args(const mam_problem* h) {
  Draw d;
  d.nb = h->nb;
  d.cum = h->bundle_cum_d;
  d.seed = h->seed;
  return d;
}

ColArgs col_args(const mam_problem* h) {
  ColArgs a{};
  a.theta = h->theta;
  a.cost = h->cost;
  a.cost_col = h->cost_col;
  a.cmul = h->cmul;
  a.gen_xi = h->gen_xi;
  a.gen_zeta = h->gen_zeta;
  a.gen_dim = h->dim;
  a.q = h->q;
  a.lam = h->lam;
  a.col_meas = h->col_meas;
  a.col_off = h->col_off_d;
  a.delta32 = h->delta32;
  a.amask = h->amask;
  a.mw = (h->ld + 31) / 32;
  a.blk = h->sharded ? h->blk_glob : h->blk;  // sharded: the global sums, one block
  a.nblk = h->sharded ? 1 : avg_blocks(h);
  a.rho_p = h->rho_d;
  a.gamma_p = h->gamma_d;
  a.t_used = h->t_used;
  a.meas_prob = h->meas_prob;
  a.rho = h->rho_m;
  a.inv_rho = h->irho_m;
  a.acc = h->acc;
  a.fx_scale = float(h->fx_scale);
  a.sched = h->sched_d;
  a.draw = draw_args(h);
  a.iter = h->iter_d;
  a.done = h->done;
  a.diag_wc = h->diag_wc;
  a.diag_lb = h->diag_lb;
  a.diag_res = h->diag_res;
  a.passes = h->passes;
  a.err = h->err_d;
  a.R = h->R;
  a.ld = h->ld;
  a.stages = h->cfg.stages;
  a.bisect_depth = h->cfg.bisect_depth;
  a.lam_floor = h->capped ? 0.f : -INFINITY;
  a.lb_cap = h->capped ? 0.f : INFINITY;
  a.sp_cnt = h->sp_cnt;
  a.sp_pairs = h->sp_pairs;
  a.d_last = h->d_last;
  a.th0 = h->th0;
  a.sp_k = h->sp_k;
  return a;
}

AvgArgs avg_args(const mam_problem* h, int reduce, int diag) {
  AvgArgs a{};
  a.P = h->P;
  a.R = h->R;
  a.prob_meas = h->prob_meas_d;
  a.S = h->S_d;
  a.inv_S = h->invS_f;
  a.inv_SFd = h->invSF_d;
  a.a_q = h->a_q_d;
  a.a = h->a_d;
  a.inv_Sd = h->invS_d;
  a.acc = h->acc;
  a.fx_f = float(h->fx_scale);
  a.fx_inv_f = float(1.0 / h->fx_scale);
  a.fx_inv_scale = 1.0 / h->fx_scale;
  a.sched = h->sched_d;
  a.draw = draw_args(h);
  a.iter = h->iter_d;
  a.t_used = h->t_used;
  a.reduce = reduce;
  a.diag = diag;
  a.pm = h->pm;
  a.p = h->p;
  a.delta32 = h->delta32;
  a.ld = h->ld;
  a.phat = h->phat;
  a.blk = h->blk;
  a.slices = h->avg_slices;
  a.d_last = h->d_last;
  return a;
}

int avg_blocks(const mam_problem* h) {
  const int rows = kAvgThreads / h->avg_slices;
  return (h->R + rows - 1) / rows;
}

// Measure slices of the averaging block: at most 8 measures per thread, and
// enough blocks to give every SM two.
static int choose_avg_slices(const mam_problem* h) {
  int mmax = 1;
  for (int i = 0; i < h->P; ++i) mmax = std::max(mmax, h->prob_meas[i + 1] - h->prob_meas[i]);
  int sl = 1;
  while (sl < 8 && (mmax + sl - 1) / sl > 8) sl *= 2;
  while (sl < 8) {
    const long long nblk = (h->R + kAvgThreads / sl - 1) / (kAvgThreads / sl);
    if (nblk * h->P >= 2LL * std::max(1, h->num_sms)) break;
    sl *= 2;
  }
  return sl;
}

static mam_status prof_event(mam_problem* h, cudaEvent_t* ev) {
  if (h->prof_used >= h->prof_events.size()) {
    cudaEvent_t e;
    MAM_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    h->prof_events.push_back(e);
  }
  *ev = h->prof_events[h->prof_used++];
  return MAM_OK;
}

// The column step of the configured kind with arguments ca.
static cudaError_t launch_column_step(mam_problem* h, const ColArgs& ca, bool diag) {
  return h->cfg.kind == 2
             ? launch_column_cluster(h->gen_cost ? -1 : h->cost_dtype, diag, h->cfg.vec,
                                     h->grid, h->cfg.threads, h->smem, h->stream, ca)
         : h->cfg.kind == 1
             ? launch_column_ring(h->cfg.vec, h->cost_dtype, diag, h->grid, h->cfg.threads,
                                  h->smem, h->stream, ca)
         : h->sparse
             ? launch_column_sparse(h->cfg.vec, h->cost_dtype, diag, h->grid, h->cfg.threads,
                                    h->smem, h->stream, ca)
             : launch_column(h->cfg.vec, h->cost_dtype, diag, h->grid, h->cfg.threads,
                             h->smem, h->stream, ca);
}

mam_status launch_iteration(mam_problem* h, bool diag) {
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (h->profiling) {
    for (auto& e : ev) MAM_TRY(prof_event(h, &e));
    MAM_CUDA(cudaEventRecord(ev[0], h->stream), "cudaEventRecord");
  }
  MAM_CUDA(launch_column_step(h, col_args(h), diag), "column kernel launch");
  if (diag && h->nb > 1) {
    // Lower bound of every measure for the v^k the column step just used
    // (the fused value covers only the drawn bundle).
    MAM_CUDA(launch_lb(h->cost_dtype, h->cost, h->cost_col, h->cmul, h->gen_xi, h->gen_zeta,
                       h->q, h->delta32,
                       h->t_used, h->meas_prob,
                       h->rho_m, h->col_meas, h->T, h->R, h->ld,
                       h->capped ? 0.f : INFINITY, h->diag_lb,
                       h->stream),
             "lower-bound kernel");
  }
  if (h->profiling) MAM_CUDA(cudaEventRecord(ev[1], h->stream), "cudaEventRecord");
  if (h->sharded) {
    MAM_TRY(shard_average(h, 1, diag));
  } else {
    const AvgArgs aa = avg_args(h, 1, diag ? 1 : 0);
    MAM_CUDA(launch_average(aa, avg_blocks(h), h->stream), "average kernel launch");
  }
  if (h->profiling) MAM_CUDA(cudaEventRecord(ev[2], h->stream), "cudaEventRecord");
  return MAM_OK;
}

static mam_status ensure_graph(mam_problem* h) {
  if (h->graph) return MAM_OK;
  cudaGraph_t g = nullptr;
  MAM_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal),
           "cudaStreamBeginCapture");
  mam_status st = MAM_OK;
  for (int i = 0; i < kGraphIters && st == MAM_OK; ++i) st = launch_iteration(h, false);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (st != MAM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return cuda_fail(h, e, "cudaGraphInstantiate");
  }
  return MAM_OK;
}

// Columns of the index sets of column steps k0 .. k0 + n - 1 (the host
// evaluates the same counter-based draw as the kernels).
static long long drawn_columns(const mam_problem* h, long long k0, int n) {
  if (h->nb <= 1) return (long long)n * (h->index_sets[0].second - h->index_sets[0].first);
  Draw d = draw_args(h);
  d.cum = h->bundle_cum.data();
  long long cols = 0;
  for (long long k = k0; k < k0 + n; ++k) {
    const auto& r = h->index_sets[draw_index_set(d, k)];
    cols += r.second - r.first;
  }
  return cols;
}

mam_status run_iterations(mam_problem* h, int n, bool diag_last) {
  if (n <= 0) return MAM_OK;
  {
    const long long cols = drawn_columns(h, h->iter, n);
    h->work_cols += cols;
    h->work_entries += cols * h->R;
  }
  const bool every = h->diag_mode == MAM_DIAG_EVERY;
  const int nd = every ? n : (diag_last ? 1 : 0);
  int plain = n - nd;
  if (h->profiling || h->sharded) {  // per-kernel events / the exchange callback
    // need individual launches
    while (plain-- > 0) MAM_TRY(launch_iteration(h, false));
    plain = 0;
  }
  // The graph is captured on the first call that has plain iterations, so
  // that a later call of kGraphIters or more does not pay the capture.
  if (plain > 0) MAM_TRY(ensure_graph(h));
  while (plain >= kGraphIters) {
    MAM_CUDA(cudaGraphLaunch(h->graph, h->stream), "cudaGraphLaunch");
    plain -= kGraphIters;
  }
  while (plain-- > 0) MAM_TRY(launch_iteration(h, false));
  for (int i = 0; i < nd; ++i) MAM_TRY(launch_iteration(h, true));
  h->iter += n;
  if (nd > 0) h->diag_iter = h->iter;
  return MAM_OK;
}

mam_status check_device_error(mam_problem* h) {
  int e = 0;
  MAM_CUDA(cudaMemcpy(&e, h->err_d, sizeof(int), cudaMemcpyDeviceToHost),
           "error word read");
  if (e == 2)
    return fail(h, MAM_ERR_CAPACITY,
                "sparse plan layout: a column's active set exceeded sparse_slots = " +
                    std::to_string(h->sp_k) + " (the iterate is invalid)");
  if (e != 0)
    return fail(h, MAM_ERR_TIMEOUT,
                "a device-side wait exceeded its bound (the iterate is invalid)");
  return MAM_OK;
}

mam_status sync(mam_problem* h) {
  MAM_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  return check_device_error(h);
}

// ------------------------------------------------------------ creation

mam_status reset_state(mam_problem* h) {
  if (h->sparse) {
    MAM_CUDA(launch_init_sparse(h->sp_cnt, h->th0, h->lam, h->q64, h->T, h->R,
                                h->theta0_mode, h->stream),
             "init kernel");
    MAM_CUDA(cudaMemsetAsync(h->d_last, 0, sizeof(float) * size_t(h->Mtot) * h->ld, h->stream),
             "memset");
  } else {
    MAM_CUDA(launch_init_theta(h->theta, h->lam, h->q64, h->T, h->R, h->ld,
                               h->theta0_mode, h->stream),
             "init kernel");
  }
  MAM_CUDA(launch_rowsum_theta0(h->q64, h->col_off_d, h->Mtot, h->R, h->theta0_mode,
                                h->fx_scale, h->pm, h->stream),
           "rowsum kernel");
  const size_t MR = size_t(h->Mtot) * h->R;
  MAM_CUDA(cudaMemsetAsync(h->p, 0, sizeof(double) * h->P * h->R, h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->acc, 0, sizeof(unsigned long long) * MR, h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->phat, 0, sizeof(double) * MR, h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->delta32, 0, sizeof(float) * size_t(h->Mtot) * h->ld, h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->diag_wc, 0, sizeof(float) * h->T, h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->diag_lb, 0, sizeof(float) * h->T, h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->diag_res, 0, sizeof(float) * h->T, h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->iter_d, 0, sizeof(long long), h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->done, 0, sizeof(unsigned), h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->blk, 0, sizeof(double) * 4 * h->P * avg_blocks(h), h->stream), "memset");
  std::vector<double> ones(h->P, 1.0);
  MAM_TRY(upload(h, h->t_used, ones.data(), ones.size()));
  if (h->sharded) {
    MAM_CUDA(cudaMemsetAsync(h->blk_glob, 0, sizeof(double) * 4, h->stream), "memset");
    MAM_TRY(shard_average(h, 0, false));
  } else {
    const AvgArgs aa = avg_args(h, 0, 0);
    MAM_CUDA(launch_average(aa, avg_blocks(h), h->stream), "average kernel launch");
  }
  h->iter = 0;
  h->diag_iter = -1;
  return sync(h);
}

// Randomized index sets (Remark 2): a column's first visit can come many
// iterations after creation, and without a stored threshold its projection
// starts with the cold search (bracket, bisection, Newton passes).  Prime the
// thresholds: project every index set once from theta^0 (exact projections
// of w = theta^0 + 2 t d^0 - c / rho), keep only the thresholds, and reset
// everything else to the state of theta^0.  The iterates are those of
// Algorithm 1 from theta^0 either way; only the starting points of the
// threshold searches change.  One index set needs no priming: its first
// iteration is that pass.
mam_status prime_thresholds(mam_problem* h) {
  if (h->nb <= 1 || h->index_sets.size() < 2) return MAM_OK;
  for (size_t i = 0; i < h->index_sets.size(); ++i) {
    ColArgs a = col_args(h);
    a.sched = h->sched_d + i;  // with one draw, index set 0 of this schedule
    a.draw.nb = 1;
    a.amask = nullptr;
    MAM_CUDA(launch_column_step(h, a, false), "threshold priming");
  }
  // The passes changed the plans, the row-sum accumulators, the counters
  // and t (not the marginals, p or the shifts, which only the averaging
  // writes): restore those to the state of theta^0 and keep the thresholds.
  if (h->sparse) {
    MAM_CUDA(launch_init_sparse(h->sp_cnt, h->th0, nullptr, h->q64, h->T, h->R,
                                h->theta0_mode, h->stream),
             "init kernel");
  } else {
    MAM_CUDA(launch_init_theta(h->theta, nullptr, h->q64, h->T, h->R, h->ld, h->theta0_mode,
                               h->stream),
             "init kernel");
  }
  MAM_CUDA(cudaMemsetAsync(h->acc, 0, sizeof(unsigned long long) * size_t(h->Mtot) * h->R,
                           h->stream),
           "memset");
  MAM_CUDA(cudaMemsetAsync(h->iter_d, 0, sizeof(long long), h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->done, 0, sizeof(unsigned), h->stream), "memset");
  MAM_CUDA(cudaMemsetAsync(h->passes, 0, sizeof(unsigned long long), h->stream), "memset");
  std::vector<double> ones(h->P, 1.0);
  MAM_TRY(upload(h, h->t_used, ones.data(), ones.size()));
  return sync(h);
}

// Generated costs: FP32 copies of the points, the barycenter points as
// coordinate planes [P][3][ld] (zero past dim and past R) and (x, y, z, eta)
// per kept column.
mam_status upload_gen_points(mam_problem* h) {
  std::vector<float> xi(size_t(h->P) * 3 * h->ld, 0.f);
  std::vector<float4> ze(size_t(h->T));
  for (int p = 0; p < h->P; ++p)
    for (int r = 0; r < h->R; ++r)
      for (int k = 0; k < h->dim; ++k)
        xi[(size_t(p) * 3 + k) * h->ld + r] =
            float(h->xi_h[(size_t(p) * h->R + r) * h->dim + k]);
  for (long long c = 0; c < h->T; ++c) {
    float v[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < h->dim; ++k) v[k] = float(h->zeta_kept[size_t(c) * h->dim + k]);
    ze[c] = make_float4(v[0], v[1], v[2], float(h->eta_h[h->meas_prob_h[h->col_meas_h[c]]]));
  }
  MAM_TRY(upload(h, h->gen_xi, xi.data(), xi.size()));
  return upload(h, h->gen_zeta, ze.data(), ze.size());
}

// Distinct values of one coordinate, keyed by bit pattern, in order of first
// appearance (open addressing); false once there are more than `limit`.
static bool distinct_values(const double* v, size_t n, size_t stride, int limit,
                            std::vector<double>& vals, std::vector<int>& idx) {
  size_t cap = 64;
  while (cap < 2 * size_t(limit)) cap <<= 1;
  std::vector<uint64_t> key(cap);
  std::vector<int> slot(cap, -1);
  vals.clear();
  idx.resize(n);
  for (size_t i = 0; i < n; ++i) {
    uint64_t b;
    std::memcpy(&b, v + i * stride, sizeof b);
    size_t h = size_t((b ^ (b >> 29)) * 0x9E3779B97F4A7C15ull) & (cap - 1);
    while (slot[h] >= 0 && key[h] != b) h = (h + 1) & (cap - 1);
    if (slot[h] < 0) {
      if (int(vals.size()) == limit) return false;
      slot[h] = int(vals.size());
      key[h] = b;
      vals.push_back(v[i * stride]);
    }
    idx[i] = slot[h];
  }
  return true;
}

// Squared-Euclidean costs of columns c0 .. c0 + ncols - 1 through the
// coordinate tables (CostTab) when every coordinate of xi and of the
// columns' points takes few distinct values (pixel grids); *done stays false
// otherwise and the direct kernel runs.  The tables hold the direct
// formula's per-coordinate squares, so the costs are the same bit for bit.
static mam_status build_cost_tabulated(mam_problem* h, const double* xi,
                                       const std::vector<double>& zk, long long c0,
                                       long long ncols, const long long* cols_d, bool* done) {
  *done = false;
  const int dim = h->dim, R = h->R;
  constexpr int kLimit = 4096;  // distinct values per coordinate
  std::vector<double> ux[3], uz[3];
  std::vector<int> ixk[3], izk[3];
  long long entries = 0;
  for (int k = 0; k < dim; ++k) {
    if (!distinct_values(xi + k, size_t(R), size_t(dim), kLimit, ux[k], ixk[k]) ||
        !distinct_values(zk.data() + k, size_t(ncols), size_t(dim), kLimit, uz[k], izk[k]))
      return MAM_OK;
    entries += (long long)ux[k].size() * (long long)uz[k].size();
  }
  // worth it only when the tables are much smaller than the costs
  if (entries > (1LL << 22) || entries * 16 > ncols * (long long)R) return MAM_OK;
  CostTab tb{};
  tb.dim = dim;
  std::vector<int> ix(size_t(dim) * R), iz(size_t(ncols) * dim);
  std::vector<double> vals;
  long long off = 0;
  for (int k = 0; k < dim; ++k) {
    tb.off[k] = off;
    tb.nx[k] = int(ux[k].size());
    off += (long long)ux[k].size() * (long long)uz[k].size();
    std::copy(ixk[k].begin(), ixk[k].end(), ix.begin() + size_t(k) * R);
    for (long long c = 0; c < ncols; ++c) iz[size_t(c) * dim + k] = izk[k][c];
  }
  // one device block: [tables][value lists][ix][iz]
  std::vector<size_t> vbeg(dim);
  for (int k = 0; k < dim; ++k) {
    vbeg[k] = vals.size();
    vals.insert(vals.end(), uz[k].begin(), uz[k].end());
    vals.insert(vals.end(), ux[k].begin(), ux[k].end());
  }
  const size_t b_tab = sizeof(double) * size_t(entries);
  const size_t b_val = sizeof(double) * vals.size();
  const size_t b_ix = sizeof(int) * ix.size(), b_iz = sizeof(int) * iz.size();
  char* dev = nullptr;
  MAM_CUDA(cudaMalloc(&dev, b_tab + b_val + b_ix + b_iz), "cudaMalloc (cost tables)");
  double* tab = reinterpret_cast<double*>(dev);
  double* dval = reinterpret_cast<double*>(dev + b_tab);
  int* dix = reinterpret_cast<int*>(dev + b_tab + b_val);
  int* diz = reinterpret_cast<int*>(dev + b_tab + b_val + b_ix);
  cudaError_t e = cudaMemcpyAsync(dval, vals.data(), b_val, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dix, ix.data(), b_ix, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(diz, iz.data(), b_iz, cudaMemcpyHostToDevice, h->stream);
  for (int k = 0; k < dim && e == cudaSuccess; ++k)
    e = launch_sqdiff_table(tab + tb.off[k], dval + vbeg[k], int(uz[k].size()),
                            dval + vbeg[k] + uz[k].size(), int(ux[k].size()), h->stream);
  if (e == cudaSuccess)
    e = launch_build_cost_tab(h->cost_dtype, h->cost, tab, tb, dix, diz, h->col_meas,
                              h->alpha_d, h->eta_d, c0, ncols, R, h->ld, h->stream, cols_d);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // (pageable sources, then free)
  cudaFree(dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "tabulated cost kernel");
  *done = true;
  return MAM_OK;
}

// Columns c0 .. c1 - 1 whose cost columns repeat an earlier one: equal point
// (bit for bit), alpha_m and eta give the same column.  reps: the columns to
// build (global indices, first of each class); dst_src: (column, its class's
// first column) for the others.  A point is keyed by the indices of its
// coordinates among their distinct values, so this applies where those are
// few (pixel grids); elsewhere every column is built.
static void repeated_cost_columns(const std::vector<double>& zk, int dim, long long c0,
                                  long long c1, const std::vector<int>& col_meas,
                                  const std::vector<double>& alpha_m,
                                  const std::vector<double>& eta_m, std::vector<long long>& reps,
                                  std::vector<long long>& dst_src) {
  const long long n = c1 - c0;
  reps.clear();
  dst_src.clear();
  auto all = [&]() {
    reps.resize(size_t(n));
    for (long long j = 0; j < n; ++j) reps[j] = c0 + j;
    dst_src.clear();
  };
  std::vector<double> vals;
  std::vector<int> idx[3];
  long long nz[3] = {1, 1, 1};
  long long key_span = 1;
  for (int k = 0; k < dim; ++k) {
    if (!distinct_values(zk.data() + k, size_t(n), size_t(dim), 4096, vals, idx[k])) return all();
    nz[k] = (long long)vals.size();
    key_span *= nz[k];
  }
  // (alpha_m, eta) classes of the measures of these columns
  std::vector<int> mcls(alpha_m.size(), -1);
  std::vector<std::pair<uint64_t, uint64_t>> cls;
  for (long long j = 0; j < n; ++j) {
    const int m = col_meas[c0 + j];
    if (mcls[m] >= 0) continue;
    uint64_t a, b;
    std::memcpy(&a, &alpha_m[m], sizeof a);
    std::memcpy(&b, &eta_m[m], sizeof b);
    int c = 0;
    while (c < int(cls.size()) && !(cls[c].first == a && cls[c].second == b)) ++c;
    if (c == int(cls.size())) {
      if (cls.size() == 64) return all();
      cls.push_back({a, b});
    }
    mcls[m] = c;
  }
  if (key_span * (long long)cls.size() > (1LL << 24)) return all();
  std::vector<int> first(size_t(key_span * (long long)cls.size()), -1);
  for (long long j = 0; j < n; ++j) {
    long long key = mcls[col_meas[c0 + j]];
    for (int k = 0; k < dim; ++k) key = key * nz[k] + idx[k][j];
    int& f = first[size_t(key)];
    if (f < 0) {
      f = int(j);
      reps.push_back(c0 + j);
    } else {
      dst_src.push_back(c0 + j);
      dst_src.push_back(c0 + f);
    }
  }
}

static mam_status create_impl(int n, const mam_desc* descs, mam_problem** out,
                              const mam_shard* shard = nullptr) {
  if (!out) return fail(nullptr, MAM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !descs) return fail(nullptr, MAM_ERR_INVALID_ARG, "need at least one problem");
  for (int i = 0; i < n; ++i) MAM_TRY(validate(&descs[i], i));
  if (shard) {
    if (n != 1) return fail(nullptr, MAM_ERR_INVALID_ARG, "a sharded problem is a single problem");
    if (!shard->allreduce)
      return fail(nullptr, MAM_ERR_INVALID_ARG, "sharded problem: allreduce callback is NULL");
    if (shard->m_begin < 0 || shard->m_end > descs[0].M || shard->m_end <= shard->m_begin)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  "sharded problem: need 0 <= m_begin < m_end <= M");
  }
  for (int i = 1; i < n; ++i) {
    if (descs[i].R != descs[0].R || descs[i].dim != descs[0].dim ||
        descs[i].cost_dtype != descs[0].cost_dtype ||
        descs[i].diag_mode != descs[0].diag_mode ||
        descs[i].theta0_mode != descs[0].theta0_mode || descs[i].capped != descs[0].capped)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  "batched problems must share R, dim, cost_dtype, diag_mode, theta0_mode "
                  "and capped");
    if (descs[i].cost_layout != descs[0].cost_layout)
      return fail(nullptr, MAM_ERR_INVALID_ARG, "batched problems must share cost_layout");
    if (descs[i].plan_layout != descs[0].plan_layout ||
        descs[i].sparse_slots != descs[0].sparse_slots)
      return fail(nullptr, MAM_ERR_INVALID_ARG,
                  "batched problems must share plan_layout and sparse_slots");
    if (descs[0].cost_layout == MAM_COST_SHARED) {
      const size_t nx = size_t(descs[0].R) * descs[0].dim;
      const size_t nz = size_t(descs[0].S[0]) * descs[0].dim;
      if (descs[i].S[0] != descs[0].S[0] || descs[i].eta != descs[0].eta ||
          std::memcmp(descs[i].xi, descs[0].xi, nx * sizeof(double)) != 0 ||
          std::memcmp(descs[i].zeta, descs[0].zeta, nz * sizeof(double)) != 0)
        return fail(nullptr, MAM_ERR_INVALID_ARG,
                    "a batch with the shared cost layout needs the same support points, "
                    "xi and eta in every problem");
    }
  }
  if (n > 1)
    for (int i = 0; i < n; ++i)
      if (descs[i].n_bundles > 1)
        return fail(nullptr, MAM_ERR_INVALID_ARG,
                    "batched problems must be deterministic (n_bundles <= 1)");

  mam_problem* h = new mam_problem();
  // measures kept by this handle: all (every problem of a batch), or a
  // sharded rank's range of the single problem
  const int mb = shard ? shard->m_begin : 0;
  const int me = shard ? shard->m_end : std::numeric_limits<int>::max();
  if (shard) {
    h->sharded = true;
    h->m_begin = mb;
    h->M_global = descs[0].M;
    h->allreduce = shard->allreduce;
    h->ar_user = shard->user;
  }
  auto bail = [&](mam_status s) {
    if (h->failed || s != MAM_OK) g_last_error = h->err;
    mam_destroy(h);
    return s;
  };
  const mam_desc& d0 = descs[0];
  h->P = n;
  h->R = d0.R;
  h->dim = d0.dim;
  h->ld = round_up(d0.R, 8);
  h->cost_dtype = d0.cost_dtype;
  h->capped = d0.capped != 0;
  h->theta0_mode = d0.theta0_mode;
  h->diag_mode = d0.diag_mode;
  h->shared_cost = d0.cost_layout == MAM_COST_SHARED;
  h->gen_cost = d0.cost_layout == MAM_COST_GENERATED;
  h->sparse = d0.plan_layout == MAM_PLAN_SPARSE;
  h->sp_k = !h->sparse ? 0 : d0.sparse_slots > 0 ? d0.sparse_slots : std::min(h->ld, 1024);
  h->n_sup = h->shared_cost ? d0.S[0] : 0;
  h->nb = (n == 1 && d0.n_bundles > 1) ? d0.n_bundles : 1;
  h->seed = d0.seed;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "device query"));
  if (d0.stream) {
    h->stream = static_cast<cudaStream_t>(d0.stream);
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaStreamCreate"));
    h->own_stream = true;
  }

  // Host layout: pruning (Section 4.3) and the per-measure constants.
  h->prob_meas.push_back(0);
  h->prob_cols.push_back(0);
  h->col_off.push_back(0);
  h->unpruned_off.push_back(0);
  std::vector<double> q64;
  std::vector<float> q32;
  std::vector<int> col_meas;
  std::vector<double> alpha_m, eta_m;
  long long uoff_global = 0;
  double qmax = 0;  // largest kept mass over every measure (all ranks' too)
  for (int i = 0; i < n; ++i) {
    const mam_desc& d = descs[i];
    double inv_sum = 0;
    std::vector<int> Sp(d.M);
    long long uoff = 0;
    for (int m = 0; m < d.M; ++m) {
      int cnt = 0;
      double Q = 0;
      for (int s = 0; s < d.S[m]; ++s) {
        cnt += d.q[uoff + s] > 0;
        if (d.q[uoff + s] > 0) Q += d.q[uoff + s];
      }
      Sp[m] = cnt;
      inv_sum += 1.0 / cnt;
      qmax = std::max(qmax, Q);
      uoff += d.S[m];
    }
    uoff = 0;
    double Qa = 0;
    int local = 0;
    for (int m = 0; m < d.M; ++m) {
      if (m < mb || m >= me) {  // another rank's measure: only its mass enters Qa
        double Q = 0;
        for (int s = 0; s < d.S[m]; ++s)
          if (d.q[uoff + s] > 0) Q += d.q[uoff + s];
        Qa += (1.0 / Sp[m]) / inv_sum * Q;
        uoff += d.S[m];
        continue;
      }
      const int gm = h->Mtot + local++;
      h->S.push_back(Sp[m]);
      h->S_unpruned.push_back(d.S[m]);
      const double am = (1.0 / Sp[m]) / inv_sum;
      h->a.push_back(am);
      h->meas_prob_h.push_back(i);
      alpha_m.push_back(d.alpha[m]);
      eta_m.push_back(d.eta);
      double Q = 0;
      for (int s = 0; s < d.S[m]; ++s) {
        const double v = d.q[uoff + s];
        if (v > 0) {
          q64.push_back(v);
          q32.push_back(float(v));
          col_meas.push_back(gm);
          h->keep.push_back(uoff_global + uoff + s);
          Q += v;
        }
      }
      Qa += am * Q;
      h->alpha_h.push_back(d.alpha[m]);
      h->Q_h.push_back(Q);
      h->col_off.push_back(h->col_off.back() + Sp[m]);
      h->unpruned_off.push_back(h->unpruned_off.back() + d.S[m]);
      uoff += d.S[m];
    }
    uoff_global += uoff;
    h->Mtot += local;
    h->prob_meas.push_back(h->Mtot);
    h->prob_cols.push_back(h->col_off.back());
    h->rho.push_back(d.rho);
    h->eta_h.push_back(d.eta);
    h->gamma.push_back(d.gamma);
    h->Qa.push_back(Qa);
  }
  h->T = h->col_off.back();
  if (h->T >= (1LL << 31) - 1)
    return bail(fail(h, MAM_ERR_INVALID_ARG, "too many kept columns (>= 2^31)"));

  // Index sets: all columns, or the bundles of Remark 2 (contiguous measures
  // of the whole problem; a sharded rank keeps the part it owns, possibly
  // none).
  if (h->nb > 1) {
    const int M = d0.M;
    double tot = 0;
    std::vector<double> beta(h->nb);
    for (int b = 0; b < h->nb; ++b) {
      const int m0 = int((long long)b * M / h->nb), m1 = int((long long)(b + 1) * M / h->nb);
      double s = 0;
      for (int m = m0; m < m1; ++m) s += d0.alpha[m];
      beta[b] = s;
      tot += s;
      const int l0 = std::min(std::max(m0, mb), std::min(me, M)) - mb;
      const int l1 = std::min(std::max(m1, mb), std::min(me, M)) - mb;
      h->index_sets.push_back({h->col_off[l0], h->col_off[l1]});
      h->index_meas.push_back({l0, l1});
    }
    if (!(tot > 0))
      return bail(fail(h, MAM_ERR_INVALID_ARG, "randomized MAM needs sum(alpha) > 0"));
    double acc = 0;
    for (int b = 0; b < h->nb; ++b) {
      acc += beta[b] / tot;
      h->bundle_cum.push_back(acc);
    }
  } else {
    h->index_sets.push_back({0, h->T});
    h->index_meas.push_back({0, h->Mtot});
  }
  // Fixed-point scale of the row-sum accumulators: every sum of pi-hat over
  // a row is at most the measure's mass, so Qmax * 2^e <= 2^61 cannot
  // overflow the signed 64-bit accumulators.
  {
    // 2 bits of headroom over the largest mass: the marginals p^(m) (row
    // sums of theta = pihat - d) and p are held in the same fixed point.
    int e2 = 59 - int(std::ceil(std::log2(qmax * 1.0001)));
    e2 = std::max(0, std::min(100, e2));
    h->fx_scale = std::ldexp(1.0, e2);
  }

  // Device buffers.
  const size_t Tld = size_t(h->T) * h->ld;
  const size_t MR = size_t(h->Mtot) * h->R;
  mam_status s = MAM_OK;
#define ALLOC(ptr, count, what) \
  if ((s = dalloc(h, &(ptr), (count), (what))) != MAM_OK) return bail(s)
  if (h->sparse) {
    ALLOC(h->sp_cnt, size_t(h->T), "sparse plan counts");
    ALLOC(h->sp_pairs, size_t(h->T) * h->sp_k, "sparse plan pairs");
    ALLOC(h->d_last, size_t(h->Mtot) * h->ld, "shifts of the last visits");
    ALLOC(h->th0, size_t(h->T), "theta^0 values");
  } else {
    ALLOC(h->theta, Tld, "plans theta");
  }
  void* costp = nullptr;
  if (!h->gen_cost) {
    const size_t ncost = h->shared_cost ? size_t(h->n_sup) * h->ld : Tld;
    char* cp = nullptr;
    ALLOC(cp, ncost * cost_elem_size(h->cost_dtype), "costs");
    costp = cp;
  } else {
    ALLOC(h->gen_xi, size_t(h->P) * 3 * h->ld, "points (fp32)");
    ALLOC(h->gen_zeta, size_t(h->T), "support points (fp32)");
  }
  h->cost = costp;
  ALLOC(h->q, size_t(h->T), "weights");
  ALLOC(h->q64, size_t(h->T), "weights (fp64)");
  ALLOC(h->lam, size_t(h->T), "thresholds");
  ALLOC(h->pm, MR, "marginals");
  ALLOC(h->acc, MR, "row-sum accumulators");
  ALLOC(h->delta32, size_t(h->Mtot) * h->ld, "shifts (fp32)");
  ALLOC(h->phat, MR, "pi-hat marginals");
  ALLOC(h->p, size_t(h->P) * h->R, "barycenters");
  ALLOC(h->t_used, size_t(h->P), "t");
  h->avg_slices = choose_avg_slices(h);
  ALLOC(h->blk, size_t(h->P) * avg_blocks(h) * 4, "block sums");
  ALLOC(h->done, 1, "arrival counter");
  ALLOC(h->diag_wc, size_t(h->T), "diagnostics");
  ALLOC(h->diag_lb, size_t(h->T), "diagnostics");
  ALLOC(h->diag_res, size_t(h->T), "diagnostics");
  ALLOC(h->diag_out, size_t(h->P) * 3, "diagnostic sums");
  ALLOC(h->passes, 1, "pass counter");
  ALLOC(h->err_d, 1, "error word");
  ALLOC(h->meas_prob, size_t(h->Mtot), "measure table");
  ALLOC(h->rho_m, size_t(h->Mtot), "rho table");
  ALLOC(h->irho_m, size_t(h->Mtot), "rho table");
  ALLOC(h->a_d, size_t(h->Mtot), "weights a");
  ALLOC(h->alpha_d, size_t(h->Mtot), "alpha");
  ALLOC(h->eta_d, size_t(h->Mtot), "eta");
  ALLOC(h->S_d, size_t(h->Mtot), "sizes");
  ALLOC(h->Sd_d, size_t(h->Mtot), "sizes");
  ALLOC(h->invS_d, size_t(h->Mtot), "sizes");
  ALLOC(h->invS_f, size_t(h->Mtot), "sizes");
  ALLOC(h->invSF_d, size_t(h->Mtot), "sizes");
  ALLOC(h->a_q_d, size_t(h->Mtot), "weights a");
  ALLOC(h->prob_meas_d, size_t(h->P) + 1, "problem table");
  ALLOC(h->rho_d, size_t(h->P), "rho");
  ALLOC(h->gamma_d, size_t(h->P), "gamma");
  ALLOC(h->col_off_d, size_t(h->Mtot) + 1, "column offsets");
  ALLOC(h->prob_cols_d, size_t(h->P) + 1, "problem columns");
  ALLOC(h->col_meas, size_t(h->T), "column table");
  ALLOC(h->bundle_cum_d, std::max<size_t>(1, h->bundle_cum.size()), "bundle table");
  ALLOC(h->iter_d, 1, "iteration counter");
  ALLOC(h->cmul, size_t(h->Mtot), "cost factors");
  if (h->shared_cost) {
    ALLOC(h->cost_col, size_t(h->T), "cost columns");
    ALLOC(h->sup_zeta_d, size_t(h->n_sup) * h->dim, "support points");
    ALLOC(h->sup_meas_d, size_t(h->n_sup), "support table");
    ALLOC(h->sup_alpha_d, 1, "support weight");
    ALLOC(h->sup_eta_d, 1, "support eta");
  }
  if (h->sharded) {
    ALLOC(h->exch_i64, size_t(h->R), "exchange buffer");
    ALLOC(h->exch_f64, size_t(h->R), "exchange buffer");
    ALLOC(h->blk_glob, 4, "global block sums");
  }
#undef ALLOC

  // Shared cost: the stored matrix is C, so alpha_m goes into the factor of
  // c in w = theta + 2 d - c / rho (and into the diagnostics' cost factor).
  std::vector<float> rho_m(h->Mtot), irho_m(h->Mtot), cmul(h->Mtot, 1.f);
  for (int m = 0; m < h->Mtot; ++m) {
    rho_m[m] = float(h->rho[h->meas_prob_h[m]]);
    const double a = (h->shared_cost || h->gen_cost) ? alpha_m[m] : 1.0;
    irho_m[m] = float(a / h->rho[h->meas_prob_h[m]]);
    cmul[m] = float(a);
  }
  if ((s = upload(h, h->cmul, cmul.data(), cmul.size())) != MAM_OK) return bail(s);
  if (h->shared_cost) {
    // Column of C of each plan column: its index in the measure's unpruned
    // support.  keep[] counts from the start of the descriptions, so the
    // measure's unpruned start there is subtracted.
    std::vector<int> cc(h->T);
    {
      long long start = 0;  // unpruned offset of measure m in the description
      int mi = 0;
      for (int i = 0; i < n; ++i) {
        const mam_desc& d = descs[i];
        for (int m = 0; m < d.M; ++m) {
          if (!(m < mb || m >= me)) {
            for (long long c = h->col_off[mi]; c < h->col_off[mi + 1]; ++c)
              cc[c] = int(h->keep[c] - start);
            ++mi;
          }
          start += d.S[m];
        }
      }
    }
    if ((s = upload(h, h->cost_col, cc.data(), cc.size())) != MAM_OK) return bail(s);
    std::vector<int> zeros(h->n_sup, 0);
    const double one = 1.0, eta0 = d0.eta;
    if ((s = upload(h, h->sup_meas_d, zeros.data(), zeros.size())) != MAM_OK) return bail(s);
    if ((s = upload(h, h->sup_alpha_d, &one, 1)) != MAM_OK) return bail(s);
    if ((s = upload(h, h->sup_eta_d, &eta0, 1)) != MAM_OK) return bail(s);
    if ((s = upload(h, h->sup_zeta_d, d0.zeta, size_t(h->n_sup) * h->dim)) != MAM_OK)
      return bail(s);
  }
  if ((s = upload(h, h->q, q32.data(), q32.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->q64, q64.data(), q64.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->meas_prob, h->meas_prob_h.data(), h->meas_prob_h.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->rho_m, rho_m.data(), rho_m.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->irho_m, irho_m.data(), irho_m.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->a_d, h->a.data(), h->a.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->alpha_d, alpha_m.data(), alpha_m.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->eta_d, eta_m.data(), eta_m.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->S_d, h->S.data(), h->S.size())) != MAM_OK) return bail(s);
  {
    std::vector<double> Sd(h->Mtot), iS(h->Mtot);
    for (int m = 0; m < h->Mtot; ++m) {
      Sd[m] = double(h->S[m]);
      iS[m] = 1.0 / double(h->S[m]);
    }
    if ((s = upload(h, h->Sd_d, Sd.data(), Sd.size())) != MAM_OK) return bail(s);
    // (pageable sources: the copy has taken the data when the call returns)
    if ((s = upload(h, h->invS_d, iS.data(), iS.size())) != MAM_OK) return bail(s);
    std::vector<float> iSf(h->Mtot);
    std::vector<double> iSF(h->Mtot);
    std::vector<long long> aq(h->Mtot);
    for (int m = 0; m < h->Mtot; ++m) {
      iSf[m] = float(iS[m]);
      iSF[m] = iS[m] / h->fx_scale;  // F = 2^e: exact
      aq[m] = std::llround(std::ldexp(h->a[m], 62));
    }
    if ((s = upload(h, h->invS_f, iSf.data(), iSf.size())) != MAM_OK) return bail(s);
    if ((s = upload(h, h->invSF_d, iSF.data(), iSF.size())) != MAM_OK) return bail(s);
    if ((s = upload(h, h->a_q_d, aq.data(), aq.size())) != MAM_OK) return bail(s);
  }
  if ((s = upload(h, h->prob_meas_d, h->prob_meas.data(), h->prob_meas.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->rho_d, h->rho.data(), h->rho.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->gamma_d, h->gamma.data(), h->gamma.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->col_off_d, h->col_off.data(), h->col_off.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->prob_cols_d, h->prob_cols.data(), h->prob_cols.size())) != MAM_OK) return bail(s);
  if ((s = upload(h, h->col_meas, col_meas.data(), col_meas.size())) != MAM_OK) return bail(s);
  h->col_meas_h = col_meas;
  if (!h->bundle_cum.empty() &&
      (s = upload(h, h->bundle_cum_d, h->bundle_cum.data(), h->bundle_cum.size())) != MAM_OK)
    return bail(s);
  e = cudaMemsetAsync(h->done, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->passes, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err_d, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "memset"));

  // Keep the kept support points and the barycenter points (backward pass).
  for (int i = 0; i < n; ++i) {
    const mam_desc& d = descs[i];
    h->xi_h.insert(h->xi_h.end(), d.xi, d.xi + size_t(d.R) * d.dim);
  }
  h->has_gen_cost = false;
  for (int i = 0; i < n; ++i) h->has_gen_cost |= descs[i].cost != nullptr;

  // Costs (eq. HugeLP), built on the device problem by problem.
  {
    double* xi_d = nullptr;
    double* zeta_d = nullptr;
    double* gen_d = nullptr;
    auto tmp_free = [&]() {
      if (xi_d) cudaFree(xi_d);
      if (zeta_d) cudaFree(zeta_d);
      if (gen_d) cudaFree(gen_d);
    };
    long long uoff_g = 0;
    for (int i = 0; i < n && s == MAM_OK; ++i) {
      const mam_desc& d = descs[i];
      const long long c0 = h->prob_cols[i], c1 = h->prob_cols[i + 1];
      long long utot = 0;
      for (int m = 0; m < d.M; ++m) utot += d.S[m];
      if (!xi_d) {
        if (cudaMalloc(&xi_d, sizeof(double) * size_t(d.R) * d.dim) != cudaSuccess) {
          cudaGetLastError();
          s = fail(h, MAM_ERR_OOM, "cudaMalloc failed for xi");
          break;
        }
      }
      e = cudaMemcpy(xi_d, d.xi, sizeof(double) * size_t(d.R) * d.dim, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) { s = cuda_fail(h, e, "xi upload"); break; }
      if (!d.cost) {
        std::vector<double> zk(size_t(c1 - c0) * d.dim);
        for (long long c = c0; c < c1; ++c)
          for (int k = 0; k < d.dim; ++k)
            zk[size_t(c - c0) * d.dim + k] = d.zeta[size_t(h->keep[c] - uoff_g) * d.dim + k];
        h->zeta_kept.insert(h->zeta_kept.end(), zk.begin(), zk.end());
        if (zeta_d) cudaFree(zeta_d);
        zeta_d = nullptr;
        if (cudaMalloc(&zeta_d, sizeof(double) * std::max<size_t>(1, zk.size())) != cudaSuccess) {
          cudaGetLastError();
          s = fail(h, MAM_ERR_OOM, "cudaMalloc failed for zeta");
          break;
        }
        e = cudaMemcpy(zeta_d, zk.data(), sizeof(double) * zk.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { s = cuda_fail(h, e, "zeta upload"); break; }
        if (h->gen_cost)  // nothing stored: the kernels compute c from the points
          e = cudaSuccess;
        else if (h->shared_cost)  // one matrix C over the common support (xi is shared too)
          e = i == 0 ? launch_build_cost(h->cost_dtype, h->cost, xi_d, h->sup_zeta_d, nullptr,
                                         h->sup_meas_d, h->sup_alpha_d, h->sup_eta_d, 0,
                                         h->n_sup, h->R, h->ld, h->dim, h->stream)
                     : cudaSuccess;
        else {
          // Repeated columns (the same point in several measures of equal
          // alpha_m and eta) are built once and copied.
          std::vector<long long> reps, dst_src;
          repeated_cost_columns(zk, d.dim, c0, c1, col_meas, alpha_m, eta_m, reps, dst_src);
          std::vector<double> zr;
          const std::vector<double>* zb = &zk;
          long long* lists = nullptr;  // device: [reps][dst_src]
          if (!dst_src.empty()) {
            zr.resize(reps.size() * size_t(d.dim));
            for (size_t j = 0; j < reps.size(); ++j)
              for (int k = 0; k < d.dim; ++k)
                zr[j * d.dim + k] = zk[size_t(reps[j] - c0) * d.dim + k];
            zb = &zr;
            e = cudaMalloc(&lists, sizeof(long long) * (reps.size() + dst_src.size()));
            if (e == cudaSuccess)
              e = cudaMemcpy(lists, reps.data(), sizeof(long long) * reps.size(),
                             cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
              e = cudaMemcpy(lists + reps.size(), dst_src.data(),
                             sizeof(long long) * dst_src.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
              e = cudaMemcpy(zeta_d, zr.data(), sizeof(double) * zr.size(),
                             cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
              if (lists) cudaFree(lists);
              s = cuda_fail(h, e, "cost column lists");
              break;
            }
          }
          const long long nb = (long long)reps.size();
          bool tabulated = false;
          s = build_cost_tabulated(h, d.xi, *zb, c0, nb, lists, &tabulated);
          if (s == MAM_OK && !tabulated)
            e = launch_build_cost(h->cost_dtype, h->cost, xi_d, zeta_d, nullptr, h->col_meas,
                                  h->alpha_d, h->eta_d, c0, nb, h->R, h->ld, h->dim,
                                  h->stream, lists);
          if (s == MAM_OK && e == cudaSuccess && lists)
            e = launch_copy_cost_columns(h->cost_dtype, h->cost, lists + reps.size(),
                                         (long long)dst_src.size() / 2, h->ld, h->stream);
          if (lists) {
            const cudaError_t e2 = cudaStreamSynchronize(h->stream);
            if (e == cudaSuccess) e = e2;
            cudaFree(lists);
          }
          if (s != MAM_OK) break;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { s = cuda_fail(h, e, "cost kernel"); break; }
      } else {
        if (d.zeta) {
          for (long long c = c0; c < c1; ++c)
            for (int k = 0; k < d.dim; ++k)
              h->zeta_kept.push_back(d.zeta[size_t(h->keep[c] - uoff_g) * d.dim + k]);
        }
        const long long chunk = std::max<long long>(1, (64LL << 20) / (8LL * d.R));
        if (!gen_d) {
          if (cudaMalloc(&gen_d, sizeof(double) * size_t(chunk) * d.R) != cudaSuccess) {
            cudaGetLastError();
            s = fail(h, MAM_ERR_OOM, "cudaMalloc failed for the cost staging buffer");
            break;
          }
        }
        std::vector<double> buf;
        for (long long cb = c0; cb < c1 && s == MAM_OK; cb += chunk) {
          const long long ce = std::min(c1, cb + chunk);
          buf.resize(size_t(ce - cb) * d.R);
          for (long long c = cb; c < ce; ++c)
            std::memcpy(&buf[size_t(c - cb) * d.R],
                        d.cost + size_t(h->keep[c] - uoff_g) * d.R, sizeof(double) * d.R);
          e = cudaMemcpy(gen_d, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice);
          if (e == cudaSuccess)
            e = launch_build_cost(h->cost_dtype, h->cost, xi_d, nullptr, gen_d, h->col_meas,
                                  h->alpha_d, h->eta_d, cb, ce - cb, h->R, h->ld, h->dim,
                                  h->stream);
          if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
          if (e != cudaSuccess) s = cuda_fail(h, e, "cost kernel");
        }
      }
      uoff_g += utot;
    }
    tmp_free();
    if (s != MAM_OK) return bail(s);
  }

  if (h->gen_cost && (s = upload_gen_points(h)) != MAM_OK) return bail(s);
  if ((s = apply_config(h, default_config(h))) != MAM_OK) return bail(s);
  if ((s = reset_state(h)) != MAM_OK) return bail(s);
  if ((s = prime_thresholds(h)) != MAM_OK) return bail(s);
  *out = h;
  return MAM_OK;
}

}  // namespace mam

// ================================================================ C ABI

extern "C" {

mam_status mam_create(const mam_desc* desc, mam_problem** out) {
  return create_impl(1, desc, out);
}

mam_status mam_create_sharded(const mam_desc* desc, const mam_shard* shard,
                              mam_problem** out) {
  if (!shard) return fail(nullptr, MAM_ERR_INVALID_ARG, "shard is NULL");
  return create_impl(1, desc, out, shard);
}

mam_status mam_batch_create(int32_t n, const mam_desc* descs, mam_problem** out) {
  return create_impl(n, descs, out);
}

#define MAM_CHECK_HANDLE(h)                                                \
  do {                                                                     \
    if (!(h)) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");    \
    if ((h)->failed) return MAM_ERR_STATE;                                 \
  } while (0)

mam_status mam_step(mam_problem* h, int32_t n_iters) {
  MAM_CHECK_HANDLE(h);
  if (n_iters < 0) return fail(h, MAM_ERR_INVALID_ARG, "n_iters must be >= 0");
  return run_iterations(h, n_iters, h->diag_mode == MAM_DIAG_LAST);
}

static mam_status objective_all(mam_problem* h, std::vector<mam_objective_t>& out) {
  MAM_TRY(sync(h));
  MAM_CUDA(launch_diag_reduce(h->diag_wc, h->diag_lb, h->diag_res, h->prob_cols_d,
                              h->sched_d, draw_args(h), h->iter_d, h->P, h->diag_out,
                              h->stream),
           "diagnostic reduction");
  // Sharded: the rank's column sums and block sums, summed over the ranks
  // (the block sums of the last averaging are the rank's own, so this is the
  // same global value whether or not the last iteration exchanged them).
  if (h->sharded) {
    MAM_TRY(shard_exchange(h, h->diag_out, 3, MAM_SUM_F64));
    MAM_TRY(shard_block_sums(h));
    MAM_TRY(shard_exchange(h, h->passes, 1, MAM_SUM_I64));
  }
  const int nblk = h->sharded ? 1 : avg_blocks(h);
  std::vector<double> sums(size_t(h->P) * 3), blk(size_t(h->P) * nblk * 4), t(h->P);
  unsigned long long passes = 0;
  MAM_CUDA(cudaMemcpyAsync(sums.data(), h->diag_out, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, h->stream), "read");
  MAM_CUDA(cudaMemcpyAsync(blk.data(), h->sharded ? h->blk_glob : h->blk,
                           sizeof(double) * blk.size(), cudaMemcpyDeviceToHost, h->stream), "read");
  MAM_CUDA(cudaMemcpyAsync(&passes, h->passes, sizeof(passes), cudaMemcpyDeviceToHost, h->stream), "read");
  MAM_CUDA(cudaMemcpyAsync(t.data(), h->t_used, sizeof(double) * t.size(), cudaMemcpyDeviceToHost, h->stream), "read");
  MAM_TRY(sync(h));
  out.resize(h->P);
  for (int i = 0; i < h->P; ++i) {
    mam_objective_t& o = out[i];
    double e = 0, eh = 0, dp = 0;
    for (int b = 0; b < nblk; ++b) {
      e += blk[(size_t(i) * nblk + b) * 4];
      eh += blk[(size_t(i) * nblk + b) * 4 + 1];
      dp += blk[(size_t(i) * nblk + b) * 4 + 2];
    }
    o.w_hat = sums[3 * i];
    o.lower_bound = sums[3 * i + 1];
    o.fp_resid = std::sqrt(sums[3 * i + 2]);
    o.dist_pihat = std::sqrt(eh);
    o.f_unbal = o.w_hat + (std::isinf(h->gamma[i]) ? 0.0 : h->gamma[i] * o.dist_pihat);
    o.dp_norm = std::sqrt(dp);
    o.t = t[i];
    o.dist_theta = std::sqrt(e);
    const double rD = h->rho[i] * o.dist_theta;
    o.t_next = (std::isinf(h->gamma[i]) || rD <= h->gamma[i]) ? 1.0 : h->gamma[i] / rD;
    o.iter = h->diag_iter;
    o.newton_passes = (int64_t)passes;
  }
  return MAM_OK;
}

mam_status mam_objective(mam_problem* h, int32_t index, mam_objective_t* out) {
  MAM_CHECK_HANDLE(h);
  if (!out || index < 0 || index >= h->P)
    return fail(h, MAM_ERR_INVALID_ARG, "bad objective index or output");
  std::vector<mam_objective_t> all;
  MAM_TRY(objective_all(h, all));
  *out = all[index];
  const double v[] = {out->w_hat, out->lower_bound, out->fp_resid, out->dist_pihat,
                      out->dist_theta, out->t};
  for (double x : v)
    if (!std::isfinite(x)) return fail(h, MAM_ERR_NONFINITE, "non-finite diagnostic");
  return MAM_OK;
}

mam_status mam_objective_all(mam_problem* h, mam_objective_t* out) {
  MAM_CHECK_HANDLE(h);
  if (!out) return fail(h, MAM_ERR_INVALID_ARG, "out is NULL");
  std::vector<mam_objective_t> all;
  MAM_TRY(objective_all(h, all));
  for (int i = 0; i < h->P; ++i) {
    out[i] = all[i];
    const double v[] = {all[i].w_hat, all[i].lower_bound, all[i].fp_resid,
                        all[i].dist_pihat, all[i].dist_theta, all[i].t};
    for (double x : v)
      if (!std::isfinite(x)) return fail(h, MAM_ERR_NONFINITE, "non-finite diagnostic");
  }
  return MAM_OK;
}

mam_status mam_solve(mam_problem* h, int32_t max_iters, double gap_tol, double w_ref,
                     int32_t check_every, int32_t* iters_done, double* gap_out) {
  MAM_CHECK_HANDLE(h);
  if (max_iters < 0 || check_every < 1 || !(gap_tol >= 0))
    return fail(h, MAM_ERR_INVALID_ARG, "bad solve arguments");
  int done = 0;
  double gap = INFINITY;
  std::vector<mam_objective_t> all;
  while (done < max_iters) {
    const int n = std::min<int>(check_every, max_iters - done);
    MAM_TRY(run_iterations(h, n, true));
    done += n;
    MAM_TRY(objective_all(h, all));
    gap = 0;
    for (int i = 0; i < h->P; ++i) {
      const mam_objective_t& o = all[i];
      const double ref = w_ref > 0 ? w_ref : o.lower_bound;
      double g = std::fabs(o.f_unbal - ref) / std::max(std::fabs(ref), 1e-300);
      if (std::isinf(h->gamma[i])) g = std::max(g, o.dist_pihat / h->Qa[i]);
      if (!std::isfinite(g)) {
        if (iters_done) *iters_done = done;
        return fail(h, MAM_ERR_NONFINITE, "non-finite gap");
      }
      gap = std::max(gap, g);
    }
    if (gap <= gap_tol) break;
  }
  if (iters_done) *iters_done = done;
  if (gap_out) *gap_out = gap;
  return MAM_OK;
}

mam_status mam_update_support(mam_problem* h, double* xi_out) {
  MAM_CHECK_HANDLE(h);
  if (h->sparse)
    return fail(h, MAM_ERR_UNSUPPORTED, "the support step needs the dense plan layout");
  if (h->P != 1) return fail(h, MAM_ERR_INVALID_ARG, "the support step needs a single problem");
  if (h->sharded)
    return fail(h, MAM_ERR_INVALID_ARG, "the support step is not offered for sharded problems");
  if (h->nb > 1)
    return fail(h, MAM_ERR_INVALID_ARG, "the support step needs the deterministic index set");
  if (h->has_gen_cost || h->zeta_kept.size() != size_t(h->T) * h->dim)
    return fail(h, MAM_ERR_INVALID_ARG,
                "the support step needs support points and the squared Euclidean cost");
  mam_status s = MAM_OK;
  if (!h->sup_acc) {  // first use: the buffers are published together
    double *xd = nullptr, *zd = nullptr;
    unsigned long long* ac = nullptr;
    if ((s = dalloc(h, &xd, size_t(h->R) * h->dim, "support")) != MAM_OK) return s;
    if ((s = dalloc(h, &zd, h->zeta_kept.size(), "support points")) != MAM_OK) return s;
    if ((s = dalloc(h, &ac, size_t(h->R) * (h->dim + 1), "support sums")) != MAM_OK) return s;
    if ((s = upload(h, xd, h->xi_h.data(), h->xi_h.size())) != MAM_OK) return s;
    if ((s = upload(h, zd, h->zeta_kept.data(), h->zeta_kept.size())) != MAM_OK) return s;
    MAM_CUDA(cudaMemsetAsync(ac, 0, sizeof(unsigned long long) * size_t(h->R) * (h->dim + 1),
                             h->stream),
             "memset");
    h->xi_dev = xd;
    h->zeta_dev = zd;
    h->sup_acc = ac;
  }
  // t of the next step, from the averaging kernel's block sums (eq.
  // Unbalanced-prox).
  double t = 1.0;
  if (!std::isinf(h->gamma[0])) {
    const int nblk = avg_blocks(h);
    std::vector<double> blk(size_t(nblk) * 4);
    MAM_CUDA(cudaMemcpyAsync(blk.data(), h->blk, sizeof(double) * blk.size(),
                             cudaMemcpyDeviceToHost, h->stream),
             "read");
    MAM_TRY(sync(h));
    double e = 0;
    for (int b = 0; b < nblk; ++b) e += blk[size_t(b) * 4];
    const double rD = h->rho[0] * std::sqrt(e);
    t = rD <= h->gamma[0] ? 1.0 : h->gamma[0] / rD;
  }
  // Fixed-point scale: every per-row sum stays below 2^61 in magnitude.
  double zmax = 1.0, mass = 0.0;
  for (double v : h->zeta_kept) zmax = std::max(zmax, std::fabs(v));
  for (int m = 0; m < h->Mtot; ++m) mass += h->alpha_h[m] * h->Q_h[m];
  if (!(mass > 0)) return fail(h, MAM_ERR_INVALID_ARG, "the support step needs sum alpha_m Q_m > 0");
  SupportArgs a{};
  a.theta = h->theta;
  a.cost = h->cost;
  a.q = h->q;
  a.lam = h->lam;
  a.col_meas = h->col_meas;
  a.delta32 = h->delta32;
  a.inv_rho = h->irho_m;
  a.cost_col = h->cost_col;
  a.gen_xi = h->gen_xi;
  a.gen_zeta = h->gen_zeta;
  a.alpha = h->alpha_d;
  a.zeta = h->zeta_dev;
  a.acc = h->sup_acc;
  {
    const double ex = std::floor(std::log2(std::ldexp(1.0, 61) / (1.01 * zmax * mass)));
    a.fx = std::ldexp(1.0, int(std::max(-960.0, std::min(960.0, ex))));  // finite scale
  }
  a.t = float(t);
  a.lam_floor = h->capped ? 0.f : -INFINITY;
  a.T = h->T;
  a.R = h->R;
  a.ld = h->ld;
  a.dim = h->dim;
  MAM_CUDA(launch_support_step(h->cost_dtype, a, h->xi_dev, h->stream), "support step");
  // The costs of the new support (FP64, rounded to the storage type; with
  // generated costs, the FP32 copy of the new support).
  if (h->gen_cost) {
    MAM_CUDA(cudaMemcpyAsync(h->xi_h.data(), h->xi_dev, sizeof(double) * h->xi_h.size(),
                             cudaMemcpyDeviceToHost, h->stream),
             "read");
    MAM_TRY(sync(h));
    MAM_TRY(upload_gen_points(h));
  } else
  MAM_CUDA(h->shared_cost
               ? launch_build_cost(h->cost_dtype, h->cost, h->xi_dev, h->sup_zeta_d, nullptr,
                                   h->sup_meas_d, h->sup_alpha_d, h->sup_eta_d, 0, h->n_sup,
                                   h->R, h->ld, h->dim, h->stream)
               : launch_build_cost(h->cost_dtype, h->cost, h->xi_dev, h->zeta_dev, nullptr,
                                   h->col_meas, h->alpha_d, h->eta_d, 0, h->T, h->R, h->ld,
                                   h->dim, h->stream),
           "cost kernel");
  MAM_CUDA(cudaMemcpyAsync(h->xi_h.data(), h->xi_dev, sizeof(double) * h->xi_h.size(),
                           cudaMemcpyDeviceToHost, h->stream),
           "read");
  MAM_TRY(sync(h));
  if (xi_out) std::memcpy(xi_out, h->xi_h.data(), sizeof(double) * h->xi_h.size());
  return MAM_OK;
}

mam_status mam_free_support(mam_problem* h, int32_t outer, int32_t inner_iters, double gap_tol,
                            int32_t check_every, double* xi_out, int32_t* iters_done) {
  MAM_CHECK_HANDLE(h);
  if (outer < 0 || inner_iters < 0 || check_every < 1 || !(gap_tol >= 0))
    return fail(h, MAM_ERR_INVALID_ARG, "bad free-support arguments");
  if (h->sparse)
    return fail(h, MAM_ERR_UNSUPPORTED, "the support step needs the dense plan layout");
  if (h->sharded)
    return fail(h, MAM_ERR_INVALID_ARG, "the support step is not offered for sharded problems");
  int total = 0;
  for (int k = 0; k < outer; ++k) {
    // Algorithm 2: the fixed-support problem on the current support ...
    int done = 0;
    if (gap_tol > 0) {
      MAM_TRY(mam_solve(h, inner_iters, gap_tol, 0.0, check_every, &done, nullptr));
    } else {
      MAM_TRY(mam_step(h, inner_iters));
      done = inner_iters;
    }
    total += done;
    // ... then the support step of Prop. 4 (costs rebuilt, theta kept).
    MAM_TRY(mam_update_support(h, xi_out));
  }
  if (outer == 0 && xi_out && h->xi_h.size() == size_t(h->R) * h->dim)
    std::memcpy(xi_out, h->xi_h.data(), sizeof(double) * h->xi_h.size());  // unchanged support
  if (iters_done) *iters_done = total;
  return MAM_OK;
}

mam_status mam_get_barycenter(mam_problem* h, double* p_out, int32_t device_ptr) {
  MAM_CHECK_HANDLE(h);
  if (!p_out) return fail(h, MAM_ERR_INVALID_ARG, "p_out is NULL");
  MAM_CUDA(cudaMemcpyAsync(p_out, h->p, sizeof(double) * h->P * h->R,
                           device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           h->stream),
           "barycenter copy");
  return sync(h);
}

mam_status mam_get_marginals(mam_problem* h, double* pm_out, int32_t device_ptr) {
  MAM_CHECK_HANDLE(h);
  if (!pm_out) return fail(h, MAM_ERR_INVALID_ARG, "pm_out is NULL");
  const size_t MR = size_t(h->Mtot) * h->R;
  if (device_ptr) {
    MAM_CUDA(launch_fx_to_double(h->pm, MR, 1.0 / h->fx_scale, pm_out, h->stream),
             "marginal conversion");
    return sync(h);
  }
  std::vector<long long> fx(MR);
  MAM_CUDA(cudaMemcpyAsync(fx.data(), h->pm, sizeof(long long) * MR, cudaMemcpyDeviceToHost,
                           h->stream),
           "marginal copy");
  MAM_TRY(sync(h));
  const double inv = 1.0 / h->fx_scale;
  for (size_t i = 0; i < MR; ++i) pm_out[i] = double(fx[i]) * inv;
  return MAM_OK;
}

// Sparse plans: theta of columns col0 .. col0 + ncols - 1, expanded on the
// device in chunks of at most 64 MB and copied to the host.
static mam_status get_theta_sparse(mam_problem* h, long long col0, long long ncols,
                                   float* out) {
  const long long chunk = std::max(1LL, (64LL << 20) / (4LL * h->R));
  float* buf = nullptr;
  MAM_CUDA(cudaMalloc(&buf, sizeof(float) * size_t(std::min(chunk, ncols)) * h->R),
           "cudaMalloc (theta expansion)");
  mam_status s = MAM_OK;
  for (long long c = 0; c < ncols && s == MAM_OK; c += chunk) {
    const long long n = std::min(chunk, ncols - c);
    cudaError_t e = launch_expand_sparse(buf, col0 + c, n, h->sp_cnt, h->sp_pairs, h->sp_k,
                                         h->d_last, h->th0, h->col_meas, h->R, h->ld,
                                         h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + size_t(c) * h->R, buf, sizeof(float) * size_t(n) * h->R,
                          cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = cuda_fail(h, e, "theta expansion");
  }
  cudaFree(buf);
  return s != MAM_OK ? s : sync(h);
}

mam_status mam_get_theta(mam_problem* h, float* theta_out) {
  MAM_CHECK_HANDLE(h);
  if (!theta_out) return fail(h, MAM_ERR_INVALID_ARG, "theta_out is NULL");
  if (h->sparse) {
    MAM_TRY(sync(h));
    return get_theta_sparse(h, 0, h->T, theta_out);
  }
  MAM_CUDA(cudaMemcpy2DAsync(theta_out, sizeof(float) * h->R, h->theta,
                             sizeof(float) * h->ld, sizeof(float) * h->R, h->T,
                             cudaMemcpyDeviceToHost, h->stream),
           "theta copy");
  return sync(h);
}

mam_status mam_get_theta_range(mam_problem* h, int64_t col0, int64_t ncols, float* theta_out) {
  MAM_CHECK_HANDLE(h);
  if (!theta_out) return fail(h, MAM_ERR_INVALID_ARG, "theta_out is NULL");
  if (col0 < 0 || ncols < 0 || col0 + ncols > h->T)
    return fail(h, MAM_ERR_INVALID_ARG, "column range outside 0..T");
  if (ncols == 0) return MAM_OK;
  if (h->sparse) {
    MAM_TRY(sync(h));
    return get_theta_sparse(h, col0, ncols, theta_out);
  }
  MAM_CUDA(cudaMemcpy2DAsync(theta_out, sizeof(float) * h->R, h->theta + size_t(col0) * h->ld,
                             sizeof(float) * h->ld, sizeof(float) * h->R, size_t(ncols),
                             cudaMemcpyDeviceToHost, h->stream),
           "theta copy");
  return sync(h);
}

mam_status mam_get_work(const mam_problem* h, int64_t* columns, int64_t* entries) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  if (columns) *columns = h->work_cols;
  if (entries) *entries = h->work_entries;
  return MAM_OK;
}

mam_status mam_get_sizes(const mam_problem* h, int32_t* n_problems, int32_t* n_measures,
                         int32_t* R, int64_t* T, int32_t* ld) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  if (n_problems) *n_problems = h->P;
  if (n_measures) *n_measures = h->Mtot;
  if (R) *R = h->R;
  if (T) *T = h->T;
  if (ld) *ld = h->ld;
  return MAM_OK;
}

mam_status mam_get_pruned_sizes(const mam_problem* h, int32_t* S_out) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  if (!S_out) return fail(const_cast<mam_problem*>(h), MAM_ERR_INVALID_ARG, "S_out is NULL");
  for (int m = 0; m < h->Mtot; ++m) S_out[m] = h->S[m];
  return MAM_OK;
}

// ------------------------------------------------------------ checkpoints

namespace {
struct StateHeader {
  uint64_t magic;
  int64_t T, iter, diag_iter;
  int32_t P, Mtot, R, ld;
  int32_t bundle_cur, bundle_prev, plan_layout, sparse_slots;
};
constexpr uint64_t kStateMagic = 0x334554415453414dull;  // "MASTATE3"

}  // namespace
}  // extern "C"

namespace mam {
std::vector<Piece> state_pieces(mam_problem* h) {
  const size_t MR = size_t(h->Mtot) * h->R;
  std::vector<Piece> plans;
  if (h->sparse)
    plans = {{h->sp_cnt, sizeof(int) * size_t(h->T)},
             {h->sp_pairs, sizeof(int2) * size_t(h->T) * h->sp_k},
             {h->d_last, sizeof(float) * size_t(h->Mtot) * h->ld}};
  else
    plans = {{h->theta, sizeof(float) * size_t(h->T) * h->ld}};
  std::vector<Piece> rest = {
          {h->lam, sizeof(float) * size_t(h->T)},
          {h->pm, sizeof(long long) * MR},
          {h->p, sizeof(double) * size_t(h->P) * h->R},
          {h->delta32, sizeof(float) * size_t(h->Mtot) * h->ld},
          {h->phat, sizeof(double) * MR},
          {h->t_used, sizeof(double) * h->P},
          {h->blk, sizeof(double) * 4 * size_t(h->P) * avg_blocks(h)},
          {h->diag_wc, sizeof(float) * size_t(h->T)},
          {h->diag_lb, sizeof(float) * size_t(h->T)},
          {h->diag_res, sizeof(float) * size_t(h->T)},
          {h->passes, sizeof(unsigned long long)},
          {h->iter_d, sizeof(long long)}};
  plans.insert(plans.end(), rest.begin(), rest.end());
  return plans;
}
}  // namespace mam

extern "C" {

mam_status mam_get_state(mam_problem* h, void* buf, size_t* bytes) {
  MAM_CHECK_HANDLE(h);
  if (!bytes) return fail(h, MAM_ERR_INVALID_ARG, "bytes is NULL");
  const auto pieces = state_pieces(h);
  size_t need = sizeof(StateHeader);
  for (auto& p : pieces) need += p.bytes;
  if (!buf) {
    *bytes = need;
    return MAM_OK;
  }
  if (*bytes < need) return fail(h, MAM_ERR_INVALID_ARG, "state buffer too small");
  MAM_TRY(sync(h));
  StateHeader hd{};
  hd.magic = kStateMagic;
  hd.T = h->T;
  hd.iter = h->iter;
  hd.diag_iter = h->diag_iter;
  hd.P = h->P;
  hd.Mtot = h->Mtot;
  hd.R = h->R;
  hd.ld = h->ld;
  hd.plan_layout = h->sparse ? MAM_PLAN_SPARSE : MAM_PLAN_DENSE;
  hd.sparse_slots = h->sp_k;
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  for (auto& p : pieces) {
    MAM_CUDA(cudaMemcpy(out + off, p.dev, p.bytes, cudaMemcpyDeviceToHost), "state");
    off += p.bytes;
  }
  *bytes = need;
  return MAM_OK;
}

mam_status mam_set_state(mam_problem* h, const void* buf, size_t bytes) {
  MAM_CHECK_HANDLE(h);
  if (!buf) return fail(h, MAM_ERR_INVALID_ARG, "buf is NULL");
  const auto pieces = state_pieces(h);
  size_t need = sizeof(StateHeader);
  for (auto& p : pieces) need += p.bytes;
  StateHeader hd;
  if (bytes < need) return fail(h, MAM_ERR_INVALID_ARG, "state buffer too small");
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.T != h->T || hd.P != h->P || hd.Mtot != h->Mtot ||
      hd.R != h->R || hd.ld != h->ld ||
      hd.plan_layout != (h->sparse ? MAM_PLAN_SPARSE : MAM_PLAN_DENSE) ||
      hd.sparse_slots != h->sp_k)
    return fail(h, MAM_ERR_INVALID_ARG, "state does not belong to this problem");
  MAM_TRY(sync(h));
  const char* in = static_cast<const char*>(buf);
  size_t off = sizeof(hd);
  for (auto& p : pieces) {
    MAM_CUDA(cudaMemcpy(p.dev, in + off, p.bytes, cudaMemcpyHostToDevice), "state");
    off += p.bytes;
  }
  h->iter = hd.iter;
  h->diag_iter = hd.diag_iter;
  return MAM_OK;
}

// ------------------------------------------------------------ config

mam_status mam_get_config(const mam_problem* h, mam_kernel_config* cfg) {
  if (!h || !cfg) return fail(nullptr, MAM_ERR_INVALID_ARG, "null argument");
  *cfg = h->cfg;
  return MAM_OK;
}

mam_status mam_set_config(mam_problem* h, const mam_kernel_config* cfg) {
  MAM_CHECK_HANDLE(h);
  if (!cfg) return fail(h, MAM_ERR_INVALID_ARG, "cfg is NULL");
  MAM_TRY(sync(h));
  const mam_kernel_config old = h->cfg;
  mam_status s = apply_config(h, *cfg);
  if (s != MAM_OK && s != MAM_ERR_CUDA) {
    const std::string msg = h->err;
    apply_config(h, old);
    h->err = msg;
  }
  return s;
}

mam_status mam_profile_enable(mam_problem* h, int32_t enable) {
  MAM_CHECK_HANDLE(h);
  MAM_TRY(sync(h));
  h->profiling = enable != 0;
  h->prof_used = 0;
  return MAM_OK;
}

mam_status mam_profile_read(mam_problem* h, double* column_ms, double* average_ms,
                            int64_t* launches) {
  MAM_CHECK_HANDLE(h);
  MAM_TRY(sync(h));
  double c = 0, a = 0;
  const size_t n = h->prof_used / 3;
  for (size_t i = 0; i < n; ++i) {
    float x = 0, y = 0;
    MAM_CUDA(cudaEventElapsedTime(&x, h->prof_events[3 * i], h->prof_events[3 * i + 1]), "cudaEventElapsedTime");
    MAM_CUDA(cudaEventElapsedTime(&y, h->prof_events[3 * i + 1], h->prof_events[3 * i + 2]), "cudaEventElapsedTime");
    c += x;
    a += y;
  }
  if (column_ms) *column_ms = c;
  if (average_ms) *average_ms = a;
  if (launches) *launches = int64_t(n);
  h->prof_used = 0;
  return MAM_OK;
}

const char* mam_last_error(const mam_problem* h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

void mam_destroy(mam_problem* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_sched(h);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  free_backward(h);
  for (cudaEvent_t e : h->prof_events) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
