// libmam: differentiation through unrolled MAM iterations.
//
// Reverse mode with checkpointing.  mam_forward_record runs K iterations of
// Algorithm 1 from theta^0 and keeps a device snapshot of the whole state
// every ckpt_every iterations (and after the last one).  mam_backward walks
// the segments from the last to the first: it restores the segment's
// snapshot, re-runs its iterations with the same kernels (the iterates are
// bit-identical because every reduction is order-independent) while the
// column kernels record each step's active sets as bit masks, and then
// applies the reverse step of each iteration in reverse order
// (mam_backward_kernels.cu).  Memory: (K / ckpt_every + 1) state snapshots
// plus (ckpt_every + 1) active-set masks of one bit per plan entry.
// With ckpt_every = 0 (automatic), when the masks of all K steps (K bits per
// plan entry) fit in a quarter of the free device memory,
// mam_forward_record keeps them from the forward pass itself, and
// mam_backward applies the reverse steps directly: no segment is restored or
// recomputed.  Otherwise (or with an explicit ckpt_every) it checkpoints.
#include "mam.h"
#include "mam_handle.h"
#include "mam_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace mam {

struct BackwardState {
  int K = 0, ck = 0, nseg = 0;
  std::vector<void*> allocs;
  size_t snap_bytes = 0;
  std::vector<char*> snaps;  // [nseg + 1]
  std::vector<long long> snap_iter, snap_diag_iter;
  bool all_masks = false;         // the masks of all K steps are kept (no recomputation)
  unsigned* mask_all = nullptr;   // [K][T][mw] active sets of every step (all_masks)
  unsigned* mask_seg = nullptr;   // [ck][T][mw] active sets of the segment's steps
  unsigned* mask_next = nullptr;  // [T][mw] active sets of the step after the segment
  float* stored = nullptr;   // [T][ld]
  double* pend = nullptr;    // [Mtot][R]
  double* red = nullptr;     // [Mtot][1 + dim][R]
  double* acc_prev = nullptr;  // [Mtot][R]
  float* part = nullptr;     // [nchunks][1 + dim][R]
  float* pend_f = nullptr;   // [Mtot][R]
  long long* chunk_begin = nullptr;  // [nchunks + 1]
  int* meas_chunk = nullptr;         // [Mtot + 1]
  int nchunks = 0;
  double* qbar = nullptr;    // [T]
  double* zetabar = nullptr; // [T][dim]
  double* xibar = nullptr;   // [R][dim]
  double* zeta = nullptr;    // [T][dim]
  double* xi = nullptr;      // [R][dim]
  ~BackwardState() {
    for (void* p : allocs) cudaFree(p);
  }
};

void free_backward(mam_problem* h) {
  delete h->bwd;
  h->bwd = nullptr;
}

namespace {

#define BWD_CUDA(x, where)                                \
  do {                                                    \
    cudaError_t _e = (x);                                 \
    if (_e != cudaSuccess) return cuda_fail(h, _e, where); \
  } while (0)
#define BWD_TRY(x)                 \
  do {                             \
    mam_status _s = (x);           \
    if (_s != MAM_OK) return _s;   \
  } while (0)

template <typename T>
mam_status balloc(mam_problem* h, BackwardState* b, T** ptr, size_t count, const char* what) {
  void* p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MAM_ERR_OOM, std::string("cudaMalloc failed for ") + what + " (" +
                                    std::to_string(count * sizeof(T)) + " bytes)");
  }
  b->allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return MAM_OK;
}

mam_status snapshot(mam_problem* h, int i) {
  BackwardState* b = h->bwd;
  size_t off = 0;
  for (const Piece& pc : state_pieces(h)) {
    BWD_CUDA(cudaMemcpyAsync(b->snaps[i] + off, pc.dev, pc.bytes, cudaMemcpyDeviceToDevice,
                             h->stream),
             "snapshot copy");
    off += (pc.bytes + 255) / 256 * 256;
  }
  b->snap_iter[i] = h->iter;
  b->snap_diag_iter[i] = h->diag_iter;
  return MAM_OK;
}

mam_status restore(mam_problem* h, int i) {
  BackwardState* b = h->bwd;
  size_t off = 0;
  for (const Piece& pc : state_pieces(h)) {
    BWD_CUDA(cudaMemcpyAsync(pc.dev, b->snaps[i] + off, pc.bytes, cudaMemcpyDeviceToDevice,
                             h->stream),
             "restore copy");
    off += (pc.bytes + 255) / 256 * 256;
  }
  h->iter = b->snap_iter[i];
  h->diag_iter = b->snap_diag_iter[i];
  return MAM_OK;
}

size_t snapshot_bytes(mam_problem* h) {
  size_t n = 0;
  for (const Piece& pc : state_pieces(h)) n += (pc.bytes + 255) / 256 * 256;
  return n;
}

}  // namespace
}  // namespace mam

using namespace mam;

extern "C" {

mam_status mam_forward_record(mam_problem* h, int32_t K, int32_t ckpt_every) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  if (h->failed) return MAM_ERR_STATE;
  if (h->P != 1) return fail(h, MAM_ERR_INVALID_ARG, "differentiation needs a single problem");
  if (h->sharded)
    return fail(h, MAM_ERR_INVALID_ARG, "differentiation is not offered for sharded problems");
  if (h->ld > kMaxCtaR || h->cfg.kind == 2)  // the cluster kernel records no active sets
    return fail(h, MAM_ERR_INVALID_ARG,
                "differentiation needs columns of at most " + std::to_string(kMaxCtaR) +
                    " rows and a one-CTA or one-warp column kernel (kind 0 or 1)");
  if (h->capped)
    return fail(h, MAM_ERR_INVALID_ARG,
                "differentiation needs columns that carry their mass (capped = 0)");
  if (std::isfinite(h->gamma[0]))
    return fail(h, MAM_ERR_INVALID_ARG, "differentiation needs the balanced problem (gamma = inf)");
  if (h->nb != 1)
    return fail(h, MAM_ERR_INVALID_ARG, "differentiation needs the deterministic index set");
  if (h->theta0_mode != 0 && h->theta0_mode != 1)
    return fail(h, MAM_ERR_INVALID_ARG, "theta0_mode must be 0 or 1");
  if (K < 1) return fail(h, MAM_ERR_INVALID_ARG, "K must be >= 1");
  const bool automatic = ckpt_every == 0;
  if (ckpt_every == 0) ckpt_every = std::max(1, int(std::lround(std::sqrt(double(K)))));
  if (ckpt_every < 1 || ckpt_every > K)
    return fail(h, MAM_ERR_INVALID_ARG, "ckpt_every must be in 1..K (0 = about sqrt(K))");
  BWD_TRY(sync(h));
  free_backward(h);
  h->bwd = new BackwardState();
  BackwardState* b = h->bwd;
  b->K = K;
  b->ck = ckpt_every;
  b->nseg = (K + ckpt_every - 1) / ckpt_every;
  b->snap_bytes = snapshot_bytes(h);
  b->snaps.assign(b->nseg + 1, nullptr);
  b->snap_iter.assign(b->nseg + 1, 0);
  b->snap_diag_iter.assign(b->nseg + 1, -1);
  const size_t Tl = size_t(h->T) * h->ld;
  const size_t MR = size_t(h->Mtot) * h->R;
  const int dim = std::max(1, h->dim);
  mam_status s = MAM_OK;
  const size_t Tm = size_t(h->T) * ((h->ld + 31) / 32);
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    b->all_masks = automatic && size_t(K) * Tm * sizeof(unsigned) <= free_b / 4;
  }
  // Keeping every step's masks needs only the first and the last state.
  for (int i = 0; i <= b->nseg && s == MAM_OK; ++i)
    if (!b->all_masks || i == 0 || i == b->nseg)
      s = balloc(h, b, &b->snaps[i], b->snap_bytes, "state snapshot");
  if (b->all_masks) {
    if (s == MAM_OK) s = balloc(h, b, &b->mask_all, Tm * size_t(K), "active sets");
  } else {
    if (s == MAM_OK) s = balloc(h, b, &b->mask_seg, Tm * b->ck, "active sets");
    if (s == MAM_OK) s = balloc(h, b, &b->mask_next, Tm, "active sets");
  }
  if (s == MAM_OK) s = balloc(h, b, &b->stored, Tl, "adjoint plan");
  if (s == MAM_OK) s = balloc(h, b, &b->pend, MR, "adjoint marginals");
  // chunks of at most kBwdChunk consecutive columns of one measure
  std::vector<long long> cb;
  std::vector<int> mc;
  for (int m = 0; m < h->Mtot; ++m) {
    mc.push_back(int(cb.size()));
    for (long long c = h->col_off[m]; c < h->col_off[m + 1]; c += kBwdChunk) cb.push_back(c);
  }
  mc.push_back(int(cb.size()));
  b->nchunks = int(cb.size());
  cb.push_back(h->col_off[h->Mtot]);
  if (s == MAM_OK) s = balloc(h, b, &b->red, MR * (1 + dim), "adjoint row sums");
  if (s == MAM_OK) s = balloc(h, b, &b->acc_prev, MR, "adjoint row sums");
  if (s == MAM_OK) s = balloc(h, b, &b->pend_f, MR, "adjoint marginals (fp32)");
  if (s == MAM_OK)
    s = balloc(h, b, &b->part, size_t(b->nchunks) * (1 + dim) * h->R, "adjoint chunk sums");
  if (s == MAM_OK) s = balloc(h, b, &b->chunk_begin, cb.size(), "chunk table");
  if (s == MAM_OK) s = balloc(h, b, &b->meas_chunk, mc.size(), "chunk table");
  if (s == MAM_OK) s = balloc(h, b, &b->qbar, size_t(h->T), "grad q");
  if (s == MAM_OK) s = balloc(h, b, &b->zetabar, size_t(h->T) * dim, "grad zeta");
  if (s == MAM_OK) s = balloc(h, b, &b->xibar, size_t(h->R) * dim, "grad xi");
  if (s == MAM_OK) s = balloc(h, b, &b->zeta, size_t(h->T) * dim, "zeta");
  if (s == MAM_OK) s = balloc(h, b, &b->xi, size_t(h->R) * dim, "xi");
  if (s != MAM_OK) {
    free_backward(h);
    return s;
  }
  BWD_CUDA(cudaMemcpy(b->chunk_begin, cb.data(), sizeof(long long) * cb.size(),
                      cudaMemcpyHostToDevice),
           "chunk table upload");
  BWD_CUDA(cudaMemcpy(b->meas_chunk, mc.data(), sizeof(int) * mc.size(), cudaMemcpyHostToDevice),
           "chunk table upload");
  if (h->zeta_kept.size() == size_t(h->T) * h->dim && h->dim > 0)
    BWD_CUDA(cudaMemcpy(b->zeta, h->zeta_kept.data(), sizeof(double) * h->zeta_kept.size(),
                        cudaMemcpyHostToDevice),
             "zeta upload");
  if (h->xi_h.size() >= size_t(h->R) * h->dim && h->dim > 0)
    BWD_CUDA(cudaMemcpy(b->xi, h->xi_h.data(), sizeof(double) * size_t(h->R) * h->dim,
                        cudaMemcpyHostToDevice),
             "xi upload");
  BWD_TRY(reset_state(h));
  if (b->all_masks) {
    // The forward kernels record every step's active sets as they go.
    BWD_TRY(snapshot(h, 0));
    for (int k = 0; k < K; ++k) {
      h->amask = b->mask_all + Tm * size_t(k);
      const mam_status st = launch_iteration(h, false);
      h->amask = nullptr;
      BWD_TRY(st);
    }
    h->iter += K;
    BWD_TRY(snapshot(h, b->nseg));
    return sync(h);
  }
  for (int seg = 0; seg < b->nseg; ++seg) {
    BWD_TRY(snapshot(h, seg));
    const int L = std::min(b->ck, K - seg * b->ck);
    BWD_TRY(run_iterations(h, L, false));
  }
  BWD_TRY(snapshot(h, b->nseg));
  return sync(h);
}

mam_status mam_backward(mam_problem* h, const double* grad_p, double* grad_q,
                        double* grad_zeta, double* grad_xi) {
  if (!h) return fail(nullptr, MAM_ERR_INVALID_ARG, "null handle");
  if (h->failed) return MAM_ERR_STATE;
  BackwardState* b = h->bwd;
  if (!b || b->K < 1) return fail(h, MAM_ERR_STATE, "call mam_forward_record first");
  if (!grad_p) return fail(h, MAM_ERR_INVALID_ARG, "grad_p is NULL");
  for (int r = 0; r < h->R; ++r)
    if (!std::isfinite(grad_p[r])) return fail(h, MAM_ERR_INVALID_ARG, "grad_p is not finite");
  const bool coords = h->dim > 0 && h->zeta_kept.size() == size_t(h->T) * h->dim &&
                      !h->has_gen_cost;
  if ((grad_zeta || grad_xi) && !coords)
    return fail(h, MAM_ERR_INVALID_ARG,
                "coordinate gradients need the squared Euclidean cost built from xi and zeta");
  const size_t Tl = size_t(h->T) * h->ld;
  const size_t MR = size_t(h->Mtot) * h->R;
  const int dim = coords ? h->dim : 0;
  const int dimA = std::max(1, h->dim);
  // thetabar^K: p^K = sum_m a_m rowsum(theta^(m),K), so every column of
  // measure m receives a_m dL/dp^K.
  std::vector<double> pend0(MR);
  for (int m = 0; m < h->Mtot; ++m)
    for (int r = 0; r < h->R; ++r) pend0[size_t(m) * h->R + r] = h->a[m] * grad_p[r];
  BWD_CUDA(cudaMemcpyAsync(b->pend, pend0.data(), sizeof(double) * MR, cudaMemcpyHostToDevice,
                           h->stream),
           "grad_p upload");
  std::vector<float> pend0f(pend0.begin(), pend0.end());
  BWD_CUDA(cudaMemcpyAsync(b->pend_f, pend0f.data(), sizeof(float) * MR, cudaMemcpyHostToDevice,
                           h->stream),
           "grad_p upload");
  BWD_CUDA(cudaMemsetAsync(b->stored, 0, sizeof(float) * Tl, h->stream), "memset");
  BWD_CUDA(cudaMemsetAsync(b->acc_prev, 0, sizeof(double) * MR, h->stream), "memset");
  BWD_CUDA(cudaMemsetAsync(b->qbar, 0, sizeof(double) * h->T, h->stream), "memset");
  BWD_CUDA(cudaMemsetAsync(b->zetabar, 0, sizeof(double) * h->T * dimA, h->stream), "memset");
  BWD_CUDA(cudaMemsetAsync(b->xibar, 0, sizeof(double) * h->R * dimA, h->stream), "memset");
  BwdArgs A{};
  A.stored = b->stored;
  A.pend = b->pend;
  A.col_meas = h->col_meas;
  A.chunk_begin = b->chunk_begin;
  A.meas_chunk = b->meas_chunk;
  A.zeta = b->zeta;
  A.xi = b->xi;
  A.alpha = h->alpha_d;
  A.Sd = h->Sd_d;
  A.inv_S = h->invS_d;
  A.a = h->a_d;
  A.part = b->part;
  A.pend_f = b->pend_f;
  A.red = b->red;
  A.acc_prev = b->acc_prev;
  A.qbar = b->qbar;
  A.zetabar = b->zetabar;
  A.xibar = b->xibar;
  A.Mtot = h->Mtot;
  A.R = h->R;
  A.ld = h->ld;
  A.dim = dim;
  A.rho = h->rho[0];
  A.mw = (h->ld + 31) / 32;
  const size_t Tm = size_t(h->T) * A.mw;
  bool have_next = false;  // the step after the segment exists (its sets are in mask_next)
  if (b->all_masks)
    for (int k = b->K - 1; k >= 0; --k) {
      A.am = b->mask_all + Tm * size_t(k);
      A.nm = k + 1 < b->K ? b->mask_all + Tm * size_t(k + 1) : nullptr;
      BWD_CUDA(launch_bwd_step(b->nchunks, h->stream, A), "adjoint step");
    }
  for (int seg = b->all_masks ? -1 : b->nseg - 1; seg >= 0; --seg) {
    BWD_TRY(restore(h, seg));
    const int L = std::min(b->ck, b->K - seg * b->ck);
    // Re-run the segment; the column kernels record each step's active sets.
    for (int j = 0; j < L; ++j) {
      h->amask = b->mask_seg + Tm * j;
      const mam_status st = launch_iteration(h, false);
      h->amask = nullptr;
      BWD_TRY(st);
    }
    for (int j = L - 1; j >= 0; --j) {
      A.am = b->mask_seg + Tm * j;
      A.nm = j + 1 < L ? b->mask_seg + Tm * (j + 1) : (have_next ? b->mask_next : nullptr);
      BWD_CUDA(launch_bwd_step(b->nchunks, h->stream, A), "adjoint step");
    }
    BWD_CUDA(cudaMemcpyAsync(b->mask_next, b->mask_seg, sizeof(unsigned) * Tm,
                             cudaMemcpyDeviceToDevice, h->stream),
             "active-set copy");
    have_next = true;
  }
  if (h->theta0_mode == 0) BWD_CUDA(launch_bwd_theta0(h->T, h->stream, A), "adjoint theta0");
  std::vector<double> qb(h->T), zb(size_t(h->T) * dimA), xb(size_t(h->R) * dimA);
  BWD_CUDA(cudaMemcpyAsync(qb.data(), b->qbar, sizeof(double) * qb.size(),
                           cudaMemcpyDeviceToHost, h->stream),
           "grad q download");
  BWD_CUDA(cudaMemcpyAsync(zb.data(), b->zetabar, sizeof(double) * zb.size(),
                           cudaMemcpyDeviceToHost, h->stream),
           "grad zeta download");
  BWD_CUDA(cudaMemcpyAsync(xb.data(), b->xibar, sizeof(double) * xb.size(),
                           cudaMemcpyDeviceToHost, h->stream),
           "grad xi download");
  BWD_TRY(restore(h, b->nseg));
  BWD_TRY(sync(h));
  const long long U = h->unpruned_off[h->Mtot];
  if (grad_q) {
    std::fill(grad_q, grad_q + U, 0.0);
    for (long long c = 0; c < h->T; ++c) grad_q[h->keep[c]] = qb[c];
  }
  if (grad_zeta) {
    std::fill(grad_zeta, grad_zeta + U * h->dim, 0.0);
    for (long long c = 0; c < h->T; ++c)
      for (int k = 0; k < h->dim; ++k) grad_zeta[h->keep[c] * h->dim + k] = zb[c * h->dim + k];
  }
  if (grad_xi)
    for (size_t i = 0; i < size_t(h->R) * h->dim; ++i) grad_xi[i] = xb[i];
  return MAM_OK;
}

}  // extern "C"
