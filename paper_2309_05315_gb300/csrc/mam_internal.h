// Internal declarations shared by the translation units of libmam.
// Nothing here is part of the public C ABI (include/mam.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mam {

// Work schedule of one index set M^k (all measures, or one bundle of
// Remark 2).  The index set's columns are contiguous in the global column
// order; CTA b of the persistent grid takes a contiguous slice of them.  The
// slice is cut at measure boundaries into segments; each segment owns one
// row of the partial row-sum buffer ("slot").  Slots of one measure are
// consecutive, so Step 3 (p^(m) = row sums of theta^(m)) sums
// partials[slot_begin[m] .. slot_end[m]) in a fixed order.
struct Sched {
  const int* cta_seg_begin;  // [G+1] first segment of each CTA
  const int4* segs;          // [nseg] (measure, col_begin, col_end, slot)
  const int* slot_begin;     // [Mtot] first slot of measure m (or 0)
  const int* slot_end;       // [Mtot] one past the last slot (== begin: none)
  long long col_begin;       // index set's first column
  long long col_end;         // one past its last column
};

// Arguments of the fused column kernel (Algorithm 1, Step 2 + Step 3
// partials, plus the fused diagnostics).
struct ColArgs {
  float* theta;              // [T][ld] plans, column-contiguous
  const void* cost;          // [T][ld] costs (float / bf16 / half)
  const float* q;            // [T] kept weights q_s (the simplex masses)
  float* lam;                // [T] last threshold lambda_s (NaN: none)
  const double* delta;       // [Mtot][R] (p - p^(m)) / S_m
  const double* t;           // [P] t^k
  const int* meas_prob;      // [Mtot] problem of each measure
  const float* rho;          // [Mtot] rho of the measure's problem
  const float* inv_rho;      // [Mtot] 1/rho
  float* partials;           // [nslot][ld] row sums of the new theta
  const Sched* sched;        // [n_sched] device array of schedules
  const int* bundle_cur;     // index of the schedule to run (device), or null
  float* diag_wc;            // [T] sum_r c_rs pi-hat_rs          (DIAG)
  float* diag_lb;            // [T] q_s * min_r (c_rs - rho d_r)  (DIAG)
  float* diag_res;           // [T] sum_r (theta'_rs - theta_rs)^2 (DIAG)
  unsigned long long* passes;// [1] threshold-search passes (summed)
  int* err;                  // [1] device error word (0 = ok)
  int R;                     // rows
  int ld;                    // padded column stride (multiple of 8)
  int stages;                // TMA pipeline depth
  int bisect_depth;          // bisection steps on a cold start
};

// Arguments of the averaging kernel (Algorithm 1, Step 1, t^k, and Step 3
// reduction of the partial row sums).
struct AvgArgs {
  int P, R, ld;
  const int* prob_meas;      // [P+1] first measure of each problem
  const int* S;              // [Mtot] pruned support sizes
  const double* a;           // [Mtot] averaging weights of eq. (pr)
  const double* rho;         // [P]
  const double* gamma;       // [P] (inf = balanced)
  const float* partials;
  const Sched* sched;
  const int* bundle_cur;     // bundle of the column step just done (or null)
  int* bundle_prev;          // receives that bundle (or null)
  int reduce;                // 1: p^(m) from partials; 0: p^(m) given
  int diag;                  // 1: also pi-hat marginals and their distance
  double* pm;                // [Mtot][R]
  double* p;                 // [P][R]
  double* delta;             // [Mtot][R]
  double* phat;              // [Mtot][R] row sums of pi-hat (DIAG)
  double* t;                 // [P] in: t of the step done; out: next t
  double* blk;               // [P][nblk][4] block partial sums
  unsigned* counter;         // [P] arrival counters (self-resetting)
  double* stat;              // [P][4] (dist_L(theta), dist_L(pi-hat), ||dp||, t used)
  // Remark 2 (single randomized problem; nb <= 1 otherwise)
  int nb;
  const double* bundle_cum;  // [nb] cumulative draw probabilities
  unsigned long long seed;
  long long* iter;           // [1] completed column steps
  int* bundle_next;          // [1] bundle of the next column step
};

// Launch helpers (mam_kernels.cu).
cudaError_t launch_column(int nv, int cost_dtype, bool diag, int grid, int threads,
                          size_t smem, cudaStream_t st, const ColArgs& a);
cudaError_t set_column_smem(int nv, int cost_dtype, bool diag, size_t smem);
int column_max_threads(int nv);
cudaError_t column_occupancy(int nv, int cost_dtype, bool diag, int threads,
                             size_t smem, int* blocks_per_sm);
cudaError_t launch_average(const AvgArgs& a, int nblk, cudaStream_t st);
cudaError_t launch_build_cost(int cost_dtype, void* cost, const double* xi,
                              const double* zeta, const double* gen_cost,
                              const int* col_meas, const double* alpha,
                              long long col0, long long ncols, int R, int ld,
                              int dim, cudaStream_t st);
cudaError_t launch_init_theta(float* theta, float* lam, const double* q,
                              long long T, int R, int ld, int mode,
                              cudaStream_t st);
cudaError_t launch_rowsum(const float* theta, const long long* col_off,
                          int Mtot, int R, int ld, double* pm, cudaStream_t st);
cudaError_t launch_diag_reduce(const float* wc, const float* lb,
                               const float* res, const long long* prob_cols,
                               const Sched* sched, const int* bundle_prev,
                               int P, double* out, cudaStream_t st);

cudaError_t launch_lb(int cost_dtype, const void* cost, const float* q,
                      const double* delta, const double* t,
                      const int* meas_prob, const float* rho,
                      const int* col_meas, long long T, int R, int ld,
                      float* diag_lb, cudaStream_t st);

constexpr int kRedSlots = 32;  // warps per CTA, max

}  // namespace mam
