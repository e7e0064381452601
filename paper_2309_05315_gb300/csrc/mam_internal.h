// Internal declarations shared by the translation units of libmam.
// Nothing here is part of the public C ABI (include/mam.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mam {

// One index set M^k (all measures, or one bundle of Remark 2): its columns
// and its measures are contiguous.  CTA b of the persistent grid of G CTAs
// takes columns [col_begin + n*b/G, col_begin + n*(b+1)/G), n = col_end -
// col_begin.
struct Sched {
  long long col_begin;
  long long col_end;
  int meas_begin;
  int meas_end;
};

// Remark 2 draws: the index set of column step k is a pure function of
// (seed, k), so every kernel that needs it recomputes it from the device
// iteration counter.
struct Draw {
  int nb;                    // bundles (<= 1: deterministic, index set 0)
  const double* cum;         // [nb] cumulative probabilities
  unsigned long long seed;
};

// Arguments of the fused column kernel (Algorithm 1, Step 2, the Step 3
// accumulation of row sums, t^k, and the fused diagnostics).
struct ColArgs {
  float* theta;              // [T][ld] plans, column-contiguous (dense layout)
  const void* cost;          // [T][ld] costs (float / bf16 / half), or [S][ld] shared
  const int* cost_col;       // [T] cost column of each plan column (shared layout), or null
  const float* cmul;         // [Mtot] factor of the stored cost: alpha_m (shared), else 1
  const float* gen_xi;       // generated costs: [P][3][ld] coordinate planes of xi
                             // (x, y, z; planes past dim and rows past R are 0), else null
  const float4* gen_zeta;    // generated costs: [T] points (x, y, z, eta) of the columns
  int gen_dim;               // coordinates used (1..3)
  const float* q;            // [T] kept weights q_s (the simplex masses)
  float* lam;                // [T] last threshold lambda_s (NaN: none)
  const int* col_meas;       // [T] measure of each column
  const long long* col_off;  // [Mtot+1] first column of each measure
  const float* delta32;      // [Mtot][ld] (p - p^(m)) / S_m in FP32, zero past R
  unsigned* amask;           // optional [T][mw] active-set bits (row r: word r/32, bit r%32)
  int mw;                    // 32-bit words per column of amask
  const double* blk;         // [P][nblk][4] averaging block sums (dist^2 in [0])
  int nblk;
  const double* rho_p;       // [P]
  const double* gamma_p;     // [P] (inf = balanced)
  double* t_used;            // [P] t^k used by this step (written)
  const int* meas_prob;      // [Mtot] problem of each measure
  const float* rho;          // [Mtot] rho of the measure's problem
  const float* inv_rho;      // [Mtot] 1/rho
  unsigned long long* acc;   // [Mtot][R] fixed-point row sums of pi-hat
  float fx_scale;            // fixed-point scale 2^e of acc
  const Sched* sched;        // [n_sched] index sets (device)
  Draw draw;
  long long* iter;           // [1] completed column steps (advanced here)
  unsigned* done;            // [1] CTA arrival counter (self-resetting)
  float* diag_wc;            // [T] sum_r c_rs pi-hat_rs          (DIAG)
  float* diag_lb;            // [T] q_s * min_r (c_rs - rho d_r)  (DIAG)
  float* diag_res;           // [T] sum_r (theta'_rs - theta_rs)^2 (DIAG)
  unsigned long long* passes;// [1] threshold-search passes (summed)
  int* err;                  // [1] device error word (0 = ok)
  int R;                     // rows
  int ld;                    // padded column stride (multiple of 8)
  int stages;                // TMA pipeline depth
  int bisect_depth;          // bisection steps on a cold start
  float lam_floor;           // lower clamp of the applied threshold: -inf, or 0
                             // for capped columns (projection onto Delta_<=(q_s))
  float lb_cap;              // upper clamp of a column's lower-bound term per unit
                             // mass: +inf, or 0 for capped columns
  // Sparse plan layout (theta = pihat - d_last, pihat as pairs; else unused)
  int* sp_cnt;               // [T] stored pairs of each column (-1: theta^0)
  int2* sp_pairs;            // [T][sp_k] (row, FP32 bits of pihat_r)
  const float* d_last;       // [Mtot][ld] d of each measure's last column step
  const float* th0;          // [T] theta^0 of each column on rows < R
  int sp_k;                  // pair slots per column (even)
};

// Arguments of the averaging kernel (Algorithm 1, Step 3 completion, Step 1
// and the distance that fixes t^k).
// Marginals are 64-bit fixed point with the scale F = 2^e of the row-sum
// accumulators: integer adds and products are exact and order-independent,
// and the FP64 pipe (a small fraction of the FP32 rate on this GPU) is left
// to per-row work.
struct AvgArgs {
  int P, R;
  const int* prob_meas;      // [P+1] first measure of each problem
  const int* S;              // [Mtot] pruned support sizes S_m
  const float* inv_S;        // [Mtot] 1 / S_m
  const double* inv_SFd;     // [Mtot] 1 / (S_m F) in FP64 (the shifts' one product)
  const long long* a_q;      // [Mtot] round(a_m 2^62), weights of eq. (pr)
  const double* a;           // [Mtot] a_m (diagnostics)
  const double* inv_Sd;      // [Mtot] 1 / S_m in FP64 (diagnostics)
  unsigned long long* acc;   // [Mtot][R] fixed-point sums of pi-hat (zeroed here)
  float fx_f;                // F
  float fx_inv_f;            // 1 / F
  double fx_inv_scale;       // 1 / F
  const Sched* sched;
  Draw draw;
  const long long* iter;     // [1] completed column steps
  const double* t_used;      // [P] t of the column step just done
  int reduce;                // 1: p^(m) from acc; 0: p^(m) given
  int diag;                  // 1: also pi-hat marginals and their distance
  long long* pm;             // [Mtot][R] p^(m) F
  double* p;                 // [P][R]
  float* delta32;            // [Mtot][ld] (p - p^(m)) / S_m, read by the column kernels
  int ld;
  double* phat;              // [Mtot][R] row sums of pi-hat (DIAG)
  double* blk;               // [P][nblk][4] block sums: dist^2, dist_hat^2, |dp|^2
  int slices;                // measure slices per block (1, 2, 4, 8)
  float* d_last;             // [Mtot][ld] sparse plans: d of each updated measure's
                             // column step (written), else null
};

constexpr int kAvgThreads = 128;  // threads per averaging block: rows x measure slices
constexpr int kAvgGroup = 4;      // measures whose loads an averaging thread batches
constexpr int kAvgKeep = 16;      // marginals an averaging thread keeps in registers

// Launch helpers (mam_kernels.cu).
cudaError_t launch_column(int nv, int cost_dtype, bool diag, int grid, int threads,
                          size_t smem, cudaStream_t st, const ColArgs& a);
cudaError_t set_column_smem(int nv, int cost_dtype, bool diag, size_t smem);
int column_max_threads(int nv);
cudaError_t column_occupancy(int nv, int cost_dtype, bool diag, int threads,
                             size_t smem, int* blocks_per_sm);
cudaError_t launch_average(const AvgArgs& a, int nblk, cudaStream_t st);
// The sparse plan layout (mam_sparse.cu).
cudaError_t launch_column_sparse(int nv, int cost_dtype, bool diag, int grid, int threads,
                                 size_t smem, cudaStream_t st, const ColArgs& a);
cudaError_t set_column_sparse_smem(int nv, int cost_dtype, bool diag, size_t smem);
cudaError_t column_sparse_occupancy(int nv, int cost_dtype, bool diag, int threads,
                                    size_t smem, int* blocks_per_sm);
cudaError_t launch_init_sparse(int* cnt, float* th0, float* lam, const double* q,
                               long long T, int R, int mode, cudaStream_t st);
cudaError_t launch_expand_sparse(float* out, long long col0, long long ncols, const int* cnt,
                                 const int2* pairs, int K, const float* d_last,
                                 const float* th0, const int* col_meas, int R, int ld,
                                 cudaStream_t st);
// One warp per column with a shared-memory ring (mam_warp_kernel.cu).
bool ring_kernel_has(int nv);
int ring_kernel_max_threads(int nv);
size_t ring_kernel_smem(int nv, int slots, int cost_bytes);
cudaError_t launch_column_ring(int nv, int cost_dtype, bool diag, int grid, int threads,
                               size_t smem, cudaStream_t st, const ColArgs& a);
cudaError_t set_column_ring_smem(int nv, int cost_dtype, bool diag, size_t smem);
cudaError_t column_ring_occupancy(int nv, int cost_dtype, bool diag, int threads,
                                  size_t smem, int* blocks_per_sm);
// One column per thread-block cluster of cs CTAs (mam_cluster_kernel.cu),
// for columns longer than one CTA holds.
int cluster_rows_per_cta(int ld, int cs);
size_t cluster_kernel_smem(int ld, int cs);
cudaError_t launch_column_cluster(int cost_dtype, bool diag, int cs, int grid, int threads,
                                  size_t smem, cudaStream_t st, const ColArgs& a);
cudaError_t set_column_cluster_smem(int cost_dtype, bool diag, size_t smem);
cudaError_t column_cluster_occupancy(int cost_dtype, bool diag, int cs, int threads,
                                     size_t smem, int* clusters);
// Squared-Euclidean costs from per-coordinate tables (mam_setup.cu): when
// the points take few distinct values per coordinate (pixel grids), the
// table of coordinate k holds fl(fl(zv_u - xv_v)^2) for every pair of
// distinct values, [nz_k][nx_k] from element off[k] of one FP64 buffer; a
// cost entry is then the same FP64 sum of the same squares the direct formula
// forms.
struct CostTab {
  int dim;
  long long off[3];  // first element of each coordinate's table
  int nx[3];         // distinct barycenter-point values of each coordinate
};
cudaError_t launch_sqdiff_table(double* tab, const double* uz, int nz, const double* ux,
                                int nx, cudaStream_t st);
// cols (optional): the columns to build, [ncols], in place of col0 + j.
cudaError_t launch_build_cost_tab(int cost_dtype, void* cost, const double* tab,
                                  const CostTab& tb, const int* ix, const int* iz,
                                  const int* col_meas, const double* alpha, const double* eta,
                                  long long col0, long long ncols, int R, int ld,
                                  cudaStream_t st, const long long* cols = nullptr);
// Copies cost column src to dst for every pair of dst_src [n][2].
cudaError_t launch_copy_cost_columns(int cost_dtype, void* cost, const long long* dst_src,
                                     long long n, int ld, cudaStream_t st);
cudaError_t launch_build_cost(int cost_dtype, void* cost, const double* xi,
                              const double* zeta, const double* gen_cost,
                              const int* col_meas, const double* alpha,
                              const double* eta, long long col0, long long ncols,
                              int R, int ld, int dim, cudaStream_t st,
                              const long long* cols = nullptr);
cudaError_t launch_init_theta(float* theta, float* lam, const double* q,
                              long long T, int R, int ld, int mode,
                              cudaStream_t st);
cudaError_t launch_rowsum_theta0(const double* q, const long long* col_off, int Mtot, int R,
                                 int mode, double fx_scale, long long* pm, cudaStream_t st);
cudaError_t launch_diag_reduce(const float* wc, const float* lb,
                               const float* res, const long long* prob_cols,
                               const Sched* sched, Draw draw,
                               const long long* iter, int P, double* out,
                               cudaStream_t st);

cudaError_t launch_lb(int cost_dtype, const void* cost, const int* cost_col,
                      const float* cmul, const float* gen_xi, const float4* gen_zeta,
                      const float* q,
                      const float* delta32, const double* t_used,
                      const int* meas_prob, const float* rho,
                      const int* col_meas, long long T, int R, int ld,
                      float lb_cap, float* diag_lb, cudaStream_t st);

// out[i] = in[i] * scale (fixed-point marginals to FP64).
cudaError_t launch_fx_to_double(const long long* in, size_t n, double scale, double* out,
                                cudaStream_t st);

constexpr int kRedSlots = 32;  // warps per CTA, max


// Reverse sweep through one balanced, deterministic iteration
// (mam_backward_kernels.cu).  thetabar = stored (column-sparse) + pend
// (broadcast along the columns of each measure).  Columns are processed in
// chunks of consecutive columns of one measure.
constexpr int kBwdChunk = 16;  // columns per chunk (at most)
struct BwdArgs {
  const unsigned* am;            // [T][mw] active-set bits of the step
  const unsigned* nm;            // [T][mw] active-set bits of the step after, or
                                 // nullptr (the stored part entering is zero)
  int mw;                        // words per column
  float* stored;                 // [T][ld] sparse part of thetabar (in: k+1, out: k)
  double* pend;                  // [Mtot][R] broadcast part of thetabar
  const int* col_meas;           // [T]
  const long long* chunk_begin;  // [nchunks + 1] first column of each chunk
  const int* meas_chunk;         // [Mtot + 1] first chunk of each measure
  const double* zeta;            // [T][dim] kept support points
  const double* xi;              // [R][dim]
  const double* alpha;           // [Mtot]
  const double* Sd;              // [Mtot]
  const double* inv_S;           // [Mtot] 1 / S_m
  const double* a;               // [Mtot]
  float* part;                   // [nchunks][1 + dim][R] chunk row sums of wbar, wbar zeta
  float* pend_f;                 // [Mtot][R] FP32 copy of pend for the column step
  double* red;                   // [Mtot][1 + dim][R] chunk sums added per measure
  double* acc_prev;              // [Mtot][R] sum_s wbar_rs of the step after (k+1)
  double* qbar;                  // [T]
  double* zetabar;               // [T][dim]
  double* xibar;                 // [R][dim]
  int Mtot, R, ld, dim;
  double rho;
};

cudaError_t launch_bwd_step(int nchunks, cudaStream_t st, const BwdArgs& a);
cudaError_t launch_bwd_theta0(long long T, cudaStream_t st, const BwdArgs& a);

}  // namespace mam
