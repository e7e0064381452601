// The library-owned problem handle (opaque behind include/mam.h) and the
// host helpers shared by libmam's translation units.
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "mam.h"
#include "mam_internal.h"

namespace mam {

constexpr int kGraphIters = 10;   // iterations per captured CUDA graph
constexpr int kMaxCtaR = 12288;   // largest column one CTA covers (threads*vec*4)
constexpr int kMaxR = 786432;     // largest column a cluster of 16 CTAs covers
                                  // (49152 rows of w, 192 KB, per CTA)

struct BackwardState;  // mam_backward.cu

}  // namespace mam

struct mam_problem {
  std::string err;
  bool failed = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, num_sms = 0;

  // sizes and modes
  int P = 1, Mtot = 0, R = 0, ld = 0, dim = 0;
  long long T = 0;
  int cost_dtype = 0, theta0_mode = 0, diag_mode = 0;
  int nb = 1;
  bool capped = false;  // columns projected onto Delta_<=(q_s) (full unbalanced extension)
  unsigned long long seed = 0;
  bool has_gen_cost = false;

  // host tables
  std::vector<int> prob_meas;           // [P+1]
  std::vector<long long> prob_cols;     // [P+1]
  std::vector<int> S, S_unpruned;       // [Mtot]
  std::vector<int> meas_prob_h;         // [Mtot]
  std::vector<long long> col_off;       // [Mtot+1] kept columns
  std::vector<long long> unpruned_off;  // [Mtot+1] unpruned entries
  std::vector<long long> keep;          // [T] unpruned index of each column
  std::vector<double> a;                // [Mtot]
  std::vector<double> rho, gamma, Qa;   // [P]
  std::vector<double> bundle_cum;       // [nb]
  std::vector<std::pair<long long, long long>> index_sets;  // column ranges
  std::vector<std::pair<int, int>> index_meas;              // measure ranges
  double fx_scale = 1.0;                // 2^e of the fixed-point row sums
  std::vector<double> xi_h;             // [P][R][dim]
  std::vector<double> zeta_kept;        // [T][dim] (when available)

  // device buffers (all in `allocs`)
  std::vector<void*> allocs;
  float* theta = nullptr;
  void* cost = nullptr;
  float* q = nullptr;
  double* q64 = nullptr;
  float* lam = nullptr;
  long long* pm = nullptr;  // [Mtot][R] p^(m) in fixed point (scale fx_scale)
  float* delta32 = nullptr;
  double* phat = nullptr;
  double* p = nullptr;
  double* t_used = nullptr;
  unsigned* done = nullptr;
  double* blk = nullptr;
  float* diag_wc = nullptr;
  float* diag_lb = nullptr;
  float* diag_res = nullptr;
  double* diag_out = nullptr;
  unsigned long long* passes = nullptr;
  int* err_d = nullptr;
  int* meas_prob = nullptr;
  float* rho_m = nullptr;
  float* irho_m = nullptr;
  double* a_d = nullptr;
  double* alpha_d = nullptr;
  double* eta_d = nullptr;  // [Mtot] eta of the measure's problem (capped; else 0)
  // free-support step (allocated on first use)
  double* xi_dev = nullptr;               // [R][dim]
  double* zeta_dev = nullptr;             // [T][dim]
  unsigned long long* sup_acc = nullptr;  // [R][dim + 1]
  std::vector<double> alpha_h, Q_h;       // [Mtot] alpha_m and kept mass Q_m
  int* S_d = nullptr;
  double* Sd_d = nullptr;
  double* invS_d = nullptr;
  float* invS_f = nullptr;
  double* invSF_d = nullptr;
  long long* a_q_d = nullptr;
  int* prob_meas_d = nullptr;
  double* rho_d = nullptr;
  double* gamma_d = nullptr;
  long long* col_off_d = nullptr;
  long long* prob_cols_d = nullptr;
  int* col_meas = nullptr;
  double* bundle_cum_d = nullptr;
  long long* iter_d = nullptr;
  unsigned long long* acc = nullptr;

  // schedules and launch configuration
  std::vector<void*> sched_allocs;
  mam::Sched* sched_d = nullptr;
  mam_kernel_config cfg{};
  int grid = 0;
  size_t smem = 0;
  int avg_slices = 8;  // measure slices of the averaging block
  cudaGraphExec_t graph = nullptr;

  // host mirrors
  long long iter = 0;
  long long diag_iter = -1;
  // work done by the column steps since create (mam_get_work)
  long long work_cols = 0;
  long long work_entries = 0;

  // per-kernel timing (mam_profile_enable)
  bool profiling = false;
  std::vector<cudaEvent_t> prof_events;
  size_t prof_used = 0;

  // sparse plan layout (MAM_PLAN_SPARSE): theta = pihat - d_last with pihat
  // held as pairs; no dense theta
  bool sparse = false;
  int sp_k = 0;               // pair slots per column (even)
  int* sp_cnt = nullptr;      // [T] stored pairs of each column (-1: theta^0)
  int2* sp_pairs = nullptr;   // [T][sp_k] (row, FP32 bits of pihat_r)
  float* d_last = nullptr;    // [Mtot][ld] d of each measure's last column step
  float* th0 = nullptr;       // [T] theta^0 of each column (rows < R)

  // generated cost layout (MAM_COST_GENERATED): no stored cost
  bool gen_cost = false;
  float* gen_xi = nullptr;     // [P][3][ld] FP32 coordinate planes (x, y, z)
  float4* gen_zeta = nullptr;  // [T] (x, y, z, eta) FP32
  std::vector<double> eta_h;   // [P] eta of each problem
  std::vector<int> col_meas_h; // [T] measure of each kept column

  // shared cost layout (MAM_COST_SHARED): one matrix C over the common support
  bool shared_cost = false;
  int n_sup = 0;                  // columns of C (points of the common support)
  int* cost_col = nullptr;        // [T] column of C of each plan column
  float* cmul = nullptr;          // [Mtot] alpha_m (shared) or 1: factor of the stored cost
  double* sup_zeta_d = nullptr;   // [n_sup][dim] the common support points
  int* sup_meas_d = nullptr;      // [n_sup] zeros (C is built as one unit-weight measure)
  double* sup_alpha_d = nullptr;  // [1] 1.0
  double* sup_eta_d = nullptr;    // [1] eta

  // measure-sharded problem (mam_create_sharded): measures m_begin ..
  // m_begin + Mtot - 1 of M_global live here
  bool sharded = false;
  int m_begin = 0, M_global = 0;
  mam_allreduce_fn allreduce = nullptr;
  void* ar_user = nullptr;
  long long* exch_i64 = nullptr;  // [R] partial, then global, sum of a_m p^(m) F
  double* exch_f64 = nullptr;     // [R] same for the pi-hat marginals (diagnostics)
  double* blk_glob = nullptr;     // [4] global sums: D^2, D-hat^2, |dp|^2, 0

  mam::BackwardState* bwd = nullptr;
  unsigned* amask = nullptr;  // set during the reverse sweep's recomputation only
};

// Early returns on a failed library call (MAM_TRY) or CUDA call (MAM_CUDA;
// needs the handle `h` in scope).
#define MAM_TRY(x)                     \
  do {                                 \
    mam_status _s = (x);               \
    if (_s != MAM_OK) return _s;       \
  } while (0)

#define MAM_CUDA(x, where)                                 \
  do {                                                     \
    cudaError_t _e = (x);                                  \
    if (_e != cudaSuccess) return mam::cuda_fail(h, _e, where); \
  } while (0)

namespace mam {

mam_status fail(mam_problem* h, mam_status code, const std::string& msg);
mam_status cuda_fail(mam_problem* h, cudaError_t e, const char* where);

// Device allocation recorded in the handle (freed by mam_destroy).
template <typename T>
mam_status dalloc(mam_problem* h, T** ptr, size_t count, const char* what) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MAM_ERR_OOM,
                std::string("cudaMalloc failed for ") + what + " (" +
                    std::to_string(count * sizeof(T)) + " bytes)");
  }
  h->allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return MAM_OK;
}
size_t cost_elem_size(int dt);
mam_status apply_config(mam_problem* h, const mam_kernel_config& c);
mam_status check_config(const mam_problem* h, const mam_kernel_config& c);
mam_kernel_config default_config(const mam_problem* h);
mam_status run_iterations(mam_problem* h, int n, bool diag_last);
mam_status launch_iteration(mam_problem* h, bool diag);
mam_status sync(mam_problem* h);
Draw draw_args(const mam_problem* h);
ColArgs col_args(const mam_problem* h);
AvgArgs avg_args(const mam_problem* h, int reduce, int diag);
int avg_blocks(const mam_problem* h);
size_t column_smem_bytes(const mam_problem* h, const mam_kernel_config& c);
void free_backward(mam_problem* h);

// One device buffer of the iteration state (everything mam_get_state saves).
struct Piece {
  void* dev;
  size_t bytes;
};
std::vector<Piece> state_pieces(mam_problem* h);
mam_status reset_state(mam_problem* h);
mam_status upload_gen_points(mam_problem* h);

// Measure-sharded problems (mam_shard.cu).
int shard_blocks(const mam_problem* h);
mam_status shard_exchange(mam_problem* h, void* buf, long long count, int dtype);
mam_status shard_block_sums(mam_problem* h);
mam_status shard_average(mam_problem* h, int reduce, bool diag);

}  // namespace mam
