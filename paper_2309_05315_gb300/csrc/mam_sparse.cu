// libmam device code for the sparse plan layout (MAM_PLAN_SPARSE) of the
// Method of Averaged Marginals (arXiv 2309.05315, Algorithm 1).
//
// Every column step sets theta' = pihat - d (Algorithm 1, Step 2), where
// pihat is the projection onto the simplex Delta_R(q_s) (Prop. 3) and is zero
// off its active set.  So a column of theta is held as the (row, value) pairs
// of its last pihat, plus the shift d of its measure's last column step
// (d_last, written by the averaging kernel); a column never visited holds
// theta^0.  The stored FP32 values are those of the dense layout: the dense
// commit stores fl(pihat_r - d_r), and fl(pihat_r + fl(0 - d_r)) is the same
// number (negation is exact), 0 - d_r on an inactive row.
//
//   column_kernel<..., SP = true>   (mam_column.cuh) the column step
//   init_sparse_kernel              theta^0: count -1, the theta^0 value, lam NaN
//   expand_sparse_kernel            theta of a column range, dense [ncols][R]
#include "mam_column.cuh"

namespace mam {
namespace {

// theta^0 of Step 0 ("Initialization" leaves it arbitrary): mode 0 holds
// q_s / R on every row (rounded once to FP32), mode 1 holds 0.  The thresholds
// become unknown (NaN) unless lam is null.
__global__ void init_sparse_kernel(int* cnt, float* th0, float* lam, const double* q,
                                   long long T, int R, int mode) {
  for (long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x; col < T;
       col += (long long)gridDim.x * blockDim.x) {
    cnt[col] = -1;
    th0[col] = mode == 0 ? float(q[col] / double(R)) : 0.f;
    if (lam) lam[col] = __int_as_float(0x7fc00000);
  }
}

// out[j][r] = theta_{r, col0 + j}, r < R: a block per column (grid-stride).
// Pass 1 writes the inactive value 0 - d_last_r (or theta^0), pass 2 adds
// pihat on the stored rows; the barrier between them orders the block's own
// global writes.
__global__ void expand_sparse_kernel(float* out, long long col0, long long ncols,
                                     const int* cnt, const int2* pairs, int K,
                                     const float* d_last, const float* th0,
                                     const int* col_meas, int R, int ld) {
  for (long long j = blockIdx.x; j < ncols; j += gridDim.x) {
    const long long col = col0 + j;
    const int n = cnt[col];
    float* o = out + size_t(j) * R;
    const float* dl = d_last + size_t(col_meas[col]) * ld;
    const float v0 = th0[col];
    for (int r = threadIdx.x; r < R; r += blockDim.x) o[r] = n < 0 ? v0 : 0.f - dl[r];
    __syncthreads();
    const int2* pr = pairs + size_t(col) * K;
    for (int i = threadIdx.x; i < n && i < K; i += blockDim.x) {
      const int2 e = pr[i];
      if ((unsigned)e.x < (unsigned)R) o[e.x] = __int_as_float(e.y) + (0.f - dl[e.x]);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_column_sparse(int nv, int cost_dtype, bool diag, int grid, int threads,
                                 size_t smem, cudaStream_t st, const ColArgs& a) {
  return col_op_any<true>(nv, cost_dtype, 0, diag, grid, threads, smem, st, &a, nullptr);
}

cudaError_t set_column_sparse_smem(int nv, int cost_dtype, bool diag, size_t smem) {
  return col_op_any<true>(nv, cost_dtype, 1, diag, 0, 0, smem, nullptr, nullptr, nullptr);
}

cudaError_t column_sparse_occupancy(int nv, int cost_dtype, bool diag, int threads,
                                    size_t smem, int* blocks_per_sm) {
  return col_op_any<true>(nv, cost_dtype, 2, diag, 0, threads, smem, nullptr, nullptr,
                          blocks_per_sm);
}

cudaError_t launch_init_sparse(int* cnt, float* th0, float* lam, const double* q,
                               long long T, int R, int mode, cudaStream_t st) {
  long long g = (T + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  init_sparse_kernel<<<int(g), 256, 0, st>>>(cnt, th0, lam, q, T, R, mode);
  return cudaGetLastError();
}

cudaError_t launch_expand_sparse(float* out, long long col0, long long ncols, const int* cnt,
                                 const int2* pairs, int K, const float* d_last,
                                 const float* th0, const int* col_meas, int R, int ld,
                                 cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  long long g = ncols < 152 * 8 ? ncols : 152 * 8;
  expand_sparse_kernel<<<int(g), 256, 0, st>>>(out, col0, ncols, cnt, pairs, K, d_last, th0,
                                               col_meas, R, ld);
  return cudaGetLastError();
}

}  // namespace mam
