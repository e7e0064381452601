// libmam: reverse mode through unrolled MAM iterations (balanced,
// deterministic, t = 1).
//
// One forward iteration (Algorithm 1) maps theta to theta' by
//   d^(m) = (p - p^(m)) / S_m,  p^(m) = row sums of theta^(m),  p = sum a_m p^(m)
//   w = theta + 2 d - c / rho,  pihat = max(w - lambda, 0) with
//   sum_r pihat = q_s,  theta' = pihat - d.
// Where the active sets A_s = {r : w_r > lambda_s} do not change, pihat is
// affine in (w, q): d pihat / d w = I_A - 1_A 1_A^T / |A| and
// d pihat / d q_s = 1_A / |A|.  Given thetabar' (the gradient w.r.t. theta')
// the reverse step is
//   wbar = [A] (thetabar' - mean_A thetabar'),   qbar_s += mean_A thetabar',
//   cbar = -wbar / rho,   dbar^(m)_r = sum_s (2 wbar_rs - thetabar'_rs),
//   pbar = sum_m dbar^(m) / S_m,   pbarm^(m) = -dbar^(m) / S_m + a_m pbar,
//   thetabar = wbar + pbarm^(m) broadcast along each column,
// and the cost c^(m)_rs = alpha_m ||xi_r - zeta_s||^2 gives
//   zetabar_s += (2 alpha_m / rho) sum_r wbar_rs (xi_r - zeta_s),
//   xibar_r   -= (2 alpha_m / rho) sum_s wbar_rs (xi_r - zeta_s).
// thetabar is kept as a column-sparse part ("stored": wbar, zero off the
// active set) plus a per-(measure,row) part ("pend": pbarm).  Since the stored
// part entering step k is the wbar of step k+1, sum_s thetabar'_rs =
// (sum_s wbar^(k+1)_rs) + S_m pend_r: the row sums of one step are reused by
// the next.
//
// The reverse step needs of the forward step only its active sets.  The
// forward column kernels, re-run over a checkpoint segment, write them as
// bit masks (row r of a column: word r / 32, bit r % 32), so the reverse step
// reads no plan iterate and no cost: it touches the stored part only where
// the step's active set or the next step's (the only rows where the stored
// part can be nonzero) has a bit.
//
// Layout of the work: a CTA owns a chunk of consecutive columns of one
// measure, one warp per column (bwd_column_kernel); then a thread owns one
// row of a chunk and adds its columns in order (bwd_chunk_rowsum_kernel);
// the chunks of a measure are added in a fixed order
// (bwd_chunk_reduce_kernel).  No atomics, so the result does not depend on
// scheduling.
#include "mam_device.cuh"
#include "mam_internal.h"

namespace mam {
namespace {

template <int N, typename V>
__device__ __forceinline__ void block_sum_n(V (&v)[N], V (*sh)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  __syncthreads();  // the previous call's readers are done
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < N; ++j) sh[warp][j] = v[j];
  }
  __syncthreads();
  const int nw = int(blockDim.x >> 5);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    V t = V(0);
    for (int w = 0; w < nw; ++w) t += sh[w][j];
    v[j] = t;
  }
}

constexpr int kBwdWarps = 8;

// One reverse step over the columns of chunk blockIdx.x, one warp per column.
// Lane l visits rows r = 32 v + l.  Per-entry arithmetic is FP32 (the FP64
// pipe of this GPU is a small fraction of its FP32 rate); per-column results
// are accumulated in FP64.
__global__ void __launch_bounds__(kBwdWarps * 32) bwd_column_kernel(const BwdArgs A) {
  extern __shared__ float pd_s[];  // [R] broadcast part of thetabar, this measure
  const int R = A.R, ld = A.ld, dim = A.dim, mw = A.mw;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long c0 = A.chunk_begin[blockIdx.x], c1 = A.chunk_begin[blockIdx.x + 1];
  const int m = A.col_meas[c0];
  for (int i = tid; i < R; i += blockDim.x) pd_s[i] = A.pend_f[size_t(m) * R + i];
  __syncthreads();
  const double coef = 2.0 * A.alpha[m] / A.rho;
  const unsigned bit = 1u << lane;
  for (long long col = c0 + warp; col < c1; col += kBwdWarps) {
    const unsigned* am = A.am + size_t(col) * mw;
    const unsigned* nm = A.nm ? A.nm + size_t(col) * mw : nullptr;
    float* st = A.stored + size_t(col) * ld;
    // mean of thetabar' over the active set; the stored part is zero off the
    // next step's active set.  Active sets are sparse: the lanes load 32 mask
    // words at a time and the warp visits only the nonzero ones (a ballot).
    float s1 = 0.f, na = 0.f;
    for (int v0 = 0; v0 < mw; v0 += 32) {
      const bool in = v0 + lane < mw;
      const unsigned aw = in ? am[v0 + lane] : 0u;
      const unsigned bw = (in && nm) ? nm[v0 + lane] : 0u;
      unsigned live = __ballot_sync(0xffffffffu, aw != 0u);
      while (live) {
        const int j = __ffs(live) - 1;
        live &= live - 1;
        const unsigned a = __shfl_sync(0xffffffffu, aw, j);
        const unsigned b = __shfl_sync(0xffffffffu, bw, j);
        if (a & bit) {
          const int r = 32 * (v0 + j) + lane;
          const float so = (b & bit) ? st[r] : 0.f;
          s1 += so + pd_s[r];
          na += 1.f;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      na += __shfl_xor_sync(0xffffffffu, na, o);
    }
    const float mean = na > 0.f ? s1 / na : 0.f;
    float zs[3] = {0.f, 0.f, 0.f}, zx[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < dim) zs[k] = float(A.zeta[size_t(col) * dim + k]);
    // wbar on the active set; zeros where the stored part was nonzero (the
    // words of either set, visited as above)
    for (int v0 = 0; v0 < mw; v0 += 32) {
      const bool in = v0 + lane < mw;
      const unsigned aw = in ? am[v0 + lane] : 0u;
      const unsigned bw = (in && nm) ? nm[v0 + lane] : 0u;
      unsigned live = __ballot_sync(0xffffffffu, (aw | bw) != 0u);
      while (live) {
        const int j = __ffs(live) - 1;
        live &= live - 1;
        const unsigned a = __shfl_sync(0xffffffffu, aw, j);
        const unsigned b = __shfl_sync(0xffffffffu, bw, j);
        if ((a | b) & bit) {
          const int r = 32 * (v0 + j) + lane;
          if (a & bit) {
            const float so = (b & bit) ? st[r] : 0.f;
            const float wb = (so + pd_s[r]) - mean;
            st[r] = wb;
#pragma unroll
            for (int k = 0; k < 3; ++k)
              if (k < dim)
                zx[k] = fmaf(wb, float(__ldg(A.xi + size_t(r) * dim + k)) - zs[k], zx[k]);
          } else {
            st[r] = 0.f;
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < dim)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) zx[k] += __shfl_xor_sync(0xffffffffu, zx[k], o);
    if (lane == 0) {
      A.qbar[col] += double(mean);
      for (int k = 0; k < dim; ++k) A.zetabar[size_t(col) * dim + k] += coef * double(zx[k]);
    }
  }
}

// Per-row sums of one chunk's new stored part: part[chunk][0][r] = sum_s
// wbar_rs, part[chunk][1 + k][r] = sum_s wbar_rs zeta_s[k], the columns added
// in order.  Grid (chunk, row block): one thread per row; wbar is zero off the
// step's active set, so only rows with a mask bit are read.
constexpr int kRsThreads = 128;
__global__ void __launch_bounds__(kRsThreads) bwd_chunk_rowsum_kernel(const BwdArgs A) {
  const long long c0 = A.chunk_begin[blockIdx.x], c1 = A.chunk_begin[blockIdx.x + 1];
  const int R = A.R, ld = A.ld, dim = A.dim, mw = A.mw;
  const int r = blockIdx.y * kRsThreads + threadIdx.x;
  if (r >= R) return;
  const int nc = int(c1 - c0);  // <= kBwdChunk
  const unsigned bit = 1u << (r & 31);
  // the chunk's mask words of this row, loaded together
  unsigned wd[kBwdChunk];
#pragma unroll
  for (int j = 0; j < kBwdChunk; ++j) wd[j] = j < nc ? A.am[size_t(c0 + j) * mw + (r >> 5)] : 0u;
  float sw = 0.f, sz[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < kBwdChunk; ++j) {
    if (wd[j] & bit) {
      const long long col = c0 + j;
      const float wb = A.stored[size_t(col) * ld + r];
      sw += wb;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k < dim) sz[k] = fmaf(wb, float(__ldg(A.zeta + size_t(col) * dim + k)), sz[k]);
    }
  }
  float* part = A.part + size_t(blockIdx.x) * (1 + dim) * R;
  part[r] = sw;
  for (int k = 0; k < dim; ++k) part[size_t(1 + k) * R + r] = sz[k];
}

// Sums the chunk partials of each measure in a fixed order:
// red[m][k][r] = sum over the chunks j of measure m of part[j][k][r]
// (k = 0: sum_s wbar_rs, k = 1..dim: sum_s wbar_rs zeta_s).  Compensated
// FP32 summation (Knuth's TwoSum: the rounding error of every addition is
// carried in a second float), so the result keeps about twice the FP32
// precision without FP64 arithmetic.  Block (kRedRows rows) x (kRedSlices
// chunk slices), grid (rows, measures, 1 + dim).
__device__ __forceinline__ void two_sum(float& s, float& c, float x) {
  const float t = s + x;
  const float z = t - s;
  c += (s - (t - z)) + (x - z);
  s = t;
}

constexpr int kRedRows = 32, kRedSlices = 8;
__global__ void __launch_bounds__(kRedRows * kRedSlices) bwd_chunk_reduce_kernel(const BwdArgs A) {
  __shared__ float sh[2][kRedSlices][kRedRows];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = blockIdx.x * kRedRows + tx;
  const int m = blockIdx.y, k = blockIdx.z;
  const int K1 = 1 + A.dim, R = A.R;
  float s = 0.f, c = 0.f;
  if (r < R) {
#pragma unroll 4
    for (int j = A.meas_chunk[m] + ty; j < A.meas_chunk[m + 1]; j += kRedSlices)
      two_sum(s, c, A.part[(size_t(j) * K1 + k) * R + r]);
  }
  sh[0][ty][tx] = s;
  sh[1][ty][tx] = c;
  __syncthreads();
  if (ty == 0 && r < R) {
    float t = 0.f, ct = 0.f;
#pragma unroll
    for (int y = 0; y < kRedSlices; ++y) {
      two_sum(t, ct, sh[0][y][tx]);
      ct += sh[1][y][tx];
    }
    A.red[(size_t(m) * K1 + k) * R + r] = double(t) + double(ct);
  }
}

// Per row r: dbar, pbar, the new broadcast part of thetabar and xibar.
// acc_prev holds sum_s wbar^(k+1)_rs (the stored part entering this step).
// Block (kRowRows rows) x (kRowSlices measure slices): a thread takes the
// measures m = y, y + kRowSlices, ... of its row (at most kRowKeep of them
// kept in registers between the two phases); pbar and the xibar terms are
// added over the slices in shared memory in a fixed order.
constexpr int kRowRows = 32, kRowSlices = 8, kRowKeep = 8;
__global__ void __launch_bounds__(kRowRows * kRowSlices) bwd_row_kernel(const BwdArgs A) {
  __shared__ double sp[kRowSlices][kRowRows];
  __shared__ double sx[3][kRowSlices][kRowRows];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = blockIdx.x * kRowRows + tx;
  const bool row = r < A.R;
  const int dim = A.dim, R = A.R, K1 = 1 + dim;
  double pb = 0.0, xs[3] = {0.0, 0.0, 0.0};
  double dkeep[kRowKeep];
  double xr[3] = {0.0, 0.0, 0.0};
  if (row)
    for (int k = 0; k < dim; ++k) xr[k] = A.xi[size_t(r) * dim + k];
  int q = 0;
  if (row) {
    for (int m = ty; m < A.Mtot; m += kRowSlices, ++q) {
      const size_t o = size_t(m) * R + r;
      const double w = A.red[size_t(m) * K1 * R + r];
      const double dbar = 2.0 * w - (A.acc_prev[o] + A.Sd[m] * A.pend[o]);
      if (q < kRowKeep) dkeep[q] = dbar;
      pb += dbar * A.inv_S[m];
      const double coef = 2.0 * A.alpha[m] / A.rho;
      for (int k = 0; k < dim; ++k)
        xs[k] += coef * (xr[k] * w - A.red[(size_t(m) * K1 + 1 + k) * R + r]);
    }
  }
  sp[ty][tx] = pb;
  for (int k = 0; k < 3; ++k) sx[k][ty][tx] = xs[k];
  __syncthreads();
  double pbar = 0.0;
#pragma unroll
  for (int y = 0; y < kRowSlices; ++y) pbar += sp[y][tx];
  if (row && ty == 0)
    for (int k = 0; k < dim; ++k) {
      double t = 0.0;
      for (int y = 0; y < kRowSlices; ++y) t += sx[k][y][tx];
      A.xibar[size_t(r) * dim + k] -= t;
    }
  if (row) {
    q = 0;
    for (int m = ty; m < A.Mtot; m += kRowSlices, ++q) {
      const size_t o = size_t(m) * R + r;
      const double w = A.red[size_t(m) * K1 * R + r];
      const double dbar = q < kRowKeep ? dkeep[q]
                                       : 2.0 * w - (A.acc_prev[o] + A.Sd[m] * A.pend[o]);
      const double pn = -dbar * A.inv_S[m] + A.a[m] * pbar;
      A.pend[o] = pn;
      A.pend_f[o] = float(pn);
      A.acc_prev[o] = w;
    }
  }
}

// theta^0_rs = q_s / R: qbar_s += sum_r thetabar^0_rs / R.
__global__ void __launch_bounds__(256) bwd_theta0_kernel(const BwdArgs A) {
  __shared__ double sh[8][4];
  const long long col = blockIdx.x;
  const int m = A.col_meas[col];
  double s[1] = {0.0};
  for (int r = threadIdx.x; r < A.R; r += blockDim.x)
    s[0] += double(A.stored[size_t(col) * A.ld + r]) + A.pend[size_t(m) * A.R + r];
  block_sum_n<1, double>(s, sh);
  if (threadIdx.x == 0) A.qbar[col] += s[0] / double(A.R);
}

}  // namespace

cudaError_t launch_bwd_step(int nchunks, cudaStream_t st, const BwdArgs& a) {
  bwd_column_kernel<<<nchunks, kBwdWarps * 32, sizeof(float) * size_t(a.R), st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bwd_chunk_rowsum_kernel<<<dim3(nchunks, (a.R + kRsThreads - 1) / kRsThreads), kRsThreads, 0,
                            st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bwd_chunk_reduce_kernel<<<dim3((a.R + kRedRows - 1) / kRedRows, a.Mtot, 1 + a.dim),
                            dim3(kRedRows, kRedSlices), 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bwd_row_kernel<<<(a.R + kRowRows - 1) / kRowRows, dim3(kRowRows, kRowSlices), 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bwd_theta0(long long T, cudaStream_t st, const BwdArgs& a) {
  bwd_theta0_kernel<<<unsigned(T), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mam
