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
// the next and no column is read twice.
//
// Layout of the work: a CTA owns a chunk of consecutive columns of one
// measure.  Columns of up to 2048 rows go one per warp (bwd_warp_kernel),
// and bwd_chunk_rowsum_kernel then takes each chunk's per-row sums (sum_s
// wbar_rs and sum_s wbar_rs zeta_s) from the columns just written.  Longer columns go one per
// CTA, a thread owning fixed rows r = tid + i * blockDim.x of every column of
// the chunk, which keeps those sums in registers (bwd_column_kernel).  The
// chunks are then added per measure (bwd_chunk_reduce_kernel).  Every sum is taken
// in a fixed order, without atomics, so the result does not depend on
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

// One reverse step over the columns of chunk blockIdx.x.  Per-entry
// arithmetic is FP32 (the FP64 pipe of this GPU is a small fraction of its
// FP32 rate); per-column and per-row results are accumulated in FP64.
template <int NVB, typename CT, int DIM>
__global__ void __launch_bounds__(kBwdMaxThreads) bwd_column_kernel(const BwdArgs A) {
  __shared__ float sh[kBwdMaxThreads / 32][4];
  constexpr int DZ = DIM > 0 ? DIM : 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long c0 = A.chunk_begin[blockIdx.x], c1 = A.chunk_begin[blockIdx.x + 1];
  const int m = A.col_meas[c0];
  const int R = A.R, ld = A.ld;
  const float irho = A.irho[m];
  const double coef = 2.0 * A.alpha[m] / A.rho;
  float d[NVB], pd[NVB], accW[NVB], accZ[NVB][DZ], xr[NVB][DZ];
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    const int r = tid + i * nt;
    d[i] = r < R ? A.delta32[size_t(m) * ld + r] : 0.f;  // t = 1: d = delta32
    pd[i] = r < R ? float(A.pend[size_t(m) * R + r]) : 0.f;
    accW[i] = 0.f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      accZ[i][k] = 0.f;
      xr[i][k] = r < R ? float(A.xi[size_t(r) * DIM + k]) : 0.f;
    }
  }
  for (long long col = c0; col < c1; ++col) {
    const float* th = A.theta + size_t(col) * ld;
    const CT* c = static_cast<const CT*>(A.cost) + size_t(col) * ld;
    float* st = A.stored + size_t(col) * ld;
    const float lam = A.lam[col];
    float tb[NVB];
    bool act[NVB];
    float v2[2] = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NVB; ++i) {
      const int r = tid + i * nt;
      act[i] = false;
      tb[i] = 0.f;
      if (r < R) {
        // w exactly as the forward column step formed it
        const float w = fmaf(-float(c[r]), irho, fmaf(2.f, d[i], th[r]));
        act[i] = w > lam;
        tb[i] = st[r] + pd[i];
        if (act[i]) {
          v2[0] += tb[i];
          v2[1] += 1.f;
        }
      }
    }
    block_sum_n<2, float>(v2, sh);
    const float mean = v2[1] > 0.f ? v2[0] / v2[1] : 0.f;
    float zs[DZ], zx[DZ];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      zs[k] = float(A.zeta[size_t(col) * DIM + k]);
      zx[k] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < NVB; ++i) {
      const int r = tid + i * nt;
      if (r >= R) continue;
      const float wb = act[i] ? tb[i] - mean : 0.f;
      st[r] = wb;
      if (act[i]) {
        accW[i] += wb;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          accZ[i][k] = fmaf(wb, zs[k], accZ[i][k]);
          zx[k] = fmaf(wb, xr[i][k] - zs[k], zx[k]);
        }
      }
    }
    if (DIM > 0) block_sum_n<DZ, float>(zx, sh);
    if (tid == 0) {
      A.qbar[col] += double(mean);
#pragma unroll
      for (int k = 0; k < DIM; ++k) A.zetabar[size_t(col) * DIM + k] += coef * double(zx[k]);
    }
  }
  // chunk partials, [chunk][1 + DIM][R]
  double* part = A.part + size_t(blockIdx.x) * (1 + DIM) * R;
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    const int r = tid + i * nt;
    if (r >= R) continue;
    part[r] = double(accW[i]);
#pragma unroll
    for (int k = 0; k < DIM; ++k) part[size_t(1 + k) * R + r] = double(accZ[i][k]);
  }
}

// The same reverse step with one warp per column (columns of up to 64 x 32
// rows); the warps of a CTA take the columns of its chunk in turn and reduce
// with shuffles only.  Lane l holds rows r = l + 32 v (v < NV).  A first pass
// over the column keeps only bit masks (active rows, rows whose stored value
// is nonzero) and the sums for the mean; a second pass touches those rows
// only, so register use stays low and the loads of the first pass overlap
// (it is branch-free, with the loads of G rows issued together).  The
// chunk's per-row sums are taken by bwd_chunk_rowsum_kernel.
constexpr int kBwdWarps = 8;

template <int NV, typename CT>
__global__ void __launch_bounds__(kBwdWarps * 32) bwd_warp_kernel(const BwdArgs A) {
  extern __shared__ float sm_w[];
  const int R = A.R, ld = A.ld, dim = A.dim;
  float* d_s = sm_w;       // [R] shift of the chunk's measure
  float* pd_s = sm_w + R;  // [R] broadcast part of thetabar
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long c0 = A.chunk_begin[blockIdx.x], c1 = A.chunk_begin[blockIdx.x + 1];
  const int m = A.col_meas[c0];
  for (int i = tid; i < R; i += blockDim.x) {
    d_s[i] = A.delta32[size_t(m) * ld + i];  // t = 1: d = delta32
    pd_s[i] = float(A.pend[size_t(m) * R + i]);
  }
  __syncthreads();
  const float irho = A.irho[m];
  const double coef = 2.0 * A.alpha[m] / A.rho;
  constexpr int G = 8;  // rows whose loads are issued together
  for (long long col = c0 + warp; col < c1; col += kBwdWarps) {
    const float* th = A.theta + size_t(col) * ld;
    const CT* c = static_cast<const CT*>(A.cost) + size_t(col) * ld;
    float* st = A.stored + size_t(col) * ld;
    const float lam = A.lam[col];
    unsigned long long act = 0ull, nz = 0ull;
    float s1 = 0.f, na = 0.f;
#pragma unroll
    for (int v0 = 0; v0 < NV; v0 += G) {
      float thv[G], cv[G], sv[G];
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int r = lane + 32 * (v0 + u);
        const bool ok = v0 + u < NV && r < R;
        thv[u] = ok ? th[r] : 0.f;
        cv[u] = ok ? float(c[r]) : INFINITY;
        sv[u] = ok ? st[r] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int v = v0 + u;
        const int r = lane + 32 * v;
        if (v < NV && r < R) {
          // w exactly as the forward column step formed it
          const float w = fmaf(-cv[u], irho, fmaf(2.f, d_s[r], thv[u]));
          const bool a = w > lam;
          nz |= (unsigned long long)(sv[u] != 0.f) << v;
          act |= (unsigned long long)a << v;
          s1 += a ? sv[u] + pd_s[r] : 0.f;
          na += a ? 1.f : 0.f;
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
    unsigned long long todo = act | nz;
    while (todo) {
      const int v = __ffsll((long long)todo) - 1;
      todo &= todo - 1ull;
      const int r = lane + 32 * v;
      if ((act >> v) & 1ull) {
        const float wb = (st[r] + pd_s[r]) - mean;
        st[r] = wb;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < dim) zx[k] = fmaf(wb, float(__ldg(A.xi + size_t(r) * dim + k)) - zs[k], zx[k]);
      } else {
        st[r] = 0.f;
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
// in order.  A thread owns rows r = tid + i * kRsThreads (i < NVB), so every
// column gives it NVB independent loads, and columns are unrolled by four.
constexpr int kRsThreads = 256;

template <int NVB>
__global__ void __launch_bounds__(kRsThreads) bwd_chunk_rowsum_kernel(const BwdArgs A) {
  const int tid = threadIdx.x;
  const long long c0 = A.chunk_begin[blockIdx.x], c1 = A.chunk_begin[blockIdx.x + 1];
  const int R = A.R, ld = A.ld, dim = A.dim;
  float sw[NVB], sz[NVB][3];
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    sw[i] = 0.f;
    sz[i][0] = sz[i][1] = sz[i][2] = 0.f;
  }
#pragma unroll 4
  for (long long col = c0; col < c1; ++col) {
    const float* st = A.stored + size_t(col) * ld;
    float zc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < dim) zc[k] = float(__ldg(A.zeta + size_t(col) * dim + k));
#pragma unroll
    for (int i = 0; i < NVB; ++i) {
      const int r = tid + i * kRsThreads;
      const float wb = r < R ? st[r] : 0.f;
      sw[i] += wb;
#pragma unroll
      for (int k = 0; k < 3; ++k) sz[i][k] = fmaf(wb, zc[k], sz[i][k]);
    }
  }
  double* part = A.part + size_t(blockIdx.x) * (1 + dim) * R;
#pragma unroll
  for (int i = 0; i < NVB; ++i) {
    const int r = tid + i * kRsThreads;
    if (r >= R) continue;
    part[r] = double(sw[i]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < dim) part[size_t(1 + k) * R + r] = double(sz[i][k]);
  }
}

// Sums the chunk partials of each measure in a fixed order:
// red[m][k][r] = sum over the chunks j of measure m of part[j][k][r]
// (k = 0: sum_s wbar_rs, k = 1..dim: sum_s wbar_rs zeta_s).  Block
// (kRedRows rows) x (kRedSlices chunk slices), grid (rows, measures, 1 + dim).
constexpr int kRedRows = 32, kRedSlices = 8;
__global__ void __launch_bounds__(kRedRows * kRedSlices) bwd_chunk_reduce_kernel(const BwdArgs A) {
  __shared__ double sh[kRedSlices][kRedRows];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = blockIdx.x * kRedRows + tx;
  const int m = blockIdx.y, k = blockIdx.z;
  const int K1 = 1 + A.dim, R = A.R;
  double s = 0.0;
  if (r < R) {
#pragma unroll 4
    for (int j = A.meas_chunk[m] + ty; j < A.meas_chunk[m + 1]; j += kRedSlices)
      s += A.part[(size_t(j) * K1 + k) * R + r];
  }
  sh[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && r < R) {
    double t = 0.0;
#pragma unroll
    for (int y = 0; y < kRedSlices; ++y) t += sh[y][tx];
    A.red[(size_t(m) * K1 + k) * R + r] = t;
  }
}

// Per row r: dbar, pbar, the new broadcast part of thetabar and xibar.
// acc_prev holds sum_s wbar^(k+1)_rs (the stored part entering this step).
__global__ void bwd_row_kernel(const BwdArgs A) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.R) return;
  const int dim = A.dim, R = A.R, K1 = 1 + dim;
  double pbar = 0.0;
  for (int m = 0; m < A.Mtot; ++m) {
    const size_t o = size_t(m) * R + r;
    const double w = A.red[size_t(m) * K1 * R + r];
    const double dbar = 2.0 * w - (A.acc_prev[o] + A.Sd[m] * A.pend[o]);
    pbar += dbar * A.inv_S[m];
  }
  for (int m = 0; m < A.Mtot; ++m) {
    const size_t o = size_t(m) * R + r;
    const double w = A.red[size_t(m) * K1 * R + r];
    const double dbar = 2.0 * w - (A.acc_prev[o] + A.Sd[m] * A.pend[o]);
    const double coef = 2.0 * A.alpha[m] / A.rho;
    for (int k = 0; k < dim; ++k) {
      const double wz = A.red[(size_t(m) * K1 + 1 + k) * R + r];
      A.xibar[size_t(r) * dim + k] -= coef * (A.xi[size_t(r) * dim + k] * w - wz);
    }
    A.pend[o] = -dbar * A.inv_S[m] + A.a[m] * pbar;
    A.acc_prev[o] = w;
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

template <int NVB, int DIM>
cudaError_t bwd_col_dt(int dt, int nchunks, int nt, cudaStream_t st, const BwdArgs& a) {
  switch (dt) {
    case 0: bwd_column_kernel<NVB, float, DIM><<<nchunks, nt, 0, st>>>(a); break;
    case 1: bwd_column_kernel<NVB, __nv_bfloat16, DIM><<<nchunks, nt, 0, st>>>(a); break;
    case 2: bwd_column_kernel<NVB, __half, DIM><<<nchunks, nt, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NVB>
cudaError_t bwd_col_nv(int dt, int dim, int nchunks, int nt, cudaStream_t st, const BwdArgs& a) {
  switch (dim) {
    case 0: return bwd_col_dt<NVB, 0>(dt, nchunks, nt, st, a);
    case 1: return bwd_col_dt<NVB, 1>(dt, nchunks, nt, st, a);
    case 2: return bwd_col_dt<NVB, 2>(dt, nchunks, nt, st, a);
    case 3: return bwd_col_dt<NVB, 3>(dt, nchunks, nt, st, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int bwd_max_rows() { return 8 * kBwdMaxThreads; }


cudaError_t launch_chunk_rowsum(int nchunks, cudaStream_t st, const BwdArgs& a) {
  const int need = (a.R + kRsThreads - 1) / kRsThreads;
  if (need <= 2) bwd_chunk_rowsum_kernel<2><<<nchunks, kRsThreads, 0, st>>>(a);
  else if (need <= 4) bwd_chunk_rowsum_kernel<4><<<nchunks, kRsThreads, 0, st>>>(a);
  else if (need <= 8) bwd_chunk_rowsum_kernel<8><<<nchunks, kRsThreads, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int NV>
cudaError_t bwd_warp_nv(int dt, int nchunks, cudaStream_t st, const BwdArgs& a) {
  const size_t smem = 2 * sizeof(float) * size_t(a.R);
  switch (dt) {
    case 0: bwd_warp_kernel<NV, float><<<nchunks, kBwdWarps * 32, smem, st>>>(a); break;
    case 1: bwd_warp_kernel<NV, __nv_bfloat16><<<nchunks, kBwdWarps * 32, smem, st>>>(a); break;
    case 2: bwd_warp_kernel<NV, __half><<<nchunks, kBwdWarps * 32, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_chunk_rowsum(nchunks, st, a);
}

cudaError_t launch_bwd_step(int cost_dtype, int nchunks, cudaStream_t st, const BwdArgs& a) {
  const int nv = (a.R + 31) / 32;
  cudaError_t e;
  if (nv <= 4) e = bwd_warp_nv<4>(cost_dtype, nchunks, st, a);
  else if (nv <= 8) e = bwd_warp_nv<8>(cost_dtype, nchunks, st, a);
  else if (nv <= 16) e = bwd_warp_nv<16>(cost_dtype, nchunks, st, a);
  else if (nv <= 25) e = bwd_warp_nv<25>(cost_dtype, nchunks, st, a);
  else if (nv <= 32) e = bwd_warp_nv<32>(cost_dtype, nchunks, st, a);
  else if (nv <= 50) e = bwd_warp_nv<50>(cost_dtype, nchunks, st, a);
  else if (nv <= 64) e = bwd_warp_nv<64>(cost_dtype, nchunks, st, a);
  else {
    // longer columns (R > 2048): one CTA of 512 threads per chunk column
    const int need = (a.R + kBwdMaxThreads - 1) / kBwdMaxThreads;
    if (need <= 6) e = bwd_col_nv<6>(cost_dtype, a.dim, nchunks, kBwdMaxThreads, st, a);
    else if (need <= 8) e = bwd_col_nv<8>(cost_dtype, a.dim, nchunks, kBwdMaxThreads, st, a);
    else return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  bwd_chunk_reduce_kernel<<<dim3((a.R + kRedRows - 1) / kRedRows, a.Mtot, 1 + a.dim),
                            dim3(kRedRows, kRedSlices), 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bwd_row_kernel<<<(a.R + 63) / 64, 64, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bwd_theta0(long long T, cudaStream_t st, const BwdArgs& a) {
  bwd_theta0_kernel<<<unsigned(T), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mam
