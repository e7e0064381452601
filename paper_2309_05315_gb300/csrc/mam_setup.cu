// libmam device code run at creation and reset (arXiv 2309.05315, eq. HugeLP
// and Algorithm 1 Step 0): the costs, theta^0 and its row sums, and a
// fixed-point to FP64 conversion for the host reads.  Kept apart from the
// per-iteration kernels of mam_kernels.cu.
#include "mam_device.cuh"

#include <cmath>

namespace mam {
namespace {

// c_rs = alpha_m * ||xi_r - zeta_s||^2 (eq. HugeLP) or alpha_m * C_rs,
// computed in FP64 without contraction, rounded to FP32, then to the storage
// type (round to nearest even).  Padding rows R..ld-1 get +inf.  zeta and gen hold the
// columns col0 .. col0+ncols-1 only.
template <typename CT>
__device__ __forceinline__ CT to_cost(float x);
template <>
__device__ __forceinline__ float to_cost<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_cost<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half to_cost<__half>(float x) {
  return __float2half_rn(x);
}

template <typename CT>
__global__ void build_cost_kernel(CT* cost, const double* xi,
                                  const double* zeta, const double* gen,
                                  const int* col_meas, const double* alpha,
                                  const double* eta, long long col0,
                                  long long ncols, int R, int ld, int dim,
                                  const long long* cols) {
  // A block per column (grid-stride); the column's measure, alpha, eta and
  // point once per column.  The additions that are exact no-ops (0 + x,
  // x - 0) are skipped: the values are those of the plain FP64 formula.
  // cols (optional) lists the columns; zeta and gen then follow the list.
  for (long long jc = blockIdx.x; jc < ncols; jc += gridDim.x) {
    const long long col = cols ? cols[jc] : col0 + jc;
    const int m = col_meas[col];
    const double al = alpha[m];
    const double et = eta ? eta[m] : 0.0;
    double z[3] = {0.0, 0.0, 0.0};
    if (!gen)
      for (int k = 0; k < dim; ++k) z[k] = zeta[jc * dim + k];
    CT* out = cost + size_t(col) * ld;
    for (int r = threadIdx.x; r < ld; r += blockDim.x) {
      double c = INFINITY;  // padding rows: w = -inf, never active
      if (r < R) {
        double acc;
        if (gen) {
          acc = gen[jc * R + r];
        } else {
          const double d0 = __dadd_rn(z[0], -xi[size_t(r) * dim]);
          acc = __dmul_rn(d0, d0);
          for (int k = 1; k < dim; ++k) {
            const double df = __dadd_rn(z[k], -xi[size_t(r) * dim + k]);
            acc = __dadd_rn(acc, __dmul_rn(df, df));
          }
        }
        if (et != 0.0) acc = __dadd_rn(acc, -et);
        c = __dmul_rn(al, acc);
      }
      out[r] = to_cost<CT>(__double2float_rn(c));
    }
  }
}

// tab[u][v] = fl(d^2), d = fl(uz_u - ux_v): the per-coordinate square of
// build_cost_kernel for every pair of distinct coordinate values.
__global__ void sqdiff_table_kernel(double* tab, const double* uz, int nz, const double* ux,
                                    int nx) {
  const long long n = (long long)nz * nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = __dadd_rn(uz[i / nx], -ux[i % nx]);
    tab[i] = __dmul_rn(d, d);
  }
}

// build_cost_kernel's values from the coordinate tables: the column's row of
// each table (its point's value index iz) is read at the row's value index
// ix; the squares are added in coordinate order and scaled as there.
// ix: [dim][R] value indices of the barycenter points; iz: [ncols][dim].
template <typename CT>
__global__ void build_cost_tab_kernel(CT* cost, const double* __restrict__ tab,
                                      const CostTab tb, const int* __restrict__ ix,
                                      const int* __restrict__ iz, const int* col_meas,
                                      const double* alpha, const double* eta, long long col0,
                                      long long ncols, int R, int ld, const long long* cols) {
  for (long long jc = blockIdx.x; jc < ncols; jc += gridDim.x) {
    const long long col = cols ? cols[jc] : col0 + jc;
    const int m = col_meas[col];
    const double al = alpha[m];
    const double et = eta ? eta[m] : 0.0;
    const double* t0 = tab + tb.off[0] + (long long)iz[jc * tb.dim] * tb.nx[0];
    const double* t1 =
        tb.dim > 1 ? tab + tb.off[1] + (long long)iz[jc * tb.dim + 1] * tb.nx[1] : nullptr;
    const double* t2 =
        tb.dim > 2 ? tab + tb.off[2] + (long long)iz[jc * tb.dim + 2] * tb.nx[2] : nullptr;
    CT* out = cost + size_t(col) * ld;
    for (int r = threadIdx.x; r < ld; r += blockDim.x) {
      double c = INFINITY;  // padding rows: w = -inf, never active
      if (r < R) {
        double acc = __ldg(t0 + __ldg(ix + r));
        if (t1) acc = __dadd_rn(acc, __ldg(t1 + __ldg(ix + R + r)));
        if (t2) acc = __dadd_rn(acc, __ldg(t2 + __ldg(ix + 2 * size_t(R) + r)));
        if (et != 0.0) acc = __dadd_rn(acc, -et);
        c = __dmul_rn(al, acc);
      }
      out[r] = to_cost<CT>(__double2float_rn(c));
    }
  }
}

// Columns with the same point, alpha_m and eta have the same cost column:
// dst_src[i] = (dst, src) copies column src onto column dst, 16 B at a time
// (a column is ld * sizeof(CT) bytes, ld a multiple of 8).
__global__ void copy_cost_columns_kernel(uint4* cost, const long long* dst_src, long long n,
                                         int vec_per_col) {
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    const uint4* s = cost + size_t(dst_src[2 * i + 1]) * vec_per_col;
    uint4* d = cost + size_t(dst_src[2 * i]) * vec_per_col;
    for (int v = threadIdx.x; v < vec_per_col; v += blockDim.x) d[v] = s[v];
  }
}

// theta^0 (Alg. 1 Step 0; "Initialization" leaves it arbitrary):
// mode 0: theta_rs = q_s / R, mode 1: 0.  Padding rows are 0 and every
// threshold starts unknown (NaN; lam = null keeps the thresholds).
__global__ void init_theta_kernel(float* theta, float* lam,
                                  const double* q, long long T, int R, int ld,
                                  int mode) {
  // A block per column (grid-stride): q_s / R once per column, rows written
  // as float4 (ld is a multiple of 8).
  const int ld4 = ld >> 2;
  for (long long col = blockIdx.x; col < T; col += gridDim.x) {
    const float v = mode == 0 ? float(q[col] / double(R)) : 0.f;
    float4* th = reinterpret_cast<float4*>(theta + size_t(col) * ld);
    for (int g = threadIdx.x; g < ld4; g += blockDim.x) {
      const int r = 4 * g;
      th[g] = make_float4(r < R ? v : 0.f, r + 1 < R ? v : 0.f, r + 2 < R ? v : 0.f,
                          r + 3 < R ? v : 0.f);
    }
    if (lam && threadIdx.x == 0) lam[col] = __int_as_float(0x7fc00000);
  }
}

// p^(m)_r F = F sum_s theta^0_rs for theta^0 (Alg. 1 Step 0), summed in
// FP64 in column order and rounded once to the 64-bit fixed point of the
// marginals.  Every row of a theta^0 column holds the same value
// (float(q_s / R), or 0), so one block per measure forms the sum and writes
// it to every row: the value a per-row sum of the stored entries would give,
// at 1/R of the work.
__global__ void rowsum_theta0_kernel(const double* q, const long long* col_off, int R,
                                     int mode, double fx_scale, long long* pm) {
  // The block forms the values of a chunk of columns, thread 0 adds them in
  // column order (the FP64 divisions leave the serial chain).
  constexpr int kChunk = 1024;
  __shared__ double v[kChunk];
  __shared__ long long v_s;
  const int m = blockIdx.x;
  double acc = 0.0;  // thread 0's running sum
  if (mode == 0)
    for (long long c0 = col_off[m]; c0 < col_off[m + 1]; c0 += kChunk) {
      const int n = int(col_off[m + 1] - c0 < kChunk ? col_off[m + 1] - c0 : kChunk);
      for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = double(float(q[c0 + i] / double(R)));
      __syncthreads();
      if (threadIdx.x == 0)
        for (int i = 0; i < n; ++i) acc += v[i];
      __syncthreads();
    }
  if (threadIdx.x == 0) v_s = __double2ll_rn(acc * fx_scale);
  __syncthreads();
  const long long sum = v_s;
  for (int r = threadIdx.x; r < R; r += blockDim.x) pm[size_t(m) * R + r] = sum;
}

}  // namespace

cudaError_t launch_build_cost(int cost_dtype, void* cost, const double* xi,
                              const double* zeta, const double* gen_cost,
                              const int* col_meas, const double* alpha,
                              const double* eta, long long col0, long long ncols,
                              int R, int ld, int dim, cudaStream_t st,
                              const long long* cols) {
  long long g = ncols < 152 * 16 ? ncols : 152 * 16;
  if (g < 1) g = 1;
  switch (cost_dtype) {
    case 0:
      build_cost_kernel<float><<<int(g), 256, 0, st>>>(
          static_cast<float*>(cost), xi, zeta, gen_cost, col_meas, alpha, eta,
          col0, ncols, R, ld, dim, cols);
      break;
    case 1:
      build_cost_kernel<__nv_bfloat16><<<int(g), 256, 0, st>>>(
          static_cast<__nv_bfloat16*>(cost), xi, zeta, gen_cost, col_meas,
          alpha, eta, col0, ncols, R, ld, dim, cols);
      break;
    case 2:
      build_cost_kernel<__half><<<int(g), 256, 0, st>>>(
          static_cast<__half*>(cost), xi, zeta, gen_cost, col_meas, alpha, eta,
          col0, ncols, R, ld, dim, cols);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sqdiff_table(double* tab, const double* uz, int nz, const double* ux,
                                int nx, cudaStream_t st) {
  long long g = ((long long)nz * nx + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  sqdiff_table_kernel<<<int(g), 256, 0, st>>>(tab, uz, nz, ux, nx);
  return cudaGetLastError();
}

cudaError_t launch_build_cost_tab(int cost_dtype, void* cost, const double* tab,
                                  const CostTab& tb, const int* ix, const int* iz,
                                  const int* col_meas, const double* alpha, const double* eta,
                                  long long col0, long long ncols, int R, int ld,
                                  cudaStream_t st, const long long* cols) {
  long long g = ncols < 152 * 16 ? ncols : 152 * 16;
  if (g < 1) g = 1;
  switch (cost_dtype) {
    case 0:
      build_cost_tab_kernel<float><<<int(g), 256, 0, st>>>(
          static_cast<float*>(cost), tab, tb, ix, iz, col_meas, alpha, eta, col0, ncols, R, ld,
          cols);
      break;
    case 1:
      build_cost_tab_kernel<__nv_bfloat16><<<int(g), 256, 0, st>>>(
          static_cast<__nv_bfloat16*>(cost), tab, tb, ix, iz, col_meas, alpha, eta, col0,
          ncols, R, ld, cols);
      break;
    case 2:
      build_cost_tab_kernel<__half><<<int(g), 256, 0, st>>>(
          static_cast<__half*>(cost), tab, tb, ix, iz, col_meas, alpha, eta, col0, ncols, R,
          ld, cols);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_copy_cost_columns(int cost_dtype, void* cost, const long long* dst_src,
                                     long long n, int ld, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int vec = int(size_t(ld) * (cost_dtype == 0 ? 4 : 2) / 16);
  long long g = n < 152 * 16 ? n : 152 * 16;
  copy_cost_columns_kernel<<<int(g), 256, 0, st>>>(static_cast<uint4*>(cost), dst_src, n, vec);
  return cudaGetLastError();
}

cudaError_t launch_init_theta(float* theta, float* lam,
                              const double* q, long long T, int R, int ld,
                              int mode, cudaStream_t st) {
  long long g = T < 152 * 16 ? T : 152 * 16;
  if (g < 1) g = 1;
  init_theta_kernel<<<int(g), ld >= 1024 ? 256 : 128, 0, st>>>(theta, lam, q, T, R, ld,
                                                                 mode);
  return cudaGetLastError();
}

__global__ void fx_to_double_kernel(const long long* in, size_t n, double scale, double* out) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    out[i] = double(in[i]) * scale;
}

cudaError_t launch_fx_to_double(const long long* in, size_t n, double scale, double* out,
                                cudaStream_t st) {
  size_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  fx_to_double_kernel<<<unsigned(g), 256, 0, st>>>(in, n, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_rowsum_theta0(const double* q, const long long* col_off, int Mtot, int R,
                                 int mode, double fx_scale, long long* pm, cudaStream_t st) {
  rowsum_theta0_kernel<<<Mtot, 256, 0, st>>>(q, col_off, R, mode, fx_scale, pm);
  return cudaGetLastError();
}

}  // namespace mam
