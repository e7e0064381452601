// libmam internal: the free-support step of Algorithm 2 (Prop. 4).
#pragma once

#include <cuda_runtime.h>

namespace mam {

// Arguments of the free-support step (Algorithm 2, Prop. 4).
struct SupportArgs {
  const float* theta;        // [T][ld]
  const void* cost;          // [T][ld] (float / bf16 / half), or [S][ld] shared
  const int* cost_col;       // [T] cost column of each plan column (shared), or null
  const float* gen_xi;       // generated costs: [3][ld] coordinate planes of xi, else null
  const float4* gen_zeta;    // generated costs: [T] (x, y, z, eta)
  const float* q;            // [T]
  const float* lam;          // [T] last thresholds (warm start; NaN: none)
  const int* col_meas;       // [T]
  const float* delta32;      // [Mtot][ld] (p - p^(m)) / S_m of the current plans
  const float* inv_rho;      // [Mtot]
  const double* alpha;       // [Mtot]
  const double* zeta;        // [T][dim] support points of the kept columns
  unsigned long long* acc;   // [R][dim + 1] fixed-point sums (zero on entry, cleared)
  double fx;                 // fixed-point scale of acc
  float t;                   // t of the next step
  float lam_floor;           // 0 for capped columns, else -inf
  long long T;
  int R, ld, dim;
};

// pi-hat of the next step -> per-row sums -> xi (rows without mass keep
// their point).
cudaError_t launch_support_step(int cost_dtype, const SupportArgs& a, double* xi,
                                cudaStream_t st);

}  // namespace mam
