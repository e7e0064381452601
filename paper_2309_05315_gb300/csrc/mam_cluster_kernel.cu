// libmam: the column step for long columns, one column per thread-block
// cluster (kernel kind 2).
//
// Step 2 of Algorithm 1 projects every plan column, R entries long, onto
// the simplex Delta_R(q_s).  A free-support grid (Theorem 1: every point
// sum_m alpha_m zeta_(m), R = (M (K - 1) + 1)^2 for K x K images, e.g.
// R = 349281 for ten 60 x 60 images) makes a column far longer than one CTA
// can hold, so a column is split across the CS CTAs (2..16) of a cluster:
// CTA k holds rows [k rpc, (k + 1) rpc) and keeps its slice of
//   w_r = theta_rs + 2 d_r - c_rs / rho
// in shared memory.  The exact threshold search (the same warm-started
// Newton/Michelot iteration with the Newton-step certificate as the
// one-CTA kernel) needs, per pass, sum_r max(w_r - l, 0), #{w_r > l},
// min_r |w_r - l| and max_r w_r over the whole column: each CTA reduces its
// slice, thread 0 writes the four values into a slot of every peer's shared
// memory (st.shared::cluster at the mapa-translated address, no multicast),
// and one cluster barrier (arrive.release / wait.acquire) makes them
// visible; every CTA then combines the CS slots in rank order, so all CTAs
// hold bit-identical totals and take the same branches.  Slots are double
// buffered: a CTA can write buffer b again only after the barrier of the
// reduction in between, which every CTA passes after reading b.
// theta and c are read once (pass 1) and theta written once (commit) per
// column; d (one R-vector per measure) is read from L2.  Row sums of pi-hat
// are added as 64-bit fixed-point integers, as in the other column kernels.
// A cluster barrier at the start (every peer's shared memory exists before
// the first remote store) and at the end (no CTA leaves while a peer could
// still write to it) brackets the kernel.  Cluster barriers are hardware
// barriers, not spin loops; every CTA of a cluster runs the same sequence of
// them because the control flow depends only on the combined totals.
#include "mam_device.cuh"

#include <cfloat>
#include <cmath>

namespace mam {
namespace {

constexpr int kClusterMax = 16;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Store v into the same shared-memory slot of CTA `peer` of the cluster.
__device__ __forceinline__ void st_peer(float4* local_slot, unsigned peer, float4 v) {
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(remote) : "r"(smem_u32(local_slot)), "r"(peer));
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};"
               :: "r"(remote), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// (sum, sum, min, max) of the whole column: CTA reduction, then the
// cluster exchange described above.  Every thread of every CTA returns the
// same value.
struct ClusterRed {
  float4* red;    // [2][kRedSlots] CTA partials per warp
  float4* slot;   // [2][kClusterMax] cluster partials per CTA rank
  int rb, cb, lane, warp, nw;
  unsigned rank, cs;

  __device__ float4 operator()(float4 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      v.z = fminf(v.z, __shfl_xor_sync(0xffffffffu, v.z, o));
      v.w = fmaxf(v.w, __shfl_xor_sync(0xffffffffu, v.w, o));
    }
    if (lane == 0) red[rb * kRedSlots + warp] = v;
    __syncthreads();
    float4 r = lane < nw ? red[rb * kRedSlots + lane]
                         : make_float4(0.f, 0.f, INFINITY, -INFINITY);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
      r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
      r.z = fminf(r.z, __shfl_xor_sync(0xffffffffu, r.z, o));
      r.w = fmaxf(r.w, __shfl_xor_sync(0xffffffffu, r.w, o));
    }
    rb ^= 1;
    float4* s = slot + cb * kClusterMax;
    if (lane == 0 && warp == 0)
      for (unsigned k = 0; k < cs; ++k) st_peer(s + rank, k, r);
    cluster_sync();
    float4 t = make_float4(0.f, 0.f, INFINITY, -INFINITY);
    for (unsigned k = 0; k < cs; ++k) {
      const float4 u = s[k];
      t.x += u.x;
      t.y += u.y;
      t.z = fminf(t.z, u.z);
      t.w = fmaxf(t.w, u.w);
    }
    cb ^= 1;
    return t;
  }
};

template <typename CT>
__device__ __forceinline__ float4 load_cost4(const CT* base, int g) {
  return CostIO<CT>::load4(base, g);
}

constexpr int kClThreads = 256;  // most threads per CTA
constexpr int kClUnroll = 4;     // float4 groups a thread loads before using any

// Column step over the clusters' share of the index set.  rpc: rows per CTA
// slice (a multiple of 4); dynamic shared memory holds rpc floats of w.
// Every thread issues the loads of kClUnroll groups (theta, c and d: 12
// independent 16-byte loads) before it uses any, so that a CTA keeps about
// 50 KB in flight.
// GEN: c is not read but computed as ||xi_r - zeta_s||^2 - eta in FP32 from
// the points (the generated cost layout; CT is unused then).
// xg: the problem's coordinate planes [3][ld]; one float4 per coordinate
// covers the group's 4 rows.
template <typename CT, bool DIAG, bool GEN>
__device__ __forceinline__ float4 cost4(const ColArgs& A, const CT* c_g, const float* xg,
                                        float4 zg, long long r, int R, int g) {
  if (!GEN) return load_cost4<CT>(c_g, g);
  const int ld = A.ld;
  const float zc[3] = {zg.x, zg.y, zg.z};
  // all three planes, independent loads issued together (planes past dim
  // hold zeros, as does zeta there)
  float4 x[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = __ldg(reinterpret_cast<const float4*>(xg + size_t(k) * ld + r));
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float dx = x[k].x - zc[k], dy = x[k].y - zc[k], dz = x[k].z - zc[k],
                dw = x[k].w - zc[k];
    s.x = fmaf(dx, dx, s.x);
    s.y = fmaf(dy, dy, s.y);
    s.z = fmaf(dz, dz, s.z);
    s.w = fmaf(dw, dw, s.w);
  }
  return make_float4(r < R ? s.x - zg.w : INFINITY, r + 1 < R ? s.y - zg.w : INFINITY,
                     r + 2 < R ? s.z - zg.w : INFINITY, r + 3 < R ? s.w - zg.w : INFINITY);
}

template <typename CT, bool DIAG, bool GEN>
__global__ void __launch_bounds__(kClThreads, 2) column_cluster_kernel(const ColArgs A, int rpc) {
  extern __shared__ __align__(16) float w_s[];
  __shared__ float4 red[2 * kRedSlots];
  __shared__ float4 slot[2 * kClusterMax];
  __shared__ double dred[kRedSlots];
  const int tid = threadIdx.x, nt = blockDim.x;
  ClusterRed cred{red, slot, 0, 0, tid & 31, tid >> 5, nt >> 5, cluster_rank(), cluster_size()};
  const int R = A.R, ld = A.ld;
  const long long r0 = (long long)cred.rank * rpc;
  const long long r1 = r0 + rpc < R ? r0 + rpc : R;
  const int ng = r1 > r0 ? int((r1 - r0 + 3) / 4) : 0;  // float4 groups of the slice
  float4* w4 = reinterpret_cast<float4*>(w_s);

  cluster_sync();  // every peer's shared memory exists before the first remote store
  const long long k_iter = *A.iter;
  const Sched sc = A.sched[draw_index_set(A.draw, k_iter)];
  const long long n_all = sc.col_end - sc.col_begin;
  const long long G = cluster_count();
  const long long cid = cluster_id();
  const long long col0 = sc.col_begin + n_all * cid / G;
  const long long ncol = sc.col_begin + n_all * (cid + 1) / G - col0;
  unsigned long long my_passes = 0;

  pdl_wait();  // the averaging kernel's shifts, block sums and cleared sums
  int m_cur = -1, p_cur = -1;
  double t_cur = 1.0;
  float tf = 1.f, rho_m = 0.f, nirho = 0.f, cm = 1.f;  // cm: factor of the stored cost
  const float* dl = nullptr;
  unsigned long long* acc_m = nullptr;
  const float fx = A.fx_scale;
  for (long long j = 0; j < ncol; ++j) {
    const long long col = col0 + j;
    const int m = A.col_meas[col];
    const float tau = A.q[col];
    const float lam_prev = A.lam[col];
    if (m != m_cur) {
      m_cur = m;
      const int pr = A.meas_prob[m];
      if (pr != p_cur) {
        p_cur = pr;
        t_cur = t_from_blocks(A.blk + size_t(pr) * A.nblk * 4, A.nblk, A.rho_p[pr],
                              A.gamma_p[pr], dred, tid, nt);
        if (tid == 0 && cred.rank == 0) A.t_used[pr] = t_cur;
      }
      tf = float(t_cur);
      rho_m = A.rho[m];
      nirho = -A.inv_rho[m];
      cm = A.cmul[m];
      dl = A.delta32 + size_t(m) * ld;
      acc_m = A.acc + size_t(m) * R;
    }
    const float* th_g = A.theta + size_t(col) * ld + r0;
    const long long ccol = A.cost_col ? (long long)A.cost_col[col] : col;
    const CT* c_g = GEN ? nullptr : static_cast<const CT*>(A.cost) + size_t(ccol) * ld + r0;
    const float* xg = GEN ? A.gen_xi + size_t(A.meas_prob[m]) * 3 * ld : nullptr;
    const float4 zg = GEN ? A.gen_zeta[col] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool pos = tau > 0.f;
    const bool warm = pos && (lam_prev == lam_prev);
    const float l0 = warm ? lam_prev : 0.f;

    // Pass 1: w into shared memory, and (f, n, gap, max) at l0.
    float4 v = make_float4(0.f, 0.f, INFINITY, -INFINITY);
    for (int g0 = tid; g0 < ng; g0 += kClUnroll * nt) {
      float4 th[kClUnroll], c[kClUnroll], dd[kClUnroll];
#pragma unroll
      for (int u = 0; u < kClUnroll; ++u) {
        const int g = g0 + u * nt;
        if (g < ng) {
          th[u] = __ldg(reinterpret_cast<const float4*>(th_g) + g);
          c[u] = cost4<CT, DIAG, GEN>(A, c_g, xg, zg, r0 + 4LL * g, R, g);
          dd[u] = __ldg(reinterpret_cast<const float4*>(dl + r0) + g);
        }
      }
#pragma unroll
      for (int u = 0; u < kClUnroll; ++u) {
        const int g = g0 + u * nt;
        if (g >= ng) break;
        float4 w;
        w.x = fmaf(c[u].x, nirho, fmaf(2.f, __fmul_rn(tf, dd[u].x), th[u].x));
        w.y = fmaf(c[u].y, nirho, fmaf(2.f, __fmul_rn(tf, dd[u].y), th[u].y));
        w.z = fmaf(c[u].z, nirho, fmaf(2.f, __fmul_rn(tf, dd[u].z), th[u].z));
        w.w = fmaf(c[u].w, nirho, fmaf(2.f, __fmul_rn(tf, dd[u].w), th[u].w));
        w4[g] = w;
        const float xs[4] = {w.x - l0, w.y - l0, w.z - l0, w.w - l0};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          v.x += fmaxf(xs[e], 0.f);
          v.y += xs[e] > 0.f ? 1.f : 0.f;
          v.z = fminf(v.z, fabsf(xs[e]));
        }
        v.w = fmaxf(v.w, fmaxf(fmaxf(w.x, w.y), fmaxf(w.z, w.w)));
      }
    }
    const float4 t1 = cred(v);
    int np = 1;
    float lam_fin = INFINITY;
    if (pos) {
      float f = t1.x, n = t1.y;
      const float gap0 = t1.z, mx = t1.w;
      float nprev = -1.f, lam = l0;
      bool bracket = !warm, done = false;
      if (warm) {
        if (n == 0.f) {
          bracket = true;  // warm start at or above max w
        } else {
          const float dlt = (f - tau) / n;
          lam = l0 + dlt;
          nprev = n;
          if (newton_certified(gap0, dlt, l0)) {
            lam_fin = lam;
            done = true;
          }
        }
      }
      for (int it = 0; it < kMaxNewton && !done; ++it) {
        if (bracket) {  // lambda* lies in [max w - tau, max w)
          float lo_b = mx - tau, hi_b = mx;
          for (int b = 0; b < A.bisect_depth; ++b) {
            const float mid = 0.5f * (lo_b + hi_b);
            float4 u = make_float4(0.f, 0.f, INFINITY, -INFINITY);
            for (int g = tid; g < ng; g += nt) {
              const float4 w = w4[g];
              const float xs[4] = {w.x - mid, w.y - mid, w.z - mid, w.w - mid};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                u.x += fmaxf(xs[e], 0.f);
                u.y += xs[e] > 0.f ? 1.f : 0.f;
              }
            }
            const float4 tb = cred(u);
            ++np;
            if (tb.x >= tau) lo_b = mid; else hi_b = mid;
          }
          lam = lo_b;
          nprev = -1.f;
          bracket = false;
        }
        // (f, n) at lam, and min_r |w_r - lam| for the certificate of the
        // Newton step from lam (a pass costs a cluster barrier)
        float4 u = make_float4(0.f, 0.f, INFINITY, -INFINITY);
        for (int g = tid; g < ng; g += nt) {
          const float4 w = w4[g];
          const float xs[4] = {w.x - lam, w.y - lam, w.z - lam, w.w - lam};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            u.x += fmaxf(xs[e], 0.f);
            u.y += xs[e] > 0.f ? 1.f : 0.f;
            u.z = fminf(u.z, fabsf(xs[e]));
          }
        }
        const float4 tn = cred(u);
        ++np;
        f = tn.x;
        const float cnt = tn.y;
        if (cnt == nprev) {  // same active set twice: lam is the threshold
          lam_fin = lam;
          break;
        }
        if (cnt == 0.f) {  // not expected from below; restart from the bracket
          bracket = true;
          continue;
        }
        nprev = cnt;
        const float dl = (f - tau) / cnt;
        const float lam_from = lam;
        lam = lam + dl;
        lam_fin = lam;  // used if the pass budget runs out (not expected)
        if (newton_certified(tn.z, dl, lam_from)) break;  // the next pass would confirm lam
      }
    }

    // Commit: theta' = pihat - d, the Step 3 row sums, the diagnostics.
    const float lam_use = fmaxf(lam_fin, A.lam_floor);
    float wc = 0.f, res = 0.f, lbmin = INFINITY;
    float4* thw = reinterpret_cast<float4*>(A.theta + size_t(col) * ld + r0);
    for (int g0 = tid; g0 < ng; g0 += kClUnroll * nt) {
      float4 ddu[kClUnroll];
#pragma unroll
      for (int u = 0; u < kClUnroll; ++u)
        if (g0 + u * nt < ng)
          ddu[u] = __ldg(reinterpret_cast<const float4*>(dl + r0) + g0 + u * nt);
#pragma unroll
      for (int u = 0; u < kClUnroll; ++u) {
        const int g = g0 + u * nt;
        if (g >= ng) break;
        const float4 w = w4[g];
        const float4 dd = ddu[u];
        const float d4[4] = {__fmul_rn(tf, dd.x), __fmul_rn(tf, dd.y), __fmul_rn(tf, dd.z),
                             __fmul_rn(tf, dd.w)};
        const float pv[4] = {fmaxf(w.x - lam_use, 0.f), fmaxf(w.y - lam_use, 0.f),
                             fmaxf(w.z - lam_use, 0.f), fmaxf(w.w - lam_use, 0.f)};
        const float4 ov = make_float4(pv[0] - d4[0], pv[1] - d4[1], pv[2] - d4[2], pv[3] - d4[3]);
        const long long rr = r0 + 4LL * g;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (pv[e] > 0.f)
            atomicAdd(acc_m + rr + e, (unsigned long long)f32_to_i64_rn(pv[e] * fx));
        if (DIAG) {
          const float4 th = __ldg(reinterpret_cast<const float4*>(th_g) + g);
          const float4 c = cost4<CT, DIAG, GEN>(A, c_g, xg, zg, rr, R, g);
          const float thv[4] = {th.x, th.y, th.z, th.w};
          const float cv[4] = {cm * c.x, cm * c.y, cm * c.z, cm * c.w};
          const float ovv[4] = {ov.x, ov.y, ov.z, ov.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (rr + e >= R) continue;
            if (pv[e] > 0.f) wc += cv[e] * pv[e];
            const float dd2 = ovv[e] - thv[e];
            res += dd2 * dd2;
            lbmin = fminf(lbmin, cv[e] - rho_m * d4[e]);
          }
        }
        thw[g] = ov;
      }
    }
    if (DIAG) {
      // (wc, res) summed and lbmin taken over the column (the max slot is unused)
      const float4 td = cred(make_float4(wc, res, lbmin, -INFINITY));
      if (tid == 0 && cred.rank == 0) {
        A.diag_wc[col] = td.x;
        A.diag_res[col] = td.y;
        A.diag_lb[col] = tau * fminf(td.z, A.lb_cap);
      }
    }
    if (tid == 0 && cred.rank == 0) A.lam[col] = lam_fin;
    my_passes += np;
  }
  if (tid == 0) {
    if (cred.rank == 0) atomicAdd(A.passes, my_passes);
    pdl_wait();
    // The last CTA to finish advances the iteration counter (every CTA has
    // read it by then).
    __threadfence();
    if (atomicAdd(A.done, 1u) == gridDim.x - 1) {
      *A.iter = k_iter + 1;
      *A.done = 0u;
    }
  }
  cluster_sync();  // no CTA leaves while a peer could still store into it
}

template <typename CT, bool DIAG, bool GEN>
cudaError_t cluster_op(int op, int cs, int grid, int threads, size_t smem, cudaStream_t st,
                       const ColArgs* a, int rpc, int* occ) {
  auto kern = column_cluster_kernel<CT, DIAG, GEN>;
  if (op == 1) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  if (op == 2) {  // resident clusters on the whole GPU
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(occ, kern, &cfg);
  }
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kern, *a, rpc);
}

template <typename CT>
cudaError_t cluster_op_d(int op, bool diag, int cs, int grid, int threads, size_t smem,
                         cudaStream_t st, const ColArgs* a, int rpc, int* occ) {
  return diag ? cluster_op<CT, true, false>(op, cs, grid, threads, smem, st, a, rpc, occ)
              : cluster_op<CT, false, false>(op, cs, grid, threads, smem, st, a, rpc, occ);
}

// dt < 0: generated costs (no stored cost type).
cudaError_t cluster_op_any(int dt, int op, bool diag, int cs, int grid, int threads,
                           size_t smem, cudaStream_t st, const ColArgs* a, int rpc, int* occ) {
  if (dt < 0)
    return diag ? cluster_op<float, true, true>(op, cs, grid, threads, smem, st, a, rpc, occ)
                : cluster_op<float, false, true>(op, cs, grid, threads, smem, st, a, rpc, occ);
  switch (dt) {
    case 0: return cluster_op_d<float>(op, diag, cs, grid, threads, smem, st, a, rpc, occ);
    case 1: return cluster_op_d<__nv_bfloat16>(op, diag, cs, grid, threads, smem, st, a, rpc, occ);
    case 2: return cluster_op_d<__half>(op, diag, cs, grid, threads, smem, st, a, rpc, occ);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int cluster_rows_per_cta(int ld, int cs) {
  const int per = (ld + cs - 1) / cs;
  return (per + 3) / 4 * 4;
}

size_t cluster_kernel_smem(int ld, int cs) {
  return size_t(cluster_rows_per_cta(ld, cs)) * sizeof(float);
}

cudaError_t launch_column_cluster(int cost_dtype, bool diag, int cs, int grid, int threads,
                                  size_t smem, cudaStream_t st, const ColArgs& a) {
  return cluster_op_any(cost_dtype, 0, diag, cs, grid, threads, smem, st, &a,
                        cluster_rows_per_cta(a.ld, cs), nullptr);
}

cudaError_t set_column_cluster_smem(int cost_dtype, bool diag, size_t smem) {
  return cluster_op_any(cost_dtype, 1, diag, 0, 0, 0, smem, nullptr, nullptr, 0, nullptr);
}

cudaError_t column_cluster_occupancy(int cost_dtype, bool diag, int cs, int threads,
                                     size_t smem, int* clusters) {
  return cluster_op_any(cost_dtype, 2, diag, cs, cs, threads, smem, nullptr, nullptr, 0,
                        clusters);
}

}  // namespace mam
