// K2 + K5: numerical coarse propagator G and the serial Parareal sweep.
//
// G (Sec. 3.1, Sec. 3.2: the same discretisation as F with a larger step) takes csteps
// implicit-Euler steps per slice.  With the larger step the system is not diagonally
// dominant, so each step is solved by BiCGSTAB (van der Vorst 1992) on the Jacobi-scaled
// system  D^{-1}(I - dtau R_h) d = D^{-1} dtau R_h w  in FP32 (the paper runs its coarse
// models in single precision, Sec. 4.1).  One thread-block cluster holds the whole state and
// the two matrix-vector operands in shared memory (same band layout as the fine stepper);
// dot products are reduced warp -> CTA -> cluster in a fixed order, so every CTA obtains
// bitwise the same scalars and the result does not depend on scheduling.
//
// The serial Parareal sweep of eq. (parareal) runs in the same kernel: for n = n_first..N-1
//   G_new = G(u_n^{k+1});  u_{n+1}^{k+1} = F_n + (G_new - G_old_n);  G_old_n = G_new,
// with FP64 partial sums of ||u_{n+1}^{k+1} - u_{n+1}^k||^2 and ||u_{n+1}^{k+1}||^2 per slice
// and, at the end, delta_k = max_n ||du_n|| / max_n ||u_n|| (reading c5).  The correction is
// evaluated as F + (G_new - G_old) so that an unchanged slice gives a zero bracket exactly.
#include <cooperative_groups.h>

#include <cmath>
#include <cstdio>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bsp {

struct SweepParams {
  ItemDesc d;       // dtau = coarse step
  SweepArgs a;
  BandShape sh;
  float h;
};

struct Band {
  int M, ncol, BH, C, rank, col, r0, jbase;
  bool active;
};

// Jacobi-scaled operator A^ y = y - invd * (off-diagonal part of dtau R_h) y at interior
// nodes; zero elsewhere.  y lives in shared memory (band) with halo rows in the
// neighbouring CTAs.
template <int K>
__device__ __forceinline__ void scaled_matvec(const Band& bd, const float* y, const float* y_prev,
                                              const float* y_next, const float4* rowt,
                                              const float* invd, float ce, float cw, float cgi,
                                              float* out) {
  const int ncol = bd.ncol, col = bd.col, r0 = bd.r0, BH = bd.BH;
  const int il = col > 0 ? col - 1 : 0;
  const int ir = col + 1 < ncol ? col + 1 : col;
  const float* up = (r0 == 0) ? (y_prev ? y_prev + (BH - 1) * ncol : y) : y + (r0 - 1) * ncol;
  float uW = up[il], uC = up[col], uE = up[ir];
  float cW = y[r0 * ncol + il], cC = y[r0 * ncol + col], cE = y[r0 * ncol + ir];
  const bool last_group = (r0 + K >= BH);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int r = r0 + k, j = bd.jbase + r;
    const float* dn = (k < K - 1 || !last_group) ? y + (r + 1) * ncol
                                                 : (y_next ? y_next : y + (BH - 1) * ncol);
    const float dW = dn[il], dC = dn[col], dE = dn[ir];
    float o = 0.f;
    if (j < bd.M - 1 && col < bd.M - 1) {
      const float4 rc = rowt[r];
      const float cg = cgi * rc.z;
      o = cC - invd[r * ncol + col] * (ce * cE + cw * cW + rc.x * dC + rc.y * uC +
                                       cg * ((dE - uE) - (dW - uW)));
    }
    out[k] = o;
    uW = cW; uC = cC; uE = cE;
    cW = dW; cC = dC; cE = dE;
  }
}

// Deterministic sum of NV per-thread values over the cluster.  Every thread returns the
// same totals.  `slot` alternates so that a fast CTA never overwrites partials that a
// slow CTA is still reading.
template <int NV>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cluster, double (&v)[NV],
                                            double* wpart, double* slots, double* bcast,
                                            int& round, int C) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) wpart[warp * NV + q] = x;
  }
  __syncthreads();
  double* slot = slots + (round & 1) * NV;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) s += wpart[w * NV + q];
      slot[q] = s;
    }
  }
  cluster.sync();
  if (threadIdx.x == 0) {
    double tot[NV];
    for (int q = 0; q < NV; ++q) tot[q] = 0.0;
    for (int c = 0; c < C; ++c) {
      const double* rs = cluster.map_shared_rank(slot, c);
      for (int q = 0; q < NV; ++q) tot[q] += rs[q];
    }
    for (int q = 0; q < NV; ++q) bcast[q] = tot[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = bcast[q];
  ++round;
}

__device__ __forceinline__ void set_far_field_c(float* u, const PayoffF& pf, float tau, float h,
                                                const Band& bd, int tid) {
  const int M = bd.M, BH = bd.BH, jbase = bd.jbase, ncol = bd.ncol;
  const bool has_last_row = (jbase <= M - 1) && (M - 1 < jbase + BH);
  const int n_entries = BH + (has_last_row ? (M - 1) : 0);
  for (int e = tid; e < n_entries; e += kThreads) {
    int r, c;
    if (e < BH) { r = e; c = M - 1; if (jbase + r > M - 1) continue; }
    else { r = M - 1 - jbase; c = e - BH; }
    u[r * ncol + c] = far_field(pf, c * h, (jbase + r) * h, tau);
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads, 1) sweep_band_kernel(const __grid_constant__ SweepParams sp) {
  cg::cluster_group cluster = cg::this_cluster();
  const ItemDesc& d = sp.d;
  const SweepArgs& a = sp.a;
  Band bd;
  bd.M = sp.sh.M; bd.ncol = sp.sh.ncol; bd.BH = sp.sh.BH; bd.C = sp.sh.C;
  bd.rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  bd.col = tid % bd.ncol;
  const int grp = tid / bd.ncol;
  bd.active = (grp < sp.sh.G) && (bd.col < bd.M);
  bd.r0 = grp * K;
  bd.jbase = bd.rank * bd.BH;
  const int M = bd.M, ncol = bd.ncol, BH = bd.BH, C = bd.C;
  const size_t MM = (size_t)M * M;
  const float h = sp.h;
  const PayoffF pf = make_payoff(d);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* u = reinterpret_cast<float*>(smem_raw);   // state
  float* P = u + BH * ncol;                        // search direction p
  float* S = P + BH * ncol;                        // s
  float* RH = S + BH * ncol;                       // shadow residual r^
  float* ID = RH + BH * ncol;                      // inverse diagonal
  float4* rowt = reinterpret_cast<float4*>(ID + BH * ncol);
  double* wpart = reinterpret_cast<double*>(rowt + BH);   // [16 warps][4]
  double* slots = wpart + (kThreads / 32) * 4;            // [2][4]
  double* bcast = slots + 8;                              // [4]

  float* u_prev = bd.rank > 0 ? cluster.map_shared_rank(u, bd.rank - 1) : nullptr;
  float* u_next = bd.rank < C - 1 ? cluster.map_shared_rank(u, bd.rank + 1) : nullptr;
  float* P_prev = bd.rank > 0 ? cluster.map_shared_rank(P, bd.rank - 1) : nullptr;
  float* P_next = bd.rank < C - 1 ? cluster.map_shared_rank(P, bd.rank + 1) : nullptr;
  float* S_prev = bd.rank > 0 ? cluster.map_shared_rank(S, bd.rank - 1) : nullptr;
  float* S_next = bd.rank < C - 1 ? cluster.map_shared_rank(S, bd.rank + 1) : nullptr;

  for (int e = tid; e < BH * ncol; e += kThreads) {
    const int r = e / ncol, c = e - r * ncol;
    const int j = bd.jbase + r;
    ID[e] = (j < M - 1 && c < M - 1) ? inv_diag(d, c, j) : 0.f;
    P[e] = 0.f; S[e] = 0.f; RH[e] = 0.f;
  }
  for (int r = tid; r < BH; r += kThreads) {
    float cs, cn, gj;
    row_coefs(d, bd.jbase + r, cs, cn, gj);
    rowt[r] = make_float4(cs, cn, gj, 0.f);
  }
  float ce = 0.f, cw = 0.f, cgi = 0.f;
  if (bd.active) column_coefs(d, bd.col, ce, cw, cgi);
  const float rdt = (float)(d.r * d.dtau);
  int round = 0;

  // initial state of the first slice
  const float* src;
  if (a.mode == SWEEP_PROP) src = a.in;
  else if (a.mode == SWEEP_INIT) src = a.U;
  else src = a.Gold + (size_t)a.n_first * MM;   // ITER: G(u_k) is unchanged -> reuse G_old_k
  for (int e = tid; e < BH * ncol; e += kThreads) {
    const int r = e / ncol, c = e - r * ncol;
    const int j = bd.jbase + r;
    u[e] = (j < M && c < M) ? src[(size_t)j * M + c] : 0.f;
  }
  __syncthreads();

  const int n_end = (a.mode == SWEEP_PROP) ? a.n_first + 1 : a.N;
  bool failed = false;
  for (int n = a.n_first; n < n_end; ++n) {
    const bool skip_g = (a.mode == SWEEP_ITER && n == a.n_first);
    if (!skip_g) {
      for (int cstep = 0; cstep < a.csteps; ++cstep) {
        const double tau_new = d.tau0 + a.slice_len * n + (cstep + 1) * d.dtau;
        set_far_field_c(u, pf, (float)tau_new, h, bd, tid);
        cluster.sync();
        // b^ = D^{-1} dtau R_h w ; x = 0 ; r = r^ = p = b^
        float x[K], rr[K], vv[K], tt[K];
        double acc[1] = {0.0};
        if (bd.active) {
          const int col = bd.col, r0 = bd.r0;
          const int il = col > 0 ? col - 1 : 0, ir = col + 1 < ncol ? col + 1 : col;
          const float* up = (r0 == 0) ? (u_prev ? u_prev + (BH - 1) * ncol : u) : u + (r0 - 1) * ncol;
          float uW = up[il], uC = up[col], uE = up[ir];
          float cW = u[r0 * ncol + il], cC = u[r0 * ncol + col], cE = u[r0 * ncol + ir];
          const bool last_group = (r0 + K >= BH);
          float part = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int r = r0 + k, j = bd.jbase + r;
            const float* dn = (k < K - 1 || !last_group) ? u + (r + 1) * ncol
                                                         : (u_next ? u_next : u + (BH - 1) * ncol);
            const float dW = dn[il], dC = dn[col], dE = dn[ir];
            float bh = 0.f;
            if (j < M - 1 && col < M - 1) {
              const float4 rc = rowt[r];
              const float cg = cgi * rc.z;
              const float b = ce * (cE - cC) - cw * (cC - cW) + rc.x * (dC - cC) - rc.y * (cC - uC) +
                              cg * ((dE - uE) - (dW - uW)) - rdt * cC;
              bh = b * ID[r * ncol + col];
            }
            x[k] = 0.f; rr[k] = bh; vv[k] = 0.f; tt[k] = 0.f;
            part += bh * bh;
            uW = cW; uC = cC; uE = cE;
            cW = dW; cC = dC; cE = dE;
          }
          acc[0] = (double)part;
        } else {
#pragma unroll
          for (int k = 0; k < K; ++k) { x[k] = rr[k] = vv[k] = tt[k] = 0.f; }
        }
        // P and RH may still be read by neighbours of the previous solve: the cluster.sync
        // above ordered those reads before these writes.
        if (bd.active) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int idx = (bd.r0 + k) * ncol + bd.col;
            P[idx] = rr[k];
            RH[idx] = rr[k];
          }
        }
        cluster_sum<1>(cluster, acc, wpart, slots, bcast, round, C);   // publishes P
        const double bnorm2 = acc[0];
        double rho = bnorm2;
        double alpha = 1.0, omega = 1.0;
        const double stop2 = a.tol * a.tol * bnorm2;
        int it = 0;
        bool conv = (bnorm2 <= 1e-60);
        while (!conv && it < a.maxit) {
          ++it;
          // v = A^ p ; alpha = rho / (r^, v)
          double red1[1] = {0.0};
          if (bd.active) {
            scaled_matvec<K>(bd, P, P_prev, P_next, rowt, ID, ce, cw, cgi, vv);
            float part = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) part += RH[(bd.r0 + k) * ncol + bd.col] * vv[k];
            red1[0] = (double)part;
          }
          cluster_sum<1>(cluster, red1, wpart, slots, bcast, round, C);
          if (red1[0] == 0.0) { failed = true; break; }
          alpha = rho / red1[0];
          // s = r - alpha v
          if (bd.active) {
#pragma unroll
            for (int k = 0; k < K; ++k) S[(bd.r0 + k) * ncol + bd.col] = rr[k] - (float)alpha * vv[k];
          }
          cluster.sync();
          // t = A^ s ; omega = (t, s) / (t, t)
          double red2[2] = {0.0, 0.0};
          if (bd.active) {
            scaled_matvec<K>(bd, S, S_prev, S_next, rowt, ID, ce, cw, cgi, tt);
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const float sv = S[(bd.r0 + k) * ncol + bd.col];
              p0 += tt[k] * sv;
              p1 += tt[k] * tt[k];
            }
            red2[0] = (double)p0; red2[1] = (double)p1;
          }
          cluster_sum<2>(cluster, red2, wpart, slots, bcast, round, C);
          omega = (red2[1] > 0.0) ? red2[0] / red2[1] : 0.0;
          // x += alpha p + omega s ; r = s - omega t
          double red3[2] = {0.0, 0.0};
          if (bd.active) {
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int idx = (bd.r0 + k) * ncol + bd.col;
              const float sv = S[idx];
              x[k] += (float)alpha * P[idx] + (float)omega * sv;
              rr[k] = sv - (float)omega * tt[k];
              p0 += RH[idx] * rr[k];
              p1 += rr[k] * rr[k];
            }
            red3[0] = (double)p0; red3[1] = (double)p1;
          }
          cluster_sum<2>(cluster, red3, wpart, slots, bcast, round, C);
          if (red3[1] <= stop2) { conv = true; break; }
          if (omega == 0.0 || rho == 0.0) { failed = true; break; }
          const double beta = (red3[0] / rho) * (alpha / omega);
          rho = red3[0];
          if (bd.active) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int idx = (bd.r0 + k) * ncol + bd.col;
              P[idx] = rr[k] + (float)beta * (P[idx] - (float)omega * vv[k]);
            }
          }
          cluster.sync();
        }
        if (!conv) failed = true;
        // u^{m+1} = w + d on interior nodes (far-field nodes already hold g(tau_new))
        if (bd.active) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int r = bd.r0 + k, j = bd.jbase + r;
            if (j < M - 1 && bd.col < M - 1) u[r * ncol + bd.col] += x[k];
          }
        }
        cluster.sync();
      }
    }

    if (a.mode == SWEEP_PROP) {
      if (bd.active) {
        for (int k = 0; k < K; ++k) {
          const int j = bd.jbase + bd.r0 + k;
          if (j < M) a.out[(size_t)j * M + bd.col] = u[(bd.r0 + k) * ncol + bd.col];
        }
      }
    } else if (a.mode == SWEEP_INIT) {
      double nr[1] = {0.0};
      if (bd.active) {
        float* Un = a.U + (size_t)(n + 1) * MM;
        float* Gn = a.Gold + (size_t)n * MM;
        for (int k = 0; k < K; ++k) {
          const int j = bd.jbase + bd.r0 + k;
          if (j < M) {
            const float g = u[(bd.r0 + k) * ncol + bd.col];
            Un[(size_t)j * M + bd.col] = g;
            Gn[(size_t)j * M + bd.col] = g;
            nr[0] += (double)g * (double)g;
          }
        }
      }
      cluster_sum<1>(cluster, nr, wpart, slots, bcast, round, C);
      if (bd.rank == 0 && tid == 0) { a.norms[2 * (n + 1)] = nr[0]; a.norms[2 * (n + 1) + 1] = 0.0; }
    } else {
      // correction u_{n+1} = F_n + (G_new - G_old_n), defect partials
      double nr[2] = {0.0, 0.0};
      if (bd.active) {
        float* Un = a.U + (size_t)(n + 1) * MM;
        const float* Fn = a.Fb + (size_t)n * MM;
        float* Gn = a.Gold + (size_t)n * MM;
        for (int k = 0; k < K; ++k) {
          const int r = bd.r0 + k, j = bd.jbase + r;
          if (j < M) {
            const size_t gi = (size_t)j * M + bd.col;
            const float gnew = u[r * ncol + bd.col];
            const float unew = Fn[gi] + (gnew - Gn[gi]);
            const float uold = Un[gi];
            Un[gi] = unew;
            Gn[gi] = gnew;
            u[r * ncol + bd.col] = unew;
            const double du = (double)unew - (double)uold;
            nr[0] += (double)unew * (double)unew;
            nr[1] += du * du;
          }
        }
      }
      cluster_sum<2>(cluster, nr, wpart, slots, bcast, round, C);
      if (bd.rank == 0 && tid == 0) { a.norms[2 * (n + 1)] = nr[0]; a.norms[2 * (n + 1) + 1] = nr[1]; }
    }
  }

  if (bd.rank == 0 && tid == 0) {
    if (failed) atomicOr(a.status, 1);
    if (a.mode == SWEEP_ITER) {
      double num = 0.0, den = 0.0;
      for (int n = 1; n <= a.N; ++n) {
        den = fmax(den, a.norms[2 * n]);
        if (n >= a.n_first + 1) num = fmax(num, a.norms[2 * n + 1]);
      }
      a.defect[0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
    }
  }
}

template <int K>
static int launch_sweep_k(const bs_grid* g, const SweepParams& sp, cudaStream_t s) {
  const BandShape& sh = sp.sh;
  const size_t smem = (size_t)5 * sh.BH * sh.ncol * sizeof(float) + (size_t)sh.BH * sizeof(float4) +
                      ((kThreads / 32) * 4 + 8 + 4) * sizeof(double);
  auto kern = sweep_band_kernel<K>;
  BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (sh.C > 8) BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sh.C, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, sp));
  return BS_OK;
}

int launch_sweep(const bs_grid* g, const ItemDesc& d, const SweepArgs& a, cudaStream_t s) {
  SweepParams sp;
  sp.d = d;
  sp.a = a;
  sp.sh = g->shape;
  sp.h = (float)(g->xmax / (g->M - 1));
  if (sp.sh.C < 1 || sp.sh.C > kMaxCluster)
    return set_error(BS_ERR_ARG, "coarse propagator: grid M=%d not supported", g->M);
  return (sp.sh.K == 8) ? launch_sweep_k<8>(g, sp, s) : launch_sweep_k<16>(g, sp, s);
}

}  // namespace bsp
