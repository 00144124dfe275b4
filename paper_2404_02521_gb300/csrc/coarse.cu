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

template <int NCOL, int NT, int K>
struct CBand {
  static constexpr int G = NT / NCOL;
  static constexpr int BH = G * K;
  static constexpr int NW = NT / 32;
};

// Jacobi-scaled operator A^ y = y - invd * (off-diagonal part of dtau R_h) y on the thread's
// column strip; zero on non-interior nodes (invd = 0 there and y = 0 there).
template <int NCOL, int K>
__device__ __forceinline__ void scaled_matvec(const float* __restrict__ y, const float* upr,
                                              const float* dnr, const float2* __restrict__ rowc,
                                              const float* __restrict__ ID, int col, int il,
                                              int ir, int r0, float ce, float cw, float cg0,
                                              float cgi, float (&out)[K]) {
  float nW = upr[il], nC = upr[col], nE = upr[ir];
  const float sDW = dnr[il], sDC = dnr[col], sDE = dnr[ir];
  float cW = y[r0 * NCOL + il], cC = y[r0 * NCOL + col], cE = y[r0 * NCOL + ir];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int r = r0 + k;
    float sW, sC, sE;
    if (k < K - 1) {
      sW = y[(r + 1) * NCOL + il]; sC = y[(r + 1) * NCOL + col]; sE = y[(r + 1) * NCOL + ir];
    } else {
      sW = sDW; sC = sDC; sE = sDE;
    }
    const float2 rc = rowc[r];
    const float cg = fmaf((float)k, cgi, cg0);
    out[k] = cC - ID[r * NCOL + col] *
                      (ce * cE + cw * cW + rc.x * sC + rc.y * nC + cg * ((sE - nE) - (sW - nW)));
    nW = cW; nC = cC; nE = cE;
    cW = sW; cC = sC; cE = sE;
  }
}

// Deterministic cluster-wide sum of NV values: butterfly within each warp, butterfly of
// the warp partials in warp 0, then one lane per CTA of the cluster reads that CTA's
// partial and warp 0 sums them by butterfly.  A butterfly gives every lane the same bits
// (each level adds the same two operands), so every CTA obtains identical totals.
// `round` alternates the slot so a fast CTA never overwrites partials still being read.
template <int NV, int NW>
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
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = lane < NW ? wpart[lane * NV + q] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if (C == 1) {
        if (lane == 0) bcast[q] = x;
      } else if (lane == 0) {
        slot[q] = x;
      }
    }
  }
  if (C > 1) {
    cluster.sync();
    if (warp == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        double x = lane < C ? cluster.map_shared_rank(slot, lane)[q] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) bcast[q] = x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = bcast[q];
  ++round;
}

template <int NCOL, int NT, int BH>
__device__ __forceinline__ void set_far_field_c(float* u, const PayoffF& pf, float tau, float h,
                                                int M, int jbase, int tid) {
  const bool has_last_row = (jbase <= M - 1) && (M - 1 < jbase + BH);
  const int n_entries = BH + (has_last_row ? (M - 1) : 0);
  for (int e = tid; e < n_entries; e += NT) {
    int r, c;
    if (e < BH) { r = e; c = M - 1; if (jbase + r > M - 1) continue; }
    else { r = M - 1 - jbase; c = e - BH; }
    u[r * NCOL + c] = far_field(pf, c * h, (jbase + r) * h, tau);
  }
}

template <int NCOL, int NT, int K>
__global__ void __launch_bounds__(NT, 1) sweep_band_kernel(const __grid_constant__ SweepParams sp) {
  using CB = CBand<NCOL, NT, K>;
  constexpr int G = CB::G, BH = CB::BH, NW = CB::NW;
  cg::cluster_group cluster = cg::this_cluster();
  const ItemDesc& d = sp.d;
  const SweepArgs& a = sp.a;
  const int M = sp.sh.M, C = sp.sh.C;
  const int rank = C > 1 ? (int)cluster.block_rank() : 0;
  const int tid = threadIdx.x;
  const int col = tid % NCOL, grp = tid / NCOL;
  const int r0 = grp * K;
  const int jbase = rank * BH;
  const size_t MM = (size_t)M * M;
  const float h = sp.h;
  const PayoffF pf = make_payoff(d);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* u = reinterpret_cast<float*>(smem_raw);   // state w / u
  float* P = u + BH * NCOL;                        // search direction p
  float* S = P + BH * NCOL;                        // s
  float* RH = S + BH * NCOL;                       // shadow residual r^
  float* ID = RH + BH * NCOL;                      // inverse diagonal (0 off the PDE rows)
  float2* rowc = reinterpret_cast<float2*>(ID + BH * NCOL);
  double* wpart = reinterpret_cast<double*>(rowc + BH);   // [NW][4]
  double* slots = wpart + NW * 4;                         // [2][4]
  double* bcast = slots + 8;                              // [4]

  const bool has_prev = rank > 0, has_next = rank < C - 1;
  auto up_row = [&](float* buf) -> const float* {
    if (grp > 0) return buf + (r0 - 1) * NCOL;
    return has_prev ? cluster.map_shared_rank(buf, rank - 1) + (BH - 1) * NCOL : buf;
  };
  auto dn_row = [&](float* buf) -> const float* {
    if (grp < G - 1) return buf + (r0 + K) * NCOL;
    return has_next ? cluster.map_shared_rank(buf, rank + 1) : buf + (BH - 1) * NCOL;
  };
  const float* u_up = up_row(u);
  const float* u_dn = dn_row(u);
  const float* P_up = up_row(P);
  const float* P_dn = dn_row(P);
  const float* S_up = up_row(S);
  const float* S_dn = dn_row(S);

  for (int e = tid; e < BH * NCOL; e += NT) {
    const int r = e / NCOL, c = e % NCOL;
    const int j = jbase + r;
    ID[e] = (j < M - 1 && c < M - 1) ? inv_diag(d, c, j) : 0.f;
    P[e] = 0.f; S[e] = 0.f; RH[e] = 0.f;
  }
  for (int r = tid; r < BH; r += NT) {
    float cs, cn, gj;
    row_coefs(d, jbase + r, cs, cn, gj);
    rowc[r] = make_float2(cs, cn);
  }
  float ce = 0.f, cw = 0.f, cgi = 0.f;
  column_coefs(d, col, ce, cw, cgi);
  const float cg0 = cgi * (float)(jbase + r0);
  const int il = col > 0 ? col - 1 : 0;
  const int ir = col + 1 < NCOL ? col + 1 : col;
  const float rdt = (float)(d.r * d.dtau);
  int round = 0;
  int iters_max = 0;

  // initial state of the first slice
  const float* src;
  if (a.mode == SWEEP_PROP) src = a.in;
  else if (a.mode == SWEEP_INIT) src = a.U;
  else src = a.Gold + (size_t)a.n_first * MM;   // ITER: G(u_k) is unchanged -> reuse G_old_k
  for (int e = tid; e < BH * NCOL; e += NT) {
    const int r = e / NCOL, c = e % NCOL;
    const int j = jbase + r;
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
        set_far_field_c<NCOL, NT, BH>(u, pf, (float)tau_new, h, M, jbase, tid);
        if (C > 1) cluster.sync(); else __syncthreads();
        // b^ = D^{-1} dtau R_h w ;  x = 0 ;  r = r^ = p = b^
        float x[K], rr[K], vv[K], tt[K];
        double acc[1];
        {
          float nW = u_up[il], nC = u_up[col], nE = u_up[ir];
          float cW = u[r0 * NCOL + il], cC = u[r0 * NCOL + col], cE = u[r0 * NCOL + ir];
          float part = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int r = r0 + k;
            float sW, sC, sE;
            if (k < K - 1) {
              sW = u[(r + 1) * NCOL + il]; sC = u[(r + 1) * NCOL + col]; sE = u[(r + 1) * NCOL + ir];
            } else {
              sW = u_dn[il]; sC = u_dn[col]; sE = u_dn[ir];
            }
            const float2 rc = rowc[r];
            const float cg = fmaf((float)k, cgi, cg0);
            const float b = ce * (cE - cC) - cw * (cC - cW) + rc.x * (sC - cC) - rc.y * (cC - nC) +
                            cg * ((sE - nE) - (sW - nW)) - rdt * cC;
            const float bh = b * ID[r * NCOL + col];
            x[k] = 0.f; rr[k] = bh; vv[k] = 0.f; tt[k] = 0.f;
            part = fmaf(bh, bh, part);
            nW = cW; nC = cC; nE = cE;
            cW = sW; cC = sC; cE = sE;
          }
          acc[0] = (double)part;
        }
        // P and RH are not read by anyone between the barrier above and the next one.
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int idx = (r0 + k) * NCOL + col;
          P[idx] = rr[k];
          RH[idx] = rr[k];
        }
        cluster_sum<1, NW>(cluster, acc, wpart, slots, bcast, round, C);   // also publishes P
        const double bnorm2 = acc[0];
        double rho = bnorm2;
        double alpha = 1.0, omega = 1.0;
        const double stop2 = a.tol * a.tol * bnorm2;
        int it = 0;
        bool conv = (bnorm2 <= 1e-60);
        while (!conv && it < a.maxit) {
          ++it;
          // v = A^ p ;  alpha = rho / (r^, v)
          scaled_matvec<NCOL, K>(P, P_up, P_dn, rowc, ID, col, il, ir, r0, ce, cw, cg0, cgi, vv);
          double red1[1];
          {
            float part = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) part = fmaf(RH[(r0 + k) * NCOL + col], vv[k], part);
            red1[0] = (double)part;
          }
          cluster_sum<1, NW>(cluster, red1, wpart, slots, bcast, round, C);
          if (red1[0] == 0.0) { failed = true; break; }
          alpha = rho / red1[0];
          const float af = (float)alpha;
          // s = r - alpha v
#pragma unroll
          for (int k = 0; k < K; ++k) S[(r0 + k) * NCOL + col] = fmaf(-af, vv[k], rr[k]);
          if (C > 1) cluster.sync(); else __syncthreads();
          // t = A^ s ;  omega = (t, s) / (t, t)
          scaled_matvec<NCOL, K>(S, S_up, S_dn, rowc, ID, col, il, ir, r0, ce, cw, cg0, cgi, tt);
          double red2[2];
          {
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const float sv = S[(r0 + k) * NCOL + col];
              p0 = fmaf(tt[k], sv, p0);
              p1 = fmaf(tt[k], tt[k], p1);
            }
            red2[0] = (double)p0; red2[1] = (double)p1;
          }
          cluster_sum<2, NW>(cluster, red2, wpart, slots, bcast, round, C);
          omega = (red2[1] > 0.0) ? red2[0] / red2[1] : 0.0;
          const float of = (float)omega;
          // x += alpha p + omega s ;  r = s - omega t
          double red3[2];
          {
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int idx = (r0 + k) * NCOL + col;
              const float sv = S[idx];
              x[k] += af * P[idx] + of * sv;
              rr[k] = fmaf(-of, tt[k], sv);
              p0 = fmaf(RH[idx], rr[k], p0);
              p1 = fmaf(rr[k], rr[k], p1);
            }
            red3[0] = (double)p0; red3[1] = (double)p1;
          }
          cluster_sum<2, NW>(cluster, red3, wpart, slots, bcast, round, C);
          if (red3[1] <= stop2) { conv = true; break; }
          if (omega == 0.0 || rho == 0.0) { failed = true; break; }
          const double beta = (red3[0] / rho) * (alpha / omega);
          rho = red3[0];
          const float bf = (float)beta;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int idx = (r0 + k) * NCOL + col;
            P[idx] = rr[k] + bf * (P[idx] - of * vv[k]);
          }
          if (C > 1) cluster.sync(); else __syncthreads();
        }
        if (!conv) failed = true;
        iters_max = it > iters_max ? it : iters_max;
        // u^{m+1} = w + d (x = 0 off the PDE rows, whose values already hold g(tau_new))
#pragma unroll
        for (int k = 0; k < K; ++k) u[(r0 + k) * NCOL + col] += x[k];
        if (C > 1) cluster.sync(); else __syncthreads();
      }
    }

    if (a.mode == SWEEP_PROP) {
      if (col < M) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = jbase + r0 + k;
          if (j < M) a.out[(size_t)j * M + col] = u[(r0 + k) * NCOL + col];
        }
      }
    } else if (a.mode == SWEEP_INIT) {
      double nr[1] = {0.0};
      if (col < M) {
        float* Un = a.U + (size_t)(n + 1) * MM;
        float* Gn = a.Gold + (size_t)n * MM;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = jbase + r0 + k;
          if (j < M) {
            const float g = u[(r0 + k) * NCOL + col];
            Un[(size_t)j * M + col] = g;
            Gn[(size_t)j * M + col] = g;
            nr[0] += (double)g * (double)g;
          }
        }
      }
      cluster_sum<1, NW>(cluster, nr, wpart, slots, bcast, round, C);
      if (rank == 0 && tid == 0) { a.norms[2 * (n + 1)] = nr[0]; a.norms[2 * (n + 1) + 1] = 0.0; }
    } else {
      // correction u_{n+1} = F_n + (G_new - G_old_n) and defect partials
      double nr[2] = {0.0, 0.0};
      if (col < M) {
        float* Un = a.U + (size_t)(n + 1) * MM;
        const float* Fn = a.Fb + (size_t)n * MM;
        float* Gn = a.Gold + (size_t)n * MM;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int r = r0 + k, j = jbase + r;
          if (j < M) {
            const size_t gi = (size_t)j * M + col;
            const float gnew = u[r * NCOL + col];
            const float unew = Fn[gi] + (gnew - Gn[gi]);
            const float uold = Un[gi];
            Un[gi] = unew;
            Gn[gi] = gnew;
            u[r * NCOL + col] = unew;
            const double du = (double)unew - (double)uold;
            nr[0] += (double)unew * (double)unew;
            nr[1] += du * du;
          }
        }
      }
      cluster_sum<2, NW>(cluster, nr, wpart, slots, bcast, round, C);
      if (rank == 0 && tid == 0) { a.norms[2 * (n + 1)] = nr[0]; a.norms[2 * (n + 1) + 1] = nr[1]; }
    }
  }

  if (rank == 0 && tid == 0) {
    if (failed) atomicOr(a.status, 1);
    atomicMax(a.status + 1, iters_max);
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

template <int NCOL, int NT, int K>
static int launch_sweep_k(const bs_grid* g, const SweepParams& sp, cudaStream_t s) {
  using CB = CBand<NCOL, NT, K>;
  const size_t smem = (size_t)5 * CB::BH * NCOL * sizeof(float) + (size_t)CB::BH * sizeof(float2) +
                      (CB::NW * 4 + 8 + 4) * sizeof(double);
  auto kern = sweep_band_kernel<NCOL, NT, K>;
  BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (sp.sh.C > 8) BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sp.sh.C, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sp.sh.C;
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
  switch (sp.sh.ncol) {
    case 32: return launch_sweep_k<32, 256, 4>(g, sp, s);
    case 64: return launch_sweep_k<64, 512, 8>(g, sp, s);
    case 128: return launch_sweep_k<128, 512, 16>(g, sp, s);
    case 256: return launch_sweep_k<256, 512, 16>(g, sp, s);
  }
  return set_error(BS_ERR_ARG, "coarse propagator: no band shape for M=%d", g->M);
}

}  // namespace bsp
