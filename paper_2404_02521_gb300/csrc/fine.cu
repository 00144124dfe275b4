// K1: fine propagator F (Sec. 3.1) -- implicit Euler steps of eq. (fd), batched over
// independent states (time slices and requests), one thread-block cluster per state.
//
// Each cluster keeps its whole M x M state on chip for all nsteps: CTA `rank` owns a band
// of BH rows (all ncol >= M columns) in shared memory, and the halo rows above and below
// the band are read from the neighbouring CTAs' shared memory (DSMEM) after a cluster
// barrier.  HBM is touched once to load the state and once to store it.
//
// Per implicit step  (I - dtau R_h) u^{m+1} = u^m  the increment  d = u^{m+1} - u^m  solves
//   (I - dtau R_h) d = dtau R_h w,   w = u^m inside, g(tau^{m+1}) on the far edges,
// with d = 0 on the far edges.  It is solved by Jacobi sweeps
//   d <- (b + sum_k c_k d_k) / (1 + sum_k c_k + r dtau),   b = dtau R_h w,
// started from the previous step's increment.  The Gershgorin bound q < 1 of the system
// (checked on the host) makes every sweep a max-norm contraction by q; the sweep count is
// chosen so that q^sweeps <= 2^-22.  The state is a compensated pair (hi, lo): u = hi + lo,
// updated by an error-free two-sum, so that increments below half an ulp of u are not lost
// over tens of thousands of steps; b is evaluated from hi.
#include <cooperative_groups.h>

#include <cstdio>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bsp {

struct FineBatch {
  ItemDesc it[kMaxItems];
  int n;
  int nsteps;
  BandShape sh;
  float h;
};

// Shape of the band kernel: NT threads, NCOL (>= M) columns, each thread owns one column
// and K consecutive rows of the band, G = NT / NCOL row groups, band height BH = G * K.
template <int NCOL, int NT, int K>
struct BandCfg {
  static constexpr int G = NT / NCOL;
  static constexpr int BH = G * K;
};

// Far-field values at tau for the band's Dirichlet nodes (column M-1 and, in the last band,
// row M-1), written into hi.  One evaluation per thread.
template <int NCOL, int NT, int BH>
__device__ __forceinline__ void set_far_field(float* hi, const PayoffF& pf, float tau, float h,
                                              int M, int jbase, int tid) {
  const bool has_last_row = (jbase <= M - 1) && (M - 1 < jbase + BH);
  const int n_entries = BH + (has_last_row ? (M - 1) : 0);
  for (int e = tid; e < n_entries; e += NT) {
    int r, c;
    if (e < BH) {
      r = e;
      c = M - 1;
      if (jbase + r > M - 1) continue;
    } else {
      r = M - 1 - jbase;
      c = e - BH;
    }
    hi[r * NCOL + c] = far_field(pf, c * h, (jbase + r) * h, tau);
  }
}

// One Jacobi sweep over the thread's column strip.  The thread's own column of the old
// increment is in dv[] (registers); west/east columns and the rows just outside the strip
// come from shared memory (rows outside the band from the neighbouring CTAs).  FIRST also
// evaluates b = dtau R_h w from hi; LAST also applies the increment to (hi, lo).
// Non-interior nodes have invd = 0, so they write a zero increment without a branch.
template <int NCOL, int K, bool FIRST, bool LAST>
__device__ __forceinline__ void fine_sweep(const float* __restrict__ rd, float* __restrict__ wr,
                                           const float* upr, const float* dnr, float* hi,
                                           const float* hup, const float* hdn,
                                           const float2* __restrict__ rowc, float (&dv)[K],
                                           float (&b)[K], const float (&invd)[K], float (&lo)[K],
                                           int col, int il, int ir, int r0, float ce, float cw,
                                           float cg0, float cgi, float rdt) {
  // rows r0-1 and r0+K (halo of the strip)
  float nW = upr[il], nC = upr[col], nE = upr[ir];
  const float sDW = dnr[il], sDC = dnr[col], sDE = dnr[ir];
  float cW = rd[r0 * NCOL + il], cE = rd[r0 * NCOL + ir];
  float hnW = 0.f, hnC = 0.f, hnE = 0.f, hcW = 0.f, hcC = 0.f, hcE = 0.f;
  float hsDW = 0.f, hsDC = 0.f, hsDE = 0.f;
  if (FIRST) {
    hnW = hup[il]; hnC = hup[col]; hnE = hup[ir];
    hcW = hi[r0 * NCOL + il]; hcC = hi[r0 * NCOL + col]; hcE = hi[r0 * NCOL + ir];
    hsDW = hdn[il]; hsDC = hdn[col]; hsDE = hdn[ir];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int r = r0 + k;
    float sW, sC, sE;
    if (k < K - 1) {
      sW = rd[(r + 1) * NCOL + il];
      sE = rd[(r + 1) * NCOL + ir];
      sC = dv[k + 1];
    } else {
      sW = sDW; sC = sDC; sE = sDE;
    }
    const float2 rc = rowc[r];
    const float cg = fmaf((float)k, cgi, cg0);
    if (FIRST) {
      float hsW, hsC, hsE;
      if (k < K - 1) {
        hsW = hi[(r + 1) * NCOL + il]; hsC = hi[(r + 1) * NCOL + col]; hsE = hi[(r + 1) * NCOL + ir];
      } else {
        hsW = hsDW; hsC = hsDC; hsE = hsDE;
      }
      b[k] = ce * (hcE - hcC) - cw * (hcC - hcW) + rc.x * (hsC - hcC) - rc.y * (hcC - hnC) +
             cg * ((hsE - hnE) - (hsW - hnW)) - rdt * hcC;
      hnW = hcW; hnC = hcC; hnE = hcE;
      hcW = hsW; hcC = hsC; hcE = hsE;
    }
    const float v = (b[k] + ce * cE + cw * cW + rc.x * sC + rc.y * nC + cg * ((sE - nE) - (sW - nW))) * invd[k];
    wr[r * NCOL + col] = v;
    nC = dv[k];
    dv[k] = v;
    nW = cW; nE = cE;
    cW = sW; cE = sE;
    if (LAST) {
      const float h0 = hi[r * NCOL + col];
      const float s = h0 + v;
      const float bb = s - h0;
      const float err = (h0 - (s - bb)) + (v - bb);
      const float l = lo[k] + err;
      const float hn = s + l;
      lo[k] = l - (hn - s);
      hi[r * NCOL + col] = hn;
    }
  }
}

template <int NCOL, int NT, int K>
__global__ void __launch_bounds__(NT, 1) fine_band_kernel(const __grid_constant__ FineBatch fb) {
  constexpr int G = BandCfg<NCOL, NT, K>::G;
  constexpr int BH = BandCfg<NCOL, NT, K>::BH;
  cg::cluster_group cluster = cg::this_cluster();
  const ItemDesc& d = fb.it[blockIdx.y];
  const int M = fb.sh.M, C = fb.sh.C;
  const int rank = C > 1 ? (int)cluster.block_rank() : 0;
  const int tid = threadIdx.x;
  const int col = tid % NCOL, grp = tid / NCOL;
  const int r0 = grp * K;
  const int jbase = rank * BH;
  const float h = fb.h;
  const PayoffF pf = make_payoff(d);

  extern __shared__ __align__(16) float smem[];
  float* hi = smem;
  float* dA = hi + BH * NCOL;
  float* dB = dA + BH * NCOL;
  float2* rowc = reinterpret_cast<float2*>(dB + BH * NCOL);

  for (int e = tid; e < BH * NCOL; e += NT) {
    const int r = e / NCOL, c = e % NCOL;
    const int j = jbase + r;
    hi[e] = (j < M && c < M) ? d.in[(size_t)j * M + c] : 0.f;
    dA[e] = 0.f;
    dB[e] = 0.f;
  }
  for (int r = tid; r < BH; r += NT) {
    float cs, cn, gj;
    row_coefs(d, jbase + r, cs, cn, gj);
    rowc[r] = make_float2(cs, cn);
  }
  if (fb.nsteps > 0) {
    __syncthreads();
    set_far_field<NCOL, NT, BH>(hi, pf, (float)(d.tau0 + d.dtau), h, M, jbase, tid);
  }

  // halo-row sources: rows r0-1 and r0+K of each buffer (clamped at the domain edges, where
  // the coefficients that would use them vanish or the node is not a PDE row)
  const bool has_prev = rank > 0, has_next = rank < C - 1;
  auto up_row = [&](float* buf) -> const float* {
    if (grp > 0) return buf + (r0 - 1) * NCOL;
    return has_prev ? cluster.map_shared_rank(buf, rank - 1) + (BH - 1) * NCOL : buf;
  };
  auto dn_row = [&](float* buf) -> const float* {
    if (grp < G - 1) return buf + (r0 + K) * NCOL;
    return has_next ? cluster.map_shared_rank(buf, rank + 1) : buf + (BH - 1) * NCOL;
  };
  const float* upA = up_row(dA);
  const float* dnA = dn_row(dA);
  const float* upB = up_row(dB);
  const float* dnB = dn_row(dB);
  const float* hup = up_row(hi);
  const float* hdn = dn_row(hi);

  float ce = 0.f, cw = 0.f, cgi = 0.f;
  column_coefs(d, col, ce, cw, cgi);
  const float cg0 = cgi * (float)(jbase + r0);
  float dv[K], b[K], invd[K], lo[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = jbase + r0 + k;
    invd[k] = (j < M - 1 && col < M - 1) ? inv_diag(d, col, j) : 0.f;
    lo[k] = 0.f;
    b[k] = 0.f;
    dv[k] = 0.f;
  }
  const int il = col > 0 ? col - 1 : 0;
  const int ir = col + 1 < NCOL ? col + 1 : col;
  const float rdt = (float)(d.r * d.dtau);
  const int m = d.sweeps;
  if (C > 1) cluster.sync(); else __syncthreads();

  int par = 0;
  for (int step = 0; step < fb.nsteps; ++step) {
    for (int s = 0; s < m; ++s) {
      const float* rd = par ? dB : dA;
      float* wr = par ? dA : dB;
      const float* upr = par ? upB : upA;
      const float* dnr = par ? dnB : dnA;
      if (s == 0)
        fine_sweep<NCOL, K, true, false>(rd, wr, upr, dnr, hi, hup, hdn, rowc, dv, b, invd, lo, col,
                                         il, ir, r0, ce, cw, cg0, cgi, rdt);
      else if (s == m - 1)
        fine_sweep<NCOL, K, false, true>(rd, wr, upr, dnr, hi, hup, hdn, rowc, dv, b, invd, lo, col,
                                         il, ir, r0, ce, cw, cg0, cgi, rdt);
      else
        fine_sweep<NCOL, K, false, false>(rd, wr, upr, dnr, hi, hup, hdn, rowc, dv, b, invd, lo,
                                          col, il, ir, r0, ce, cw, cg0, cgi, rdt);
      // After the first sweep has read hi, move the far-field data to the next step (the
      // last sweep, at least one barrier later, leaves those nodes unchanged).
      if (s == 1 && step + 1 < fb.nsteps)
        set_far_field<NCOL, NT, BH>(hi, pf, (float)(d.tau0 + (step + 2) * d.dtau), h, M, jbase, tid);
      par ^= 1;
      if (C > 1) cluster.sync(); else __syncthreads();
    }
  }

  if (col < M) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = jbase + r0 + k;
      if (j < M) d.out[(size_t)j * M + col] = hi[(r0 + k) * NCOL + col] + lo[k];
    }
  }
}

template <int NCOL, int NT, int K>
static int launch_band(const bs_grid* g, const FineBatch& fb, cudaStream_t s) {
  constexpr int BH = BandCfg<NCOL, NT, K>::BH;
  const size_t smem = (size_t)3 * BH * NCOL * sizeof(float) + (size_t)BH * sizeof(float2);
  auto kern = fine_band_kernel<NCOL, NT, K>;
  BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (fb.sh.C > 8) BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(fb.sh.C, fb.n, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = fb.sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, fb));
  return BS_OK;
}

int launch_fine(const bs_grid* g, const ItemDesc* items, int n, int nsteps, cudaStream_t s) {
  const BandShape sh = g->shape;
  if (sh.C < 1 || sh.C > kMaxCluster)
    return set_error(BS_ERR_ARG, "fine_propagate_batched: grid M=%d is not supported by the "
                                 "cluster-resident stepper", g->M);
  for (int base = 0; base < n; base += kMaxItems) {
    FineBatch fb;
    fb.n = (n - base) < kMaxItems ? (n - base) : kMaxItems;
    for (int k = 0; k < fb.n; ++k) fb.it[k] = items[base + k];
    fb.nsteps = nsteps;
    fb.sh = sh;
    fb.h = (float)(g->xmax / (g->M - 1));
    int rc;
    switch (sh.ncol) {
      case 32: rc = launch_band<32, 256, 4>(g, fb, s); break;
      case 64: rc = launch_band<64, 512, 8>(g, fb, s); break;
      case 128: rc = launch_band<128, 512, 16>(g, fb, s); break;
      case 256: rc = launch_band<256, 512, 16>(g, fb, s); break;
      default: rc = set_error(BS_ERR_ARG, "fine_propagate_batched: no band shape for M=%d", g->M);
    }
    if (rc != BS_OK) return rc;
  }
  return BS_OK;
}

}  // namespace bsp
