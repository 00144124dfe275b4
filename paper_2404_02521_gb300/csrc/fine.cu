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

// One Jacobi sweep over the thread's column strip.  FIRST also evaluates b from hi;
// LAST also applies the increment to (hi, lo).
template <int K, bool FIRST, bool LAST>
__device__ __forceinline__ void fine_sweep(const float* __restrict__ rd, const float* rd_prev,
                                           const float* rd_next, float* __restrict__ wr,
                                           float* hi, const float* hi_prev, const float* hi_next,
                                           const float4* rowt, float* b, const float* invd,
                                           float* lo, int col, int r0, int jbase, int M,
                                           int ncol, int BH, float ce, float cw, float cgi,
                                           float rdt) {
  const int il = col > 0 ? col - 1 : 0;
  const int ir = col + 1 < ncol ? col + 1 : col;
  const float* up = (r0 == 0) ? (rd_prev ? rd_prev + (BH - 1) * ncol : rd) : rd + (r0 - 1) * ncol;
  float uW = up[il], uC = up[col], uE = up[ir];
  float cW = rd[r0 * ncol + il], cC = rd[r0 * ncol + col], cE = rd[r0 * ncol + ir];
  float huW = 0.f, huC = 0.f, huE = 0.f, hcW = 0.f, hcC = 0.f, hcE = 0.f;
  if (FIRST) {
    const float* hup = (r0 == 0) ? (hi_prev ? hi_prev + (BH - 1) * ncol : hi) : hi + (r0 - 1) * ncol;
    huW = hup[il]; huC = hup[col]; huE = hup[ir];
    hcW = hi[r0 * ncol + il]; hcC = hi[r0 * ncol + col]; hcE = hi[r0 * ncol + ir];
  }
  const bool last_group = (r0 + K >= BH);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int r = r0 + k;
    const int j = jbase + r;
    const float* dn;
    const float* hdn = nullptr;
    if (k < K - 1 || !last_group) {
      dn = rd + (r + 1) * ncol;
      if (FIRST) hdn = hi + (r + 1) * ncol;
    } else {
      dn = rd_next ? rd_next : rd + (BH - 1) * ncol;
      if (FIRST) hdn = hi_next ? hi_next : hi + (BH - 1) * ncol;
    }
    const float dW = dn[il], dC = dn[col], dE = dn[ir];
    float hdW = 0.f, hdC = 0.f, hdE = 0.f;
    if (FIRST) { hdW = hdn[il]; hdC = hdn[col]; hdE = hdn[ir]; }
    if (j < M - 1 && col < M - 1) {
      const float4 rc = rowt[r];
      const float cg = cgi * rc.z;
      if (FIRST) {
        b[k] = ce * (hcE - hcC) - cw * (hcC - hcW) + rc.x * (hdC - hcC) - rc.y * (hcC - huC) +
               cg * ((hdE - huE) - (hdW - huW)) - rdt * hcC;
      }
      const float v =
          (b[k] + ce * cE + cw * cW + rc.x * dC + rc.y * uC + cg * ((dE - uE) - (dW - uW))) * invd[k];
      wr[r * ncol + col] = v;
      if (LAST) {
        const float h0 = hi[r * ncol + col];
        const float s = h0 + v;
        const float bb = s - h0;
        const float err = (h0 - (s - bb)) + (v - bb);
        const float l = lo[k] + err;
        const float hn = s + l;
        lo[k] = l - (hn - s);
        hi[r * ncol + col] = hn;
      }
    }
    uW = cW; uC = cC; uE = cE;
    cW = dW; cC = dC; cE = dE;
    if (FIRST) {
      huW = hcW; huC = hcC; huE = hcE;
      hcW = hdW; hcC = hdC; hcE = hdE;
    }
  }
}

// Far-field values at tau for the band's Dirichlet nodes, written into hi.
__device__ __forceinline__ void set_far_field(float* hi, const PayoffF& pf, float tau, float h,
                                              int M, int ncol, int BH, int jbase, int tid) {
  const bool has_last_row = (jbase <= M - 1) && (M - 1 < jbase + BH);
  const int n_entries = BH + (has_last_row ? (M - 1) : 0);
  for (int e = tid; e < n_entries; e += kThreads) {
    int r, c;
    if (e < BH) { r = e; c = M - 1; if (jbase + r > M - 1) continue; }
    else { r = M - 1 - jbase; c = e - BH; }
    hi[r * ncol + c] = far_field(pf, c * h, (jbase + r) * h, tau);
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads, 1) fine_band_kernel(const __grid_constant__ FineBatch fb) {
  cg::cluster_group cluster = cg::this_cluster();
  const ItemDesc& d = fb.it[blockIdx.y];
  const int M = fb.sh.M, ncol = fb.sh.ncol, BH = fb.sh.BH, C = fb.sh.C;
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int col = tid % ncol, grp = tid / ncol;
  const bool active = (grp < fb.sh.G) && (col < M);
  const int r0 = grp * K;
  const int jbase = rank * BH;
  const float h = fb.h;
  const PayoffF pf = make_payoff(d);

  extern __shared__ __align__(16) float smem[];
  float* hi = smem;
  float* dA = hi + BH * ncol;
  float* dB = dA + BH * ncol;
  float4* rowt = reinterpret_cast<float4*>(dB + BH * ncol);

  for (int e = tid; e < BH * ncol; e += kThreads) {
    const int r = e / ncol, c = e - (e / ncol) * ncol;
    const int j = jbase + r;
    hi[e] = (j < M && c < M) ? d.in[(size_t)j * M + c] : 0.f;
    dA[e] = 0.f;
    dB[e] = 0.f;
  }
  for (int r = tid; r < BH; r += kThreads) {
    float cs, cn, gj;
    row_coefs(d, jbase + r, cs, cn, gj);
    rowt[r] = make_float4(cs, cn, gj, 0.f);
  }
  if (fb.nsteps > 0) {
    __syncthreads();
    set_far_field(hi, pf, (float)(d.tau0 + d.dtau), h, M, ncol, BH, jbase, tid);
  }

  float* hi_prev = rank > 0 ? cluster.map_shared_rank(hi, rank - 1) : nullptr;
  float* hi_next = rank < C - 1 ? cluster.map_shared_rank(hi, rank + 1) : nullptr;
  float* dA_prev = rank > 0 ? cluster.map_shared_rank(dA, rank - 1) : nullptr;
  float* dA_next = rank < C - 1 ? cluster.map_shared_rank(dA, rank + 1) : nullptr;
  float* dB_prev = rank > 0 ? cluster.map_shared_rank(dB, rank - 1) : nullptr;
  float* dB_next = rank < C - 1 ? cluster.map_shared_rank(dB, rank + 1) : nullptr;

  float ce = 0.f, cw = 0.f, cgi = 0.f;
  float b[K], invd[K], lo[K];
  if (active) column_coefs(d, col, ce, cw, cgi);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = jbase + r0 + k;
    invd[k] = (active && j < M) ? inv_diag(d, col, j) : 0.f;
    lo[k] = 0.f;
    b[k] = 0.f;
  }
  const float rdt = (float)(d.r * d.dtau);
  const int m = d.sweeps;
  cluster.sync();

  int par = 0;
  for (int step = 0; step < fb.nsteps; ++step) {
    for (int s = 0; s < m; ++s) {
      const float* rd = par ? dB : dA;
      float* wr = par ? dA : dB;
      const float* rp = par ? dB_prev : dA_prev;
      const float* rn = par ? dB_next : dA_next;
      if (active) {
        if (s == 0)
          fine_sweep<K, true, false>(rd, rp, rn, wr, hi, hi_prev, hi_next, rowt, b, invd, lo, col,
                                     r0, jbase, M, ncol, BH, ce, cw, cgi, rdt);
        else if (s == m - 1)
          fine_sweep<K, false, true>(rd, rp, rn, wr, hi, hi_prev, hi_next, rowt, b, invd, lo, col,
                                     r0, jbase, M, ncol, BH, ce, cw, cgi, rdt);
        else
          fine_sweep<K, false, false>(rd, rp, rn, wr, hi, hi_prev, hi_next, rowt, b, invd, lo,
                                      col, r0, jbase, M, ncol, BH, ce, cw, cgi, rdt);
      }
      // After the first sweep has read hi, move the far-field data to the next step.
      if (s == 1 && step + 1 < fb.nsteps)
        set_far_field(hi, pf, (float)(d.tau0 + (step + 2) * d.dtau), h, M, ncol, BH, jbase, tid);
      par ^= 1;
      cluster.sync();
    }
  }

  if (active) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = jbase + r0 + k;
      if (j < M) d.out[(size_t)j * M + col] = hi[(r0 + k) * ncol + col] + lo[k];
    }
  }
}

template <int K>
static int launch_band(const bs_grid* g, const FineBatch& fb, cudaStream_t s) {
  const BandShape& sh = fb.sh;
  const size_t smem = (size_t)3 * sh.BH * sh.ncol * sizeof(float) + (size_t)sh.BH * sizeof(float4);
  auto kern = fine_band_kernel<K>;
  BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (sh.C > 8) BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sh.C, fb.n, 1);
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
    int rc = (sh.K == 8) ? launch_band<8>(g, fb, s) : launch_band<16>(g, fb, s);
    if (rc != BS_OK) return rc;
  }
  return BS_OK;
}

}  // namespace bsp
