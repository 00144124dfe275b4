// K1: fine propagator F (Sec. 3.1) -- implicit Euler steps of eq. (fd), batched over
// independent states (time slices and requests), one thread-block cluster per state.
//
// Each cluster keeps its whole M x M state on chip for all nsteps (band layout of
// band.cuh): HBM is touched once to load the state and once to store it.
//
// Per implicit step  (I - dtau R_h) u^{m+1} = u^m  the increment  d = u^{m+1} - u^m  solves
//   (I - dtau R_h) d = dtau R_h w,   w = u^m inside, g(tau^{m+1}) on the far edges,
// with d = 0 on the far edges.  It is solved by Jacobi sweeps
//   d <- (b + sum_k c_k d_k) / (1 + sum_k c_k + r dtau),   b = dtau R_h w,
// started from the previous step's increment.  The Gershgorin bound q < 1 of the system
// (checked on the host) makes every sweep a max-norm contraction by q; the sweep count is
// chosen so that q^sweeps is below a target (2^-22 for the first, cold-started step of a
// launch, 2^-10 for the warm-started steps after it).  The state is a compensated
// pair (hi, lo): u = hi + lo, updated by an error-free two-sum, so that increments below half
// an ulp of u are not lost over tens of thousands of steps; b is evaluated from hi.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "band.cuh"

namespace bsp {

struct FineBatch {
  ItemDesc it[kMaxItems];
  int n;
  int nsteps;
  BandShape sh;
  float h;
};

__device__ __forceinline__ void cl_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// b = dtau R_h w at one node from the 3x3 neighbourhood of hi (eq. fd in index units).  This
// file is compiled without implicit contraction; the multiply-adds are explicit, so every
// kernel that instantiates the stencil rounds it alike.
__device__ __forceinline__ float rhs_point(float ce, float cw, float cs, float cn, float cg, float rdt,
                                           float nW, float nC, float nE, float cW, float cC,
                                           float cE, float sW, float sC, float sE) {
  float t = ce * (cE - cC);
  t = fmaf(-cw, cC - cW, t);
  t = fmaf(cs, sC - cC, t);
  t = fmaf(-cn, cC - nC, t);
  t = fmaf(cg, (sE - nE) - (sW - nW), t);
  return fmaf(-rdt, cC, t);
}

// Jacobi update of one node from the old increments around it: the four axis neighbours join
// b in one chain of fused multiply-adds, then the mixed term, then the diagonal scale.
__device__ __forceinline__ float jacobi_point(float b, float invd, float ce, float cw, float cs,
                                              float cn, float cg, float nW, float nC, float nE,
                                              float cW, float cE, float sW, float sC, float sE) {
  const float t = fmaf(cn, nC, fmaf(cs, sC, fmaf(ce, cE, fmaf(cw, cW, b))));
  return fmaf(cg, (sE - nE) - (sW - nW), t) * invd;
}

// Asynchronous 4-byte global -> shared copy; with ok == false the destination is zero-filled
// and nothing is read.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Compensated update (hi, lo) += v: error-free two-sum, then renormalise.
__device__ __forceinline__ float two_sum_update(float h0, float v, float& lo) {
  const float s = h0 + v;
  const float bb = s - h0;
  const float err = (h0 - (s - bb)) + (v - bb);
  const float l = lo + err;
  const float hn = s + l;
  lo = l - (hn - s);
  return hn;
}

// Initial guess of the next step from this step's increment v: with extrap, the linear
// extrapolation 2 d_m - d_{m-1} (d_{m-1} from dp, own rows), else v itself; dp <- v.
__device__ __forceinline__ float next_guess(float v, float* dp, int e, bool extrap) {
  if (!dp) return v;
  const float prev = dp[e];
  dp[e] = v;
  return extrap ? fmaf(2.f, v, -prev) : v;
}

// next_guess with the mode fixed at compile time, so that the sweeps carry no per-node select:
// XM = 0 no history (guess = v), 1 history kept (guess = v), 2 history kept and the guess
// extrapolated.
template <int XM>
__device__ __forceinline__ float next_guess_x(float v, float* dp, int e) {
  if (XM == 0) return v;
  const float prev = dp[e];
  dp[e] = v;
  return XM == 2 ? fmaf(2.f, v, -prev) : v;
}

// One Jacobi sweep over the thread's column strip (own band rows r0..r0+K-1, plane rows
// r0+1..r0+K).  Strip rows 1..K-2 read only rows of the strip itself, written by this CTA
// in the previous sweep; they are updated before the cluster wait.  The two end rows read
// the rows just outside the strip (other row groups or the halo copies of the neighbouring
// CTAs) and are updated after it, so the barrier latency overlaps the interior work.
// The thread's own column of the old increment is in dv[]; lo[k] is the compensation word of
// strip row k (registers, or shared memory through StripLo).  FIRST also evaluates
// b = dtau R_h w from hi; LAST also applies the increment to (hi, lo) of the PDE nodes and
// leaves the next step's initial guess (next_guess_x<XM>, history in dp) in wr and dv[].  Nodes
// that are not PDE rows have invd = 0 and write a zero increment; LAST leaves their hi
// (Dirichlet data) to the far-field update, which may follow it directly, unless UNCOND: then
// every node takes the compensated update, which leaves hi as it is where v = 0 and lo = 0 (a
// kernel may choose this only where each far-field value is written by the thread that owns
// the node, after its sweep).  The plane rows are addressed from per-thread base pointers at
// the row north of the strip, so every access in the unrolled rows is a constant offset.
template <class CFG, bool FIRST, bool LAST, class LoT, int XM = 0, bool UNCOND = false>
__device__ __forceinline__ void fine_sweep(const float* __restrict__ rd, float* __restrict__ wr,
                                           float* hi, const HaloPush& wr_push,
                                           const HaloPush& hi_push, const float4* __restrict__ rowc,
                                           float (&dv)[CFG::K], float (&b)[CFG::K],
                                           const float (&invd)[CFG::K], LoT& lo,
                                           int col, int il, int ir, int r0, float ce, float cw,
                                           float cgi, float rdt, bool clustered,
                                           float* dp = nullptr) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K;
  static_assert(K >= 4, "strip needs interior rows");
  const int p0 = r0 + 1;
  // base pointers at plane row p0 - 1 = r0 (the row north of the strip)
  const float* rW = rd + r0 * NCOL + il;
  const float* rC = rd + r0 * NCOL + col;
  const float* rE = rd + r0 * NCOL + ir;
  const float* hW = hi + r0 * NCOL + il;
  const float* hC = hi + r0 * NCOL + col;
  const float* hE = hi + r0 * NCOL + ir;
  float* hO = hi + r0 * NCOL + col;
  float* wO = wr + r0 * NCOL + col;
  float* dO = dp ? dp + r0 * NCOL + col : nullptr;   // own row k at dO[k * NCOL]
  const float4* rcs = rowc + r0;
  // rows 0 and 1 of the strip (plane rows p0, p0 + 1 at offsets 1, 2)
  const float r0W = rW[NCOL], r0E = rE[NCOL];
  const float r1W = rW[2 * NCOL], r1E = rE[2 * NCOL];
  const float dv1_old = dv[1];
  float nW = r0W, nC = dv[0], nE = r0E;
  float cW = r1W, cE = r1E;
  float h0W = 0.f, h0C = 0.f, h0E = 0.f, h1W = 0.f, h1C = 0.f, h1E = 0.f;
  float hnW = 0.f, hnC = 0.f, hnE = 0.f, hcW = 0.f, hcC = 0.f, hcE = 0.f;
  if (FIRST) {
    h0W = hW[NCOL]; h0C = hC[NCOL]; h0E = hE[NCOL];
    h1W = hW[2 * NCOL]; h1C = hC[2 * NCOL]; h1E = hE[2 * NCOL];
    hnW = h0W; hnC = h0C; hnE = h0E;
    hcW = h1W; hcC = h1C; hcE = h1E;
  }
#pragma unroll
  for (int k = 1; k <= K - 2; ++k) {
    const float sW = rW[(k + 2) * NCOL], sE = rE[(k + 2) * NCOL];
    const float sC = dv[k + 1];
    const float4 rc = rcs[k];
    const float cg = cgi * rc.z;
    if (FIRST) {
      const float hsW = hW[(k + 2) * NCOL], hsC = hC[(k + 2) * NCOL], hsE = hE[(k + 2) * NCOL];
      b[k] = rhs_point(ce, cw, rc.x, rc.y, cg, rdt, hnW, hnC, hnE, hcW, hcC, hcE, hsW, hsC, hsE);
      hnW = hcW; hnC = hcC; hnE = hcE;
      hcW = hsW; hcC = hsC; hcE = hsE;
    }
    const float v = jacobi_point(b[k], invd[k], ce, cw, rc.x, rc.y, cg, nW, nC, nE, cW, cE, sW, sC, sE);
    const float g = LAST ? next_guess_x<XM>(v, dO, k * NCOL) : v;
    wO[(k + 1) * NCOL] = g;
    nC = dv[k];
    dv[k] = g;
    nW = cW; nE = cE;
    cW = sW; cE = sE;
    if (LAST && (UNCOND || invd[k] != 0.f)) hO[(k + 1) * NCOL] = two_sum_update(hO[(k + 1) * NCOL], v, lo[k]);
  }
  if (clustered) cl_wait();
  {  // last strip row: north = old row K-2 (window), south = plane row p0+K
    constexpr int k = K - 1;
    const int p = p0 + k;
    const float sW = rW[(k + 2) * NCOL], sC = rC[(k + 2) * NCOL], sE = rE[(k + 2) * NCOL];
    const float4 rc = rcs[k];
    const float cg = cgi * rc.z;
    if (FIRST) {
      const float hsW = hW[(k + 2) * NCOL], hsC = hC[(k + 2) * NCOL], hsE = hE[(k + 2) * NCOL];
      b[k] = rhs_point(ce, cw, rc.x, rc.y, cg, rdt, hnW, hnC, hnE, hcW, hcC, hcE, hsW, hsC, hsE);
    }
    const float v = jacobi_point(b[k], invd[k], ce, cw, rc.x, rc.y, cg, nW, nC, nE, cW, cE, sW, sC, sE);
    const float g = LAST ? next_guess_x<XM>(v, dO, k * NCOL) : v;
    band_store<CFG>(wr, wr_push, p - 1, col, g);
    dv[k] = g;
    if (LAST && (UNCOND || invd[k] != 0.f))
      band_store<CFG>(hi, hi_push, p - 1, col, two_sum_update(hO[(k + 1) * NCOL], v, lo[k]));
  }
  {  // first strip row: north = plane row p0-1, south = old row 1
    const int p = p0;
    const float qW = rW[0], qC = rC[0], qE = rE[0];
    const float4 rc = rcs[0];
    const float cg = cgi * rc.z;
    if (FIRST) {
      const float hqW = hW[0], hqC = hC[0], hqE = hE[0];
      b[0] = rhs_point(ce, cw, rc.x, rc.y, cg, rdt, hqW, hqC, hqE, h0W, h0C, h0E, h1W, h1C, h1E);
    }
    const float v = jacobi_point(b[0], invd[0], ce, cw, rc.x, rc.y, cg, qW, qC, qE, r0W, r0E, r1W,
                                 dv1_old, r1E);
    const float g = LAST ? next_guess_x<XM>(v, dO, 0) : v;
    band_store<CFG>(wr, wr_push, p - 1, col, g);
    dv[0] = g;
    if (LAST && (UNCOND || invd[0] != 0.f))
      band_store<CFG>(hi, hi_push, p - 1, col, two_sum_update(hO[NCOL], v, lo[0]));
  }
}

// The commit of a step whose last sweep has already run as a FIRST sweep (its result is in
// dv[] and in the own rows of the plane wr): the compensated update of hi by v = dv[k] and
// the next step's initial guess into wr and dv[], with the band-edge rows mirrored into the
// neighbours -- what a LAST sweep does after its Jacobi update.  The caller separates it from
// that sweep by a block and cluster barrier: the sweep's right-hand side read hi around
// every node, here hi is written.
template <class CFG, class LoT>
__device__ __forceinline__ void fine_commit(float* __restrict__ wr, const HaloPush& wr_push, float* hi,
                                            const HaloPush& hi_push, float (&dv)[CFG::K],
                                            const float (&invd)[CFG::K], LoT& lo, int col, int r0, float* dp,
                                            bool extrap) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int p = r0 + 1 + k;
    const float v = dv[k];
    const float g = next_guess(v, dp, (r0 + k) * NCOL + col, extrap);
    band_store<CFG>(wr, wr_push, p - 1, col, g);
    dv[k] = g;
    if (invd[k] != 0.f) band_store<CFG>(hi, hi_push, p - 1, col, two_sum_update(hi[p * NCOL + col], v, lo[k]));
  }
}

// The compensation words of a thread's strip rows in a shared-memory plane of own rows.
template <class CFG>
struct StripLo {
  float* p;   // the thread's entry of its first strip row
  __device__ __forceinline__ float& operator[](int k) const { return p[k * CFG::NCOL]; }
};

template <class CFG>
__global__ void __launch_bounds__(CFG::NT, 1) fine_band_kernel(const __grid_constant__ FineBatch fb) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K, BH = CFG::BH, PLANE = CFG::PLANE;
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
  float* dA = hi + PLANE;
  float* dB = dA + PLANE;
  float* DP = dB + PLANE;   // d_{m-1}, own rows [BH*NCOL]
  float4* rowc = reinterpret_cast<float4*>(DP + BH * NCOL);

  band_load<CFG>(hi, d.in, M, jbase, tid);
  for (int e = tid; e < PLANE; e += CFG::NT) {
    dA[e] = 0.f;
    dB[e] = 0.f;
  }
  for (int r = tid; r < BH; r += CFG::NT) {
    float cs, cn, gj;
    row_coefs(d, jbase + r, cs, cn, gj);
    rowc[r] = make_float4(cs, cn, gj, 0.f);   // gj = (float)j exactly
  }
  const HaloPush hi_push = halo_push<CFG>(cluster, hi, rank, C);
  const HaloPush pA = halo_push<CFG>(cluster, dA, rank, C);
  const HaloPush pB = halo_push<CFG>(cluster, dB, rank, C);
  cluster_barrier(cluster, C);   // neighbours' loads done before far-field mirrors land
  if (fb.nsteps > 0) band_far_field<CFG>(hi, hi_push, pf, (float)(d.tau0 + d.dtau), h, M, jbase, tid);

  float ce = 0.f, cw = 0.f, cgi = 0.f;
  column_coefs(d, col, ce, cw, cgi);
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
  const float rdt = d.rdt;
  cluster_barrier(cluster, C);

  // Split cluster barrier: each sweep arrives after its writes and waits (inside the sweep)
  // only before the rows that read other CTAs' data; one arrive here opens the first phase.
  const bool clustered = C > 1;
  if (clustered) cl_arrive();
  int par = 0;
  // Sweeps per step: the first step starts cold (zero increment), the next ones up to step
  // xstart - 1 from the previous increment, every later one from the extrapolation
  // 2 d_{m-1} - d_{m-2}, which the last sweep of the step before leaves in the plane
  // (next_guess).
  for (int step = 0; step < fb.nsteps; ++step) {
    const int m = step_sweeps(d, step);
    for (int s = 0; s < m; ++s) {
      const float* rd = par ? dB : dA;
      float* wr = par ? dA : dB;
      const HaloPush& wp = par ? pA : pB;
      if (s == 0)
        fine_sweep<CFG, true, false>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col, il, ir, r0,
                                     ce, cw, cgi, rdt, clustered);
      else if (s == m - 1) {
        if (step + 1 >= d.xstart)
          fine_sweep<CFG, false, true, decltype(lo), 2>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col, il, ir,
                                                        r0, ce, cw, cgi, rdt, clustered, DP);
        else
          fine_sweep<CFG, false, true, decltype(lo), 1>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col, il, ir,
                                                        r0, ce, cw, cgi, rdt, clustered, DP);
      }
      else
        fine_sweep<CFG, false, false>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col, il, ir,
                                      r0, ce, cw, cgi, rdt, clustered);
      // After the first sweep has read hi (every CTA has: the second sweep waited on the
      // cluster barrier), move the far-field data to the next step; the last sweep -- this
      // one when a step has two sweeps -- writes only PDE nodes.
      if (s == 1 && step + 1 < fb.nsteps)
        band_far_field<CFG>(hi, hi_push, pf, (float)(d.tau0 + (step + 2) * d.dtau), h, M, jbase, tid);
      par ^= 1;
      if (clustered) cl_arrive();
      __syncthreads();
    }
  }
  if (clustered) cl_wait();   // no CTA leaves while a neighbour may still store into it

  if (col < M) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = jbase + r0 + k;
      if (j < M) d.out[(size_t)j * M + col] = hi[(r0 + k + 1) * NCOL + col] + lo[k];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Cluster tiles for grids that do not fit one cluster (M > 256), temporally blocked: one launch
// runs several whole implicit steps on a region (or, when a step's sweeps exceed the halo, a
// part of that step's sweeps).  A cluster of C CTAs owns a region of 256 columns x 32C rows
// (CTA `rank` holds rows 32 rank .. 32 rank + 31 in the band layout of band.cuh, so the rows
// between its CTAs are exchanged over DSMEM every sweep like the band stepper's).  Only the
// region's outer edges are cut: they hold values that are not updated, and every sweep's
// result is exact one node further from them -- the first sweep of a step forms b from hi one
// node further in, the last one applies the increment where it is exact, so the state stays
// exact as far in as the increment.  After a launch's H sweeps in all (over all its steps) an
// interior of I x I nodes at offset (H, H) matches a whole-grid solve bit for bit (the domain
// edges need no halo: zero coefficients at x = 0, y = 0, Dirichlet at the far edges).  The
// grid is covered by ntx^2 such interiors.  (hi, lo, increment, previous increment) of every
// node go to the other half of a ping-pong workspace between launches, so HBM carries
// 32 bytes per node per launch and 32 / s per node-step for s steps per launch; the
// increment slot holds the next step's initial guess (extrapolated from the third step on,
// as in the band stepper).  Where M is a multiple of 4 the region origin is too, and the
// region arrives as 16-byte asynchronous copies; otherwise as 4-byte ones.
// ---------------------------------------------------------------------------------------
// Two region layouts.  A: 256 columns x 256 rows (8 CTAs of 32 rows; 512 threads of one column
// x 16 rows), at most 24 sweeps per launch, so interiors keep >= 208 nodes.  B: 288 x 288 (9
// CTAs of 32 rows, a non-portable cluster size; 576 threads of one column x 16 rows), at most
// 16 sweeps per launch, interiors of 256: 1024 x 1024 takes 4 x 4 regions instead of A's 5 x 5
// (19% fewer nodes computed), 512 x 512 2 x 2 instead of 3 x 3.  The launch picks the layout
// with less work in waves of co-resident clusters (tile_layout).  Both keep 16-row strips; A in 128 registers per
// thread, B in 96 (a CTA of 576 threads is allocated registers for 20 warps).
typedef BandCfg<256, 512, 16> CTileCfgA;
typedef BandCfg<288, 576, 16> CTileCfgB;
constexpr int kCTileMaxHalo = 24;    // layout A: sweeps per launch (a multiple of 4)
constexpr int kCTileMaxHaloB = 16;   // layout B

struct CTileBatch {
  ItemDesc it[kMaxItems];
  float* ws;        // per item: [2][hi, lo, increment, previous increment][M*M]
  int n, M, H, I, ntx, C;
  float h;
};

// Asynchronous 16-byte global -> shared copy (L2 only); ok == false zero-fills.
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0)
               : "memory");
}

// Far-field data of the launch's steps.  A launch evaluates g(x, y, tau) once per step for the
// far-edge nodes it holds -- the column i = M - 1 on this CTA's plane rows and the row
// j = M - 1 on the region's columns -- into a shared-memory table, at one place in the code
// (an inlined far_field may contract its products into fused multiply-adds differently at
// different call sites, which would make a result depend on the launch plan); the steps copy
// their values from it.  The work is spread over the CTA's threads.
constexpr int kCTileMaxSteps = kCTileMaxHalo / 2;   // steps have at least two sweeps
template <class CFG>
struct FarTable {
  static constexpr int W = (CFG::BH + 2) + CFG::NCOL;   // far column rows, then far row columns
  static constexpr int FLOATS = kCTileMaxSteps * W;
};

template <class CFG>
__device__ __forceinline__ void far_table_fill(float* ff, const PayoffF& pf, const ItemDesc& d, int step0,
                                               int nstep, float h, int M, int ix0, int jb, int tid) {
  constexpr int W = FarTable<CFG>::W, PR = CFG::BH + 2;
  const int cfar = M - 1 - ix0;          // region column of i = M - 1
  const int pfar = M - jb;               // plane row of j = M - 1
  const bool has_col = cfar >= 0 && cfar < CFG::NCOL, has_row = pfar >= 0 && pfar < PR;
  if (!has_col && !has_row) return;
  for (int e = tid; e < nstep * W; e += CFG::NT) {
    const int t = e / W, q = e - t * W;
    const float tau = (float)(d.tau0 + (step0 + t + 1) * d.dtau);
    int i, j;
    if (q < PR) {
      if (!has_col) continue;
      i = M - 1;
      j = jb + q - 1;
    } else {
      if (!has_row) continue;
      i = ix0 + (q - PR);
      j = M - 1;
    }
    if (i >= 0 && i < M && j >= 0 && j < M) ff[e] = far_field(pf, (float)i * h, (float)j * h, tau);
  }
}

// Step t's far-field data on this thread's own region rows, mirrored into the neighbours'
// halo rows by band_store.  The region's cut halo rows are left as they are (they are beyond
// the exact part).
template <class CFG>
__device__ __forceinline__ void ctile_far_field(float* hi, const HaloPush& hp, const float* ff, int t, int M,
                                                int ig, int jrow0, int r0, int col) {
  constexpr int W = FarTable<CFG>::W, PR = CFG::BH + 2;
  const float* row = ff + t * W;
  if (ig == M - 1) {
#pragma unroll
    for (int k = 0; k < CFG::K; ++k) {
      const int j = jrow0 + k;
      if (j >= 0 && j < M) band_store<CFG>(hi, hp, r0 + k, col, row[r0 + k + 1]);
    }
  } else if (ig >= 0 && ig < M - 1) {
    const int k = M - 1 - jrow0;
    if (k >= 0 && k < CFG::K) band_store<CFG>(hi, hp, r0 + k, col, row[PR + col]);
  }
}

// Launch of steps [step0, step0 + nstep) of every item; with nstep == 1 only the sweeps
// [s_begin, s_end) of that step (the step is applied if it ends in this launch).  `first`:
// the state comes from the items' inputs (no increments yet); `last`: the result goes to the
// items' outputs instead of the workspace.
template <class CFG, int VEC>
__global__ void __launch_bounds__(CFG::NT, 1) fine_ctile_kernel(const __grid_constant__ CTileBatch tb,
                                                                int step0, int nstep, int first, int last,
                                                                int par, int s_begin, int s_end) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K, BH = CFG::BH, PLANE = CFG::PLANE;
  static_assert(VEC == 1 || VEC == 4, "4-byte or 16-byte copies");
  cg::cluster_group cluster = cg::this_cluster();
  const int C = tb.C;
  const int rank = (int)cluster.block_rank();
  const ItemDesc& d = tb.it[blockIdx.z];
  const int M = tb.M, H = tb.H, I = tb.I;
  const size_t MM = (size_t)M * M;
  const int tx = (int)blockIdx.y % tb.ntx, ty = (int)blockIdx.y / tb.ntx;
  const int ix0 = tx * I - H, jy0 = ty * I - H;   // region origin (multiples of VEC)
  const int jb = jy0 + rank * BH;                 // row of this CTA's first own row
  float* ws = tb.ws + (size_t)blockIdx.z * 8 * MM;
  const float* hi_g = first ? d.in : ws + (size_t)(par * 4 + 0) * MM;
  const float* lo_g = ws + (size_t)(par * 4 + 1) * MM;
  const float* dv_g = ws + (size_t)(par * 4 + 2) * MM;
  const float* dp_g = ws + (size_t)(par * 4 + 3) * MM;
  float* hi_o = ws + (size_t)((par ^ 1) * 4 + 0) * MM;
  float* lo_o = ws + (size_t)((par ^ 1) * 4 + 1) * MM;
  float* dv_o = ws + (size_t)((par ^ 1) * 4 + 2) * MM;
  float* dp_o = ws + (size_t)((par ^ 1) * 4 + 3) * MM;
  const int tid = threadIdx.x;
  const int col = tid % NCOL, grp = tid / NCOL;
  const int r0 = grp * K;
  const PayoffF pf = make_payoff(d);

  extern __shared__ __align__(16) float smem[];
  float* hi = smem;
  float* dA = hi + PLANE;
  float* dB = dA + PLANE;
  float* DP = dB + PLANE;   // previous increment, own rows [BH*NCOL]
  float* LO = DP + BH * NCOL;   // compensation words, own rows [BH*NCOL]
  float* FF = LO + BH * NCOL;   // far-field table [kCTileMaxSteps][FarTable::W]
  float4* rowc = reinterpret_cast<float4*>(FF + FarTable<CFG>::FLOATS);
  // Own rows and both halo rows of hi and of the increment (the halo rows between CTAs are
  // the neighbours' own rows and are kept current by DSMEM pushes during the sweeps), and
  // the own rows of the previous increment and of lo: asynchronous copies, all in flight at
  // once, zero-filled outside the domain (with VEC = 4 a chunk lies wholly inside or outside:
  // M and the region origin are multiples of 4).
  // The second increment plane needs only its halo rows: the launch's first sweep reads the
  // first plane and writes every own row of the second before anything reads it.
  for (int e = tid * VEC; e < PLANE; e += CFG::NT * VEC) {
    const int pr = e / NCOL, c = e % NCOL;
    const int j = jb + pr - 1, i = ix0 + c;
    const bool in = (i >= 0 && i < M && j >= 0 && j < M);
    const size_t gi = in ? (size_t)j * M + i : 0;
    const bool halo = pr == 0 || pr == BH + 1;
    if constexpr (VEC == 4) {
      cp_async16(hi + e, hi_g + gi, in);
      cp_async16(dA + e, dv_g + gi, in && !first);
      if (halo) cp_async16(dB + e, dv_g + gi, in && !first);
    } else {
      cp_async4(hi + e, hi_g + gi, in);
      cp_async4(dA + e, dv_g + gi, in && !first);
      if (halo) cp_async4(dB + e, dv_g + gi, in && !first);
    }
  }
  for (int e = tid * VEC; e < BH * NCOL; e += CFG::NT * VEC) {
    const int r = e / NCOL, c = e % NCOL;
    const int j = jb + r, i = ix0 + c;
    const bool in = (i >= 0 && i < M && j >= 0 && j < M);
    const size_t gi = in ? (size_t)j * M + i : 0;
    if constexpr (VEC == 4) {
      cp_async16(DP + e, dp_g + gi, in && !first);
      cp_async16(LO + e, lo_g + gi, in && !first);
    } else {
      cp_async4(DP + e, dp_g + gi, in && !first);
      cp_async4(LO + e, lo_g + gi, in && !first);
    }
  }
  for (int r = tid; r < BH; r += CFG::NT) {
    float cs, cn, gj;
    row_coefs(d, jb + r, cs, cn, gj);
    rowc[r] = make_float4(cs, cn, gj, 0.f);   // gj = (float)j exactly
  }
  far_table_fill<CFG>(FF, pf, d, step0, nstep, tb.h, M, ix0, jb, tid);
  const int ig = ix0 + col;
  float ce = 0.f, cw = 0.f, cgi = 0.f;
  column_coefs(d, ig, ce, cw, cgi);
  cp_async_wait_all();
  __syncthreads();
  // the far-field data of the first step on every plane row this thread covers (own rows and,
  // for the edge groups, the halo row next to them), locally: the neighbours' halo rows are
  // still being loaded
  {
    const int pa = grp == 0 ? 0 : r0 + 1, pb = grp == CFG::G - 1 ? BH + 1 : r0 + K;
    if (ig == M - 1) {
      for (int pr = pa; pr <= pb; ++pr) {
        const int j = jb + pr - 1;
        if (j >= 0 && j < M) hi[pr * NCOL + col] = FF[pr];
      }
    } else if (ig >= 0 && ig < M - 1) {
      const int pr = M - jb;   // plane row of j = M - 1
      if (pr >= pa && pr <= pb) hi[pr * NCOL + col] = FF[(BH + 2) + col];
    }
  }
  float dv[K], b[K], invd[K];
  StripLo<CFG> lo{LO + r0 * NCOL + col};   // compensation words stay in shared memory
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = jb + r0 + k;
    const bool pde = ig >= 0 && ig < M - 1 && j >= 0 && j < M - 1;
    invd[k] = pde ? inv_diag(d, ig, j) : 0.f;
    if (!pde) lo[k] = 0.f;
    b[k] = 0.f;
    dv[k] = dA[(r0 + k + 1) * NCOL + col];
  }
  const int il = col > 0 ? col - 1 : 0;
  const int ir = col + 1 < NCOL ? col + 1 : col;
  const float rdt = d.rdt;
  const HaloPush hi_push = halo_push<CFG>(cluster, hi, rank, C);
  const HaloPush pA = halo_push<CFG>(cluster, dA, rank, C);
  const HaloPush pB = halo_push<CFG>(cluster, dB, rank, C);
  cluster_barrier(cluster, C);   // every CTA's loads are done before the first push lands

  cl_arrive();
  int p = 0;
  for (int t = 0; t < nstep; ++t) {
    const int step = step0 + t;
    const int m_item = step_sweeps(d, step);
    const int sa = nstep == 1 ? s_begin : 0;
    const int sb = nstep == 1 ? min(s_end, m_item) : m_item;
    const int nsw = max(0, sb - sa);
    const bool commit = nsw > 0 && sb == m_item;
    const bool extrap = step + 1 >= d.xstart;
    for (int s = 0; s < nsw; ++s) {
      const float* rd = p ? dB : dA;
      float* wr = p ? dA : dB;
      const HaloPush& wp = p ? pA : pB;
      const bool fst = s == 0, lst = commit && s == nsw - 1;
      if (fst && lst) {
        // A one-sweep piece that commits its step (an item whose step ends one sweep into a
        // launch of a split step): the sweep forms b from hi, so hi is updated only after
        // every thread of the cluster has passed it.
        fine_sweep<CFG, true, false>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col, il, ir, r0, ce, cw,
                                     cgi, rdt, true);
        cl_arrive();
        __syncthreads();
        cl_wait();
        fine_commit<CFG>(wr, wp, hi, hi_push, dv, invd, lo, col, r0, DP, extrap);
      } else if (fst)
        fine_sweep<CFG, true, false>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col, il, ir, r0, ce, cw,
                                     cgi, rdt, true);
      else if (lst) {
        // unconditional commit: the far-field data are set by the owning thread after the sweep
        if (extrap)
          fine_sweep<CFG, false, true, decltype(lo), 2, true>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col,
                                                              il, ir, r0, ce, cw, cgi, rdt, true, DP);
        else
          fine_sweep<CFG, false, true, decltype(lo), 1, true>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col,
                                                              il, ir, r0, ce, cw, cgi, rdt, true, DP);
      }
      else
        fine_sweep<CFG, false, false>(rd, wr, hi, wp, hi_push, rowc, dv, b, invd, lo, col, il, ir, r0, ce, cw,
                                      cgi, rdt, true);
      // After the second sweep of a step every CTA has passed the first one, which read hi:
      // move the far-field data on to the next step of this launch (the last sweep writes
      // only PDE nodes, so this may follow it directly).
      if (s == 1 && t + 1 < nstep) ctile_far_field<CFG>(hi, hi_push, FF, t + 1, M, ig, jb + r0, r0, col);
      p ^= 1;
      cl_arrive();
      __syncthreads();
    }
  }
  cl_wait();   // no CTA leaves while a neighbour may still store into it

  // the interior of the region
  if (col >= H && col < H + I && ig < M) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int rr = rank * BH + r0 + k, j = jb + r0 + k;
      if (rr >= H && rr < H + I && j < M) {
        const size_t gi = (size_t)j * M + ig;
        const float hv = hi[(r0 + k + 1) * NCOL + col];
        if (last) {
          d.out[gi] = hv + lo[k];
        } else {
          hi_o[gi] = hv;
          lo_o[gi] = lo[k];
          dv_o[gi] = dv[k];
          dp_o[gi] = DP[(r0 + k) * NCOL + col];
        }
      }
    }
  }
}

// u_out = hi + lo from the second workspace half (after a single launch)
__global__ void ctile_finish_kernel(const __grid_constant__ CTileBatch tb) {
  const ItemDesc& d = tb.it[blockIdx.y];
  const size_t MM = (size_t)tb.M * tb.M;
  const float* ws = tb.ws + (size_t)blockIdx.y * 8 * MM;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < MM) d.out[e] = ws[4 * MM + e] + ws[5 * MM + e];
}

// The largest sweep count of any item in step `step`.
static int max_step_sweeps(const ItemDesc* items, int n, int step) {
  int m = 1;
  for (int k = 0; k < n; ++k) m = std::max(m, step_sweeps(items[k], step));
  return m;
}

// One launch of the tile stepper: steps [step0, step0 + nstep), or sweeps [s0, s1) of step0
// (nstep == 1), with H sweeps in all (the halo).
struct CTileLaunch {
  int step0, nstep, s0, s1, H;
};

// Launch plan: whole steps are packed into a launch while their sweeps (the largest count of
// any item, step by step) add up to at most kCTileMaxHalo; a step with more sweeps than that is
// split evenly over several launches.
static void ctile_plan(const ItemDesc* items, int n, int nsteps, int hmax, std::vector<CTileLaunch>& plan) {
  plan.clear();
  int step = 0;
  while (step < nsteps) {
    const int m = max_step_sweeps(items, n, step);
    if (m > hmax) {
      const int nl = (m + hmax - 1) / hmax;
      const int chunk = (m + nl - 1) / nl;
      for (int l = 0; l < nl; ++l) {
        const int s0 = l * chunk, s1 = std::min(m, s0 + chunk);
        plan.push_back({step, 1, s0, s1, s1 - s0});
      }
      ++step;
      continue;
    }
    int h = m, k = 1;
    while (step + k < nsteps) {
      const int mk = max_step_sweeps(items, n, step + k);
      if (h + mk > hmax) break;
      h += mk;
      ++k;
    }
    plan.push_back({step, k, 0, 1 << 30, h});
    step += k;
  }
}

// Region geometry of a launch with h sweeps: halo H (a multiple of 4 with 16-byte copies), ntx
// interiors of I nodes per axis, clusters of C CTAs.
template <class CFG>
static void ctile_geometry(int M, int h, bool vec, CTileBatch& tb) {
  const int NC = CFG::NCOL;
  const int H = vec ? ((std::max(2, h) + 3) / 4) * 4 : std::max(2, h);
  int ntx = (M + (NC - 2 * H) - 1) / (NC - 2 * H);
  int I;
  for (;; ++ntx) {
    I = (M + ntx - 1) / ntx;
    if (vec) I = ((I + 3) / 4) * 4;
    if (I + 2 * H <= NC) break;
  }
  tb.H = H;
  tb.I = I;
  tb.ntx = ntx;
  tb.C = (I + 2 * H + CFG::BH - 1) / CFG::BH;
}

template <class CFG>
static size_t ctile_smem() {
  return (size_t)3 * CFG::PLANE * sizeof(float) + (size_t)2 * CFG::BH * CFG::NCOL * sizeof(float) +
         (size_t)FarTable<CFG>::FLOATS * sizeof(float) + (size_t)CFG::BH * sizeof(float4);
}

// Clusters of C CTAs of a layout that the current device runs at once (0 if unknown),
// measured once per device, layout and C through the occupancy API.
template <class CFG>
static int tile_capacity(int C) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, C});
  if (it != cache.end()) return it->second;
  const size_t smem = ctile_smem<CFG>();
  auto kern = fine_ctile_kernel<CFG, 4>;
  int n = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(CFG::NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) ||
      cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache[{dev, C}] = n;
  return n;
}

// The region layout of a launch batch of nb states (1 = A, 2 = B; BS_OPT_FINE_TILE forces
// one): the one with less work per launch, counted as waves of clusters (states x regions
// over the clusters the device holds at once) times the nodes of a region, B's nodes weighted
// by kTileCostB; with an unknown capacity, the nodes of all regions.  A on a tie.  Both give
// the same result bit for bit.  At 1024 x 1024 the device holds 15 clusters of 8 or of 9
// CTAs: one state (25 A regions or 16 B regions, two waves either way) goes to A, eight or
// more to B.
constexpr double kTileCostB = 1.12;   // B's time per node over A's (more launches, 96 registers),
                                      // from 64 states x 64 steps at 1024^2
static int tile_layout(int M, int nb) {
  if (g_opt.fine_tile == 1 || g_opt.fine_tile == 2) return g_opt.fine_tile;
  CTileBatch ta, tb;
  ctile_geometry<CTileCfgA>(M, kCTileMaxHalo, M % 4 == 0, ta);
  ctile_geometry<CTileCfgB>(M, kCTileMaxHaloB, M % 4 == 0, tb);
  const double ra = (double)CTileCfgA::NCOL * (ta.C * CTileCfgA::BH);   // nodes of a region
  const double rb = (double)CTileCfgB::NCOL * (tb.C * CTileCfgB::BH);
  const double ca = (double)nb * ta.ntx * ta.ntx, cb = (double)nb * tb.ntx * tb.ntx;   // clusters
  const int capa = tile_capacity<CTileCfgA>(ta.C), capb = tile_capacity<CTileCfgB>(tb.C);
  double wa = ca * ra, wb = cb * rb;
  if (capa > 0 && capb > 0) {
    wa = std::ceil(ca / capa) * ra;
    wb = std::ceil(cb / capb) * rb;
  }
  wb *= kTileCostB;
  return wb < wa ? 2 : 1;
}

template <class CFG>
static int launch_ctiles(const bs_grid* g, const ItemDesc* items, int n, int nsteps, int hmax, cudaStream_t s) {
  const int M = g->M;
  const size_t MM = (size_t)M * M;
  int rc = ensure(const_cast<bs_grid*>(g)->ws_fine, (size_t)std::min(n, kMaxItems) * 8 * MM * sizeof(float));
  if (rc) return rc;
  const size_t smem = ctile_smem<CFG>();
  // 16-byte copies need M and every input state 16-byte aligned (the workspace is)
  bool vec = M % 4 == 0;
  for (int k = 0; k < n; ++k) vec = vec && ((uintptr_t)items[k].in % 16 == 0);
  auto kern = vec ? fine_ctile_kernel<CFG, 4> : fine_ctile_kernel<CFG, 1>;
  BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (CFG::NCOL / CFG::BH > 8) BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  std::vector<CTileLaunch> plan;
  for (int base = 0; base < n; base += kMaxItems) {
    CTileBatch tb;
    tb.n = std::min(n - base, kMaxItems);
    for (int k = 0; k < tb.n; ++k) tb.it[k] = items[base + k];
    tb.ws = (float*)g->ws_fine.ptr;
    tb.M = M;
    tb.h = (float)(g->xmax / (M - 1));
    ctile_plan(tb.it, tb.n, nsteps, hmax, plan);
    int par = 0;
    const int nl = (int)plan.size();
    for (int l = 0; l < nl; ++l) {
      const CTileLaunch& L = plan[(size_t)l];
      ctile_geometry<CFG>(M, L.H, vec, tb);
      const bool first = l == 0, final_launch = l == nl - 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(tb.C, tb.ntx * tb.ntx, tb.n);
      cfg.blockDim = dim3(CFG::NT, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = tb.C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      // A launch that reads u_in must not write u_out (they may alias): a single launch keeps
      // its result in the workspace and u_out is formed in a separate pass.
      BS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, tb, L.step0, L.nstep, (int)first, (int)(final_launch && !first),
                                     par, L.s0, L.s1));
      par ^= 1;
    }
    if (nl == 1) {
      ctile_finish_kernel<<<dim3((unsigned)((MM + 255) / 256), tb.n), 256, 0, s>>>(tb);
      BS_CUDA_TRY(cudaGetLastError());
    }
  }
  return BS_OK;
}

static int launch_ctiles(const bs_grid* g, const ItemDesc* items, int n, int nsteps, cudaStream_t s) {
  return tile_layout(g->M, std::min(n, kMaxItems)) == 2
             ? launch_ctiles<CTileCfgB>(g, items, n, nsteps, kCTileMaxHaloB, s)
             : launch_ctiles<CTileCfgA>(g, items, n, nsteps, kCTileMaxHalo, s);
}

int fine_launches(const bs_grid* g, const ItemDesc* items, int n, int nsteps) {
  const int chunks = (n + kMaxItems - 1) / kMaxItems;
  if (g->shape.C >= 1 && g->shape.C <= kMaxCluster) return chunks;
  if (nsteps < 1) return 0;
  const int hmax = tile_layout(g->M, std::min(n, kMaxItems)) == 2 ? kCTileMaxHaloB : kCTileMaxHalo;
  int total = 0;
  std::vector<CTileLaunch> plan;
  for (int base = 0; base < n; base += kMaxItems) {
    const int nb = std::min(n - base, kMaxItems);
    ctile_plan(items + base, nb, nsteps, hmax, plan);
    total += (int)plan.size() + (plan.size() == 1 ? 1 : 0);
  }
  return total;
}

// Band layouts of the 129..256-column grids.  The default: 8 CTAs of 32 rows (512 threads, one
// column x 16 rows each).  For one or a few states: 16 CTAs of 16 rows (256 threads), each on
// an SM of its own (its shared memory is padded so that no second CTA shares the SM), so that
// a state's steps run on twice the SMs at half the warps per SM -- 2.03 against 3.06 ms for
// 512 steps of one 256 x 256 state, but more waves for a large batch.  Every node is computed
// with the same operations from its global indices in both, so results agree bit for bit.
typedef BandCfg<256, 512, 16> Band256;
typedef BandCfg<256, 256, 16> Band256x16;
constexpr size_t kBandSpreadSmem = 120 * 1024;   // above half an SM's shared memory
constexpr double kBand16Time = 0.66;             // Band256x16's time per state over Band256's

template <class CFG>
static size_t band_smem(bool spread) {
  const size_t b = (size_t)3 * CFG::PLANE * sizeof(float) + (size_t)CFG::BH * CFG::NCOL * sizeof(float) +
                   (size_t)CFG::BH * sizeof(float4);
  return spread ? std::max(b, kBandSpreadSmem) : b;
}

template <class CFG>
static int launch_band(const FineBatch& fb, cudaStream_t s, bool spread = false) {
  const size_t smem = band_smem<CFG>(spread);
  auto kern = fine_band_kernel<CFG>;
  BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (fb.sh.C > 8) BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(fb.sh.C, fb.n, 1);
  cfg.blockDim = dim3(CFG::NT, 1, 1);
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

// Clusters of the fine band kernel that the device runs at once (0 if unknown), measured once
// per device, layout and cluster size.
template <class CFG>
static int band_capacity(const BandShape& sh, bool spread = false) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  const int key = sh.C * 2 + (spread ? 1 : 0);
  auto it = cache.find({dev, key});
  if (it != cache.end()) return it->second;
  const size_t smem = band_smem<CFG>(spread);
  auto kern = fine_band_kernel<CFG>;
  int n = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sh.C, 1, 1);
  cfg.blockDim = dim3(CFG::NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (sh.C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) ||
      cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache[{dev, key}] = n;
  return n;
}

static BandShape band16_shape(const BandShape& sh) {
  BandShape s16 = sh;
  s16.G = 1;
  s16.BH = 16;
  s16.C = (sh.M + 15) / 16;
  return s16;
}

// Whether a launch of n states on a 256-column band grid takes the 16-CTA layout: fewer
// waves times time per state (BS_OPT_FINE_TILE 1 or 2 forces the 8- or the 16-CTA layout).
static bool use_band16(const BandShape& sh, int n) {
  if (sh.ncol != 256) return false;
  if (g_opt.fine_tile == 1 || g_opt.fine_tile == 2) return g_opt.fine_tile == 2;
  const int cap8 = band_capacity<Band256>(sh), cap16 = band_capacity<Band256x16>(band16_shape(sh), true);
  if (cap8 <= 0 || cap16 <= 0) return false;
  const double t8 = std::ceil((double)n / cap8), t16 = std::ceil((double)n / cap16) * kBand16Time;
  return t16 < t8;
}

int fine_cluster_capacity(const bs_grid* g) {
  const BandShape sh = g->shape;
  if (sh.C < 1 || sh.C > kMaxCluster) return 0;
  switch (sh.ncol) {
    case 32: return band_capacity<BandCfg<32, 256, 4>>(sh);
    case 64: return band_capacity<BandCfg<64, 512, 8>>(sh);
    case 128: return band_capacity<BandCfg<128, 512, 16>>(sh);
    case 256: return band_capacity<Band256>(sh);
  }
  return 0;
}

int launch_fine(const bs_grid* g, const ItemDesc* items, int n, int nsteps, cudaStream_t s) {
  const BandShape sh = g->shape;
  if (sh.C < 1 || sh.C > kMaxCluster) return launch_ctiles(g, items, n, nsteps, s);
  const bool b16 = use_band16(sh, std::min(n, kMaxItems));
  for (int base = 0; base < n; base += kMaxItems) {
    FineBatch fb;
    fb.n = (n - base) < kMaxItems ? (n - base) : kMaxItems;
    for (int k = 0; k < fb.n; ++k) fb.it[k] = items[base + k];
    fb.nsteps = nsteps;
    fb.sh = b16 ? band16_shape(sh) : sh;
    fb.h = (float)(g->xmax / (g->M - 1));
    int rc;
    switch (sh.ncol) {
      case 32: rc = launch_band<BandCfg<32, 256, 4>>(fb, s); break;
      case 64: rc = launch_band<BandCfg<64, 512, 8>>(fb, s); break;
      case 128: rc = launch_band<BandCfg<128, 512, 16>>(fb, s); break;
      case 256: rc = b16 ? launch_band<Band256x16>(fb, s, true) : launch_band<Band256>(fb, s); break;
      default: rc = set_error(BS_ERR_ARG, "fine_propagate_batched: no band shape for M=%d", g->M);
    }
    if (rc != BS_OK) return rc;
  }
  return BS_OK;
}

}  // namespace bsp
