// K2 + K5: numerical coarse propagator G and the serial Parareal sweep.
//
// G (Sec. 3.1, Sec. 3.2: the same discretisation as F with a larger step) takes csteps
// implicit-Euler steps per slice.  With the larger step the system is not diagonally
// dominant, so each step is solved by BiCGSTAB (van der Vorst 1992) on the Jacobi-scaled
// system  D^{-1}(I - dtau R_h) d = D^{-1} dtau R_h w  in FP32 (the paper runs its coarse
// models in single precision, Sec. 4.1).  One thread-block cluster holds the whole state and
// the two matrix-vector operands in shared memory (band layout of band.cuh).
//
// Reductions: per-thread partial sums, a warp butterfly, then one warp per CTA adds the warp
// partials of all CTAs in a fixed order -- in FP32 for the Krylov dot products, in FP64 for
// the Parareal defect norms.  A butterfly adds the same two operands on both lanes of every
// pair, so all lanes -- and all CTAs, which read the same partials in the same order -- get
// bitwise the same total.  The BiCGSTAB scalars (alpha, omega, beta) are computed once per
// CTA by that warp and broadcast through shared memory.  FP64 is kept off the iteration: at
// this GPU's FP64 rate, FP64 butterflies and divisions on one warp cost more than the rest of
// an iteration.
//
// The serial Parareal sweep of eq. (parareal) runs in the same kernel: for n = n_first..N-1
//   G_new = G(u_n^{k+1});  u_{n+1}^{k+1} = F_n + (G_new - G_old_n);  G_old_n = G_new,
// with FP64 sums of ||u_{n+1}^{k+1} - u_{n+1}^k||^2 and ||u_{n+1}^{k+1}||^2 per slice and, at
// the end, delta_k = max_n ||du_n|| / max_n ||u_n|| (reading c5).  The correction is
// evaluated as F + (G_new - G_old) so that an unchanged slice gives a zero bracket exactly.
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>

#include "band.cuh"

namespace bsp {

constexpr int kKrylovAttempts = 3;   // BiCGSTAB starts per implicit step (restarts on breakdown)

constexpr int kMaxBandRows = 256;   // rows of the largest band-variant grid, padding included

struct SweepParams {
  ItemDesc d;       // dtau = coarse step
  SweepArgs a;
  BandShape sh;
  float h;
  // Row coefficients {cs, cn, (float)j, 0} of every band row, in the launch's constant
  // parameter space: the rows of a strip are the same for a whole warp (for a whole CTA in
  // one-group variants), so the stencil reads them as uniform constant loads rather than
  // shared-memory loads.  Owner and neighbour read the same values (halo rows included).
  float4 rowc[kMaxBandRows];
};

// BiCGSTAB scalar state shared by a CTA (identical in every CTA of the cluster).  The
// Krylov dot products and scalars are FP32 like the vectors; only the Parareal norms are
// FP64 (tot), since FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU
// and sits on the serial path of every iteration.
struct Scal {
  double tot[4];    // FP64 totals of the last cluster_sum<double>
  float totf[4];    // FP32 totals of the last cluster_sum<float>
  float rho, alpha, omega, stop2;
  float af, of, bf;
  int conv, fail;
};

__device__ __forceinline__ double* scal_tot(Scal* s, double) { return s->tot; }
__device__ __forceinline__ float* scal_tot(Scal* s, float) { return s->totf; }

// Jacobi-scaled operator at one node:
//   (A^ y)_C = y_C - invd * (ce y_E + cw y_W + cs y_S + cn y_N + cg ((y_SE - y_NE) - (y_SW - y_NW)))
// (N = row j-1, S = row j+1), with every rounding explicit, so that a halo row evaluated by a
// neighbour equals bit for bit the same row evaluated by its owner.
__device__ __forceinline__ float scaled_node(float nW, float nC, float nE, float cW, float cC, float cE, float sW,
                                             float sC, float sE, float4 rc, float id, float ce, float cw,
                                             float cgi) {
  const float cg = cgi * rc.z;
  float acc = ce * cE;
  acc = fmaf(cw, cW, acc);
  acc = fmaf(rc.x, sC, acc);
  acc = fmaf(rc.y, nC, acc);
  acc = fmaf(cg, (sE - nE) - (sW - nW), acc);
  return fmaf(-id, acc, cC);
}

// A^ y at one row; yrow points at the row's first column, the rows above and below are
// yrow -+ ncol.
__device__ __forceinline__ float scaled_row(const float* yrow, int ncol, int col, int il, int ir, float4 rc,
                                            float id, float ce, float cw, float cgi) {
  const float* n = yrow - ncol;
  const float* s = yrow + ncol;
  return scaled_node(n[il], n[col], n[ir], yrow[il], yrow[col], yrow[ir], s[il], s[col], s[ir], rc, id, ce, cw,
                     cgi);
}

// scaled_matvec with the strip's own values y_C taken from registers (c[k] equals the plane's
// own row r0 + k): the vertical neighbours inside the strip come from registers too, so each
// row loads only its west and east neighbours (and the strip's first and last rows one more).
template <class CFG>
__device__ __forceinline__ void scaled_matvec_rc(const float* __restrict__ y, const float (&c)[CFG::K],
                                                 const float4* __restrict__ rowc,
                                                 const float* __restrict__ ID, int col, int il, int ir, int r0,
                                                 float ce, float cw, float cgi, float (&out)[CFG::K]) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K;
  const int p0 = r0 + 1;
  float nW = y[(p0 - 1) * NCOL + il], nC = y[(p0 - 1) * NCOL + col], nE = y[(p0 - 1) * NCOL + ir];
  float cW = y[p0 * NCOL + il], cC = c[0], cE = y[p0 * NCOL + ir];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int p = p0 + k;
    const float sW = y[(p + 1) * NCOL + il], sE = y[(p + 1) * NCOL + ir];
    const float sC = k + 1 < K ? c[k + 1 < K ? k + 1 : k] : y[(p + 1) * NCOL + col];
    out[k] = scaled_node(nW, nC, nE, cW, cC, cE, sW, sC, sE, rowc[p - 1], ID[(p - 1) * NCOL + col], ce, cw, cgi);
    nW = cW; nC = cC; nE = cE;
    cW = sW; cC = sC; cE = sE;
  }
}

template <class T>
__device__ __forceinline__ T warp_butterfly(T x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Cluster-wide sum of NV per-thread values of type T.  Each warp reduces its values by a
// butterfly; warp 0 adds the warp partials (wpart) and lanes 0..C-1 store the CTA partial into
// slot `rank` of every CTA of the cluster; after one cluster barrier, thread 0 of every CTA
// adds the C partials in rank order, so every CTA gets bitwise the same totals in
// scal_tot(sc) (type T), and runs `fin(sc)` before the closing CTA barrier.  `round`
// alternates two slot arrays so that a fast CTA never overwrites partials that a slow CTA is
// still adding.  slots: double[2][kMaxCluster][4]; wpart: double[NW][4].
template <class CFG, int NV, class T, class Fin>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, const T (&v)[NV], double* slots,
                                            double* wpart, Scal* sc, int& round, int rank, int C,
                                            Fin fin) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* slot = reinterpret_cast<T*>(slots) + (round & 1) * (kMaxCluster * 4);
  T* wp = reinterpret_cast<T*>(wpart);
  T x[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) x[q] = warp_butterfly<T>(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) wp[warp * 4 + q] = x[q];
  }
  __syncthreads();
  if (warp == 0) {
    T c[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) c[q] = warp_butterfly<T>(lane < CFG::NW ? wp[lane * 4 + q] : T(0));
    if (lane < C) {
      T* dst = (C > 1 ? cl.map_shared_rank(slot, lane) : slot) + rank * 4;
#pragma unroll
      for (int q = 0; q < NV; ++q) dst[q] = c[q];
    }
  }
  if (C > 1) cl.sync(); else __syncthreads();
  if (threadIdx.x == 0) {
    T* out = scal_tot(sc, T(0));
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      T acc = T(0);
      for (int i = 0; i < C; ++i) acc += slot[i * 4 + q];
      out[q] = acc;
    }
    fin(sc);
  }
  __syncthreads();
  ++round;
}

// BiCGSTAB scalar updates shared by the band and global kernels (run by one thread per CTA).
struct KrylovFin {
  // start: totf = {(b^, b^), (r, r)}
  static __device__ __forceinline__ void start(Scal* s, float tol) {
    s->rho = s->totf[1];
    s->stop2 = tol * tol * s->totf[0];
    s->conv = s->totf[1] <= s->stop2 || !(s->totf[0] > 1e-30f);
    s->fail = 0;
    s->alpha = s->omega = 1.f;
  }
  // after v = A^ p: totf = {(r^, v), (r, r)}
  static __device__ __forceinline__ void alpha(Scal* s) {
    if (s->totf[1] <= s->stop2) { s->conv = 1; return; }
    if (s->totf[0] == 0.f) { s->fail = 1; return; }
    s->alpha = s->rho / s->totf[0];
    s->af = s->alpha;
  }
  // after t = A^ s: totf = {(t, s), (t, t), (r^, s), (r^, t)}
  static __device__ __forceinline__ void omega(Scal* s) {
    s->omega = s->totf[1] > 0.f ? s->totf[0] / s->totf[1] : 0.f;
    s->of = s->omega;
    const float rho_new = s->totf[2] - s->omega * s->totf[3];
    if (s->omega == 0.f || s->rho == 0.f) { s->fail = 1; s->bf = 0.f; return; }
    s->bf = (rho_new / s->rho) * (s->alpha / s->omega);
    s->rho = rho_new;
  }
};

// ---------------------------------------------------------------------------------------
// Point-to-point cluster exchange for the BiCGSTAB iterations.  A round moves every CTA's
// partial sums to every CTA of the cluster, plus (optionally) one halo row from each band
// neighbour, with st.async stores into the receivers' shared memory.  Each store completes
// its byte count on the receiver's mbarrier for that round's parity; a CTA waits on its own
// mbarrier until all expected bytes have landed.  No cluster-wide barrier and no fence are
// needed: the complete-tx of st.async releases the data and the mbarrier wait acquires it.
//
// Buffer reuse: rounds alternate two mbarriers and two partial-slot arrays.  A CTA sends
// round r+2 data only after round r+1 has completed for it, which needs this CTA's round r+1
// partial, which this CTA sends only after it has finished reading the round r slots (and
// the round r halo rows; halo rows of v are double-buffered by iteration parity since they
// are read once more after the following round).
// ---------------------------------------------------------------------------------------
constexpr int kXchgWaitPolls = 1 << 22;   // bound on mbarrier polls per round

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(uint64_t* mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}
// the local arrival of a round, announcing the bytes the round's stores will complete
__device__ __forceinline__ void mbar_arm(uint64_t* mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* mb, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void st_async_f32(uint32_t dst, float v, uint32_t mb) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];\n" ::"r"(dst),
               "r"(__float_as_uint(v)), "r"(mb)
               : "memory");
}
__device__ __forceinline__ void st_async_v2(uint32_t dst, float a, float b, uint32_t mb) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];\n" ::"r"(dst),
               "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(mb)
               : "memory");
}
__device__ __forceinline__ void st_async_v4(uint32_t dst, float a, float b, float c, float d, uint32_t mb) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];\n" ::"r"(dst),
      "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
      "r"(mb)
      : "memory");
}

struct Xchg {
  uint64_t* mb;     // [2] mbarriers (one per round parity), arrival count 1
  float* kslot;     // [2][kMaxCluster][4] partial sums by source rank
  float* wpart;     // [NW][4] warp partials
  uint32_t phase;   // bit b: parity of the current phase of mb[b]
  int round;
  bool dead;        // a wait ran out: skip further waits (the sweep reports an error)
};

// One exchange round: sum NV values over the cluster (every CTA gets bitwise the same totals:
// the CTA partials are added in rank order).  The caller has already sent the halo rows
// this round carries; halo_bytes is what this CTA receives of them.
template <class CFG, int NV>
__device__ __forceinline__ void xround(Xchg& xs, const float (&v)[NV], float (&tot)[NV], int rank, int C,
                                       uint32_t halo_bytes) {
  static_assert(NV == 2 || NV == 4, "partials travel as one v2 or v4 store");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = xs.round & 1;
  if (threadIdx.x == 0) mbar_arm(xs.mb + b, (uint32_t)(C * NV * 4) + halo_bytes);
  float w[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) w[q] = warp_butterfly<float>(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) xs.wpart[warp * 4 + q] = w[q];
  }
  __syncthreads();
  float* slot = xs.kslot + b * (kMaxCluster * 4);
  if (warp == 0) {
    float c[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) c[q] = warp_butterfly<float>(lane < CFG::NW ? xs.wpart[lane * 4 + q] : 0.f);
    if (lane < C) {
      const uint32_t dst = cluster_addr(smem_addr(slot + rank * 4), lane);
      const uint32_t mb = cluster_addr(smem_addr(xs.mb + b), lane);
      if constexpr (NV == 2) st_async_v2(dst, c[0], c[1], mb);
      else st_async_v4(dst, c[0], c[1], c[2], c[3], mb);
    }
  }
  if (!xs.dead) {
    const uint32_t par = (xs.phase >> b) & 1u;
    int polls = 0;
    while (!mbar_test(xs.mb + b, par)) {
      if (++polls >= kXchgWaitPolls) {
        xs.dead = true;
        break;
      }
    }
  }
  xs.phase ^= 1u << b;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    float acc = 0.f;
    for (int i = 0; i < C; ++i) acc += slot[i * 4 + q];
    tot[q] = acc;
  }
  ++xs.round;
}

// v with its sign flipped where bit k of `bits` is set: the product with the shadow residual
// r^ = sign(r_0) of row k.
__device__ __forceinline__ float signed_by(float v, uint32_t bits, int k) {
  return __int_as_float(__float_as_int(v) ^ (int)((bits >> k) << 31));
}

// Q = M^{-1} y = 2 y - A^ y on the strip's own rows and, for the edge groups, on the halo row
// next to the band (y has DH = 2 halo rows, its own values also in yc; Q has one halo row).
// The own rows of Q are also returned in q.  Outside the domain Q stays zero.
template <class CFG, int DH>
__device__ __forceinline__ void precond_apply(const float* __restrict__ y, const float (&yc)[CFG::K],
                                              float* __restrict__ Q, float (&q)[CFG::K],
                                              const float4* __restrict__ rowc, const float* __restrict__ ID,
                                              int col, int il, int ir, int r0, int grp, float ce, float cw,
                                              float cgi, bool has_up, bool has_down, float4 rc_top, float id_top,
                                              float4 rc_bot, float id_bot) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K, BH = CFG::BH;
  scaled_matvec_rc<CFG>(y + (DH - 1) * NCOL, yc, rowc, ID, col, il, ir, r0, ce, cw, cgi, q);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    q[k] = fmaf(2.f, yc[k], -q[k]);
    Q[(r0 + k + 1) * NCOL + col] = q[k];
  }
  if (grp == 0 && has_up) {
    const float* yr = y + (DH - 1) * NCOL;
    Q[col] = fmaf(2.f, yr[col], -scaled_row(yr, NCOL, col, il, ir, rc_top, id_top, ce, cw, cgi));
  }
  if (grp == CFG::G - 1 && has_down) {
    const float* yr = y + (BH + DH) * NCOL;
    Q[(BH + 1) * NCOL + col] = fmaf(2.f, yr[col], -scaled_row(yr, NCOL, col, il, ir, rc_bot, id_bot, ce, cw, cgi));
  }
}

// Q = M^{-1} y with the degree-2 Neumann polynomial M^{-1} = I + 1.5 E + E^2, E = I - A^,
// evaluated as y + E w with w = 1.5 y + E y:  w = 2.5 y - A^ y,  Q = (y + w) - A^ w.  w goes to
// the plane W (two halo rows each side; the edge groups evaluate them from y, which has
// DH = 3 halo rows), then Q to its plane on the own rows and one halo row each side; the own
// rows of Q are also returned in q.  Owner and neighbour evaluate a row with the same
// operations in the same order (scaled_node, fmaf, then an add and a subtract), so a halo row
// of W or Q equals its owner's row bit for bit and M^{-1} is the same operator on every CTA.
// Outside the domain W and Q stay zero.
template <class CFG>
__device__ __forceinline__ void precond_apply2(const float* __restrict__ y, const float (&yc)[CFG::K],
                                               float* __restrict__ W, float* __restrict__ Q, float (&q)[CFG::K],
                                               const float4* __restrict__ rowc, const float* __restrict__ ID,
                                               int col, int il, int ir, int r0, int grp, float ce, float cw,
                                               float cgi, bool has_up, bool has_down, const float4 (&rc_top)[2],
                                               const float (&id_top)[2], const float4 (&rc_bot)[2],
                                               const float (&id_bot)[2]) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K, BH = CFG::BH, DH = 3;
  float wk[K];
  scaled_matvec_rc<CFG>(y + (DH - 1) * NCOL, yc, rowc, ID, col, il, ir, r0, ce, cw, cgi, wk);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    wk[k] = fmaf(2.5f, yc[k], -wk[k]);
    W[(r0 + k + 2) * NCOL + col] = wk[k];
  }
  if (grp == 0 && has_up) {   // band rows -1 and -2 (W rows 1 and 0)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float* yr = y + (DH - 1 - t) * NCOL;
      W[(1 - t) * NCOL + col] = fmaf(2.5f, yr[col], -scaled_row(yr, NCOL, col, il, ir, rc_top[t], id_top[t], ce, cw, cgi));
    }
  }
  if (grp == CFG::G - 1 && has_down) {   // band rows BH and BH + 1 (W rows BH + 2, BH + 3)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float* yr = y + (BH + DH + t) * NCOL;
      W[(BH + 2 + t) * NCOL + col] = fmaf(2.5f, yr[col], -scaled_row(yr, NCOL, col, il, ir, rc_bot[t], id_bot[t], ce, cw, cgi));
    }
  }
  __syncthreads();
  scaled_matvec_rc<CFG>(W + NCOL, wk, rowc, ID, col, il, ir, r0, ce, cw, cgi, q);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    q[k] = (yc[k] + wk[k]) - q[k];
    Q[(r0 + k + 1) * NCOL + col] = q[k];
  }
  if (grp == 0 && has_up) {
    const float* wr = W + NCOL;
    Q[col] = (y[(DH - 1) * NCOL + col] + wr[col]) - scaled_row(wr, NCOL, col, il, ir, rc_top[0], id_top[0], ce, cw, cgi);
  }
  if (grp == CFG::G - 1 && has_down) {
    const float* wr = W + (BH + 2) * NCOL;
    Q[(BH + 1) * NCOL + col] = (y[(BH + DH) * NCOL + col] + wr[col]) -
                               scaled_row(wr, NCOL, col, il, ir, rc_bot[0], id_bot[0], ce, cw, cgi);
  }
}

// Shared-memory layout of sweep_band_kernel (floats first, every array a multiple of 16 B).
// The polynomial preconditioner needs the p and s planes with halo rows on each side as deep
// as its degree plus one and one more plane (Q); the degree-2 polynomial (POLY2) also the plane
// W with two halo rows, and strips of at least three rows (each edge group sends its DH rows);
// quadratic extrapolation (QUAD) one more own-row plane.  Each is used where it fits in the
// 227 KB of a CTA (the degree-2 polynomial first: it saves the most iterations).
template <class CFG>
struct SweepSmem {
  static constexpr int NCOL = CFG::NCOL, BH = CFG::BH, PLANE = CFG::PLANE, NW = CFG::NW;
  static constexpr size_t TAIL_BYTES = 2 * kMaxCluster * 4 * 8 + NW * 4 * 8 + 16 + sizeof(Scal);
  static constexpr size_t floats(int dh, bool q, bool w, bool quad) {
    return PLANE + 2 * (size_t)(BH + 2 * dh) * NCOL + (q ? PLANE : 0) + (w ? (size_t)(BH + 4) * NCOL : 0) +
           (2 + (quad ? 1 : 0)) * (size_t)BH * NCOL + 6 * (size_t)dh * NCOL + 2 * kMaxCluster * 4 + NW * 4;
  }
  static constexpr bool fits(size_t f) { return f * 4 + TAIL_BYTES <= 227 * 1024; }
  static constexpr bool POLY2 = CFG::K >= 3 && fits(floats(3, true, true, false));
  static constexpr bool POLY = POLY2 || fits(floats(2, true, false, false));
  static constexpr int DH = POLY2 ? 3 : POLY ? 2 : 1;   // halo rows of the p and s planes
  static constexpr bool QUAD = fits(floats(DH, POLY, POLY2, true));
  static constexpr int DPLANE = (BH + 2 * DH) * NCOL;
  static constexpr size_t u = 0, P = u + PLANE, S = P + DPLANE;         // u: one halo row; p, s: DH
  static constexpr size_t Q = S + DPLANE;        // preconditioned direction, one halo row (POLY only)
  static constexpr size_t W = Q + (POLY ? PLANE : 0);   // degree-2 intermediate, two halo rows (POLY2)
  static constexpr size_t ID = W + (POLY2 ? (size_t)(BH + 4) * NCOL : 0), XP = ID + BH * NCOL;   // own rows
  static constexpr size_t XQ = XP + BH * NCOL;   // d_{m-3}, own rows (QUAD only)
  static constexpr size_t VH = XQ + (QUAD ? BH * NCOL : 0);   // [2 parity][top DH, bottom DH rows][NCOL] v halo
  static constexpr size_t TH = VH + 4 * DH * NCOL;   // [top DH, bottom DH rows][NCOL] t halo rows
  static constexpr size_t KSLOT = TH + 2 * DH * NCOL;   // [2][kMaxCluster][4] exchange partials
  static constexpr size_t KWP = KSLOT + 2 * kMaxCluster * 4;   // [NW][4]
  static constexpr size_t FLOATS = KWP + NW * 4;
  // doubles after the floats: slots [2][kMaxCluster][4], wpart [NW][4]; then mbarriers, Scal
  static constexpr size_t SLOTS_B = FLOATS * 4, WPART_B = SLOTS_B + 2 * kMaxCluster * 4 * 8;
  static constexpr size_t MB_B = WPART_B + NW * 4 * 8, SCAL_B = MB_B + 16;
  static constexpr size_t BYTES = SCAL_B + sizeof(Scal);
  static_assert(FLOATS % 4 == 0, "16-byte alignment of the double arrays");
  static_assert(FLOATS == floats(DH, POLY, POLY2, QUAD), "layout and fit test agree");
  static_assert(CFG::K >= DH, "the edge groups send DH rows");
};

// Halo targets of a plane with DH halo rows on each side: own rows 0..DH-1 mirror into rows
// BH+DH.. of rank-1's plane, own rows BH-DH..BH-1 into rows 0.. of rank+1's plane.
template <class CFG, int DH>
__device__ __forceinline__ HaloPush deep_push(cg::cluster_group& cl, float* plane, int rank, int C) {
  HaloPush h;
  h.prev_bottom = rank > 0 ? cl.map_shared_rank(plane, rank - 1) + (CFG::BH + DH) * CFG::NCOL : nullptr;
  h.next_top = rank < C - 1 ? cl.map_shared_rank(plane, rank + 1) : nullptr;
  return h;
}
template <class CFG, int DH>
__device__ __forceinline__ void deep_store(float* plane, const HaloPush& h, int r, int c, float v) {
  plane[(r + DH) * CFG::NCOL + c] = v;
  if (r < DH && h.prev_bottom) h.prev_bottom[r * CFG::NCOL + c] = v;
  if (r >= CFG::BH - DH && h.next_top) h.next_top[(r - (CFG::BH - DH)) * CFG::NCOL + c] = v;
}

template <class CFG>
__global__ void __launch_bounds__(CFG::NT, 1) sweep_band_kernel(const __grid_constant__ SweepParams sp) {
  constexpr int NCOL = CFG::NCOL, K = CFG::K, BH = CFG::BH, G = CFG::G;
  using L = SweepSmem<CFG>;
  constexpr int DH = L::DH;
  cg::cluster_group cluster = cg::this_cluster();
  const ItemDesc& d = sp.d;
  const SweepArgs& a = sp.a;
  const int M = sp.sh.M, C = sp.sh.C;
  const int rank = C > 1 ? (int)cluster.block_rank() : 0;
  const int tid = threadIdx.x;
  const int col = tid % NCOL, grp = G == 1 ? 0 : tid / NCOL;
  const int r0 = grp * K;   // a compile-time 0 in one-group variants: uniform row indices
  const int jbase = rank * BH;
  const size_t MM = (size_t)M * M;
  const float h = sp.h;
  const PayoffF pf = make_payoff(d);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* fs = reinterpret_cast<float*>(smem_raw);
  float* u = fs + L::u;      // state w / u          [PLANE]
  float* P = fs + L::P;      // search direction p   [DPLANE]: own row r at plane row r + DH
  float* S = fs + L::S;      // s                    [DPLANE]
  float* Q = fs + L::Q;      // M^{-1} p, M^{-1} s   [PLANE] (L::POLY)
  float* W = fs + L::W;      // 2.5 y - A^ y          [(BH + 4) * NCOL] (L::POLY2)
  const float* P1 = P + (DH - 1) * NCOL;   // p and s seen with one halo row
  const float* S1 = S + (DH - 1) * NCOL;
  float* ID = fs + L::ID;    // inverse diagonal     [BH*NCOL]
  float* XP = fs + L::XP;    // increment before xw  [BH*NCOL]
  float* XQ = fs + L::XQ;    // the one before that  [BH*NCOL] (L::QUAD)
  float* VH = fs + L::VH;
  float* TH = fs + L::TH;
  const float4* rowc = sp.rowc + jbase;   // own band rows (index r0 + k)
  double* slots = reinterpret_cast<double*>(smem_raw + L::SLOTS_B);
  double* wpart = reinterpret_cast<double*>(smem_raw + L::WPART_B);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + L::MB_B);
  Scal* sc = reinterpret_cast<Scal*>(smem_raw + L::SCAL_B);

  const HaloPush pu = halo_push<CFG>(cluster, u, rank, C);
  const HaloPush pP = deep_push<CFG, DH>(cluster, P, rank, C);
  const HaloPush pS = deep_push<CFG, DH>(cluster, S, rank, C);
  static_assert(K <= 32, "one sign bit per strip row");
  const bool has_up = rank > 0, has_down = rank < C - 1;
  // receivers of this thread's halo stores (v and t rows): group 0 sends band rows 0..DH-1 to
  // the bottom halo of rank-1, group G-1 sends band rows BH-DH..BH-1 to the top halo of rank+1
  const bool send_up = grp == 0 && has_up, send_down = grp == G - 1 && has_down;
  const uint32_t halo_bytes = (uint32_t)((has_up ? 1 : 0) + (has_down ? 1 : 0)) * DH * NCOL * 4;

  for (int e = tid; e < BH * NCOL; e += CFG::NT) {
    const int r = e / NCOL, c = e % NCOL;
    const int j = jbase + r;
    ID[e] = (j < M - 1 && c < M - 1) ? inv_diag(d, c, j) : 0.f;
  }
  for (int e = tid; e < L::DPLANE; e += CFG::NT) {
    P[e] = 0.f; S[e] = 0.f;
  }
  if (L::POLY)
    for (int e = tid; e < CFG::PLANE; e += CFG::NT) Q[e] = 0.f;
  if (L::POLY2)
    for (int e = tid; e < (BH + 4) * NCOL; e += CFG::NT) W[e] = 0.f;
  for (int e = tid; e < 6 * DH * NCOL; e += CFG::NT) VH[e] = 0.f;   // VH and TH
  if (tid == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  Xchg xs;
  xs.mb = mbar;
  xs.kslot = fs + L::KSLOT;
  xs.wpart = fs + L::KWP;
  xs.phase = 0;
  xs.round = 0;
  xs.dead = false;
  float ce = 0.f, cw = 0.f, cgi = 0.f;
  column_coefs(d, col, ce, cw, cgi);
  const int il = col > 0 ? col - 1 : 0;
  const int ir = col + 1 < NCOL ? col + 1 : col;
  // coefficients of the halo rows next to the band (rows jbase-1 and jbase+BH), where the
  // edge groups evaluate the preconditioner
  // coefficients of the halo rows next to the band (rows jbase-1, jbase-2 and jbase+BH,
  // jbase+BH+1), where the edge groups evaluate the preconditioner
  float4 rc_top[2], rc_bot[2];
  float id_top[2], id_bot[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    rc_top[t] = rc_bot[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    id_top[t] = id_bot[t] = 0.f;
  }
  if (L::POLY) {
#pragma unroll
    for (int t = 0; t < (L::POLY2 ? 2 : 1); ++t) {
      const int jt = jbase - 1 - t, jb = jbase + BH + t;
      if (grp == 0 && has_up) {
        rc_top[t] = sp.rowc[jt];
        id_top[t] = (jt < M - 1 && col < M - 1) ? inv_diag(d, col, jt) : 0.f;
      }
      if (grp == G - 1 && has_down) {
        rc_bot[t] = sp.rowc[jb];
        id_bot[t] = (jb < M - 1 && col < M - 1) ? inv_diag(d, col, jb) : 0.f;
      }
    }
  }
  const float rdt = d.rdt;
  const float tol = (float)a.tol;
  int round = 0;
  int iters_max = 0, iters_total = 0, nsolves = 0;
  int kit = 0;   // BiCGSTAB iterations run by this kernel (parity of the v halo buffers)
  bool failed = false;

  // batched PROP: this cluster's state
  const bool batched = a.mode == SWEEP_PROP && a.nprop > 0;
  const PropItem pit = batched ? a.prop[blockIdx.y] : PropItem{a.in, a.out, d.tau0};
  // initial state of the first slice (own rows and halo rows)
  // slices of this launch (a chunk of the sweep, or all of it)
  const int n_lo = a.n_end > 0 ? a.n_begin : a.n_first;
  const int n_hi = a.n_end > 0 ? a.n_end : (a.mode == SWEEP_PROP ? a.n_first + 1 : a.N);
  const float* src;
  if (a.mode == SWEEP_PROP) src = pit.in;
  else if (a.mode == SWEEP_INIT) src = a.U + (size_t)n_lo * MM;
  else if (n_lo == a.n_first) src = a.Gold + (size_t)a.n_first * MM;   // G(u_k) unchanged: G_old_k
  else src = a.U + (size_t)n_lo * MM;                                    // corrected by the chunk before
  band_load<CFG>(u, src, M, jbase, tid);
  cluster_barrier(cluster, C);   // also publishes the mbarrier initialisation

  // Initial guess of each solve: the extrapolation of the previous coarse increments --
  // quadratic 3 d_{m-1} - 3 d_{m-2} + d_{m-3} where the third history plane fits in shared
  // memory, else linear 2 d_{m-1} - d_{m-2} (d_{m-1} after one step, 0 at the start).  The
  // increments of consecutive steps vary smoothly: the linear start saves about 30% of the
  // BiCGSTAB iterations against the previous increment, the quadratic one 30% more.
  float xw[K];   // d_{m-1}; XP holds d_{m-2}, XQ d_{m-3} (own rows)
#pragma unroll
  for (int k = 0; k < K; ++k) xw[k] = 0.f;
  int nhist = 0;
  for (int n = n_lo; n < n_hi; ++n) {
    const bool skip_g = (a.mode == SWEEP_ITER && n == a.n_first);
    if (!skip_g) {
      for (int cstep = 0; cstep < a.csteps; ++cstep) {
        const double tau_new = pit.tau0 + a.slice_len * n + (cstep + 1) * d.dtau;
        band_far_field<CFG>(u, pu, pf, (float)tau_new, h, M, jbase, tid);
        cluster_barrier(cluster, C);
        if (L::QUAD && nhist >= 3) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int e = (r0 + k) * NCOL + col;
            const float d2 = XP[e], d3 = XQ[e];
            XQ[e] = d2;
            XP[e] = xw[k];
            xw[k] = 3.f * (xw[k] - d2) + d3;
          }
        } else if (nhist >= 2) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int e = (r0 + k) * NCOL + col;
            const float dprev = XP[e];
            if (L::QUAD) XQ[e] = dprev;
            XP[e] = xw[k];
            xw[k] = 2.f * xw[k] - dprev;
          }
        } else if (nhist == 1) {
#pragma unroll
          for (int k = 0; k < K; ++k) XP[(r0 + k) * NCOL + col] = xw[k];
        }
        // per thread: x, r (s after the first round of an iteration), v, t and p of the strip
        float x[K], rr[K], vv[K], tt[K], pk[K];
        int it = 0;
        bool conv = false;
        // A breakdown (a zero denominator in alpha, omega or beta) restarts the solve from
        // the current iterate with a fresh shadow residual.
        for (int attempt = 0; attempt < kKrylovAttempts; ++attempt) {
          // a restart rewrites the neighbours' P halo rows: they must have left the iteration
          if (attempt > 0) cluster_barrier(cluster, C);
          // b^ = D^{-1} dtau R_h w;  x = initial guess;  r = p = b^ - A^ x;  r^ = sign(r)
          float bb_part = 0.f, rabs_part = 0.f;
          {
            const int p0 = r0 + 1;
            float nW = u[(p0 - 1) * NCOL + il], nC = u[(p0 - 1) * NCOL + col], nE = u[(p0 - 1) * NCOL + ir];
            float cW = u[p0 * NCOL + il], cC = u[p0 * NCOL + col], cE = u[p0 * NCOL + ir];
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int p = p0 + k;
              const float sW = u[(p + 1) * NCOL + il], sC = u[(p + 1) * NCOL + col],
                          sE = u[(p + 1) * NCOL + ir];
              const float4 rc = rowc[p - 1];
              const float cg = cgi * rc.z;
              const float bb = ce * (cE - cC) - cw * (cC - cW) + rc.x * (sC - cC) - rc.y * (cC - nC) +
                               cg * ((sE - nE) - (sW - nW)) - rdt * cC;
              const float bh = bb * ID[(p - 1) * NCOL + col];
              x[k] = xw[k]; rr[k] = bh; vv[k] = 0.f; tt[k] = 0.f;
              bb_part = fmaf(bh, bh, bb_part);
              nW = cW; nC = cC; nE = cE;
              cW = sW; cC = sC; cE = sE;
            }
          }
          // x goes through the s plane (free until the first iteration writes s), so that p can
          // take r right after the product without a reduction in between
#pragma unroll
          for (int k = 0; k < K; ++k) deep_store<CFG, DH>(S, pS, r0 + k, col, x[k]);
          cluster_barrier(cluster, C);
          scaled_matvec_rc<CFG>(S1, x, rowc, ID, col, il, ir, r0, ce, cw, cgi, vv);
          // The shadow residual r^ = sign(r_0) (+1 where r_0 = 0): its dot products need no
          // loads, only the thread's K sign bits, and (r^, r_0) = sum |r_0| > 0.  On the CPU
          // model of the workload it takes the iterations of r^ = r_0.
          uint32_t rsign = 0;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            rr[k] -= vv[k];
            rsign |= (rr[k] < 0.f ? 1u : 0u) << k;
            rabs_part += fabsf(rr[k]);
            deep_store<CFG, DH>(P, pP, r0 + k, col, rr[k]);
            pk[k] = rr[k];
          }
          cluster_barrier(cluster, C);
          // rho = (r^, r_0), the stopping threshold and the start test arrive with the first
          // exchange round (the first iteration's)
          float rho = 0.f, stop2 = 0.f;
          bool first = true;
          conv = false;
          bool fail = false;
          // r on the halo rows (kept by the threads that own those columns of the edge groups;
          // the P halo rows hold r here)
          float rh_top[DH], rh_bot[DH];
#pragma unroll
          for (int t = 0; t < DH; ++t) {
            rh_top[t] = grp == 0 ? P[t * NCOL + col] : 0.f;
            rh_bot[t] = grp == G - 1 ? P[(BH + DH + t) * NCOL + col] : 0.f;
          }
          // BiCGSTAB iterations with two exchange rounds each.  The halo rows of s and p are
          // computed locally from r, v and t on the halo rows (v and t arrive with the rounds),
          // so the matrix-vector products need no cluster barrier.
          //
          // POLY: right preconditioning with M^{-1} = 2I - A^, the first two terms of the
          // Neumann series of A^{-1} (A^ = I - (off-diagonal part), so M^{-1} A^ is closer to
          // I): v = A^ M^{-1} p, t = A^ M^{-1} s, x += alpha M^{-1} p + omega M^{-1} s.  It
          // halves the iterations for one more stencil evaluation per product; M^{-1} y on the
          // row next to the band needs y two rows into the halo, so p, s, v and t keep two
          // halo rows.
          while (!conv && it < a.maxit) {
            ++it;
            const int par = kit & 1;
            float* vh_top = VH + (2 * par) * DH * NCOL;
            float* vh_bot = vh_top + DH * NCOL;
            // v = A^ p (POLY: A^ M^{-1} p) ;  alpha = rho / (r^, v) ;  (r, r) for the stopping test
            if constexpr (L::POLY2) {
              float qk[K];
              precond_apply2<CFG>(P, pk, W, Q, qk, rowc, ID, col, il, ir, r0, grp, ce, cw, cgi, has_up, has_down,
                                  rc_top, id_top, rc_bot, id_bot);
              __syncthreads();
              scaled_matvec_rc<CFG>(Q, qk, rowc, ID, col, il, ir, r0, ce, cw, cgi, vv);
            } else if constexpr (L::POLY) {
              float qk[K];
              precond_apply<CFG, DH>(P, pk, Q, qk, rowc, ID, col, il, ir, r0, grp, ce, cw, cgi, has_up, has_down,
                                     rc_top[0], id_top[0], rc_bot[0], id_bot[0]);
              __syncthreads();
              scaled_matvec_rc<CFG>(Q, qk, rowc, ID, col, il, ir, r0, ce, cw, cgi, vv);
            } else {
              scaled_matvec_rc<CFG>(P1, pk, rowc, ID, col, il, ir, r0, ce, cw, cgi, vv);
            }
            {
              const uint32_t mb = smem_addr(xs.mb + (xs.round & 1));
#pragma unroll
              for (int t = 0; t < DH; ++t) {
                if (send_up)
                  st_async_f32(cluster_addr(smem_addr(vh_bot + t * NCOL + col), rank - 1), vv[t],
                               cluster_addr(mb, rank - 1));
                if (send_down)
                  st_async_f32(cluster_addr(smem_addr(vh_top + t * NCOL + col), rank + 1), vv[K - DH + t],
                               cluster_addr(mb, rank + 1));
              }
            }
            float p1[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < K; ++k) {
              p1[0] += signed_by(vv[k], rsign, k);
              p1[1] = fmaf(rr[k], rr[k], p1[1]);
            }
            float ta[4];
            if (first) {
              // the first round also carries (b^, b^) and (r^, r_0)
              const float p1x[4] = {p1[0], p1[1], bb_part, rabs_part};
              xround<CFG, 4>(xs, p1x, ta, rank, C, halo_bytes);
              first = false;
              stop2 = tol * tol * ta[2];
              rho = ta[3];
              if (!xs.dead && (ta[1] <= stop2 || !(ta[2] > 1e-30f))) {   // the guess already solves it
                --it;
                conv = true;
                break;
              }
            } else {
              float t2[2];
              xround<CFG, 2>(xs, p1, t2, rank, C, halo_bytes);
              ta[0] = t2[0];
              ta[1] = t2[1];
            }
            if (xs.dead) { conv = true; break; }
            if (ta[1] <= stop2) { conv = true; break; }
            if (ta[0] == 0.f) { fail = true; break; }
            const float af = rho / ta[0];
            // s = r - alpha v (rr holds s from here on), own rows and halo rows
#pragma unroll
            for (int k = 0; k < K; ++k) {
              if constexpr (L::POLY) x[k] = fmaf(af, Q[(r0 + k + 1) * NCOL + col], x[k]);   // x += alpha M^{-1} p
              else x[k] = fmaf(af, pk[k], x[k]);
              rr[k] = fmaf(-af, vv[k], rr[k]);
              S[(r0 + k + DH) * NCOL + col] = rr[k];
            }
#pragma unroll
            for (int t = 0; t < DH; ++t) {
              if (grp == 0) S[t * NCOL + col] = has_up ? fmaf(-af, vh_top[t * NCOL + col], rh_top[t]) : 0.f;
              if (grp == G - 1)
                S[(BH + DH + t) * NCOL + col] = has_down ? fmaf(-af, vh_bot[t * NCOL + col], rh_bot[t]) : 0.f;
            }
            __syncthreads();
            // t = A^ s (POLY: A^ M^{-1} s) ;  omega = (t, s) / (t, t) ;  rho_new = (r^, s) - omega (r^, t)
            if constexpr (L::POLY2) {
              float qk[K];
              precond_apply2<CFG>(S, rr, W, Q, qk, rowc, ID, col, il, ir, r0, grp, ce, cw, cgi, has_up, has_down,
                                  rc_top, id_top, rc_bot, id_bot);
              __syncthreads();
              scaled_matvec_rc<CFG>(Q, qk, rowc, ID, col, il, ir, r0, ce, cw, cgi, tt);
            } else if constexpr (L::POLY) {
              float qk[K];
              precond_apply<CFG, DH>(S, rr, Q, qk, rowc, ID, col, il, ir, r0, grp, ce, cw, cgi, has_up, has_down,
                                     rc_top[0], id_top[0], rc_bot[0], id_bot[0]);
              __syncthreads();
              scaled_matvec_rc<CFG>(Q, qk, rowc, ID, col, il, ir, r0, ce, cw, cgi, tt);
            } else {
              scaled_matvec_rc<CFG>(S1, rr, rowc, ID, col, il, ir, r0, ce, cw, cgi, tt);
            }
            {
              const uint32_t mb = smem_addr(xs.mb + (xs.round & 1));
#pragma unroll
              for (int t = 0; t < DH; ++t) {
                if (send_up)
                  st_async_f32(cluster_addr(smem_addr(TH + (DH + t) * NCOL + col), rank - 1), tt[t],
                               cluster_addr(mb, rank - 1));
                if (send_down)
                  st_async_f32(cluster_addr(smem_addr(TH + t * NCOL + col), rank + 1), tt[K - DH + t],
                               cluster_addr(mb, rank + 1));
              }
            }
            float p2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < K; ++k) {
              p2[0] = fmaf(tt[k], rr[k], p2[0]);
              p2[1] = fmaf(tt[k], tt[k], p2[1]);
              p2[2] += signed_by(rr[k], rsign, k);
              p2[3] += signed_by(tt[k], rsign, k);
            }
            float tb[4];
            xround<CFG, 4>(xs, p2, tb, rank, C, halo_bytes);
            if (xs.dead) { conv = true; break; }
            const float of = tb[1] > 0.f ? tb[0] / tb[1] : 0.f;
            const float rho_new = tb[2] - of * tb[3];
            float bf = 0.f;
            if (of == 0.f || rho == 0.f) fail = true;
            else bf = (rho_new / rho) * (af / of);
            rho = rho_new;
            // x += omega s (POLY: omega M^{-1} s) ;  r = s - omega t ;  p = r + beta (p - omega v)
#pragma unroll
            for (int k = 0; k < K; ++k) {
              if constexpr (L::POLY) x[k] = fmaf(of, Q[(r0 + k + 1) * NCOL + col], x[k]);
              else x[k] = fmaf(of, rr[k], x[k]);
              rr[k] = fmaf(-of, tt[k], rr[k]);
              pk[k] = fmaf(bf, fmaf(-of, vv[k], pk[k]), rr[k]);
              P[(r0 + k + DH) * NCOL + col] = pk[k];
            }
#pragma unroll
            for (int t = 0; t < DH; ++t) {
              if (grp == 0) {
                float* pp = P + t * NCOL + col;
                rh_top[t] = has_up ? fmaf(-of, TH[t * NCOL + col], S[t * NCOL + col]) : 0.f;
                *pp = has_up ? fmaf(bf, fmaf(-of, vh_top[t * NCOL + col], *pp), rh_top[t]) : 0.f;
              }
              if (grp == G - 1) {
                float* pp = P + (BH + DH + t) * NCOL + col;
                rh_bot[t] = has_down ? fmaf(-of, TH[(DH + t) * NCOL + col], S[(BH + DH + t) * NCOL + col]) : 0.f;
                *pp = has_down ? fmaf(bf, fmaf(-of, vh_bot[t * NCOL + col], *pp), rh_bot[t]) : 0.f;
              }
            }
            __syncthreads();
            ++kit;
            if (fail) break;
          }
          if (conv || !fail) break;
#pragma unroll
          for (int k = 0; k < K; ++k) xw[k] = x[k];
        }
        if (!conv) failed = true;
        iters_max = it > iters_max ? it : iters_max;
        iters_total += it;
        ++nsolves;
#pragma unroll
        for (int k = 0; k < K; ++k) xw[k] = x[k];
        nhist = nhist < 3 ? nhist + 1 : 3;
        // u^{m+1} = w + d (d = 0 off the PDE rows, whose values already hold g(tau_new))
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int idx = (r0 + k + 1) * NCOL + col;
          band_store<CFG>(u, pu, r0 + k, col, u[idx] + x[k]);
        }
        cluster_barrier(cluster, C);
      }
    }

    if (a.mode == SWEEP_PROP) {
      if (col < M) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = jbase + r0 + k;
          if (j < M) pit.out[(size_t)j * M + col] = u[(r0 + k + 1) * NCOL + col];
        }
      }
    } else if (a.mode == SWEEP_INIT) {
      // The norms: each thread adds its K nodes in FP32, the sum over threads and CTAs is
      // FP64 (FP64 runs at a small fraction of the FP32 rate on this part; per-node FP64
      // arithmetic took a few microseconds per slice on the 16 SMs of the cluster).
      float nf = 0.f;
      if (col < M) {
        float* Un = a.U + (size_t)(n + 1) * MM;
        float* Gn = a.Gold + (size_t)n * MM;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = jbase + r0 + k;
          if (j < M) {
            const float g = u[(r0 + k + 1) * NCOL + col];
            Un[(size_t)j * M + col] = g;
            Gn[(size_t)j * M + col] = g;
            nf = fmaf(g, g, nf);
          }
        }
      }
      double nr[1] = {(double)nf};
      double* norms = a.norms;
      const int slot_n = n + 1;
      cluster_sum<CFG, 1>(cluster, nr, slots, wpart, sc, round, rank, C, [norms, slot_n, rank](Scal* s) {
        if (rank == 0) { norms[2 * slot_n] = s->tot[0]; norms[2 * slot_n + 1] = 0.0; }
      });
    } else {
      // correction u_{n+1} = F_n + (G_new - G_old_n) and defect partials (per thread in FP32:
      // u_new - u_old of nearby values is exact, Sterbenz; over threads and CTAs in FP64)
      float nf[2] = {0.f, 0.f};
      float* Un = a.U + (size_t)(n + 1) * MM;
      const float* Fn = a.Fb + (size_t)n * MM;
      float* Gn = a.Gold + (size_t)n * MM;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = jbase + r0 + k;
        if (col < M && j < M) {
          const size_t gi = (size_t)j * M + col;
          const float gnew = u[(r0 + k + 1) * NCOL + col];
          const float unew = Fn[gi] + (gnew - Gn[gi]);
          const float uold = Un[gi];
          Un[gi] = unew;
          Gn[gi] = gnew;
          band_store<CFG>(u, pu, r0 + k, col, unew);
          const float du = unew - uold;
          nf[0] = fmaf(unew, unew, nf[0]);
          nf[1] = fmaf(du, du, nf[1]);
        }
      }
      double nr[2] = {(double)nf[0], (double)nf[1]};
      double* norms = a.norms;
      const int slot_n = n + 1;
      cluster_sum<CFG, 2>(cluster, nr, slots, wpart, sc, round, rank, C, [norms, slot_n, rank](Scal* s) {
        if (rank == 0) { norms[2 * slot_n] = s->tot[0]; norms[2 * slot_n + 1] = s->tot[1]; }
      });
    }
  }
  cluster_barrier(cluster, C);   // no CTA leaves while another may still address its memory

  if (rank == 0 && tid == 0) {
    if (failed) atomicOr(a.status, 1);
    atomicMax(a.status + 1, iters_max);
    atomicAdd(a.status + 2, iters_total);
    atomicAdd(a.status + 3, nsolves);
    if (a.mode == SWEEP_ITER && n_hi == a.N) {
      double num = 0.0, den = 0.0;
      for (int n = 1; n <= a.N; ++n) {
        den = fmax(den, a.norms[2 * n]);
        if (n >= a.n_first + 1) num = fmax(num, a.norms[2 * n + 1]);
      }
      a.defect[0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
    }
  }
  if (xs.dead && tid == 0) atomicOr(a.status, 2);
}

// Dynamic shared memory of sweep_band_kernel.
template <class CFG>
static size_t sweep_smem_bytes() {
  return SweepSmem<CFG>::BYTES;
}

// The shared memory a CTA may claim on the current device (0 if the query fails).
static size_t smem_optin_bytes() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (size_t)v;
}

// {cs, cn, (float)j, 0} of rows 0..kMaxBandRows-1 from the item's host-rounded constants, in
// double and rounded once (the same on every host).
static void fill_row_coefs(SweepParams& sp) {
  const double ay = sp.d.ay, my = sp.d.my;
  for (int j = 0; j < kMaxBandRows; ++j) {
    const double b = ay * ((double)j * j), n = my * j;
    sp.rowc[j] = make_float4((float)(b + n), (float)(b - n), (float)j, 0.f);
  }
}

template <class CFG>
static int launch_sweep_k(const SweepParams& sp, cudaStream_t s) {
  // A single system (the serial sweep, one PROP state) claims all of each SM's shared memory,
  // so that no CTA of a concurrent kernel (the fine propagator of the pipelined driver) shares
  // its SMs: the sweep is the serial critical path, and an SM shared with a stencil kernel
  // issues its iterations up to a third slower.  Batched PROP packs its clusters as usual.
  const bool batched = sp.a.mode == SWEEP_PROP && sp.a.nprop > 0;
  size_t smem = sweep_smem_bytes<CFG>();
  if (!batched) {
    static const size_t optin = smem_optin_bytes();
    if (optin > smem) smem = optin;
  }
  auto kern = sweep_band_kernel<CFG>;
  BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (sp.sh.C > 8) BS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sp.sh.C, sp.a.mode == SWEEP_PROP && sp.a.nprop > 0 ? sp.a.nprop : 1, 1);
  cfg.blockDim = dim3(CFG::NT, 1, 1);
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

// ---------------------------------------------------------------------------------------
// Grids beyond one cluster's shared memory (M > 256): the same BiCGSTAB and Parareal sweep
// with the vectors in a global workspace.  One cluster of CG CTAs owns the system; CTA rank
// handles rows [rank*BHg, rank*BHg + BHg).  Each stencil pass stages its operand rows (R rows
// of the band plus one halo row on each side) in shared memory once, so every value crosses
// L2 once rather than nine times; the rows written by other CTAs are read with ld.global.cg
// (L2, never a stale L1 line), ordered by the cluster barrier's release/acquire.
// ---------------------------------------------------------------------------------------
constexpr int kGThreads = 1024;
struct GCfg {
  static constexpr int NW = kGThreads / 32;
};

struct GlobalVecs {
  float *u, *x, *xp, *xq, *r, *rh, *p, *v, *s, *t, *id, *q;   // q: M^{-1} p, then M^{-1} s
};
constexpr int kGlobalVecs = 12;

struct GSweepParams {
  ItemDesc d;
  SweepArgs a;
  GlobalVecs w;
  int M, C;
  float h;
};

__device__ __forceinline__ void g_coefs(const ItemDesc& d, int i, int j, float& ce, float& cw,
                                        float& cs, float& cn, float& cg) {
  float cgi, gj;
  column_coefs(d, i, ce, cw, cgi);
  row_coefs(d, j, cs, cn, gj);
  cg = cgi * gj;
}

// Shared-memory tiles of the stencil passes: rows ra-1 .. rb of an M-column vector with row
// stride S = M + 8; column c sits at index c + 4, so columns -1 and M read the zero pads and
// 16-byte copies land aligned.  Rows outside the grid are zero.
constexpr int kTilePad = 4;
__host__ __device__ inline int g_tile_stride(int M) { return M + 2 * kTilePad; }

__device__ __forceinline__ void g_stage(const float* __restrict__ y, float* __restrict__ tile, int M, int ra, int rb) {
  const int S = g_tile_stride(M);
  const int rows = rb - ra + 2;   // ra-1 .. rb
  if ((M & 3) == 0) {
    const int q = M >> 2;
#pragma unroll 4
    for (int idx = threadIdx.x; idx < rows * q; idx += kGThreads) {
      const int r = idx / q, c4 = idx - r * q;
      const int j = ra - 1 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j >= 0 && j < M) v = __ldcg(reinterpret_cast<const float4*>(y + (size_t)j * M) + c4);
      *reinterpret_cast<float4*>(tile + r * S + kTilePad + 4 * c4) = v;
    }
  } else {
#pragma unroll 4
    for (int idx = threadIdx.x; idx < rows * M; idx += kGThreads) {
      const int r = idx / M, c = idx - r * M;
      const int j = ra - 1 + r;
      tile[r * S + kTilePad + c] = (j >= 0 && j < M) ? __ldcg(y + (size_t)j * M + c) : 0.f;
    }
  }
}

// A^ y at node (i, j) from a tile whose first row is ra - 1.
__device__ __forceinline__ float g_tile_matvec(const float* tile, int S, int ra, int i, int j, float id, float ce,
                                               float cw, float cs, float cn, float cg) {
  const float* c = tile + (j - ra + 1) * S + kTilePad + i;
  const float yc = c[0], yw = c[-1], ye = c[1];
  const float yn = c[-S], ys = c[S], ynw = c[-S - 1], yne = c[-S + 1], ysw = c[S - 1], yse = c[S + 1];
  return yc - id * (ce * ye + cw * yw + cs * ys + cn * yn + cg * ((yse - yne) - (ysw - ynw)));
}

// Rows of a band per staged pass: two tiles of R + 2 rows in the dynamic shared memory.
__host__ __device__ inline int g_tile_rows(int M, int BHg, size_t smem_bytes) {
  const int fit = (int)(smem_bytes / (2 * sizeof(float) * (size_t)g_tile_stride(M))) - 2;
  return fit < BHg ? (fit > 0 ? fit : 1) : BHg;
}
constexpr size_t kGTileBytes = 200 * 1024;   // dynamic shared memory of the global sweep

// Visits the nodes e = b0 + tid, b0 + tid + kGThreads, ... < b1 as f(e, i, j), stepping (i, j)
// instead of dividing e by M at every node (a 64-bit division is a long instruction sequence).
template <class F>
__device__ __forceinline__ void g_nodes(size_t b0, size_t b1, int M, F f) {
  const int step_j = kGThreads / M, step_i = kGThreads - step_j * M;
  size_t e = b0 + threadIdx.x;
  int j = (int)(e / (size_t)M), i = (int)(e - (size_t)j * M);
  for (; e < b1; e += kGThreads) {
    f(e, i, j);
    i += step_i;
    j += step_j;
    if (i >= M) {
      i -= M;
      ++j;
    }
  }
}

// One stencil pass over the CTA's rows j0..j1-1: stage y0 (and y1) tile by tile, then run
// body(e, i, j, ra) for every node of the tile's rows (ra: the tile's first own row).
template <class Body>
__device__ __forceinline__ void g_pass(const float* y0, const float* y1, float* t0, float* t1, int M, int j0, int j1,
                                       int R, Body body) {
  for (int ra = j0; ra < j1; ra += R) {
    const int rb = min(j1, ra + R);
    g_stage(y0, t0, M, ra, rb);
    if (y1) g_stage(y1, t1, M, ra, rb);
    __syncthreads();
    g_nodes((size_t)ra * M, (size_t)rb * M, M, [&](size_t e, int i, int j) { body(e, i, j, ra); });
    __syncthreads();   // the tiles are restaged next
  }
}

__global__ void __launch_bounds__(kGThreads, 1) sweep_global_kernel(const __grid_constant__ GSweepParams gp) {
  cg::cluster_group cluster = cg::this_cluster();
  const ItemDesc& d = gp.d;
  const SweepArgs& a = gp.a;
  const bool batched = a.mode == SWEEP_PROP && a.nprop > 0;
  const PropItem pit = batched ? a.prop[blockIdx.y] : PropItem{a.in, a.out, d.tau0};
  // per-state workspace of a batched PROP launch
  GlobalVecs w = gp.w;
  if (batched) {
    const size_t off = (size_t)blockIdx.y * kGlobalVecs * (size_t)gp.M * gp.M;
    w.u += off; w.x += off; w.xp += off; w.xq += off; w.r += off; w.rh += off;
    w.p += off; w.v += off; w.s += off; w.t += off; w.id += off; w.q += off;
  }
  const int M = gp.M, C = gp.C;
  const int rank = C > 1 ? (int)cluster.block_rank() : 0;
  const int tid = threadIdx.x;
  const size_t MM = (size_t)M * M;
  const int BHg = (M + C - 1) / C;
  const int j0 = rank * BHg, j1 = min(M, j0 + BHg);
  const size_t e0 = (size_t)j0 * M, e1 = (size_t)j1 * M;
  const PayoffF pf = make_payoff(d);
  const float rdt = d.rdt;
  const float tol = (float)a.tol;
  __shared__ double slots[2 * kMaxCluster * 4];
  __shared__ double wpart[GCfg::NW * 4];
  __shared__ Scal scs;
  Scal* sc = &scs;
  extern __shared__ __align__(16) float gtiles[];
  const int S = g_tile_stride(M);
  const int R = g_tile_rows(M, BHg, kGTileBytes);
  float* T0 = gtiles;
  float* T1 = gtiles + (R + 2) * S;
  for (int idx = tid; idx < 2 * (R + 2) * S; idx += kGThreads) gtiles[idx] = 0.f;   // pads stay zero
  int round = 0, iters_max = 0, iters_total = 0, nsolves = 0, nhist = 0;
  bool failed = false;
  auto barrier = [&]() { __threadfence(); cluster_barrier(cluster, C); };

  const int n_lo = a.n_end > 0 ? a.n_begin : a.n_first;
  const int n_hi = a.n_end > 0 ? a.n_end : (a.mode == SWEEP_PROP ? a.n_first + 1 : a.N);
  g_nodes(e0, e1, M, [&](size_t e, int i, int j) {
    w.id[e] = (i < M - 1 && j < M - 1) ? inv_diag(d, i, j) : 0.f;
    w.x[e] = 0.f;
    w.xp[e] = 0.f;
    w.xq[e] = 0.f;
    w.q[e] = 0.f;
    const float* src = a.mode == SWEEP_PROP   ? pit.in
                       : a.mode == SWEEP_INIT ? a.U + (size_t)n_lo * MM
                       : n_lo == a.n_first    ? a.Gold + (size_t)a.n_first * MM
                                              : a.U + (size_t)n_lo * MM;
    w.u[e] = src[e];
  });
  barrier();
  for (int n = n_lo; n < n_hi; ++n) {
    const bool skip_g = (a.mode == SWEEP_ITER && n == a.n_first);
    if (!skip_g) {
      for (int cstep = 0; cstep < a.csteps; ++cstep) {
        const float tau_new = (float)(pit.tau0 + a.slice_len * n + (cstep + 1) * d.dtau);
        // initial guess 3 d_{m-1} - 3 d_{m-2} + d_{m-3} (see the band kernel); x holds d_{m-1}
        g_nodes(e0, e1, M, [&](size_t e, int i, int j) {
          if (i == M - 1 || j == M - 1) w.u[e] = far_field(pf, i * gp.h, j * gp.h, tau_new);
          const float d1 = w.x[e], d2 = w.xp[e];
          if (nhist >= 3) w.x[e] = 3.f * (d1 - d2) + w.xq[e];
          else if (nhist == 2) w.x[e] = 2.f * d1 - d2;
          w.xq[e] = d2;
          w.xp[e] = d1;
        });
        barrier();
        int it = 0;
        // restart from the current iterate after a breakdown (see the band kernel)
        for (int attempt = 0; attempt < kKrylovAttempts; ++attempt) {
          if (attempt > 0) barrier();   // the other CTAs' last x updates are visible
          // b^ = D^{-1} dtau R_h w ;  r = b^ - A^ x (x = previous increment)
          float part[2] = {0.f, 0.f};
          g_pass(w.u, w.x, T0, T1, M, j0, j1, R, [&](size_t e, int i, int j, int ra) {
            float bh = 0.f, rr = 0.f;
            if (i < M - 1 && j < M - 1) {
              float ce, cw, cs, cn, cg;
              g_coefs(d, i, j, ce, cw, cs, cn, cg);
              const float* y = T0 + (j - ra + 1) * S + kTilePad + i;
              const float c = y[0], yw = y[-1], ye = y[1], yn = y[-S], ys = y[S];
              const float ynw = y[-S - 1], yne = y[-S + 1], ysw = y[S - 1], yse = y[S + 1];
              const float b = ce * (ye - c) - cw * (c - yw) + cs * (ys - c) - cn * (c - yn) +
                              cg * ((yse - yne) - (ysw - ynw)) - rdt * c;
              const float id = w.id[e];
              bh = b * id;
              rr = bh - g_tile_matvec(T1, S, ra, i, j, id, ce, cw, cs, cn, cg);
            }
            w.r[e] = rr;
            w.rh[e] = rr;
            part[0] = fmaf(bh, bh, part[0]);
            part[1] = fmaf(rr, rr, part[1]);
          });
          cluster_sum<GCfg, 2>(cluster, part, slots, wpart, sc, round, rank, C,
                               [tol](Scal* s) { KrylovFin::start(s, tol); });
          for (size_t e = e0 + tid; e < e1; e += kGThreads) w.p[e] = w.r[e];
          barrier();
          // Right-preconditioned with M^{-1} = 2I - A^ (see the band kernel): v = A^ M^{-1} p,
          // t = A^ M^{-1} s, x += alpha M^{-1} p + omega M^{-1} s.  Each preconditioner
          // application reads its operand's neighbours, hence one more barrier before the
          // product that reads q.
          while (!sc->conv && it < a.maxit) {
            ++it;
            g_pass(w.p, nullptr, T0, T1, M, j0, j1, R, [&](size_t e, int i, int j, int ra) {
              float qv = 0.f;
              if (i < M - 1 && j < M - 1) {
                float ce, cw, cs, cn, cg;
                g_coefs(d, i, j, ce, cw, cs, cn, cg);
                qv = fmaf(2.f, T0[(j - ra + 1) * S + kTilePad + i],
                          -g_tile_matvec(T0, S, ra, i, j, w.id[e], ce, cw, cs, cn, cg));
              }
              w.q[e] = qv;
            });
            barrier();
            float p1[2] = {0.f, 0.f};
            g_pass(w.q, nullptr, T0, T1, M, j0, j1, R, [&](size_t e, int i, int j, int ra) {
              float vv = 0.f;
              if (i < M - 1 && j < M - 1) {
                float ce, cw, cs, cn, cg;
                g_coefs(d, i, j, ce, cw, cs, cn, cg);
                vv = g_tile_matvec(T0, S, ra, i, j, w.id[e], ce, cw, cs, cn, cg);
              }
              w.v[e] = vv;
              const float rr = w.r[e];
              p1[0] = fmaf(w.rh[e], vv, p1[0]);
              p1[1] = fmaf(rr, rr, p1[1]);
            });
            // every CTA has read its neighbours' q before this reduction's barrier
            cluster_sum<GCfg, 2>(cluster, p1, slots, wpart, sc, round, rank, C, [](Scal* s) { KrylovFin::alpha(s); });
            if (sc->conv || sc->fail) break;
            const float af = sc->af;
            for (size_t e = e0 + tid; e < e1; e += kGThreads) {
              w.x[e] = fmaf(af, w.q[e], w.x[e]);
              w.s[e] = fmaf(-af, w.v[e], w.r[e]);
            }
            barrier();
            g_pass(w.s, nullptr, T0, T1, M, j0, j1, R, [&](size_t e, int i, int j, int ra) {
              float qv = 0.f;
              if (i < M - 1 && j < M - 1) {
                float ce, cw, cs, cn, cg;
                g_coefs(d, i, j, ce, cw, cs, cn, cg);
                qv = fmaf(2.f, T0[(j - ra + 1) * S + kTilePad + i],
                          -g_tile_matvec(T0, S, ra, i, j, w.id[e], ce, cw, cs, cn, cg));
              }
              w.q[e] = qv;
            });
            barrier();
            float p2[4] = {0.f, 0.f, 0.f, 0.f};
            g_pass(w.q, nullptr, T0, T1, M, j0, j1, R, [&](size_t e, int i, int j, int ra) {
              float tt = 0.f;
              if (i < M - 1 && j < M - 1) {
                float ce, cw, cs, cn, cg;
                g_coefs(d, i, j, ce, cw, cs, cn, cg);
                tt = g_tile_matvec(T0, S, ra, i, j, w.id[e], ce, cw, cs, cn, cg);
              }
              w.t[e] = tt;
              const float sv = w.s[e], rh = w.rh[e];
              p2[0] = fmaf(tt, sv, p2[0]);
              p2[1] = fmaf(tt, tt, p2[1]);
              p2[2] = fmaf(rh, sv, p2[2]);
              p2[3] = fmaf(rh, tt, p2[3]);
            });
            cluster_sum<GCfg, 4>(cluster, p2, slots, wpart, sc, round, rank, C, [](Scal* s) { KrylovFin::omega(s); });
            const float of = sc->of, bf = sc->bf;
            for (size_t e = e0 + tid; e < e1; e += kGThreads) {
              const float sv = w.s[e], pv = w.p[e], tt = w.t[e];
              w.x[e] = fmaf(of, w.q[e], w.x[e]);
              const float rr = fmaf(-of, tt, sv);
              w.r[e] = rr;
              w.p[e] = fmaf(bf, fmaf(-of, w.v[e], pv), rr);
            }
            if (sc->fail) break;
            barrier();
          }
          if (sc->conv || !sc->fail) break;
        }
        if (!sc->conv) failed = true;
        iters_max = it > iters_max ? it : iters_max;
        iters_total += it;
        ++nsolves;
        nhist = nhist < 3 ? nhist + 1 : 3;
        for (size_t e = e0 + tid; e < e1; e += kGThreads) w.u[e] += w.x[e];
        barrier();
      }
    }
    if (a.mode == SWEEP_PROP) {
      for (size_t e = e0 + tid; e < e1; e += kGThreads) pit.out[e] = w.u[e];
    } else {
      double nr[2] = {0.0, 0.0};
      float* Un = a.U + (size_t)(n + 1) * MM;
      const float* Fn = a.Fb + (size_t)n * MM;
      float* Gn = a.Gold + (size_t)n * MM;
      for (size_t e = e0 + tid; e < e1; e += kGThreads) {
        const float gnew = w.u[e];
        // squares in FP32 (u_new - u_old of nearby values is exact), sums in FP64
        if (a.mode == SWEEP_INIT) {
          Un[e] = gnew;
          Gn[e] = gnew;
          nr[0] += (double)(gnew * gnew);
        } else {
          const float unew = Fn[e] + (gnew - Gn[e]);
          const float du = unew - Un[e];
          Un[e] = unew;
          Gn[e] = gnew;
          w.u[e] = unew;
          nr[0] += (double)(unew * unew);
          nr[1] += (double)(du * du);
        }
      }
      double* norms = a.norms;
      const int slot_n = n + 1;
      const bool iter = a.mode == SWEEP_ITER;
      cluster_sum<GCfg, 2>(cluster, nr, slots, wpart, sc, round, rank, C, [norms, slot_n, rank, iter](Scal* s) {
        if (rank == 0) { norms[2 * slot_n] = s->tot[0]; norms[2 * slot_n + 1] = iter ? s->tot[1] : 0.0; }
      });
      barrier();
    }
  }
  if (rank == 0 && tid == 0) {
    if (failed) atomicOr(a.status, 1);
    atomicMax(a.status + 1, iters_max);
    atomicAdd(a.status + 2, iters_total);
    atomicAdd(a.status + 3, nsolves);
    if (a.mode == SWEEP_ITER && n_hi == a.N) {
      double num = 0.0, den = 0.0;
      for (int n = 1; n <= a.N; ++n) {
        den = fmax(den, a.norms[2 * n]);
        if (n >= a.n_first + 1) num = fmax(num, a.norms[2 * n + 1]);
      }
      a.defect[0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
    }
  }
}

static cudaLaunchConfig_t global_launch_config(int C, int nst, cudaStream_t s, cudaLaunchAttribute (&attr)[1]) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, nst, 1);
  cfg.blockDim = dim3(kGThreads, 1, 1);
  cfg.dynamicSmemBytes = kGTileBytes;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Cluster size of the global-memory sweep: 16 CTAs where the device can hold such a cluster,
// else 8 (0: neither).
static int global_cluster_ctas(int) {
  if (cudaFuncSetAttribute(sweep_global_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGTileBytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int C : {16, 8}) {
    if (C > 8 &&
        cudaFuncSetAttribute(sweep_global_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = global_launch_config(C, 1, nullptr, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, sweep_global_kernel, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    return C;
  }
  return 0;
}

static int launch_sweep_global(const bs_grid* g, const ItemDesc& d, const SweepArgs& a, cudaStream_t s) {
  const int M = g->M;
  const size_t MM = (size_t)M * M;
  const int nst = a.mode == SWEEP_PROP && a.nprop > 0 ? a.nprop : 1;
  int rc = ensure(const_cast<bs_grid*>(g)->ws_coarse, (size_t)nst * kGlobalVecs * MM * sizeof(float));
  if (rc) return rc;
  GSweepParams gp;
  gp.d = d;
  gp.a = a;
  float* base = (float*)g->ws_coarse.ptr;
  gp.w = GlobalVecs{base,          base + MM,     base + 2 * MM, base + 3 * MM, base + 4 * MM,  base + 5 * MM,
                    base + 6 * MM, base + 7 * MM, base + 8 * MM, base + 9 * MM, base + 10 * MM, base + 11 * MM};
  gp.M = M;
  gp.h = (float)(g->xmax / (M - 1));
  const int C = global_cluster_ctas(M);
  if (C == 0) return set_error(BS_ERR_CUDA, "coarse propagator: no cluster shape available for M=%d", M);
  const int R = g_tile_rows(M, (M + C - 1) / C, kGTileBytes);
  if ((size_t)2 * (R + 2) * g_tile_stride(M) * sizeof(float) > kGTileBytes)
    return set_error(BS_ERR_ARG, "coarse propagator: M=%d exceeds the global solver's tile size", M);
  gp.C = C;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = global_launch_config(C, nst, s, attr);
  BS_CUDA_TRY(cudaLaunchKernelEx(&cfg, sweep_global_kernel, gp));
  return BS_OK;
}

// ---------------------------------------------------------------------------------------
// Band variants of the cluster-resident coarse sweep.  A variant fixes the columns per CTA
// (NCOL >= M), the threads per CTA and the rows per thread; its cluster size follows from M.
// More CTAs per system shorten the arithmetic of each BiCGSTAB iteration but not its cluster
// barriers, so the best variant depends on M and on the machine: coarse_autotune times the
// candidates once per M (a few short PROP solves) and caches the winner for the process, so
// that every solve of that grid size runs the same kernel and reduction order.
// ---------------------------------------------------------------------------------------
struct CoarseVariant {
  int ncol, nt, k;
  bool is_default;   // the shape used when no measurement is available
};
static const CoarseVariant kCoarseVariants[] = {
    {32, 256, 4, true},   {32, 128, 2, false},  {64, 512, 8, true},   {64, 256, 4, false},
    {128, 512, 16, true}, {128, 512, 4, false}, {256, 512, 16, true}, {256, 512, 8, false},
    {256, 256, 16, false}, {128, 256, 8, false}};
constexpr int kNumCoarseVariants = (int)(sizeof(kCoarseVariants) / sizeof(kCoarseVariants[0]));
static_assert(kNumCoarseVariants == 10, "launch_variant and variant_launchable list every variant");

static int variant_ncol(int M) {
  return M <= 32 ? 32 : M <= 64 ? 64 : M <= 128 ? 128 : M <= 256 ? 256 : 0;
}

static BandShape variant_shape(int v, int M) {
  const CoarseVariant& cv = kCoarseVariants[v];
  BandShape sh = {};
  sh.M = M;
  sh.ncol = cv.ncol;
  sh.G = cv.nt / cv.ncol;
  sh.K = cv.k;
  sh.BH = sh.G * sh.K;
  sh.C = (M + sh.BH - 1) / sh.BH;
  return sh;
}

static bool variant_fits(int v, int M) {
  return kCoarseVariants[v].ncol == variant_ncol(M) && variant_shape(v, M).C <= kMaxCluster;
}

static int launch_variant(int v, SweepParams sp, cudaStream_t s) {
  sp.sh = variant_shape(v, sp.sh.M);
  fill_row_coefs(sp);
  switch (v) {
    case 0: return launch_sweep_k<BandCfg<32, 256, 4>>(sp, s);
    case 1: return launch_sweep_k<BandCfg<32, 128, 2>>(sp, s);
    case 2: return launch_sweep_k<BandCfg<64, 512, 8>>(sp, s);
    case 3: return launch_sweep_k<BandCfg<64, 256, 4>>(sp, s);
    case 4: return launch_sweep_k<BandCfg<128, 512, 16>>(sp, s);
    case 5: return launch_sweep_k<BandCfg<128, 512, 4>>(sp, s);
    case 6: return launch_sweep_k<BandCfg<256, 512, 16>>(sp, s);
    case 7: return launch_sweep_k<BandCfg<256, 512, 8>>(sp, s);
    case 8: return launch_sweep_k<BandCfg<256, 256, 16>>(sp, s);
    case 9: return launch_sweep_k<BandCfg<128, 256, 8>>(sp, s);
  }
  return set_error(BS_ERR_ARG, "coarse propagator: no band variant %d", v);
}

// Whether the device can hold one cluster of the variant (clusters above 8 CTAs are
// non-portable and depend on the GPC layout).
template <class CFG>
static bool cluster_fits(const BandShape& sh) {
  const size_t smem = sweep_smem_bytes<CFG>();
  auto kern = sweep_band_kernel<CFG>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (sh.C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return false;
  }
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
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

static bool variant_launchable(int v, int M) {
  if (!variant_fits(v, M)) return false;
  const BandShape sh = variant_shape(v, M);
  switch (v) {
    case 0: return cluster_fits<BandCfg<32, 256, 4>>(sh);
    case 1: return cluster_fits<BandCfg<32, 128, 2>>(sh);
    case 2: return cluster_fits<BandCfg<64, 512, 8>>(sh);
    case 3: return cluster_fits<BandCfg<64, 256, 4>>(sh);
    case 4: return cluster_fits<BandCfg<128, 512, 16>>(sh);
    case 5: return cluster_fits<BandCfg<128, 512, 4>>(sh);
    case 6: return cluster_fits<BandCfg<256, 512, 16>>(sh);
    case 7: return cluster_fits<BandCfg<256, 512, 8>>(sh);
    case 8: return cluster_fits<BandCfg<256, 256, 16>>(sh);
    case 9: return cluster_fits<BandCfg<128, 256, 8>>(sh);
  }
  return false;
}

static int default_variant(int M) {
  for (int v = 0; v < kNumCoarseVariants; ++v)
    if (kCoarseVariants[v].is_default && variant_fits(v, M)) return v;
  return -1;
}

static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_tuned;   // (device, M) -> variant

int coarse_cached_variant(int device, int M) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find({device, M});
  return it != g_tuned.end() ? it->second : default_variant(M);
}

// The variant measured for (device, M) in this process, or -1 if none was measured yet.
int coarse_tuned_variant(int device, int M) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find({device, M});
  return it != g_tuned.end() ? it->second : -1;
}

// Times every launchable variant on a PROP solve of `steps` coarse steps from the payoff
// state of d (best of three after one warm-up) and caches the fastest for (device, M).
int coarse_autotune(bs_grid* g, const ItemDesc& d, cudaStream_t s, int steps, int* chosen) {
  const int M = g->M;
  const size_t MM = (size_t)M * M;
  float* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = default_variant(M);
  float best_ms = 1e30f;
  int rc = BS_OK;
  note_device_alloc();
  if (cudaMalloc(&buf, 2 * MM * sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = cuda_error(cudaGetLastError(), "coarse_autotune");
  }
  if (rc == BS_OK) rc = launch_payoff(g, d, buf, s);
  for (int v = 0; rc == BS_OK && v < kNumCoarseVariants; ++v) {
    if (!variant_launchable(v, M)) continue;
    SweepParams sp;
    sp.d = d;
    sp.d.tau0 = 0.0;
    sp.a = SweepArgs{};
    sp.a.mode = SWEEP_PROP;
    sp.a.N = 1;
    sp.a.csteps = steps;
    sp.a.in = buf;
    sp.a.out = buf + MM;
    sp.a.status = g->status;
    sp.a.tol = g_opt.krylov_tol;
    sp.a.maxit = g_opt.krylov_maxit;
    sp.sh.M = M;
    sp.h = (float)(g->xmax / (M - 1));
    float t_min = 1e30f;
    for (int rep = 0; rc == BS_OK && rep < 4; ++rep) {
      if (cudaEventRecord(e0, s) != cudaSuccess) { rc = cuda_error(cudaGetLastError(), "coarse_autotune"); break; }
      if ((rc = launch_variant(v, sp, s))) break;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "coarse_autotune");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < t_min) t_min = ms;
    }
    if (rc == BS_OK && t_min < best_ms) {
      best_ms = t_min;
      best = v;
    }
  }
  if (buf) cudaFree(buf);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // the tuning solves' iteration counts are not the caller's
  if (rc == BS_OK && cudaMemsetAsync(g->status, 0, kStatusWords * sizeof(int), s) != cudaSuccess)
    rc = cuda_error(cudaGetLastError(), "coarse_autotune");
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[{g->device, M}] = best;
  }
  g->coarse_variant = best;
  if (chosen) *chosen = best;
  return BS_OK;
}

// The band variant the coarse sweep of g runs: forced by the option, else measured once per
// grid size (from the cache while a stream is being captured).
static int resolve_variant(const bs_grid* g, const ItemDesc& d, cudaStream_t s, int* v) {
  bs_grid* gm = const_cast<bs_grid*>(g);
  // one measurement per (device, M) for the whole process: every grid of that size then runs
  // the same kernel and reduction order
  if (g_opt.coarse_variant < 0 && gm->coarse_variant < 0) gm->coarse_variant = coarse_tuned_variant(g->device, g->M);
  if (g_opt.coarse_variant < 0 && gm->coarse_variant < 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
    if (capturing) {
      gm->coarse_variant = coarse_cached_variant(g->device, g->M);
    } else {
      int rc = coarse_autotune(gm, d, s, kAutotuneSteps, nullptr);
      if (rc) return rc;
    }
  }
  *v = g_opt.coarse_variant >= 0 ? g_opt.coarse_variant : gm->coarse_variant;
  if (*v < 0 || *v >= kNumCoarseVariants || !variant_fits(*v, g->M))
    return set_error(BS_ERR_ARG, "coarse propagator: band variant %d does not fit M=%d", *v, g->M);
  return BS_OK;
}

template <class CFG>
static void variant_features(int* poly, int* quad) {
  *poly = SweepSmem<CFG>::POLY2 ? 2 : SweepSmem<CFG>::POLY ? 1 : 0;
  *quad = SweepSmem<CFG>::QUAD ? 1 : 0;
}

int coarse_variant_info(int v, int M, int* ctas, int* threads, int* rows, int* poly, int* quad) {
  if (v < 0 || v >= kNumCoarseVariants || M < 2 || !variant_fits(v, M))
    return set_error(BS_ERR_ARG, "bs_coarse_variant_info: no band variant %d for M=%d", v, M);
  const BandShape sh = variant_shape(v, M);
  int pl = 0, qd = 0;
  switch (v) {
    case 0: variant_features<BandCfg<32, 256, 4>>(&pl, &qd); break;
    case 1: variant_features<BandCfg<32, 128, 2>>(&pl, &qd); break;
    case 2: variant_features<BandCfg<64, 512, 8>>(&pl, &qd); break;
    case 3: variant_features<BandCfg<64, 256, 4>>(&pl, &qd); break;
    case 4: variant_features<BandCfg<128, 512, 16>>(&pl, &qd); break;
    case 5: variant_features<BandCfg<128, 512, 4>>(&pl, &qd); break;
    case 6: variant_features<BandCfg<256, 512, 16>>(&pl, &qd); break;
    case 7: variant_features<BandCfg<256, 512, 8>>(&pl, &qd); break;
    case 8: variant_features<BandCfg<256, 256, 16>>(&pl, &qd); break;
    case 9: variant_features<BandCfg<128, 256, 8>>(&pl, &qd); break;
  }
  if (ctas) *ctas = sh.C;
  if (threads) *threads = kCoarseVariants[v].nt;
  if (rows) *rows = kCoarseVariants[v].k;
  if (poly) *poly = pl;
  if (quad) *quad = qd;
  return BS_OK;
}

int coarse_cluster_ctas(const bs_grid* g, const ItemDesc& d, cudaStream_t s, int* ctas) {
  if (variant_ncol(g->M) == 0) {
    *ctas = global_cluster_ctas(g->M);
    return BS_OK;
  }
  int v = -1;
  int rc = resolve_variant(g, d, s, &v);
  if (rc) return rc;
  *ctas = variant_shape(v, g->M).C;
  return BS_OK;
}

int launch_sweep(const bs_grid* g, const ItemDesc& d, const SweepArgs& a, cudaStream_t s) {
  SweepParams sp;
  sp.d = d;
  sp.a = a;
  sp.sh = g->shape;
  sp.h = (float)(g->xmax / (g->M - 1));
  if (variant_ncol(g->M) == 0) return launch_sweep_global(g, d, a, s);
  int v = -1;
  int rc = resolve_variant(g, d, s, &v);
  if (rc) return rc;
  sp.sh.M = g->M;
  return launch_variant(v, sp, s);
}

}  // namespace bsp
