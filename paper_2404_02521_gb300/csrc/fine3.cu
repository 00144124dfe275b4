// F for three assets: eq. (bse_general) with n = 3, discretised like eq. (fd) (second
// differences along each axis, four-point cross differences for each pair, centred first
// differences: a 19-point stencil) and stepped by implicit Euler, for B states at once.
//
// Each step solves (I - dtau R_h) d = dtau R_h u (increment form, far-face Dirichlet data at
// the new time level) by Jacobi sweeps whose count follows from the Gershgorin bound q of the
// system (q < 0.8; the first step from d = 0 to q^m <= 2^-22, later steps from the previous
// increment to q^m <= 2^-10, at least 2), and carries u as a compensated (hi, lo) FP32 pair.
// Stencil coefficients are products of host-rounded FP32 constants and exact integer node
// indices (x_p = i_p h, so h cancels).
//
// One launch of f3_sweep_kernel per Jacobi sweep.  A block owns kF3TileI x kF3TileJ columns
// (i, j) and kF3PlanesPerBlock planes k; it stages the halo tile of the old increment (one
// node on every side, zero outside the grid) in shared memory with asynchronous 4-byte copies
// that are all in flight at once, and loads its columns' own operands (b, and for the last
// sweep hi and lo) into registers before its single barrier.  Each thread then walks its
// column (i, j) up through the block's planes.  The first sweep of a step also stages hi and
// forms b = dtau R_h hi (the RHS phase); the last sweep also adds the increment to (hi, lo)
// (APPLY) and writes the far faces of the next step (FACE).  So a step is its sweeps alone;
// f3_phase_kernel remains only for the INIT and OUT passes of a launch (and the FACE pass
// before the first step).
//
// Layout: u[(k*M + j)*M + i] with i the index of asset 1 (fastest), j of asset 2, k of
// asset 3.  Nodes with an index M - 1 carry Dirichlet data; nodes with an index 0 carry the
// PDE row itself (every coefficient that would reach index -1 is a multiple of that index).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "fine3.cuh"

namespace bsp {

// The pointwise phases of a step (one launch each): INIT copies u_in into (hi, lo = 0) and
// zeroes the increment; FACE writes the far-face data at tau; RHS forms b = dtau R_h hi;
// APPLY adds the increment to (hi, lo); OUT writes hi + lo.
__global__ void __launch_bounds__(kF3Threads) f3_phase_kernel(const __grid_constant__ F3Batch fb, int phase,
                                                              int step, int cur) {
  const F3Item& it = fb.it[blockIdx.y];
  const int M = fb.M, n3 = M * M * M;
  const int e = blockIdx.x * kF3Threads + threadIdx.x;
  if (e >= n3) return;
  int i, j, k;
  f3_node(e, M, i, j, k);
  const bool pde = i < M - 1 && j < M - 1 && k < M - 1;
  float* d = cur ? it.dB : it.dA;
  switch (phase) {
    case F3_INIT:
      it.hi[e] = it.in[e];
      it.lo[e] = 0.f;
      it.dA[e] = 0.f;
      it.dB[e] = 0.f;
      break;
    case F3_FACE:
      if (!pde) {
        it.hi[e] = f3_far_field(fb, i, j, k, it.tau0 + (step + 1) * fb.dtau);
      }
      break;
    case F3_RHS:
      it.b[e] = pde ? f3_offdiag(it.hi, fb.c, M, i, j, k) - (f3_diag(fb.c, i, j, k) - 1.0f) * it.hi[e] : 0.f;
      break;
    case F3_APPLY:
      if (pde) {
        const float h0 = it.hi[e], v = d[e];
        const float s = h0 + v, bb = s - h0;
        const float err = (h0 - (s - bb)) + (v - bb);
        const float l = it.lo[e] + err;
        const float hn = s + l;
        it.lo[e] = l - (hn - s);
        it.hi[e] = hn;
      }
      break;
    case F3_OUT:
      it.out[e] = it.hi[e] + it.lo[e];
      break;
  }
}

// Asynchronous 4-byte global -> shared copy (all of a thread's copies in flight at once);
// with ok == false the destination is zero-filled and nothing is read.
__device__ __forceinline__ void f3_cp_async4(float* dst, const float* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}

// Halo tile of one block: kF3TileI x kF3TileJ columns and kF3PlanesPerBlock planes plus one
// node on every side, i fastest.  Entries outside the grid are 0 (their weights are 0 too).
constexpr int kHI = kF3TileI + 2, kHJ = kF3TileJ + 2, kHK = kF3PlanesPerBlock + 2;
constexpr int kTileFloats = kHI * kHJ * kHK;

// Off-diagonal part of dtau R_h at the node of tile index L (column coefficients precomputed;
// no guards: a neighbour at index -1 is 0 in the tile and has weight 0).
struct F3Col {
  float wxp, wxm, wyp, wym, cxy, cxz, cyz;
};
__device__ __forceinline__ float f3_tile_offdiag(const float* t, int L, const F3Col& w, float az, float mz,
                                                 float fk) {
  constexpr int X = 1, Y = kHI, Z = kHI * kHJ;
  float acc = w.wxp * t[L + X];
  acc = fmaf(w.wxm, t[L - X], acc);
  acc = fmaf(w.wyp, t[L + Y], acc);
  acc = fmaf(w.wym, t[L - Y], acc);
  acc = fmaf(az + mz, t[L + Z], acc);
  acc = fmaf(az - mz, t[L - Z], acc);
  acc = fmaf(w.cxy, (t[L + X + Y] + t[L - X - Y]) - (t[L + X - Y] + t[L - X + Y]), acc);
  acc = fmaf(w.cxz * fk, (t[L + X + Z] + t[L - X - Z]) - (t[L + X - Z] + t[L - X + Z]), acc);
  acc = fmaf(w.cyz * fk, (t[L + Y + Z] + t[L - Y - Z]) - (t[L + Y - Z] + t[L - Y + Z]), acc);
  return acc;
}

// One Jacobi sweep: d_new = (b + offdiag(d_old)) / diag at PDE nodes, 0 elsewhere.  A block
// stages its halo tile of d_old in shared memory (asynchronous copies, coalesced along i),
// then each thread walks its column (i, j) up through the block's planes.  The first sweep of
// a step also stages the state and forms b = dtau R_h hi (RHS); the last one also adds its
// increment to (hi, lo) (APPLY) and writes the far faces of step face_step (FACE; -1: none).
// A step has at least two sweeps, so no launch both reads the state's neighbours and writes
// the state.
enum { F3S_FIRST = 1, F3S_LAST = 2 };
template <int FLAGS>
__global__ void __launch_bounds__(kF3TileI * kF3TileJ, 4) f3_sweep_kernel(const __grid_constant__ F3Batch fb,
                                                                         int cur, int tiles_i, int face_step) {
  constexpr bool first = FLAGS & F3S_FIRST, last = FLAGS & F3S_LAST;
  __shared__ float sd[kTileFloats];
  __shared__ float sh[first ? kTileFloats : 1];
  const F3Item& it = fb.it[blockIdx.z];
  const int M = fb.M;
  const int tj = blockIdx.x / tiles_i;   // uniform per block
  const int i0 = (blockIdx.x - tj * tiles_i) * kF3TileI, j0 = tj * kF3TileJ;
  const int k0 = blockIdx.y * kF3PlanesPerBlock;
  const float* __restrict__ din = cur ? it.dB : it.dA;
  float* __restrict__ dout = cur ? it.dA : it.dB;
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const int col = j * M + i, sz = M * M;
  const bool active = i < M && j < M, pdecol = i < M - 1 && j < M - 1;
  // the column's own operands for every plane, loaded with the tile (no load waits per plane)
  float bq[kF3PlanesPerBlock], hq[last ? kF3PlanesPerBlock : 1], lq[last ? kF3PlanesPerBlock : 1];
#pragma unroll
  for (int kk = 0; kk < kF3PlanesPerBlock; ++kk) {
    const int k = k0 + kk, e = k * sz + col;
    const bool pde = pdecol && k < M - 1;
    if (!first) bq[kk] = pde ? __ldg(it.b + e) : 0.f;
    if (last) {
      hq[kk] = pde ? it.hi[e] : 0.f;
      lq[kk] = pde ? it.lo[e] : 0.f;
    }
  }
  for (int q = threadIdx.y * kF3TileI + threadIdx.x; q < kTileFloats; q += kF3TileI * kF3TileJ) {
    const int ck = q / (kHI * kHJ);
    const int rem = q - ck * (kHI * kHJ);
    const int bj = rem / kHI;
    const int gi = i0 - 1 + (rem - bj * kHI), gj = j0 - 1 + bj, gk = k0 - 1 + ck;
    const bool in = gi >= 0 && gi < M && gj >= 0 && gj < M && gk >= 0 && gk < M;
    const int ge = in ? (gk * M + gj) * M + gi : 0;
    f3_cp_async4(sd + q, din + ge, in);
    if (first) f3_cp_async4(sh + q, it.hi + ge, in);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();   // the only barrier: threads outside the grid leave after it
  if (!active) return;
  const int k1 = min(k0 + kF3PlanesPerBlock, M);
  const bool face = last && face_step >= 0;
  const float tau_face = it.tau0 + (face_step + 1) * fb.dtau;
  if (!pdecol) {   // far-face column: no unknowns
    for (int k = k0; k < k1; ++k) {
      dout[k * sz + col] = 0.f;
      if (face) it.hi[k * sz + col] = f3_far_field(fb, i, j, k, tau_face);
    }
    return;
  }
  const F3Coef& c = fb.c;
  const float fi = (float)i, fj = (float)j;
  const float ax = c.A[0] * (fi * fi), ay = c.A[1] * (fj * fj);
  const float mx = c.D[0] * fi, my = c.D[1] * fj;
  const F3Col w = {ax + mx, ax - mx, ay + my, ay - my, c.Cxy * (fi * fj), c.Cxz * fi, c.Cyz * fj};
  const float dxy = 1.0f + 2.0f * (ax + ay) + c.rdt;
  const int L0 = (1 * kHJ + threadIdx.y + 1) * kHI + threadIdx.x + 1;   // tile index of plane k0
#pragma unroll
  for (int kk = 0; kk < kF3PlanesPerBlock; ++kk) {
    const int k = k0 + kk;
    if (k >= k1) break;
    const int e = k * sz + col;
    if (k == M - 1) {
      dout[e] = 0.f;   // far face
      if (face) it.hi[e] = f3_far_field(fb, i, j, k, tau_face);
      break;
    }
    const int L = L0 + kk * (kHI * kHJ);
    const float fk = (float)k;
    const float az = c.A[2] * (fk * fk), mz = c.D[2] * fk;
    const float diag = dxy + 2.0f * az;
    float bv;
    if (first) {   // RHS: b = offdiag(hi) - (diag - 1) hi
      bv = f3_tile_offdiag(sh, L, w, az, mz, fk) - (diag - 1.0f) * sh[L];
      it.b[e] = bv;
    } else {
      bv = bq[kk];
    }
    const float dn = (bv + f3_tile_offdiag(sd, L, w, az, mz, fk)) / diag;
    dout[e] = dn;
    if (last) {   // APPLY: compensated add of the increment
      const float h0 = hq[kk];
      const float sm = h0 + dn, bb = sm - h0;
      const float err = (h0 - (sm - bb)) + (dn - bb);
      const float l = lq[kk] + err;
      const float hn = sm + l;
      it.lo[e] = l - (hn - sm);
      it.hi[e] = hn;
    }
  }
}

// Gershgorin bound of I - dtau R_h over the PDE nodes: max of sum |off-diagonal| / diagonal.
static double f3_contraction_scan(int M, const bs_params3& p, double dtau) {
  double q = 0.0;
  const double rho[3][3] = {{1.0, p.rho[0], p.rho[1]}, {p.rho[0], 1.0, p.rho[2]}, {p.rho[1], p.rho[2], 1.0}};
  for (int k = 0; k <= M - 2; ++k)
    for (int j = 0; j <= M - 2; ++j)
      for (int i = 0; i <= M - 2; ++i) {
        const int id[3] = {i, j, k};
        double off = 0.0, diag = 1.0 + dtau * p.r;
        for (int a = 0; a < 3; ++a) {
          const double dif = 0.5 * p.sigma[a] * p.sigma[a] * id[a] * id[a], drift = 0.5 * p.r * id[a];
          off += std::fabs(dif + drift) + std::fabs(dif - drift);
          diag += dtau * 2.0 * dif;
        }
        for (int a = 0; a < 3; ++a)
          for (int b = a + 1; b < 3; ++b)
            off += 4.0 * std::fabs(0.25 * rho[a][b] * p.sigma[a] * p.sigma[b]) * id[a] * id[b];
        q = std::fmax(q, dtau * off / diag);
      }
  return q;
}

// The scan visits (M-1)^3 nodes (milliseconds at 128^3), and parareal_solve3 asks for the same
// bound on every F call: the last few results are kept per (M, parameters, dtau).
double f3_contraction(int M, const bs_params3& p, double dtau) {
  struct Entry {
    double key[9];
    double q;
  };
  static std::mutex mu;
  static Entry cache[8];
  static int used = 0, next = 0;
  const double key[9] = {(double)M, p.sigma[0], p.sigma[1], p.sigma[2], p.rho[0], p.rho[1], p.rho[2], p.r, dtau};
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int e = 0; e < used; ++e)
      if (std::memcmp(cache[e].key, key, sizeof(key)) == 0) return cache[e].q;
  }
  const double q = f3_contraction_scan(M, p, dtau);
  std::lock_guard<std::mutex> lock(mu);
  std::memcpy(cache[next].key, key, sizeof(key));
  cache[next].q = q;
  next = (next + 1) % 8;
  used = used < 8 ? used + 1 : 8;
  return q;
}

static int f3_sweeps(double q, bool cold) {
  const double target = cold ? 1.0 / 4194304.0 : 1.0 / 1024.0;
  if (q <= 0.0) return 2;
  const int m = (int)std::ceil(std::log(target) / std::log(q));
  return m < 2 ? 2 : m;
}

int f3_check(int M, double xmax, const bs_params3* p) {
  if (!p) return set_error(BS_ERR_ARG, "params3 is NULL");
  if (M < 4 || M > 128) return set_error(BS_ERR_ARG, "three-asset grid: M=%d out of [4, 128]", M);
  if (!(xmax > 0.0)) return set_error(BS_ERR_ARG, "three-asset grid: xmax must be > 0");
  for (int a = 0; a < 3; ++a) {
    if (!(p->sigma[a] > 0.0)) return set_error(BS_ERR_ARG, "sigma must be > 0");
    if (!(std::fabs(p->rho[a]) < 1.0)) return set_error(BS_ERR_ARG, "|rho| must be < 1");
  }
  // the correlation matrix must be positive definite (its determinant, the 2x2 minors are
  // positive already)
  const double r12 = p->rho[0], r13 = p->rho[1], r23 = p->rho[2];
  if (!(1.0 - r12 * r12 - r13 * r13 - r23 * r23 + 2.0 * r12 * r13 * r23 > 0.0))
    return set_error(BS_ERR_ARG, "the correlation matrix is not positive definite");
  if (!(p->r >= 0.0)) return set_error(BS_ERR_ARG, "r must be >= 0");
  if (p->payoff != BS_PAYOFF_BASKET && p->payoff != BS_PAYOFF_EXCHANGE)
    return set_error(BS_ERR_ARG, "three-asset payoff must be BS_PAYOFF_BASKET or BS_PAYOFF_EXCHANGE");
  if (p->reserved != 0) return set_error(BS_ERR_ARG, "bs_params3.reserved must be 0");
  return BS_OK;
}

F3Batch f3_batch(int M, double xmax, const bs_params3& p, double dtau) {
  F3Batch fb = {};
  fb.M = M;
  fb.h = (float)(xmax / (M - 1));
  for (int a = 0; a < 3; ++a) {
    fb.c.A[a] = (float)(0.5 * p.sigma[a] * p.sigma[a] * dtau);
    fb.c.D[a] = (float)(0.5 * p.r * dtau);
    fb.w[a] = (float)p.w[a];
  }
  fb.c.Cxy = (float)(0.25 * p.rho[0] * p.sigma[0] * p.sigma[1] * dtau);
  fb.c.Cxz = (float)(0.25 * p.rho[1] * p.sigma[0] * p.sigma[2] * dtau);
  fb.c.Cyz = (float)(0.25 * p.rho[2] * p.sigma[1] * p.sigma[2] * dtau);
  fb.c.rdt = (float)(p.r * dtau);
  fb.kind = p.payoff;
  fb.K = (float)p.strike;
  fb.r = (float)p.r;
  fb.dtau = (float)dtau;
  fb.ex = PayoffF{};
  fb.ex.kind = BS_PAYOFF_EXCHANGE;
  fb.ex.s1 = (float)p.sigma[0];
  fb.ex.s2 = (float)p.sigma[1];
  fb.ex.rho = (float)p.rho[0];
  fb.ex.r = (float)p.r;
  return fb;
}

__global__ void f3_payoff_kernel(float* u, int M, float h, int kind, float w0, float w1, float w2, float K) {
  const int n3 = M * M * M;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n3) return;
  int i, j, k;
  f3_node(e, M, i, j, k);
  const float x = i * h, y = j * h, z = k * h;
  u[e] = kind == BS_PAYOFF_BASKET ? fmaxf(w0 * x + w1 * y + w2 * z - K, 0.f) : fmaxf(x - y, 0.f);
}

}  // namespace bsp

using namespace bsp;

extern "C" {

int bs_payoff3(int M, double xmax, const bs_params3* p, float* u, bs_stream stream) {
  int rc = f3_check(M, xmax, p);
  if (rc) return rc;
  if (!u) return set_error(BS_ERR_ARG, "bs_payoff3: NULL state");
  const int n3 = M * M * M;
  f3_payoff_kernel<<<(n3 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      u, M, (float)(xmax / (M - 1)), p->payoff, (float)p->w[0], (float)p->w[1], (float)p->w[2], (float)p->strike);
  BS_CUDA_TRY(cudaGetLastError());
  return BS_OK;
}

int fine_propagate3(int M, double xmax, const bs_params3* p, const float* const* u_in, float* const* u_out,
                    const double* tau0, int B, double dtau, int nsteps, bs_stream stream) {
  int rc = f3_check(M, xmax, p);
  if (rc) return rc;
  if (!u_in || !u_out || !tau0) return set_error(BS_ERR_ARG, "fine_propagate3: NULL argument");
  if (B < 1 || nsteps < 0) return set_error(BS_ERR_ARG, "fine_propagate3: B=%d nsteps=%d", B, nsteps);
  if (!(dtau > 0.0)) return set_error(BS_ERR_ARG, "fine_propagate3: dtau <= 0");
  for (int b = 0; b < B; ++b)
    if (!u_in[b] || !u_out[b]) return set_error(BS_ERR_ARG, "fine_propagate3: NULL state %d", b);
  const double q = f3_contraction(M, *p, dtau);
  if (!(q < 0.8))
    return set_error(BS_ERR_ARG, "fine_propagate3: Jacobi bound %.3f >= 0.8 (take smaller steps)", q);
  const int m0 = f3_sweeps(q, true), m1 = f3_sweeps(q, false);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n3 = (size_t)M * M * M;
  const unsigned blocks = (unsigned)((n3 + kF3Threads - 1) / kF3Threads);
  for (int base = 0; base < B; base += kF3MaxItems) {
    const int nb = B - base < kF3MaxItems ? B - base : kF3MaxItems;
    float* ws = nullptr;
    note_device_alloc();
    BS_CUDA_TRY(cudaMallocAsync((void**)&ws, (size_t)nb * 5 * n3 * sizeof(float), s));
    F3Batch fb = f3_batch(M, xmax, *p, dtau);
    fb.n = nb;
    for (int t = 0; t < nb; ++t) {
      F3Item& it = fb.it[t];
      float* w = ws + (size_t)t * 5 * n3;
      it.in = u_in[base + t];
      it.out = u_out[base + t];
      it.hi = w;
      it.lo = w + n3;
      it.b = w + 2 * n3;
      it.dA = w + 3 * n3;
      it.dB = w + 4 * n3;
      it.tau0 = (float)tau0[base + t];
    }
    const dim3 grid(blocks, nb);
    const int tiles_i = (M + kF3TileI - 1) / kF3TileI, tiles_j = (M + kF3TileJ - 1) / kF3TileJ;
    const dim3 sgrid((unsigned)(tiles_i * tiles_j), (unsigned)((M + kF3PlanesPerBlock - 1) / kF3PlanesPerBlock),
                     (unsigned)nb);
    const dim3 sblock(kF3TileI, kF3TileJ);
    f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_INIT, 0, 0);
    if (nsteps > 0) f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_FACE, 0, 0);
    int cur = 0;   // 0: the increment is in dA
    for (int step = 0; step < nsteps; ++step) {
      const int m = step == 0 ? m0 : m1;   // >= 2
      for (int sw = 0; sw < m; ++sw) {
        const int face_step = step + 1 < nsteps ? step + 1 : -1;
        if (sw == 0)
          f3_sweep_kernel<F3S_FIRST><<<sgrid, sblock, 0, s>>>(fb, cur, tiles_i, face_step);
        else if (sw == m - 1)
          f3_sweep_kernel<F3S_LAST><<<sgrid, sblock, 0, s>>>(fb, cur, tiles_i, face_step);
        else
          f3_sweep_kernel<0><<<sgrid, sblock, 0, s>>>(fb, cur, tiles_i, face_step);
        cur ^= 1;
      }
    }
    f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_OUT, nsteps, cur);
    BS_CUDA_TRY(cudaGetLastError());
    BS_CUDA_TRY(cudaFreeAsync(ws, s));
  }
  return BS_OK;
}

}  // extern "C"
