// Three-asset operator (eq. bse_general with n = 3): the 19-point stencil and far-face
// data shared by the three-asset kernels (fine3.cu, krylov3.cu).  Layout u[(k*M + j)*M + i],
// i the index of asset 1; coefficients are host-rounded FP32 constants times exact integer
// node indices (x_p = i_p h, h cancels).
#pragma once

#include "common.cuh"

namespace bsp {

constexpr int kF3MaxItems = 32;
constexpr int kF3Threads = 256;
constexpr int kF3TileI = 32, kF3TileJ = 8;   // sweep kernel: columns per block
constexpr int kF3PlanesPerBlock = 8;         // sweep kernel: planes of k per thread

struct F3Item {
  const float* in;
  float* out;
  float* hi;   // [M^3] state, high part
  float* lo;   // [M^3] compensation
  float* b;    // [M^3] dtau R_h u of the step
  float* dA;   // [M^3] increment ping-pong
  float* dB;
  float tau0;
};

struct F3Coef {
  float A[3];      // 1/2 sigma_p^2 dtau      (times i_p^2: diffusion weight of +-1 along p)
  float D[3];      // 1/2 r dtau              (times i_p: drift weight, + on +1, - on -1)
  float Cxy, Cxz, Cyz;   // 1/4 rho_pq sigma_p sigma_q dtau (times i_p i_q: cross weight)
  float rdt;       // r dtau
};

struct F3Batch {
  F3Item it[kF3MaxItems];
  int n, M;
  float h;
  F3Coef c;
  int kind;        // BS_PAYOFF_BASKET or BS_PAYOFF_EXCHANGE
  float w[3], K;   // basket: max(w.x - K e^{-r tau}, 0) on the far faces
  PayoffF ex;      // exchange: Margrabe in (x_1, x_2) on the far faces
  float r;
  float dtau;
};

__device__ __forceinline__ void f3_node(int e, int M, int& i, int& j, int& k) {
  const int MM = M * M;
  k = e / MM;
  const int rem = e - k * MM;
  j = rem / M;
  i = rem - j * M;
}

__device__ __forceinline__ float f3_far_field(const F3Batch& fb, int i, int j, int k, float tau) {
  const float x = i * fb.h, y = j * fb.h, z = k * fb.h;
  if (fb.kind == BS_PAYOFF_BASKET)
    return fmaxf(fb.w[0] * x + fb.w[1] * y + fb.w[2] * z - fb.K * expf(-fb.r * tau), 0.0f);
  return far_field(fb.ex, x, y, tau);
}

// Off-diagonal part of dtau R_h applied to y at a PDE node (i, j, k <= M-2): the 18
// neighbours; a neighbour at index -1 has weight 0 and is not read.
__device__ __forceinline__ float f3_offdiag(const float* __restrict__ y, const F3Coef& c, int M, int i, int j,
                                            int k) {
  const int e = (k * M + j) * M + i;
  const int sx = 1, sy = M, sz = M * M;
  const float fi = (float)i, fj = (float)j, fk = (float)k;
  const float ax = c.A[0] * (fi * fi), ay = c.A[1] * (fj * fj), az = c.A[2] * (fk * fk);
  const float mx = c.D[0] * fi, my = c.D[1] * fj, mz = c.D[2] * fk;
  float acc = (ax + mx) * __ldg(y + e + sx) + (ay + my) * __ldg(y + e + sy) + (az + mz) * __ldg(y + e + sz);
  if (i > 0) acc = fmaf(ax - mx, __ldg(y + e - sx), acc);
  if (j > 0) acc = fmaf(ay - my, __ldg(y + e - sy), acc);
  if (k > 0) acc = fmaf(az - mz, __ldg(y + e - sz), acc);
  // cross pairs: +(++ and --) - (+- and -+)
  {
    float s = __ldg(y + e + sx + sy);
    if (i > 0 && j > 0) s += __ldg(y + e - sx - sy);
    if (j > 0) s -= __ldg(y + e + sx - sy);
    if (i > 0) s -= __ldg(y + e - sx + sy);
    acc = fmaf(c.Cxy * (fi * fj), s, acc);
  }
  {
    float s = __ldg(y + e + sx + sz);
    if (i > 0 && k > 0) s += __ldg(y + e - sx - sz);
    if (k > 0) s -= __ldg(y + e + sx - sz);
    if (i > 0) s -= __ldg(y + e - sx + sz);
    acc = fmaf(c.Cxz * (fi * fk), s, acc);
  }
  {
    float s = __ldg(y + e + sy + sz);
    if (j > 0 && k > 0) s += __ldg(y + e - sy - sz);
    if (k > 0) s -= __ldg(y + e + sy - sz);
    if (j > 0) s -= __ldg(y + e - sy + sz);
    acc = fmaf(c.Cyz * (fj * fk), s, acc);
  }
  return acc;
}

__device__ __forceinline__ float f3_diag(const F3Coef& c, int i, int j, int k) {
  const float fi = (float)i, fj = (float)j, fk = (float)k;
  return 1.0f + 2.0f * (c.A[0] * (fi * fi) + c.A[1] * (fj * fj) + c.A[2] * (fk * fk)) + c.rdt;
}

// host helpers (fine3.cu)
int f3_check(int M, double xmax, const bs_params3* p);                 // BS_OK or BS_ERR_ARG
F3Batch f3_batch(int M, double xmax, const bs_params3& p, double dtau);  // coefficients of one step
double f3_contraction(int M, const bs_params3& p, double dtau);         // Gershgorin bound q
enum { F3_INIT = 0, F3_FACE = 1, F3_RHS = 2, F3_APPLY = 3, F3_OUT = 4 };
__global__ void f3_phase_kernel(const __grid_constant__ F3Batch fb, int phase, int step, int cur);
// G over one slice for one state, BiCGSTAB per implicit step (krylov3.cu)
int coarse_propagate3_krylov(int M, double xmax, const bs_params3& p, const float* u_in, float* u_out, double tau0,
                             double dtau, int nsteps, double tol, int maxit, cudaStream_t s);

}  // namespace bsp
