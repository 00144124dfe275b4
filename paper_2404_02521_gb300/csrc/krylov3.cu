// Numerical coarse model G for three assets (Sec. 3.2 with n = 3): implicit-Euler steps whose
// systems are too stiff for Jacobi, solved by BiCGSTAB (van der Vorst 1992) on the
// Jacobi-scaled increment system D^{-1}(I - dtau R_h) d = D^{-1} dtau R_h u in FP32, one state.
// The iteration is driven from the host: each BiCGSTAB iteration is a short chain of kernels
// (products with the 19-point stencil, vector updates, block partial sums) and one-block
// kernels that add the partials in a fixed order and update the scalars in device memory;
// the host reads the convergence flag once per kK3Batch iterations: once the device sets
// conv or fail, the kernels of the iterations still queued return at once.  Each step starts
// from the previous step's increment; a breakdown restarts from the current iterate.
#include <algorithm>
#include <cmath>

#include "fine3.cuh"

namespace bsp {

constexpr int kK3Threads = 256;
constexpr int kK3Attempts = 3;
constexpr int kK3Batch = 4;   // iterations queued per host check

struct K3Vecs {
  float *x, *r, *rh, *p, *v, *s, *t, *id, *b;   // x is the F3 item's increment buffer dA
};

struct K3Scal {
  float rho, alpha, omega, beta, stop2;
  int conv, fail, zero;   // zero: b^ vanishes, the solution is d = 0
  int pending;            // omega or rho vanished: finish this iteration, then stop
};

// block partial sums of up to 4 values: warp butterfly, then warp 0 over the warp sums
__device__ __forceinline__ void k3_partials(float (&v)[4], int nv, float* out) {
  __shared__ float ws[kK3Threads / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < nv; ++q) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    if (lane == 0) ws[warp][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < nv; ++q) {
      float a = 0.f;
      for (int w = 0; w < kK3Threads / 32; ++w) a += ws[w][q];
      out[4 * blockIdx.x + q] = a;
    }
  }
}

// A^ y = y - invd * offdiag(y) at a PDE node
__device__ __forceinline__ float k3_scaled(const float* y, const F3Coef& c, int M, int i, int j, int k, int e,
                                           float invd) {
  return y[e] - invd * f3_offdiag(y, c, M, i, j, k);
}

enum { K3_INIT = 0, K3_V = 1, K3_S = 2, K3_T = 3, K3_UPDATE = 4 };

// The vector phases of an iteration.  INIT: invd, b^ = invd b, r = r^ = p = b^ - A^ x with
// partials (b^, b^), (r, r).  V: v = A^ p, partial (r^, v).  S: s = r - alpha v.  T: t = A^ s,
// partials (t, s), (t, t), (r^, s), (r^, t).  UPDATE: x += alpha p + omega s, r = s - omega t,
// p = r + beta (p - omega v), partial (r, r).
__global__ void __launch_bounds__(kK3Threads) k3_phase_kernel(const __grid_constant__ F3Batch fb, K3Vecs w,
                                                              const K3Scal* sc, int phase, float* partials) {
  if (phase != K3_INIT && (sc->conv || sc->fail)) return;   // uniform: the iteration is over
  const int M = fb.M, n3 = M * M * M;
  const int e = blockIdx.x * kK3Threads + threadIdx.x;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (e < n3) {
    int i, j, k;
    f3_node(e, M, i, j, k);
    const bool pde = i < M - 1 && j < M - 1 && k < M - 1;
    switch (phase) {
      case K3_INIT: {
        const float invd = pde ? 1.0f / f3_diag(fb.c, i, j, k) : 0.f;
        w.id[e] = invd;
        const float bh = invd * w.b[e];
        const float r = pde ? bh - k3_scaled(w.x, fb.c, M, i, j, k, e, invd) : 0.f;
        w.r[e] = r;
        w.rh[e] = r;
        w.p[e] = r;
        acc[0] = bh * bh;
        acc[1] = r * r;
        break;
      }
      case K3_V: {
        const float v = pde ? k3_scaled(w.p, fb.c, M, i, j, k, e, w.id[e]) : 0.f;
        w.v[e] = v;
        acc[0] = w.rh[e] * v;
        break;
      }
      case K3_S:
        w.s[e] = fmaf(-sc->alpha, w.v[e], w.r[e]);
        break;
      case K3_T: {
        const float t = pde ? k3_scaled(w.s, fb.c, M, i, j, k, e, w.id[e]) : 0.f;
        const float s = w.s[e], rh = w.rh[e];
        w.t[e] = t;
        acc[0] = t * s;
        acc[1] = t * t;
        acc[2] = rh * s;
        acc[3] = rh * t;
        break;
      }
      case K3_UPDATE: {
        const float a = sc->alpha, o = sc->omega, be = sc->beta;
        const float s = w.s[e], pv = w.p[e];
        w.x[e] += a * pv + o * s;
        const float r = fmaf(-o, w.t[e], s);
        w.r[e] = r;
        w.p[e] = fmaf(be, fmaf(-o, w.v[e], pv), r);
        acc[0] = r * r;
        break;
      }
    }
  }
  if (phase == K3_S) return;
  k3_partials(acc, 4, partials);
}

enum { K3F_START = 0, K3F_ALPHA = 1, K3F_OMEGA = 2, K3F_CONV = 3 };

// One thread adds the block partials in block order and updates the scalars.
__global__ void k3_finish_kernel(const float* partials, int nblocks, K3Scal* sc, int mode, float tol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (mode != K3F_START && (sc->conv || sc->fail)) return;
  float t[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < 4; ++q) t[q] += partials[4 * b + q];
  switch (mode) {
    case K3F_START:
      sc->rho = t[1];
      sc->stop2 = tol * tol * t[0];
      sc->zero = !(t[0] > 1e-30f) ? 1 : 0;
      sc->conv = (t[1] <= sc->stop2 || sc->zero) ? 1 : 0;
      sc->fail = 0;
      sc->pending = 0;
      break;
    case K3F_ALPHA:
      if (t[0] == 0.f) { sc->fail = 1; sc->alpha = 0.f; break; }
      sc->alpha = sc->rho / t[0];
      break;
    case K3F_OMEGA: {
      const float om = t[1] > 0.f ? t[0] / t[1] : 0.f;
      const float rho_new = t[2] - om * t[3];
      sc->omega = om;
      if (om == 0.f || sc->rho == 0.f) { sc->pending = 1; sc->beta = 0.f; break; }
      sc->beta = (rho_new / sc->rho) * (sc->alpha / om);
      sc->rho = rho_new;
      break;
    }
    case K3F_CONV:
      sc->conv = t[0] <= sc->stop2 ? 1 : 0;
      if (sc->pending) sc->fail = 1;
      break;
  }
}

// G over one slice for one state: nsteps implicit steps of size dtau from tau0, each solved by
// BiCGSTAB to relative residual tol (at most maxit iterations per attempt).
int coarse_propagate3_krylov(int M, double xmax, const bs_params3& p, const float* u_in, float* u_out, double tau0,
                             double dtau, int nsteps, double tol, int maxit, cudaStream_t s) {
  const size_t n3 = (size_t)M * M * M;
  const int nblocks = (int)((n3 + kK3Threads - 1) / kK3Threads);
  float* ws = nullptr;
  const size_t fl = 12 * n3 + (size_t)4 * nblocks;
  note_device_alloc();
  BS_CUDA_TRY(cudaMallocAsync((void**)&ws, fl * sizeof(float) + sizeof(K3Scal), s));
  F3Batch fb = f3_batch(M, xmax, p, dtau);
  fb.n = 1;
  F3Item& it = fb.it[0];
  it.in = u_in;
  it.out = u_out;
  it.hi = ws;
  it.lo = ws + n3;
  it.b = ws + 2 * n3;
  it.dA = ws + 3 * n3;
  it.dB = ws + 4 * n3;
  it.tau0 = (float)tau0;
  K3Vecs w;
  w.x = it.dA;
  w.b = it.b;
  w.r = ws + 5 * n3;
  w.rh = ws + 6 * n3;
  w.p = ws + 7 * n3;
  w.v = ws + 8 * n3;
  w.s = ws + 9 * n3;
  w.t = ws + 10 * n3;
  w.id = ws + 11 * n3;
  float* partials = ws + 12 * n3;
  K3Scal* dsc = reinterpret_cast<K3Scal*>(ws + fl);
  const dim3 grid((unsigned)nblocks, 1);
  int rc = BS_OK;
  auto finish = [&](int mode) { k3_finish_kernel<<<1, 32, 0, s>>>(partials, nblocks, dsc, mode, (float)tol); };
  f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_INIT, 0, 0);
  for (int step = 0; step < nsteps && rc == BS_OK; ++step) {
    f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_FACE, step, 0);
    f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_RHS, step, 0);
    bool conv = false;
    for (int attempt = 0; attempt < kK3Attempts && !conv && rc == BS_OK; ++attempt) {
      k3_phase_kernel<<<grid, kK3Threads, 0, s>>>(fb, w, dsc, K3_INIT, partials);
      finish(K3F_START);
      K3Scal h = {};
      for (int itn = 0; itn <= maxit;) {
        if (cudaMemcpyAsync(&h, dsc, sizeof(K3Scal), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          rc = cuda_error(cudaGetLastError(), "three-asset coarse BiCGSTAB");
          break;
        }
        if (h.conv) {
          conv = true;
          if (h.zero && cudaMemsetAsync(w.x, 0, n3 * sizeof(float), s) != cudaSuccess)
            rc = cuda_error(cudaGetLastError(), "three-asset coarse BiCGSTAB");
          break;
        }
        if (h.fail || itn == maxit) break;
        const int nb = std::min(kK3Batch, maxit - itn);
        for (int b = 0; b < nb; ++b) {
          k3_phase_kernel<<<grid, kK3Threads, 0, s>>>(fb, w, dsc, K3_V, partials);
          finish(K3F_ALPHA);
          k3_phase_kernel<<<grid, kK3Threads, 0, s>>>(fb, w, dsc, K3_S, partials);
          k3_phase_kernel<<<grid, kK3Threads, 0, s>>>(fb, w, dsc, K3_T, partials);
          finish(K3F_OMEGA);
          k3_phase_kernel<<<grid, kK3Threads, 0, s>>>(fb, w, dsc, K3_UPDATE, partials);
          finish(K3F_CONV);
        }
        itn += nb;
      }
      if (rc == BS_OK && !conv && !h.fail) break;   // the iteration cap, not a breakdown
    }
    if (rc == BS_OK && !conv)
      rc = set_error(BS_ERR_NOCONV, "three-asset coarse BiCGSTAB: no convergence within %d iterations", maxit);
    if (rc == BS_OK) f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_APPLY, step, 0);
  }
  if (rc == BS_OK) f3_phase_kernel<<<grid, kF3Threads, 0, s>>>(fb, F3_OUT, nsteps, 0);
  if (rc == BS_OK) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_error(e, "three-asset coarse BiCGSTAB");
  }
  cudaFreeAsync(ws, s);
  return rc;
}

}  // namespace bsp

using namespace bsp;

extern "C" int coarse_propagate3(int M, double xmax, const bs_params3* p, const float* u_in, float* u_out,
                                 double tau0, double dtau_slice, int nsteps, bs_stream stream) {
  int rc = f3_check(M, xmax, p);
  if (rc) return rc;
  if (!u_in || !u_out) return set_error(BS_ERR_ARG, "coarse_propagate3: NULL state");
  if (!(dtau_slice > 0.0) || nsteps < 1)
    return set_error(BS_ERR_ARG, "coarse_propagate3: dtau_slice=%g nsteps=%d", dtau_slice, nsteps);
  return coarse_propagate3_krylov(M, xmax, *p, u_in, u_out, tau0, dtau_slice / nsteps, nsteps, g_opt.krylov_tol,
                                  g_opt.krylov_maxit, (cudaStream_t)stream);
}
