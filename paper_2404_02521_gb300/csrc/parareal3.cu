// Parareal (eq. parareal) for three assets: F is the Jacobi-stepped three-asset propagator of
// fine3.cu, G the same implicit scheme with fewer, larger steps solved by BiCGSTAB
// (krylov3.cu; the numerical coarse model of Sec. 3.2 for n = 3).  The iteration runs from
// the host: F on slices k..N-1 in one batched call, then the serial sweep
// n = k..N-1 of G, the correction u_{n+1} = F_n + (G_new - G_old_n) and the FP64 defect
// norms (reading c5), with G skipped on the exact slice n = k (G_old_k is unchanged).
#include <cmath>
#include <vector>

#include "fine3.cuh"

namespace bsp {

constexpr int kP3Threads = 256;
constexpr int kP3Blocks = 304;   // 2 per SM: the correction kernel's grid (grid-stride)

// mode 0: u_{n+1} = G_old = G_new (the initial sweep); mode 1: the correction.  FP32 squares
// per thread (u_new - u_old of nearby values is exact), FP64 partials per block.
__global__ void __launch_bounds__(kP3Threads) p3_correct_kernel(int mode, size_t n3, float* __restrict__ Unext,
                                                                const float* __restrict__ Fn,
                                                                const float* __restrict__ Gnew,
                                                                float* __restrict__ Gold, double* partials) {
  float s0 = 0.f, s1 = 0.f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n3; e += (size_t)gridDim.x * blockDim.x) {
    const float g = Gnew[e];
    if (mode == 0) {
      Unext[e] = g;
      Gold[e] = g;
      s0 = fmaf(g, g, s0);
    } else {
      const float unew = Fn[e] + (g - Gold[e]);
      const float du = unew - Unext[e];
      Unext[e] = unew;
      Gold[e] = g;
      s0 = fmaf(unew, unew, s0);
      s1 = fmaf(du, du, s1);
    }
  }
  double n0 = s0, n1 = s1;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n0 += __shfl_xor_sync(0xffffffffu, n0, off);
    n1 += __shfl_xor_sync(0xffffffffu, n1, off);
  }
  __shared__ double r0[kP3Threads / 32], r1[kP3Threads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { r0[warp] = n0; r1[warp] = n1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kP3Threads / 32; ++w) { a += r0[w]; b += r1[w]; }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// norms[2 n] = ||u_n||^2, norms[2 n + 1] = ||du_n||^2 from the block partials (fixed order).
__global__ void p3_sum_kernel(const double* partials, int nblocks, double* norms) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblocks; ++i) { a += partials[2 * i]; b += partials[2 * i + 1]; }
  norms[0] = a;
  norms[1] = b;
}

}  // namespace bsp

using namespace bsp;

extern "C" int parareal_solve3(int M, double xmax, const bs_params3* p, double T, int N, int fine_steps,
                               int coarse_steps, double tol, int Kmax, float* u_out, int* k_done,
                               double* defect_hist, bs_stream stream) {
  if (!p || !u_out || !k_done) return set_error(BS_ERR_ARG, "parareal_solve3: NULL argument");
  if (!(T > 0.0) || N < 1 || fine_steps < 1 || coarse_steps < 1 || Kmax < 0 || Kmax > N)
    return set_error(BS_ERR_ARG, "parareal_solve3: T=%g N=%d fine_steps=%d coarse_steps=%d Kmax=%d", T, N,
                     fine_steps, coarse_steps, Kmax);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n3 = (size_t)M * M * M;
  const double slice = T / N;
  const double dtf = slice / fine_steps, dtg = slice / coarse_steps;
  int rc = bs_payoff3(M, xmax, p, u_out, stream);   // also checks M, xmax and p
  if (rc) return rc;
  // workspace: F[N], G_old[N], G_new, then FP64 block partials [N + 1][blocks][2] and norms
  const int nblocks = (int)std::min<size_t>((n3 + kP3Threads - 1) / kP3Threads, kP3Blocks);
  const size_t fbytes = ((2 * (size_t)N + 1) * n3 * sizeof(float) + 255) / 256 * 256;
  unsigned char* ws = nullptr;
  note_device_alloc();
  BS_CUDA_TRY(cudaMallocAsync((void**)&ws, fbytes + (size_t)nblocks * 2 * sizeof(double) +
                                               (size_t)(N + 1) * 2 * sizeof(double), s));
  float* Fb = reinterpret_cast<float*>(ws);
  float* Gold = Fb + (size_t)N * n3;
  float* Gnew = Gold + (size_t)N * n3;
  double* partials = reinterpret_cast<double*>(ws + fbytes);
  double* norms = partials + (size_t)nblocks * 2;
  std::vector<double> hnorms(2 * (size_t)(N + 1), 0.0);
  auto U = [&](int n) { return u_out + (size_t)n * n3; };
  auto G = [&](int n, float* out) -> int {   // G(u_n) over slice n: BiCGSTAB per coarse step
    return coarse_propagate3_krylov(M, xmax, *p, U(n), out, n * slice, dtg, coarse_steps, g_opt.krylov_tol,
                                    g_opt.krylov_maxit, s);
  };
  auto correct = [&](int mode, int n) -> int {
    p3_correct_kernel<<<nblocks, kP3Threads, 0, s>>>(mode, n3, U(n + 1), Fb + (size_t)n * n3, Gnew,
                                                     Gold + (size_t)n * n3, partials);
    p3_sum_kernel<<<1, 32, 0, s>>>(partials, nblocks, norms + 2 * (size_t)(n + 1));
    BS_CUDA_TRY(cudaGetLastError());
    return BS_OK;
  };
  auto fail = [&](int code) {
    cudaFreeAsync(ws, s);
    return code;
  };
  // initial sweep: u_{n+1} = G(u_n)
  for (int n = 0; n < N; ++n) {
    if ((rc = G(n, Gnew)) || (rc = correct(0, n))) return fail(rc);
  }
  int k = 0;
  bool converged = false;
  std::vector<const float*> fin((size_t)N);
  std::vector<float*> fout((size_t)N);
  std::vector<double> ft0((size_t)N);
  for (; k < Kmax; ++k) {
    const int B = N - k;   // slices below k are exact
    for (int n = k; n < N; ++n) {
      fin[n - k] = U(n);
      fout[n - k] = Fb + (size_t)n * n3;
      ft0[n - k] = n * slice;
    }
    if ((rc = fine_propagate3(M, xmax, p, fin.data(), fout.data(), ft0.data(), B, dtf, fine_steps, stream)))
      return fail(rc);
    for (int n = k; n < N; ++n) {
      if (n == k) {
        // G of the exact slice is unchanged: G_new = G_old_k, so u_{k+1} = F_k exactly
        if (cudaMemcpyAsync(Gnew, Gold + (size_t)n * n3, n3 * sizeof(float), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
          return fail(cuda_error(cudaGetLastError(), "parareal_solve3"));
      } else if ((rc = G(n, Gnew))) {
        return fail(rc);
      }
      if ((rc = correct(1, n))) return fail(rc);
    }
    if (cudaMemcpyAsync(hnorms.data(), norms, hnorms.size() * sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(cuda_error(cudaGetLastError(), "parareal_solve3"));
    double num = 0.0, den = 0.0;
    for (int n = 1; n <= N; ++n) {
      den = std::fmax(den, hnorms[2 * n]);
      if (n >= k + 1) num = std::fmax(num, hnorms[2 * n + 1]);
    }
    const double defect = den > 0.0 ? std::sqrt(num) / std::sqrt(den) : std::sqrt(num);
    if (defect_hist) defect_hist[k] = defect;
    if (defect <= tol) {
      ++k;
      converged = true;
      break;
    }
  }
  *k_done = k;
  BS_CUDA_TRY(cudaFreeAsync(ws, s));
  BS_CUDA_TRY(cudaStreamSynchronize(s));
  // after N iterations every slice is exact (serial fine stepping), whatever the last defect
  if (!converged && k < N)
    return set_error(BS_ERR_MAXITER, "parareal_solve3: tol %g not met after %d iterations", tol, k);
  return BS_OK;
}
