// parareal_solve_noalloc: Parareal with the numerical coarse model for callers that may not
// allocate device memory -- for example a latency-critical pricing path where a device
// allocation (which can synchronise the whole device and take milliseconds) is forbidden,
// or a host framework that owns all device memory through its own allocator and does not
// allow raw cudaMalloc calls from libraries it embeds.
//
// The fine and coarse buffers, the per-slice norms, the status word and the defect scalar
// live in one file-scope device array of fixed size (every GPU that loads this library
// holds it until the process exits).  The caller still provides u_out.  This entry point
// calls no cudaMalloc, cudaFree or allocating library routine.
#include <mutex>

#include "common.cuh"

namespace bsp {

constexpr size_t kNoAllocMaxNM2 = size_t(1) << 22;   // N * M * M <= 4,194,304
constexpr int kNoAllocMaxN = 1024;
constexpr size_t kNoAllocStatusOff = 0;                                  // int[kStatusWords]
constexpr size_t kNoAllocDefectOff = 256;                                // double[8]
constexpr size_t kNoAllocNormsOff = 512;                                 // double[2(N+1)]
constexpr size_t kNoAllocBufOff =
    kNoAllocNormsOff + ((2 * (kNoAllocMaxN + 1) * sizeof(double) + 255) / 256) * 256;
constexpr size_t kNoAllocBytes = kNoAllocBufOff + 2 * kNoAllocMaxNM2 * sizeof(float);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices] = {};
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device, looked up once per device.
// In host code the array's name is only a host-side stand-in, never a device address.
static int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(BS_ERR_ARG, "parareal_solve_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  return BS_OK;
}

}  // namespace bsp

using namespace bsp;

extern "C" int parareal_solve_noalloc(int M, double xmax, const bs_params* p, int N,
                                      int fine_steps, int coarse_steps, double tol, int Kmax,
                                      float* u_out, int* k_done, double* defect_hist,
                                      bs_stream stream) {
  if (!u_out || !k_done) return set_error(BS_ERR_ARG, "parareal_solve_noalloc: NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  if (M < 4 || M > 4096 || !(xmax > 0.0))
    return set_error(BS_ERR_ARG, "parareal_solve_noalloc: M=%d xmax=%g", M, xmax);
  if (N < 1 || fine_steps < 1 || coarse_steps < 1 || Kmax < 0 || Kmax > N || !(p->T > 0.0))
    return set_error(BS_ERR_ARG, "parareal_solve_noalloc: N=%d fine_steps=%d coarse_steps=%d Kmax=%d",
                     N, fine_steps, coarse_steps, Kmax);
  if (N > kNoAllocMaxN || (size_t)N * M * M > kNoAllocMaxNM2)
    return set_error(BS_ERR_ARG,
                     "parareal_solve_noalloc: N*M*M = %zu exceeds the fixed scratch capacity of "
                     "%zu nodes (N <= %d); use parareal_solve",
                     (size_t)N * M * M, kNoAllocMaxNM2, kNoAllocMaxN);
  const BandShape shape = band_shape(M);
  if (shape.C < 1 || shape.C > kMaxCluster)
    return set_error(BS_ERR_ARG,
                     "parareal_solve_noalloc: M=%d exceeds the limit M <= 256 (grids that fit one "
                     "thread-block cluster); use parareal_solve", M);
  const double slice = p->T / N;
  const double dtau_f = slice / fine_steps;
  const double q = jacobi_contraction(M, *p, dtau_f);
  const int sweeps = sweeps_for(q, START_WARM), sweeps0 = sweeps_for(q, START_COLD);
  const int sweepsx = sweeps_for(q, START_EXTRAP), sweepsxl = sweeps_for(q, START_EXTRAP_LATE);
  if (sweeps == 0)
    return set_error(BS_ERR_ARG,
                     "parareal_solve_noalloc: the fine step's Jacobi bound %.3f is >= 0.8 (only the "
                     "Jacobi stepper runs without allocation); use more fine steps or parareal_solve", q);

  unsigned char* base = nullptr;
  if ((rc = noalloc_scratch(&base))) return rc;
  int* status = reinterpret_cast<int*>(base + kNoAllocStatusOff);
  double* defect = reinterpret_cast<double*>(base + kNoAllocDefectOff);
  double* norms = reinterpret_cast<double*>(base + kNoAllocNormsOff);
  const size_t MM = (size_t)M * M;
  float* Fb = reinterpret_cast<float*>(base + kNoAllocBufOff);
  float* Gold = Fb + (size_t)N * MM;

  // A grid description on the stack: the launchers read only M, xmax and the band shape.
  bs_grid g{};
  g.M = M;
  g.xmax = xmax;
  g.shape = shape;
  g.status = status;
  g.dscal = defect;
  // the measured coarse variant if this process has one for M (tuning would allocate)
  BS_CUDA_TRY(cudaGetDevice(&g.device));
  g.coarse_variant = coarse_cached_variant(g.device, M);
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: the status word must start at zero
  BS_CUDA_TRY(cudaMemsetAsync(status, 0, kStatusWords * sizeof(int), s));

  ItemDesc dc = make_item(*p, 0.0, slice / coarse_steps);
  if ((rc = launch_payoff(&g, dc, u_out, s))) return rc;
  SweepArgs a = {};
  a.N = N;
  a.csteps = coarse_steps;
  a.slice_len = slice;
  a.U = u_out;
  a.Fb = Fb;
  a.Gold = Gold;
  a.norms = norms;
  a.defect = defect;
  a.status = status;
  a.tol = g_opt.krylov_tol;
  a.maxit = g_opt.krylov_maxit;
  a.mode = SWEEP_INIT;
  a.n_first = 0;
  if ((rc = launch_sweep(&g, dc, a, s))) return rc;

  ItemDesc items[kMaxItems];
  int k = 0;
  bool converged = false;
  for (; k < Kmax; ++k) {
    // F on slices k..N-1, in launches of at most kMaxItems states
    for (int n0 = k; n0 < N; n0 += kMaxItems) {
      const int B = (N - n0) < kMaxItems ? (N - n0) : kMaxItems;
      for (int i = 0; i < B; ++i) {
        const int n = n0 + i;
        ItemDesc d = make_item(*p, n * slice, dtau_f);
        d.in = u_out + (size_t)n * MM;
        d.out = Fb + (size_t)n * MM;
        d.sweeps = sweeps;
        d.sweeps0 = sweeps0;
        d.sweepsx = sweepsx;
        d.sweepsxl = sweepsxl;
        items[i] = d;
      }
      if ((rc = launch_fine(&g, items, B, fine_steps, s))) return rc;
    }
    a.mode = SWEEP_ITER;
    a.n_first = k;
    if ((rc = launch_sweep(&g, dc, a, s))) return rc;
    double host_defect = 0.0;
    int host_status = 0;
    BS_CUDA_TRY(cudaMemcpyAsync(&host_defect, defect, sizeof(double), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaStreamSynchronize(s));
    if (defect_hist) defect_hist[k] = host_defect;
    if (host_status) {
      *k_done = k + 1;
      if (host_status & 2)
        return set_error(BS_ERR_CUDA, "parareal_solve_noalloc: a cluster exchange of the coarse sweep timed out");
      return set_error(BS_ERR_NOCONV, "parareal_solve_noalloc: a coarse BiCGSTAB solve hit its iteration cap");
    }
    if (host_defect <= tol) {
      ++k;
      converged = true;
      break;
    }
  }
  *k_done = k;
  if (Kmax == 0) BS_CUDA_TRY(cudaStreamSynchronize(s));
  // after N iterations every slice is exact (serial fine stepping), whatever the last defect
  if (!converged && k < N)
    return set_error(BS_ERR_MAXITER, "parareal_solve_noalloc: tol %g not met after %d iterations", tol, k);
  return BS_OK;
}
