// Shared device/host definitions of the Black-Scholes Parareal library (sm_103a).
//
// Grid and operator conventions (eq. fd, Sec. 3.2):
//   nodes x_i = i*h, h = xmax/(M-1); state u[j*M + i] (row = y index j, column = x index i).
//   In index units the coefficients of dtau*R_h are, at node (i, j):
//     east  (i+1, j): dtau*(s1^2 i^2/2 + r i/2)      west  (i-1, j): dtau*(s1^2 i^2/2 - r i/2)
//     south (i, j+1): dtau*(s2^2 j^2/2 + r j/2)      north (i, j-1): dtau*(s2^2 j^2/2 - r j/2)
//     cross: +dtau*rho s1 s2 i j/4 on (i+1, j+1), (i-1, j-1); minus on (i+1, j-1), (i-1, j+1)
//     centre: -(sum of the four axis weights) - dtau*r
//   because x_i/h = i, so the spacing h cancels from every term of eq. (fd).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bsparareal.h"

namespace bsp {

constexpr int kMaxItems = 96;        // items per fine launch (kernel-parameter descriptors)
constexpr int kThreads = 512;        // threads per CTA of the band kernels
constexpr int kMaxCluster = 16;
constexpr int kStatusWords = 4;   // status words of a grid (see bs_grid::status)

// Per-item description carried in kernel parameters.
struct ItemDesc {
  const float* in;
  float* out;
  double tau0, dtau;
  double s1, s2, rho, r;
  double K, w1, w2, K2, cash;
  int payoff;
  int sweeps;     // fine: Jacobi sweeps of the second step of a launch (warm start)
  int sweeps0;    // fine: Jacobi sweeps of the first step of a launch (cold start)
  int sweepsx;    // fine: Jacobi sweeps of steps xstart .. xlate-1 (extrapolated start)
  int sweepsxl;   // fine: Jacobi sweeps of steps >= xlate (extrapolated, transients decayed)
  int xstart;     // fine: first step of a launch that starts from the extrapolated guess (>= 2)
  int xlate;      // fine: first step that uses sweepsxl (>= xstart)
  // Stencil constants of eq. (fd) in index units, rounded once from FP64 on the host:
  // east/west = ax*i^2 +- mx*i, south/north = ay*j^2 +- my*j, cross = gxy*i*j, rdt = r*dtau.
  float ax, mx, ay, my, gxy, rdt;
};

// Band decomposition of an M x M slice over a cluster of C CTAs: each CTA owns BH = G*K
// consecutive rows of ncol (>= M, multiple of 32) columns; thread t works on column
// t % ncol and rows (t / ncol)*K .. +K-1 of the band.
struct BandShape {
  int M, ncol, G, K, BH, C;
};

// FP32 payoff / far-field data, evaluated on the device.
struct PayoffF {
  int kind;
  float K, w1, w2, K2, cash, s1, s2, rho, r;
};

__host__ __device__ inline PayoffF make_payoff(const ItemDesc& d) {
  PayoffF p;
  p.kind = d.payoff;
  p.K = (float)d.K; p.w1 = (float)d.w1; p.w2 = (float)d.w2; p.K2 = (float)d.K2;
  p.cash = (float)d.cash; p.s1 = (float)d.s1; p.s2 = (float)d.s2; p.rho = (float)d.rho;
  p.r = (float)d.r;
  return p;
}

// Bivariate standard normal CDF by integrating its derivative in the correlation
// (Plackett's identity dB/drho = phi2(h, k; rho)) from 0 to rho with 20-point
// Gauss-Legendre quadrature in FP32; used only for the cash-or-nothing far field.
__device__ inline float bvn_cdf_f(float h, float k, float rho) {
  // Gauss-Legendre nodes/weights on [-1, 1], 20 points (positive half; symmetric).
  const float xg[10] = {0.0765265211f, 0.2277858511f, 0.3737060887f, 0.5108670020f,
                        0.6360536807f, 0.7463319065f, 0.8391169718f, 0.9122344283f,
                        0.9639719273f, 0.9931285992f};
  const float wg[10] = {0.1527533871f, 0.1491729865f, 0.1420961093f, 0.1316886384f,
                        0.1181945320f, 0.1019301198f, 0.0832767416f, 0.0626720483f,
                        0.0406014298f, 0.0176140071f};
  float base = normcdff(h) * normcdff(k);
  if (rho == 0.0f) return base;
  float acc = 0.0f;
  for (int q = 0; q < 10; ++q) {
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      float t = 0.5f * rho * (1.0f + sgn * xg[q]);
      float om = 1.0f - t * t;
      float e = __expf(-(h * h - 2.0f * t * h * k + k * k) / (2.0f * om));
      acc += wg[q] * e * rsqrtf(om);
    }
  }
  return base + 0.5f * rho * acc * 0.15915494309f;  // 1/(2 pi)
}

// Far-field Dirichlet value g(x, y, tau) (reading of the boundary: exchange -> Margrabe,
// basket -> forward value max(w1 x + w2 y - K e^{-r tau}, 0), one-asset -> Black-Scholes
// call in x, cash-or-nothing -> eq. solution).  At tau = 0 every branch is the payoff.
__device__ inline float far_field(const PayoffF& p, float x, float y, float tau) {
  switch (p.kind) {
    case BS_PAYOFF_BASKET:
      return fmaxf(p.w1 * x + p.w2 * y - p.K * expf(-p.r * tau), 0.0f);
    case BS_PAYOFF_EXCHANGE: {
      if (y <= 0.0f) return x;
      if (x <= 0.0f) return 0.0f;
      float v = p.s1 * p.s1 + p.s2 * p.s2 - 2.0f * p.rho * p.s1 * p.s2;
      if (tau <= 0.0f || v <= 0.0f) return fmaxf(x - y, 0.0f);
      float sq = sqrtf(v * tau);
      float d1 = (logf(x / y) + 0.5f * v * tau) / sq;
      float d2 = d1 - sq;
      return x * normcdff(d1) - y * normcdff(d2);
    }
    case BS_PAYOFF_CALL1: {
      if (x <= 0.0f) return 0.0f;
      if (tau <= 0.0f) return fmaxf(x - p.K, 0.0f);
      float sq = p.s1 * sqrtf(tau);
      float d1 = (logf(x / p.K) + (p.r + 0.5f * p.s1 * p.s1) * tau) / sq;
      float d2 = d1 - sq;
      return x * normcdff(d1) - p.K * expf(-p.r * tau) * normcdff(d2);
    }
    case BS_PAYOFF_CASH_OR_NOTHING: {
      if (tau <= 0.0f) return (x >= p.K && y >= p.K2) ? p.cash : 0.0f;
      if (x <= 0.0f || y <= 0.0f) return 0.0f;
      float st = sqrtf(tau);
      float dx = (logf(x / p.K) + (p.r - 0.5f * p.s1 * p.s1) * tau) / (p.s1 * st);
      float dy = (logf(y / p.K2) + (p.r - 0.5f * p.s2 * p.s2) * tau) / (p.s2 * st);
      return p.cash * expf(-p.r * tau) * bvn_cdf_f(dx, dy, p.rho);
    }
  }
  return 0.0f;
}

// Payoff u(tau = 0) at (x, y).
__device__ inline float payoff_value(const PayoffF& p, float x, float y) {
  switch (p.kind) {
    case BS_PAYOFF_BASKET: return fmaxf(p.w1 * x + p.w2 * y - p.K, 0.0f);
    case BS_PAYOFF_EXCHANGE: return fmaxf(x - y, 0.0f);
    case BS_PAYOFF_CALL1: return fmaxf(x - p.K, 0.0f);
    case BS_PAYOFF_CASH_OR_NOTHING: return (x >= p.K && y >= p.K2) ? p.cash : 0.0f;
  }
  return 0.0f;
}

// Coefficients of dtau*R_h at a node, in index units (see the file header).
struct Coef {
  float e, w, s, n, g, rdt, invd;   // invd = 1 / (1 + e + w + s + n + rdt)
};

// Stencil coefficients of node (i, j) in FP32 from the item's constants.  Each is a product
// of a correctly rounded constant and an exact integer (i, j < 2^12), so it is within a few
// ulps of the FP64 value; the kernels evaluate them without FP64 arithmetic, which runs at a
// small fraction of the FP32 rate on this GPU.
__device__ __forceinline__ void column_coefs(const ItemDesc& d, int i, float& ce, float& cw,
                                             float& cgi) {
  const float fi = (float)i;
  const float a = d.ax * (fi * fi), m = d.mx * fi;
  ce = a + m;
  cw = a - m;
  cgi = d.gxy * fi;
}

__device__ __forceinline__ void row_coefs(const ItemDesc& d, int j, float& cs, float& cn, float& gj) {
  const float fj = (float)j;
  const float b = d.ay * (fj * fj), n = d.my * fj;
  cs = b + n;
  cn = b - n;
  gj = fj;
}

// 1 / (1 + dtau (sigma1^2 i^2 + sigma2^2 j^2 + r)), the inverse diagonal of I - dtau R_h.
__device__ __forceinline__ float inv_diag(const ItemDesc& d, int i, int j) {
  const float fi = (float)i, fj = (float)j;
  const float diag = 1.0f + (2.0f * (d.ax * (fi * fi)) + 2.0f * (d.ay * (fj * fj)) + d.rdt);
  return 1.0f / diag;
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

#define BS_CUDA_TRY(call)                                      \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::bsp::cuda_error(e_, #call); \
  } while (0)

ItemDesc make_item(const bs_params& p, double tau0, double dtau);
int check_params(const bs_params* p);
double jacobi_contraction(int M, const bs_params& p, double dtau);
enum SweepStart { START_WARM = 0, START_COLD = 1, START_EXTRAP = 2, START_EXTRAP_LATE = 3 };

// Jacobi sweeps of step `step` (0-based) of a fine launch for this item.
__host__ __device__ inline int step_sweeps(const ItemDesc& d, int step) {
  return step == 0 ? d.sweeps0 : step < d.xstart ? d.sweeps : step < d.xlate ? d.sweepsx : d.sweepsxl;
}
int sweeps_for(double q, int start);
BandShape band_shape(int M);

struct Options {
  int fine_sweeps = 0;
  double jacobi_target = 1.0 / 1024.0;            // warm-started steps: q^m <= 2^-10
  double jacobi_target_cold = 1.0 / 4194304.0;    // first step of a launch: q^m <= 2^-22
  double jacobi_target_extrap = 1.0 / 64.0;       // extrapolated starts: q^m <= 2^-6
  // ... from step extrap_late on: two sweeps (the structural minimum) wherever q <= 0.707
  double jacobi_target_extrap_late = 0.5;
  int extrap_start = 2;                           // first extrapolated step of a launch
  int extrap_late = 16;                           // first step with the late target
  int pipeline = 1;                               // parareal_solve overlaps F with the sweep
  // Relative residual of the coarse BiCGSTAB solves (numerical G).  G only has to be a good,
  // deterministic approximation: on the 256 x 256 exchange workloads tolerances from 1e-6 to
  // 1e-4 gave the same Parareal iterations and defects and the same distance to serial fine
  // stepping (FP32 rounding level), 1e-5 a third fewer iterations than 1e-6.
  double krylov_tol = 1e-5;
  // ... of the fine Krylov steps (F for step sizes beyond Jacobi): F defines the answer
  double fine_krylov_tol = 1e-6;
  int krylov_maxit = 400;
  int phase_timing = 0;
  int coarse_variant = -1;   // >= 0: force this coarse band variant; -1: measured per grid size
  int fine_tile = 0;         // region layout of the fine tiles (M > 256): 0 auto, 1 or 2 forced
};
extern Options g_opt;

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};
int ensure(Workspace& w, size_t bytes);
// Counts a device allocation made by the library (every cudaMalloc / cudaMallocAsync /
// cudaMallocHost site calls it; read by bs_device_allocations).
void note_device_alloc();

}  // namespace bsp

struct bs_grid {
  int M;
  double xmax;
  int device;
  bsp::BandShape shape;
  int* status;                 // device int[kStatusWords]: [0] bit 0 = Krylov cap hit, bit 1 =
                               // a cluster exchange timed out; [1] max iterations, [2] total
                               // iterations, [3] solves
  double* dscal;               // device: scalar outputs (defect)
  double* dnorms;              // device: per-slice squared norms / defects
  bsp::Workspace ws_par;       // Parareal F / Gold buffers
  bsp::Workspace ws_fine;      // tile fine stepper (M > 256): ping-pong hi, lo, increment
  bsp::Workspace ws_coarse;    // global-memory coarse solver (M > 256): Krylov vectors
  int coarse_variant = -1;     // band variant of the coarse sweep (-1: not chosen yet)
  int coarse_M = 0;            // numerical G on an Mc x Mc grid with resampling (0: this grid)
  bs_grid* coarse_grid = nullptr;   // that grid (created on first use)
  bsp::Workspace ws_rs;        // resampling buffers and defect partials
  void* pipe = nullptr;        // pipelined driver: second stream and events (pipeline.cu)
  // cached contraction
  double q_key[6];
  double q_val;
  // phase accounting (bs_phase_stats)
  double ms_fine = 0.0, ms_coarse = 0.0;
  int n_fine = 0, n_coarse = 0, n_other = 0;
};

// Kernel launchers implemented in the .cu files.
namespace bsp {
int launch_fine(const bs_grid* g, const ItemDesc* items, int n, int nsteps, cudaStream_t s);
int fine_launches(const bs_grid* g, const ItemDesc* items, int n, int nsteps);   // kernels launch_fine enqueues
int launch_payoff(const bs_grid* g, const ItemDesc& d, float* u, cudaStream_t s);
// Jacobi sweeps per fine step on this grid (cached contraction bound; 0 if q >= 0.8)
int grid_sweeps(bs_grid* g, const bs_params& p, double dtau, int start = START_WARM);
// Coarse numerical propagation / Parareal serial sweep (see coarse.cu).
enum { SWEEP_PROP = 0, SWEEP_INIT = 1, SWEEP_ITER = 2 };
// Independent states propagated by one batched SWEEP_PROP launch (one cluster each): the
// Krylov fine propagator for steps whose Jacobi bound is too large.
constexpr int kMaxProp = 64;
struct PropItem {
  const float* in;
  float* out;
  double tau0;
};

struct SweepArgs {
  int mode;
  int n_first, N;
  int csteps;           // implicit steps per slice
  double slice_len;     // tau length of one slice
  const float* in;      // SWEEP_PROP: input state
  float* out;           // SWEEP_PROP: output state
  float* U;             // [N+1][M*M]
  const float* Fb;      // [N][M*M]
  float* Gold;          // [N][M*M]
  double* norms;        // [2*(N+1)]: ||U_n||^2 and ||dU_n||^2 (iteration)
  double* defect;       // scalar out
  int* status;
  double tol;           // relative residual of the Krylov solve
  int maxit;
  int nprop;            // SWEEP_PROP: > 0 -> cluster blockIdx.y propagates prop[blockIdx.y]
  PropItem prop[kMaxProp];
  // INIT / ITER in chunks: with n_end > 0 the launch runs slices n_begin .. n_end-1 only,
  // starting from U[n_begin] (written by the chunk before) unless n_begin == n_first; the
  // defect is formed by the launch that ends at N.  n_end == 0: the whole sweep.
  int n_begin, n_end;
};
int launch_sweep(const bs_grid* g, const ItemDesc& d, const SweepArgs& a, cudaStream_t s);
// F by BiCGSTAB per implicit step for items whose Jacobi bound is >= 0.8 (capi.cu)
int launch_krylov_fine(bs_grid* g, const ItemDesc* items, int n, int nsteps, cudaStream_t s);
int coarse_cached_variant(int device, int M);   // tuned (or default) variant, no allocation
int coarse_tuned_variant(int device, int M);    // tuned variant, -1 if none measured yet
// Numerical G on the grid's coarse grid with bilinear resampling (resampled.cu).
int resampled_propagate(bs_grid* g, const ItemDesc& d, const float* in, float* out, double tau0, int nsteps,
                        cudaStream_t s);
int resampled_sweep(bs_grid* g, const ItemDesc& d, const SweepArgs& a, cudaStream_t s);
int resampled_launches_per_slice();
// Pipelined Parareal with the numerical G on the state grid (pipeline.cu).
// Pipelined driver: whether N slices are enough to pipeline, and the slices per chunk.
bool pipeline_eligible(int N);
int pipeline_chunk(bs_grid* g, const ItemDesc& dc, int N, cudaStream_t s, int* S);
int fine_cluster_capacity(const bs_grid* g);   // fine band clusters the device runs at once (0: unknown)
int coarse_cluster_ctas(const bs_grid* g, const ItemDesc& d, cudaStream_t s, int* ctas);
int coarse_variant_info(int v, int M, int* ctas, int* threads, int* rows, int* poly, int* quad);
int parareal_pipelined(bs_grid* g, const bs_params* p, int N, int fine_steps, int coarse_steps, double tol,
                       int Kmax, float* u_out, bool user_u0, int* k_done, double* defect_hist,
                       cudaStream_t s);
void pipe_destroy(bs_grid* g);
// coarse steps of each timed tuning solve: past the cold start from the payoff, so that the
// extrapolated initial guesses of the steady state weigh in
constexpr int kAutotuneSteps = 16;
int coarse_autotune(bs_grid* g, const ItemDesc& d, cudaStream_t s, int steps, int* chosen);
// PINO coarse propagator (pino.cu)
int pino_check(const bs_pino* net, int M);
int pino_propagate(bs_pino* net, const bs_grid* g, const ItemDesc& d, const float* in, float* out,
                   double tau0, double dtau, cudaStream_t s);
int pino_propagate_batched(bs_pino* net, const bs_grid* g, const ItemDesc* items, const float* const* in,
                           float* const* out, int B, cudaStream_t s);   // items[b].tau0, .dtau: the slice
int pino_sweep(bs_pino* net, const bs_grid* g, const ItemDesc& d, const SweepArgs& a,
               double* partials, cudaStream_t s);
size_t pino_partials_bytes(int M, int N);
int pino_error_flag(const bs_pino* net, int* flag);
int pino_launches_per_step(const bs_pino* net, int M);
}  // namespace bsp
