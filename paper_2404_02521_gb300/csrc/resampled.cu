// Numerical coarse propagator on a coarser grid (the resolution change of Sec. 4.4, applied
// to the numerical coarse model of Sec. 3.2): for a state u on the M x M grid,
//     G(u) = P( G_c(R u) ),   far field at the slice's end,
// where R restricts bilinearly to the Mc x Mc grid of the same domain, G_c takes the coarse
// implicit-Euler steps there (the BiCGSTAB cluster sweep in PROP mode), and P prolongs the
// coarse state back bilinearly (spatially coarsened Parareal: fine-scale components, which F
// damps within a slice, are dropped by G as well; passing them through G undamped makes
// Parareal stall).  For the serial Parareal sweep every slice is one
// restrict / coarse-solve / apply triple; the apply kernel also forms the correction
// u_{n+1} = F_n + (G_new - G_old) and FP64 block sums of the defect norms, reduced in a fixed
// order by a final kernel (same definition as the same-grid sweep).
#include "common.cuh"

namespace bsp {

enum { RS_PROP = 0, RS_INIT = 1, RS_ITER = 2, RS_ITER_SKIP = 3 };

// bilinear sample of a node field on an Mi grid at fractional node index (tx, ty)
__device__ __forceinline__ float rs_bilinear(const float* u, int Mi, float tx, float ty) {
  int i0 = min((int)floorf(tx), Mi - 2), j0 = min((int)floorf(ty), Mi - 2);
  i0 = max(i0, 0);
  j0 = max(j0, 0);
  const float fx = tx - i0, fy = ty - j0;
  const float* r0 = u + (size_t)j0 * Mi;
  const float* r1 = r0 + Mi;
  const float a = r0[i0] * (1.f - fx) + r0[i0 + 1] * fx;
  const float c = r1[i0] * (1.f - fx) + r1[i0 + 1] * fx;
  return a * (1.f - fy) + c * fy;
}

__global__ void rs_restrict_kernel(const float* __restrict__ u, int M, float* __restrict__ uc, int Mc) {
  const size_t P = (size_t)Mc * Mc;
  const float ratio = (float)(M - 1) / (float)(Mc - 1);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)((unsigned)e / (unsigned)Mc), i = (int)(e - (size_t)j * Mc);
    uc[e] = rs_bilinear(u, M, i * ratio, j * ratio);
  }
}

struct RsApply {
  int mode, M, Mc;
  float h, tau_new;
  PayoffF pf;
  float* out;           // PROP: G(u_n)
  const float* c_out;   // G_c(R u_n) on the coarse grid
  float* Unext;         // Parareal: u_{n+1}
  const float* Fn;      // Parareal: F(u_n)
  float* Gold;          // Parareal: G_old_n
  double* partials;     // Parareal: [blocks][2] sums of u^2 and du^2
};

// Blocks of the apply kernel: a grid-stride loop gives each thread several nodes, whose
// squares it adds in FP32 before one FP64 reduction (one node per thread made the FP64
// butterfly the bottleneck at this part's FP64 rate).
constexpr int kRsApplyBlocks = 608;
static int rs_apply_blocks(size_t MM) { return (int)std::min<size_t>((MM + 255) / 256, kRsApplyBlocks); }

__global__ void rs_apply_kernel(const __grid_constant__ RsApply a) {
  const int M = a.M;
  const size_t MM = (size_t)M * M;
  const float ratio = (float)(a.Mc - 1) / (float)(M - 1);
  float s0 = 0.f, s1 = 0.f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MM; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)((unsigned)e / (unsigned)M), i = (int)(e - (size_t)j * M);
    float g;
    if (a.mode == RS_ITER_SKIP) {
      g = a.Gold[e];
    } else if (i == M - 1 || j == M - 1) {
      g = far_field(a.pf, i * a.h, j * a.h, a.tau_new);
    } else {
      g = rs_bilinear(a.c_out, a.Mc, i * ratio, j * ratio);
    }
    if (a.mode == RS_PROP) {
      a.out[e] = g;
    } else if (a.mode == RS_INIT) {
      a.Unext[e] = g;
      a.Gold[e] = g;
      s0 = fmaf(g, g, s0);
    } else {
      // u_new - u_old of nearby values is exact in FP32
      const float unew = a.Fn[e] + (g - a.Gold[e]);
      const float du = unew - a.Unext[e];
      a.Unext[e] = unew;
      a.Gold[e] = g;
      s0 = fmaf(unew, unew, s0);
      s1 = fmaf(du, du, s1);
    }
  }
  if (a.mode == RS_PROP) return;
  double n0 = s0, n1 = s1;
  __shared__ double r0[32], r1[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n0 += __shfl_xor_sync(0xffffffffu, n0, off);
    n1 += __shfl_xor_sync(0xffffffffu, n1, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { r0[warp] = n0; r1[warp] = n1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += r0[w]; s1 += r1[w]; }
    a.partials[2 * blockIdx.x] = s0;
    a.partials[2 * blockIdx.x + 1] = s1;
  }
}

// norms of slices n_lo..N from the block partials (fixed order), then
// delta = max_{n > n_first} ||du_n|| / max_n ||u_n||  (reading c5).
__global__ void rs_defect_kernel(const double* partials, int nblocks, int n_lo, int N, int n_first,
                                 double* norms, double* defect, int iter) {
  const int lane = threadIdx.x;
  for (int n = n_lo; n <= N; ++n) {
    const double* p = partials + (size_t)n * 2 * nblocks;
    double s0 = 0.0, s1 = 0.0;
    for (int b = lane; b < nblocks; b += 32) { s0 += p[2 * b]; s1 += p[2 * b + 1]; }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, off);
      s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    if (lane == 0) {
      norms[2 * n] = s0;
      norms[2 * n + 1] = iter ? s1 : 0.0;
    }
  }
  if (lane == 0 && iter) {
    double num = 0.0, den = 0.0;
    for (int n = 1; n <= N; ++n) {
      den = fmax(den, norms[2 * n]);
      if (n >= n_first + 1) num = fmax(num, norms[2 * n + 1]);
    }
    defect[0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
  }
}

// Coarse grid and buffers of a state grid: [R u, G_c(R u)] (Mc^2 floats each) and the block
// partials [(N+1)][blocks][2].
static int rs_ensure(bs_grid* g, int N, float** c_in, float** c_out, double** partials) {
  const int Mc = g->coarse_M;
  if (!g->coarse_grid || g->coarse_grid->M != Mc) {
    if (g->coarse_grid) bs_grid_destroy(g->coarse_grid);
    g->coarse_grid = nullptr;
    int rc = bs_grid_create(Mc, g->xmax, &g->coarse_grid);
    if (rc) return rc;
  }
  const size_t MM = (size_t)g->M * g->M, P = (size_t)Mc * Mc;
  const size_t nblocks = (size_t)rs_apply_blocks(MM);
  const size_t fbytes = ((2 * P * sizeof(float)) + 255) / 256 * 256;
  int rc = ensure(g->ws_rs, fbytes + (size_t)(N + 1) * nblocks * 2 * sizeof(double));
  if (rc) return rc;
  *c_in = (float*)g->ws_rs.ptr;
  *c_out = *c_in + P;
  *partials = (double*)((unsigned char*)g->ws_rs.ptr + fbytes);
  return BS_OK;
}

// One coarse step sequence of one slice on the coarse grid: c_out = G_c(c_in).
static int rs_coarse(bs_grid* g, const ItemDesc& d, const float* c_in, float* c_out, double tau0, int csteps,
                     cudaStream_t s) {
  ItemDesc dc = d;
  dc.tau0 = tau0;
  SweepArgs a = {};
  a.mode = SWEEP_PROP;
  a.n_first = 0;
  a.N = 1;
  a.csteps = csteps;
  a.slice_len = 0.0;
  a.in = c_in;
  a.out = c_out;
  a.status = g->status;
  a.tol = g_opt.krylov_tol;
  a.maxit = g_opt.krylov_maxit;
  return launch_sweep(g->coarse_grid, dc, a, s);
}

static RsApply rs_args(const bs_grid* g, const ItemDesc& d, int mode, double tau_new, const float* c_out) {
  RsApply ra = {};
  ra.mode = mode;
  ra.M = g->M;
  ra.Mc = g->coarse_M;
  ra.h = (float)(g->xmax / (g->M - 1));
  ra.tau_new = (float)tau_new;
  ra.pf = make_payoff(d);
  ra.c_out = c_out;
  return ra;
}

// coarse_propagate on a grid with a coarse grid: d.dtau is the coarse step, nsteps of them.
int resampled_propagate(bs_grid* g, const ItemDesc& d, const float* in, float* out, double tau0, int nsteps,
                        cudaStream_t s) {
  float *c_in, *c_out;
  double* partials;
  int rc = rs_ensure(g, 1, &c_in, &c_out, &partials);
  if (rc) return rc;
  const int Mc = g->coarse_M;
  rs_restrict_kernel<<<(Mc * Mc + 255) / 256, 256, 0, s>>>(in, g->M, c_in, Mc);
  BS_CUDA_TRY(cudaGetLastError());
  if ((rc = rs_coarse(g, d, c_in, c_out, tau0, nsteps, s))) return rc;
  RsApply ra = rs_args(g, d, RS_PROP, tau0 + nsteps * d.dtau, c_out);
  ra.out = out;
  const size_t MM = (size_t)g->M * g->M;
  rs_apply_kernel<<<rs_apply_blocks(MM), 256, 0, s>>>(ra);
  BS_CUDA_TRY(cudaGetLastError());
  return BS_OK;
}

// One serial Parareal sweep (SWEEP_INIT or SWEEP_ITER) with the resampled numerical G.
int resampled_sweep(bs_grid* g, const ItemDesc& d, const SweepArgs& a, cudaStream_t s) {
  float *c_in, *c_out;
  double* partials;
  int rc = rs_ensure(g, a.N, &c_in, &c_out, &partials);
  if (rc) return rc;
  const int M = g->M, Mc = g->coarse_M;
  const size_t MM = (size_t)M * M;
  const int nblocks = rs_apply_blocks(MM);
  // slices of this call: the whole sweep, or the range [n_begin, n_end) (a partitioned sweep)
  const int n_lo = a.n_end > 0 ? a.n_begin : a.n_first;
  const int n_hi = a.n_end > 0 ? a.n_end : a.N;
  for (int n = n_lo; n < n_hi; ++n) {
    const bool skip = (a.mode == SWEEP_ITER && n == a.n_first);
    const float* un = a.U + (size_t)n * MM;
    const double tau_n = n * a.slice_len;
    if (!skip) {
      rs_restrict_kernel<<<(Mc * Mc + 255) / 256, 256, 0, s>>>(un, M, c_in, Mc);
      BS_CUDA_TRY(cudaGetLastError());
      if ((rc = rs_coarse(g, d, c_in, c_out, tau_n, a.csteps, s))) return rc;
    }
    const int mode = a.mode == SWEEP_INIT ? RS_INIT : (skip ? RS_ITER_SKIP : RS_ITER);
    RsApply ra = rs_args(g, d, mode, tau_n + a.slice_len, c_out);
    ra.Unext = a.U + (size_t)(n + 1) * MM;
    ra.Fn = a.Fb + (size_t)n * MM;
    ra.Gold = a.Gold + (size_t)n * MM;
    ra.partials = partials + (size_t)(n + 1) * 2 * nblocks;
    rs_apply_kernel<<<nblocks, 256, 0, s>>>(ra);
    BS_CUDA_TRY(cudaGetLastError());
  }
  // norms of the slices this call wrote (and, for a whole sweep, the defect)
  const int n_norm = a.n_end > 0 ? n_lo + 1 : (a.mode == SWEEP_INIT ? 1 : a.n_first + 1);
  rs_defect_kernel<<<1, 32, 0, s>>>(partials, nblocks, n_norm, n_hi, a.n_first, a.norms, a.defect,
                                    a.mode == SWEEP_ITER ? 1 : 0);
  BS_CUDA_TRY(cudaGetLastError());
  return BS_OK;
}

// kernels per slice of a sweep (restrict, coarse solve, apply)
int resampled_launches_per_slice() { return 3; }

}  // namespace bsp
