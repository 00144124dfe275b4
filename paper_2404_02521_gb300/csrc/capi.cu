// C ABI of the Black-Scholes Parareal library: handles, argument checks, the payoff kernel
// (K6) and the Parareal driver loop (eq. parareal, Sec. 3.1).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace bsp {

static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  return set_error(e == cudaErrorMemoryAllocation ? BS_ERR_OOM : BS_ERR_CUDA, "%s failed: %s",
                   what, cudaGetErrorString(e));
}

int check_params(const bs_params* p) {
  if (!p) return set_error(BS_ERR_ARG, "params is NULL");
  if (!(p->sigma1 > 0.0) || !(p->sigma2 > 0.0)) return set_error(BS_ERR_ARG, "sigma must be > 0");
  if (!(std::fabs(p->rho) < 1.0)) return set_error(BS_ERR_ARG, "|rho| must be < 1");
  if (!(p->r >= 0.0)) return set_error(BS_ERR_ARG, "r must be >= 0");
  if (p->payoff < BS_PAYOFF_BASKET || p->payoff > BS_PAYOFF_CASH_OR_NOTHING)
    return set_error(BS_ERR_ARG, "unknown payoff %d", p->payoff);
  if (p->reserved != 0) return set_error(BS_ERR_ARG, "bs_params.reserved must be 0");
  if (p->payoff == BS_PAYOFF_CASH_OR_NOTHING && !(std::fabs(p->rho) <= 0.95))
    return set_error(BS_ERR_ARG, "cash-or-nothing far field needs |rho| <= 0.95");
  return BS_OK;
}

ItemDesc make_item(const bs_params& p, double tau0, double dtau) {
  ItemDesc d;
  d.in = nullptr;
  d.out = nullptr;
  d.tau0 = tau0;
  d.dtau = dtau;
  d.s1 = p.sigma1; d.s2 = p.sigma2; d.rho = p.rho; d.r = p.r;
  d.K = p.strike; d.w1 = p.w1; d.w2 = p.w2; d.K2 = p.strike2; d.cash = p.cash;
  d.payoff = p.payoff;
  d.sweeps = 0;
  d.sweeps0 = 0;
  d.sweepsx = 0;
  d.sweepsxl = 0;
  d.xstart = g_opt.extrap_start;
  d.xlate = g_opt.extrap_late > g_opt.extrap_start ? g_opt.extrap_late : g_opt.extrap_start;
  d.ax = (float)(0.5 * p.sigma1 * p.sigma1 * dtau);
  d.mx = (float)(0.5 * p.r * dtau);
  d.ay = (float)(0.5 * p.sigma2 * p.sigma2 * dtau);
  d.my = (float)(0.5 * p.r * dtau);
  d.gxy = (float)(0.25 * p.rho * p.sigma1 * p.sigma2 * dtau);
  d.rdt = (float)(p.r * dtau);
  return d;
}

// max over PDE rows (0 <= i, j <= M-2) of sum |off-diagonal| / diagonal of I - dtau R_h.
double jacobi_contraction(int M, const bs_params& p, double dtau) {
  double q = 0.0;
  const double g = std::fabs(p.rho) * p.sigma1 * p.sigma2;
  for (int j = 0; j <= M - 2; ++j) {
    const double bj = 0.5 * p.sigma2 * p.sigma2 * j * j, nj = 0.5 * p.r * j;
    const double offy = std::fabs(bj + nj) + std::fabs(bj - nj);
    for (int i = 0; i <= M - 2; ++i) {
      const double ai = 0.5 * p.sigma1 * p.sigma1 * i * i, mi = 0.5 * p.r * i;
      const double off = dtau * (std::fabs(ai + mi) + std::fabs(ai - mi) + offy + g * i * j);
      const double diag = 1.0 + dtau * (2.0 * ai + 2.0 * bj + p.r);
      q = std::fmax(q, off / diag);
    }
  }
  return q;
}

Options g_opt;

// Sweeps so that q^m <= target (at least 2: the first sweep forms b, the last applies d).
int sweeps_for(double q, int start) {
  if (!(q < 0.8)) return 0;
  if (g_opt.fine_sweeps > 0) return g_opt.fine_sweeps;
  if (q <= 0.0) return 2;
  const double target = start == START_COLD          ? g_opt.jacobi_target_cold
                        : start == START_EXTRAP      ? g_opt.jacobi_target_extrap
                        : start == START_EXTRAP_LATE ? g_opt.jacobi_target_extrap_late
                                                     : g_opt.jacobi_target;
  int m = (int)std::ceil(std::log(target) / std::log(q));
  return m < 2 ? 2 : m;
}

// Band shapes of the cluster-resident kernels (NCOL columns, NT threads, K rows per thread,
// band height BH = (NT / NCOL) * K, cluster size C = ceil(M / BH)).
BandShape band_shape(int M) {
  BandShape s = {};
  s.M = M;
  if (M <= 32) { s.ncol = 32; s.G = 8; s.K = 4; }
  else if (M <= 64) { s.ncol = 64; s.G = 8; s.K = 8; }
  else if (M <= 128) { s.ncol = 128; s.G = 4; s.K = 16; }
  else if (M <= 256) { s.ncol = 256; s.G = 2; s.K = 16; }
  else { s.C = 0; return s; }
  s.BH = s.G * s.K;
  s.C = (M + s.BH - 1) / s.BH;
  return s;
}

static std::atomic<long long> g_dev_allocs{0};

void note_device_alloc() { g_dev_allocs.fetch_add(1, std::memory_order_relaxed); }

int ensure(Workspace& w, size_t bytes) {
  if (w.bytes >= bytes) return BS_OK;
  if (w.ptr) cudaFree(w.ptr);
  w.ptr = nullptr;
  w.bytes = 0;
  note_device_alloc();
  BS_CUDA_TRY(cudaMalloc(&w.ptr, bytes));
  w.bytes = bytes;
  return BS_OK;
}

__global__ void payoff_kernel(PayoffF pf, float* u, int M, float h) {
  const size_t n = (size_t)M * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)((unsigned)e / (unsigned)M), i = (int)(e - (size_t)j * M);
    u[e] = payoff_value(pf, i * h, j * h);
  }
}

int launch_payoff(const bs_grid* g, const ItemDesc& d, float* u, cudaStream_t s) {
  const int M = g->M;
  const size_t n = (size_t)M * M;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  payoff_kernel<<<blocks, 256, 0, s>>>(make_payoff(d), u, M, (float)(g->xmax / (M - 1)));
  BS_CUDA_TRY(cudaGetLastError());
  return BS_OK;
}

int grid_sweeps(bs_grid* g, const bs_params& p, double dtau, int start) {
  const double key[6] = {p.sigma1, p.sigma2, p.rho, p.r, dtau, (double)g->M};
  if (std::memcmp(key, g->q_key, sizeof(key)) != 0) {
    g->q_val = jacobi_contraction(g->M, p, dtau);
    std::memcpy(g->q_key, key, sizeof(key));
  }
  return sweeps_for(g->q_val, start);
}

// Fine propagation of items whose Jacobi bound is too large for the sweep steppers: every
// implicit step is solved by BiCGSTAB (the coarse solver), one cluster per state, in batched
// SWEEP_PROP launches of states that share their parameters and step size.
int launch_krylov_fine(bs_grid* g, const ItemDesc* items, int n, int nsteps, cudaStream_t s) {
  auto same = [](const ItemDesc& a, const ItemDesc& b) {
    return a.s1 == b.s1 && a.s2 == b.s2 && a.rho == b.rho && a.r == b.r && a.K == b.K && a.w1 == b.w1 &&
           a.w2 == b.w2 && a.K2 == b.K2 && a.cash == b.cash && a.payoff == b.payoff && a.dtau == b.dtau;
  };
  int i = 0;
  while (i < n) {
    SweepArgs a = {};
    a.mode = SWEEP_PROP;
    a.n_first = 0;
    a.N = 1;
    a.csteps = nsteps;
    a.slice_len = 0.0;
    a.status = g->status;
    a.tol = g_opt.fine_krylov_tol;
    a.maxit = g_opt.krylov_maxit;
    int j = i;
    while (j < n && j - i < kMaxProp && same(items[i], items[j])) {
      a.prop[j - i] = PropItem{items[j].in, items[j].out, items[j].tau0};
      ++j;
    }
    a.nprop = j - i;
    g->n_fine += 1;
    int rc = launch_sweep(g, items[i], a, s);
    if (rc) return rc;
    i = j;
  }
  return BS_OK;
}

}  // namespace bsp

using namespace bsp;

namespace bsp {
int launch_physics_loss(const bs_grid* g, const bs_params* p, const float* const* u_pred,
                        const float* const* u_prev, const double* dtau, int B, double* loss,
                        float* const* grad, cudaStream_t s);
}  // namespace bsp

extern "C" {

const char* bs_last_error(void) { return g_err; }

int bs_device_allocations(long long* count) {
  if (!count) return set_error(BS_ERR_ARG, "bs_device_allocations: NULL argument");
  *count = g_dev_allocs.load(std::memory_order_relaxed);
  return BS_OK;
}

int bs_grid_create(int M, double xmax, bs_grid** out) {
  g_err[0] = 0;
  if (!out) return set_error(BS_ERR_ARG, "bs_grid_create: out is NULL");
  *out = nullptr;
  if (M < 4 || M > 4096) return set_error(BS_ERR_ARG, "bs_grid_create: M=%d out of [4, 4096]", M);
  if (!(xmax > 0.0)) return set_error(BS_ERR_ARG, "bs_grid_create: xmax must be > 0");
  bs_grid* g = new bs_grid();
  g->M = M;
  g->xmax = xmax;
  g->shape = band_shape(M);
  std::memset(g->q_key, 0, sizeof(g->q_key));
  g->q_val = 0.0;
  cudaError_t e = cudaGetDevice(&g->device);
  note_device_alloc();
  note_device_alloc();
  if (e == cudaSuccess) e = cudaMalloc(&g->status, kStatusWords * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->status, 0, kStatusWords * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&g->dscal, 8 * sizeof(double));
  g->dnorms = nullptr;
  if (e != cudaSuccess) {
    delete g;
    return cuda_error(e, "bs_grid_create");
  }
  *out = g;
  return BS_OK;
}

int bs_grid_destroy(bs_grid* g) {
  if (!g) return BS_OK;
  cudaFree(g->status);
  cudaFree(g->dscal);
  if (g->dnorms) cudaFree(g->dnorms);
  if (g->ws_par.ptr) cudaFree(g->ws_par.ptr);
  if (g->ws_fine.ptr) cudaFree(g->ws_fine.ptr);
  if (g->ws_coarse.ptr) cudaFree(g->ws_coarse.ptr);
  if (g->ws_rs.ptr) cudaFree(g->ws_rs.ptr);
  pipe_destroy(g);
  if (g->coarse_grid) bs_grid_destroy(g->coarse_grid);
  delete g;
  return BS_OK;
}

int bs_payoff(const bs_grid* g, const bs_params* p, float* u, bs_stream stream) {
  if (!g || !u) return set_error(BS_ERR_ARG, "bs_payoff: NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  const_cast<bs_grid*>(g)->n_other += 1;
  return launch_payoff(g, make_item(*p, 0.0, 0.0), u, (cudaStream_t)stream);
}

int bs_fine_sweeps(const bs_grid* g, const bs_params* p, double dtau, int first_step) {
  if (!g || check_params(p) || !(dtau > 0.0)) return 0;
  if (first_step < 0 || first_step > 3) return 0;
  return grid_sweeps(const_cast<bs_grid*>(g), *p, dtau, first_step);
}

int fine_propagate_batched(const bs_grid* g, const bs_params* p, const float* const* u_in,
                           float* const* u_out, const double* tau0, const double* dtau,
                           int nsteps, int B, bs_stream stream) {
  if (!g || !p || !u_in || !u_out || !tau0 || !dtau)
    return set_error(BS_ERR_ARG, "fine_propagate_batched: NULL argument");
  if (B < 1 || nsteps < 0) return set_error(BS_ERR_ARG, "fine_propagate_batched: B=%d nsteps=%d", B, nsteps);
  std::vector<ItemDesc> items((size_t)B);
  for (int b = 0; b < B; ++b) {
    int rc = check_params(&p[b]);
    if (rc) return rc;
    if (!u_in[b] || !u_out[b]) return set_error(BS_ERR_ARG, "fine_propagate_batched: NULL state %d", b);
    if (!(dtau[b] > 0.0)) return set_error(BS_ERR_ARG, "fine_propagate_batched: dtau[%d] <= 0", b);
    ItemDesc d = make_item(p[b], tau0[b], dtau[b]);
    d.in = u_in[b];
    d.out = u_out[b];
    d.sweeps = grid_sweeps(const_cast<bs_grid*>(g), p[b], dtau[b]);
    d.sweeps0 = grid_sweeps(const_cast<bs_grid*>(g), p[b], dtau[b], START_COLD);
    d.sweepsx = grid_sweeps(const_cast<bs_grid*>(g), p[b], dtau[b], START_EXTRAP);
    d.sweepsxl = grid_sweeps(const_cast<bs_grid*>(g), p[b], dtau[b], START_EXTRAP_LATE);
    items[(size_t)b] = d;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (nsteps == 0) {
    for (int b = 0; b < B; ++b)
      if (u_out[b] != u_in[b])
        BS_CUDA_TRY(cudaMemcpyAsync(u_out[b], u_in[b], sizeof(float) * g->M * g->M,
                                    cudaMemcpyDeviceToDevice, s));
    return BS_OK;
  }
  // Jacobi bound < 0.8: the sweep steppers; otherwise BiCGSTAB per step
  std::vector<ItemDesc> jac, kry;
  for (const ItemDesc& d : items) (d.sweeps > 0 ? jac : kry).push_back(d);
  int rc = BS_OK;
  if (!jac.empty()) {
    const_cast<bs_grid*>(g)->n_fine += fine_launches(g, jac.data(), (int)jac.size(), nsteps);
    if ((rc = launch_fine(g, jac.data(), (int)jac.size(), nsteps, s))) return rc;
  }
  if (!kry.empty()) rc = launch_krylov_fine(const_cast<bs_grid*>(g), kry.data(), (int)kry.size(), nsteps, s);
  return rc;
}

int coarse_propagate(const bs_grid* g, int kind, const bs_pino* net, const bs_params* p,
                     const float* u_in, float* u_out, double tau0, double dtau_slice, int nsteps,
                     bs_stream stream) {
  if (!g || !u_in || !u_out) return set_error(BS_ERR_ARG, "coarse_propagate: NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  if (!(dtau_slice > 0.0)) return set_error(BS_ERR_ARG, "coarse_propagate: dtau_slice <= 0");
  if (kind == BS_COARSE_NUM) {
    if (net) return set_error(BS_ERR_ARG, "coarse_propagate: net must be NULL for BS_COARSE_NUM");
    if (nsteps < 1) return set_error(BS_ERR_ARG, "coarse_propagate: nsteps < 1");
    ItemDesc d = make_item(*p, tau0, dtau_slice / nsteps);
    if (g->coarse_M > 0 && g->coarse_M != g->M) {
      const_cast<bs_grid*>(g)->n_coarse += resampled_launches_per_slice();
      return resampled_propagate(const_cast<bs_grid*>(g), d, u_in, u_out, tau0, nsteps, (cudaStream_t)stream);
    }
    SweepArgs a = {};
    a.mode = SWEEP_PROP;
    a.n_first = 0;
    a.N = 1;
    a.csteps = nsteps;
    a.slice_len = 0.0;
    a.in = u_in;
    a.out = u_out;
    a.status = g->status;
    a.tol = g_opt.krylov_tol;
    a.maxit = g_opt.krylov_maxit;
    const_cast<bs_grid*>(g)->n_coarse += 1;
    return launch_sweep(g, d, a, (cudaStream_t)stream);
  }
  if (kind == BS_COARSE_PINO) {
    const_cast<bs_grid*>(g)->n_coarse += 1;
    return pino_propagate(const_cast<bs_pino*>(net), g, make_item(*p, tau0, dtau_slice), u_in, u_out,
                          tau0, dtau_slice, (cudaStream_t)stream);
  }
  return set_error(BS_ERR_ARG, "coarse_propagate: unknown kind %d", kind);
}

int coarse_propagate_batched(const bs_grid* g, int kind, const bs_pino* net, const bs_params* p,
                             const float* const* u_in, float* const* u_out, const double* tau0,
                             double dtau_slice, int nsteps, int B, bs_stream stream) {
  if (!g || !p || !u_in || !u_out || !tau0) return set_error(BS_ERR_ARG, "coarse_propagate_batched: NULL argument");
  if (B < 1) return set_error(BS_ERR_ARG, "coarse_propagate_batched: B=%d", B);
  if (!(dtau_slice > 0.0)) return set_error(BS_ERR_ARG, "coarse_propagate_batched: dtau_slice <= 0");
  for (int b = 0; b < B; ++b) {
    int rc = check_params(&p[b]);
    if (rc) return rc;
    if (!u_in[b] || !u_out[b]) return set_error(BS_ERR_ARG, "coarse_propagate_batched: NULL state %d", b);
  }
  cudaStream_t s = (cudaStream_t)stream;
  bs_grid* gm = const_cast<bs_grid*>(g);
  if (kind == BS_COARSE_PINO) {
    std::vector<ItemDesc> items((size_t)B);
    for (int b = 0; b < B; ++b) items[(size_t)b] = make_item(p[b], tau0[b], dtau_slice);
    gm->n_coarse += ((B + 127) / 128) * pino_launches_per_step(const_cast<bs_pino*>(net), gm->M);
    return pino_propagate_batched(const_cast<bs_pino*>(net), g, items.data(), u_in, u_out, B, s);
  }
  if (kind != BS_COARSE_NUM) return set_error(BS_ERR_ARG, "coarse_propagate_batched: unknown kind %d", kind);
  if (net) return set_error(BS_ERR_ARG, "coarse_propagate_batched: net must be NULL for BS_COARSE_NUM");
  if (nsteps < 1) return set_error(BS_ERR_ARG, "coarse_propagate_batched: nsteps < 1");
  if (g->coarse_M > 0 && g->coarse_M != g->M) {   // resampled G: state after state
    for (int b = 0; b < B; ++b) {
      gm->n_coarse += resampled_launches_per_slice();
      int rc = resampled_propagate(gm, make_item(p[b], tau0[b], dtau_slice / nsteps), u_in[b], u_out[b], tau0[b],
                                   nsteps, s);
      if (rc) return rc;
    }
    return BS_OK;
  }
  // one cluster per state, one launch per run of consecutive states with the same parameters
  auto same = [](const bs_params& a, const bs_params& b) {
    return a.sigma1 == b.sigma1 && a.sigma2 == b.sigma2 && a.rho == b.rho && a.r == b.r && a.strike == b.strike &&
           a.w1 == b.w1 && a.w2 == b.w2 && a.payoff == b.payoff && a.strike2 == b.strike2 && a.cash == b.cash;
  };
  int i = 0;
  while (i < B) {
    SweepArgs a = {};
    a.mode = SWEEP_PROP;
    a.n_first = 0;
    a.N = 1;
    a.csteps = nsteps;
    a.slice_len = 0.0;
    a.status = g->status;
    a.tol = g_opt.krylov_tol;
    a.maxit = g_opt.krylov_maxit;
    int j = i;
    while (j < B && j - i < kMaxProp && same(p[i], p[j])) {
      a.prop[j - i] = PropItem{u_in[j], u_out[j], tau0[j]};
      ++j;
    }
    a.nprop = j - i;
    gm->n_coarse += 1;
    int rc = launch_sweep(g, make_item(p[i], 0.0, dtau_slice / nsteps), a, s);
    if (rc) return rc;
    i = j;
  }
  return BS_OK;
}

int bs_set_option(int option, double value) {
  switch (option) {
    case BS_OPT_FINE_SWEEPS:
      if (!(value == 0.0 || (value >= 2.0 && value <= 256.0)))
        return set_error(BS_ERR_ARG, "BS_OPT_FINE_SWEEPS must be 0 or in [2, 256]");
      g_opt.fine_sweeps = (int)value;
      return BS_OK;
    case BS_OPT_JACOBI_TARGET:
      if (!(value > 0.0 && value < 1.0)) return set_error(BS_ERR_ARG, "BS_OPT_JACOBI_TARGET must be in (0, 1)");
      g_opt.jacobi_target = value;
      return BS_OK;
    case BS_OPT_JACOBI_TARGET_COLD:
      if (!(value > 0.0 && value < 1.0)) return set_error(BS_ERR_ARG, "BS_OPT_JACOBI_TARGET_COLD must be in (0, 1)");
      g_opt.jacobi_target_cold = value;
      return BS_OK;
    case BS_OPT_EXTRAP_START:
      if (!(value == std::floor(value) && value >= 2.0 && value <= 1e9))
        return set_error(BS_ERR_ARG, "BS_OPT_EXTRAP_START must be an integer >= 2");
      g_opt.extrap_start = (int)value;
      return BS_OK;
    case BS_OPT_PIPELINE:
      g_opt.pipeline = value != 0.0;
      return BS_OK;
    case BS_OPT_EXTRAP_LATE:
      if (!(value == std::floor(value) && value >= 2.0 && value <= 1e9))
        return set_error(BS_ERR_ARG, "BS_OPT_EXTRAP_LATE must be an integer >= 2");
      g_opt.extrap_late = (int)value;
      return BS_OK;
    case BS_OPT_JACOBI_TARGET_EXTRAP_LATE:
      if (!(value > 0.0 && value < 1.0)) return set_error(BS_ERR_ARG, "BS_OPT_JACOBI_TARGET_EXTRAP_LATE must be in (0, 1)");
      g_opt.jacobi_target_extrap_late = value;
      return BS_OK;
    case BS_OPT_JACOBI_TARGET_EXTRAP:
      if (!(value > 0.0 && value < 1.0)) return set_error(BS_ERR_ARG, "BS_OPT_JACOBI_TARGET_EXTRAP must be in (0, 1)");
      g_opt.jacobi_target_extrap = value;
      return BS_OK;
    case BS_OPT_COARSE_VARIANT:
      if (!(value == std::floor(value) && value >= -1.0 && value < 64.0))
        return set_error(BS_ERR_ARG, "BS_OPT_COARSE_VARIANT must be -1 or a variant index");
      g_opt.coarse_variant = (int)value;
      return BS_OK;
    case BS_OPT_KRYLOV_TOL:
      if (!(value > 0.0 && value < 1.0)) return set_error(BS_ERR_ARG, "BS_OPT_KRYLOV_TOL must be in (0, 1)");
      g_opt.krylov_tol = value;
      return BS_OK;
    case BS_OPT_FINE_KRYLOV_TOL:
      if (!(value > 0.0 && value < 1.0)) return set_error(BS_ERR_ARG, "BS_OPT_FINE_KRYLOV_TOL must be in (0, 1)");
      g_opt.fine_krylov_tol = value;
      return BS_OK;
    case BS_OPT_PHASE_TIMING:
      g_opt.phase_timing = value != 0.0;
      return BS_OK;
    case BS_OPT_KRYLOV_MAXIT:
      if (!(value >= 1.0 && value <= 100000.0)) return set_error(BS_ERR_ARG, "BS_OPT_KRYLOV_MAXIT must be in [1, 1e5]");
      g_opt.krylov_maxit = (int)value;
      return BS_OK;
    case BS_OPT_FINE_TILE:
      if (!(value == 0.0 || value == 1.0 || value == 2.0))
        return set_error(BS_ERR_ARG, "BS_OPT_FINE_TILE must be 0, 1 or 2");
      g_opt.fine_tile = (int)value;
      return BS_OK;
  }
  return set_error(BS_ERR_ARG, "bs_set_option: unknown option %d", option);
}

int bs_grid_set_coarse(bs_grid* g, int Mc) {
  if (!g) return set_error(BS_ERR_ARG, "bs_grid_set_coarse: NULL grid");
  if (Mc != 0 && (Mc < 8 || Mc > g->M))
    return set_error(BS_ERR_ARG, "bs_grid_set_coarse: Mc=%d must be 0 or in [8, M=%d]", Mc, g->M);
  g->coarse_M = Mc == g->M ? 0 : Mc;
  return BS_OK;
}

int bs_fine_steps_for(int M, const bs_params* p, int N, int min_steps, double qmax, int* steps) {
  if (!steps) return set_error(BS_ERR_ARG, "bs_fine_steps_for: NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  if (M < 4 || M > 4096 || N < 1 || min_steps < 1 || !(qmax > 0.0 && qmax < 0.8))
    return set_error(BS_ERR_ARG, "bs_fine_steps_for: M=%d N=%d min_steps=%d qmax=%g", M, N, min_steps, qmax);
  const double slice = p->T / N;
  for (long long s = min_steps; s <= (1 << 20); s *= 2) {
    if (jacobi_contraction(M, *p, slice / (double)s) <= qmax) {
      *steps = (int)s;
      return BS_OK;
    }
  }
  return set_error(BS_ERR_ARG, "bs_fine_steps_for: no step count up to 2^20 reaches q <= %g", qmax);
}

int bs_coarse_variant_info(int variant, int M, int* ctas, int* threads, int* rows, int* poly, int* quad) {
  return coarse_variant_info(variant, M, ctas, threads, rows, poly, quad);
}

int bs_coarse_variant(bs_grid* g, const bs_params* p, double dtau_coarse, int* variant,
                      bs_stream stream) {
  if (!g || !variant) return set_error(BS_ERR_ARG, "bs_coarse_variant: NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  if (!(dtau_coarse > 0.0)) return set_error(BS_ERR_ARG, "bs_coarse_variant: dtau_coarse <= 0");
  *variant = -1;
  if (g->M > 256) return BS_OK;
  if (g_opt.coarse_variant >= 0) {   // forced by BS_OPT_COARSE_VARIANT
    *variant = g_opt.coarse_variant;
    return BS_OK;
  }
  if (g->coarse_variant < 0) g->coarse_variant = coarse_tuned_variant(g->device, g->M);
  if (g->coarse_variant < 0) {
    rc = coarse_autotune(g, make_item(*p, 0.0, dtau_coarse), (cudaStream_t)stream, kAutotuneSteps, nullptr);
    if (rc) return rc;
  }
  *variant = g->coarse_variant;
  return BS_OK;
}

int bs_grid_stats(bs_grid* g, int* krylov_iters_max, int* krylov_failed, int* krylov_iters_total,
                  int* krylov_solves) {
  if (!g) return set_error(BS_ERR_ARG, "bs_grid_stats: NULL grid");
  int h[kStatusWords] = {};
  BS_CUDA_TRY(cudaMemcpy(h, g->status, kStatusWords * sizeof(int), cudaMemcpyDeviceToHost));
  BS_CUDA_TRY(cudaMemset(g->status, 0, kStatusWords * sizeof(int)));
  if (krylov_iters_max) *krylov_iters_max = h[1];
  if (krylov_failed) *krylov_failed = h[0];   // bit 0: iteration cap, bit 1: exchange timeout
  if (krylov_iters_total) *krylov_iters_total = h[2];
  if (krylov_solves) *krylov_solves = h[3];
  return BS_OK;
}

int bs_phase_stats(bs_grid* g, double* fine_ms, int* fine_launches, double* coarse_ms,
                   int* coarse_launches, int* other_launches) {
  if (!g) return set_error(BS_ERR_ARG, "bs_phase_stats: NULL grid");
  if (fine_ms) *fine_ms = g->ms_fine;
  if (coarse_ms) *coarse_ms = g->ms_coarse;
  if (fine_launches) *fine_launches = g->n_fine;
  if (coarse_launches) *coarse_launches = g->n_coarse;
  if (other_launches) *other_launches = g->n_other;
  g->ms_fine = g->ms_coarse = 0.0;
  g->n_fine = g->n_coarse = g->n_other = 0;
  return BS_OK;
}

// CUDA events bracketing one launch group on the caller's stream (BS_OPT_PHASE_TIMING).
struct PhaseTimer {
  cudaEvent_t e[2] = {nullptr, nullptr};
  bool on = false;
  int begin(cudaStream_t s) {
    if (!on) return BS_OK;
    if (!e[0]) {
      BS_CUDA_TRY(cudaEventCreate(&e[0]));
      BS_CUDA_TRY(cudaEventCreate(&e[1]));
    }
    BS_CUDA_TRY(cudaEventRecord(e[0], s));
    return BS_OK;
  }
  int end(cudaStream_t s) {
    if (on) BS_CUDA_TRY(cudaEventRecord(e[1], s));
    return BS_OK;
  }
  // after the stream has been synchronised
  double elapsed() const {
    float ms = 0.f;
    if (on && e[0]) cudaEventElapsedTime(&ms, e[0], e[1]);
    return (double)ms;
  }
  ~PhaseTimer() {
    if (e[0]) cudaEventDestroy(e[0]);
    if (e[1]) cudaEventDestroy(e[1]);
  }
};

int parareal_sweep_range(const bs_grid* gc, const bs_params* p, int N, int coarse_steps, int k, int n_begin,
                         int n_end, float* U, const float* Fb, float* Gold, double* norms, bs_stream stream) {
  bs_grid* g = const_cast<bs_grid*>(gc);
  if (!g || !U || !Gold || !norms || (k >= 0 && !Fb))
    return set_error(BS_ERR_ARG, "parareal_sweep_range: NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  if (N < 1 || coarse_steps < 1 || !(p->T > 0.0) || k < -1 || k >= N || n_begin < 0 || n_end > N ||
      n_begin >= n_end || (k >= 0 && n_begin < k))
    return set_error(BS_ERR_ARG, "parareal_sweep_range: N=%d coarse_steps=%d k=%d range [%d, %d)", N,
                     coarse_steps, k, n_begin, n_end);
  const double slice = p->T / N;
  const ItemDesc dc = make_item(*p, 0.0, slice / coarse_steps);
  SweepArgs a = {};
  a.N = N;
  a.csteps = coarse_steps;
  a.slice_len = slice;
  a.U = U;
  a.Fb = Fb;
  a.Gold = Gold;
  a.norms = norms;
  a.defect = g->dscal;   // scratch: the caller forms the defect from the norms
  a.status = g->status;
  a.tol = g_opt.krylov_tol;
  a.maxit = g_opt.krylov_maxit;
  a.mode = k < 0 ? SWEEP_INIT : SWEEP_ITER;
  a.n_first = k < 0 ? 0 : k;
  a.n_begin = n_begin;
  a.n_end = n_end;
  cudaStream_t s = (cudaStream_t)stream;
  if (g->coarse_M > 0 && g->coarse_M != g->M) {
    g->n_coarse += (n_end - n_begin) * resampled_launches_per_slice() + 1;
    return resampled_sweep(g, dc, a, s);
  }
  g->n_coarse += 1;
  return launch_sweep(g, dc, a, s);
}

int parareal_solve(const bs_grid* gc, const bs_params* p, int N, int fine_steps, int coarse_kind,
                   int coarse_steps, const bs_pino* net, double tol, int Kmax, float* u_out,
                   int* k_done, double* defect_hist, bs_stream stream) {
  bs_grid* g = const_cast<bs_grid*>(gc);
  if (!g || !u_out || !k_done) return set_error(BS_ERR_ARG, "parareal_solve: NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  const bool user_u0 = (coarse_kind & BS_PARAREAL_USER_U0) != 0;
  coarse_kind &= ~BS_PARAREAL_USER_U0;
  if (N < 1 || fine_steps < 1 || Kmax < 0 || Kmax > N || !(p->T > 0.0))
    return set_error(BS_ERR_ARG, "parareal_solve: N=%d fine_steps=%d Kmax=%d T=%g", N, fine_steps,
                     Kmax, p->T);
  if (coarse_kind != BS_COARSE_NUM && coarse_kind != BS_COARSE_PINO)
    return set_error(BS_ERR_ARG, "parareal_solve: coarse kind %d unsupported", coarse_kind);
  const bool pino = coarse_kind == BS_COARSE_PINO;
  if (pino && (rc = pino_check(net, g->M))) return rc;
  if (!pino && coarse_steps < 1) return set_error(BS_ERR_ARG, "parareal_solve: coarse_steps < 1");
  if (pino) coarse_steps = 1;
  cudaStream_t s = (cudaStream_t)stream;
  const int M = g->M;
  const size_t MM = (size_t)M * M;
  const double slice = p->T / N;
  const double dtau_f = slice / fine_steps;
  const int sweeps = grid_sweeps(g, *p, dtau_f);
  const int sweeps0 = grid_sweeps(g, *p, dtau_f, START_COLD);
  const int sweepsx = grid_sweeps(g, *p, dtau_f, START_EXTRAP);
  const int sweepsxl = grid_sweeps(g, *p, dtau_f, START_EXTRAP_LATE);
  const bool krylov_f = sweeps == 0;   // Jacobi bound >= 0.8: F by BiCGSTAB per step
  // numerical G on this grid: F overlapped with the chunked coarse sweep (Krylov F of grids
  // beyond one cluster shares the coarse solver's global workspace and stays sequential)
  if (!pino && g_opt.pipeline && pipeline_eligible(N) && !(krylov_f && g->M > 256))
    return parareal_pipelined(g, p, N, fine_steps, coarse_steps, tol, Kmax, u_out, user_u0, k_done,
                              defect_hist, s);
  const size_t part_bytes = pino ? pino_partials_bytes(M, N) : 0;
  rc = ensure(g->ws_par, sizeof(float) * 2 * (size_t)N * MM + sizeof(double) * 2 * (N + 1) + part_bytes);
  if (rc) return rc;
  float* Fb = (float*)g->ws_par.ptr;
  float* Gold = Fb + (size_t)N * MM;
  double* norms = (double*)(Gold + (size_t)N * MM);
  double* partials = norms + 2 * (N + 1);
  bs_pino* pnet = const_cast<bs_pino*>(net);
  // one serial coarse sweep (numerical: one persistent cluster kernel; PINO: per slice the
  // network kernels and the correction), counted into the grid's launch statistics
  const bool resampled = !pino && g->coarse_M > 0 && g->coarse_M != g->M;
  auto sweep = [&](const ItemDesc& d, const SweepArgs& sa) -> int {
    if (resampled) {
      for (int n = sa.n_first; n < sa.N; ++n)
        g->n_coarse += (sa.mode == SWEEP_ITER && n == sa.n_first) ? 1 : resampled_launches_per_slice();
      g->n_coarse += 1;
      return resampled_sweep(g, d, sa, s);
    }
    if (!pino) {
      g->n_coarse += 1;
      return launch_sweep(g, d, sa, s);
    }
    const int per_slice = pino_launches_per_step(pnet, g->M);
    for (int n = sa.n_first; n < sa.N; ++n)
      g->n_coarse += (sa.mode == SWEEP_ITER && n == sa.n_first) ? 1 : per_slice;
    g->n_coarse += 1;
    return pino_sweep(pnet, g, d, sa, partials, s);
  };
  BS_CUDA_TRY(cudaMemsetAsync(g->status, 0, kStatusWords * sizeof(int), s));
  PhaseTimer tf, tc;
  tf.on = tc.on = g_opt.phase_timing != 0;

  ItemDesc dc = make_item(*p, 0.0, slice / coarse_steps);
  if (!user_u0) {
    rc = launch_payoff(g, dc, u_out, s);
    if (rc) return rc;
    g->n_other += 1;
  }
  SweepArgs a = {};
  a.N = N;
  a.csteps = coarse_steps;
  a.slice_len = slice;
  a.U = u_out;
  a.Fb = Fb;
  a.Gold = Gold;
  a.norms = norms;
  a.defect = g->dscal;
  a.status = g->status;
  a.tol = g_opt.krylov_tol;
  a.maxit = g_opt.krylov_maxit;
  a.mode = SWEEP_INIT;
  a.n_first = 0;
  if ((rc = tc.begin(s))) return rc;
  rc = sweep(dc, a);
  if (rc) return rc;
  if ((rc = tc.end(s))) return rc;
  double ms_c = 0.0, ms_f = 0.0;
  if (tc.on) {
    BS_CUDA_TRY(cudaStreamSynchronize(s));
    ms_c += tc.elapsed();
  }

  std::vector<ItemDesc> items((size_t)N);
  int k = 0;
  int status = BS_ERR_MAXITER;
  for (; k < Kmax; ++k) {
    // F on slices k..N-1 (slices below k are already exact)
    const int B = N - k;
    for (int n = k; n < N; ++n) {
      ItemDesc d = make_item(*p, n * slice, dtau_f);
      d.in = u_out + (size_t)n * MM;
      d.out = Fb + (size_t)n * MM;
      d.sweeps = sweeps;
      d.sweeps0 = sweeps0;
      d.sweepsx = sweepsx;
      d.sweepsxl = sweepsxl;
      items[(size_t)(n - k)] = d;
    }
    if ((rc = tf.begin(s))) return rc;
    if (krylov_f) {
      rc = launch_krylov_fine(g, items.data(), B, fine_steps, s);
    } else {
      rc = launch_fine(g, items.data(), B, fine_steps, s);
      g->n_fine += fine_launches(g, items.data(), B, fine_steps);
    }
    if (rc) return rc;
    if ((rc = tf.end(s))) return rc;
    a.mode = SWEEP_ITER;
    a.n_first = k;
    if ((rc = tc.begin(s))) return rc;
    rc = sweep(dc, a);
    if (rc) return rc;
    if ((rc = tc.end(s))) return rc;
    double host[1];
    int hstat = 0;
    BS_CUDA_TRY(cudaMemcpyAsync(host, g->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaMemcpyAsync(&hstat, g->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaStreamSynchronize(s));
    if (pino) {
      int perr = 0;
      if ((rc = pino_error_flag(pnet, &perr))) return rc;
      if (perr) return set_error(BS_ERR_CUDA, "parareal_solve: a PINO tensor-core tile timed out");
    }
    ms_f += tf.elapsed();
    ms_c += tc.elapsed();
    if (defect_hist) defect_hist[k] = host[0];
    if (hstat) {
      *k_done = k + 1;
      g->ms_fine += ms_f;
      g->ms_coarse += ms_c;
      if (hstat & 2)
        return set_error(BS_ERR_CUDA, "parareal_solve: a cluster exchange of the coarse sweep timed out");
      return set_error(BS_ERR_NOCONV, "parareal_solve: a coarse BiCGSTAB solve hit its iteration cap");
    }
    if (host[0] <= tol) {
      ++k;
      status = BS_OK;
      break;
    }
  }
  *k_done = k;
  g->ms_fine += ms_f;
  g->ms_coarse += ms_c;
  if (Kmax == 0) BS_CUDA_TRY(cudaStreamSynchronize(s));
  // after N iterations every slice is exact (serial fine stepping), whatever the last defect
  if (status == BS_ERR_MAXITER && k < N)
    return set_error(BS_ERR_MAXITER, "parareal_solve: tol %g not met after %d iterations", tol, k);
  return BS_OK;
}

int pino_physics_loss(const bs_grid* g, const bs_params* p, const float* const* u_pred,
                      const float* const* u_prev, const double* dtau, int B, double* loss,
                      float* const* grad, bs_stream stream) {
  if (!g || !p || !u_pred || !u_prev || !dtau || !loss)
    return set_error(BS_ERR_ARG, "pino_physics_loss: NULL argument");
  if (B < 1) return set_error(BS_ERR_ARG, "pino_physics_loss: B=%d", B);
  for (int b = 0; b < B; ++b) {
    int rc = check_params(&p[b]);
    if (rc) return rc;
    if (!u_pred[b] || !u_prev[b] || (grad && !grad[b]))
      return set_error(BS_ERR_ARG, "pino_physics_loss: NULL state %d", b);
    if (grad && (grad[b] == u_pred[b] || grad[b] == u_prev[b]))
      return set_error(BS_ERR_ARG, "pino_physics_loss: grad[%d] aliases an input", b);
    if (!(dtau[b] > 0.0)) return set_error(BS_ERR_ARG, "pino_physics_loss: dtau[%d] <= 0", b);
  }
  return launch_physics_loss(g, p, u_pred, u_prev, dtau, B, loss, grad, (cudaStream_t)stream);
}

}  // extern "C"
