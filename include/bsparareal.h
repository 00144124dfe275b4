/*
 * bsparareal.h -- C ABI of the GB300 (sm_103a) Parareal library for the two-asset
 * Black-Scholes equation.
 *
 * Method: Ibrahim, Goetschel, Ruprecht, "Space-time parallel scaling of Parareal with a
 * physics-informed Fourier Neural Operator coarse propagator applied to the Black-Scholes
 * equation" (PASC'25).  Section and equation names below refer to that paper.
 *
 * Conventions
 *  - Every entry point returns an int status: BS_OK (0) or a negative BS_ERR_* code.
 *    bs_last_error() returns a message for the last failure on the calling host thread.
 *  - Grids are square: M nodes per axis including both ends, x_i = i*xmax/(M-1)
 *    (the paper uses dx = dy, Sec. 3.2).  A state is a row-major float array u[j*M + i]
 *    with j the y (second asset) index and i the x (first asset) index.
 *  - Device pointers are owned by the caller.  Handles (bs_grid, bs_pino) are owned by
 *    the library and released with the matching *_destroy call.
 *  - Work is enqueued on the caller's CUDA stream (a cudaStream_t / CUstream; NULL is the
 *    legacy default stream) and is asynchronous unless a function says "synchronous".
 *  - A handle may be used by one stream at a time: internal workspace is reused between
 *    calls in stream order.
 *  - Time is tau = T - t (eq. bse_change_variable); tau = 0 is the payoff.
 */
#ifndef BSPARAREAL_H
#define BSPARAREAL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* bs_stream;      /* same type as cudaStream_t */

typedef struct bs_grid bs_grid;             /* opaque: grid size + internal workspace */
typedef struct bs_pino bs_pino;             /* opaque: PINO weights resident on the GPU */

enum {
  BS_OK = 0,
  BS_ERR_ARG = -1,      /* invalid argument (NULL pointer, size, unsupported combination) */
  BS_ERR_CUDA = -2,     /* a CUDA runtime call failed; message has the CUDA error string */
  BS_ERR_NOCONV = -3,   /* an inner Krylov solve hit its iteration cap */
  BS_ERR_MAXITER = -4,  /* Parareal reached Kmax < N without meeting tol (results still valid) */
  BS_ERR_OOM = -5,      /* device allocation failed */
  BS_ERR_FILE = -6      /* weight file missing, truncated or malformed */
};

enum {
  BS_PAYOFF_BASKET = 0,          /* max(w1*x + w2*y - K, 0) */
  BS_PAYOFF_EXCHANGE = 1,        /* max(x - y, 0) */
  BS_PAYOFF_CALL1 = 2,           /* max(x - K, 0): one-asset call, y is a spectator */
  BS_PAYOFF_CASH_OR_NOTHING = 3  /* c if x >= S1 and y >= S2 else 0 (Sec. 3.2) */
};

enum { BS_COARSE_NUM = 0, BS_COARSE_PINO = 1 };
/* Flag or-ed into parareal_solve's coarse_kind: u_out[0..M*M) already holds the initial state
 * u(tau = 0) on entry (for example a tabulated payoff uploaded by the caller); without it the
 * payoff of p is written there.  The far-field data still follow p->payoff. */
enum { BS_PARAREAL_USER_U0 = 0x100 };

/* Model and payoff parameters (eq. bse: sigma1, sigma2, rho, r; Sec. 3.2 payoff). */
typedef struct {
  double sigma1, sigma2;   /* volatilities, > 0 */
  double rho;              /* correlation, |rho| < 1 */
  double r;                /* risk-free rate, >= 0 */
  double T;                /* maturity (tau runs over [0, T]) */
  double strike;           /* K (basket, one-asset call) or S1 (cash-or-nothing) */
  double w1, w2;           /* basket weights */
  int payoff;              /* BS_PAYOFF_* */
  int reserved;            /* must be 0 */
  double strike2;          /* S2 (cash-or-nothing) */
  double cash;             /* c  (cash-or-nothing) */
} bs_params;

/* Message describing the last failure on this host thread ("" if none). */
const char* bs_last_error(void);

/* Number of device allocations (cudaMalloc, cudaMallocAsync) and pinned host allocations the
 * library has made in this process, into *count (a diagnostic: it lets a caller check that a
 * call allocated nothing).  Host-only.  BS_ERR_ARG for a NULL pointer. */
int bs_device_allocations(long long* count);

/* Create a grid of M x M nodes on [0, xmax]^2 (4 <= M <= 4096, xmax > 0).  Selects the
 * device that is current on the calling thread.  *g receives the handle. */
int bs_grid_create(int M, double xmax, bs_grid** g);
int bs_grid_destroy(bs_grid* g);

/* Write the payoff u(tau = 0) (Sec. 3.2; reading of the boundary: the far edges carry the
 * same closed-form data as at tau = 0) into the device array u[M*M].  Asynchronous. */
int bs_payoff(const bs_grid* g, const bs_params* p, float* u, bs_stream stream);

/* Fine propagator F of Sec. 3.1 for B independent states at once (eq. fd with implicit
 * Euler, Sec. 3.2).  For item b, nsteps implicit-Euler steps of size dtau[b] are taken
 * from tau0[b]:  (I - dtau R_h) u^{m+1} = u^m, with the 9-point centred operator R_h of
 * eq. (fd), the PDE row itself on x = 0 and y = 0 (its coefficients vanish there), and
 * far-field Dirichlet data g(x, y, tau^{m+1}) on x = xmax and y = xmax (exchange: Margrabe;
 * basket: max(w1 x + w2 y - K e^{-r tau}, 0); one-asset: Black-Scholes call; cash-or-nothing:
 * eq. solution).  Each implicit system is solved in FP32 by Jacobi sweeps whose count
 * follows from the Gershgorin contraction q of the system (q < 0.8), or, for items with
 * q >= 0.8, by BiCGSTAB per step to BS_OPT_FINE_KRYLOV_TOL; the state is carried as a
 * compensated (hi, lo) float pair across steps and rounded to float on output.
 *
 *  p[B], tau0[B], dtau[B]  host arrays (per-item parameters)
 *  u_in[B], u_out[B]       host arrays of device pointers to float[M*M]; u_out[b] may
 *                          equal u_in[b] (in place)
 *  nsteps >= 0, 1 <= B
 * Results for an item do not depend on B or on the other items.  Asynchronous: only
 * enqueues kernels, so after one call with the same grid and batch it can be captured into
 * a CUDA graph.
 * Errors: BS_ERR_ARG (NULL, B < 1, dtau <= 0), BS_ERR_CUDA.  A BiCGSTAB step that hits its
 * iteration cap is reported by the next synchronous call on this grid as BS_ERR_NOCONV. */
int fine_propagate_batched(const bs_grid* g, const bs_params* p,
                           const float* const* u_in, float* const* u_out,
                           const double* tau0, const double* dtau, int nsteps, int B,
                           bs_stream stream);

/* Three assets: eq. (bse_general) with n = 3 (the paper treats n = 2; its general form
 * extends eq. (fd) to a 19-point stencil: second differences along each axis, four-point
 * cross differences for each pair, centred first differences).  Grid: M nodes per axis
 * including both ends on [0, xmax]^3, u[(k*M + j)*M + i] with i the index of asset 1. */
typedef struct {
  double sigma[3];   /* volatilities, > 0 */
  double rho[3];     /* correlations rho_12, rho_13, rho_23 (a positive definite matrix) */
  double r;          /* risk-free rate, >= 0 */
  double strike;     /* K of the basket */
  double w[3];       /* basket weights */
  int payoff;        /* BS_PAYOFF_BASKET: max(w.x - K, 0), far faces max(w.x - K e^{-r tau}, 0);
                        BS_PAYOFF_EXCHANGE: max(x_1 - x_2, 0), far faces Margrabe in (x_1, x_2) */
  int reserved;      /* must be 0 */
} bs_params3;

/* The payoff of p on the M^3 grid into device float[M^3] u.  Asynchronous.
 * Errors: BS_ERR_ARG (M outside [4, 128], invalid parameters, NULL), BS_ERR_CUDA. */
int bs_payoff3(int M, double xmax, const bs_params3* p, float* u, bs_stream stream);

/* F for three assets on B states at once: nsteps implicit-Euler steps of size dtau from
 * tau0[b], (I - dtau R_h) u^{m+1} = u^m with the 19-point R_h and far-face Dirichlet data
 * at tau^{m+1}; solved by Jacobi sweeps (count from the Gershgorin bound q of the system,
 * q < 0.8) in FP32 with a compensated (hi, lo) state.  u_in[b], u_out[b]: device
 * float[M^3] (may alias).  Allocates its workspace stream-ordered (5 M^3 floats per state).
 * Asynchronous.  Results for a state do not depend on B or on the other states.
 * Errors: BS_ERR_ARG (as bs_payoff3; NULL pointers, B < 1, dtau <= 0, q >= 0.8),
 * BS_ERR_CUDA. */
int fine_propagate3(int M, double xmax, const bs_params3* p, const float* const* u_in, float* const* u_out,
                    const double* tau0, int B, double dtau, int nsteps, bs_stream stream);

/* G for three assets, one state: nsteps implicit-Euler steps of size dtau_slice/nsteps from
 * tau0 with the 19-point operator, each solved by BiCGSTAB on the Jacobi-scaled increment
 * system in FP32 to BS_OPT_KRYLOV_TOL (any step size).  u_in, u_out: device float[M^3] (may
 * alias).  Allocates its workspace stream-ordered (12 M^3 floats).  Synchronous (the host
 * checks convergence every four iterations).  Errors: BS_ERR_ARG (as bs_payoff3, NULL, dtau_slice <= 0,
 * nsteps < 1), BS_ERR_NOCONV (BS_OPT_KRYLOV_MAXIT reached), BS_ERR_CUDA. */
int coarse_propagate3(int M, double xmax, const bs_params3* p, const float* u_in, float* u_out,
                      double tau0, double dtau_slice, int nsteps, bs_stream stream);

/* Parareal (eq. parareal) for three assets on [0, T] with N slices: F = fine_steps Jacobi
 * steps per slice (fine_propagate3), G = coarse_steps steps of the same scheme solved by
 * BiCGSTAB (coarse_propagate3); iterate until delta_k <= tol (reading c5, FP64 norms) or
 * k = Kmax.
 *  u_out        device float[(N+1)*M^3]: u_0 (the payoff) .. u_N on return
 *  k_done       host int: iterations performed;  defect_hist  host double[Kmax] or NULL
 * Synchronous.  Returns BS_OK (converged, or k_done = N: every slice exact), BS_ERR_MAXITER
 * (tol not met within Kmax < N), BS_ERR_ARG (as fine_propagate3, or N, steps, Kmax out of
 * range), BS_ERR_NOCONV (a coarse BiCGSTAB solve hit its cap), BS_ERR_CUDA. */
int parareal_solve3(int M, double xmax, const bs_params3* p, double T, int N, int fine_steps,
                    int coarse_steps, double tol, int Kmax, float* u_out, int* k_done,
                    double* defect_hist, bs_stream stream);

/* Coarse propagator G of Sec. 3.1 for one state.
 *  kind = BS_COARSE_NUM: nsteps implicit-Euler steps of size dtau_slice/nsteps with the
 *    same operator as F (Sec. 3.2: the numerical coarse model is the same discretisation
 *    with a larger step), solved by BiCGSTAB in FP32 (the paper runs its coarse models in
 *    single precision, Sec. 4.1).  net must be NULL.
 *  kind = BS_COARSE_PINO: one evaluation of the PINO (Sec. 3.4-3.5) mapping u(tau0) and
 *    the interval (tau0, tau0 + dtau_slice) to u(tau0 + dtau_slice); nsteps is ignored.
 * u_in, u_out: device float[M*M] (may alias).  Asynchronous: only enqueues kernels, so
 * after one call on this grid (which picks the band variant) it can be captured into a CUDA
 * graph.
 * Errors: BS_ERR_ARG, BS_ERR_CUDA.  A Krylov solve that hits its iteration cap is reported
 * by the next synchronous call on this grid as BS_ERR_NOCONV. */
int coarse_propagate(const bs_grid* g, int kind, const bs_pino* net, const bs_params* p,
                     const float* u_in, float* u_out, double tau0, double dtau_slice,
                     int nsteps, bs_stream stream);

/* Coarse propagator G for B independent states at once (the same grid): as coarse_propagate
 * for item b with p[b], u_in[b] -> u_out[b], starting at tau0[b], over dtau_slice.
 *  kind = BS_COARSE_NUM: one thread-block cluster per state, one launch per run of
 *    consecutive items with equal parameters (at most 64 states each); on a grid with a
 *    coarse grid (bs_grid_set_coarse) the states are propagated one after another.
 *  kind = BS_COARSE_PINO: the network on up to 128 states per launch chain (every GEMM of the
 *    chain carries the states as extra rows or grid blocks); nsteps is ignored.
 * For concurrent solves or requests whose coarse steps are due together (a slice of each).
 * Results for an item do not depend on B or on the other items (bitwise).
 *  p[B], u_in[B], u_out[B], tau0[B]  host arrays (u_in/u_out: device float[M*M], may alias)
 * Asynchronous.  Errors: BS_ERR_ARG (NULL, B < 1, dtau_slice <= 0, nsteps < 1 for NUM, a
 * network for NUM or none for PINO), BS_ERR_OOM, BS_ERR_CUDA. */
int coarse_propagate_batched(const bs_grid* g, int kind, const bs_pino* net, const bs_params* p,
                             const float* const* u_in, float* const* u_out, const double* tau0,
                             double dtau_slice, int nsteps, int B, bs_stream stream);

/* Load PINO weights (Sec. 3.5: FNO backbone with lifting, L Fourier layers, projection;
 * batch norm folded into the pointwise weights) from a little-endian file written by
 * paper_2404_02521_gb300/pino_train.py.  Weights are converted to BF16 on load.
 * Synchronous.  Errors: BS_ERR_FILE, BS_ERR_ARG, BS_ERR_OOM. */
int pino_load(const char* path, bs_pino** net);
int pino_destroy(bs_pino* net);

/* PDE term of the PINO training loss (Sec. 3.5, eq. bs_totalloss, MSE_f) for B predicted
 * slices on the device.  A prediction u_pred[b] of u(tau + dtau[b]) from u_prev[b] = u(tau) is
 * scored at the collocation points that carry a PDE row, 0 <= i, j <= M-2 (the far edges hold
 * Dirichlet data), by the residual of eq. (bse_change_variable) discretised by eq. (fd) with
 * the slice as one implicit-Euler step:
 *   r = (u_pred - u_prev) / dtau - R_h u_pred,     loss[b] = sum r^2 / (M-1)^2,
 * and, where grad is given, grad[b] = d loss[b] / d u_pred[b] on every node (the adjoint of the
 * residual: 2/(M-1)^2 (r / dtau - R_h^T r)), so that a training loop can back-propagate it.
 *  p[B], dtau[B]          host arrays (per-item parameters and slice lengths, dtau > 0)
 *  u_pred[B], u_prev[B]   host arrays of device pointers to float[M*M] (read only)
 *  loss                   device double[B], overwritten (FP64 sums of FP32 residuals; the
 *                         order of the block sums may vary, so the last bits may too)
 *  grad                   NULL, or a host array of B device pointers to float[M*M] (written;
 *                         must not alias u_pred or u_prev)
 * Asynchronous.  Errors: BS_ERR_ARG (NULL, B < 1, dtau <= 0, bad parameters), BS_ERR_CUDA. */
int pino_physics_loss(const bs_grid* g, const bs_params* p, const float* const* u_pred,
                      const float* const* u_prev, const double* dtau, int B, double* loss,
                      float* const* grad, bs_stream stream);

/* Parareal, eq. (parareal): u_{n+1}^{k+1} = G(u_n^{k+1}) + F(u_n^k) - G(u_n^k) on N slices
 * of [0, p->T], starting from the payoff and one serial coarse sweep.  F takes fine_steps
 * implicit-Euler steps per slice; G is the numerical model with coarse_steps steps per slice
 * or the PINO.  Iterates until delta_k = max_n ||u_n^{k+1} - u_n^k||_2 / max_n ||u_n^{k+1}||_2
 * <= tol (FP64 reductions on the GPU) or k = Kmax (Kmax <= N; Kmax = N reproduces the serial
 * fine solution bitwise).
 *  u_out        device float[(N+1)*M*M]: u_0..u_N on return
 *  k_done       host int: iterations performed
 *  defect_hist  host double[Kmax] (may be NULL): delta_k per iteration
 * Synchronous (returns after the stream has drained).
 * Returns BS_OK on convergence (delta_k <= tol, or k_done = N: after N iterations every slice
 * is serial fine stepping exactly), BS_ERR_MAXITER if tol was not met within Kmax < N (u_out
 * then holds the last iterate), BS_ERR_NOCONV if a coarse Krylov solve failed. */
int parareal_solve(const bs_grid* g, const bs_params* p, int N, int fine_steps,
                   int coarse_kind, int coarse_steps, const bs_pino* net, double tol,
                   int Kmax, float* u_out, int* k_done, double* defect_hist,
                   bs_stream stream);

/* One serial coarse sweep of eq. (parareal) over the slices [n_begin, n_end) of a solve with N
 * slices of [0, p->T], numerical G (coarse_steps implicit steps per slice, on the grid's
 * coarse grid if bs_grid_set_coarse set one).  For drivers that partition the slices over
 * several GPUs: each GPU sweeps its own contiguous range once it holds u_{n_begin} (the
 * serial sweep's hand-off), and the Parareal defect is formed across GPUs from the norms.
 *  k = -1: the initial sweep, U[n+1] = Gold[n] = G(U[n]);
 *  k >= 0: iteration k, U[n+1] = Fb[n] + (G(U[n]) - Gold[n]), Gold[n] = G(U[n]) (reading c6),
 *          with n_begin >= k; slice k's G is Gold[k] unchanged (u_k is exact after k
 *          iterations), so for n_begin == k it is not recomputed.
 *  U     device float[(N+1)*M*M], Fb and Gold device float[N*M*M]: full-size arrays indexed by
 *        the global slice number; only U[n_begin .. n_end], Fb[n_begin .. n_end-1] and
 *        Gold[n_begin .. n_end-1] are read or written.
 *  norms device double[2*(N+1)]: for n in (n_begin, n_end], norms[2n] = ||U[n]||^2 and
 *        norms[2n+1] = ||U[n]_new - U[n]_old||^2 (FP64 reductions; 0 for k = -1).  The defect of
 *        iteration k is sqrt(max_{n > k} norms[2n+1]) / sqrt(max_{n >= 1} norms[2n]) over all
 *        slices of all GPUs (reading c5).
 * Asynchronous (enqueues kernels on `stream`).  Errors: BS_ERR_ARG (NULL, ranges), BS_ERR_CUDA;
 * a coarse BiCGSTAB solve that hits its cap is reported by the next bs_grid_stats call. */
int parareal_sweep_range(const bs_grid* g, const bs_params* p, int N, int coarse_steps, int k, int n_begin,
                         int n_end, float* U, const float* Fb, float* Gold, double* norms, bs_stream stream);

/* Number of Jacobi sweeps F uses per implicit step for these parameters and step size on
 * this grid, by how the step's solve starts: first_step = 1 for the first step of a launch
 * (zero increment), 0 for a step started from the previous increment (the second step; every
 * step before BS_OPT_EXTRAP_START), 2 for a step started from the extrapolation of the two
 * previous increments, 3 for such a step from BS_OPT_EXTRAP_LATE on.
 * 0 if Jacobi does not apply or first_step is out of range.  Host-only helper. */
int bs_fine_sweeps(const bs_grid* g, const bs_params* p, double dtau, int first_step);

/* Solver options (process-wide; set them before launching work, not concurrently with it).
 *  BS_OPT_FINE_SWEEPS    Jacobi sweeps per fine step, >= 2; 0 = derive from the contraction
 *                        bound (default)
 *  BS_OPT_JACOBI_TARGET  the derived sweep count of a warm-started step (each step starts
 *                        from the previous step's increment) makes q^sweeps <= this
 *                        (default 2^-10)
 *  BS_OPT_JACOBI_TARGET_COLD  the same for the first step of a launch, which starts from a
 *                        zero increment (default 2^-22)
 *  BS_OPT_JACOBI_TARGET_EXTRAP  the same for the steps of a launch from BS_OPT_EXTRAP_START
 *                        on, which start from the extrapolation 2 d_{m-1} - d_{m-2} of the
 *                        previous two increments (default 2^-6).  For a mode with
 *                        dtau*lambda = a the extrapolation error is a^2 |d| against a |d| for
 *                        the warm start: much smaller for slow modes, not for stiff ones
 *  BS_OPT_EXTRAP_START   index (>= 2) of the first step of a launch that starts from the
 *                        extrapolated guess; the steps before it are warm-started (default 2)
 *  BS_OPT_EXTRAP_LATE    index of the first step that uses the late target below (default
 *                        16: stiff modes, whose extrapolation is poor, decay by at least a
 *                        factor 2 per step and are gone by then)
 *  BS_OPT_JACOBI_TARGET_EXTRAP_LATE  the extrapolated-start target from BS_OPT_EXTRAP_LATE on
 *                        (default 0.5: two sweeps, the structural minimum, wherever q <= 0.707;
 *                        at the 1024 x 1024 large-solve step, q = 0.63, the error against the FP64
 *                        oracle after 1024 steps is 6e-8 max|V| with two, three or five sweeps)
 *  BS_OPT_PIPELINE       1 (default): parareal_solve with the numerical G (on the state grid
 *                        or on a coarse grid) and N >= 8 splits each coarse sweep into chunks
 *                        of consecutive slices (as many as F runs in one wave beside the
 *                        sweep's cluster, at most a quarter of them) and runs F for a chunk on
 *                        a second stream as soon as the sweep has produced its input states
 *                        (F of the next iteration speculatively, before the defect is known,
 *                        where a state fits one cluster or from the second iteration on); 0: F
 *                        and the sweep alternate as whole phases
 *  BS_OPT_KRYLOV_TOL     relative residual at which a coarse BiCGSTAB solve (numerical G) stops
 *                        (1e-5; G need only be a deterministic approximation of F)
 *  BS_OPT_FINE_KRYLOV_TOL  ... a fine BiCGSTAB step (F for step sizes beyond Jacobi) stops (1e-6)
 *  BS_OPT_KRYLOV_MAXIT   iteration cap of a coarse BiCGSTAB solve (default 400)
 *  BS_OPT_PHASE_TIMING   1: parareal_solve brackets its fine and coarse launches with CUDA
 *                        events on the caller's stream (read back by bs_phase_stats); 0: off
 *  BS_OPT_COARSE_VARIANT  -1 (default): the coarse sweep of grids with M <= 256 uses the band
 *                        variant measured fastest for that M (bs_coarse_variant); k >= 0:
 *                        always variant k (it must fit the grid, else the launch fails with
 *                        BS_ERR_ARG).  Variants differ in work split and reduction order
 *                        and, where their shared memory allows, use a polynomial
 *                        preconditioner and quadratic initial-guess extrapolation (all solve
 *                        the same systems to the same Krylov tolerance).
 *  BS_OPT_FINE_TILE      layout of the fine stepper: 0 (default) per launch, the one with less
 *                        work counted in waves of co-resident clusters; 1 or 2 forces one.
 *                        Grids with M > 256 run as overlapping cluster tiles: layout 1 on
 *                        regions of 256 x 256 nodes (8 CTAs, up to 24 sweeps per launch),
 *                        layout 2 on regions of 288 x 288 (9 CTAs, up to 16 sweeps).  Grids
 *                        with 128 < M <= 256 keep a state in one cluster: layout 1 on 8 CTAs
 *                        of 32 rows, layout 2 on 16 CTAs of 16 rows (one CTA per SM; faster
 *                        for one or a few states).  Smaller grids have one layout.  All
 *                        layouts give the same result bit for bit.
 * Returns BS_OK or BS_ERR_ARG for an unknown option or an out-of-range value. */
enum { BS_OPT_FINE_SWEEPS = 0, BS_OPT_JACOBI_TARGET = 1, BS_OPT_KRYLOV_TOL = 2,
       BS_OPT_KRYLOV_MAXIT = 3, BS_OPT_PHASE_TIMING = 4, BS_OPT_JACOBI_TARGET_COLD = 5,
       BS_OPT_COARSE_VARIANT = 6, BS_OPT_JACOBI_TARGET_EXTRAP = 7, BS_OPT_EXTRAP_START = 8,
       BS_OPT_EXTRAP_LATE = 9, BS_OPT_JACOBI_TARGET_EXTRAP_LATE = 10, BS_OPT_PIPELINE = 11,
       BS_OPT_FINE_KRYLOV_TOL = 12, BS_OPT_FINE_TILE = 13 };
int bs_set_option(int option, double value);

/* Numerical coarse propagator on a coarser grid (the resolution change of Sec. 4.4 applied to
 * the numerical coarse model): with Mc > 0, BS_COARSE_NUM on this grid computes
 *     G(u) = P(G_c(R u)),   far-field data at the slice's end,
 * where R restricts bilinearly to Mc x Mc nodes of the same domain, G_c takes the coarse
 * implicit-Euler steps there, and P prolongs the coarse state bilinearly (spatially
 * coarsened Parareal; converges quickly for smooth payoffs such as the basket).  This applies
 * to coarse_propagate and parareal_solve (serial sweep: restrict, coarse solve and apply per
 * slice).  Mc = 0 (default) or Mc = M: the coarse steps run on this grid.  Host-only.
 * BS_ERR_ARG unless Mc is 0 or in [8, M]. */
int bs_grid_set_coarse(bs_grid* g, int Mc);

/* Fine steps per slice for a time step whose Jacobi bound q (the Gershgorin contraction of
 * I - dtau R_h on an M x M grid, independent of xmax) is at most qmax: the smallest
 * min_steps * 2^k (k >= 0, at most 2^20) with q(T / (N * steps)) <= qmax.  This is the rule
 * the serving runtime applies to requests with fine_steps <= 0 (min_steps 64, qmax 0.7).
 * Host-only.  BS_ERR_ARG for invalid arguments, qmax outside (0, 0.8), or no such count. */
int bs_fine_steps_for(int M, const bs_params* p, int N, int min_steps, double qmax, int* steps);

/* Coarse-sweep autotuner (no counterpart in the paper, which has one CPU code path).  For
 * M <= 256 the serial coarse sweep runs on one thread-block cluster; the band variants
 * (columns per CTA, threads per CTA, rows per thread, hence cluster size) trade per-iteration
 * arithmetic against cluster-barrier latency.  The first coarse launch on a grid times each
 * variant that the device can launch on a short PROP solve from the payoff of p with coarse
 * step dtau_coarse, and caches the fastest per (device, M) for the process; this call runs
 * that measurement now (if not already done) and returns the chosen variant index in
 * *variant (-1 for M > 256, which uses the global-memory solver; the forced index when
 * BS_OPT_COARSE_VARIANT is set, without measuring).  Synchronous on `stream`;
 * allocates and frees two M*M FP32 buffers.  Returns BS_OK, BS_ERR_ARG or BS_ERR_CUDA. */
int bs_coarse_variant(bs_grid* g, const bs_params* p, double dtau_coarse, int* variant,
                      bs_stream stream);

/* Shape and solver features of band variant `variant` on an M x M grid (M <= 256, the
 * variant's column count must cover M): *ctas = CTAs of its cluster, *threads = threads per
 * CTA, *rows = rows per thread, *poly = the degree of its polynomial preconditioner (0: none;
 * 1: M^{-1} = 2I - A^, two more scaled 9-point products per BiCGSTAB iteration; 2: M^{-1} =
 * I + 1.5E + E^2 with E = I - A^, four more), *quad = 1 if its initial guesses extrapolate
 * quadratically.  Each feature is used where the variant's shared memory holds its extra
 * planes (and, for degree 2, its strips have at least three rows).  Any output pointer may be
 * NULL.  Host-only.  Returns BS_OK or BS_ERR_ARG (unknown variant, or one that does not fit M). */
int bs_coarse_variant_info(int variant, int M, int* ctas, int* threads, int* rows, int* poly, int* quad);

/* Diagnostics of the coarse solves enqueued on this grid since the last parareal_solve or
 * bs_grid_stats call: the largest BiCGSTAB iteration count, whether any solve hit its cap,
 * the summed iteration count and the number of implicit-Euler solves.  Any output pointer
 * may be NULL.  Synchronous (waits for the device), then resets the counters. */
int bs_grid_stats(bs_grid* g, int* krylov_iters_max, int* krylov_failed, int* krylov_iters_total,
                  int* krylov_solves);

/* Per-phase accounting on this grid since the last call: kernel launches of the fine
 * propagator, of the coarse propagator / serial Parareal sweep, and of everything else
 * (payoff), and -- when BS_OPT_PHASE_TIMING is on -- the summed CUDA-event durations of the
 * fine and coarse launches made by parareal_solve.  Host-only (the event times were read
 * when parareal_solve synchronised); resets the counters.  Any pointer may be NULL. */
int bs_phase_stats(bs_grid* g, double* fine_ms, int* fine_launches, double* coarse_ms,
                   int* coarse_launches, int* other_launches);

/* Parareal with the numerical coarse model, for callers that cannot allocate device memory:
 * code on a latency-critical pricing path where a device allocation (which may synchronise
 * the whole device and take milliseconds) is not allowed, or code embedded in a host
 * framework that owns all device memory through its own allocator.  The paper has no
 * counterpart to this entry point.  It runs the phase-by-phase Parareal iteration of
 * parareal_solve with coarse_kind = BS_COARSE_NUM and BS_OPT_PIPELINE = 0 (F on all open
 * slices, then the serial coarse sweep), with the same kernels, but takes the grid as M and
 * xmax instead of a bs_grid handle and keeps its scratch (fine and coarse slice buffers,
 * norms, status) in one fixed device array inside the library: about 32 MiB, held by every
 * GPU that loads the library until the process exits.  It calls no cudaMalloc, cudaFree or
 * allocating library routine (bs_device_allocations does not move across a call).
 *  - Capacity: N * M * M <= 4,194,304, N <= 1024 and M <= 256 (grids whose state fits one
 *    thread-block cluster; for example N = 64 slices of 256 x 256); larger problems return
 *    BS_ERR_ARG with a message naming the limit.  Use parareal_solve beyond these limits.
 *  - The fine step must have a Jacobi bound below 0.8 (bs_fine_sweeps(...) > 0): F runs the
 *    Jacobi stepper only; other steps return BS_ERR_ARG.
 *  - The coarse sweep uses the band variant that bs_coarse_variant has measured for M in this
 *    process (by a parareal_solve or coarse_propagate call on an M x M grid, or by
 *    bs_coarse_variant), else the default variant for M; it never runs the autotuner (which
 *    allocates).  With the same variant the iterates equal parareal_solve's bit for bit; with
 *    another they agree within the coarse Krylov tolerance (variants add in other orders).
 *  - The caller still owns u_out (device float[(N+1)*M*M]); k_done and defect_hist as in
 *    parareal_solve.  Synchronous, same return codes as parareal_solve.
 *  - The first call on a device looks up the array's device address (which may also load the
 *    library's device code); make that first call before any stream capture.
 *  - All calls share the one array: calls that overlap on the GPU (two host threads, or two
 *    streams) race and must be serialised by the caller. */
int parareal_solve_noalloc(int M, double xmax, const bs_params* p, int N, int fine_steps,
                           int coarse_steps, double tol, int Kmax, float* u_out, int* k_done,
                           double* defect_hist, bs_stream stream);

/* ---------------------------------------------------------------------------------------
 * Serving: continuous batching of Parareal pricing requests (no counterpart in the paper,
 * which prices one option per run).
 *
 * A server owns one device arena of hbm_budget_bytes.  Each admitted request keeps its whole
 * Parareal state in the arena -- U [N+1][M][M], F and G_old [N][M][M] in FP32 and 2(N+1) FP64
 * norms, request_bytes = (3N+1) M^2 * 4 + 16 (N+1), rounded up to 256 -- from admission to
 * completion (a PINO request also keeps its defect partials there, (N+1) ceil(M^2/256) x 16
 * bytes).  Requests are admitted in submission order while one of max_active slots is
 * free and the arena has room (first fit); a request that does not fit waits.  Every
 * request runs the Parareal of parareal_solve (eq. parareal; reading c5 stopping norm) with
 * its own coarse model -- numerical G on its grid, numerical G on a coarse grid, or the
 * PINO -- on its own CUDA stream; the fine propagation of all requests due at the same time
 * is batched into one fine_propagate launch per (grid size, fine steps), and the serial
 * coarse sweeps of different requests overlap on their streams (PINO sweeps share the
 * network's workspace and run one after another on one server stream).  A request's result
 * does not depend on what it was batched with: every slice of a fine launch is computed
 * independently, and each coarse sweep belongs to one request.
 *
 * The server is driven by the caller: bs_server_progress polls the requests' CUDA events
 * (no blocking), retires finished requests, admits waiting ones and launches the next
 * batched work; call it in a loop.  bs_server_poll returns finished requests.  A server is
 * used from one host thread at a time (calls are serialised by an internal lock).
 * --------------------------------------------------------------------------------------- */
typedef struct bs_server bs_server;       /* opaque */

typedef struct {
  size_t hbm_budget_bytes;   /* device arena for request state, >= 1 MiB */
  int max_active;            /* requests on the device at once (one CUDA stream each), 1..256 */
} bs_server_config;

typedef struct {
  bs_params p;               /* option parameters; p.T is the maturity */
  int M;                     /* grid nodes per axis, 4..4096 */
  double xmax;               /* domain [0, xmax]^2 */
  int N;                     /* time slices */
  int fine_steps;            /* implicit steps per slice of F; <= 0: 64, doubled until the
                                Jacobi bound of a step is <= 0.7 */
  int coarse_steps;          /* implicit steps per slice of the numerical G, >= 1 */
  double tol;                /* Parareal tolerance on the defect (> 0) */
  int Kmax;                  /* iteration cap, 1..N */
  float* u_out;              /* [M*M] caller buffer (host or device) for u(T) = U[N]; it
                                must stay valid until the request is reported done */
  /* The coarse model (zero-initialised: the numerical G on the request's own grid). */
  int coarse_kind;           /* BS_COARSE_NUM or BS_COARSE_PINO */
  int coarse_M;              /* BS_COARSE_NUM only: 0 = G on the request's grid; 8..M = G on an
                                coarse_M x coarse_M grid with bilinear resampling, the form
                                bs_grid_set_coarse selects for parareal_solve */
  const bs_pino* net;        /* BS_COARSE_PINO: the network (coarse_steps is then ignored);
                                the caller keeps it loaded until the request is done */
} bs_request;

typedef struct {
  long long id;              /* from bs_server_submit */
  int status;                /* BS_OK, BS_ERR_MAXITER (u_out holds the last iterate),
                                BS_ERR_NOCONV or BS_ERR_CUDA */
  int iterations;            /* Parareal iterations run */
  double defect;             /* last defect */
  double latency_ms;         /* host time from bs_server_submit to completion */
  int fine_steps;            /* fine steps per slice used */
} bs_result;

typedef struct {
  size_t arena_bytes, arena_used;
  long long fine_batches;    /* batched fine launches (groups) */
  long long fine_items;      /* slices propagated by them */
  long long coarse_sweeps;   /* coarse sweeps launched */
  long long launches;        /* kernels launched by the server */
} bs_server_stats_t;

/* Allocates the arena (cudaMalloc) and per-slot streams, events and pinned words on the
 * current device.  BS_ERR_ARG for a budget below 1 MiB or max_active outside 1..256. */
int bs_server_create(const bs_server_config* cfg, bs_server** out);
/* Queues a request (copied); *id identifies it in bs_server_poll.  Host-only.  BS_ERR_ARG
 * for invalid sizes or parameters, for explicit fine_steps whose Jacobi bound is >= 0.8, for
 * an unknown coarse_kind, a coarse_M outside {0} U [8, M], a PINO request without a network
 * of the supported shape or with coarse_M set, or for a request larger than the whole arena. */
int bs_server_submit(bs_server* s, const bs_request* r, long long* id);
/* Advances the server without blocking (see above); *active and *pending (either may be
 * NULL) receive the numbers of admitted and waiting requests.  The first request of a grid
 * size M <= 256 runs the coarse autotuner once (a few milliseconds, synchronous). */
int bs_server_progress(bs_server* s, int* active, int* pending);
/* Moves up to max_results finished requests into out[] (oldest first); *n receives the count. */
int bs_server_poll(bs_server* s, bs_result* out, int max_results, int* n);
int bs_server_stats(bs_server* s, bs_server_stats_t* st);
/* Waits for the device, then releases everything (requests still in flight are dropped). */
int bs_server_destroy(bs_server* s);

#ifdef __cplusplus
}
#endif
#endif /* BSPARAREAL_H */
