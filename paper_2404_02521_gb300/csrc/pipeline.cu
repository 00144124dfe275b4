// Pipelined Parareal driver (numerical G, on the state grid or on the grid's coarse grid).
//
// Eq. (parareal) needs F(u_n^k) only when the sweep of iteration k-1 has produced u_n^k, so F
// and the serial coarse sweep need not alternate as whole phases.  Each sweep is split into
// chunks of S consecutive slices, launched one after another on an internal stream of the
// highest priority (so that a sweep chunk's 16-CTA cluster is placed before an F chunk that
// becomes ready at the same moment); the F launch of a chunk goes to a low-priority stream
// and waits (cudaStreamWaitEvent) for the sweep chunk that finished its input states.  Both
// streams start after the caller's stream and the caller's stream waits for both at the end.
// The sweep chunk of iteration k waits for the F chunk of iteration k over the same slices.
// The first input of F chunk c, u_{cS}, is the last state sweep chunk c-1 writes, and the next
// sweep rewrites it while F chunk c may still be waiting for SMs; so each sweep chunk also
// copies its last state into a snapshot (two sets, by iteration parity) that F chunk c reads.
// F of iteration k+1 is launched before the host has read the defect of iteration k
// (speculatively: it writes only the F workspace, and is wasted if iteration k converged), so
// it runs on the SMs the 16-CTA coarse cluster leaves free while the sweep continues.  All ordering is between whole kernels through stream
// events; no kernel waits on another.  Results: the same Parareal iteration; on the state grid
// the coarse solves restart their extrapolated initial guesses at chunk boundaries, so G agrees
// with the unchunked sweep to the Krylov tolerance, not bitwise; with G on a coarse grid every
// slice's coarse solve starts afresh anyway, and the result is the phase-by-phase driver's bit
// for bit.  F of the next iteration is speculated only where it is cheap (grids whose states
// live in one cluster) or from the second iteration on: on the tiled grids one F pass is most
// of a solve, and a solve that converges after one iteration would pay for a second.
#include <vector>

#include "common.cuh"

namespace bsp {

struct PipeState {
  cudaStream_t ss = nullptr;            // sweep chunks (highest priority)
  cudaStream_t sf = nullptr;            // F chunks
  std::vector<cudaEvent_t> ev_s, ev_f;  // per chunk: sweep chunk done, F chunk done
  std::vector<cudaEvent_t> timing;      // start/end pairs (phase timing)
  size_t next_timing = 0;
};

static int pipe_state(bs_grid* g, int chunks, PipeState** out) {
  if (!g->pipe) {
    PipeState* ps = new PipeState();
    // A sweep chunk's cluster needs 16 SMs of one GPC; when it and an F chunk become ready
    // together, the higher stream priority places the cluster first.
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&ps->ss, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ps->sf, cudaStreamNonBlocking, lo) != cudaSuccess) {
      if (ps->ss) cudaStreamDestroy(ps->ss);
      delete ps;
      return cuda_error(cudaGetLastError(), "parareal pipeline: streams");
    }
    g->pipe = ps;
  }
  PipeState* ps = static_cast<PipeState*>(g->pipe);
  while ((int)ps->ev_s.size() < chunks) {
    cudaEvent_t a, b;
    BS_CUDA_TRY(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    BS_CUDA_TRY(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    ps->ev_s.push_back(a);
    ps->ev_f.push_back(b);
  }
  ps->next_timing = 0;
  *out = ps;
  return BS_OK;
}

void pipe_destroy(bs_grid* g) {
  PipeState* ps = static_cast<PipeState*>(g->pipe);
  if (!ps) return;
  for (cudaEvent_t e : ps->ev_s) cudaEventDestroy(e);
  for (cudaEvent_t e : ps->ev_f) cudaEventDestroy(e);
  for (cudaEvent_t e : ps->timing) cudaEventDestroy(e);
  if (ps->sf) cudaStreamDestroy(ps->sf);
  if (ps->ss) cudaStreamDestroy(ps->ss);
  delete ps;
  g->pipe = nullptr;
}

// A start/end event pair for phase timing (created on first use, reused across solves).
static int timing_pair(PipeState* ps, cudaEvent_t* a, cudaEvent_t* b) {
  while (ps->timing.size() < ps->next_timing + 2) {
    cudaEvent_t e;
    BS_CUDA_TRY(cudaEventCreate(&e));
    ps->timing.push_back(e);
  }
  *a = ps->timing[ps->next_timing];
  *b = ps->timing[ps->next_timing + 1];
  ps->next_timing += 2;
  return BS_OK;
}

bool pipeline_eligible(int N) { return N >= 8; }

// Slices per chunk.  An F chunk should run in one wave beside the sweep's cluster: the fine
// clusters the device holds at once, less those the coarse cluster displaces (its CTAs over
// the fine cluster's, rounded up: both take whole SMs of one GPC).  A chunk that spills into a
// second wave, or an F wave that leaves no GPC for the sweep's cluster, stalls the sweep --
// on the 256 x 256 workload chunks of 16 slices took 60 ms per solve, of 12 slices 48, and the
// 13 of this rule 44.
// At most a quarter of the slices, so that F starts early and the sweep drains soon.
int pipeline_chunk(bs_grid* g, const ItemDesc& dc, int N, cudaStream_t s, int* S) {
  int quarter = (N + 3) / 4;
  const int cap = fine_cluster_capacity(g);
  if (cap > 0) {
    int cc = 0;
    int rc = coarse_cluster_ctas(g, dc, s, &cc);
    if (rc) return rc;
    const int cf = g->shape.C;
    const int wave = cap - (cc + cf - 1) / cf;
    if (wave >= 1 && wave < quarter) quarter = wave;
  }
  *S = quarter;
  return BS_OK;
}

int parareal_pipelined(bs_grid* g, const bs_params* p, int N, int fine_steps, int coarse_steps, double tol,
                       int Kmax, float* u_out, bool user_u0, int* k_done, double* defect_hist,
                       cudaStream_t caller) {
  const int M = g->M;
  const size_t MM = (size_t)M * M;
  const double slice = p->T / N;
  const double dtau_f = slice / fine_steps;
  const int sweeps = grid_sweeps(g, *p, dtau_f);
  const int sweeps0 = grid_sweeps(g, *p, dtau_f, START_COLD);
  const int sweepsx = grid_sweeps(g, *p, dtau_f, START_EXTRAP);
  const int sweepsxl = grid_sweeps(g, *p, dtau_f, START_EXTRAP_LATE);
  const bool krylov_f = sweeps == 0;
  const bool resampled = g->coarse_M > 0 && g->coarse_M != g->M;
  const bool cheap_f = g->shape.C >= 1 && g->shape.C <= kMaxCluster;   // a state per cluster
  const ItemDesc dc = make_item(*p, 0.0, slice / coarse_steps);
  int S = 0;
  int rc = pipeline_chunk(g, dc, N, caller, &S);
  if (rc) return rc;
  const int chunks = (N + S - 1) / S;
  // F buffers, G_old, the slice norms, then two sets (by iteration parity) of chunk-boundary
  // snapshots: snap[par][c] holds u_{cS} of the iterate that F of that parity reads
  const size_t base = sizeof(float) * 2 * (size_t)N * MM + sizeof(double) * 2 * (N + 1);
  const size_t snap_off = (base + 255) & ~(size_t)255;
  rc = ensure(g->ws_par, snap_off + sizeof(float) * 2 * (size_t)chunks * MM);
  if (rc) return rc;
  float* Fb = (float*)g->ws_par.ptr;
  float* Gold = Fb + (size_t)N * MM;
  double* norms = (double*)(Gold + (size_t)N * MM);
  float* snap = (float*)((unsigned char*)g->ws_par.ptr + snap_off);
  auto snap_at = [&](int parity, int c) { return snap + ((size_t)parity * chunks + c) * MM; };
  PipeState* ps;
  if ((rc = pipe_state(g, chunks, &ps))) return rc;
  cudaStream_t sf = ps->sf, s = ps->ss;
  // both internal streams start after everything the caller enqueued before this call
  BS_CUDA_TRY(cudaEventRecord(ps->ev_f[0], caller));
  BS_CUDA_TRY(cudaStreamWaitEvent(s, ps->ev_f[0], 0));
  BS_CUDA_TRY(cudaStreamWaitEvent(sf, ps->ev_f[0], 0));
  const bool timing = g_opt.phase_timing != 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> t_fine, t_coarse;

  BS_CUDA_TRY(cudaMemsetAsync(g->status, 0, kStatusWords * sizeof(int), s));
  if (!user_u0) {
    if ((rc = launch_payoff(g, dc, u_out, s))) return rc;
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

  // sweep chunks of one iteration (mode, first slice k), each after the F chunk it reads
  auto sweep_chunks = [&](int mode, int k, bool wait_f) -> int {
    for (int c = 0; c < chunks; ++c) {
      const int lo = std::max(k, c * S), hi = std::min(N, (c + 1) * S);
      if (lo >= hi) continue;
      if (wait_f) BS_CUDA_TRY(cudaStreamWaitEvent(s, ps->ev_f[c], 0));
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      if (timing) {
        int r = timing_pair(ps, &t0, &t1);
        if (r) return r;
        BS_CUDA_TRY(cudaEventRecord(t0, s));
      }
      a.mode = mode;
      a.n_first = k;
      a.n_begin = lo;
      a.n_end = hi;
      int r;
      if (resampled) {
        r = resampled_sweep(g, dc, a, s);
        g->n_coarse += (hi - lo) * resampled_launches_per_slice() + 1;
      } else {
        r = launch_sweep(g, dc, a, s);
        g->n_coarse += 1;
      }
      if (r) return r;
      // u_hi is the first input of the next F chunk, which may not have read it yet when the
      // next iteration's sweep chunk c overwrites it: that F chunk reads this copy instead
      if (hi < N) {
        const int par = mode == SWEEP_INIT ? 0 : (k + 1) & 1;
        BS_CUDA_TRY(cudaMemcpyAsync(snap_at(par, c + 1), u_out + (size_t)hi * MM, sizeof(float) * MM,
                                    cudaMemcpyDeviceToDevice, s));
      }
      if (timing) {
        BS_CUDA_TRY(cudaEventRecord(t1, s));
        t_coarse.emplace_back(t0, t1);
      }
      BS_CUDA_TRY(cudaEventRecord(ps->ev_s[c], s));
    }
    return BS_OK;
  };
  // F chunks of iteration k on the second stream, each after the sweep chunk that wrote its
  // input states
  std::vector<ItemDesc> items;
  auto fine_chunks = [&](int k) -> int {
    for (int c = 0; c < chunks; ++c) {
      const int lo = std::max(k, c * S), hi = std::min(N, (c + 1) * S);
      if (lo >= hi) continue;
      BS_CUDA_TRY(cudaStreamWaitEvent(sf, ps->ev_s[c], 0));
      items.clear();
      for (int n = lo; n < hi; ++n) {
        ItemDesc d = make_item(*p, n * slice, dtau_f);
        // u_{cS} is rewritten by this iteration's sweep chunk c-1 while k < cS
        d.in = (n == c * S && c >= 1 && k < n) ? snap_at(k & 1, c) : u_out + (size_t)n * MM;
        d.out = Fb + (size_t)n * MM;
        d.sweeps = sweeps;
        d.sweeps0 = sweeps0;
        d.sweepsx = sweepsx;
        d.sweepsxl = sweepsxl;
        items.push_back(d);
      }
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      if (timing) {
        int r = timing_pair(ps, &t0, &t1);
        if (r) return r;
        BS_CUDA_TRY(cudaEventRecord(t0, sf));
      }
      int r;
      if (krylov_f) {
        r = launch_krylov_fine(g, items.data(), (int)items.size(), fine_steps, sf);
      } else {
        r = launch_fine(g, items.data(), (int)items.size(), fine_steps, sf);
        g->n_fine += fine_launches(g, items.data(), (int)items.size(), fine_steps);
      }
      if (r) return r;
      if (timing) {
        BS_CUDA_TRY(cudaEventRecord(t1, sf));
        t_fine.emplace_back(t0, t1);
      }
      BS_CUDA_TRY(cudaEventRecord(ps->ev_f[c], sf));
    }
    return BS_OK;
  };

  if ((rc = sweep_chunks(SWEEP_INIT, 0, false))) return rc;
  int k = 0;
  int status = BS_ERR_MAXITER;
  if (Kmax > 0 && (rc = fine_chunks(0))) return rc;
  double prev_defect = 1e300;
  bool f_launched = true;   // F of iteration k is enqueued
  for (; k < Kmax; ++k) {
    if (!f_launched && (rc = fine_chunks(k))) return rc;
    if ((rc = sweep_chunks(SWEEP_ITER, k, true))) return rc;
    // The next iteration's F, before this iteration's defect is known -- unless the last
    // defect was already within 10 tol: then this iteration is likely the final one, and a
    // wasted F would only slow its sweep down (the two share the GPU).
    f_launched = k + 1 < Kmax && prev_defect > 10.0 * tol && (cheap_f || k >= 1);
    if (f_launched && (rc = fine_chunks(k + 1))) return rc;
    double host = 0.0;
    int hstat = 0;
    BS_CUDA_TRY(cudaMemcpyAsync(&host, g->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaMemcpyAsync(&hstat, g->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaStreamSynchronize(s));
    if (defect_hist) defect_hist[k] = host;
    prev_defect = host;
    if (hstat) {
      *k_done = k + 1;
      BS_CUDA_TRY(cudaStreamSynchronize(sf));
      if (hstat & 2)
        return set_error(BS_ERR_CUDA, "parareal_solve: a cluster exchange of the coarse sweep timed out");
      return set_error(BS_ERR_NOCONV, "parareal_solve: a coarse BiCGSTAB solve hit its iteration cap");
    }
    if (host <= tol) {
      ++k;
      status = BS_OK;
      break;
    }
  }
  *k_done = k;
  // work enqueued on the caller's stream after this call is ordered after all of it,
  // including the speculative F
  BS_CUDA_TRY(cudaEventRecord(ps->ev_f[0], sf));
  BS_CUDA_TRY(cudaEventRecord(ps->ev_s[0], s));
  BS_CUDA_TRY(cudaStreamWaitEvent(caller, ps->ev_f[0], 0));
  BS_CUDA_TRY(cudaStreamWaitEvent(caller, ps->ev_s[0], 0));
  if (timing) {
    BS_CUDA_TRY(cudaStreamSynchronize(sf));
    BS_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    for (auto& e : t_fine) {
      cudaEventElapsedTime(&ms, e.first, e.second);
      g->ms_fine += ms;
    }
    for (auto& e : t_coarse) {
      cudaEventElapsedTime(&ms, e.first, e.second);
      g->ms_coarse += ms;
    }
  }
  if (Kmax == 0) BS_CUDA_TRY(cudaStreamSynchronize(s));
  // after N iterations every slice is exact (serial fine stepping), whatever the last defect
  if (status == BS_ERR_MAXITER && k < N)
    return set_error(BS_ERR_MAXITER, "parareal_solve: tol %g not met after %d iterations", tol, k);
  return BS_OK;
}

}  // namespace bsp
