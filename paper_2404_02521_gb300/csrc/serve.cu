// Serving loop: continuous batching of Parareal pricing requests on one GPU.
//
// The paper prices one option per run; a pricing service receives many requests of
// different grid sizes and slice counts.  This runtime keeps each admitted request's whole
// Parareal state (U, F, G_old and the norms) resident in one device arena sized by an HBM
// budget, and advances every request through its own state machine
//     admitted -> payoff + initial coarse sweep -> { F on slices k..N-1 -> correcting
//     coarse sweep -> defect } * -> copy of u(T) -> done
// driven by CUDA events that the host polls, so requests that arrive while others are on the
// GPU are admitted as soon as a slot and arena space are free.  Requests whose fine
// propagation is due at the same time are batched: their slices go into one
// fine_propagate launch per grid size (the fine kernels treat every slice independently,
// so a result does not depend on what it was batched with).  Coarse sweeps, serial within a
// request, run on the request's own stream and overlap across requests.  Each request
// brings its coarse model: the numerical G on its grid or on a coarse grid (its own grid
// object carries the coarse grid and its buffers), or the PINO, whose sweeps share the
// network's workspace and so run in order on one server stream, ordered against the
// request's stream by events.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace bsp {

constexpr size_t kArenaAlign = 256;

// First-fit allocator over [0, capacity) of the device arena.
class Arena {
 public:
  void reset(size_t capacity) {
    free_.clear();
    if (capacity) free_[0] = capacity;
    cap_ = capacity;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t capacity() const { return cap_; }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0, used_ = 0;
};

enum Phase { PH_FREE = 0, PH_INIT, PH_READY_F, PH_G, PH_COPY };

struct Slot {
  Phase phase = PH_FREE;
  long long id = 0;
  bs_request r{};
  bs_grid* g = nullptr;          // per-request grid: status, defect, coarse workspace
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  double* h_defect = nullptr;    // pinned
  int* h_status = nullptr;       // pinned
  size_t off = 0, bytes = 0;
  float *U = nullptr, *Fb = nullptr, *Gold = nullptr;
  double* norms = nullptr;
  double* partials = nullptr;    // PINO requests: the sweep's defect partials
  int k = 0, sweeps = 0, sweeps0 = 0, sweepsx = 0, sweepsxl = 0, result = BS_OK;
  double defect = 0.0, t_submit = 0.0;
};

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace bsp

struct bs_server {
  bs_server_config cfg{};
  int device = 0;
  unsigned char* arena_base = nullptr;
  bsp::Arena arena;
  std::vector<bsp::Slot> slots;
  std::deque<std::pair<long long, bs_request>> pending;
  std::deque<double> pending_t;
  std::deque<bs_result> done;
  std::map<int, std::vector<bs_grid*>> grid_pool;   // M -> reusable per-request grids
  std::map<int, bs_grid*> class_grid;               // M -> grid owning the fine workspace
  std::map<int, cudaStream_t> batch_stream;         // M -> stream of its batched F launches
  std::vector<cudaEvent_t> batch_events;
  size_t next_batch_event = 0;
  cudaStream_t pino_stream = nullptr;               // every PINO sweep, in order
  long long next_id = 1;
  std::mutex mu;
  // statistics
  long long fine_batches = 0, fine_items = 0, coarse_sweeps = 0, launches = 0;
};

namespace bsp {

// Request state in the arena: U [N+1][M][M], F [N][M][M], G_old [N][M][M] (FP32), the
// per-slice norms [2(N+1)] (FP64) and, for a PINO request, the sweep's defect partials.
static size_t state_bytes(const bs_request& r) {
  const size_t MM = (size_t)r.M * r.M;
  return ((size_t)(3 * r.N + 1) * MM * sizeof(float) + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
}
static size_t norms_bytes(const bs_request& r) {
  return (sizeof(double) * 2 * (r.N + 1) + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
}
static size_t request_bytes(const bs_request& r) {
  const size_t part = r.coarse_kind == BS_COARSE_PINO ? pino_partials_bytes(r.M, r.N) : 0;
  return state_bytes(r) + (part ? norms_bytes(r) + part : sizeof(double) * 2 * (r.N + 1));
}

static cudaEvent_t batch_event(bs_server* sv);

// One coarse sweep of a request (SweepArgs filled in by the caller) with its coarse model,
// ordered after the work already on the request's stream; counts its launches.
static int request_sweep(bs_server* sv, Slot& sl, const ItemDesc& dc, const SweepArgs& a) {
  const bs_request& r = sl.r;
  int rc;
  if (r.coarse_kind == BS_COARSE_PINO) {
    // the network's workspace (activations, slice descriptors) serves one sweep at a time
    cudaEvent_t e0 = batch_event(sv);
    BS_CUDA_TRY(cudaEventRecord(e0, sl.st));
    BS_CUDA_TRY(cudaStreamWaitEvent(sv->pino_stream, e0, 0));
    if ((rc = pino_sweep(const_cast<bs_pino*>(r.net), sl.g, dc, a, sl.partials, sv->pino_stream))) return rc;
    cudaEvent_t e1 = batch_event(sv);
    BS_CUDA_TRY(cudaEventRecord(e1, sv->pino_stream));
    BS_CUDA_TRY(cudaStreamWaitEvent(sl.st, e1, 0));
    sv->launches += (long long)(a.N - a.n_first) * pino_launches_per_step(r.net, r.M) + 1;
  } else if (sl.g->coarse_M > 0) {
    if ((rc = resampled_sweep(sl.g, dc, a, sl.st))) return rc;
    sv->launches += (long long)(a.N - a.n_first) * resampled_launches_per_slice() + 1;
  } else {
    if ((rc = launch_sweep(sl.g, dc, a, sl.st))) return rc;
    sv->launches += 1;
  }
  sv->coarse_sweeps += 1;
  return BS_OK;
}

// 64 steps per slice, doubled until the Jacobi bound of a fine step is at most 0.7
static int auto_fine_steps(const bs_request& r) {
  int s = 0;
  return bs_fine_steps_for(r.M, &r.p, r.N, 64, 0.7, &s) == BS_OK ? s : 0;
}

static int take_grid(bs_server* sv, int M, double xmax, bs_grid** out) {
  auto& pool = sv->grid_pool[M];
  for (size_t i = 0; i < pool.size(); ++i) {
    if (pool[i]->xmax == xmax) {
      *out = pool[i];
      pool.erase(pool.begin() + (long)i);
      return BS_OK;
    }
  }
  int rc = bs_grid_create(M, xmax, out);
  if (rc) return rc;
  (*out)->coarse_variant = coarse_cached_variant(sv->device, M);
  return BS_OK;
}

static cudaEvent_t batch_event(bs_server* sv) {
  cudaEvent_t e = sv->batch_events[sv->next_batch_event % sv->batch_events.size()];
  ++sv->next_batch_event;
  return e;
}

static int class_setup(bs_server* sv, const bs_request& r) {
  if (sv->class_grid.count(r.M)) return BS_OK;
  bs_grid* g = nullptr;
  int rc = bs_grid_create(r.M, r.xmax, &g);
  if (rc) return rc;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    bs_grid_destroy(g);
    return cuda_error(cudaGetLastError(), "bs_server: stream");
  }
  // one measurement of the coarse band variant per grid size and process, before any request
  // uses it (a variant this process has already measured for M is kept)
  if (r.M <= 256 && g_opt.coarse_variant < 0 && coarse_tuned_variant(sv->device, r.M) < 0) {
    const int cs = r.coarse_steps > 0 ? r.coarse_steps : 1;
    rc = coarse_autotune(g, make_item(r.p, 0.0, r.p.T / r.N / cs), s, kAutotuneSteps, nullptr);
    if (rc) {
      cudaStreamDestroy(s);
      bs_grid_destroy(g);
      return rc;
    }
  }
  sv->class_grid[r.M] = g;
  sv->batch_stream[r.M] = s;
  return BS_OK;
}

// Admit one request into a free slot: arena space, payoff and the initial coarse sweep.
static int admit(bs_server* sv, Slot& sl, long long id, const bs_request& r, double t_submit) {
  int rc = class_setup(sv, r);
  if (rc) return rc;
  sl.id = id;
  sl.r = r;
  sl.t_submit = t_submit;
  sl.k = 0;
  sl.result = BS_OK;
  sl.defect = 0.0;
  const size_t MM = (size_t)r.M * r.M;
  float* base = reinterpret_cast<float*>(sv->arena_base + sl.off);
  sl.U = base;
  sl.Fb = base + (size_t)(r.N + 1) * MM;
  sl.Gold = sl.Fb + (size_t)r.N * MM;
  const size_t fbytes = state_bytes(r);
  sl.norms = reinterpret_cast<double*>(sv->arena_base + sl.off + fbytes);
  sl.partials = r.coarse_kind == BS_COARSE_PINO
                    ? reinterpret_cast<double*>(sv->arena_base + sl.off + fbytes + norms_bytes(r))
                    : nullptr;
  if ((rc = take_grid(sv, r.M, r.xmax, &sl.g))) return rc;
  // the numerical G's grid (a pooled grid keeps the coarse grid of its last request until
  // this call changes it)
  if ((rc = bs_grid_set_coarse(sl.g, r.coarse_kind == BS_COARSE_NUM ? r.coarse_M : 0))) return rc;
  const double slice = r.p.T / r.N;
  const double dtau_f = slice / r.fine_steps;
  sl.sweeps = grid_sweeps(sl.g, r.p, dtau_f, START_WARM);
  sl.sweeps0 = grid_sweeps(sl.g, r.p, dtau_f, START_COLD);
  sl.sweepsx = grid_sweeps(sl.g, r.p, dtau_f, START_EXTRAP);
  sl.sweepsxl = grid_sweeps(sl.g, r.p, dtau_f, START_EXTRAP_LATE);
  BS_CUDA_TRY(cudaMemsetAsync(sl.g->status, 0, kStatusWords * sizeof(int), sl.st));
  const ItemDesc dc = make_item(r.p, 0.0, slice / r.coarse_steps);
  if ((rc = launch_payoff(sl.g, dc, sl.U, sl.st))) return rc;
  SweepArgs a = {};
  a.mode = SWEEP_INIT;
  a.n_first = 0;
  a.N = r.N;
  a.csteps = r.coarse_steps;
  a.slice_len = slice;
  a.U = sl.U;
  a.Fb = sl.Fb;
  a.Gold = sl.Gold;
  a.norms = sl.norms;
  a.defect = sl.g->dscal;
  a.status = sl.g->status;
  a.tol = g_opt.krylov_tol;
  a.maxit = g_opt.krylov_maxit;
  if ((rc = request_sweep(sv, sl, dc, a))) return rc;
  BS_CUDA_TRY(cudaEventRecord(sl.ev, sl.st));
  sv->launches += 1;   // the payoff
  sl.phase = PH_INIT;
  return BS_OK;
}

static void finish(bs_server* sv, Slot& sl) {
  bs_result res{};
  res.id = sl.id;
  res.status = sl.result;
  res.iterations = sl.k;
  res.defect = sl.defect;
  res.latency_ms = now_ms() - sl.t_submit;
  res.fine_steps = sl.r.fine_steps;
  sv->done.push_back(res);
  sv->arena.release(sl.off, sl.bytes);
  sv->grid_pool[sl.r.M].push_back(sl.g);
  sl.g = nullptr;
  sl.phase = PH_FREE;
}

// Enqueue the copy of u(T) = U[N] to the caller's buffer; the request is done after it.
static int start_copy(bs_server* sv, Slot& sl) {
  const size_t MM = (size_t)sl.r.M * sl.r.M;
  BS_CUDA_TRY(cudaMemcpyAsync(sl.r.u_out, sl.U + (size_t)sl.r.N * MM, MM * sizeof(float), cudaMemcpyDefault,
                              sl.st));
  BS_CUDA_TRY(cudaEventRecord(sl.ev, sl.st));
  sl.phase = PH_COPY;
  return BS_OK;
}

// One group of requests with the same grid size and fine steps per slice: one batched F
// launch on the group's stream, then each request's correcting sweep on its own stream.
static int launch_group(bs_server* sv, const std::vector<Slot*>& grp) {
  const int M = grp[0]->r.M, fs = grp[0]->r.fine_steps;
  const size_t MM = (size_t)M * M;
  std::vector<ItemDesc> items;
  for (Slot* sl : grp) {
    const double slice = sl->r.p.T / sl->r.N;
    for (int n = sl->k; n < sl->r.N; ++n) {
      ItemDesc d = make_item(sl->r.p, n * slice, slice / fs);
      d.in = sl->U + (size_t)n * MM;
      d.out = sl->Fb + (size_t)n * MM;
      d.sweeps = sl->sweeps;
      d.sweeps0 = sl->sweeps0;
      d.sweepsx = sl->sweepsx;
      d.sweepsxl = sl->sweepsxl;
      items.push_back(d);
    }
  }
  cudaStream_t bst = sv->batch_stream[M];
  bs_grid* cg = sv->class_grid[M];
  int rc = launch_fine(cg, items.data(), (int)items.size(), fs, bst);
  if (rc) return rc;
  sv->launches += fine_launches(cg, items.data(), (int)items.size(), fs);
  sv->fine_batches += 1;
  sv->fine_items += (long long)items.size();
  cudaEvent_t be = batch_event(sv);
  BS_CUDA_TRY(cudaEventRecord(be, bst));
  for (Slot* sl : grp) {
    BS_CUDA_TRY(cudaStreamWaitEvent(sl->st, be, 0));
    const double slice = sl->r.p.T / sl->r.N;
    const ItemDesc dc = make_item(sl->r.p, 0.0, slice / sl->r.coarse_steps);
    SweepArgs a = {};
    a.mode = SWEEP_ITER;
    a.n_first = sl->k;
    a.N = sl->r.N;
    a.csteps = sl->r.coarse_steps;
    a.slice_len = slice;
    a.U = sl->U;
    a.Fb = sl->Fb;
    a.Gold = sl->Gold;
    a.norms = sl->norms;
    a.defect = sl->g->dscal;
    a.status = sl->g->status;
    a.tol = g_opt.krylov_tol;
    a.maxit = g_opt.krylov_maxit;
    if ((rc = request_sweep(sv, *sl, dc, a))) return rc;
    BS_CUDA_TRY(cudaMemcpyAsync(sl->h_defect, sl->g->dscal, sizeof(double), cudaMemcpyDeviceToHost, sl->st));
    BS_CUDA_TRY(cudaMemcpyAsync(sl->h_status, sl->g->status, sizeof(int), cudaMemcpyDeviceToHost, sl->st));
    BS_CUDA_TRY(cudaEventRecord(sl->ev, sl->st));
    sl->phase = PH_G;
  }
  return BS_OK;
}

static int progress(bs_server* sv) {
  int rc;
  // 1. completions
  for (Slot& sl : sv->slots) {
    if (sl.phase == PH_FREE || sl.phase == PH_READY_F) continue;
    const cudaError_t q = cudaEventQuery(sl.ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return cuda_error(q, "bs_server: request event");
    if (sl.phase == PH_INIT) {
      sl.phase = PH_READY_F;
    } else if (sl.phase == PH_G) {
      sl.defect = *sl.h_defect;
      const int st = *sl.h_status;
      ++sl.k;
      if (st & 2) {
        sl.result = BS_ERR_CUDA;
      } else if (st) {
        sl.result = BS_ERR_NOCONV;
      } else if (sl.defect <= sl.r.tol || sl.k >= sl.r.N) {   // k = N: every slice is exact
        sl.result = BS_OK;
      } else if (sl.k >= sl.r.Kmax) {
        sl.result = BS_ERR_MAXITER;
      } else {
        sl.phase = PH_READY_F;
        continue;
      }
      if ((rc = start_copy(sv, sl))) return rc;
    } else if (sl.phase == PH_COPY) {
      finish(sv, sl);
    }
  }
  // 2. admissions, in arrival order, while a slot and arena space are free
  while (!sv->pending.empty()) {
    Slot* free_slot = nullptr;
    for (Slot& sl : sv->slots)
      if (sl.phase == PH_FREE) { free_slot = &sl; break; }
    if (!free_slot) break;
    // a copy: pop_front below destroys the queued element (and may free its block)
    const bs_request r = sv->pending.front().second;
    const size_t bytes = request_bytes(r);
    size_t off = 0;
    if (!sv->arena.alloc(bytes, &off)) break;   // wait for memory to free up
    free_slot->off = off;
    free_slot->bytes = bytes;
    const long long id = sv->pending.front().first;
    const double t = sv->pending_t.front();
    sv->pending.pop_front();
    sv->pending_t.pop_front();
    if ((rc = admit(sv, *free_slot, id, r, t))) {
      sv->arena.release(off, bytes);
      free_slot->phase = PH_FREE;
      return rc;
    }
  }
  // 3. batched fine propagation for every request whose F is due
  std::map<std::pair<int, int>, std::vector<Slot*>> groups;
  for (Slot& sl : sv->slots)
    if (sl.phase == PH_READY_F) groups[{sl.r.M, sl.r.fine_steps}].push_back(&sl);
  for (auto& kv : groups)
    if ((rc = launch_group(sv, kv.second))) return rc;
  return BS_OK;
}

}  // namespace bsp

using namespace bsp;

extern "C" {

int bs_server_create(const bs_server_config* cfg, bs_server** out) {
  if (!cfg || !out) return set_error(BS_ERR_ARG, "bs_server_create: NULL argument");
  *out = nullptr;
  if (cfg->hbm_budget_bytes < (size_t)(1 << 20) || cfg->max_active < 1 || cfg->max_active > 256)
    return set_error(BS_ERR_ARG, "bs_server_create: budget %zu B, max_active %d", cfg->hbm_budget_bytes,
                     cfg->max_active);
  bs_server* sv = new bs_server();
  sv->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&sv->device);
  note_device_alloc();
  if (e == cudaSuccess) e = cudaMalloc(&sv->arena_base, cfg->hbm_budget_bytes);
  if (e != cudaSuccess) {
    delete sv;
    return cuda_error(e, "bs_server_create: arena");
  }
  sv->arena.reset(cfg->hbm_budget_bytes);
  sv->slots.resize((size_t)cfg->max_active);
  for (Slot& sl : sv->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    note_device_alloc();
    note_device_alloc();
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_defect, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_status, sizeof(int));
  }
  sv->batch_events.resize(64);
  for (auto& be : sv->batch_events)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&be, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->pino_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    bs_server_destroy(sv);
    return cuda_error(e, "bs_server_create");
  }
  *out = sv;
  return BS_OK;
}

int bs_server_submit(bs_server* sv, const bs_request* r, long long* id) {
  if (!sv || !r || !id) return set_error(BS_ERR_ARG, "bs_server_submit: NULL argument");
  int rc = check_params(&r->p);
  if (rc) return rc;
  if (r->M < 4 || r->M > 4096 || !(r->xmax > 0.0) || r->N < 1 || r->coarse_steps < 1 || !r->u_out ||
      !(r->tol > 0.0) || r->Kmax < 1 || r->Kmax > r->N)
    return set_error(BS_ERR_ARG, "bs_server_submit: M=%d N=%d coarse_steps=%d Kmax=%d", r->M, r->N,
                     r->coarse_steps, r->Kmax);
  if (r->coarse_kind != BS_COARSE_NUM && r->coarse_kind != BS_COARSE_PINO)
    return set_error(BS_ERR_ARG, "bs_server_submit: unknown coarse_kind %d", r->coarse_kind);
  if (r->coarse_M != 0 && (r->coarse_kind != BS_COARSE_NUM || r->coarse_M < 8 || r->coarse_M > r->M))
    return set_error(BS_ERR_ARG, "bs_server_submit: coarse_M=%d needs the numerical G and 8 <= coarse_M <= M=%d",
                     r->coarse_M, r->M);
  if (r->coarse_kind == BS_COARSE_PINO && (rc = pino_check(r->net, r->M))) return rc;
  bs_request q = *r;
  if (q.coarse_kind == BS_COARSE_PINO) q.coarse_steps = 1;
  if (q.fine_steps <= 0) q.fine_steps = auto_fine_steps(q);
  if (q.fine_steps <= 0 || !(jacobi_contraction(q.M, q.p, q.p.T / q.N / q.fine_steps) < 0.8))
    return set_error(BS_ERR_ARG, "bs_server_submit: fine steps give a Jacobi bound >= 0.8");
  if (request_bytes(q) > sv->arena.capacity())
    return set_error(BS_ERR_ARG, "bs_server_submit: request needs %zu B, budget %zu B", request_bytes(q),
                     sv->arena.capacity());
  std::lock_guard<std::mutex> lock(sv->mu);
  *id = sv->next_id++;
  sv->pending.emplace_back(*id, q);
  sv->pending_t.push_back(now_ms());
  return BS_OK;
}

int bs_server_progress(bs_server* sv, int* active, int* pending) {
  if (!sv) return set_error(BS_ERR_ARG, "bs_server_progress: NULL server");
  std::lock_guard<std::mutex> lock(sv->mu);
  int rc = progress(sv);
  if (active) {
    int n = 0;
    for (const Slot& sl : sv->slots) n += sl.phase != PH_FREE;
    *active = n;
  }
  if (pending) *pending = (int)sv->pending.size();
  return rc;
}

int bs_server_poll(bs_server* sv, bs_result* out, int max_results, int* n) {
  if (!sv || !n || (max_results > 0 && !out)) return set_error(BS_ERR_ARG, "bs_server_poll: NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  int c = 0;
  while (c < max_results && !sv->done.empty()) {
    out[c++] = sv->done.front();
    sv->done.pop_front();
  }
  *n = c;
  return BS_OK;
}

int bs_server_stats(bs_server* sv, bs_server_stats_t* st) {
  if (!sv || !st) return set_error(BS_ERR_ARG, "bs_server_stats: NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  st->arena_bytes = sv->arena.capacity();
  st->arena_used = sv->arena.used();
  st->fine_batches = sv->fine_batches;
  st->fine_items = sv->fine_items;
  st->coarse_sweeps = sv->coarse_sweeps;
  st->launches = sv->launches;
  return BS_OK;
}

int bs_server_destroy(bs_server* sv) {
  if (!sv) return BS_OK;
  cudaDeviceSynchronize();
  for (Slot& sl : sv->slots) {
    if (sl.g) bs_grid_destroy(sl.g);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.h_defect) cudaFreeHost(sl.h_defect);
    if (sl.h_status) cudaFreeHost(sl.h_status);
  }
  for (auto& kv : sv->grid_pool)
    for (bs_grid* g : kv.second) bs_grid_destroy(g);
  for (auto& kv : sv->class_grid) bs_grid_destroy(kv.second);
  for (auto& kv : sv->batch_stream) cudaStreamDestroy(kv.second);
  if (sv->pino_stream) cudaStreamDestroy(sv->pino_stream);
  for (auto& be : sv->batch_events)
    if (be) cudaEventDestroy(be);
  if (sv->arena_base) cudaFree(sv->arena_base);
  delete sv;
  return BS_OK;
}

}  // extern "C"
