// extern "C" entry points of include/cardiac_bddc.h: argument checks,
// error capture (no exception crosses the boundary) and the Newton drivers
// of Section 2 (load steps, Newton on Eq. tangent problem).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <cmath>
#include <new>
#include <string>

#include "bddc.h"
#include "fem.h"
#include "krylov.h"

namespace cbddc {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// bit 0: tensor cores on; bit 1: three-part split for the sweep updates;
// bit 2: three-part split for the other FP32 setup products
static std::atomic<int> g_tensor_cores{1};
bool tensor_cores_enabled() { return (g_tensor_cores.load(std::memory_order_relaxed) & 1) != 0; }
bool tensor_cores_for(bool sweep) {
  const int m = g_tensor_cores.load(std::memory_order_relaxed);
  return (m & 1) && !(m & (sweep ? 16 : 8));
}
bool tc_sweep_ks1() { return (g_tensor_cores.load(std::memory_order_relaxed) & 32) == 0; }
bool tc_other_ks1() { return (g_tensor_cores.load(std::memory_order_relaxed) & 64) != 0; }
int tc_parts(bool sweep) { return (g_tensor_cores.load(std::memory_order_relaxed) & (sweep ? 2 : 4)) ? 3 : 2; }

// Launch timer: event pairs recorded on the launching stream, one pool per
// kernel class; several classes can be recorded at the same time.
namespace {
constexpr int kTimerClasses = 16;
struct ClassTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  int depth = 0;      // nesting of begin/end of this class (multilevel recursion)
  bool open = false;  // the outermost begin recorded an event
  int64_t launches = 0;
  double flops = 0.0, bytes = 0.0;
  static constexpr size_t kMax = 65536;
  void reset() {
    used = 0;
    depth = 0;
    open = false;
    launches = 0;
    flops = bytes = 0.0;
  }
};
ClassTimer g_timers[kTimerClasses];
int g_timer_primary = 0;  // the class passed to cbddc_timer_start
}  // namespace

bool timer_active(int kernel_class) {
  return kernel_class > 0 && kernel_class < kTimerClasses && g_timers[kernel_class].on;
}

// Only the outermost begin/end pair of a class is recorded: the multilevel
// apply runs the level-2 apply inside the level-1 one, and its work is
// already counted in the outer call's flops and bytes.
void timer_begin(int kernel_class, cudaStream_t s) {
  if (!timer_active(kernel_class)) return;
  ClassTimer& t = g_timers[kernel_class];
  if (t.depth++ > 0) return;
  t.open = false;
  if (t.used + 2 > ClassTimer::kMax) return;
  while (t.pool.size() < t.used + 2) {
    cudaEvent_t e;
    CB_CUDA(cudaEventCreate(&e));
    t.pool.push_back(e);
  }
  CB_CUDA(cudaEventRecord(t.pool[t.used], s));
  t.open = true;
}

void timer_end(int kernel_class, cudaStream_t s, double flops, double bytes) {
  if (!timer_active(kernel_class)) return;
  ClassTimer& t = g_timers[kernel_class];
  if (t.depth == 0) return;
  if (--t.depth > 0 || !t.open) return;
  CB_CUDA(cudaEventRecord(t.pool[t.used + 1], s));
  t.open = false;
  t.used += 2;
  t.launches += 1;
  t.flops += flops;
  t.bytes += bytes;
}

static void timer_totals(int kernel_class, double* total_ms, int64_t* launches, double* flops, double* bytes) {
  const ClassTimer& t = g_timers[kernel_class];
  double ms = 0.0;
  for (size_t i = 0; i + 1 < t.used; i += 2) {
    CB_CUDA(cudaEventSynchronize(t.pool[i + 1]));
    float v = 0.f;
    CB_CUDA(cudaEventElapsedTime(&v, t.pool[i], t.pool[i + 1]));
    ms += v;
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = t.launches;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
}

template <typename F>
static int guard(F&& f) {
  try {
    f();
    return CBDDC_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return CBDDC_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return CBDDC_EINVAL;
  } catch (...) {
    set_last_error("unknown error");
    return CBDDC_EINVAL;
  }
}

// Reads and clears the device status word (synchronises the stream).
static int take_status(fem_problem* P, cudaStream_t s) {
  int h = 0;
  CB_CUDA(cudaMemcpyAsync(&h, P->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaMemsetAsync(P->status.p, 0, sizeof(int), s));
  CB_CUDA(cudaStreamSynchronize(s));
  return h;
}

static void fill_tangent(fem_problem* P, fem_tangent* K) {
  if (!K) return;
  K->vals = P->bsr_vals.p;
  K->row_ptr = P->bsr_row_ptr.p;
  K->col_idx = P->bsr_col.p;
  K->n_block_rows = P->n_free_nodes;
  K->nnzb = P->nnzb;
}

static int sweep_block_of(const bddc_options* opt) { return opt->sweep_block == 128 ? 128 : 64; }

static bddc_options options_of(const solve_options* opt) {
  bddc_options bo{};
  bo.precision = opt->precision;
  bo.primal = opt->primal;
  bo.pivot_tol = opt->pivot_tol;
  bo.levels = opt->levels;
  bo.n_parts2 = opt->n_parts2;
  bo.part2 = opt->part2;
  bo.primal2 = opt->primal2;
  bo.precision2 = opt->precision2;
  bo.scaling = opt->scaling;
  bo.coarse = opt->coarse;
  bo.sweep_block = opt->sweep_block;
  bo.tile_order = opt->tile_order;
  return bo;
}

static void ensure_ctx(fem_problem* P, const solve_options* opt, bddc_ctx** C) {
  if (*C) return;
  bddc_options bo = options_of(opt);
  const int pi = opt->precision == CBDDC_FP32 ? 1 : 0;
  if (opt->autotune && P->tuned_to[pi] >= 0) {
    bo.sweep_block = P->tuned_nb[pi];
    bo.tile_order = P->tuned_to[pi];
  }
  bddc_ctx* c = new bddc_ctx;
  try {
    bddc_create(P, &bo, c);
  } catch (...) {
    delete c;
    throw;
  }
  if (opt->autotune) {
    c->ms_setup_tuned = P->tuned_ms[pi];
    c->ms_setup_default = P->default_ms[pi];
  }
  *C = c;
}


static void ensure_work(bddc_ctx* C, int64_t n) {
  if (C->nw_r.n != (size_t)n) {
    C->nw_r.alloc(n);
    C->nw_b.alloc(n);
    C->nw_delta.alloc(n);
    C->nw_d.alloc(n);
  }
}

struct Events {
  cudaEvent_t e[5];
  Events() {
    for (auto& x : e) CB_CUDA(cudaEventCreate(&x));
  }
  ~Events() {
    for (auto& x : e) cudaEventDestroy(x);
  }
  float ms(int a, int b) const {
    float v = 0.f;
    cudaEventElapsedTime(&v, e[a], e[b]);
    return v;
  }
};

// Autotuning of the setup (solve_options.autotune): on the tangent at d,
// one timed setup (after an untimed one) per candidate {sweep block 64 /
// 128 (FP32 only)} x {tile order 0 / 1}; the fastest is cached in P per
// precision.  Returns the time spent (ms).
static float autotune_setup(fem_problem* P, const solve_options* opt, double lam, const double* d,
                            cudaStream_t s) {
  const int pi = opt->precision == CBDDC_FP32 ? 1 : 0;
  if (P->tuned_to[pi] >= 0) return 0.f;
  const auto t0 = std::chrono::steady_clock::now();
  {
    DVec<double> rtmp;
    rtmp.alloc(P->n_free);
    assemble(P, d, lam, rtmp.p, true, s);
    CB_CUDA(cudaStreamSynchronize(s));
  }
  CB_CHECK(!(take_status(P, s) & DEV_INVERTED), CBDDC_EINVERTED, "J <= 0 at a quadrature point");
  std::vector<int> nbs{64};
  if (opt->precision == CBDDC_FP32) nbs.push_back(128);
  float best = 1e30f, dflt = 0.f;
  int best_nb = 64, best_to = 0;
  for (int nb : nbs) {
    for (int to = 0; to < 2; ++to) {
      bddc_options bo = options_of(opt);
      bo.sweep_block = nb;
      bo.tile_order = to;
      std::unique_ptr<bddc_ctx> c(new bddc_ctx);
      bddc_create(P, &bo, c.get());
      bddc_run_setup(c.get(), s);
      Events ev;
      CB_CUDA(cudaEventRecord(ev.e[0], s));
      bddc_run_setup(c.get(), s);
      CB_CUDA(cudaEventRecord(ev.e[1], s));
      CB_CUDA(cudaEventSynchronize(ev.e[1]));
      const int st = take_status(P, s);
      if (st & (DEV_PIVOT | DEV_TIMEOUT)) continue;  // not a usable candidate
      const float ms = ev.ms(0, 1);
      if (nb == 64 && to == 0) dflt = ms;
      if (ms < best) {
        best = ms;
        best_nb = nb;
        best_to = to;
      }
    }
  }
  P->tuned_nb[pi] = best_nb;
  P->tuned_to[pi] = best_to;
  P->tuned_ms[pi] = best < 1e30f ? best : 0.f;
  P->default_ms[pi] = dflt;
  return std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// One Newton step at load lam: assemble residual + tangent, BDDC setup,
// GMRES on DF(d) delta = -F(d), d += delta.  Returns the GMRES status.
static int newton_step_impl(fem_problem* P, bddc_ctx** Cp, const solve_options* opt, double lam,
                            double* d, newton_record* rec, cudaStream_t s) {
  float tune_ms = 0.f;
  if (opt->autotune && *Cp == nullptr) tune_ms = autotune_setup(P, opt, lam, d, s);
  ensure_ctx(P, opt, Cp);
  bddc_ctx* C = *Cp;
  const int64_t n = P->n_free;
  ensure_work(C, n);
  Events ev;
  CB_CUDA(cudaEventRecord(ev.e[0], s));
  assemble(P, d, lam, C->nw_r.p, true, s);
  CB_CUDA(cudaEventRecord(ev.e[1], s));
  const int st = take_status(P, s);
  CB_CHECK(!(st & DEV_INVERTED), CBDDC_EINVERTED, "J <= 0 at a quadrature point");
  const double rn = device_norm(P, C->gm, C->nw_r.p, s);
  CB_CUDA(cudaEventRecord(ev.e[2], s));
  bddc_run_setup(C, s);
  CB_CUDA(cudaEventRecord(ev.e[3], s));
  const int st2 = take_status(P, s);
  CB_CHECK(!(st2 & DEV_TIMEOUT), CBDDC_ETIMEOUT, "a tensor-core setup kernel timed out on a device wait");
  CB_CHECK(!(st2 & DEV_PIVOT), CBDDC_EPIVOT, "tiny pivot in a local factorisation");
  axpby(-1.0, C->nw_r.p, 0.0, C->nw_r.p, C->nw_b.p, n, s);
  int its = 0;
  double rel = 0.0;
  const int gst = gmres_run(P, C, C->gm, C->nw_b.p, C->nw_delta.p, opt->restart > 0 ? opt->restart : 100,
                            opt->max_gmres > 0 ? opt->max_gmres : 1000,
                            opt->gmres_rtol > 0 ? opt->gmres_rtol : 1e-8, &its, &rel, s);
  axpby(1.0, d, 1.0, C->nw_delta.p, d, n, s);
  CB_CUDA(cudaEventRecord(ev.e[4], s));
  CB_CUDA(cudaEventSynchronize(ev.e[4]));
  if (rec) {
    rec->load = lam;
    rec->gmres_its = its;
    rec->res = rn;
    rec->ms_assemble = ev.ms(0, 1);
    rec->ms_setup = ev.ms(2, 3);
    rec->ms_gmres = ev.ms(3, 4);
    rec->ms_total = ev.ms(0, 4);
    rec->gmres_relres = rel;
    rec->gmres_reorth = C->gm.reorth;
    rec->ms_autotune = tune_ms;
  }
  return gst;
}

}  // namespace cbddc

using namespace cbddc;

extern "C" {

int fem_problem_create(const fem_problem_desc* desc, fem_problem** out) {
  return guard([&] {
    CB_CHECK(out != nullptr, CBDDC_EINVAL, "null output handle");
    *out = nullptr;
    fem_problem* P = new fem_problem;
    try {
      build_problem(desc, P);
    } catch (...) {
      delete P;
      throw;
    }
    *out = P;
  });
}

void fem_problem_destroy(fem_problem* P) { delete P; }

int fem_problem_get_info(const fem_problem* P, fem_problem_info* info) {
  return guard([&] {
    CB_CHECK(P && info, CBDDC_EINVAL, "null argument");
    info->n_free = P->n_free;
    info->n_block_rows = P->n_free_nodes;
    info->nnzb = P->nnzb;
    info->n_parts = P->n_parts;
    info->n_vertices = (int)P->vertices.size();
    info->n_edges = (int)P->edges.size();
    info->n_faces = (int)P->faces.size();
    int64_t mx = 0, sm = 0;
    for (auto& s : P->subs) {
      mx = std::max<int64_t>(mx, 3 * (int64_t)s.nodes.size());
      sm += 3 * (int64_t)s.nodes.size();
    }
    info->max_local_dofs = mx;
    info->sum_local_dofs = sm;
    info->device_bytes = P->device_bytes();
  });
}

int fem_residual(fem_problem* P, const double* d, double load_factor, double* residual,
                 cbddc_stream_t stream) {
  int inverted = 0;
  int rc = guard([&] {
    CB_CHECK(P && d && residual, CBDDC_EINVAL, "null argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    assemble(P, d, load_factor, residual, false, s);
    inverted = take_status(P, s) & DEV_INVERTED;
  });
  if (rc == CBDDC_OK && inverted) {
    set_last_error("J <= 0 at a quadrature point");
    return CBDDC_EINVERTED;
  }
  return rc;
}

int fem_assemble_tangent(fem_problem* P, const double* d, double load_factor, double* residual,
                         fem_tangent* K, cbddc_stream_t stream) {
  int inverted = 0;
  int rc = guard([&] {
    CB_CHECK(P && d, CBDDC_EINVAL, "null argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    assemble(P, d, load_factor, residual, true, s);
    inverted = take_status(P, s) & DEV_INVERTED;
    fill_tangent(P, K);
  });
  if (rc == CBDDC_OK && inverted) {
    set_last_error("J <= 0 at a quadrature point");
    return CBDDC_EINVERTED;
  }
  return rc;
}

int fem_tangent_copy(const fem_problem* P, double* vals, int32_t* row_ptr, int32_t* col_idx,
                     cbddc_stream_t stream) {
  return guard([&] {
    CB_CHECK(P != nullptr, CBDDC_EINVAL, "null problem");
    CB_CHECK(P->has_tangent, CBDDC_EINVAL, "no tangent assembled yet");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (vals)
      CB_CUDA(cudaMemcpyAsync(vals, P->bsr_vals.p, P->bsr_vals.bytes(), cudaMemcpyDeviceToDevice, s));
    if (row_ptr)
      CB_CUDA(cudaMemcpyAsync(row_ptr, P->bsr_row_ptr.p, P->bsr_row_ptr.bytes(), cudaMemcpyDeviceToDevice, s));
    if (col_idx)
      CB_CUDA(cudaMemcpyAsync(col_idx, P->bsr_col.p, P->bsr_col.bytes(), cudaMemcpyDeviceToDevice, s));
  });
}

int fem_spmv(fem_problem* P, const double* x, double* y, cbddc_stream_t stream) {
  return guard([&] {
    CB_CHECK(P && x && y, CBDDC_EINVAL, "null argument");
    CB_CHECK(P->has_tangent, CBDDC_EINVAL, "no tangent assembled yet");
    bsr_spmv(P, x, y, reinterpret_cast<cudaStream_t>(stream));
  });
}

int fem_set_time_state(fem_problem* P, double dt, const double* d_prev, const double* d_prev2) {
  return guard([&] {
    CB_CHECK(P != nullptr, CBDDC_EINVAL, "null problem");
    CB_CHECK(dt >= 0.0 && std::isfinite(dt), CBDDC_EINVAL, "dt must be finite and >= 0");
    if (dt > 0.0) CB_CHECK(d_prev && d_prev2, CBDDC_EINVAL, "previous displacements missing");
    P->dt = dt;
    P->d_prev = dt > 0.0 ? d_prev : nullptr;
    P->d_prev2 = dt > 0.0 ? d_prev2 : nullptr;
  });
}

int bddc_setup(fem_problem* P, const fem_tangent* K, const bddc_options* opt, bddc_ctx** inout,
               cbddc_stream_t stream) {
  return guard([&] {
    CB_CHECK(P && opt && inout, CBDDC_EINVAL, "null argument");
    CB_CHECK(P->has_tangent, CBDDC_EINVAL, "no tangent assembled yet");
    (void)K;  // the element matrices of the last assembly are used
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (*inout == nullptr) {
      bddc_ctx* c = new bddc_ctx;
      try {
        bddc_create(P, opt, c);
      } catch (...) {
        delete c;
        throw;
      }
      *inout = c;
    } else {
      bddc_ctx* c = *inout;
      CB_CHECK(c->P == P && c->precision == opt->precision && c->primal == opt->primal &&
                   c->levels == (opt->levels >= 3 ? 3 : 2) && c->scaling == opt->scaling &&
                   c->coarse == opt->coarse && c->nb == sweep_block_of(opt),
               CBDDC_EINVAL, "context was created for another problem or options");
    }
    bddc_run_setup(*inout, s);
    const int st = take_status(P, s);
    CB_CHECK(!(st & DEV_TIMEOUT), CBDDC_ETIMEOUT, "a tensor-core setup kernel timed out on a device wait");
    CB_CHECK(!(st & DEV_PIVOT), CBDDC_EPIVOT, "tiny pivot in a local factorisation");
  });
}

int bddc_apply(bddc_ctx* C, const double* r, double* z, cbddc_stream_t stream) {
  return guard([&] {
    CB_CHECK(C && r && z, CBDDC_EINVAL, "null argument");
    CB_CHECK(r != z, CBDDC_EINVAL, "r and z must not alias");
    bddc_run_apply(C, r, z, reinterpret_cast<cudaStream_t>(stream));
  });
}

void bddc_destroy(bddc_ctx* C) { delete C; }

int bddc_apply_noalloc(bddc_ctx* C, const double* r, double* z, cbddc_stream_t stream) {
  return guard([&] {
    CB_CHECK(C && r && z, CBDDC_EINVAL, "null argument");
    CB_CHECK(r != z, CBDDC_EINVAL, "r and z must not alias");
    bddc_run_apply_noalloc(C, r, z, reinterpret_cast<cudaStream_t>(stream));
  });
}

int bddc_get_info(const bddc_ctx* C, bddc_info* info) {
  return guard([&] {
    CB_CHECK(C && info, CBDDC_EINVAL, "null argument");
    info->n_primal = C->n_pi;
    info->n_primal2 = C->next ? C->next->n_pi : 0;
    info->precision = C->precision;
    info->local_bytes = C->local_bytes;
    info->device_bytes = C->device_bytes();
    info->setup_flops = C->setup_flops;
    info->sweep_block = C->nb;
    info->tile_order = C->tile_order;
    info->ms_setup_tuned = C->ms_setup_tuned;
    info->ms_setup_default = C->ms_setup_default;
  });
}

int gmres_solve(fem_problem* P, bddc_ctx* C, const double* b, double* x, const gmres_options* opt,
                gmres_report* rep, cbddc_stream_t stream) {
  int gst = CBDDC_OK;
  int rc = guard([&] {
    CB_CHECK(P && C && b && x && opt, CBDDC_EINVAL, "null argument");
    CB_CHECK(C->P == P, CBDDC_EINVAL, "context belongs to another problem");
    int its = 0;
    double rel = 0.0;
    gst = gmres_run(P, C, C->gm, b, x, opt->restart > 0 ? opt->restart : 100,
                    opt->max_iters > 0 ? opt->max_iters : 1000, opt->rtol > 0 ? opt->rtol : 1e-8, &its,
                    &rel, reinterpret_cast<cudaStream_t>(stream));
    if (rep) {
      rep->iterations = its;
      rep->converged = gst == CBDDC_OK;
      rep->rel_residual = rel;
    }
  });
  if (rc != CBDDC_OK) return rc;
  if (gst != CBDDC_OK) set_last_error("GMRES did not converge");
  return gst;
}

int newton_step(fem_problem* P, bddc_ctx** ctx, const solve_options* opt, double load_factor, double* d,
                newton_record* rec, cbddc_stream_t stream) {
  int gst = CBDDC_OK;
  int rc = guard([&] {
    CB_CHECK(P && ctx && opt && d, CBDDC_EINVAL, "null argument");
    gst = newton_step_impl(P, ctx, opt, load_factor, d, rec, reinterpret_cast<cudaStream_t>(stream));
  });
  if (rc != CBDDC_OK) return rc;
  if (gst != CBDDC_OK) set_last_error("GMRES did not converge");
  return gst;
}

int newton_step_host(fem_problem* P, bddc_ctx** ctx, const solve_options* opt, double load_factor,
                     double* d_host, newton_record* rec, cbddc_stream_t stream) {
  int gst = CBDDC_OK;
  int rc = guard([&] {
    CB_CHECK(P && ctx && opt && d_host, CBDDC_EINVAL, "null argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ensure_ctx(P, opt, ctx);
    ensure_work(*ctx, P->n_free);
    double* dd = (*ctx)->nw_d.p;
    const size_t bytes = P->n_free * sizeof(double);
    CB_CUDA(cudaMemcpyAsync(dd, d_host, bytes, cudaMemcpyHostToDevice, s));
    gst = newton_step_impl(P, ctx, opt, load_factor, dd, rec, s);
    CB_CUDA(cudaMemcpyAsync(d_host, dd, bytes, cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaStreamSynchronize(s));
  });
  if (rc != CBDDC_OK) return rc;
  if (gst != CBDDC_OK) set_last_error("GMRES did not converge");
  return gst;
}

int newton_gmres_solve(fem_problem* P, const solve_options* opt, double* d, solve_report* rep,
                       cbddc_stream_t stream) {
  bddc_ctx* C = nullptr;
  int rc = guard([&] {
    CB_CHECK(P && opt && d && rep, CBDDC_EINVAL, "null argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    *rep = solve_report{};
    const int64_t n = P->n_free;
    const double tol = opt->newton_rtol > 0 ? opt->newton_rtol : 1e-8;
    const int nsteps = std::max(1, opt->load_steps);
    const int max_newton = opt->max_newton > 0 ? opt->max_newton : 25;
    const int max_halv = opt->max_halvings >= 0 ? opt->max_halvings : 6;
    ensure_ctx(P, opt, &C);
    ensure_work(C, n);
    DVec<double> dtry;
    dtry.alloc(n);
    std::vector<double> targets;
    for (int k = 1; k <= nsteps; ++k) targets.push_back((double)k / nsteps);
    double lam_prev = 0.0;
    while (!targets.empty()) {
      const double lam = targets.front();
      CB_CUDA(cudaMemcpyAsync(dtry.p, d, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      bool ok = false;
      bool failed = false;
      assemble(P, dtry.p, lam, C->nw_r.p, false, s);
      if (take_status(P, s) & DEV_INVERTED) failed = true;
      double r0 = failed ? 0.0 : device_norm(P, C->gm, C->nw_r.p, s);
      double rn = r0;
      for (int it = 0; it < max_newton && !failed; ++it) {
        if (rn <= tol * r0 || rn == 0.0) { ok = true; break; }
        newton_record rec{};
        int gst = CBDDC_OK;
        try {
          gst = newton_step_impl(P, &C, opt, lam, dtry.p, &rec, s);
        } catch (const Error& e) {
          if (e.code != CBDDC_EINVERTED && e.code != CBDDC_EPIVOT) throw;
          failed = true;
          break;
        }
        rec.newton = it;
        rec.res0 = r0;
        if (rep->n_records < CBDDC_MAX_RECORDS) rep->rec[rep->n_records++] = rec;
        rep->newton_steps++;
        rep->total_gmres_its += rec.gmres_its;
        if (gst != CBDDC_OK) { failed = true; break; }
        assemble(P, dtry.p, lam, C->nw_r.p, false, s);
        if (take_status(P, s) & DEV_INVERTED) { failed = true; break; }
        rn = device_norm(P, C->gm, C->nw_r.p, s);
        if (!std::isfinite(rn)) { failed = true; break; }
      }
      if (!ok && !failed && rn <= tol * r0) ok = true;
      if (ok) {
        CB_CUDA(cudaMemcpyAsync(d, dtry.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        lam_prev = lam;
        targets.erase(targets.begin());
        rep->load_steps_done++;
        rep->final_rel_residual = r0 > 0 ? rn / r0 : 0.0;
      } else {
        rep->halvings++;
        CB_CHECK(rep->halvings <= max_halv, CBDDC_ENOCONV, "Newton failed to converge");
        targets.insert(targets.begin(), 0.5 * (lam_prev + lam));
      }
    }
    CB_CUDA(cudaStreamSynchronize(s));
  });
  delete C;
  if (rep) rep->status = rc;
  return rc;
}

const char* cbddc_last_error(void) { return g_last_error.c_str(); }

uint64_t cbddc_kernel_launches(void) { return g_launches.load(); }

int cbddc_set_tensor_cores(int mode) { return g_tensor_cores.exchange(mode & 127); }

int cbddc_timer_start(int kernel_class) {
  return guard([&] {
    CB_CHECK(kernel_class >= 0 && kernel_class <= CBDDC_TIMER_SETUP_GEMM_F64, CBDDC_EINVAL, "bad kernel class");
    for (auto& t : g_timers) {
      t.on = false;
      t.reset();
    }
    g_timer_primary = kernel_class;
    if (kernel_class > 0) g_timers[kernel_class].on = true;
  });
}

int cbddc_timer_enable(int kernel_class) {
  return guard([&] {
    CB_CHECK(kernel_class > 0 && kernel_class <= CBDDC_TIMER_SETUP_GEMM_F64, CBDDC_EINVAL, "bad kernel class");
    ClassTimer& t = g_timers[kernel_class];
    if (!t.on) {
      t.reset();
      t.on = true;
    }
  });
}

int cbddc_timer_result(int kernel_class, double* total_ms, int64_t* launches, double* flops, double* bytes) {
  return guard([&] {
    CB_CHECK(kernel_class > 0 && kernel_class <= CBDDC_TIMER_SETUP_GEMM_F64, CBDDC_EINVAL, "bad kernel class");
    timer_totals(kernel_class, total_ms, launches, flops, bytes);
  });
}

int cbddc_timer_stop(double* total_ms, int64_t* launches, double* flops, double* bytes) {
  return guard([&] {
    if (g_timer_primary > 0) {
      timer_totals(g_timer_primary, total_ms, launches, flops, bytes);
    } else {
      if (total_ms) *total_ms = 0.0;
      if (launches) *launches = 0;
      if (flops) *flops = 0.0;
      if (bytes) *bytes = 0.0;
    }
    for (auto& t : g_timers) {
      t.on = false;
      t.reset();
    }
    g_timer_primary = 0;
  });
}

}  // extern "C"
