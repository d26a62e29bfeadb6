// C ABI of the DMK Stokes near-field library (see include/dmk_stokes.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "common.cuh"


namespace {

thread_local std::string g_last_error;

dmk_status_t set_err(dmk_stokes_plan_t plan, dmk_status_t code, const std::string& msg) {
  g_last_error = msg;
  if (plan) plan->p.last_error = msg;
  return code;
}

bool valid_plan(dmk_stokes_plan_t plan) { return plan && plan->p.magic == dmk::kPlanMagic; }

dmk_status_t validate_opts(const dmk_stokes_opts_t* o, std::string& msg) {
  if (!o) { msg = "opts is NULL"; return DMK_ERR_INVALID_ARG; }
  if (o->dim != 2 && o->dim != 3) { msg = "dim must be 2 or 3"; return DMK_ERR_INVALID_ARG; }
  if (o->periodic != 0 && o->periodic != 1) { msg = "periodic must be 0 or 1"; return DMK_ERR_INVALID_ARG; }
  if (o->kernels < 1 || o->kernels > 3) { msg = "kernels must be a nonzero mask of 1|2"; return DMK_ERR_INVALID_ARG; }
  if (o->precision != 0 && o->precision != 1) { msg = "precision must be 0 or 1"; return DMK_ERR_INVALID_ARG; }
  if (o->components != DMK_COMPONENTS_ALL && o->components != DMK_COMPONENTS_NEAR &&
      o->components != DMK_COMPONENTS_EWALD) {
    msg = "components must be 0, 1 or 2";
    return DMK_ERR_INVALID_ARG;
  }
  if (o->leaf_capacity < 0 || o->leaf_capacity > (1 << 20)) { msg = "leaf_capacity out of range"; return DMK_ERR_INVALID_ARG; }
  if (o->n_rhs < 1 || o->n_rhs > 16) { msg = "n_rhs must be in 1..16"; return DMK_ERR_INVALID_ARG; }
  if (o->bandlimit != 0 && (o->bandlimit < 2 || o->bandlimit > 36)) {
    msg = "bandlimit (3c/pi) must be 0 or in 2..36";
    return DMK_ERR_INVALID_ARG;
  }
  if (!(o->eps >= 1e-12 * (1 - 1e-9) && o->eps <= 1e-3 * (1 + 1e-9))) {
    msg = "eps must lie in [1e-12, 1e-3] (Table 2 range)";
    return DMK_ERR_INVALID_ARG;
  }
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(o->box_lo[a])) { msg = "box_lo not finite"; return DMK_ERR_INVALID_ARG; }
  if (o->components == DMK_COMPONENTS_EWALD &&
      !(o->periodic == 1 && o->dim == 3 && o->kernels == DMK_KERNEL_STOKESLET && o->n_rhs == 1)) {
    msg = "components = DMK_COMPONENTS_EWALD is provided for the periodic 3D Stokeslet with one force column";
    return DMK_ERR_UNSUPPORTED;
  }
  if (o->components == DMK_COMPONENTS_ALL && o->n_rhs != 1) {
    msg = "components = DMK_COMPONENTS_ALL (the DMK far field) takes one force column";
    return DMK_ERR_UNSUPPORTED;
  }
  if (o->n_rhs != 1 && (o->kernels & DMK_KERNEL_STRESSLET)) {
    msg = "the stresslet takes one density column (n_rhs = 1)";
    return DMK_ERR_UNSUPPORTED;
  }
  return DMK_OK;
}

// Kernel tables depend only on (dim, c, FP32 tolerance); the 2D ones take a
// few tens of milliseconds of host quadrature (App. B), so every process keeps
// the tables it has built and plans with the same parameters copy them.
// Truncation of the FP32 tables (Chebyshev tail relative to max |f|): a tenth
// of eps, no lower than FP32 rounding of the pair terms can use.
double fp32_table_tol(double eps) { return std::max(eps / 10.0, 1e-8); }

bool cached_tables(int dim, double c, double fp32_tol, dmk::KernelTables* out) {
  struct Entry {
    int dim;
    double c, tol;
    std::unique_ptr<dmk::KernelTables> tables;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  std::lock_guard<std::mutex> lk(mu);
  for (const Entry& e : cache)
    if (e.dim == dim && e.c == c && e.tol == fp32_tol) {
      *out = *e.tables;
      return true;
    }
  auto t = std::make_unique<dmk::KernelTables>();
  if (dmk::build_tables(dim, c, fp32_tol, t.get()) != 0) return false;
  *out = *t;
  if (cache.size() < 64) cache.push_back(Entry{dim, c, fp32_tol, std::move(t)});
  return true;
}

}  // namespace

namespace dmk {
namespace {
// pinned slots: blocks of 256 slots of 16 int32, handed out from a free list
struct PinnedPool {
  std::mutex mu;
  std::vector<int32_t*> free_list;
};
PinnedPool& pinned_pool() {
  static PinnedPool pool;   // blocks stay allocated until the process exits
  return pool;
}
}  // namespace

int32_t* pinned_slot() {
  PinnedPool& pool = pinned_pool();
  std::lock_guard<std::mutex> lk(pool.mu);
  if (pool.free_list.empty()) {
    void* b = nullptr;
    if (cudaMallocHost(&b, 256 * 16 * sizeof(int32_t)) != cudaSuccess)
      throw Error{DMK_ERR_NOMEM, "pinned host allocation failed"};
    for (int k = 255; k >= 0; --k) pool.free_list.push_back(static_cast<int32_t*>(b) + 16 * k);
  }
  int32_t* r = pool.free_list.back();
  pool.free_list.pop_back();
  return r;
}

void pinned_release(int32_t* slot) {
  PinnedPool& pool = pinned_pool();
  std::lock_guard<std::mutex> lk(pool.mu);
  pool.free_list.push_back(slot);
}
}  // namespace dmk

namespace {

void configure_pool(int dev) {
  static std::mutex mu;
  static std::set<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(dev)) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;   // keep freed blocks cached in the pool
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done.insert(dev);
}

void release(dmk::Plan& p) {
  dmk::ewald_free(p);
  dmk::far_free(p);
  if (p.aux) cudaFreeAsync(p.aux, p.stream);
  p.aux = nullptr;
  p.aux_bytes = 0;
  dmk::free_tree(p.tree, p.stream);
  p.fsorted = nullptr;
  p.reduce_buf = nullptr;
  p.status = nullptr;
  p.arena.release();
  if (p.h_status) dmk::pinned_release(p.h_status);
  p.h_status = nullptr;
}

dmk_status_t make_plan(const dmk_stokes_opts_t* opts, int32_t n_sys, const int64_t* h_offsets,
                       const double* d_src, const double* d_trg, int64_t n_trg, void* stream,
                       dmk_stokes_plan_t* out) {
  if (!out) return set_err(nullptr, DMK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::string msg;
  dmk_status_t st = validate_opts(opts, msg);
  if (st != DMK_OK) return set_err(nullptr, st, msg);
  if (n_sys < 1 || !h_offsets) return set_err(nullptr, DMK_ERR_INVALID_ARG, "bad system offsets");
  if (h_offsets[0] != 0) return set_err(nullptr, DMK_ERR_INVALID_ARG, "h_offsets[0] must be 0");
  for (int k = 0; k < n_sys; ++k)
    if (h_offsets[k + 1] < h_offsets[k]) return set_err(nullptr, DMK_ERR_INVALID_ARG, "h_offsets decreasing");
  const int64_t N = h_offsets[n_sys];
  if (N >= (int64_t(1) << 31)) return set_err(nullptr, DMK_ERR_INVALID_ARG, "too many points (>= 2^31)");
  if (N > 0 && !d_src) return set_err(nullptr, DMK_ERR_INVALID_ARG, "d_src is NULL");
  if (d_trg && n_sys != 1) return set_err(nullptr, DMK_ERR_UNSUPPORTED, "separate targets need a single system");
  if (opts && opts->components == DMK_COMPONENTS_EWALD && (n_sys != 1 || d_trg))
    return set_err(nullptr, DMK_ERR_UNSUPPORTED, "components = EWALD needs a single system, targets = sources");
  if (opts && opts->components == DMK_COMPONENTS_ALL && n_sys != 1)
    return set_err(nullptr, DMK_ERR_UNSUPPORTED, "components = ALL needs a single system");
  if (d_trg && (n_trg < 0 || n_trg >= (int64_t(1) << 31)))
    return set_err(nullptr, DMK_ERR_INVALID_ARG, "n_trg out of range");

  dmk_stokes_plan_t plan = new (std::nothrow) dmk_stokes_plan_s();
  if (!plan) return set_err(nullptr, DMK_ERR_NOMEM, "host allocation failed");
  dmk::Plan& p = plan->p;
  p.opts = *opts;
  p.stream = static_cast<cudaStream_t>(stream);
  plan->last_stream = p.stream;
  try {
    DMK_CUDA_TRY(cudaGetDevice(&p.device));
    configure_pool(p.device);
    double c = opts->bandlimit > 0 ? opts->bandlimit * M_PI / 3.0 : dmk::bandlimit_for_eps(opts->eps, opts->kernels);
    if (c <= 0) throw dmk::Error{DMK_ERR_INVALID_ARG, "eps outside Table 2 range"};
    if (!cached_tables(opts->dim, c, fp32_table_tol(opts->eps), &p.tables))
      throw dmk::Error{DMK_ERR_UNSUPPORTED, "kernel tables could not be built for this dimension"};
    p.leaf_capacity = opts->leaf_capacity > 0 ? opts->leaf_capacity
                                              : dmk::leaf_capacity_for_eps(opts->eps, opts->dim);
    if (opts->components == DMK_COMPONENTS_EWALD) p.uniform_level = dmk::ewald_level(N, opts->leaf_capacity);
    p.tree.N = N;
    p.tree.n_sys = n_sys;
    // one arena block for the tree (~80 bytes per point) and the evaluation workspace
    p.arena.s = p.stream;
    p.fsorted_bytes = dmk::eval_workspace_bytes(p.opts, N, d_trg ? n_trg : N);
    p.arena.reserve(p.fsorted_bytes + static_cast<size_t>(N) * 96 + 32 * static_cast<size_t>(n_sys) +
                    (size_t(8) << 20));
    p.status = p.arena.alloc<int>(1);
    DMK_CUDA_TRY(cudaMemsetAsync(p.status, 0, sizeof(int), p.stream));
    p.h_status = dmk::pinned_slot();
    dmk::build_tree(p, d_src, h_offsets);
    if (d_trg) dmk::build_targets(p, d_trg, n_trg);
    if (p.uniform_level > 0) dmk::ewald_setup(p, p.uniform_level);
    if (opts->components == DMK_COMPONENTS_ALL) dmk::far_setup(p);
    p.fsorted = p.arena.alloc<char>(p.fsorted_bytes);
    p.reduce_buf = p.arena.alloc<double>(4 * n_sys);
    DMK_CUDA_TRY(cudaGetLastError());
    // everything above is complete when the call returns: the plan may then be
    // used from any stream and the coordinate buffer reused
    DMK_CUDA_TRY(cudaStreamSynchronize(p.stream));
  } catch (const dmk::Error& e) {
    release(p);
    delete plan;
    return set_err(nullptr, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    release(p);
    delete plan;
    return set_err(nullptr, DMK_ERR_NOMEM, "host allocation failed");
  }
  p.magic = dmk::kPlanMagic;
  *out = plan;
  return DMK_OK;
}

}  // namespace

dmk_status_t dmk::record_error(dmk_stokes_plan_t plan, dmk_status_t code, const std::string& msg) {
  return set_err(plan, code, msg);
}

extern "C" {

dmk_status_t dmk_stokes_plan(const dmk_stokes_opts_t* opts, int64_t n_src, const double* d_src,
                             int64_t n_trg, const double* d_trg, void* stream, dmk_stokes_plan_t* out) {
  if (out) *out = nullptr;
  if (n_src < 0) return set_err(nullptr, DMK_ERR_INVALID_ARG, "n_src < 0");
  if (!d_trg && n_trg != n_src && n_trg != 0)
    return set_err(nullptr, DMK_ERR_INVALID_ARG, "d_trg is NULL (targets are the sources) but n_trg != n_src");
  int64_t offs[2] = {0, n_src};
  if (!d_trg && n_trg == 0 && n_src > 0) {
    // an empty set of separate targets (no valid pointer exists for it)
    static const double kNoTarget[3] = {0.0, 0.0, 0.0};
    return make_plan(opts, 1, offs, d_src, kNoTarget, 0, stream, out);
  }
  return make_plan(opts, 1, offs, d_src, d_trg, n_trg, stream, out);
}

dmk_status_t dmk_stokes_plan_batched(const dmk_stokes_opts_t* opts, int32_t n_sys, const int64_t* h_offsets,
                                     const double* d_src, void* stream, dmk_stokes_plan_t* out) {
  if (out) *out = nullptr;
  if (n_sys > 65535) return set_err(nullptr, DMK_ERR_INVALID_ARG, "n_sys > 65535");
  return make_plan(opts, n_sys, h_offsets, d_src, nullptr, 0, stream, out);
}

// The gradient and adjoint workspace (aux) is allocated on the plan's stream
// by the first call that needs it, and the stream synchronised so that any
// stream may use it; later calls reuse it.
static void ensure_aux(dmk_stokes_plan_t plan, size_t bytes) {
  dmk::Plan& p = plan->p;
  if (bytes == 0 || p.aux_bytes >= bytes) return;
  if (p.aux) {
    // a smaller workspace from an earlier call: let its work finish first
    DMK_CUDA_TRY(cudaStreamSynchronize(plan->last_stream));
    cudaFreeAsync(p.aux, p.stream);
  }
  p.aux = nullptr;
  p.aux_bytes = 0;
  DMK_CUDA_TRY(cudaMallocAsync(&p.aux, bytes, p.stream));
  DMK_CUDA_TRY(cudaStreamSynchronize(p.stream));
  p.aux_bytes = bytes;
}

static dmk_status_t run_eval(dmk_stokes_plan_t plan, const double* d_f, const double* d_g, const double* d_n,
                             double* d_u, double* d_gradu, void* stream) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  dmk::Plan& p = plan->p;
  const int64_t N = p.tree.N;
  const int64_t NT = p.tree.sep ? p.tree.NT : N;
  const bool want_s = p.opts.kernels & DMK_KERNEL_STOKESLET;
  const bool want_t = p.opts.kernels & DMK_KERNEL_STRESSLET;
  if (N > 0) {
    if (want_s && !d_f) return set_err(plan, DMK_ERR_INVALID_ARG, "d_f is NULL but the Stokeslet is requested");
    if (want_t && (!d_g || !d_n)) return set_err(plan, DMK_ERR_INVALID_ARG, "d_g / d_n NULL but the stresslet is requested");
  }
  if (NT > 0 && !d_u && !d_gradu) return set_err(plan, DMK_ERR_INVALID_ARG, "d_u is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  plan->last_stream = s;
  if ((p.ewald || p.far) && d_gradu)
    return set_err(plan, DMK_ERR_UNSUPPORTED, "the gradient of components = ALL / EWALD is not provided");
  try {
    if (d_gradu && N > 0) ensure_aux(plan, dmk::aux_bytes_grad(p.opts, N));
    if (p.trace) DMK_CUDA_TRY(cudaEventRecord(p.trace[0], s));
    dmk::launch_near(p, want_s ? d_f : nullptr, want_t ? d_g : nullptr, want_t ? d_n : nullptr, d_u, d_gradu, s);
    if (p.trace) DMK_CUDA_TRY(cudaEventRecord(p.trace[1], s));
    if (p.ewald && d_u) dmk::ewald_far(p, d_f, d_u, s);   // + the Fourier part (Ewald far field)
    if (p.far && d_u) dmk::far_run(p, want_s ? d_f : nullptr, want_t ? d_g : nullptr, want_t ? d_n : nullptr, d_u, s);
  } catch (const dmk::Error& e) {
    return set_err(plan, e.code, e.msg);
  }
  return DMK_OK;
}

dmk_status_t dmk_stokes_eval(dmk_stokes_plan_t plan, const double* d_f, const double* d_g, const double* d_n,
                             double* d_u, void* stream) {
  if (valid_plan(plan) && (plan->p.tree.sep ? plan->p.tree.NT : plan->p.tree.N) > 0 && !d_u)
    return set_err(plan, DMK_ERR_INVALID_ARG, "d_u is NULL");
  return run_eval(plan, d_f, d_g, d_n, d_u, nullptr, stream);
}

dmk_status_t dmk_stokes_eval_grad(dmk_stokes_plan_t plan, const double* d_f, const double* d_g,
                                  const double* d_n, double* d_u, double* d_gradu, void* stream) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  if (plan->p.opts.dim != 3) return set_err(plan, DMK_ERR_UNSUPPORTED, "the gradient is provided in 3D");
  if (plan->p.opts.n_rhs != 1)
    return set_err(plan, DMK_ERR_UNSUPPORTED, "the gradient is provided for n_rhs = 1");
  if ((plan->p.tree.sep ? plan->p.tree.NT : plan->p.tree.N) > 0 && !d_gradu)
    return set_err(plan, DMK_ERR_INVALID_ARG, "d_gradu is NULL");
  return run_eval(plan, d_f, d_g, d_n, d_u, d_gradu, stream);
}

dmk_status_t dmk_stokes_eval_adjoint(dmk_stokes_plan_t plan, const double* d_f, const double* d_w, double* d_v,
                                     double* d_gx, void* stream) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  dmk::Plan& p = plan->p;
  if (p.opts.dim != 3) return set_err(plan, DMK_ERR_UNSUPPORTED, "the adjoint is provided in 3D");
  if (p.opts.kernels != DMK_KERNEL_STOKESLET)
    return set_err(plan, DMK_ERR_UNSUPPORTED, "the adjoint is provided for the Stokeslet only");
  if (p.opts.n_rhs != 1) return set_err(plan, DMK_ERR_UNSUPPORTED, "the adjoint is provided for n_rhs = 1");
  if (p.tree.sep) return set_err(plan, DMK_ERR_UNSUPPORTED, "the adjoint is provided for targets = sources");
  if (p.ewald || p.far) return set_err(plan, DMK_ERR_UNSUPPORTED, "the adjoint of components = ALL / EWALD is not provided");
  const int64_t N = p.tree.N;
  if (N > 0 && (!d_f || !d_w || !d_v || !d_gx))
    return set_err(plan, DMK_ERR_INVALID_ARG, "d_f, d_w, d_v and d_gx are required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  plan->last_stream = s;
  try {
    if (N > 0) ensure_aux(plan, dmk::aux_bytes_adjoint(p.opts, N));
    dmk::launch_adjoint(p, d_f, d_w, d_v, d_gx, s, p.aux);
  } catch (const dmk::Error& e) {
    return set_err(plan, e.code, e.msg);
  }
  return DMK_OK;
}

dmk_status_t dmk_stokes_autotune(const dmk_stokes_opts_t* opts, int64_t n_src, const double* d_src,
                                 const double* d_f, const double* d_g, const double* d_n, double* d_u,
                                 int32_t n_cand, const int32_t* h_leaf_capacity, int32_t repeats, void* stream,
                                 double* h_ms, int32_t* h_best) {
  if (!opts || n_cand < 1 || !h_leaf_capacity || repeats < 1 || !h_best)
    return set_err(nullptr, DMK_ERR_INVALID_ARG, "bad autotune arguments");
  for (int k = 0; k < n_cand; ++k)
    if (h_leaf_capacity[k] < 1) return set_err(nullptr, DMK_ERR_INVALID_ARG, "candidate leaf capacity < 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_err(nullptr, DMK_ERR_CUDA, "cudaEventCreate failed");
  std::vector<double> med(n_cand);
  dmk_status_t st = DMK_OK;
  for (int k = 0; k < n_cand && st == DMK_OK; ++k) {
    dmk_stokes_opts_t o = *opts;
    o.leaf_capacity = h_leaf_capacity[k];
    std::vector<float> ms;
    for (int r = 0; r <= repeats && st == DMK_OK; ++r) {   // the first run warms the pools up, untimed
      cudaEventRecord(e0, s);
      dmk_stokes_plan_t plan = nullptr;
      st = dmk_stokes_plan(&o, n_src, d_src, n_src, nullptr, stream, &plan);
      if (st == DMK_OK) st = dmk_stokes_eval(plan, d_f, d_g, d_n, d_u, stream);
      if (plan) dmk_stokes_destroy(plan);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = set_err(nullptr, DMK_ERR_CUDA, "autotune timing failed");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) ms.push_back(t);
    }
    if (st != DMK_OK) break;
    std::sort(ms.begin(), ms.end());
    med[k] = ms[ms.size() / 2];
    if (h_ms) h_ms[k] = med[k];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DMK_OK) return st;
  *h_best = static_cast<int32_t>(std::min_element(med.begin(), med.end()) - med.begin());
  return DMK_OK;
}

dmk_status_t dmk_stokes_eval_traced(dmk_stokes_plan_t plan, const double* d_f, const double* d_g, const double* d_n,
                                    double* d_u, void* stream, double* h_stage_ms, int32_t n_stages) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  if (!h_stage_ms || n_stages < 1 || n_stages > 9) return set_err(plan, DMK_ERR_INVALID_ARG, "h_stage_ms / n_stages");
  if (!d_u) return set_err(plan, DMK_ERR_INVALID_ARG, "d_u is NULL");
  dmk::Plan& p = plan->p;
  cudaEvent_t ev[10];
  int made = 0;
  for (; made < 10; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  if (made < 10) {
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    return set_err(plan, DMK_ERR_CUDA, "cudaEventCreate failed");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // stages without work (no far field) take zero time: record every event once first
  for (int i = 0; i < 10; ++i) cudaEventRecord(ev[i], s);
  p.trace = ev;
  dmk_status_t st = run_eval(plan, d_f, d_g, d_n, d_u, nullptr, stream);
  p.trace = nullptr;
  if (st == DMK_OK) {
    if (!p.far) cudaEventRecord(ev[9], s);
    if (cudaEventSynchronize(ev[9]) != cudaSuccess) st = set_err(plan, DMK_ERR_CUDA, "traced evaluation failed");
  }
  if (st == DMK_OK) {
    for (int i = 0; i < n_stages; ++i) {
      float ms = 0.f;
      int a = i, b = i + 1;
      if (!p.far && i >= 1) {           // no far field: everything after the near pass is empty
        h_stage_ms[i] = 0.0;
        continue;
      }
      cudaEventElapsedTime(&ms, ev[a], ev[b]);
      h_stage_ms[i] = ms;
    }
  }
  for (int i = 0; i < 10; ++i) cudaEventDestroy(ev[i]);
  return st;
}

dmk_status_t dmk_stokes_far_info(dmk_stokes_plan_t plan, int32_t info[8]) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  if (!info) return set_err(plan, DMK_ERR_INVALID_ARG, "info is NULL");
  dmk::far_info(plan->p, info);
  return DMK_OK;
}

dmk_status_t dmk_stokes_tc_wait_selftest(void* stream, int32_t* h_timed_out) {
  if (!h_timed_out) return set_err(nullptr, DMK_ERR_INVALID_ARG, "h_timed_out is NULL");
  try {
    *h_timed_out = dmk::tc_wait_selftest(static_cast<cudaStream_t>(stream)) ? 1 : 0;
  } catch (const dmk::Error& e) {
    return set_err(nullptr, e.code, e.msg);
  }
  return DMK_OK;
}

dmk_status_t dmk_stokes_sync_status(dmk_stokes_plan_t plan) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  dmk::Plan& p = plan->p;
  cudaError_t e = cudaStreamSynchronize(plan->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
  if (e != cudaSuccess) return set_err(plan, DMK_ERR_CUDA, cudaGetErrorString(e));
  e = cudaMemcpy(p.h_status, p.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_err(plan, DMK_ERR_CUDA, cudaGetErrorString(e));
  int st = *p.h_status;
  if (st & dmk::ST_NONFINITE) return set_err(plan, DMK_ERR_INVALID_ARG, "non-finite coordinate");
  if (st & dmk::ST_OUT_OF_RANGE) return set_err(plan, DMK_ERR_OUT_OF_RANGE, "point outside the unit box");
  if (st & (dmk::ST_NEAR_OVERFLOW | dmk::ST_TREE_INCONSISTENT))
    return set_err(plan, DMK_ERR_CUDA, "internal tree inconsistency");
  if (st & dmk::ST_TC_TIMEOUT) return set_err(plan, DMK_ERR_CUDA, "tensor-core wait timed out in the far field");
  return DMK_OK;
}

dmk_status_t dmk_stokes_plan_stats(dmk_stokes_plan_t plan, int64_t stats[10]) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  if (!stats) return set_err(plan, DMK_ERR_INVALID_ARG, "stats is NULL");
  dmk::Plan& p = plan->p;
  const dmk::DeviceTree& T = p.tree;
  std::vector<int32_t> lvl(T.n_leaf), cnt(T.n_leaf), off(T.n_leaf + 1), nl(T.n_near);
  cudaStream_t s = p.stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return set_err(plan, DMK_ERR_CUDA, "stream sync failed");
  if (T.n_leaf > 0) {
    cudaMemcpy(lvl.data(), T.leaf_level, T.n_leaf * sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaMemcpy(cnt.data(), T.leaf_count, T.n_leaf * sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaMemcpy(off.data(), T.near_off, (T.n_leaf + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
  }
  if (T.n_near > 0) cudaMemcpy(nl.data(), T.near_leaf, T.n_near * sizeof(int32_t), cudaMemcpyDeviceToHost);
  std::vector<int32_t> tst(T.sep ? T.n_leaf + 1 : 0);
  if (T.sep && T.n_leaf > 0)
    cudaMemcpy(tst.data(), T.leaf_tstart, (T.n_leaf + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
  int64_t issued = 0;
  int maxl = 0;
  for (int i = 0; i < T.n_leaf; ++i) {
    maxl = std::max(maxl, lvl[i]);
    int64_t src = 0;
    for (int e = off[i]; e < off[i + 1]; ++e) src += cnt[nl[e]];
    // targets of leaf i times the sources of its near leaves (the target itself excluded)
    issued += T.sep ? int64_t(tst[i + 1] - tst[i]) * src : int64_t(cnt[i]) * src - cnt[i];
  }
  stats[0] = T.n_leaf;
  stats[1] = maxl;
  stats[2] = T.n_near;
  stats[3] = T.n_tile;
  stats[4] = issued;
  stats[5] = static_cast<int64_t>(std::lround(p.tables.c * 3.0 / M_PI));
  stats[6] = p.leaf_capacity;
  stats[7] = T.N;
  if (p.useful_pairs < 0) {
    try {
      p.useful_pairs = dmk::count_useful_pairs(p);
    } catch (const dmk::Error& e) {
      return set_err(plan, e.code, e.msg);
    }
  }
  stats[8] = p.useful_pairs;
  stats[9] = p.launches;
  return DMK_OK;
}

dmk_status_t dmk_stokes_plan_tree(dmk_stokes_plan_t plan, int32_t* perm, int32_t* leaf_level, int32_t* leaf_start,
                                  int32_t* leaf_count, int64_t* leaf_coords, int32_t* near_off,
                                  int32_t* near_leaf, int32_t* near_q) {
  if (!valid_plan(plan)) return set_err(nullptr, DMK_ERR_BAD_PLAN, "invalid plan handle");
  dmk::Plan& p = plan->p;
  const dmk::DeviceTree& T = p.tree;
  const int D = p.opts.dim;
  if (cudaStreamSynchronize(p.stream) != cudaSuccess) return set_err(plan, DMK_ERR_CUDA, "stream sync failed");
  auto cp = [](void* dst, const void* src, size_t bytes) {
    if (dst && bytes) cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
  };
  cp(perm, T.perm, T.N * sizeof(int32_t));
  cp(leaf_level, T.leaf_level, T.n_leaf * sizeof(int32_t));
  cp(leaf_start, T.leaf_start, T.n_leaf * sizeof(int32_t));
  cp(leaf_count, T.leaf_count, T.n_leaf * sizeof(int32_t));
  cp(near_off, T.near_off, (T.n_leaf + 1) * sizeof(int32_t));
  cp(near_leaf, T.near_leaf, T.n_near * sizeof(int32_t));
  if (leaf_coords) {
    std::vector<uint64_t> anc(T.n_leaf);
    std::vector<int32_t> lv(T.n_leaf);
    cp(anc.data(), T.leaf_anchor, T.n_leaf * sizeof(uint64_t));
    cp(lv.data(), T.leaf_level, T.n_leaf * sizeof(int32_t));
    for (int i = 0; i < T.n_leaf; ++i) {
      int64_t c[3];
      if (D == 3) dmk::leaf_coords<3>(anc[i], lv[i], T.M, c);
      else dmk::leaf_coords<2>(anc[i], lv[i], T.M, c);
      for (int a = 0; a < D; ++a) leaf_coords[int64_t(i) * D + a] = c[a];
    }
  }
  if (near_q) {
    std::vector<int32_t> q(T.n_near);
    cp(q.data(), T.near_q, T.n_near * sizeof(int32_t));
    for (int64_t e = 0; e < T.n_near; ++e)
      for (int a = 0; a < D; ++a) near_q[e * D + a] = dmk::unpack_q(q[e], a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(plan, DMK_ERR_CUDA, cudaGetErrorString(e));
  return DMK_OK;
}

dmk_status_t dmk_stokes_kernel_table(int32_t dim, double eps, int32_t kernels, int32_t which, int32_t fp32,
                                     double* out_c, double* out_phi0, double* coef, int32_t max_terms,
                                     int32_t* n_terms) {
  if (dim != 2 && dim != 3) return set_err(nullptr, DMK_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (which < 0 || which > 6 || (dim == 2 && which >= 4 && which != 6) || (dim == 3 && which == 6))
    return set_err(nullptr, DMK_ERR_INVALID_ARG, "bad table id");
  double c = dmk::bandlimit_for_eps(eps, kernels);
  if (c <= 0) return set_err(nullptr, DMK_ERR_INVALID_ARG, "eps outside Table 2 range");
  static thread_local dmk::KernelTables tb;
  if (dmk::build_tables(dim, c, fp32_table_tol(eps), &tb) != 0)
    return set_err(nullptr, DMK_ERR_UNSUPPORTED, "table build failed");
  if (out_c) *out_c = tb.c;
  if (out_phi0) *out_phi0 = tb.phi0;
  if (which == 6) {
    if (n_terms) *n_terms = 1;
    if (coef && max_terms > 0) coef[0] = tb.self2d_m0;
    return DMK_OK;
  }
  int n = fp32 ? tb.n32[which] : tb.n64[which];
  if (n_terms) *n_terms = n;
  if (coef)
    for (int k = 0; k < std::min(n, max_terms); ++k) coef[k] = fp32 ? tb.p32[which][k] : tb.p64[which][k];
  return DMK_OK;
}

void dmk_stokes_destroy(dmk_stokes_plan_t plan) {
  if (!valid_plan(plan)) return;
  // frees go on the plan's stream; order them after work queued on the last
  // stream an evaluation used
  if (plan->last_stream != plan->p.stream) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(ev, plan->last_stream);
      cudaStreamWaitEvent(plan->p.stream, ev, 0);
      cudaEventDestroy(ev);
    }
  }
  plan->p.magic = 0;
  release(plan->p);
  delete plan;
}

const char* dmk_stokes_last_error(dmk_stokes_plan_t plan) {
  if (valid_plan(plan)) return plan->p.last_error.c_str();
  return g_last_error.c_str();
}

}  // extern "C"
