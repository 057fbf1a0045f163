// capi.cu — the C ABI of include/sym.h: handle life cycle, plan upload, executor calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "plan.h"
#include "reach.h"
#include "refine.h"
#include "sym.h"

struct sym_handle_s {
  sym::Plan plan;
  int precision = SYM_PREC_FP64;
  bool host_only = true;
  int device = -1;
  cudaStream_t stream = nullptr;
  sym::DevPlan dp;
  // device allocations owned by the handle
  void *d_sn = nullptr, *d_rows = nullptr, *d_rel = nullptr, *d_amap = nullptr, *d_updt = nullptr,
       *d_upde = nullptr, *d_tasks = nullptr, *d_perm = nullptr;
  double *d_Lx = nullptr;
  double *d_Linv = nullptr;  // inverses of the diagonal tiles (FP64 factor)
  float *d_Lfinv = nullptr;  // the same for an FP32 factor
  long long *d_status = nullptr;
  long long *h_status = nullptr;  // pinned: [0] holds the reset value, [1] receives the status
  double *d_y = nullptr;          // solve work array
  void *d_cptr = nullptr, *d_contrib = nullptr;  // contribution lists of the forward solve
  double *d_t = nullptr;          // forward-solve buffer (SOLVE_MAXRHS x tsize per matrix)
  int64_t y_cap = 0;
  double *d_stage = nullptr;      // staging for the host-pointer variants
  int64_t stage_cap = 0;
  int64_t device_bytes = 0;
  bool factored = false;
  bool pivots_valid = false;  // a factorization of a mixed-precision handle has been enqueued
  int64_t err_col = -1;
  // batches of matrices with this pattern: capacity (matrices whose factor fits), the size of
  // the last factored batch and its per-matrix failing columns
  int32_t bcap = 1;
  int32_t nbatch = 1;
  std::vector<int64_t> batch_err;
  int32_t fgraph_nb = 0;
  int64_t fgraph_stride = 0;
  int32_t sgraph_nb = 0;
  int64_t sgraph_bx[2] = {0, 0};
  // CUDA graphs of the launch sequences (replayed while their arguments stay the same)
  bool use_graphs = true;
  bool prepared = false;
  bool solve_prepared = false;
  cudaStream_t capture_stream = nullptr;
  sym::PrecondGraph pgraph;       // the FP32 preconditioner of the refined solve, as a graph
  cudaGraphExec_t fgraph = nullptr;
  const double *fgraph_ax = nullptr;
  cudaGraphExec_t sgraph = nullptr;
  const void *sgraph_key[3] = {nullptr, nullptr, nullptr};
  int64_t sgraph_ikey[3] = {0, 0, 0};
  // mixed precision: FP32 panels, a copy of A's values, CSR of P A P^T, refinement work
  float *d_Lf = nullptr;
  double *d_Axc = nullptr;
  double *d_anorm = nullptr;
  double *d_anorm_work = nullptr;
  void *d_csr_p = nullptr, *d_csr_i = nullptr, *d_csr_map = nullptr;
  double *d_rwork = nullptr;
  int64_t rwork_cap = 0;
  double *h_eta = nullptr;  // pinned, 256 doubles
  // FP64 pivots of the FP32 factor and their breakdown ratio min_k d_k / C_kk per matrix
  double *d_piv = nullptr;             // n per matrix
  void *d_dpos = nullptr;              // int64[n]: index in Ax of C_kk
  sym::PivotInfo *d_pivinfo = nullptr; // per matrix
  sym::PivotInfo *h_pivinfo = nullptr; // pinned copy, per matrix
  double pivot_threshold = 1.0 / 65536.0;
  double refine_tol = 1e-12;
  int32_t refine_max_iter = 100;
  int32_t last_iterations = 0;
  double last_berr = 0.0;
  // lookahead streams of the factor
  cudaStream_t aux_stream = nullptr;
  std::vector<cudaEvent_t> la_events;
  cudaEvent_t la_fork = nullptr, la_join = nullptr;
  sym::TwoStreams two;
  bool fused_levels = true;  // narrow levels as one launch per phase (SYM_FLAG_NO_FUSED_LEVELS)
  bool lookahead = true;  // run the factor schedule's auxiliary-stream launches concurrently
  // per-kernel profiling
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  double prof_ms[sym::NUM_KINDS] = {};
  std::vector<double> last_launch_ms[2];  // per launch of the last profiled factor / solve
  int64_t prof_launches[sym::NUM_KINDS] = {};
  double prof_flops[sym::NUM_KINDS] = {};
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SYM_ERR_OOM : SYM_ERR_CUDA;
}

#define CUDA_TRY(expr, what)                       \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

template <typename V>
int upload(const std::vector<V> &v, void **dst, int64_t &bytes) {
  size_t sz = v.size() * sizeof(V);
  if (sz == 0) sz = sizeof(V);
  CUDA_TRY(cudaMalloc(dst, sz), "cudaMalloc(plan)");
  bytes += (int64_t)sz;
  if (!v.empty()) CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice), "cudaMemcpy(plan)");
  return SYM_OK;
}

int ensure_events(sym_handle_s *h, size_t count) {
  while (h->events.size() < count) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e), "cudaEventCreate");
    h->events.push_back(e);
  }
  return SYM_OK;
}

// After the traced work has finished: add each launch's elapsed time to its kind.
int collect_trace(sym_handle_s *h, const sym::LaunchTrace &tr, double flop_scale, bool solve) {
  CUDA_TRY(cudaStreamSynchronize(h->stream), "profile sync");
  std::vector<double> &last = h->last_launch_ms[solve ? 1 : 0];
  last.clear();
  for (size_t i = 0; i < tr.kinds.size(); ++i) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, h->events[i], h->events[i + 1]), "cudaEventElapsedTime");
    h->prof_ms[tr.kinds[i]] += ms;
    h->prof_launches[tr.kinds[i]] += 1;
    last.push_back(ms);
  }
  for (int k = 0; k < sym::NUM_KINDS; ++k) {
    const bool is_solve = k >= sym::S_FGATHER;
    if (is_solve == solve) h->prof_flops[k] += h->plan.kind_flops[k] * flop_scale;
  }
  return SYM_OK;
}

void release_device(sym_handle_s *h) {
  for (cudaEvent_t e : h->la_events) cudaEventDestroy(e);
  if (h->la_fork) cudaEventDestroy(h->la_fork);
  if (h->la_join) cudaEventDestroy(h->la_join);
  if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
  {
    void *mp[] = {h->d_Linv, h->d_Lfinv, h->d_Lf, h->d_Axc, h->d_anorm, h->d_anorm_work, h->d_csr_p, h->d_csr_i,
                  h->d_csr_map, h->d_rwork, h->d_piv, h->d_dpos, h->d_pivinfo};
    for (void *p : mp)
      if (p) cudaFree(p);
    if (h->h_eta) cudaFreeHost(h->h_eta);
    if (h->h_pivinfo) cudaFreeHost(h->h_pivinfo);
  }
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  if (h->fgraph) cudaGraphExecDestroy(h->fgraph);
  if (h->sgraph) cudaGraphExecDestroy(h->sgraph);
  sym::precond_graph_reset(h->pgraph);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  void *ptrs[] = {h->d_sn, h->d_rows, h->d_rel, h->d_amap, h->d_updt, h->d_upde, h->d_tasks,
                  h->d_perm, h->d_Lx, h->d_status, h->d_y, h->d_stage, h->d_cptr, h->d_contrib, h->d_t};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (h->h_status) cudaFreeHost(h->h_status);
}

int ensure_rwork(sym_handle_s *h, int64_t count) {
  if (count <= h->rwork_cap) return SYM_OK;
  if (h->d_rwork) cudaFree(h->d_rwork);
  h->d_rwork = nullptr;
  h->rwork_cap = 0;
  CUDA_TRY(cudaMalloc(&h->d_rwork, sizeof(double) * (count > 0 ? count : 1)), "cudaMalloc(refinement work)");
  h->rwork_cap = count;
  return SYM_OK;
}

sym::RefineCtx refine_ctx(sym_handle_s *h, int32_t b = 0) {
  sym::RefineCtx r;
  r.dp = &h->dp;
  r.fwd = &h->plan.fwd_launches;
  r.bwd = &h->plan.bwd_launches;
  r.Lf = h->d_Lf + (int64_t)b * h->plan.storage();
  r.Lfinv = h->d_Lfinv + (int64_t)b * h->plan.dinv_storage;
  r.cp = (const int64_t *)h->d_csr_p;
  r.ci = (const int32_t *)h->d_csr_i;
  r.cmap = (const int64_t *)h->d_csr_map;
  r.Ax = h->d_Axc + (int64_t)b * h->plan.nnz_a;
  r.anorm = h->d_anorm + b;
  r.anorm_work = h->d_anorm_work;
  r.work = h->d_rwork;
  r.n = h->plan.n;
  return r;
}

// Everything one factorization enqueues after the status reset (the part a graph captures).
sym::Batch factor_batch(const sym_handle_s *h, int32_t nbatch, int64_t stride) {
  sym::Batch bt;
  bt.count = nbatch;
  bt.lx = h->plan.storage();
  bt.ax = stride;
  bt.dinv = h->plan.dinv_storage;
  bt.piv = h->plan.n;
  bt.nnz = h->plan.nnz_a;
  return bt;
}

cudaError_t enqueue_factor(sym_handle_s *h, const double *Ax, int32_t nbatch, int64_t stride, cudaStream_t st,
                           sym::LaunchTrace *tr) {
  const sym::Batch bt = factor_batch(h, nbatch, stride);
  if (h->precision == SYM_PREC_MIXED) {
    const int64_t nnz = h->plan.nnz_a;
    if (nnz > 0) {
      cudaError_t e = cudaMemcpy2DAsync(h->d_Axc, sizeof(double) * nnz, Ax, sizeof(double) * (nbatch > 1 ? stride : nnz),
                                        sizeof(double) * nnz, nbatch, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = sym::run_factor<float>(h->dp, h->plan.factor_launches, Ax, h->d_Lf, h->d_Lfinv, h->d_status,
                                           st, tr, bt, h->aux_stream ? &h->two : nullptr);
    if (e != cudaSuccess) return e;
    for (int32_t b = 0; b < nbatch; ++b) {
      e = sym::refine_anorm(refine_ctx(h, b), st);
      if (e != cudaSuccess) return e;
    }
    return sym::pivot_ratio(h->d_piv, h->plan.n, h->d_Axc, h->plan.nnz_a, (const int64_t *)h->d_dpos, nbatch,
                            h->d_pivinfo, st);
  }
  return sym::run_factor<double>(h->dp, h->plan.factor_launches, Ax, h->d_Lx, h->d_Linv, h->d_status, st, tr, bt,
                                 h->aux_stream ? &h->two : nullptr);
}

void drop_graphs(sym_handle_s *h) {
  if (h->fgraph) cudaGraphExecDestroy(h->fgraph);
  if (h->sgraph) cudaGraphExecDestroy(h->sgraph);
  h->fgraph = nullptr;
  h->sgraph = nullptr;
  sym::precond_graph_reset(h->pgraph);
}

// Room for the factors of nbatch matrices (panels, diagonal inverses, pivot status and, for the
// mixed precision, the copies of A's values and their norms). Growing drops the captured graphs
// (they hold the old addresses) and the current factor.
int ensure_batch(sym_handle_s *h, int32_t nbatch) {
  if (nbatch <= h->bcap) return SYM_OK;
  drop_graphs(h);
  h->factored = false;
  const auto &P = h->plan;
  auto regrow = [&](void **p, size_t bytes, const char *what) -> int {
    if (*p) cudaFree(*p);
    *p = nullptr;
    CUDA_TRY(cudaMalloc(p, bytes > 0 ? bytes : 8), what);
    return SYM_OK;
  };
  const size_t nb = (size_t)nbatch;
  int rc = SYM_OK;
  if (h->precision == SYM_PREC_FP64) {
    rc = regrow((void **)&h->d_Lx, sizeof(double) * P.storage() * nb, "cudaMalloc(L batch)");
    if (!rc) rc = regrow((void **)&h->d_Linv, sizeof(double) * P.dinv_storage * nb, "cudaMalloc(inverses batch)");
  } else {
    rc = regrow((void **)&h->d_Lf, sizeof(float) * P.storage() * nb, "cudaMalloc(L batch)");
    if (!rc) rc = regrow((void **)&h->d_Lfinv, sizeof(float) * P.dinv_storage * nb, "cudaMalloc(inverses batch)");
    if (!rc) rc = regrow((void **)&h->d_Axc, sizeof(double) * P.nnz_a * nb, "cudaMalloc(A copies)");
    h->dp.axc = h->d_Axc;
    if (!rc) rc = regrow((void **)&h->d_anorm, sizeof(double) * nb, "cudaMalloc(norms)");
    if (!rc) rc = regrow((void **)&h->d_piv, sizeof(double) * P.n * nb, "cudaMalloc(pivots)");
    if (!rc) rc = regrow((void **)&h->d_pivinfo, sizeof(sym::PivotInfo) * nb, "cudaMalloc(pivot ratios)");
    if (!rc) {
      if (h->h_pivinfo) cudaFreeHost(h->h_pivinfo);
      h->h_pivinfo = nullptr;
      cudaError_t e = cudaMallocHost(&h->h_pivinfo, sizeof(sym::PivotInfo) * nb);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocHost(pivot ratios)");
    }
    h->dp.piv = h->d_piv;
  }
  if (!rc) rc = regrow((void **)&h->d_status, sizeof(long long) * nb, "cudaMalloc(status batch)");
  if (!rc) rc = regrow((void **)&h->d_t, sizeof(double) * sym::SOLVE_MAXRHS * P.tsize * nb, "cudaMalloc(solve buffer batch)");
  h->dp.t = h->d_t;
  if (!rc) {
    if (h->h_status) cudaFreeHost(h->h_status);
    h->h_status = nullptr;
    cudaError_t e = cudaMallocHost(&h->h_status, 2 * sizeof(long long) * nb);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocHost(status batch)");
  }
  if (rc) {
    h->bcap = 0;  // partially reallocated: unusable until a successful ensure_batch
    return rc;
  }
  h->bcap = nbatch;
  return SYM_OK;
}

int ensure_capture_stream(sym_handle_s *h) {
  if (h->capture_stream) return SYM_OK;
  int lo = 0, hi = 0;
  CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
  CUDA_TRY(cudaStreamCreateWithPriority(&h->capture_stream, cudaStreamNonBlocking, hi), "cudaStreamCreate");
  return SYM_OK;
}

// The lookahead's auxiliary stream and one event per factor launch (created once).
int ensure_two_streams(sym_handle_s *h) {
  if (h->aux_stream) return SYM_OK;
  int lo = 0, hi = 0;
  CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
  CUDA_TRY(cudaStreamCreateWithPriority(&h->aux_stream, cudaStreamNonBlocking, lo), "cudaStreamCreate");
  const size_t nl = h->plan.factor_launches.size();
  h->la_events.resize(nl, nullptr);
  for (size_t i = 0; i < nl; ++i)
    CUDA_TRY(cudaEventCreateWithFlags(&h->la_events[i], cudaEventDisableTiming), "cudaEventCreate");
  CUDA_TRY(cudaEventCreateWithFlags(&h->la_fork, cudaEventDisableTiming), "cudaEventCreate");
  CUDA_TRY(cudaEventCreateWithFlags(&h->la_join, cudaEventDisableTiming), "cudaEventCreate");
  h->two.aux = h->aux_stream;
  h->two.events = &h->la_events;
  h->two.fork = h->la_fork;
  h->two.join = h->la_join;
  h->two.prio_high = hi;
  h->two.prio_low = lo;
  return SYM_OK;
}

int ensure_y(sym_handle_s *h, int64_t count) {
  if (count <= h->y_cap) return SYM_OK;
  if (h->d_y) cudaFree(h->d_y);
  h->d_y = nullptr;
  h->y_cap = 0;
  CUDA_TRY(cudaMalloc(&h->d_y, sizeof(double) * (count > 0 ? count : 1)), "cudaMalloc(solve work)");
  h->y_cap = count;
  return SYM_OK;
}

int ensure_stage(sym_handle_s *h, int64_t count) {
  if (count <= h->stage_cap) return SYM_OK;
  if (h->d_stage) cudaFree(h->d_stage);
  h->d_stage = nullptr;
  h->stage_cap = 0;
  CUDA_TRY(cudaMalloc(&h->d_stage, sizeof(double) * (count > 0 ? count : 1)), "cudaMalloc(staging)");
  h->stage_cap = count;
  return SYM_OK;
}

int check_device(sym_handle_s *h) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (h->host_only) return fail(SYM_ERR_STATE, "handle was analyzed with SYM_FLAG_HOST_ONLY");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != h->device) return fail(SYM_ERR_STATE, "the current device is not the handle's device");
  return SYM_OK;
}

int finish_status(sym_handle_s *h) {
  CUDA_TRY(cudaStreamSynchronize(h->stream), "factor");
  const int32_t nb = h->nbatch;
  h->batch_err.assign(nb, -1);
  h->err_col = -1;
  int32_t bad = 0;
  for (int32_t b = 0; b < nb; ++b)
    if (h->h_status[h->bcap + b] == -1) {
      h->factored = false;
      return fail(SYM_ERR_TIMEOUT, "a bounded device wait of the factorization ran out");
    }
  for (int32_t b = 0; b < nb; ++b) {
    const long long s = h->h_status[h->bcap + b];
    if (s != LLONG_MAX) {
      h->batch_err[b] = (s >= 0 && s < h->plan.n) ? h->plan.perm[s] : -1;
      if (bad++ == 0) h->err_col = h->batch_err[b];
    }
  }
  if (bad) {
    h->factored = false;
    return fail(SYM_ERR_NOT_SPD, "matrix is not positive definite (pivot at column " +
                                     std::to_string(h->err_col) + (nb > 1 ? " of the first failing matrix)" : ")"));
  }
  h->factored = true;
  return SYM_OK;
}

}  // namespace

extern "C" {

int sym_options_default(sym_options *opt) {
  if (!opt) return SYM_ERR_INVALID;
  std::memset(opt, 0, sizeof(*opt));
  opt->ordering = SYM_ORDER_GIVEN;
  opt->amalgamate = 1;
  opt->nrelax[0] = 4;
  opt->nrelax[1] = 16;
  opt->nrelax[2] = 48;
  opt->zrelax_permille[0] = 800;
  opt->zrelax_permille[1] = 100;
  opt->zrelax_permille[2] = 50;
  opt->flags = 0;
  return SYM_OK;
}

int sym_analyze(int64_t n, const int64_t *Ap, const int32_t *Ai, sym_handle *out) {
  return sym_analyze_perm(n, Ap, Ai, nullptr, nullptr, out);
}

static int analyze_impl(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm,
                        const sym_options *opt_in, sym_handle *out,
                        const std::vector<sym::AmalgamationRule> *rules, const std::vector<int32_t> *fund_rule);

int sym_analyze_perm(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm,
                     const sym_options *opt_in, sym_handle *out) {
  return analyze_impl(n, Ap, Ai, perm, opt_in, out, nullptr, nullptr);
}

int sym_analyze_rules(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm,
                      const sym_options *opt, int32_t nrules, const int32_t *rules, int64_t nfund,
                      const int32_t *fund_rule, sym_handle *out) {
  if (!out) return fail(SYM_ERR_INVALID, "null output handle");
  *out = nullptr;
  if (nrules < 1 || !rules || nfund < 0 || (nfund > 0 && !fund_rule))
    return fail(SYM_ERR_INVALID, "bad amalgamation rule table");
  std::vector<sym::AmalgamationRule> R(nrules);
  for (int32_t r = 0; r < nrules; ++r) {
    const int32_t *q = rules + 7 * r;
    R[r].amalgamate = q[0];
    for (int i = 0; i < 3; ++i) {
      R[r].nrelax[i] = q[1 + i];
      R[r].zrelax_permille[i] = q[4 + i];
      if (q[1 + i] < 0 || q[4 + i] < 0 || q[4 + i] > 1000) return fail(SYM_ERR_INVALID, "bad amalgamation rule");
    }
  }
  std::vector<int32_t> F(fund_rule, fund_rule + nfund);
  for (int32_t f : F)
    if (f < 0 || f >= nrules) return fail(SYM_ERR_INVALID, "rule index out of range");
  return analyze_impl(n, Ap, Ai, perm, opt, out, &R, &F);
}

static int analyze_impl(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm,
                        const sym_options *opt_in, sym_handle *out,
                        const std::vector<sym::AmalgamationRule> *rules, const std::vector<int32_t> *fund_rule) {
  if (!out) return fail(SYM_ERR_INVALID, "null output handle");
  *out = nullptr;
  sym_options opt;
  if (opt_in) opt = *opt_in;
  else sym_options_default(&opt);
  if (opt.ordering != SYM_ORDER_NATURAL && opt.ordering != SYM_ORDER_GIVEN && opt.ordering != SYM_ORDER_AUTO)
    return fail(SYM_ERR_INVALID, "unknown ordering");
  if (opt.precision != SYM_PREC_FP64 && opt.precision != SYM_PREC_MIXED)
    return fail(SYM_ERR_INVALID, "unknown precision");
  for (int i = 0; i < 3; ++i)
    if (opt.nrelax[i] < 0 || opt.zrelax_permille[i] < 0 || opt.zrelax_permille[i] > 1000)
      return fail(SYM_ERR_INVALID, "bad amalgamation parameters");
  sym_handle_s *h = new (std::nothrow) sym_handle_s();
  if (!h) return fail(SYM_ERR_OOM, "host allocation");
  try {
    std::string err;
    int rc = sym::analyze(n, Ap, Ai, perm, opt, h->plan, err, rules, fund_rule);
    if (rc != SYM_OK) {
      delete h;
      return fail(rc, err);
    }
    h->precision = opt.precision;
    if (h->precision == SYM_PREC_MIXED) sym::build_permuted_csr(Ap, Ai, h->plan);
  } catch (const std::bad_alloc &) {
    delete h;
    return fail(SYM_ERR_OOM, "host allocation during analysis");
  } catch (const std::exception &e) {
    delete h;
    return fail(SYM_ERR_INVALID, e.what());
  }
  h->host_only = (opt.flags & SYM_FLAG_HOST_ONLY) != 0;
  h->use_graphs = (opt.flags & SYM_FLAG_NO_GRAPHS) == 0;
  h->lookahead = (opt.flags & SYM_FLAG_ONE_STREAM) == 0;
  h->fused_levels = (opt.flags & SYM_FLAG_NO_FUSED_LEVELS) == 0;
  if (!h->host_only) {
    int rc = SYM_OK;
    auto &P = h->plan;
    int64_t bytes = 0;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGetDevice");
    if (!rc) rc = upload(P.snodes, &h->d_sn, bytes);
    if (!rc) rc = upload(P.rows, &h->d_rows, bytes);
    if (!rc) rc = upload(P.rel, &h->d_rel, bytes);
    if (!rc) rc = upload(P.amap, &h->d_amap, bytes);
    if (!rc) rc = upload(P.upd_tasks, &h->d_updt, bytes);
    if (!rc) rc = upload(P.upd_entries, &h->d_upde, bytes);
    if (!rc) rc = upload(P.tasks, &h->d_tasks, bytes);
    if (!rc) rc = upload(P.perm, &h->d_perm, bytes);
    if (!rc) rc = upload(P.contrib_ptr, &h->d_cptr, bytes);
    if (!rc) rc = upload(P.contrib, &h->d_contrib, bytes);
    if (!rc) {
      const int64_t tb = (int64_t)sizeof(double) * sym::SOLVE_MAXRHS * (P.tsize > 0 ? P.tsize : 1);
      e = cudaMalloc(&h->d_t, tb);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(solve buffer)");
      else bytes += tb;
    }
    if (!rc && h->precision == SYM_PREC_FP64) {
      e = cudaMalloc(&h->d_Lx, sizeof(double) * (P.storage() > 0 ? P.storage() : 1));
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(L)");
      else bytes += sizeof(double) * P.storage();
    }
    if (!rc && h->precision == SYM_PREC_FP64) {
      e = cudaMalloc(&h->d_Linv, sizeof(double) * (P.dinv_storage > 0 ? P.dinv_storage : 1));
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(diagonal inverses)");
      else bytes += sizeof(double) * P.dinv_storage;
    }
    if (!rc && h->precision == SYM_PREC_MIXED) {
      e = cudaMalloc(&h->d_Lfinv, sizeof(float) * (P.dinv_storage > 0 ? P.dinv_storage : 1));
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(diagonal inverses)");
      else bytes += sizeof(float) * P.dinv_storage;
    }
    if (!rc && h->precision == SYM_PREC_MIXED) {
      e = cudaMalloc(&h->d_Lf, sizeof(float) * (P.storage() > 0 ? P.storage() : 1));
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(L)");
      else bytes += sizeof(float) * P.storage();
      if (!rc) rc = upload(P.csr_p, &h->d_csr_p, bytes);
      if (!rc) rc = upload(P.csr_i, &h->d_csr_i, bytes);
      if (!rc) rc = upload(P.csr_map, &h->d_csr_map, bytes);
      if (!rc) {
        e = cudaMalloc(&h->d_Axc, sizeof(double) * (P.nnz_a > 0 ? P.nnz_a : 1));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(A copy)");
        else bytes += sizeof(double) * P.nnz_a;
      }
      if (!rc) {
        e = cudaMalloc(&h->d_anorm, sizeof(double));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(norm)");
      }
      if (!rc) {
        e = cudaMalloc(&h->d_anorm_work, sizeof(double) * (P.n + 512));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(norm work)");
      }
      if (!rc) {
        e = cudaMallocHost(&h->h_eta, 256 * sizeof(double));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocHost(refinement)");
      }
      if (!rc) rc = ensure_rwork(h, sym::refine_work_doubles(P.n, 1));
      if (!rc) {
        std::vector<int64_t> dpos(P.n);
        for (int64_t k = 0; k < P.n; ++k) dpos[k] = Ap[P.perm[k]];  // the diagonal leads each column
        rc = upload(dpos, &h->d_dpos, bytes);
      }
      if (!rc) {
        e = cudaMalloc(&h->d_piv, sizeof(double) * (P.n > 0 ? P.n : 1));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(pivots)");
        else bytes += sizeof(double) * P.n;
      }
      if (!rc) {
        e = cudaMalloc(&h->d_pivinfo, sizeof(sym::PivotInfo));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(pivot ratio)");
      }
      if (!rc) {
        e = cudaMallocHost(&h->h_pivinfo, sizeof(sym::PivotInfo));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocHost(pivot ratio)");
      }
    }
    if (!rc) {
      e = cudaMalloc(&h->d_status, sizeof(long long));
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(status)");
    }
    if (!rc) {
      e = cudaMallocHost(&h->h_status, 2 * sizeof(long long));  // [reset value, result] for one matrix
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocHost(status)");
    }
    if (rc) {
      release_device(h);
      delete h;
      return rc;
    }
    h->device_bytes = bytes;
    h->dp.sn = (const sym::SNode *)h->d_sn;
    h->dp.rows = (const int32_t *)h->d_rows;
    h->dp.rel = (const int32_t *)h->d_rel;
    h->dp.amap = (const int64_t *)h->d_amap;
    h->dp.upd_tasks = (const sym::UpdTask *)h->d_updt;
    h->dp.upd_entries = (const sym::UpdEntry *)h->d_upde;
    h->dp.tasks = (const sym::Int4 *)h->d_tasks;
    h->dp.perm = (const int32_t *)h->d_perm;
    h->dp.cptr = (const int64_t *)h->d_cptr;
    h->dp.contrib = (const int32_t *)h->d_contrib;
    h->dp.t = h->d_t;
    h->dp.tsize = P.tsize;
    h->dp.n = P.n;
    h->dp.nnz_a = P.nnz_a;
    h->dp.storage = P.storage();
    h->dp.tensor_cores = (opt.flags & SYM_FLAG_NO_TENSOR_CORES) == 0;
    h->dp.piv = h->d_piv;
    for (int c = 0; c < 2; ++c) h->dp.variant[c] = h->plan.variant[c].data();
    h->dp.batch_warp = h->plan.batch_warp.data();
    h->dp.batch_lanes = h->plan.batch_lanes.data();
    h->dp.batch_panel = (opt.flags & SYM_FLAG_NO_FUSED_LEVELS) ? nullptr : h->plan.batch_panel.data();
    for (int c = 0; c < 2; ++c) h->dp.panel_apart[c] = h->plan.panel_apart[c].data();
    if (!(opt.flags & SYM_FLAG_NO_FUSED_LEVELS)) {
      h->dp.fwd_panel = h->plan.fwd_panel.data();
      h->dp.bwd_panel = h->plan.bwd_panel.data();
      h->dp.nfwd_panel = (int64_t)h->plan.fwd_panel.size();
      h->dp.nbwd_panel = (int64_t)h->plan.bwd_panel.size();
    }
    h->dp.axc = h->d_Axc;
    h->dp.dpos = (const int64_t *)h->d_dpos;
  }
  *out = h;
  return SYM_OK;
}

int sym_set_stream(sym_handle h, void *stream) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  h->stream = (cudaStream_t)stream;
  return SYM_OK;
}

}  // extern "C"

namespace {

int factor_impl(sym_handle h, int32_t nbatch, const double *Ax, int64_t stride) {
  int rc = check_device(h);
  if (rc) return rc;
  if (!Ax && h->plan.nnz_a > 0) return fail(SYM_ERR_INVALID, "null Ax");
  if (nbatch < 1 || (nbatch > 1 && stride < h->plan.nnz_a)) return fail(SYM_ERR_INVALID, "bad batch arguments");
  if (nbatch > 65535) return fail(SYM_ERR_LIMIT, "more than 65535 matrices in one batch");
  rc = ensure_batch(h, nbatch);
  if (rc) return rc;
  h->factored = false;
  h->nbatch = nbatch;
  for (int32_t b = 0; b < nbatch; ++b) h->h_status[b] = LLONG_MAX;
  CUDA_TRY(cudaMemcpyAsync(h->d_status, h->h_status, sizeof(long long) * nbatch, cudaMemcpyHostToDevice, h->stream),
           "status reset");
  if (!h->prepared) {
    CUDA_TRY(h->precision == SYM_PREC_MIXED ? sym::prepare_factor<float>() : sym::prepare_factor<double>(),
             "factor set-up");
    if (h->lookahead) {
      rc = ensure_two_streams(h);
      if (rc) return rc;
    }
    h->prepared = true;
  }
  sym::LaunchTrace tr, *trp = nullptr;
  if (h->profiling) {
    rc = ensure_events(h, h->plan.factor_launches.size() + 3);
    if (rc) return rc;
    tr.events = &h->events;
    trp = &tr;
  }
  if (!trp && h->use_graphs) {
    // Replay the captured launch sequence; capture it again when Ax or the batch moved.
    if (!h->fgraph || h->fgraph_ax != Ax || h->fgraph_nb != nbatch || h->fgraph_stride != stride) {
      rc = ensure_capture_stream(h);
      if (rc) return rc;
      if (h->fgraph) cudaGraphExecDestroy(h->fgraph);
      h->fgraph = nullptr;
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal), "capture factor");
      cudaError_t e = enqueue_factor(h, Ax, nbatch, stride, h->capture_stream, nullptr);
      cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(e != cudaSuccess ? e : e2, "capture factor");
      }
      e = cudaGraphInstantiate(&h->fgraph, g, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "instantiate factor graph");
      h->fgraph_ax = Ax;
      h->fgraph_nb = nbatch;
      h->fgraph_stride = stride;
    }
    CUDA_TRY(cudaGraphLaunch(h->fgraph, h->stream), "factor graph");
  } else {
    CUDA_TRY(enqueue_factor(h, Ax, nbatch, stride, h->stream, trp), "factor kernels");
  }
  if (trp) {
    rc = collect_trace(h, tr, (double)nbatch, false);
    if (rc) return rc;
  }
  CUDA_TRY(cudaMemcpyAsync(h->h_status + h->bcap, h->d_status, sizeof(long long) * nbatch, cudaMemcpyDeviceToHost,
                           h->stream),
           "status read");
  if (h->precision == SYM_PREC_MIXED && h->plan.n > 0)
    CUDA_TRY(cudaMemcpyAsync(h->h_pivinfo, h->d_pivinfo, sizeof(sym::PivotInfo) * nbatch, cudaMemcpyDeviceToHost,
                             h->stream),
             "pivot ratio read");
  h->pivots_valid = h->precision == SYM_PREC_MIXED;
  return SYM_OK;
}

int solve_impl(sym_handle h, int32_t nbatch, int32_t nrhs, const double *B, int64_t ldb, int64_t bstride,
               double *X, int64_t ldx, int64_t xstride) {
  int rc = check_device(h);
  if (rc) return rc;
  if (!h->factored) return fail(SYM_ERR_STATE, "no successful factorization to solve with");
  const int64_t n = h->plan.n;
  if (nrhs < 0 || ldb < n || ldx < n || (nrhs > 0 && n > 0 && (!B || !X)))
    return fail(SYM_ERR_INVALID, "bad solve arguments");
  if (nbatch < 1 || nbatch > h->nbatch) return fail(SYM_ERR_INVALID, "batch larger than the factored batch");
  if (nbatch > 1 && (bstride < ldb * (int64_t)nrhs || xstride < ldx * (int64_t)nrhs))
    return fail(SYM_ERR_INVALID, "bad batch strides");
  if (!h->solve_prepared) {
    CUDA_TRY((h->precision == SYM_PREC_MIXED ? sym::prepare_solve<float, float>()
                                             : sym::prepare_solve<double, double>()),
             "solve set-up");
    h->solve_prepared = true;
  }
  if (h->precision == SYM_PREC_MIXED) {
    // FP64 conjugate gradients preconditioned with the FP32 factor, per matrix, up to 64
    // right-hand sides at a time.
    int32_t iters = 0;
    double berr = 0.0;
    bool conv = true;
    for (int32_t b = 0; b < nbatch; ++b)
      for (int32_t c0 = 0; c0 < nrhs; c0 += 64) {
        const int32_t nc = nrhs - c0 < 64 ? nrhs - c0 : 64;
        rc = ensure_rwork(h, sym::refine_work_doubles(n, nc));
        if (rc) return rc;
        sym::RefineResult res;
        sym::RefineCtx ctx = refine_ctx(h, b);
        if (nbatch == 1 && h->use_graphs) {  // (a batch's matrices would each need their own graph)
          rc = ensure_capture_stream(h);
          if (rc) return rc;
          ctx.pgraph = &h->pgraph;
          ctx.capture = h->capture_stream;
        }
        if (sym::refine_solve(ctx, nc, B + b * bstride + (int64_t)c0 * ldb, ldb,
                              X + b * xstride + (int64_t)c0 * ldx, ldx, h->refine_tol, h->refine_max_iter, h->h_eta,
                              &res, h->stream) != 0)
          return cuda_fail(cudaGetLastError(), "refinement");
        iters = res.iterations > iters ? res.iterations : iters;
        berr = res.backward_error > berr ? res.backward_error : berr;
        conv = conv && res.converged;
      }
    h->last_iterations = iters;
    h->last_berr = berr;
    if (!conv) return fail(SYM_ERR_NO_CONVERGENCE, "refinement reached its iteration limit above tolerance");
    return SYM_OK;
  }
  rc = ensure_y(h, n * (int64_t)nrhs * nbatch);
  if (rc) return rc;
  sym::Batch bt;
  bt.count = nbatch;
  bt.lx = h->plan.storage();
  bt.dinv = h->plan.dinv_storage;
  bt.y = n * (int64_t)nrhs;
  bt.b = bstride;
  bt.x = xstride;
  bt.t = (int64_t)sym::SOLVE_MAXRHS * h->plan.tsize;
  sym::LaunchTrace tr, *trp = nullptr;
  if (h->profiling) {
    const size_t passes = (size_t)(nrhs + 7) / 8;
    rc = ensure_events(h, passes * (h->plan.fwd_launches.size() + h->plan.bwd_launches.size()) + 4);
    if (rc) return rc;
    tr.events = &h->events;
    trp = &tr;
  }
  if (!trp && h->use_graphs && n > 0 && nrhs > 0) {
    const bool same = h->sgraph && h->sgraph_key[0] == B && h->sgraph_key[1] == X &&
                      h->sgraph_key[2] == h->d_y && h->sgraph_ikey[0] == nrhs && h->sgraph_ikey[1] == ldb &&
                      h->sgraph_ikey[2] == ldx && h->sgraph_nb == nbatch && h->sgraph_bx[0] == bstride &&
                      h->sgraph_bx[1] == xstride;
    if (!same) {
      rc = ensure_capture_stream(h);
      if (rc) return rc;
      if (h->sgraph) cudaGraphExecDestroy(h->sgraph);
      h->sgraph = nullptr;
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal), "capture solve");
      cudaError_t e = sym::run_solve<double>(h->dp, h->plan.fwd_launches, h->plan.bwd_launches, h->d_Lx, h->d_Linv,
                                             nrhs, B, ldb, X, ldx, h->d_y, h->capture_stream, nullptr, bt);
      cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(e != cudaSuccess ? e : e2, "capture solve");
      }
      e = cudaGraphInstantiate(&h->sgraph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "instantiate solve graph");
      h->sgraph_key[0] = B;
      h->sgraph_key[1] = X;
      h->sgraph_key[2] = h->d_y;
      h->sgraph_ikey[0] = nrhs;
      h->sgraph_ikey[1] = ldb;
      h->sgraph_ikey[2] = ldx;
      h->sgraph_nb = nbatch;
      h->sgraph_bx[0] = bstride;
      h->sgraph_bx[1] = xstride;
    }
    CUDA_TRY(cudaGraphLaunch(h->sgraph, h->stream), "solve graph");
    return SYM_OK;
  }
  CUDA_TRY(sym::run_solve<double>(h->dp, h->plan.fwd_launches, h->plan.bwd_launches, h->d_Lx, h->d_Linv, nrhs, B,
                                  ldb, X, ldx, h->d_y, h->stream, trp, bt),
           "solve kernels");
  if (trp) return collect_trace(h, tr, (double)nrhs * nbatch, true);
  return SYM_OK;
}

}  // namespace

extern "C" {

int sym_factor_async(sym_handle h, const double *Ax) { return factor_impl(h, 1, Ax, 0); }

int sym_factor_batch(sym_handle h, int32_t nbatch, const double *Ax, int64_t stride) {
  int rc = factor_impl(h, nbatch, Ax, stride);
  if (rc) return rc;
  return finish_status(h);
}

int sym_batch_error_columns(sym_handle h, int64_t *cols) {
  if (!h || !cols) return fail(SYM_ERR_INVALID, "null argument");
  for (size_t b = 0; b < h->batch_err.size(); ++b) cols[b] = h->batch_err[b];
  return SYM_OK;
}

int sym_solve_batch(sym_handle h, int32_t nbatch, int32_t nrhs, const double *B, int64_t ldb, int64_t bstride,
                    double *X, int64_t ldx, int64_t xstride) {
  return solve_impl(h, nbatch, nrhs, B, ldb, bstride, X, ldx, xstride);
}

int sym_status(sym_handle h) {
  int rc = check_device(h);
  if (rc) return rc;
  return finish_status(h);
}

int sym_factor(sym_handle h, const double *Ax) {
  int rc = sym_factor_async(h, Ax);
  if (rc) return rc;
  return finish_status(h);
}

int sym_factor_host(sym_handle h, const double *Ax) {
  int rc = check_device(h);
  if (rc) return rc;
  if (!Ax && h->plan.nnz_a > 0) return fail(SYM_ERR_INVALID, "null Ax");
  rc = ensure_stage(h, h->plan.nnz_a);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(h->d_stage, Ax, sizeof(double) * h->plan.nnz_a, cudaMemcpyHostToDevice, h->stream),
           "copy Ax");
  return sym_factor(h, h->d_stage);
}

int sym_solve_multi(sym_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx) {
  return solve_impl(h, 1, nrhs, B, ldb, 0, X, ldx, 0);
}

}  // extern "C"

namespace sym {
// What a solve with a caller-supplied work array needs of the handle: a device handle whose
// device is current, a successful factorization, and an FP64 factor.
int check_solve_ready(sym_handle h) {
  int rc = check_device(h);
  if (rc) return rc;
  if (!h->factored) return fail(SYM_ERR_STATE, "no successful factorization to solve with");
  if (h->precision != SYM_PREC_FP64) return fail(SYM_ERR_STATE, "this entry point needs an FP64 factor");
  return SYM_OK;
}

// Solve with a work array supplied by the caller (at least n * nrhs doubles); performs no
// allocation and records no profile events.
int solve_with_work(sym_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                    double *work) {
  int rc = check_solve_ready(h);
  if (rc) return rc;
  if (!h->solve_prepared) {
    CUDA_TRY((sym::prepare_solve<double, double>()), "solve set-up");
    h->solve_prepared = true;
  }
  const int64_t n = h->plan.n;
  if (nrhs < 0 || ldb < n || ldx < n || (nrhs > 0 && n > 0 && (!B || !X)))
    return fail(SYM_ERR_INVALID, "bad solve arguments");
  CUDA_TRY(sym::run_solve<double>(h->dp, h->plan.fwd_launches, h->plan.bwd_launches, h->d_Lx, h->d_Linv, nrhs, B, ldb,
                                  X, ldx, work, h->stream),
           "solve kernels");
  return SYM_OK;
}
int set_error(int code, const char *msg) { return fail(code, msg); }
int64_t plan_n(sym_handle h) { return h ? h->plan.n : 0; }
}  // namespace sym

extern "C" {

int sym_solve(sym_handle h, const double *b, double *x) {
  return sym_solve_multi(h, 1, b, h ? h->plan.n : 0, x, h ? h->plan.n : 0);
}

int sym_solve_host(sym_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx) {
  int rc = check_device(h);
  if (rc) return rc;
  const int64_t n = h->plan.n;
  if (nrhs < 0 || ldb < n || ldx < n) return fail(SYM_ERR_INVALID, "bad solve arguments");
  rc = ensure_stage(h, 2 * n * (int64_t)nrhs);
  if (rc) return rc;
  double *dB = h->d_stage, *dX = h->d_stage + n * (int64_t)nrhs;
  CUDA_TRY(cudaMemcpy2DAsync(dB, sizeof(double) * n, B, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                             cudaMemcpyHostToDevice, h->stream),
           "copy B");
  rc = sym_solve_multi(h, nrhs, dB, n, dX, n);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpy2DAsync(X, sizeof(double) * ldx, dX, sizeof(double) * n, sizeof(double) * n, nrhs,
                             cudaMemcpyDeviceToHost, h->stream),
           "copy X");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "solve");
  return SYM_OK;
}

int sym_info(sym_handle h, sym_stats *s) {
  if (!h || !s) return fail(SYM_ERR_INVALID, "null argument");
  const auto &P = h->plan;
  std::memset(s, 0, sizeof(*s));
  s->n = P.n;
  s->nnz_a = P.nnz_a;
  s->nnz_l = P.nnz_l;
  s->storage_l = P.storage();
  s->flops = P.flops;
  s->solve_flops = 2.0 * (2.0 * (double)P.nnz_l - (double)P.n);
  s->nsuper_fund = (int32_t)P.fsuper.size() - 1;
  s->nsuper = P.nsuper();
  s->nlevels = (int32_t)P.levelptr.size() - 1;
  s->max_ncols = P.max_ncols;
  s->npairs = (int64_t)P.desc.size();
  // kernels one matrix launches: the schedule's launches (+ zeroing and scatter, + the two
  // permutations) minus those of fused narrow levels that a factor, or a solve with one
  // right-hand side, skips by default
  s->nlaunch_factor = (int64_t)P.factor_launches.size() + 2;
  s->nlaunch_solve = (int64_t)P.fwd_launches.size() + (int64_t)P.bwd_launches.size() + 2;
  if (h->fused_levels) {
    const bool f32 = h->precision != SYM_PREC_FP64;
    for (const sym::PanelForm &pf : P.batch_panel)
      if (pf.role == sym::PANEL_COVERED && !P.panel_apart[0][pf.head] &&
          sym::panel_lanes_for(P.batch_panel[pf.head], 1, f32) > 0)
        --s->nlaunch_factor;
    for (const auto *forms : {&P.fwd_panel, &P.bwd_panel})
      for (const sym::PanelForm &pf : *forms)
        if (pf.role == sym::PANEL_COVERED && sym::solve_lanes_for((*forms)[pf.head], 1, !f32) > 0) --s->nlaunch_solve;
  }
  s->analyze_seconds = P.analyze_seconds;
  s->device_bytes = h->device_bytes;
  s->upd_tasks = (int64_t)P.upd_tasks.size();
  s->upd_entries = (int64_t)P.upd_entries.size();
  int64_t dense = 0;
  for (const auto &L : P.factor_launches)
    if (L.kind != sym::K_UPDATE) dense += L.count;
  s->dense_tasks = dense;
  s->exec_flops = 0.0;
  for (int k = sym::K_SCATTER; k <= sym::K_TRTRI; ++k) s->exec_flops += P.kind_flops[k];
  s->update_flops = P.update_flops;
  s->ordering_method = P.ordering_method;
  s->ordering_flops_md = P.ordering_flops[0];
  s->ordering_flops_nd = P.ordering_flops[1];
  return SYM_OK;
}

int sym_last_error_column(sym_handle h, int64_t *col) {
  if (!h || !col) return fail(SYM_ERR_INVALID, "null argument");
  *col = h->err_col;
  return SYM_OK;
}

int sym_get_batch_factor_host(sym_handle h, int32_t index, double *Lx_host) {
  int rc = check_device(h);
  if (rc) return rc;
  if (!Lx_host || index < 0 || index >= h->bcap) return fail(SYM_ERR_INVALID, "bad argument");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "sync");
  const int64_t st = h->plan.storage();
  if (h->precision == SYM_PREC_MIXED) {
    std::vector<float> tmp(st);
    CUDA_TRY(cudaMemcpy(tmp.data(), h->d_Lf + index * st, sizeof(float) * st, cudaMemcpyDeviceToHost), "copy L");
    for (int64_t i = 0; i < st; ++i) Lx_host[i] = tmp[i];
    return SYM_OK;
  }
  CUDA_TRY(cudaMemcpy(Lx_host, h->d_Lx + index * st, sizeof(double) * st, cudaMemcpyDeviceToHost), "copy L");
  return SYM_OK;
}

int sym_get_factor_host(sym_handle h, double *Lx_host) {
  int rc = check_device(h);
  if (rc) return rc;
  if (!Lx_host) return fail(SYM_ERR_INVALID, "null output");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "sync");
  if (h->precision == SYM_PREC_MIXED) {
    std::vector<float> tmp(h->plan.storage());
    CUDA_TRY(cudaMemcpy(tmp.data(), h->d_Lf, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost), "copy L");
    for (size_t i = 0; i < tmp.size(); ++i) Lx_host[i] = tmp[i];
    return SYM_OK;
  }
  CUDA_TRY(cudaMemcpy(Lx_host, h->d_Lx, sizeof(double) * h->plan.storage(), cudaMemcpyDeviceToHost), "copy L");
  return SYM_OK;
}

int64_t sym_export(sym_handle h, int32_t what, void *out) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  const auto &P = h->plan;
  const void *src = nullptr;
  int64_t count = 0;
  size_t esz = 0;
  switch (what) {
#define EXP(id, vec)          \
  case id:                    \
    src = P.vec.data();       \
    count = (int64_t)P.vec.size(); \
    esz = sizeof(P.vec[0]);   \
    break;
    EXP(SYM_EXPORT_PERM, perm)
    EXP(SYM_EXPORT_PARENT, parent)
    EXP(SYM_EXPORT_COLCOUNT, colcount)
    EXP(SYM_EXPORT_FSUPER, fsuper)
    EXP(SYM_EXPORT_SUPER, super)
    EXP(SYM_EXPORT_ROWPTR, rowptr)
    EXP(SYM_EXPORT_ROWS, rows)
    EXP(SYM_EXPORT_SPARENT, sparent)
    EXP(SYM_EXPORT_DESCPTR, descptr)
    EXP(SYM_EXPORT_DESC, desc)
    EXP(SYM_EXPORT_DESCR0, descr0)
    EXP(SYM_EXPORT_DESCNIN, descnin)
    EXP(SYM_EXPORT_RELPTR, relptr)
    EXP(SYM_EXPORT_REL, rel)
    EXP(SYM_EXPORT_LEVEL, level)
    EXP(SYM_EXPORT_LEVELPTR, levelptr)
    EXP(SYM_EXPORT_LEVELLIST, levellist)
    EXP(SYM_EXPORT_LXPTR, lxptr)
    EXP(SYM_EXPORT_CONTRIB_PTR, contrib_ptr)
    EXP(SYM_EXPORT_CONTRIB, contrib)
#undef EXP
#define EXPB(id, vec, words)                                                     \
  case id:                                                                       \
    src = P.vec.data();                                                          \
    count = (int64_t)P.vec.size() * (int64_t)(sizeof(P.vec[0]) / (words));       \
    esz = (words);                                                               \
    break;
    EXPB(SYM_EXPORT_FACTOR_LAUNCHES, factor_launches, 8)
    EXPB(SYM_EXPORT_FWD_LAUNCHES, fwd_launches, 8)
    EXPB(SYM_EXPORT_BWD_LAUNCHES, bwd_launches, 8)
    static_assert(sizeof(sym::Launch) == 40, "launch record layout");
    EXPB(SYM_EXPORT_TASKS, tasks, 4)
    EXPB(SYM_EXPORT_UPD_TASKS, upd_tasks, 8)
    EXPB(SYM_EXPORT_UPD_ENTRIES, upd_entries, 8)
    EXPB(SYM_EXPORT_BATCH_PANEL, batch_panel, 4)
    EXPB(SYM_EXPORT_FWD_PANEL, fwd_panel, 4)
    EXPB(SYM_EXPORT_BWD_PANEL, bwd_panel, 4)
    static_assert(sizeof(sym::PanelForm) == 16, "panel form record layout");
#undef EXPB
    default:
      return fail(SYM_ERR_INVALID, "unknown export item");
  }
  if (out && count > 0) std::memcpy(out, src, (size_t)count * esz);
  return count;
}

int sym_set_refinement(sym_handle h, double tol, int32_t max_iter) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (!(tol > 0.0) || max_iter < 1) return fail(SYM_ERR_INVALID, "bad refinement parameters");
  h->refine_tol = tol;
  h->refine_max_iter = max_iter;
  return SYM_OK;
}

int sym_refinement_info(sym_handle h, int32_t *iterations, double *backward_error) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (iterations) *iterations = h->last_iterations;
  if (backward_error) *backward_error = h->last_berr;
  return SYM_OK;
}

int sym_pivot_info(sym_handle h, int32_t index, double *min_ratio, int64_t *column, int32_t *breakdown) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (h->precision != SYM_PREC_MIXED) return fail(SYM_ERR_STATE, "pivot ratios belong to mixed-precision handles");
  if (!h->pivots_valid) return fail(SYM_ERR_STATE, "no factorization yet");
  if (index < 0 || index >= h->nbatch) return fail(SYM_ERR_INVALID, "matrix index out of range");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "pivot ratio");
  const sym::PivotInfo &pi = h->h_pivinfo[index];
  const bool any = h->plan.n > 0 && pi.column >= 0;
  if (min_ratio) *min_ratio = any ? pi.min_ratio : 1.0;
  if (column) *column = any ? h->plan.perm[pi.column] : -1;
  if (breakdown) *breakdown = any && pi.min_ratio < h->pivot_threshold ? 1 : 0;
  return SYM_OK;
}

int sym_autotune(sym_handle h, int32_t nbatch, const double *Ax, int64_t stride, int32_t reps, int32_t *tuned,
                 int32_t *changed) {
  int rc = check_device(h);
  if (rc) return rc;
  if (reps < 1 || reps > 100) return fail(SYM_ERR_INVALID, "reps outside 1..100");
  if (nbatch < 1) return fail(SYM_ERR_INVALID, "nbatch must be at least 1");
  auto &P = h->plan;
  const size_t nl = P.factor_launches.size();
  std::vector<int8_t> &var = P.variant[nbatch > 1 ? 1 : 0];  // one matrix and batches are tuned apart
  // fused narrow levels: one fused launch against the level's separate launches (a batch's only
  // where its panels fit the fused kernel)
  std::vector<int8_t> &apart = P.panel_apart[nbatch > 1 ? 1 : 0];
  const bool f32 = h->precision != SYM_PREC_FP64;
  std::vector<size_t> heads;
  if (h->dp.batch_panel)
    for (size_t li = 0; li < nl; ++li)
      if (P.batch_panel[li].role == sym::PANEL_FUSED && sym::panel_lanes_for(P.batch_panel[li], (unsigned)nbatch, f32) > 0)
        heads.push_back(li);
  if (tuned) *tuned = 0;
  if (changed) *changed = 0;
  // time every launch in the forms given by set(v) (kernel by kernel, CUDA events, reps
  // factorizations each), keeping the user's profile
  const bool prof0 = h->profiling;
  double ms0[sym::NUM_KINDS], fl0[sym::NUM_KINDS];
  int64_t nl0[sym::NUM_KINDS];
  std::memcpy(ms0, h->prof_ms, sizeof ms0);
  std::memcpy(fl0, h->prof_flops, sizeof fl0);
  std::memcpy(nl0, h->prof_launches, sizeof nl0);
  auto time_forms = [&](const std::function<void(int)> &set, std::vector<double> (&t)[2]) {
    for (int v = 0; v < 2 && !rc; ++v) {
      t[v].assign(nl, 0.0);
      set(v);
      drop_graphs(h);
      h->profiling = true;
      for (int32_t r = 0; r < reps && !rc; ++r) {
        rc = factor_impl(h, nbatch, Ax, stride);
        if (!rc) rc = finish_status(h);
        if (!rc && h->last_launch_ms[0].size() == nl + 1)
          for (size_t li = 0; li < nl; ++li) t[v][li] += h->last_launch_ms[0][li + 1];
      }
    }
  };
  int32_t ntun = 0, nchg = 0;
  std::vector<double> t[2];
  if (!heads.empty()) {
    std::fill(var.begin(), var.end(), 0);
    time_forms([&](int v) { for (size_t hd : heads) apart[hd] = (int8_t)v; }, t);
    for (size_t hd : heads) {  // the level's launches in either form (covered ones take ~0 fused)
      double sum[2] = {0.0, 0.0};
      for (size_t li = 0; li < nl; ++li)
        if (P.batch_panel[li].role != sym::PANEL_NONE && P.batch_panel[li].head == (int32_t)hd)
          for (int v = 0; v < 2; ++v) sum[v] += t[v][li];
      apart[hd] = !rc && sum[1] < sum[0] ? 1 : 0;
      ++ntun;
      nchg += apart[hd];
    }
  }
  std::vector<char> tunable(nl, 0);
  int32_t nform = 0;
  for (size_t li = 0; li < nl; ++li) {
    // launches of a level that stays fused have one form
    const sym::PanelForm *pf = h->dp.batch_panel ? &P.batch_panel[li] : nullptr;
    const bool fused = pf && pf->role != sym::PANEL_NONE && !apart[pf->head] &&
                       std::find(heads.begin(), heads.end(), (size_t)pf->head) != heads.end();
    nform += tunable[li] = !fused && sym::factor_launch_has_alternative(P.factor_launches[li], nbatch,
                                                                        h->precision == SYM_PREC_FP64);
  }
  if (nform > 0 && !rc) {
    time_forms([&](int v) { for (size_t li = 0; li < nl; ++li) var[li] = tunable[li] ? (int8_t)v : 0; }, t);
    for (size_t li = 0; li < nl; ++li) {
      var[li] = tunable[li] && !rc && t[1][li] < t[0][li] ? 1 : 0;
      nchg += var[li];
    }
  }
  ntun += nform;
  h->profiling = prof0;
  std::memcpy(h->prof_ms, ms0, sizeof ms0);
  std::memcpy(h->prof_flops, fl0, sizeof fl0);
  std::memcpy(h->prof_launches, nl0, sizeof nl0);
  drop_graphs(h);
  if (tuned) *tuned = ntun;
  if (changed) *changed = nchg;
  return rc;
}

int sym_set_tc_wait(sym_handle h, uint64_t limit_ns, int32_t withhold_mma) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (limit_ns < 1000 || limit_ns > 10000000000ull) return fail(SYM_ERR_INVALID, "wait limit outside [1 us, 10 s]");
  if (withhold_mma != 0 && withhold_mma != 1) return fail(SYM_ERR_INVALID, "withhold_mma must be 0 or 1");
  if (h->dp.tc_wait_ns != limit_ns || h->dp.tc_withhold != withhold_mma) drop_graphs(h);  // baked-in arguments
  h->dp.tc_wait_ns = limit_ns;
  h->dp.tc_withhold = withhold_mma;
  return SYM_OK;
}

int sym_set_pivot_threshold(sym_handle h, double threshold) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (!(threshold >= 0.0 && threshold <= 1.0)) return fail(SYM_ERR_INVALID, "threshold outside [0, 1]");
  h->pivot_threshold = threshold;
  return SYM_OK;
}

int sym_profile(sym_handle h, int32_t mode) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (mode == SYM_PROFILE_ON) h->profiling = true;
  else if (mode == SYM_PROFILE_OFF) h->profiling = false;
  else if (mode == SYM_PROFILE_RESET) {
    for (int k = 0; k < sym::NUM_KINDS; ++k) {
      h->prof_ms[k] = 0.0;
      h->prof_launches[k] = 0;
      h->prof_flops[k] = 0.0;
    }
  } else {
    return fail(SYM_ERR_INVALID, "unknown profile mode");
  }
  return SYM_OK;
}

int64_t sym_profile_launches(sym_handle h, int32_t which, double *ms) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (which != 0 && which != 1) return fail(SYM_ERR_INVALID, "which must be 0 (factor) or 1 (solve)");
  const std::vector<double> &v = h->last_launch_ms[which];
  if (ms && !v.empty()) std::memcpy(ms, v.data(), v.size() * sizeof(double));
  return (int64_t)v.size();
}

int sym_profile_read(sym_handle h, int32_t kind, double *ms, int64_t *launches, double *flops) {
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  if (kind < 0 || kind >= sym::NUM_KINDS) return fail(SYM_ERR_INVALID, "unknown kernel kind");
  if (ms) *ms = h->prof_ms[kind];
  if (launches) *launches = h->prof_launches[kind];
  if (flops) *flops = h->prof_flops[kind];
  return SYM_OK;
}

}  // extern "C"

struct sym_reach_s {
  sym_handle h = nullptr;
  sym::Reach r;
  sym::DevPlan dp;
  void *d_pbeta = nullptr, *d_cols = nullptr, *d_snodes = nullptr, *d_ut = nullptr, *d_ue = nullptr,
       *d_tasks = nullptr;
};

namespace {
void reach_release(sym_reach_s *r) {
  void *p[] = {r->d_pbeta, r->d_cols, r->d_snodes, r->d_ut, r->d_ue, r->d_tasks};
  for (void *q : p)
    if (q) cudaFree(q);
}
}  // namespace

extern "C" {

int sym_reach_analyze(sym_handle h, int64_t nnzb, const int32_t *bidx, sym_reach *out) {
  if (!out) return fail(SYM_ERR_INVALID, "null output");
  *out = nullptr;
  if (!h) return fail(SYM_ERR_INVALID, "null handle");
  int rc = h->host_only ? SYM_OK : check_device(h);
  if (rc) return rc;
  if (nnzb < 0 || (nnzb > 0 && !bidx)) return fail(SYM_ERR_INVALID, "bad right-hand side pattern");
  sym_reach_s *r = new (std::nothrow) sym_reach_s();
  if (!r) return fail(SYM_ERR_OOM, "host allocation");
  r->h = h;
  std::string err;
  try {
    rc = sym::build_reach(h->plan, nnzb, bidx, r->r, err);
  } catch (const std::bad_alloc &) {
    rc = SYM_ERR_OOM;
    err = "host allocation";
  }
  if (rc) {
    delete r;
    return fail(rc, err);
  }
  if (h->host_only) {  // inspection only: the reach can be exported but not solved with
    *out = r;
    return SYM_OK;
  }
  int64_t bytes = 0;
  rc = upload(r->r.pbeta, &r->d_pbeta, bytes);
  if (!rc) rc = upload(r->r.cols, &r->d_cols, bytes);
  if (!rc) rc = upload(r->r.snodes, &r->d_snodes, bytes);
  if (!rc) rc = upload(r->r.upd_tasks, &r->d_ut, bytes);
  if (!rc) rc = upload(r->r.upd_entries, &r->d_ue, bytes);
  if (!rc) rc = upload(r->r.tasks, &r->d_tasks, bytes);
  if (rc) {
    reach_release(r);
    delete r;
    return rc;
  }
  r->dp = h->dp;
  r->dp.upd_tasks = (const sym::UpdTask *)r->d_ut;
  r->dp.upd_entries = (const sym::UpdEntry *)r->d_ue;
  r->dp.tasks = (const sym::Int4 *)r->d_tasks;
  *out = r;
  return SYM_OK;
}

int64_t sym_reach_size(sym_reach r) { return r ? (int64_t)r->r.cols.size() : fail(SYM_ERR_INVALID, "null reach"); }

int sym_reach_indices(sym_reach r, int32_t *idx) {
  if (!r || !idx) return fail(SYM_ERR_INVALID, "null argument");
  const auto &perm = r->h->plan.perm;
  for (size_t t = 0; t < r->r.cols.size(); ++t) idx[t] = perm[r->r.cols[t]];
  return SYM_OK;
}

int64_t sym_reach_export(sym_reach r, int32_t what, void *out) {
  if (!r) return fail(SYM_ERR_INVALID, "null reach");
  const std::vector<int32_t> *v = what == 0 ? &r->r.cols : what == 1 ? &r->r.snodes : nullptr;
  if (!v) return fail(SYM_ERR_INVALID, "unknown item");
  if (out && !v->empty()) std::memcpy(out, v->data(), v->size() * sizeof(int32_t));
  return (int64_t)v->size();
}

int sym_solve_lower_sparse(sym_handle h, sym_reach r, const double *bvals, double *xvals) {
  int rc = check_device(h);
  if (rc) return rc;
  if (!r || r->h != h) return fail(SYM_ERR_INVALID, "reach set of another handle");
  if (!h->factored) return fail(SYM_ERR_STATE, "no successful factorization to solve with");
  if (h->precision != SYM_PREC_FP64) return fail(SYM_ERR_STATE, "the sparse solve needs an FP64 factor");
  if ((!bvals && !r->r.pbeta.empty()) || (!xvals && !r->r.cols.empty())) return fail(SYM_ERR_INVALID, "null vector");
  if (!h->solve_prepared) {
    CUDA_TRY((sym::prepare_solve<double, double>()), "solve set-up");
    h->solve_prepared = true;
  }
  rc = ensure_y(h, h->plan.n);
  if (rc) return rc;
  CUDA_TRY(sym::run_sparse_lower(r->dp, r->r.fwd, h->d_Lx, h->d_Linv, (const int32_t *)r->d_snodes,
                                 (int64_t)r->r.snodes.size(), (const int32_t *)r->d_pbeta, bvals,
                                 (int64_t)r->r.pbeta.size(), (const int32_t *)r->d_cols, (int64_t)r->r.cols.size(),
                                 h->d_y, xvals, h->stream),
           "sparse solve");
  return SYM_OK;
}

void sym_reach_free(sym_reach r) {
  if (!r) return;
  reach_release(r);
  delete r;
}

const char *sym_error_string(int code) {
  switch (code) {
    case SYM_OK: return "ok";
    case SYM_ERR_INVALID: return "invalid argument or pattern";
    case SYM_ERR_NOT_SPD: return "matrix is not positive definite";
    case SYM_ERR_CUDA: return "CUDA error";
    case SYM_ERR_OOM: return "out of memory";
    case SYM_ERR_STATE: return "call out of order";
    case SYM_ERR_TIMEOUT: return "device wait timed out";
    case SYM_ERR_LIMIT: return "size limit exceeded";
    case SYM_ERR_NO_CONVERGENCE: return "refinement did not converge";
    default: return "unknown error";
  }
}

const char *sym_last_error_string(void) { return g_last_error.c_str(); }

void sym_free(sym_handle h) {
  if (!h) return;
  if (!h->host_only) release_device(h);
  delete h;
}

}  // extern "C"
