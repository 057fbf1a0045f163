// refine.h — FP64 conjugate-gradient refinement around an FP32 factor (internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "kernels.h"
#include "plan.h"

namespace sym {

// One application of the FP32 preconditioner (solves with the FP32 factor, ~500 short kernels)
// captured as a CUDA graph and replayed at every CG iteration; owned by the handle, rebuilt when
// a key changes.
struct PrecondGraph {
  cudaGraphExec_t exec = nullptr;
  const void *key[4] = {nullptr, nullptr, nullptr, nullptr};  // input, output, FP32 work, factor
  int nrhs = 0;
};
void precond_graph_reset(PrecondGraph &g);

struct RefineCtx {
  const DevPlan *dp = nullptr;
  const std::vector<Launch> *fwd = nullptr;
  const std::vector<Launch> *bwd = nullptr;
  const float *Lf = nullptr;      // FP32 factor panels
  const float *Lfinv = nullptr;   // inverses of its diagonal tiles
  const int64_t *cp = nullptr;    // CSR of P A P^T (both triangles)
  const int32_t *ci = nullptr;
  const int64_t *cmap = nullptr;  // value of entry p is Ax[cmap[p]]
  const double *Ax = nullptr;     // device copy of A's values (caller's order)
  double *anorm = nullptr;        // device scalar ||A||_inf
  double *anorm_work = nullptr;   // fixed scratch of refine_anorm (n + 512 doubles); a captured
                                  // factor graph references it, so it never moves
  double *work = nullptr;         // at least refine_work_doubles(n, nrhs) doubles
  int64_t n = 0;
  PrecondGraph *pgraph = nullptr;  // non-null: replay the preconditioner as a graph, captured on
  cudaStream_t capture = nullptr;  // this (non-default) stream
};

struct RefineResult {
  int iterations = 0;
  double backward_error = 0.0;
  bool converged = true;
};

// Doubles of work space refine_solve needs for n x nrhs (nrhs <= 64).
int64_t refine_work_doubles(int64_t n, int nrhs);

// ||A||_inf into *ctx.anorm (uses ctx.anorm_work).
cudaError_t refine_anorm(const RefineCtx &ctx, cudaStream_t st);

// Solve A X = B (nrhs <= 64 columns, DEVICE pointers) to normwise backward error <= tol by
// preconditioned CG; host_eta: pinned buffer of 256 doubles. Returns 0, or -1 on a CUDA error.
int refine_solve(const RefineCtx &ctx, int nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                 double tol, int max_iter, double *host_eta, RefineResult *res, cudaStream_t st);

}  // namespace sym
