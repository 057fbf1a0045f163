// kernels.h — host entry points of the CUDA kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "plan.h"

namespace sym {

// Device copy of the plan arrays the kernels read.
struct DevPlan {
  const SNode *sn = nullptr;
  const int32_t *rows = nullptr;
  const int32_t *rel = nullptr;
  const int64_t *amap = nullptr;
  const UpdTask *upd_tasks = nullptr;
  const UpdEntry *upd_entries = nullptr;
  const Int4 *tasks = nullptr;
  const int32_t *perm = nullptr;
  const int64_t *cptr = nullptr;     // contribution lists of the forward solve (n + 1)
  const int32_t *contrib = nullptr;
  void *t = nullptr;                 // forward-solve buffer: SOLVE_MAXRHS x tsize of the solve type
  int64_t tsize = 0;
  int64_t n = 0;
  int64_t nnz_a = 0;
  int64_t storage = 0;
  bool tensor_cores = true;          // FP32 updates on tcgen05 (false: the FP32 SIMT kernel)
  uint64_t tc_wait_ns = 1000000000ull;  // limit of each bounded wait of the tensor-core update
  int32_t tc_withhold = 0;           // failure-path test: the tensor-core update issues no MMA
                                     // and no commit, so its first wait runs out
  double *piv = nullptr;             // FP32 factors: the FP64 pivot d_k of every permuted column k
                                     // (n per matrix), written by the POTRF kernels; else null
  const int8_t *batch_warp = nullptr;  // HOST array, one per factor launch: a batch's default form
                                       // of the launch is one warp per (tile, matrix) (full-tile
                                       // FP64 updates with small entries)
  const int8_t *batch_lanes = nullptr;     // HOST array, one per factor launch: a batch's lanes
                                           // per matrix for small-tile updates (Plan::batch_lanes)
  const PanelForm *batch_panel = nullptr;  // HOST array, one per factor launch: the fused narrow
                                           // levels (Plan::batch_panel); null: none
  const int8_t *panel_apart[2] = {nullptr, nullptr};  // HOST arrays (Plan::panel_apart): levels
                                           // the autotuner runs as separate launches ([0] one
                                           // matrix, [1] batches); null: none
  const PanelForm *fwd_panel = nullptr;    // HOST arrays (Plan::fwd_panel, bwd_panel): the fused
  const PanelForm *bwd_panel = nullptr;    // narrow solve levels; null: none
  int64_t nfwd_panel = 0, nbwd_panel = 0;  // their lengths (the solve lists' launch counts)
  const int8_t *variant[2] = {nullptr, nullptr};  // HOST arrays, one entry per factor launch,
                                     // [0] for one matrix, [1] for batches: 1 runs the launch's
                                     // alternative kernel form (see factor_launch_has_alternative),
                                     // as the autotuner chose; null or 0: the default form
  const double *axc = nullptr;       // FP32 factors: the FP64 copy of A's values (nnz_a per matrix)
  const int64_t *dpos = nullptr;     // FP32 factors: index in A's values of C_kk, per column k
};

// Several matrices with one pattern (blockIdx.y = matrix): offsets, in elements, from one matrix to
// the next of the panels (lx), of A's values (ax), of the diagonal-tile inverses (dinv), of the
// permuted solve block (y) and of the caller's right-hand sides (b) and solutions (x). The
// default describes a single matrix.
struct Batch {
  int32_t count = 1;
  int64_t lx = 0, ax = 0, dinv = 0, y = 0, b = 0, x = 0, t = 0, piv = 0, nnz = 0;  // nnz: DevPlan::axc
};

// Second stream for the factor's lookahead: aux runs the launches with stream == 1 at low
// priority; events[i] is recorded after launch i (at least one event per launch); fork/join
// attach aux to the main stream (also inside a CUDA-graph capture).
struct TwoStreams {
  cudaStream_t aux = nullptr;
  std::vector<cudaEvent_t> *events = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int prio_high = 0, prio_low = 0;
};

// Optional per-launch timing: when non-null, an event is recorded before the first launch and
// after every launch on the same stream; kinds[i] is the Kind of launch i (K_SCATTER for the
// zero + scatter pair, S_PERM for the permutations of the solve).
struct LaunchTrace {
  std::vector<cudaEvent_t> *events = nullptr;  // at least launches + 3 events
  std::vector<int32_t> kinds;
  int used = 0;
};

// Per-device function attributes the factor kernels need (call with the device current, before
// the first run_factor and outside stream capture).
template <typename T>
cudaError_t prepare_factor();

// Per-device function attributes of the solve kernels (with the device current, outside capture).
template <typename T, typename V>
cudaError_t prepare_solve();

// External updates of FP32 factors on the tensor cores (tc_update.cu): the attribute the kernel
// needs (once per device, outside capture), and one launch of grid.x tiles of the UpdTask list
// from toff. A bounded wait that runs out records -1 in status.
cudaError_t prepare_update_tc();
cudaError_t launch_update_tc(dim3 grid, cudaStream_t st, int prio, const DevPlan &d, float *Lx, int64_t toff,
                             const Batch &bt, long long *status);

// Whether a factor launch has a second kernel form (the autotuner times both). A batch
// (nbatch > 1): FP64 updates with lanes mapped to matrices (default for small tiles and for full
// tiles with small entries, DevPlan::batch_warp) against one warp per (tile, matrix) (small tiles;
// full tiles with small entries, in global memory) or one CTA per tile and matrix (the default of
// full tiles with large entries); small-tile POTRF, TRSM and TRTRI, one warp per (tile, matrix)
// or one CTA per tile and matrix. One matrix: clustered FP64 updates or one CTA per tile; FP32
// full-tile updates on the tensor cores or the SIMT pipes; small-tile POTRF and TRTRI, one CTA or
// one warp per tile. fp64: the factor's precision.
bool factor_launch_has_alternative(const Launch &L, int32_t nbatch, bool fp64);

// Numeric factorization: scatter A into the zeroed panels, then run the launch schedule.
// status: device int64, receives the smallest failing (permuted) column, or stays INT64_MAX;
// -1 when a bounded device wait ran out.
template <typename T>
cudaError_t run_factor(const DevPlan &d, const std::vector<Launch> &launches, const double *Ax,
                       T *Lx, T *Linv, long long *status, cudaStream_t st, LaunchTrace *trace = nullptr,
                       const Batch &bt = Batch(), const TwoStreams *two = nullptr);

// Solve with nrhs right-hand sides: y = P b, forward sweep, backward sweep, x = P^T y.
// y: device work array of n * nrhs (ld n); Linv: the diagonal-tile inverses run_factor wrote.
template <typename T>
cudaError_t run_solve(const DevPlan &d, const std::vector<Launch> &fwd, const std::vector<Launch> &bwd,
                      const T *Lx, const T *Linv, int nrhs, const double *B, int64_t ldb, double *X,
                      int64_t ldx, double *y, cudaStream_t st, LaunchTrace *trace = nullptr,
                      const Batch &bt = Batch());

// The forward and backward sweeps alone on a permuted block y (n x nrhs, ld n) of type V.
template <typename T, typename V>
cudaError_t run_sweeps(const DevPlan &d, const std::vector<Launch> &fwd, const std::vector<Launch> &bwd,
                       const T *Lx, const T *Linv, int nrhs, V *y, cudaStream_t st, LaunchTrace *trace = nullptr,
                       const Batch &bt = Batch());

// Forward solve L y = P b for a sparse b on a pruned schedule: zero the reached supernodes'
// columns of y, scatter b (permuted positions pbeta), run the pruned forward sweep, gather the
// nr reached columns into x.
cudaError_t run_sparse_lower(const DevPlan &d, const std::vector<Launch> &fwd, const double *Lx,
                             const double *Linv, const int32_t *snodes, int64_t nsn, const int32_t *pbeta,
                             const double *bvals, int64_t nb, const int32_t *cols, int64_t nr, double *y,
                             double *x, cudaStream_t st);

// The breakdown measure of an FP32 factor's pivots: for matrix b of the batch, the smallest
// ratio d_k / C_kk of the FP64 pivot to the diagonal entry of C = P A P^T, and its column k
// (smallest k on ties). Ax: A's values (matrix b at Ax + b * axstride); dpos[k]: index in Ax of
// C_kk.
struct PivotInfo {
  double min_ratio;
  int64_t column;
};
cudaError_t pivot_ratio(const double *piv, int64_t n, const double *Ax, int64_t axstride, const int64_t *dpos,
                        int32_t nbatch, PivotInfo *out, cudaStream_t st);

// y = P B and X = P^T y for nrhs columns.
template <typename V>
cudaError_t permute_in(const DevPlan &d, int nrhs, const double *B, int64_t ldb, V *y, cudaStream_t st);
template <typename V>
cudaError_t permute_out(const DevPlan &d, int nrhs, const V *y, double *X, int64_t ldx, cudaStream_t st);

}  // namespace sym
