// kernels.cu — CUDA kernels (sm_103a) of the supernodal left-looking Cholesky numeric phase and
// the supernodal triangular solves, plus the host loops that walk the precomputed schedule.
//
// Paper mapping (Sec. 3.2, VS-Block + VI-Prune on left-looking Cholesky): for each supernode J,
//   (a) update: L_J -= sum over descendants K (the block prune-set) of L_K[R1,:] L_K[R0,:]^T,
//       scattered through the relative row maps, one CTA (or cluster) per NB x NB tile of J —
//       k_update_flat (FP64), k_update_f32 (FP32), k_update_tc (FP32 on the tensor cores,
//       tc_update.cu);
//   (b) dense Cholesky of the diagonal block — k_potrf (per diagonal tile; k_potrf_r for FP32
//       tiles of order NB) and
//   (c) dense triangular solves on the rows below it — k_trsm (k_trsm_r for FP32 tiles of
//       NB columns), with k_gemm applying the
//       trailing updates inside J when J is wider than one tile.
// Supernodes of one level of the supernodal tree are independent and run in the same launches.
// The solve follows Sec. 3.1: diagonal block first, then the off-diagonal part; the forward
// sweep gathers each supernode's input from its descendants, the backward sweep (L^T) gathers
// from the rows below the diagonal block.
//
// The FP64 path is bound by the FP64 FMA pipe (about 2 DFMA per clock per SM on GB300), so the
// kernels keep that pipe busy with useful work: a flat map of output elements onto threads for
// the updates, register tiles of 2 x 8 outputs per thread for the in-supernode GEMM, operand
// chunks staged in shared memory, warp-uniform guards that skip whole warps outside ragged
// tiles, and no atomics in the factorization (every tile is owned by one CTA or cluster,
// descendants are applied in a fixed order, so results are deterministic).
#include <cooperative_groups.h>
#include <type_traits>

#include <cmath>

#include <cstdint>
#include <utility>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace sym {
namespace {

constexpr int THREADS = 256;
constexpr int KC = 16;  // inner-dimension chunk staged in shared memory (k_gemm)
constexpr int KCU = 8;  // the same for the FP64 update kernels (accumulator tile in shared memory)
// Small-tile variants: a launch whose tiles all have at most 32 rows and columns (or, for TRSM,
// at most 32 columns) runs kernels sized for 32 x 32 tiles with 128 threads, so that many more
// CTAs share an SM than the 64 x 64 forms allow (the batched workloads and the lower levels of the
// supernodal tree are made of such tiles).
constexpr int SMALL_TB = SMALL_TILE;
template <int TB>
struct TileCfg {
  static constexpr int threads = TB == NB ? THREADS : 128;
};

// Inner-dimension chunks per storage type: FP64 is bound by its pipe, so small chunks suffice; at
// the FP32 rate a chunk must carry enough multiply-adds to cover the latency of staging the next.
template <typename T>
struct Chunk {
  static constexpr int gemm = KC;
};
template <>
struct Chunk<float> {
  static constexpr int upd = 32, gemm = 64;
};

__device__ __forceinline__ int64_t d_row_tile_base(int32_t i, int32_t ncols, int32_t ncb) {
  return i < ncb ? (int64_t)i * NB : (int64_t)ncols + (int64_t)(i - ncb) * NB;
}
__device__ __forceinline__ int d_row_tile_rows(int32_t i, int32_t ncols, int32_t nrows, int32_t ncb) {
  int64_t base = d_row_tile_base(i, ncols, ncb);
  int64_t end = i < ncb ? ncols : nrows;
  int64_t r = end - base;
  return (int)(r < NB ? r : NB);
}

// r[i][j] -= A[kk][lane + 32 i] * B[kk][w + 8 j] for kk < kc, for the first NI row halves and the
// first NJ column slots of this warp. The shapes are template parameters so that no FMA of an
// inactive slot is ever issued (a run-time guard would be if-converted into predicated FMAs,
// which still occupy the FP64 pipe).
template <int NI, int NJ, int KMAX, typename T>
__device__ __forceinline__ void fma_chunk(T (&r)[2][8], const T (*As)[NB], const T (*Bs)[NB], int kc,
                                          int lane, int w) {
#pragma unroll 2
  for (int kk = 0; kk < kc; ++kk) {
    const T a0 = As[kk][lane];
    const T a1 = NI > 1 ? As[kk][lane + 32] : T(0);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const T bv = Bs[kk][w + 8 * j];
      r[0][j] = fma(-a0, bv, r[0][j]);
      if (NI > 1) r[1][j] = fma(-a1, bv, r[1][j]);
    }
  }
}

// Warp-uniform dispatch on (ni, nj); every case is its own straight-line loop.
template <int KMAX, typename T>
__device__ __forceinline__ void fma_chunk_dispatch(T (&r)[2][8], const T (*As)[NB], const T (*Bs)[NB],
                                                   int kc, int lane, int w, int ni, int nj) {
#define SYM_CASE(J)                                                  \
  case J:                                                            \
    if (ni > 1) fma_chunk<2, J, KMAX>(r, As, Bs, kc, lane, w);       \
    else fma_chunk<1, J, KMAX>(r, As, Bs, kc, lane, w);              \
    break;
  switch (nj) {
    SYM_CASE(1)
    SYM_CASE(2)
    SYM_CASE(3)
    SYM_CASE(4)
    SYM_CASE(5)
    SYM_CASE(6)
    SYM_CASE(7)
    SYM_CASE(8)
    default:
      break;
  }
#undef SYM_CASE
}

// Reciprocal square root of d > 0 in FP64: with a seed x0 of relative error e0 (the hardware
// approximation of PTX rsqrt.approx.f64, |e0| < 2^-20 measured over 2^20 random d) and
// e = 1 - d x0^2, the exact value is x0 (1 - e)^(-1/2) = x0 (1 + e/2 + 3e^2/8 + 5e^3/16 + ...).
// Keeping the terms through e^2 leaves a relative error of about 5 e^3 / 16 < 2^-56, so one step
// reaches double precision up to rounding (a Householder step of order 3; d x is within one ulp
// of sqrt(d) over the same sample). The chain is five dependent operations, which keeps the
// serial pivot path of a Cholesky short on a GPU whose FP64 pipe is narrow (a single-precision
// seed would add two conversions, ~40% more latency per pivot). Outside (1e-30, 1e30) it falls
// back to 1/sqrt.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double x0;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(x0) : "d"(d));
  const double e = fma(-d * x0, x0, 1.0);
  const double p = fma(0.375, e, 0.5);
  return fma(x0 * e, p, x0);
}

// The same in FP32: the single-precision seed plus one Newton step x <- x (3 - d x^2) / 2.
__device__ __forceinline__ float rsqrt_newton(float d) {
  const float x = rsqrtf(d);
  return x * fmaf(-0.5f * d * x, x, 1.5f);
}
template <typename T>
__device__ __forceinline__ T rsqrt_of(T d) {
  return rsqrt_newton(d);
}

// ---------------------------------------------------------------------------------------------
// Scatter of A into the zeroed panels (the temporary block storage of Sec. 2.3.2).
template <typename T>
__global__ void k_zero(T *__restrict__ x, int64_t count, const Batch bt) {
  x += blockIdx.y * bt.lx;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < count; i += stride) x[i] = T(0);
}

template <typename T>
__global__ void k_scatter(const double *__restrict__ Ax, const int64_t *__restrict__ amap,
                          T *__restrict__ Lx, int64_t nnz, const Batch bt) {
  Ax += blockIdx.y * bt.ax;
  Lx += blockIdx.y * bt.lx;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < nnz; i += stride) Lx[amap[i]] = (T)Ax[i];
}

// ---------------------------------------------------------------------------------------------
// (a) External update of one tile (bi, bj) of supernode J by all its descendant entries: FP32
// factors use the 4 x 8 register tile below, FP64 factors the flat element map further down.
// FP32 register tile: r[i][j] -= A[kk][4 rg + i] * B[kk][8 cg + j] for kk < kc, with one 16-byte
// load of A and two of B per step (3 shared-memory loads per 32 multiply-adds; the FP32 pipe is
// 32 times faster than FP64 on this part, so operand traffic, not arithmetic, bounds a thinner
// tile: the 2 x 8 form issues 10 loads per 16 multiply-adds and measured 26% FMA-pipe use).
constexpr int F32_THREADS = 128;
__device__ __forceinline__ void f32_chunk(float (&r)[4][8], const float (*As)[NB], const float (*Bs)[NB], int kc,
                                          int rg, int cg) {
#pragma unroll 4
  for (int kk = 0; kk < kc; ++kk) {
    const float4 a = *reinterpret_cast<const float4 *>(&As[kk][4 * rg]);
    const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][8 * cg]);
    const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][8 * cg + 4]);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) r[i][j] = fmaf(-av[i], bv[j], r[i][j]);
  }
}

// (a'') The external update for an FP32 factor: 128 threads, thread (rg, cg) = (tid % 16, tid / 16)
// owns rows 4 rg .. 4 rg + 3 and columns 8 cg .. 8 cg + 7 of an entry's m x n block.
__global__ void __launch_bounds__(F32_THREADS) k_update_f32(const SNode *__restrict__ sn,
                                                            const UpdTask *__restrict__ tasks,
                                                            const UpdEntry *__restrict__ ents,
                                                            const int32_t *__restrict__ rel,
                                                            float *__restrict__ Lx, int64_t toff, const Batch bt) {
  constexpr int KU = Chunk<float>::upd;
  Lx += blockIdx.y * bt.lx;
  __shared__ float acc[NB][NB + 1];  // [col][row]
  __shared__ __align__(16) float As[KU][NB];
  __shared__ __align__(16) float Bs[KU][NB];
  __shared__ int prow[NB], pcol[NB];
  const UpdTask t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.J];
  const int64_t rb = d_row_tile_base(t.bi, sj.ncols, sj.ncb);
  const int tm = d_row_tile_rows(t.bi, sj.ncols, sj.nrows, sj.ncb);
  const int cb = t.bj * NB;
  const int tn = min(NB, sj.ncols - cb);
  float *C = Lx + sj.lx + (int64_t)cb * sj.nrows + rb;
  const int tid = threadIdx.x, rg = tid & 15, cg = tid >> 4;
  for (int idx = tid; idx < tm * tn; idx += F32_THREADS) {
    int r = idx % tm, c = idx / tm;
    acc[c][r] = C[(int64_t)c * sj.nrows + r];
  }
  for (int64_t e = t.e0; e < t.e1; ++e) {
    const UpdEntry E = ents[e];
    const SNode sk = sn[E.K];
    if (tid < E.m) prow[tid] = rel[E.relr + tid] - (int)rb;
    if (tid >= NB && tid - NB < E.n) pcol[tid - NB] = rel[E.relc + tid - NB] - cb;
    __syncthreads();
    const bool active = 4 * rg < E.m && 8 * cg < E.n;
    float r[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int a = 4 * rg + i, b = 8 * cg + j;
        r[i][j] = (a < E.m && b < E.n) ? acc[pcol[b]][prow[a]] : 0.f;
      }
    const float *Kp = Lx + sk.lx;
    for (int k0 = 0; k0 < sk.ncols; k0 += KU) {
      const int kc = min(KU, sk.ncols - k0);
      for (int idx = tid; idx < KU * NB; idx += F32_THREADS) {
        int a = idx % NB, kk = idx / NB;
        const float *col = Kp + (int64_t)(k0 + kk) * sk.nrows;
        As[kk][a] = (a < E.m && kk < kc) ? col[E.r_lo + a] : 0.f;
        Bs[kk][a] = (a < E.n && kk < kc) ? col[E.c_lo + a] : 0.f;
      }
      __syncthreads();
      if (active) f32_chunk(r, As, Bs, kc, rg, cg);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int a = 4 * rg + i, b = 8 * cg + j;
        if (a < E.m && b < E.n) acc[pcol[b]][prow[a]] = r[i][j];
      }
    __syncthreads();
  }
  __syncthreads();
  for (int idx = tid; idx < tm * tn; idx += F32_THREADS) {
    int r = idx % tm, c = idx / tm;
    C[(int64_t)c * sj.nrows + r] = acc[c][r];
  }
}

// (c'') The trailing update inside J for an FP32 factor, with the same 4 x 8 register tile.
__global__ void __launch_bounds__(F32_THREADS) k_gemm_f32(const SNode *__restrict__ sn,
                                                          const Int4 *__restrict__ tasks,
                                                          float *__restrict__ Lx, int64_t toff, const Batch bt) {
  constexpr int KG = Chunk<float>::gemm;
  Lx += blockIdx.y * bt.lx;
  __shared__ __align__(16) float As[KG][NB];
  __shared__ __align__(16) float Bs[KG][NB];
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int i = t.b, j = t.c, s = t.d & 0xffff;
  int64_t rb = d_row_tile_base(i, sj.ncols, sj.ncb);
  int tm = d_row_tile_rows(i, sj.ncols, sj.nrows, sj.ncb);
  const int half = t.d >> 16;  // 0: whole tile; 1, 2: its first or second 32 rows
  if (half) {
    rb += (half - 1) * (NB / 2);
    tm = max(0, min(NB / 2, tm - (half - 1) * (NB / 2)));
  }
  const int tn = min(NB, sj.ncols - j * NB);
  const int ks = min(NB, sj.ncols - s * NB);
  const float *P = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows;  // column block s
  float *C = Lx + sj.lx + (int64_t)(j * NB) * sj.nrows + rb;
  const int tid = threadIdx.x, rg = tid & 15, cg = tid >> 4;
  const bool active = 4 * rg < tm && 8 * cg < tn;
  float r[4][8];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int a = 4 * rg + ii, b = 8 * cg + jj;
      r[ii][jj] = (a < tm && b < tn) ? C[(int64_t)b * sj.nrows + a] : 0.f;
    }
  for (int k0 = 0; k0 < ks; k0 += KG) {
    const int kc = min(KG, ks - k0);
    for (int idx = tid; idx < KG * NB; idx += F32_THREADS) {
      int a = idx % NB, kk = idx / NB;
      const float *col = P + (int64_t)(k0 + kk) * sj.nrows;
      As[kk][a] = (a < tm && kk < kc) ? col[rb + a] : 0.f;
      Bs[kk][a] = (a < tn && kk < kc) ? col[(int64_t)j * NB + a] : 0.f;
    }
    __syncthreads();
    if (active) f32_chunk(r, As, Bs, kc, rg, cg);
    __syncthreads();
  }
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int a = 4 * rg + ii, b = 8 * cg + jj;
      if (a < tm && b < tn) C[(int64_t)b * sj.nrows + a] = r[ii][jj];
    }
}

// r[j] -= A[kk][a_j] * B[kk][b_j] for kk < kc and the first J element slots of this thread
// (a_j = ab[j] & 0xff, b_j = ab[j] >> 8).
constexpr int FLAT_SLOTS = 8;  // output elements per thread and pass
template <int J, int TB, typename T>
__device__ __forceinline__ void flat_chunk(T (&r)[FLAT_SLOTS], const int (&ab)[FLAT_SLOTS], const T (*As)[TB],
                                           const T (*Bs)[TB], int kc) {
#pragma unroll 2
  for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
    for (int j = 0; j < J; ++j) r[j] = fma(-As[kk][ab[j] & 0xff], Bs[kk][ab[j] >> 8], r[j]);
  }
}

template <int TB, typename T>
__device__ __forceinline__ void flat_chunk_dispatch(T (&r)[FLAT_SLOTS], const int (&ab)[FLAT_SLOTS],
                                                    const T (*As)[TB], const T (*Bs)[TB], int kc, int jw) {
#define SYM_CASE(J) \
  case J:           \
    flat_chunk<J, TB>(r, ab, As, Bs, kc); \
    break;
  switch (jw) {
    SYM_CASE(1) SYM_CASE(2) SYM_CASE(3) SYM_CASE(4) SYM_CASE(5) SYM_CASE(6) SYM_CASE(7) SYM_CASE(8)
    default:
      break;
  }
#undef SYM_CASE
}

// (a') The same external update for an FP64 factor, with a flat map of the entry's output
// elements onto the threads: element e of an entry (e < m n, or e < m (m + 1) / 2 on a diagonal
// tile, whose strictly upper part is never needed) goes to thread e % 256, slot e / 256; slots
// are taken 8 at a time (one pass over ncols(K) per 2048 elements) to keep three CTAs per SM.
// Every multiply-add is then useful except in the last slot of a partial warp (a register-
// blocked form, computing whole 32-row halves and full squares on diagonal tiles, was 92% useful
// on the 64^3 workload). Each multiply-add takes its own two operands from shared memory, which
// the narrow FP64 pipe leaves ample room for (one warp-wide DFMA per sub-partition every 64
// cycles). Every element accumulates its entries' products in entry order, k ascending.
template <typename T, int TB, bool CLUSTER>
__global__ void __launch_bounds__(TileCfg<TB>::threads, TB == NB ? (CLUSTER ? 2 : 3) : 6)
    k_update_flat(const SNode *__restrict__ sn, const UpdTask *__restrict__ tasks,
                  const UpdEntry *__restrict__ ents, const int32_t *__restrict__ rel, T *__restrict__ Lx,
                  int64_t toff, const Batch bt) {
  constexpr int TT = TileCfg<TB>::threads;
  Lx += blockIdx.y * bt.lx;
  __shared__ T acc[TB][TB + 1];  // [col][row]
  __shared__ T As[KCU][TB];
  __shared__ T Bs[KCU][TB];
  __shared__ int prow[TB], pcol[TB];
  // A launch with few tiles runs each tile on a thread-block cluster: rank r applies entries
  // r, r + cs, ... to its own accumulator (rank 0 starts from the tile, the others from zero) and
  // rank 0 adds the others' partial tiles in rank order through distributed shared memory, so the
  // result does not depend on scheduling.
  // (CLUSTER = false: one CTA per tile, without the cluster bookkeeping and its registers.)
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = CLUSTER ? (int)cluster.num_blocks() : 1;
  const int rank = CLUSTER ? (int)cluster.block_rank() : 0;
  const UpdTask t = tasks[toff + blockIdx.x / cs];
  const SNode sj = sn[t.J];
  const int64_t rb = d_row_tile_base(t.bi, sj.ncols, sj.ncb);
  const int tm = d_row_tile_rows(t.bi, sj.ncols, sj.nrows, sj.ncb);
  const int cb = t.bj * NB;
  const int tn = min(NB, sj.ncols - cb);
  const bool diag = t.bi == t.bj;  // rows and columns of the tile are the same positions
  T *C = Lx + sj.lx + (int64_t)cb * sj.nrows + rb;
  const int tid = threadIdx.x, w = tid >> 5;
  for (int idx = tid; idx < tm * tn; idx += TT) {  // only the tile's own part is read
    int r = idx % tm, c = idx / tm;
    acc[c][r] = rank == 0 ? C[(int64_t)c * sj.nrows + r] : T(0);
  }
  for (int64_t e = t.e0 + rank; e < t.e1; e += cs) {
    const UpdEntry E = ents[e];
    const SNode sk = sn[E.K];
    if (tid < E.m) prow[tid] = rel[E.relr + tid] - (int)rb;
    if (tid >= TB && tid - TB < E.n) pcol[tid - TB] = rel[E.relc + tid - TB] - cb;
    __syncthreads();
    const int cnt = diag ? E.m * (E.m + 1) / 2 : E.m * E.n;
    const T *Kp = Lx + sk.lx;
    // Operands of one chunk: only rows the entry has and values of K it reaches are staged and
    // read.
    auto stage = [&](int k0, int kc) {
      for (int idx = tid; idx < kc * TB; idx += TT) {
        const int a = idx % TB, kk = idx / TB;
        const T *col = Kp + (int64_t)(k0 + kk) * sk.nrows;
        if (a < E.m) As[kk][a] = col[E.r_lo + a];
        if (a < E.n) Bs[kk][a] = col[E.c_lo + a];
      }
    };
    auto decode = [&](int el, int &a, int &b) {
      if (diag) {  // row-major lower triangle: el = a (a + 1) / 2 + b, b <= a
        a = (int)((sqrtf(8.0f * el + 1.0f) - 1.0f) * 0.5f);
        while ((a + 1) * (a + 2) / 2 <= el) ++a;
        while (a * (a + 1) / 2 > el) --a;
        b = el - a * (a + 1) / 2;
      } else {
        a = el % E.m;
        b = el / E.m;
      }
    };
    if (cnt <= TT) {
      // At most one element per thread (most entries of the lower levels and of small
      // matrices): no slot arrays, and warps without an element skip the multiply-adds and the
      // bookkeeping (the same operations in the same order as one slot of the general pass).
      const bool has = tid < cnt, wact = 32 * w < cnt;  // wact: warp-uniform
      int a = 0, b = 0;
      T r = T(0);
      if (has) {
        decode(tid, a, b);
        r = acc[pcol[b]][prow[a]];
      }
      for (int k0 = 0; k0 < sk.ncols; k0 += KCU) {
        const int kc = min(KCU, sk.ncols - k0);
        stage(k0, kc);
        __syncthreads();
        if (wact) {
#pragma unroll 2
          for (int kk = 0; kk < kc; ++kk) r = fma(-As[kk][a], Bs[kk][b], r);
        }
        __syncthreads();
      }
      if (has) acc[pcol[b]][prow[a]] = r;
    } else {
      for (int e0 = 0; e0 < cnt; e0 += FLAT_SLOTS * TT) {  // block-uniform passes
        const int rem = cnt - e0;
        const int nslot = min(FLAT_SLOTS, (rem + TT - 1) / TT);
        const int jw = TT * (nslot - 1) + 32 * w < rem ? nslot : nslot - 1;  // warp-uniform
        int ab[FLAT_SLOTS];
        T r[FLAT_SLOTS];
#pragma unroll
        for (int j = 0; j < FLAT_SLOTS; ++j) {
          const int el = e0 + tid + TT * j;
          int a = 0, b = 0;
          if (el < cnt) decode(el, a, b);
          ab[j] = a | (b << 8);
          r[j] = el < cnt ? acc[pcol[b]][prow[a]] : T(0);
        }
        for (int k0 = 0; k0 < sk.ncols; k0 += KCU) {
          const int kc = min(KCU, sk.ncols - k0);
          stage(k0, kc);
          __syncthreads();
          flat_chunk_dispatch<TB>(r, ab, As, Bs, kc, jw);
          __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < FLAT_SLOTS; ++j) {
          const int el = e0 + tid + TT * j;
          if (el < cnt) acc[pcol[ab[j] >> 8]][prow[ab[j] & 0xff]] = r[j];
        }
      }
    }
    __syncthreads();
  }
  if (!CLUSTER) {
    __syncthreads();
    for (int idx = tid; idx < tm * tn; idx += TT) {
      int r = idx % tm, c = idx / tm;
      C[(int64_t)c * sj.nrows + r] = acc[c][r];
    }
    return;
  }
  cluster.sync();  // every rank's partial tile is complete
  if (rank == 0) {
    for (int idx = tid; idx < tm * tn; idx += TT) {
      int r = idx % tm, c = idx / tm;
      T v = acc[c][r];
      for (int o = 1; o < cs; ++o) v += cluster.map_shared_rank(&acc[0][0], o)[c * (TB + 1) + r];
      C[(int64_t)c * sj.nrows + r] = v;
    }
  }
  cluster.sync();  // keep the other ranks' shared memory alive until rank 0 has read it
}

// ---------------------------------------------------------------------------------------------
// (b) Dense Cholesky of diagonal tile s of supernode J, in shared memory, column by column
// (right-looking). Column c+1 is on the critical path: warp 0 applies column c to it, takes its
// pivot and scales it, while the other warps apply column c to columns c+2.. — one barrier per
// column. A pivot that is not positive (or NaN) records its permuted column in *status (atomic
// min) and is replaced by 1 so the kernel finishes with finite values.
//
// An FP32 factor keeps its pivot chain in FP64: each diagonal entry is carried in FP64 (dd) as
// C_kk in FP64 plus the updates the earlier kernels accumulated in FP32 (the stored value minus
// C_kk rounded to FP32, a difference formed exactly), the tile's own updates l^2 are subtracted
// in FP64, and the pivot's reciprocal square root is taken in FP64; the off-diagonal entries and
// the column scaling stay in FP32. Every pivot d_k is stored in piv (FP64), from which the
// factorization's breakdown ratio min_k d_k / C_kk is formed.
__device__ __forceinline__ double diag64(float stored, const double *__restrict__ axc, const int64_t *__restrict__ dpos,
                                         int64_t g) {
  if (!axc) return (double)stored;
  const double c = axc[dpos[g]];
  return c + ((double)stored - (double)(float)c);
}

template <typename T, int TB>
__global__ void __launch_bounds__(TileCfg<TB>::threads) k_potrf(const SNode *__restrict__ sn,
                                                                const Int4 *__restrict__ tasks,
                                                                T *__restrict__ Lx, long long *status,
                                                                double *__restrict__ piv,
                                                                const double *__restrict__ axc,
                                                                const int64_t *__restrict__ dpos, int64_t toff,
                                                                const Batch bt) {
  constexpr int TT = TileCfg<TB>::threads;
  constexpr bool F64PIV = std::is_same<T, float>::value;
  Lx += blockIdx.y * bt.lx;
  status += blockIdx.y;
  __shared__ T a[TB][TB + 1];                      // [col][row]
  __shared__ unsigned short tri[TB * (TB - 1) / 2];  // packed lower triangle: (i << 8) | j, i >= j
  __shared__ double dd[F64PIV ? TB : 1];             // FP64 diagonal (FP32 factors)
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int s = t.b;
  const int ts = min(TB, sj.ncols - s * NB);  // a TB < NB launch holds tiles of order <= TB
  T *D = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + s * NB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (axc) axc += blockIdx.y * bt.nnz;
  for (int idx = tid; idx < ts * ts; idx += TT) {  // only the lower triangle is read
    int rr = idx % ts, c = idx / ts;
    if (rr >= c) {
      const T v = D[(int64_t)c * sj.nrows + rr];
      a[c][rr] = v;
      if (F64PIV && rr == c) dd[c] = diag64((float)v, axc, dpos, sj.first + s * NB + c);
    }
  }
  // Row-major packed index of the lower triangle: idx = i (i + 1) / 2 + j. The first
  // m (m + 1) / 2 entries are the triangle of order m, whatever m is; the largest trailing
  // triangle has order ts - 2.
  for (int idx = tid; idx < ts * (ts - 1) / 2; idx += TT) {
    int i = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= idx) ++i;
    while (i * (i + 1) / 2 > idx) --i;
    tri[idx] = (unsigned short)((i << 8) | (idx - i * (i + 1) / 2));
  }
  __syncthreads();
  // warp 0: pivot of column c (already updated by columns < c) and scaling of the column
  auto finish_column = [&](int c) {
    if constexpr (F64PIV) {
      // the pivot in FP64; its reciprocal square root only to FP32 accuracy, which is all the
      // FP32 column scaling can use (a further FP64 chain would only lengthen the serial path)
      double d = dd[c];
      if (!(d > 0.0)) {
        if (lane == 0) atomicMin(status, (long long)(sj.first + s * NB + c));
        d = 1.0;
      }
      if (lane == 0 && piv) piv[blockIdx.y * bt.piv + sj.first + s * NB + c] = d;
      const float df = (float)d;
      const float xf = rsqrt_newton(df);
      __syncwarp();
      for (int r = c + lane; r < ts; r += 32) a[c][r] = r == c ? (T)(df * xf) : a[c][r] * xf;  // d x = sqrt(d)
    } else {
      T d = a[c][c];
      if (!(d > T(0))) {
        if (lane == 0) atomicMin(status, (long long)(sj.first + s * NB + c));
        d = T(1);
      }
      const T x = rsqrt_of(d);
      __syncwarp();
      for (int r = c + lane; r < ts; r += 32) a[c][r] = r == c ? d * x : a[c][r] * x;  // d x = sqrt(d)
    }
  };
  if (warp == 0 && ts > 0) finish_column(0);
  __syncthreads();
  for (int c = 0; c + 1 < ts; ++c) {
    if (warp == 0) {
      const T l = a[c][c + 1];
      for (int r = c + 1 + lane; r < ts; r += 32) {
        if (F64PIV && r == c + 1) dd[r] = fma(-(double)l, (double)l, dd[r]);
        else a[c + 1][r] = fma(-a[c][r], l, a[c + 1][r]);
      }
      __syncwarp();
      finish_column(c + 1);
    } else if (F64PIV && warp == 1) {  // the FP64 diagonal of the trailing columns, one warp
      for (int rr = c + 2 + lane; rr < ts; rr += 32) dd[rr] = fma(-(double)a[c][rr], (double)a[c][rr], dd[rr]);
    } else {
      const int m = ts - c - 2;  // trailing lower triangle of order m, rows/cols c+2..ts-1
      const int tot = m * (m + 1) / 2;
      const int w0 = F64PIV ? 64 : 32;  // threads below w0 have other work
      for (int idx = tid - w0; idx < tot; idx += TT - w0) {
        const int ij = tri[idx];
        const int rr = c + 2 + (ij >> 8), cc = c + 2 + (ij & 0xff);
        if (!F64PIV || rr != cc) a[cc][rr] = fma(-a[c][rr], a[c][cc], a[cc][rr]);
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ts * ts; idx += TT) {
    int rr = idx % ts, c = idx / ts;
    D[(int64_t)c * sj.nrows + rr] = rr >= c ? a[c][rr] : T(0);
  }
}

// (c) Tile (i, s) <- tile * L_ss^{-T}: forward substitution over the tile's columns.
template <typename T, int TB>
__global__ void __launch_bounds__(TileCfg<TB>::threads) k_trsm(const SNode *__restrict__ sn,
                                                               const Int4 *__restrict__ tasks,
                                                               T *__restrict__ Lx, int64_t toff, const Batch bt) {
  constexpr int TT = TileCfg<TB>::threads;
  Lx += blockIdx.y * bt.lx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*Ls)[TB + 1] = reinterpret_cast<T(*)[TB + 1]>(smem_raw);                        // [col][row], lower
  T(*X)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(reinterpret_cast<T *>(smem_raw) + TB * (TB + 1));  // [col][row]
  T *dinv = reinterpret_cast<T *>(smem_raw) + TB * (TB + 1) + TB * (NB + 1);
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int i = t.b, s = t.c;
  const int ts = min(TB, sj.ncols - s * NB);  // a TB < NB launch holds tiles of <= TB columns
  int64_t rb = d_row_tile_base(i, sj.ncols, sj.ncb);
  int tm = d_row_tile_rows(i, sj.ncols, sj.nrows, sj.ncb);
  const int half = t.d >> 16;  // 0: whole tile; 1, 2: its first or second 32 rows
  if (half) {
    rb += (half - 1) * (NB / 2);
    tm = max(0, min(NB / 2, tm - (half - 1) * (NB / 2)));
  }
  const T *D = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + s * NB;
  T *B = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + rb;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < ts * ts; idx += TT) {  // lower triangle of L_ss
    int r = idx % ts, c = idx / ts;
    if (r >= c) Ls[c][r] = D[(int64_t)c * sj.nrows + r];
  }
  for (int idx = tid; idx < tm * ts; idx += TT) {
    int r = idx % tm, c = idx / tm;
    X[c][r] = B[(int64_t)c * sj.nrows + r];
  }
  __syncthreads();
  if (tid < ts) dinv[tid] = T(1) / Ls[tid][tid];
  __syncthreads();
  // Thread (r, g) owns row r and columns c+1+g, c+1+g+GR, ...: the tile's rows are spread over
  // GR = TT / tm column groups, so the threads of a warp are all busy whatever tm is (a warp-wide
  // FP64 instruction costs its pipe slot however few lanes are active).
  const int GR = tm > 0 ? TT / tm : 1;
  const int r = tm > 0 ? tid % tm : 0, g = tm > 0 ? tid / tm : GR;  // g >= GR: idle
  for (int c = 0; c < ts; ++c) {
    if (g < GR) {
      const T xc = X[c][r] * dinv[c];  // X(r, c) is final once columns < c are applied
      for (int cc = c + 1 + g; cc < ts; cc += GR) X[cc][r] = fma(-xc, Ls[c][cc], X[cc][r]);
    }
    __syncthreads();
    if (g == 0) X[c][r] *= dinv[c];
  }
  __syncthreads();
  for (int idx = tid; idx < tm * ts; idx += TT) {
    int r = idx % tm, c = idx / tm;
    B[(int64_t)c * sj.nrows + r] = X[c][r];
  }
}

// (b') FP32 diagonal tiles of order up to NB with the column chain in registers. Warp w of the
// first eight owns the columns w, w + 8, ... (lane l: rows l and l + 32 of each), the oldest
// unfinished one in v[0]; a column is published in shared memory once final. Step c, one barrier:
// the owner of column c applies column c - 1 to it, takes the FP64 pivot, scales the column and
// publishes it; every owner applies column c - 1 to its other columns right of it; warp 8
// subtracts l(k, c - 1)^2 from the FP64 diagonal of the rows k > c. Every element and every pivot
// sees the operations of k_potrf in the same order, so the factors are bit-identical; what
// changes is that the trailing columns stay in registers (k_potrf looks up a packed index and
// goes through shared memory for every update, and its barrier waits for those chains).
constexpr int PR_OWNERS = 8, PR_THREADS = 32 * (PR_OWNERS + 1);

__global__ void __launch_bounds__(PR_THREADS) k_potrf_r(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                       float *__restrict__ Lx, long long *status,
                                                       double *__restrict__ piv, const double *__restrict__ axc,
                                                       const int64_t *__restrict__ dpos, int64_t toff,
                                                       const Batch bt) {
  Lx += blockIdx.y * bt.lx;
  status += blockIdx.y;
  if (axc) axc += blockIdx.y * bt.nnz;
  __shared__ float col[NB][NB + 1];  // [c][row]: column c once final, zero above the diagonal
  __shared__ double dd[NB];          // FP64 diagonal (see k_potrf)
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int s = t.b;
  const int ts = min(NB, sj.ncols - s * NB);
  const int64_t ld = sj.nrows;
  float *D = Lx + sj.lx + (int64_t)(s * NB) * ld + s * NB;
  const int64_t g0 = sj.first + (int64_t)s * NB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float v[8][2];  // owners: column cn + 8 u at rows lane, lane + 32
  int cn = warp;
  if (warp < PR_OWNERS) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cc = warp + 8 * u, r = lane + 32 * h;
        v[u][h] = (cc < ts && r < ts && r >= cc) ? D[(int64_t)cc * ld + r] : 0.f;
      }
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r < ts) dd[r] = diag64(D[(int64_t)r * ld + r], axc, dpos, g0 + r);
    }
  }
  __syncthreads();
  for (int c = 0; c < ts; ++c) {
    if (warp < PR_OWNERS) {
      float p0 = 0.f, p1 = 0.f;  // column c - 1 at this lane's rows
      if (c > 0) {
        p0 = col[c - 1][lane];
        p1 = col[c - 1][lane + 32];
      }
      const bool own = cn == c;  // warp-uniform
      if (own) {
        double d = dd[c];
        if (c > 0) {
          const float l = col[c - 1][c];
          v[0][0] = fma(-p0, l, v[0][0]);
          v[0][1] = fma(-p1, l, v[0][1]);
          d = fma(-(double)l, (double)l, d);
        }
        if (!(d > 0.0)) {
          if (lane == 0) atomicMin(status, (long long)(g0 + c));
          d = 1.0;
        }
        if (lane == 0 && piv) piv[blockIdx.y * bt.piv + g0 + c] = d;
        const float df = (float)d;
        const float xf = rsqrt_newton(df);  // d x = sqrt(d)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = lane + 32 * h;
          col[c][r] = r == c ? df * xf : r > c ? v[0][h] * xf : 0.f;
        }
      }
      if (c > 0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int cc = cn + 8 * u;
          if ((u > 0 || !own) && cc < ts) {
            const float l = col[c - 1][cc];
            v[u][0] = fma(-p0, l, v[u][0]);
            v[u][1] = fma(-p1, l, v[u][1]);
          }
        }
      }
      if (own) {
#pragma unroll
        for (int u = 0; u < 7; ++u) {
          v[u][0] = v[u + 1][0];
          v[u][1] = v[u + 1][1];
        }
        v[7][0] = v[7][1] = 0.f;
        cn += 8;
      }
    } else if (c > 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        if (k > c && k < ts) {
          const float l = col[c - 1][k];
          dd[k] = fma(-(double)l, (double)l, dd[k]);
        }
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ts * ts; idx += PR_THREADS) {
    const int r = idx % ts, c = idx / ts;
    D[(int64_t)c * ld + r] = col[c][r];
  }
}

// (c'') Panel TRSM of full tiles with the tile in registers: thread (r, g) owns row r of the tile
// and the columns g, g + 4, ... (the oldest unfinished one in x[0]). Step c, one barrier: every
// thread applies the solved column c - 1 to its columns right of it, and the owners of column c
// publish X(:, c) = B(:, c) / L_cc. Same operations in the same order as k_trsm (bit-identical),
// without a shared-memory round trip per update. The number of columns a thread still updates
// selects a fully unrolled form, so no multiply-add is issued for a finished column (a predicated
// FP64 instruction would still take its pipe slot), and warps whose rows are all past the tile
// skip the arithmetic.
template <int N, typename T>
__device__ __forceinline__ void trsm_axpy(T (&x)[NB / 4], T xp, const T *lrow, int cn) {
#pragma unroll
  for (int u = 0; u < N; ++u) x[u] = fma(-xp, lrow[cn + 4 * u], x[u]);
}

template <typename T>
__global__ void __launch_bounds__(THREADS) k_trsm_r(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                    T *__restrict__ Lx, int64_t toff, const Batch bt) {
  static_assert(THREADS == 4 * NB, "four column groups of NB rows");
  Lx += blockIdx.y * bt.lx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*Ls)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);  // [col][row], lower triangle of L_ss
  T(*xs)[NB + 1] = Ls + NB;                                    // [col][row]: solved columns
  T *dinv = reinterpret_cast<T *>(xs + NB);
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int i = t.b, s = t.c;
  const int ts = min(NB, sj.ncols - s * NB);
  int64_t rb = d_row_tile_base(i, sj.ncols, sj.ncb);
  int tm = d_row_tile_rows(i, sj.ncols, sj.nrows, sj.ncb);
  const int half = t.d >> 16;  // 0: whole tile; 1, 2: its first or second 32 rows
  if (half) {
    rb += (half - 1) * (NB / 2);
    tm = max(0, min(NB / 2, tm - (half - 1) * (NB / 2)));
  }
  const int64_t ld = sj.nrows;
  const T *D = Lx + sj.lx + (int64_t)(s * NB) * ld + s * NB;
  T *B = Lx + sj.lx + (int64_t)(s * NB) * ld + rb;
  const int tid = threadIdx.x, r = tid & (NB - 1), g = tid >> 6;
  const bool live = (r & ~31) < tm;  // warp-uniform: some row of this warp is in the tile
  for (int idx = tid; idx < ts * ts; idx += THREADS) {
    const int rr = idx % ts, c = idx / ts;
    if (rr >= c) Ls[c][rr] = D[(int64_t)c * ld + rr];
  }
  T x[NB / 4];
  int cn = g;  // the column in x[0]
#pragma unroll
  for (int u = 0; u < NB / 4; ++u) {
    const int cc = g + 4 * u;
    x[u] = (r < tm && cc < ts) ? B[(int64_t)cc * ld + r] : T(0);
  }
  __syncthreads();
  if (tid < ts) dinv[tid] = T(1) / Ls[tid][tid];
  __syncthreads();
  for (int c = 0; c < ts; ++c) {
    if (c > 0 && live && cn < ts) {
      const T xp = xs[c - 1][r];
      const T *lrow = Ls[c - 1];
#define SYM_CASE(N)                      \
  case N:                                \
    trsm_axpy<N>(x, xp, lrow, cn);       \
    break;
      switch ((ts - cn + 3) >> 2) {  // columns cn, cn + 4, ... below ts (1..16)
        SYM_CASE(1) SYM_CASE(2) SYM_CASE(3) SYM_CASE(4) SYM_CASE(5) SYM_CASE(6) SYM_CASE(7) SYM_CASE(8)
        SYM_CASE(9) SYM_CASE(10) SYM_CASE(11) SYM_CASE(12) SYM_CASE(13) SYM_CASE(14) SYM_CASE(15) SYM_CASE(16)
        default:
          break;
      }
#undef SYM_CASE
    }
    if (cn == c) {  // uniform within a warp (its lanes share g)
      xs[c][r] = x[0] * dinv[c];
#pragma unroll
      for (int u = 0; u < NB / 4 - 1; ++u) x[u] = x[u + 1];
      x[NB / 4 - 1] = T(0);
      cn += 4;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < tm * ts; idx += THREADS) {
    const int rr = idx % tm, c = idx / tm;
    B[(int64_t)c * ld + rr] = xs[c][rr];
  }
}

// (c') Trailing update inside J: tile (i, j) -= tile (i, s) * tile (j, s)^T.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_gemm(const SNode *__restrict__ sn,
                                                  const Int4 *__restrict__ tasks,
                                                  T *__restrict__ Lx, int64_t toff, const Batch bt) {
  Lx += blockIdx.y * bt.lx;
  constexpr int KG = Chunk<T>::gemm;
  __shared__ T As[KG][NB];
  __shared__ T Bs[KG][NB];
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int i = t.b, j = t.c, s = t.d & 0xffff;
  int64_t rb = d_row_tile_base(i, sj.ncols, sj.ncb);
  int tm = d_row_tile_rows(i, sj.ncols, sj.nrows, sj.ncb);
  const int half = t.d >> 16;  // 0: whole tile; 1, 2: its first or second 32 rows
  if (half) {
    rb += (half - 1) * (NB / 2);
    tm = max(0, min(NB / 2, tm - (half - 1) * (NB / 2)));
  }
  const int tn = min(NB, sj.ncols - j * NB);
  const int ks = min(NB, sj.ncols - s * NB);
  const T *P = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows;  // column block s
  T *C = Lx + sj.lx + (int64_t)(j * NB) * sj.nrows + rb;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ni = tm > 32 ? 2 : 1;
  const int nj = tn > w ? (tn - w + 7) / 8 : 0;
  T r[2][8];
#pragma unroll
  for (int ii = 0; ii < 2; ++ii)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      int a = lane + 32 * ii, b = w + 8 * jj;
      r[ii][jj] = (a < tm && b < tn) ? C[(int64_t)b * sj.nrows + a] : T(0);
    }
  for (int k0 = 0; k0 < ks; k0 += KG) {
    const int kc = min(KG, ks - k0);
    for (int idx = tid; idx < KG * NB; idx += THREADS) {
      int a = idx % NB, kk = idx / NB;
      const T *col = P + (int64_t)(k0 + kk) * sj.nrows;
      As[kk][a] = (a < tm && kk < kc) ? col[rb + a] : T(0);
      Bs[kk][a] = (a < tn && kk < kc) ? col[(int64_t)j * NB + a] : T(0);
    }
    __syncthreads();
    fma_chunk_dispatch<KG>(r, As, Bs, kc, lane, w, ni, nj);
    __syncthreads();
  }
#pragma unroll
  for (int ii = 0; ii < 2; ++ii)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      int a = lane + 32 * ii, b = w + 8 * jj;
      if (a < tm && b < tn) C[(int64_t)b * sj.nrows + a] = r[ii][jj];
    }
}

// ---------------------------------------------------------------------------------------------
// Programmatic dependent launch (the solve's chain of short kernels). A kernel launched with the
// programmatic-serialization attribute may start once every CTA of the kernel before it in the
// stream has executed pdl_trigger(); it stages what does not depend on its predecessor (tasks,
// supernode records, tiles of L and of the inverses, all constant during a solve) and calls
// pdl_wait() — which returns once the predecessor has completed and its writes are visible —
// before it reads or writes y or t. Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Where a kernel lets its successor launch, by solve type (measured at 64^3, 4 right-hand sides).
// FP32 kernels are short: triggering at their start lets a chain of successors launch and stage
// their tiles ahead (refined mixed solve 29.7 -> 13.8 ms). FP64 kernels are long and bound by the
// FP64 pipe: successors launched that early crowd the SMs (13.3 ms against 10.7 without the
// attribute), while triggering once the dependency is met keeps one kernel ahead (8.6 ms).
template <typename V>
__device__ __forceinline__ void pdl_trigger_early() {
  if constexpr (sizeof(V) == 4) pdl_trigger();
}
template <typename V>
__device__ __forceinline__ void pdl_wait_then_trigger() {
  pdl_wait();
  if constexpr (sizeof(V) != 4) pdl_trigger();
}

// ---------------------------------------------------------------------------------------------
// Solve kernels. y is the permuted right-hand side block, n x nrhs, leading dimension n, of the
// vector type V (double for the FP64 path; float for the preconditioner of the mixed path). The
// factor is read in its storage type T and the arithmetic is done in V.
template <typename V>
__global__ void k_perm_in(const int32_t *__restrict__ perm, const double *__restrict__ B, int64_t ldb,
                          V *__restrict__ y, int64_t n, int nrhs, const Batch bt) {
  B += blockIdx.y * bt.b;
  y += blockIdx.y * bt.y;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n * nrhs; i += stride) {
    int64_t k = i % n, c = i / n;
    y[i] = (V)B[c * ldb + perm[k]];
  }
}
template <typename V>
__global__ void k_perm_out(const int32_t *__restrict__ perm, const V *__restrict__ y,
                           double *__restrict__ X, int64_t ldx, int64_t n, int nrhs, const Batch bt) {
  y += blockIdx.y * bt.y;
  X += blockIdx.y * bt.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n * nrhs; i += stride) {
    int64_t k = i % n, c = i / n;
    X[c * ldx + perm[k]] = (double)y[i];
  }
}

constexpr int MAXRHS = 8;  // right-hand sides handled per pass of the solve kernels
static_assert(MAXRHS == SOLVE_MAXRHS, "solve pass width");

// Runs STMT with the compile-time constant NR equal to the run-time count nr (1..MAXRHS).
#define SYM_NR_DISPATCH(nr, STMT)           \
  switch (nr) {                             \
    case 1: { constexpr int NR = 1; STMT; } break; \
    case 2: { constexpr int NR = 2; STMT; } break; \
    case 3: { constexpr int NR = 3; STMT; } break; \
    case 4: { constexpr int NR = 4; STMT; } break; \
    case 5: { constexpr int NR = 5; STMT; } break; \
    case 6: { constexpr int NR = 6; STMT; } break; \
    case 7: { constexpr int NR = 7; STMT; } break; \
    default: { constexpr int NR = 8; STMT; } break; \
  }
constexpr int BG = SOLVE_BG;  // columns per backward-gather CTA

// Forward gather: y(cols of tile bj of J) -= sum over descendant entries of L_K(rows) y_K.
// A thread-block cluster of cs CTAs shares one tile: CTA r takes entries r, r + cs, ...; rank 0
// adds the partial sums of all ranks in rank order through distributed shared memory, so the
// result does not depend on scheduling. Per entry the n rows of K's panel are read column by
// column (coalesced): thread t takes row t % nb and every groups-th column of K.
template <typename T, typename V>
__global__ void __launch_bounds__(THREADS) k_fgather(const SNode *__restrict__ sn,
                                                     const Int4 *__restrict__ tasks,
                                                     const UpdTask *__restrict__ utasks,
                                                     const UpdEntry *__restrict__ ents,
                                                     const int32_t *__restrict__ rel,
                                                     const T *__restrict__ Lx, V *__restrict__ y,
                                                     int64_t n, int r0, int nr, int64_t toff, const Batch bt) {
  Lx += blockIdx.y * bt.lx;
  y += blockIdx.y * bt.y;
  __shared__ V acc[MAXRHS][NB];
  __shared__ V part[THREADS][MAXRHS + 1];
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const Int4 t = tasks[toff + blockIdx.x / cs];
  const SNode sj = sn[t.a];
  const int bj = t.b;
  const UpdTask u = utasks[t.c];
  const int cb = bj * NB;
  const int tn = min(NB, sj.ncols - cb);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < MAXRHS * NB; idx += THREADS) acc[idx / NB][idx % NB] = V(0);
  __syncthreads();
  for (int64_t e = u.e0 + rank; e < u.e1; e += cs) {
    const UpdEntry E = ents[e];
    const SNode sk = sn[E.K];
    int nb = 1;
    while (nb < E.n) nb <<= 1;  // rows per group (power of two, <= NB)
    const int groups = THREADS / nb;
    const int b = tid & (nb - 1), kg = tid / nb;
    V s[MAXRHS];
#pragma unroll
    for (int q = 0; q < MAXRHS; ++q) s[q] = V(0);
    if (b < E.n) {
      const T *rowp = Lx + sk.lx + E.c_lo + b;
      const V *yk = y + (int64_t)r0 * n + sk.first;
      constexpr int U = 8;  // loads in flight per thread
      int k = kg;
      for (; k + (U - 1) * groups < sk.ncols; k += U * groups) {
        V l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) l[u] = (V)rowp[(int64_t)(k + u * groups) * sk.nrows];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int q = 0; q < MAXRHS; ++q)
            if (q < nr) s[q] = fma(l[u], yk[(int64_t)q * n + k + u * groups], s[q]);
      }
      for (; k < sk.ncols; k += groups) {
        const V l = (V)rowp[(int64_t)k * sk.nrows];
#pragma unroll
        for (int q = 0; q < MAXRHS; ++q)
          if (q < nr) s[q] = fma(l, yk[(int64_t)q * n + k], s[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < MAXRHS; ++q) part[tid][q] = s[q];
    __syncthreads();
    for (int idx = tid; idx < E.n * nr; idx += THREADS) {
      const int bb = idx % E.n, q = idx / E.n;
      V v = V(0);
      for (int g = 0; g < groups; ++g) v += part[g * nb + bb][q];
      acc[q][rel[E.relc + bb] - cb] += v;
    }
    __syncthreads();
  }
  cluster.sync();  // every rank's partial sums are complete
  if (rank == 0) {
    for (int idx = tid; idx < MAXRHS * NB; idx += THREADS) {
      const int r = idx % NB, c = idx / NB;
      if (r < tn && c < nr) {
        V v = acc[c][r];
        for (int o = 1; o < cs; ++o) v += cluster.map_shared_rank(&acc[0][0], o)[c * NB + r];
        y[(int64_t)(r0 + c) * n + sj.first + cb + r] -= v;
      }
    }
  }
  cluster.sync();  // keep the other ranks' shared memory alive until rank 0 has read it
}

// Forward push (the right-looking half of the forward solve, Sec. 3.1's y_rows -= L_off y_J
// written as a product per supernode): once the level's supernodes are solved, CTA {J, i, ch}
// forms t = L_J(rows of row tile i, columns of chunk ch) y_J(chunk) for a row tile below J's
// diagonal block and stores it at J's place in t. The panel is read once, column by column
// (64 consecutive rows: coalesced); y_J's chunk is staged in shared memory. NR right-hand sides
// are a template parameter so no multiply-add is issued for an absent one.
template <typename T, typename V, int NR>
__global__ void __launch_bounds__(THREADS) k_fpush(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                   const T *__restrict__ Lx, const V *__restrict__ y,
                                                   V *__restrict__ t, int64_t tsize, int64_t n, int r0,
                                                   int64_t toff, const Batch bt) {
  Lx += blockIdx.y * bt.lx;
  y += blockIdx.y * bt.y;
  t += blockIdx.y * bt.t;
  __shared__ V ys[NR][SOLVE_CW];  // reused for the partial sums [4][NR][NB] after the products
  pdl_trigger_early<V>();
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  const int64_t rb = d_row_tile_base(tk.b, sj.ncols, sj.ncb);
  const int tm = d_row_tile_rows(tk.b, sj.ncols, sj.nrows, sj.ncb);
  const int c0 = tk.c * SOLVE_CW, cw = min(SOLVE_CW, sj.ncols - c0);
  const int tid = threadIdx.x;
  pdl_wait_then_trigger<V>();  // y_J is the predecessor's output
  for (int idx = tid; idx < NR * SOLVE_CW; idx += THREADS) {
    const int c = idx % SOLVE_CW, q = idx / SOLVE_CW;
    ys[q][c] = c < cw ? y[(int64_t)(r0 + q) * n + sj.first + c0 + c] : V(0);
  }
  __syncthreads();
  const int r = tid & (NB - 1), g = tid >> 6;  // row r of the tile, columns g, g + 4, ...
  V acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = V(0);
  if (r < tm) {
    const T *col = Lx + sj.lx + (int64_t)c0 * sj.nrows + rb + r;
    constexpr int U = 8;  // loads in flight per thread
    int c = g;
    for (; c + 4 * (U - 1) < cw; c += 4 * U) {
      V l[U];
#pragma unroll
      for (int u = 0; u < U; ++u) l[u] = (V)col[(int64_t)(c + 4 * u) * sj.nrows];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = fma(l[u], ys[q][c + 4 * u], acc[q]);
    }
    for (; c < cw; c += 4) {
      const V l = (V)col[(int64_t)c * sj.nrows];
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] = fma(l, ys[q][c], acc[q]);
    }
  }
  __syncthreads();  // ys is reused below
  V *part = &ys[0][0];  // [g][q][r]: 4 * NR * NB <= NR * SOLVE_CW
#pragma unroll
  for (int q = 0; q < NR; ++q) part[(g * NR + q) * NB + r] = acc[q];
  __syncthreads();
  const int64_t base = sj.tx + (int64_t)tk.c * (sj.nrows - sj.ncols) + (rb - sj.ncols);
  for (int idx = tid; idx < NR * NB; idx += THREADS) {
    const int rr = idx % NB, q = idx / NB;
    if (rr < tm) {
      const V v = (part[(0 * NR + q) * NB + rr] + part[(1 * NR + q) * NB + rr]) +
                  (part[(2 * NR + q) * NB + rr] + part[(3 * NR + q) * NB + rr]);
      t[(int64_t)q * tsize + base + rr] = v;
    }
  }
}

// Forward sum: column g of J subtracts what its descendants pushed to row g, the entries of t
// named by its contribution list, added in list order (one thread per column).
template <typename V, int NR>
__global__ void __launch_bounds__(THREADS) k_fsum(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                  const int64_t *__restrict__ cptr, const int32_t *__restrict__ contrib,
                                                  const V *__restrict__ t, int64_t tsize, V *__restrict__ y,
                                                  int64_t n, int r0, int64_t toff, const Batch bt) {
  y += blockIdx.y * bt.y;
  t += blockIdx.y * bt.t;
  pdl_trigger_early<V>();
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  const int c = tk.b * 256 + threadIdx.x;
  pdl_wait_then_trigger<V>();  // t and y are the predecessors' output
  if (c >= sj.ncols) return;
  const int64_t gcol = sj.first + c;
  V acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = V(0);
#pragma unroll 4
  for (int64_t p = cptr[gcol]; p < cptr[gcol + 1]; ++p) {
    const int64_t e = contrib[p];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] += t[(int64_t)q * tsize + e];
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) y[(int64_t)(r0 + q) * n + gcol] -= acc[q];
}

// Backward gather: z(cols c0..c0+BG) -= L_J(rows below the diagonal block, cols)^T z(those rows).
// One CTA per BG-column slice. The rows are taken in chunks of 256: z at the chunk's rows is
// gathered once into shared memory, then each warp takes two columns, its lanes striding over the
// chunk's rows (coalesced panel reads), and a warp shuffle reduces each column at the end.
template <typename T, typename V, int NR>
__global__ void __launch_bounds__(THREADS) k_bgather(const SNode *__restrict__ sn,
                                                     const int32_t *__restrict__ rows,
                                                     const Int4 *__restrict__ tasks,
                                                     const T *__restrict__ Lx, V *__restrict__ y,
                                                     int64_t n, int r0, int64_t toff, const Batch bt) {
  static_assert(BG == 2 * (THREADS / 32), "two columns per warp");
  constexpr int RC = 256;
  Lx += blockIdx.y * bt.lx;
  y += blockIdx.y * bt.y;
  __shared__ V zg[NR][RC];
  pdl_trigger_early<V>();
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int c0 = t.b * BG;
  const int tn = min(BG, sj.ncols - c0);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int32_t *R = rows + sj.rowp;
  // columns w and w + 8 of the slice; an absent column reads column c0 (valid) and is not stored
  const int ca = w, cb = w + 8;
  const T *cola = Lx + sj.lx + (int64_t)(c0 + (ca < tn ? ca : 0)) * sj.nrows;
  const T *colb = Lx + sj.lx + (int64_t)(c0 + (cb < tn ? cb : 0)) * sj.nrows;
  V sa[NR], sb[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) sa[q] = sb[q] = V(0);
  pdl_wait_then_trigger<V>();  // z is the predecessor's output
  for (int rc0 = sj.ncols; rc0 < sj.nrows; rc0 += RC) {
    const int rc = min(RC, sj.nrows - rc0);
    for (int idx = tid; idx < NR * RC; idx += THREADS) {
      const int rr = idx % RC, q = idx / RC;
      if (rr < rc) zg[q][rr] = y[(int64_t)(r0 + q) * n + R[rc0 + rr]];
    }
    __syncthreads();
    if (cb < tn) {  // both columns of the warp (warp-uniform branches)
#pragma unroll 4
      for (int rr = lane; rr < rc; rr += 32) {
        const V la = (V)cola[rc0 + rr], lb = (V)colb[rc0 + rr];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const V z = zg[q][rr];
          sa[q] = fma(la, z, sa[q]);
          sb[q] = fma(lb, z, sb[q]);
        }
      }
    } else if (ca < tn) {  // slices of at most 8 columns: no work for an absent second column
#pragma unroll 4
      for (int rr = lane; rr < rc; rr += 32) {
        const V la = (V)cola[rc0 + rr];
#pragma unroll
        for (int q = 0; q < NR; ++q) sa[q] = fma(la, zg[q][rr], sa[q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    V va = sa[q], vb = sb[q];
    for (int o = 16; o > 0; o >>= 1) {
      va += __shfl_xor_sync(0xffffffffu, va, o);
      vb += __shfl_xor_sync(0xffffffffu, vb, o);
    }
    if (lane == 0) {
      if (ca < tn) y[(int64_t)(r0 + q) * n + sj.first + c0 + ca] -= va;
      if (cb < tn) y[(int64_t)(r0 + q) * n + sj.first + c0 + cb] -= vb;
    }
  }
}

// Shared-memory layout of the solve steps: the inverse of the diagonal tile and one panel tile,
// each [col][row] with padding, plus the right-hand-side tile before and after the diagonal solve.
template <typename V, int TB>
struct StepSmem {
  V Li[TB][TB + 1];
  V Lt[TB][TB + 1];
  V vs[MAXRHS][TB];
  V ys[MAXRHS][TB];
};
template <typename V, int TB>
constexpr size_t step_smem() { return sizeof(StepSmem<V, TB>); }

// Solves one diagonal tile u of J in place in global memory: y_u <- L_uu^{-1} y_u (forward) or
// z_u <- L_uu^{-T} z_u (backward), with the precomputed inverse staged in shared memory.
template <typename T, typename V, bool TRANS, int TB>
__device__ void write_solved_tile(StepSmem<V, TB> &S, const SNode &sj, const T *__restrict__ Linv, int u,
                                  V *__restrict__ y, int64_t n, int r0, int nr) {
  constexpr int TT = TileCfg<TB>::threads;
  const int tu = min(TB, sj.ncols - u * NB);
  const int64_t g0 = sj.first + u * NB;
  const int tid = threadIdx.x;
  __syncthreads();  // S may still be in use by the caller
  const T *Li = Linv + sj.dx + (int64_t)u * NB * NB;
  for (int idx = tid; idx < tu * tu; idx += TT) S.Li[idx / tu][idx % tu] = (V)Li[idx];
  pdl_wait_then_trigger<V>();
  for (int idx = tid; idx < MAXRHS * TB; idx += TT) {
    int r = idx % TB, c = idx / TB;
    S.vs[c][r] = (r < tu && c < nr) ? y[(int64_t)(r0 + c) * n + g0 + r] : V(0);
  }
  __syncthreads();
  for (int idx = tid; idx < tu * nr; idx += TT) {
    const int r = idx % tu, q = idx / tu;
    V a0 = V(0), a1 = V(0);
    if (!TRANS) {
      int k = 0;
      for (; k + 1 <= r; k += 2) {
        a0 = fma(S.Li[k][r], S.vs[q][k], a0);
        a1 = fma(S.Li[k + 1][r], S.vs[q][k + 1], a1);
      }
      if (k <= r) a0 = fma(S.Li[k][r], S.vs[q][k], a0);
    } else {
      int k = r;
      for (; k + 1 < tu; k += 2) {
        a0 = fma(S.Li[r][k], S.vs[q][k], a0);
        a1 = fma(S.Li[r][k + 1], S.vs[q][k + 1], a1);
      }
      if (k < tu) a0 = fma(S.Li[r][k], S.vs[q][k], a0);
    }
    y[(int64_t)(r0 + q) * n + g0 + r] = a0 + a1;
  }
}

// Forward step of column tile s inside J (tasks {J, i, s}). CTAs i > s read the not yet solved
// y_s, form ys = L_ss^{-1} y_s themselves from the precomputed inverse and apply
// y_i -= L_is ys. No CTA of this launch may overwrite y_s, so the solved values are written one
// step late: the CTA i = s writes the solved y_{s-1} (read by nobody now) and, for the last
// tile of J (no readers of y_s), the solved y_s as well. Tiles are staged in shared memory with
// all their loads in flight at once.
template <typename T, typename V, int TB>
__global__ void __launch_bounds__(TileCfg<TB>::threads) k_fstep(const SNode *__restrict__ sn,
                                                                const Int4 *__restrict__ tasks,
                                                                const T *__restrict__ Lx, const T *__restrict__ Linv,
                                                                V *__restrict__ y, int64_t n, int r0, int nr,
                                                                int64_t toff, const Batch bt) {
  constexpr int TT = TileCfg<TB>::threads;
  Lx += blockIdx.y * bt.lx;
  Linv += blockIdx.y * bt.dinv;
  y += blockIdx.y * bt.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem<V, TB> &S = *reinterpret_cast<StepSmem<V, TB> *>(smem_raw);
  pdl_trigger_early<V>();
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int i = t.b, s = t.c;
  if (i == s) {
    if (s >= 1) write_solved_tile<T, V, false, TB>(S, sj, Linv, s - 1, y, n, r0, nr);
    if (s == sj.ncb - 1) write_solved_tile<T, V, false, TB>(S, sj, Linv, s, y, n, r0, nr);
    return;
  }
  const int ts = min(TB, sj.ncols - s * NB);  // a TB < NB launch holds supernodes of <= TB columns
  const int tm = min(TB, sj.ncols - i * NB);
  const int64_t g0 = sj.first + s * NB;
  const int tid = threadIdx.x;
  const T *Li = Linv + sj.dx + (int64_t)s * NB * NB;                  // ts x ts, column-major, lower
  const T *Lt = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + i * NB;  // rows of tile i, cols of tile s
  for (int idx = tid; idx < ts * ts; idx += TT) S.Li[idx / ts][idx % ts] = (V)Li[idx];
  for (int idx = tid; idx < TB * ts; idx += TT) {
    const int r = idx % TB, c = idx / TB;
    if (r < tm) S.Lt[c][r] = (V)Lt[(int64_t)c * sj.nrows + r];
  }
  pdl_wait_then_trigger<V>();  // y is the predecessor's output
  for (int idx = tid; idx < MAXRHS * TB; idx += TT) {
    int r = idx % TB, c = idx / TB;
    S.vs[c][r] = (r < ts && c < nr) ? y[(int64_t)(r0 + c) * n + g0 + r] : V(0);
  }
  __syncthreads();
  for (int idx = tid; idx < ts * nr; idx += TT) {
    const int r = idx % ts, q = idx / ts;
    V a0 = V(0), a1 = V(0);
    int k = 0;
    for (; k + 1 <= r; k += 2) {
      a0 = fma(S.Li[k][r], S.vs[q][k], a0);
      a1 = fma(S.Li[k + 1][r], S.vs[q][k + 1], a1);
    }
    if (k <= r) a0 = fma(S.Li[k][r], S.vs[q][k], a0);
    S.ys[q][r] = a0 + a1;
  }
  __syncthreads();
  for (int idx = tid; idx < tm * nr; idx += TT) {
    const int r = idx % tm, q = idx / tm;
    V a0 = V(0), a1 = V(0);
    int k = 0;
    for (; k + 1 < ts; k += 2) {
      a0 = fma(S.Lt[k][r], S.ys[q][k], a0);
      a1 = fma(S.Lt[k + 1][r], S.ys[q][k + 1], a1);
    }
    if (k < ts) a0 = fma(S.Lt[k][r], S.ys[q][k], a0);
    y[(int64_t)(r0 + q) * n + sj.first + i * NB + r] -= a0 + a1;
  }
}

// Backward step of column tile s inside J (tasks {J, i, s}, s descending): CTAs i < s form
// zs = L_ss^{-T} z_s and apply z_i -= L_si^T zs; the CTA i = s writes the solved z_{s+1} and,
// for tile 0, the solved z_0 (the mirror image of the forward step). Launched for supernodes of
// at most SMALL_TILE columns; wider ones take the cluster form (k_step_c).
template <typename T, typename V, int TB>
__global__ void __launch_bounds__(TileCfg<TB>::threads) k_bstep(const SNode *__restrict__ sn,
                                                                const Int4 *__restrict__ tasks,
                                                                const T *__restrict__ Lx, const T *__restrict__ Linv,
                                                                V *__restrict__ y, int64_t n, int r0, int nr,
                                                                int64_t toff, const Batch bt) {
  constexpr int TT = TileCfg<TB>::threads;
  Lx += blockIdx.y * bt.lx;
  Linv += blockIdx.y * bt.dinv;
  y += blockIdx.y * bt.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem<V, TB> &S = *reinterpret_cast<StepSmem<V, TB> *>(smem_raw);
  pdl_trigger_early<V>();
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int i = t.b, s = t.c;
  if (i == s) {
    if (s + 1 < sj.ncb) write_solved_tile<T, V, true, TB>(S, sj, Linv, s + 1, y, n, r0, nr);
    if (s == 0) write_solved_tile<T, V, true, TB>(S, sj, Linv, 0, y, n, r0, nr);
    return;
  }
  const int ts = min(TB, sj.ncols - s * NB);  // a TB < NB launch holds supernodes of <= TB columns
  const int ti = min(TB, sj.ncols - i * NB);
  const int64_t g0 = sj.first + s * NB;
  const int tid = threadIdx.x;
  const T *Li = Linv + sj.dx + (int64_t)s * NB * NB;                  // ts x ts, column-major, lower
  const T *Lt = Lx + sj.lx + (int64_t)(i * NB) * sj.nrows + s * NB;  // rows of tile s, cols of tile i
  for (int idx = tid; idx < ts * ts; idx += TT) S.Li[idx / ts][idx % ts] = (V)Li[idx];
  for (int idx = tid; idx < TB * ti; idx += TT) {
    const int k = idx % TB, c = idx / TB;
    if (k < ts) S.Lt[c][k] = (V)Lt[(int64_t)c * sj.nrows + k];
  }
  pdl_wait_then_trigger<V>();  // y is the predecessor's output
  for (int idx = tid; idx < MAXRHS * TB; idx += TT) {
    int r = idx % TB, c = idx / TB;
    S.vs[c][r] = (r < ts && c < nr) ? y[(int64_t)(r0 + c) * n + g0 + r] : V(0);
  }
  __syncthreads();
  for (int idx = tid; idx < ts * nr; idx += TT) {
    const int r = idx % ts, q = idx / ts;
    V a0 = V(0), a1 = V(0);
    int k = r;
    for (; k + 1 < ts; k += 2) {  // (L^-1)(k, r) for k >= r
      a0 = fma(S.Li[r][k], S.vs[q][k], a0);
      a1 = fma(S.Li[r][k + 1], S.vs[q][k + 1], a1);
    }
    if (k < ts) a0 = fma(S.Li[r][k], S.vs[q][k], a0);
    S.ys[q][r] = a0 + a1;
  }
  __syncthreads();
  for (int idx = tid; idx < ti * nr; idx += TT) {
    const int c = idx % ti, q = idx / ti;
    V a0 = V(0), a1 = V(0);
    int k = 0;
    for (; k + 1 < ts; k += 2) {
      a0 = fma(S.Lt[c][k], S.ys[q][k], a0);
      a1 = fma(S.Lt[c][k + 1], S.ys[q][k + 1], a1);
    }
    if (k < ts) a0 = fma(S.Lt[c][k], S.ys[q][k], a0);
    y[(int64_t)(r0 + q) * n + sj.first + i * NB + c] -= a0 + a1;
  }
}

// Cluster forms of the solve steps (tiles of up to NB columns). A task {J, i, s} runs on a
// thread-block cluster of four CTAs; CTA q of the cluster owns the 16 rows (forward) or columns
// (backward) 16 q .. 16 q + 15 of tile i. Forward, launch s (s = -1 .. ncb - 2):
//   every task applies the solved tile s (if s >= 0) to its rows: y_i -= L_is y_s;
//   the task i = s + 1 then solves its tile in place, y_i <- L_ii^{-1} y_i, each CTA taking its
//   16 rows of the inverse and the whole updated tile, gathered from the four CTAs through
//   distributed shared memory.
// Backward, launch s (s = ncb .. 1): z_i -= L_si^T z_s (s < ncb), and the task i = s - 1 solves
// z_i <- L_ii^{-T} z_i. So the tile a step solves is written once, already solved, and read by
// the next launch only: no CTA applies the inverse of another tile, and the critical path of a
// step is one quarter tile's update plus one quarter of its solve.
constexpr int QR = 16;  // rows (or columns) per CTA of a cluster task

template <typename V, int NR>
struct StepCSmem {
  V L[NB][QR + 1];     // [k][row]: this CTA's rows of L_is (forward) or L_si^T (backward)
  V I[NB][QR + 1];     // [k][row]: this CTA's rows of L_ii^{-1} (forward) or of L_ii^{-T}
  V ys[NR][NB];        // the solved tile s
  V yq[NR][QR];        // this CTA's rows of tile i after the update (read by the cluster)
  V yf[NR][NB];        // the whole updated tile i (solving tasks)
};

// 16-lane sum (lanes l and l ^ 8, ^4, ^2, ^1 are partners; lane g of each 16 holds part g).
template <typename V>
__device__ __forceinline__ V sum16(V v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, typename V, int NR, bool FWD>
__global__ void __launch_bounds__(THREADS) k_step_c(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                    const T *__restrict__ Lx, const T *__restrict__ Linv,
                                                    V *__restrict__ y, int64_t n, int r0, int64_t toff,
                                                    const Batch bt) {
  Lx += blockIdx.y * bt.lx;
  Linv += blockIdx.y * bt.dinv;
  y += blockIdx.y * bt.y;
  __shared__ StepCSmem<V, NR> S;
  cg::cluster_group cluster = cg::this_cluster();
  pdl_trigger_early<V>();
  const int q = (int)cluster.block_rank();
  const Int4 t = tasks[toff + blockIdx.x / 4];
  const SNode sj = sn[t.a];
  const int i = t.b, s = t.c;
  const int ti = min(NB, sj.ncols - i * NB);
  const bool has_s = FWD ? s >= 0 : s < sj.ncb;
  const int ts = has_s ? min(NB, sj.ncols - s * NB) : 0;
  const bool solves = FWD ? i == s + 1 : i == s - 1;
  const int o0 = QR * q, rq = max(0, min(QR, ti - o0));  // this CTA's rows (columns) of tile i
  const int tid = threadIdx.x, o = tid >> 4, g = tid & 15;  // output o, k-group g (k = g + 16 j)
  const int64_t gi = sj.first + (int64_t)i * NB, gs = sj.first + (int64_t)s * NB;
  // Stage what does not depend on the previous launch: the rows of L and of the inverse.
  if (has_s) {
    for (int idx = tid; idx < QR * ts; idx += THREADS) {
      int r, k;
      const T *src;
      if (FWD) {  // L_is(o0 + r, k): for fixed k, 16 consecutive rows of column s NB + k
        r = idx % QR, k = idx / QR;
        src = Lx + sj.lx + (int64_t)(s * NB + k) * sj.nrows + i * NB + o0 + r;
      } else {    // L_si(k, o0 + r): for fixed r, consecutive k of column i NB + o0 + r
        k = idx % ts, r = idx / ts;
        src = Lx + sj.lx + (int64_t)(i * NB + o0 + r) * sj.nrows + s * NB + k;
      }
      S.L[k][r] = r < rq ? (V)*src : V(0);
    }
  }
  if (solves) {
    const T *Li = Linv + sj.dx + (int64_t)i * NB * NB;  // ti x ti, column-major, lower
    for (int idx = tid; idx < QR * ti; idx += THREADS) {
      int r, k;
      V v;
      if (FWD) {  // (L^-1)(o0 + r, k)
        r = idx % QR, k = idx / QR;
        v = r < rq ? (V)Li[(int64_t)k * ti + o0 + r] : V(0);
      } else {    // (L^-T)(o0 + r, k) = (L^-1)(k, o0 + r)
        k = idx % ti, r = idx / ti;
        v = r < rq ? (V)Li[(int64_t)(o0 + r) * ti + k] : V(0);
      }
      S.I[k][r] = v;
    }
  }
  pdl_wait_then_trigger<V>();  // y is the predecessor's output
  for (int idx = tid; idx < NR * NB; idx += THREADS) {
    const int k = idx % NB, c = idx / NB;
    if (has_s && k < ts) S.ys[c][k] = y[(int64_t)(r0 + c) * n + gs + k];
  }
  __syncthreads();
  // y_i(o) -= sum_k L(o, k) ys(k) for this CTA's outputs o: 16 lanes per output split k.
  V acc[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = V(0);
  if (o < QR) {
    for (int k = g; k < ts; k += 16) {
      const V l = S.L[k][o];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = fma(l, S.ys[c][k], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = sum16(acc[c]);
  if (g == 0 && o < rq) {
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const int64_t at = (int64_t)(r0 + c) * n + gi + o0 + o;
      const V v = y[at] - acc[c];
      if (solves) S.yq[c][o] = v;
      else y[at] = v;
    }
  }
  if (!solves) return;  // (uniform across the cluster: its four CTAs share the task)
  cluster.sync();       // every quarter of the updated tile is in its CTA's shared memory
  for (int idx = tid; idx < NR * ti; idx += THREADS) {
    const int k = idx % ti, c = idx / ti;
    const V *rem = cluster.map_shared_rank(&S.yq[0][0], k / QR);
    S.yf[c][k] = rem[c * QR + k % QR];
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = V(0);
  if (o < QR) {
    const int lo = FWD ? 0 : o0 + o, hi = FWD ? o0 + o + 1 : ti;  // the inverse's nonzeros
    for (int k = lo + ((g - lo) & 15); k < hi; k += 16) {
      const V l = S.I[k][o];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = fma(l, S.yf[c][k], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = sum16(acc[c]);
  if (g == 0 && o < rq) {
#pragma unroll
    for (int c = 0; c < NR; ++c) y[(int64_t)(r0 + c) * n + gi + o0 + o] = acc[c];
  }
  cluster.sync();  // keep this CTA's quarter alive until the others have read it
}

// Inverse of diagonal tile s of J (in FP64 from the factored tile), stored column-major ts x ts
// at Linv + dx + s NB^2. Solves L X = I row by row of X: row c is final once scaled by
// 1 / L(c, c); it is then eliminated from the rows below.
template <typename T, int TB>
__global__ void __launch_bounds__(TileCfg<TB>::threads) k_trtri(const SNode *__restrict__ sn,
                                                                const Int4 *__restrict__ tasks,
                                                                const T *__restrict__ Lx, T *__restrict__ Linv,
                                                                int64_t toff, const Batch bt) {
  constexpr int TT = TileCfg<TB>::threads, G = TT / TB;  // G column groups of TB rows
  Lx += blockIdx.y * bt.lx;
  Linv += blockIdx.y * bt.dinv;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double(*a)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(smem_raw);  // L, [col][row]
  double(*x)[TB + 1] = a + TB;                                          // X, [col][row]
  double *dinv = reinterpret_cast<double *>(smem_raw) + 2 * TB * (TB + 1);
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int s = t.b;
  const int ts = min(TB, sj.ncols - s * NB);  // a TB < NB launch holds tiles of order <= TB
  const T *D = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + s * NB;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < ts * ts; idx += TT) {
    int r = idx % ts, c = idx / ts;
    a[c][r] = r >= c ? (double)D[(int64_t)c * sj.nrows + r] : 0.0;
    x[c][r] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid < ts) dinv[tid] = 1.0 / a[tid][tid];
  __syncthreads();
  if (tid == 0 && ts > 0) x[0][0] *= dinv[0];  // row 0 is final
  __syncthreads();
  // Step c: row c of X is final and scaled; the rows below subtract l(r, c) times it, and row
  // c + 1, now final, is scaled by 1 / L(c+1, c+1) by the threads that updated it. Each element
  // gets the operations (and roundings) of an elimination that scales row c as it is used.
  const int r = tid % TB, jg = tid / TB;
  for (int c = 0; c + 1 < ts; ++c) {
    if (r > c && r < ts) {
      const double l = a[c][r];
      const double sc = r == c + 1 ? dinv[r] : 1.0;
      for (int j = jg; j <= c; j += G) {
        const double v = fma(-l, x[j][c], x[j][r]);
        x[j][r] = r == c + 1 ? v * sc : v;
      }
      if (r == c + 1 && jg == (c + 1) % G) x[r][r] *= sc;
    }
    __syncthreads();
  }
  T *out = Linv + sj.dx + (int64_t)s * NB * NB;
  for (int idx = tid; idx < ts * ts; idx += TT) {
    const int rr = idx % ts, c = idx / ts;
    out[(int64_t)c * ts + rr] = rr >= c ? (T)x[c][rr] : T(0);
  }
}

// (e) Warp-per-tile forms of POTRF and TRTRI for launches whose diagonal tiles all have order
// <= 32 (leaves of the supernodal tree, small matrices, batches of them). One warp owns one tile,
// WT_WARPS tiles per CTA; the lower triangles sit packed in shared memory and the work of each
// column step is mapped flat onto the lanes (the (row, column) pairs it updates), so that one
// warp-wide FP64 instruction carries up to 32 useful operations — on this part it occupies the
// FP64 pipe of its sub-partition for the same time with 3 active lanes as with 32 — and no
// CTA-wide barrier is needed. Every element sees the operations of k_potrf / k_trtri in the
// same order: the results are bit-identical to the one-tile-per-CTA forms.
constexpr int WT_WARPS = 4;
constexpr int WT_PACK = SMALL_TILE * (SMALL_TILE + 1) / 2;  // packed lower triangle of order 32

// Column-major packed lower triangle of order ts: element (r, c), r >= c.
__device__ __forceinline__ int pk(int ts, int c, int r) { return c * (2 * ts - c + 1) / 2 + (r - c); }

// Row-major enumeration of a lower triangle: el = a (a + 1) / 2 + b with b <= a.
__device__ __forceinline__ void tri_decode(int el, int &a, int &b) {
  a = (int)((sqrtf(8.0f * el + 1.0f) - 1.0f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= el) ++a;
  while (a * (a + 1) / 2 > el) --a;
  b = el - a * (a + 1) / 2;
}

// External update of small tiles in a batch: one warp per (tile, matrix), the same tile of
// WT_WARPS consecutive matrices per CTA, each warp's tile in its own shared memory. A batch's small
// supernodes give entries of a few dozen elements; in the one-CTA-per-tile form most of the
// CTA's warps sit idle behind its barriers. Here a warp's lanes take an entry's elements (lower
// triangle only on diagonal tiles) and run their sums over ncols(K) with operands read through
// L1; no barrier wider than the warp. Deterministic: entries in order, k ascending.
template <typename T>
__global__ void __launch_bounds__(32 * WT_WARPS) k_update_wb(const SNode *__restrict__ sn,
                                                             const UpdTask *__restrict__ tasks,
                                                             const UpdEntry *__restrict__ ents,
                                                             const int32_t *__restrict__ rel, T *__restrict__ Lx,
                                                             int64_t toff, int32_t nmat, const Batch bt) {
  __shared__ T acc[WT_WARPS][SMALL_TILE][SMALL_TILE + 1];  // [col][row] per warp
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t mat = blockIdx.y * WT_WARPS + w;
  if (mat >= nmat) return;  // warp-uniform; only warp-level synchronization below
  Lx += (int64_t)mat * bt.lx;
  const UpdTask t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.J];
  const int64_t rb = d_row_tile_base(t.bi, sj.ncols, sj.ncb);
  const int tm = d_row_tile_rows(t.bi, sj.ncols, sj.nrows, sj.ncb);
  const int cb = t.bj * NB;
  const int tn = min(NB, sj.ncols - cb);
  const bool diag = t.bi == t.bj;
  T(*A)[SMALL_TILE + 1] = acc[w];
  T *C = Lx + sj.lx + (int64_t)cb * sj.nrows + rb;
  for (int idx = lane; idx < tm * tn; idx += 32) {
    const int r = idx % tm, c = idx / tm;
    A[c][r] = C[(int64_t)c * sj.nrows + r];
  }
  __syncwarp();
  for (int64_t e = t.e0; e < t.e1; ++e) {
    const UpdEntry E = ents[e];
    const SNode sk = sn[E.K];
    const int64_t ld = sk.nrows;
    const int cnt = diag ? E.m * (E.m + 1) / 2 : E.m * E.n;
    for (int el = lane; el < cnt; el += 32) {
      int a, b;
      if (diag) tri_decode(el, a, b);
      else a = el % E.m, b = el / E.m;
      const int pr = rel[E.relr + a] - (int)rb, pc = rel[E.relc + b] - cb;
      const T *pa = Lx + sk.lx + E.r_lo + a, *pb = Lx + sk.lx + E.c_lo + b;
      T r = A[pc][pr];
#pragma unroll 4
      for (int k = 0; k < sk.ncols; ++k) r = fma(-pa[k * ld], pb[k * ld], r);
      A[pc][pr] = r;
    }
    __syncwarp();
  }
  for (int idx = lane; idx < tm * tn; idx += 32) {
    const int r = idx % tm, c = idx / tm;
    C[(int64_t)c * sj.nrows + r] = A[c][r];
  }
}

// The same for tiles of any size (batches): one warp per (tile, matrix), each element of an entry
// read, updated and written back in global memory by one lane (the tile is not staged: a 64 x 64
// accumulator per warp would leave room for few warps). The entries of a tile are applied in
// order, k ascending, as in every other form (bit-identical results); __syncwarp orders one
// entry's writes before the next entry's reads of the same elements.
template <typename T>
__global__ void __launch_bounds__(32 * WT_WARPS) k_update_wg(const SNode *__restrict__ sn,
                                                             const UpdTask *__restrict__ tasks,
                                                             const UpdEntry *__restrict__ ents,
                                                             const int32_t *__restrict__ rel, T *__restrict__ Lx,
                                                             int64_t toff, int32_t nmat, const Batch bt) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t mat = blockIdx.y * WT_WARPS + w;
  if (mat >= nmat) return;  // warp-uniform; only warp-level synchronization below
  Lx += (int64_t)mat * bt.lx;
  const UpdTask t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.J];
  const int64_t rb = d_row_tile_base(t.bi, sj.ncols, sj.ncb);
  const int cb = t.bj * NB;
  const bool diag = t.bi == t.bj;
  T *C = Lx + sj.lx + (int64_t)cb * sj.nrows + rb;
  for (int64_t e = t.e0; e < t.e1; ++e) {
    const UpdEntry E = ents[e];
    const SNode sk = sn[E.K];
    const int64_t ld = sk.nrows;
    const int cnt = diag ? E.m * (E.m + 1) / 2 : E.m * E.n;
    for (int el = lane; el < cnt; el += 32) {
      int a, b;
      if (diag) tri_decode(el, a, b);
      else a = el % E.m, b = el / E.m;
      const int pr = rel[E.relr + a] - (int)rb, pc = rel[E.relc + b] - cb;
      const T *pa = Lx + sk.lx + E.r_lo + a, *pb = Lx + sk.lx + E.c_lo + b;
      T *cp = C + (int64_t)pc * sj.nrows + pr;
      T r = *cp;
#pragma unroll 4
      for (int k = 0; k < sk.ncols; ++k) r = fma(-pa[k * ld], pb[k * ld], r);
      *cp = r;
    }
    __syncwarp();
  }
}

// Lanes l of a warp with l % MW < nm (the lanes of the warp's nm matrices).
__device__ __forceinline__ unsigned present_lanes(int MW, int nm) {
  unsigned mask = 0;
  for (int l = 0; l < 32; ++l)
    if ((l & (MW - 1)) < nm) mask |= 1u << l;
  return mask;
}

// The same for a batch with lanes mapped to matrices (tiles of any size, updated in global
// memory): one warp per (tile, MW = 32 / G matrices), WT_WARPS matrix groups per CTA; lane
// q * MW + m takes the elements q, q + G, ... of every entry for matrix m (consecutive elements
// are consecutive rows, so the G lanes of a matrix read neighbouring operands). The small-tile
// levels of a batch have entries of a few dozen elements and tiles of a few entries; a warp per
// (tile, matrix) leaves most lanes idle and spends its time on latency. Element by element the
// operations of k_update_wb and k_update_wg, in their order (bit-identical).
template <typename T, int G>
__global__ void __launch_bounds__(32 * WT_WARPS) k_update_mb(const SNode *__restrict__ sn,
                                                             const UpdTask *__restrict__ tasks,
                                                             const UpdEntry *__restrict__ ents,
                                                             const int32_t *__restrict__ rel, T *__restrict__ Lx,
                                                             int64_t toff, int32_t nmat, const Batch bt) {
  constexpr int MW = 32 / G;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, m = lane & (MW - 1), q = lane / MW;
  const int32_t mat0 = (blockIdx.y * WT_WARPS + w) * MW;
  if (mat0 + m >= nmat) return;  // lanes of absent matrices leave; the barriers name the others
  const unsigned mask = present_lanes(MW, nmat - mat0);
  Lx += (int64_t)(mat0 + m) * bt.lx;
  const UpdTask t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.J];
  const int64_t rb = d_row_tile_base(t.bi, sj.ncols, sj.ncb);
  const int cb = t.bj * NB;
  const bool diag = t.bi == t.bj;
  T *C = Lx + sj.lx + (int64_t)cb * sj.nrows + rb;
  for (int64_t e = t.e0; e < t.e1; ++e) {
    const UpdEntry E = ents[e];
    const SNode sk = sn[E.K];
    const int64_t ld = sk.nrows;
    const int cnt = diag ? E.m * (E.m + 1) / 2 : E.m * E.n;
    for (int el = q; el < cnt; el += G) {
      int a, b;
      if (diag) tri_decode(el, a, b);
      else a = el % E.m, b = el / E.m;
      const int pr = rel[E.relr + a] - (int)rb, pc = rel[E.relc + b] - cb;
      const T *pa = Lx + sk.lx + E.r_lo + a, *pb = Lx + sk.lx + E.c_lo + b;
      T *cp = C + (int64_t)pc * sj.nrows + pr;
      T r = *cp;
#pragma unroll 4
      for (int k = 0; k < sk.ncols; ++k) r = fma(-pa[k * ld], pb[k * ld], r);
      *cp = r;
    }
    __syncwarp(mask);  // an entry's writes before the next entry's reads of the same elements
  }
}

// TRSM of a batch's narrow tiles (ts <= SMALL_TILE columns, <= NB rows): one warp per (tile,
// matrix), four matrices per CTA, each warp's L_ss and 32-row chunk of the tile in its own shared
// memory. Within a chunk the rows are spread over 32 / rows column groups as in k_trsm and each
// element sees k_trsm's operations in the same order (bit-identical); warp barriers only.
template <typename T>
constexpr size_t trsm_w_smem() { return (size_t)WT_WARPS * sizeof(T) * (2 * SMALL_TILE * (SMALL_TILE + 1) + SMALL_TILE); }

template <typename T>
__global__ void __launch_bounds__(32 * WT_WARPS) k_trsm_w(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                          T *__restrict__ Lx, int64_t toff, int32_t nmat,
                                                          const Batch bt) {
  constexpr int TW = SMALL_TILE, PW = 2 * TW * (TW + 1) + TW;  // per warp: Ls, X, dinv
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t mat = blockIdx.y * WT_WARPS + w;
  if (mat >= nmat) return;  // warp-uniform; only warp-level synchronization below
  T(*Ls)[TW + 1] = reinterpret_cast<T(*)[TW + 1]>(reinterpret_cast<T *>(smem_raw) + w * PW);  // [col][row]
  T(*X)[TW + 1] = Ls + TW;                                                                    // [col][row]
  T *dinv = reinterpret_cast<T *>(X + TW);
  Lx += (int64_t)mat * bt.lx;
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int i = t.b, s = t.c;
  const int ts = min(TW, sj.ncols - s * NB);
  int64_t rb = d_row_tile_base(i, sj.ncols, sj.ncb);
  int tm = d_row_tile_rows(i, sj.ncols, sj.nrows, sj.ncb);
  const int half = t.d >> 16;  // 0: whole tile; 1, 2: its first or second 32 rows
  if (half) {
    rb += (half - 1) * (NB / 2);
    tm = max(0, min(NB / 2, tm - (half - 1) * (NB / 2)));
  }
  const T *D = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + s * NB;
  for (int idx = lane; idx < ts * ts; idx += 32) {
    const int r = idx % ts, c = idx / ts;
    if (r >= c) Ls[c][r] = D[(int64_t)c * sj.nrows + r];
  }
  __syncwarp();
  if (lane < ts) dinv[lane] = T(1) / Ls[lane][lane];
  for (int r0 = 0; r0 < tm; r0 += 32) {
    const int cm = min(32, tm - r0);  // rows of this chunk
    T *B = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + rb + r0;
    __syncwarp();
    for (int idx = lane; idx < cm * ts; idx += 32) {
      const int r = idx % cm, c = idx / cm;
      X[c][r] = B[(int64_t)c * sj.nrows + r];
    }
    __syncwarp();
    const int GR = 32 / cm, r = lane % cm, g = lane / cm;  // g >= GR: idle
    for (int c = 0; c < ts; ++c) {
      if (g < GR) {
        const T xc = X[c][r] * dinv[c];  // X(r, c) is final once columns < c are applied
        for (int cc = c + 1 + g; cc < ts; cc += GR) X[cc][r] = fma(-xc, Ls[c][cc], X[cc][r]);
      }
      __syncwarp();
      if (g == 0) X[c][r] *= dinv[c];
    }
    __syncwarp();
    for (int idx = lane; idx < cm * ts; idx += 32) {
      const int rr = idx % cm, c = idx / cm;
      B[(int64_t)c * sj.nrows + rr] = X[c][rr];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * WT_WARPS) k_potrf_w(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                           int64_t ntask, T *__restrict__ Lx, long long *status,
                                                           double *__restrict__ piv, const double *__restrict__ axc,
                                                           const int64_t *__restrict__ dpos, int64_t toff,
                                                           const Batch bt) {
  constexpr bool F64PIV = std::is_same<T, float>::value;  // FP64 pivot chain of FP32 factors (k_potrf)
  Lx += blockIdx.y * bt.lx;
  status += blockIdx.y;
  __shared__ T tri[WT_WARPS][WT_PACK];
  __shared__ double ddw[WT_WARPS][F64PIV ? SMALL_TILE : 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t task = (int64_t)blockIdx.x * WT_WARPS + w;
  if (task >= ntask) return;  // warp-uniform; only warp-level synchronization below
  const Int4 t = tasks[toff + task];
  const SNode sj = sn[t.a];
  const int s = t.b;
  const int ts = min(SMALL_TILE, sj.ncols - s * NB);
  T *D = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + s * NB;
  T *a = tri[w];
  double *dd = ddw[w];
  if (axc) axc += blockIdx.y * bt.nnz;
  for (int c = 0; c < ts; ++c)
    if (lane >= c && lane < ts) {
      const T v = D[(int64_t)c * sj.nrows + lane];
      a[pk(ts, c, lane)] = v;
      if (F64PIV && lane == c) dd[c] = diag64((float)v, axc, dpos, sj.first + s * NB + c);
    }
  __syncwarp();
  for (int c = 0; c < ts; ++c) {
    if constexpr (F64PIV) {  // FP64 pivot, FP32 reciprocal square root (as in k_potrf)
      double d = dd[c];
      if (!(d > 0.0)) {
        if (lane == 0) atomicMin(status, (long long)(sj.first + s * NB + c));
        d = 1.0;
      }
      if (lane == 0 && piv) piv[blockIdx.y * bt.piv + sj.first + s * NB + c] = d;
      const float df = (float)d;
      const float xf = rsqrt_newton(df);
      __syncwarp();  // every lane has read the pivot
      if (lane >= c && lane < ts) a[pk(ts, c, lane)] = lane == c ? (T)(df * xf) : a[pk(ts, c, lane)] * xf;
    } else {
      T d = a[pk(ts, c, c)];
      if (!(d > T(0))) {
        if (lane == 0) atomicMin(status, (long long)(sj.first + s * NB + c));
        d = T(1);
      }
      const T x = rsqrt_of(d);
      __syncwarp();  // every lane has read the pivot
      if (lane >= c && lane < ts) a[pk(ts, c, lane)] = lane == c ? d * x : a[pk(ts, c, lane)] * x;
    }
    __syncwarp();
    const int m = ts - 1 - c;  // trailing triangle: rows and columns c+1 .. ts-1
    if (F64PIV && lane >= c + 1 && lane < ts)  // the FP64 diagonal, one lane per trailing column
      dd[lane] = fma(-(double)a[pk(ts, c, lane)], (double)a[pk(ts, c, lane)], dd[lane]);
    for (int el = lane; el < m * (m + 1) / 2; el += 32) {
      int ia, ib;
      tri_decode(el, ia, ib);
      const int rr = c + 1 + ia, cc = c + 1 + ib;
      if (!F64PIV || rr != cc) a[pk(ts, cc, rr)] = fma(-a[pk(ts, c, rr)], a[pk(ts, c, cc)], a[pk(ts, cc, rr)]);
    }
    __syncwarp();
  }
  for (int c = 0; c < ts; ++c)
    if (lane < ts) D[(int64_t)c * sj.nrows + lane] = lane >= c ? a[pk(ts, c, lane)] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(32 * WT_WARPS) k_trtri_w(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                           int64_t ntask, const T *__restrict__ Lx,
                                                           T *__restrict__ Linv, int64_t toff, const Batch bt) {
  Lx += blockIdx.y * bt.lx;
  Linv += blockIdx.y * bt.dinv;
  __shared__ double la[WT_WARPS][WT_PACK], lxv[WT_WARPS][WT_PACK], dv[WT_WARPS][SMALL_TILE];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t task = (int64_t)blockIdx.x * WT_WARPS + w;
  if (task >= ntask) return;  // warp-uniform
  const Int4 t = tasks[toff + task];
  const SNode sj = sn[t.a];
  const int s = t.b;
  const int ts = min(SMALL_TILE, sj.ncols - s * NB);
  const T *D = Lx + sj.lx + (int64_t)(s * NB) * sj.nrows + s * NB;
  double *a = la[w], *x = lxv[w], *dinv = dv[w];
  for (int c = 0; c < ts; ++c)
    if (lane >= c && lane < ts) {
      a[pk(ts, c, lane)] = (double)D[(int64_t)c * sj.nrows + lane];
      x[pk(ts, c, lane)] = lane == c ? 1.0 : 0.0;
    }
  __syncwarp();
  if (lane < ts) dinv[lane] = 1.0 / a[pk(ts, lane, lane)];
  __syncwarp();
  if (lane == 0 && ts > 0) x[pk(ts, 0, 0)] *= dinv[0];  // row 0 is final
  __syncwarp();
  // As in k_trtri: row c is final and scaled; row c + 1 is scaled by the lanes that update it.
  for (int c = 0; c + 1 < ts; ++c) {
    const int m = ts - 1 - c;  // rows c+1 .. ts-1 of columns 0 .. c
    for (int el = lane; el < m * (c + 1); el += 32) {
      const int r = c + 1 + el % m, j = el / m;
      const double v = fma(-a[pk(ts, c, r)], x[pk(ts, j, c)], x[pk(ts, j, r)]);
      x[pk(ts, j, r)] = r == c + 1 ? v * dinv[r] : v;
    }
    if (lane == 31) x[pk(ts, c + 1, c + 1)] *= dinv[c + 1];  // (no update touches it at step c)
    __syncwarp();
  }
  T *out = Linv + sj.dx + (int64_t)s * NB * NB;
  for (int c = 0; c < ts; ++c)
    if (lane < ts) out[(int64_t)c * ts + lane] = lane >= c ? (T)x[pk(ts, c, lane)] : T(0);
}

// Narrow levels of a batch in one launch: for every supernode of the level (at most SMALL_TILE
// columns, one column tile) the POTRF of its diagonal block, the TRSM of the rows below it and
// the TRTRI of the diagonal block. One warp per (supernode, MW = 32 / G matrices); lane
// q * MW + m works on matrix m of the warp and owns the panel rows r with r % G == q. On tiles of
// a few columns the warp-per-(tile, matrix) forms leave most lanes of every FP64 instruction idle
// (the FP64 pipe takes a warp instruction's full time whatever its active lanes); here every lane
// carries a matrix. The warp's panels sit in shared memory, element e (column-major, ld nrows) of
// matrix m at e * MP + m: with one lane per matrix (MP = 33, padded) the lanes of a step touch one
// element of 32 matrices, with G lanes per matrix (MP = MW) consecutive rows of MW matrices, both
// free of bank conflicts. Panels are staged with cp.async, every copy in flight at once. The
// factor is right-looking over the panel's columns; each element sees the operations of
// k_potrf_w (rows of the diagonal block) and k_trsm_w (rows below it) in their order, and the
// inverse those of k_trtri_w.
// Asynchronous copy of one element from global to shared memory (cp.async, 4 or 8 bytes, both
// addresses aligned to the size); cp_async_wait_all waits for this thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void *smem_dst, const void *gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gsrc), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copies between global memory (np contiguous elements per matrix, matrix mm's at
// base + mm * mstride, mm < nm) and a warp's lanes-to-matrices layout (element e of matrix mm at
// S[e * MP + mm]). One lane per matrix (G = 1, MP = 33): consecutive lanes on consecutive
// elements of one matrix (coalesced, and the padded rows keep the shared accesses apart). G > 1
// (MP = MW): consecutive lanes on consecutive shared addresses, the MW matrices fastest (with a
// stride of MW elements the first mapping would put the lanes on few banks).
template <typename T, int G>
__device__ __forceinline__ void stage_in(T *S, const T *base, int64_t mstride, int np, int nm) {
  constexpr int MW = 32 / G, MP = G == 1 ? 33 : MW;
  const int lane = threadIdx.x & 31;
  if constexpr (G == 1) {
    for (int mm = 0; mm < nm; ++mm)
      for (int e = lane; e < np; e += 32) cp_async_elem<sizeof(T)>(S + e * MP + mm, base + mm * mstride + e);
  } else {
    for (int i = lane; i < np * MW; i += 32) {
      const int mm = i & (MW - 1);
      if (mm < nm) cp_async_elem<sizeof(T)>(S + i, base + mm * mstride + i / MW);
    }
  }
}
template <typename T, int G>
__device__ __forceinline__ void stage_out(T *base, int64_t mstride, const T *S, int np, int nm) {
  constexpr int MW = 32 / G, MP = G == 1 ? 33 : MW;
  const int lane = threadIdx.x & 31;
  if constexpr (G == 1) {
    for (int mm = 0; mm < nm; ++mm)
      for (int e = lane; e < np; e += 32) base[mm * mstride + e] = S[e * MP + mm];
  } else {
    for (int i = lane; i < np * MW; i += 32) {
      const int mm = i & (MW - 1);
      if (mm < nm) base[mm * mstride + i / MW] = S[i];
    }
  }
}

template <typename T, int G>
__global__ void __launch_bounds__(32) k_panel_b(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                T *__restrict__ Lx, T *__restrict__ Linv, long long *status,
                                                double *__restrict__ piv, const double *__restrict__ axc,
                                                const int64_t *__restrict__ dpos, int64_t toff, int32_t nmat,
                                                int32_t ncmax, const Batch bt) {
  constexpr int MW = 32 / G, MP = G == 1 ? 33 : MW;  // matrices per warp, element stride
  constexpr bool F64PIV = std::is_same<T, float>::value;  // FP64 pivot chain of FP32 factors
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *dv = reinterpret_cast<double *>(smem_raw);     // ncmax x MW: 1 / L_cc in FP64
  double *dd = dv + (size_t)ncmax * MW;                   // FP32: ncmax x MW FP64 pivots
  double *xd = dd + (F64PIV ? (size_t)ncmax * MW : 0);    // FP32: strict lower inverse, packed rows
  T *S = reinterpret_cast<T *>(xd + (F64PIV ? (size_t)ncmax * (ncmax - 1) / 2 * MW : 0));
  const int lane = threadIdx.x, m = lane & (MW - 1), q = lane / MW;
  const int32_t mat0 = blockIdx.y * MW, mat = mat0 + m;
  const bool act = mat < nmat;
  const int nm = min(MW, nmat - mat0);  // matrices of this warp
  const Int4 t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.a];
  const int nc = sj.ncols, nr = sj.nrows, np = nc * nr;
  stage_in<T, G>(S, Lx + (int64_t)mat0 * bt.lx + sj.lx, bt.lx, np, nm);  // every copy in flight at once
  cp_async_wait_all();
  __syncwarp();
  T *const Sm = S + m;     // this lane's matrix: element (r, c) at Sm[c * ld + r * MP]
  const int ld = nr * MP;  // column stride
  if constexpr (F64PIV) {  // the FP64 diagonal of the updated block (as k_potrf_w loads it)
    const double *ax = axc ? axc + (int64_t)(act ? mat : mat0) * bt.nnz : nullptr;
    for (int c = q; c < nc; c += G) dd[c * MW + m] = act ? diag64((float)Sm[c * ld + c * MP], ax, dpos, sj.first + c) : 1.0;
    __syncwarp();
  }
  for (int c = 0; c < nc; ++c) {
    // pivot: every lane of the matrix computes it; the owner of row c stores L_cc below
    T x, lcc;
    if constexpr (F64PIV) {
      double d = dd[c * MW + m];
      if (!(d > 0.0)) {
        if (act && q == 0) atomicMin(status + mat, (long long)(sj.first + c));
        d = 1.0;
      }
      if (act && q == 0 && piv) piv[(int64_t)mat * bt.piv + sj.first + c] = d;
      const float df = (float)d;
      x = rsqrt_newton(df);
      lcc = df * x;
    } else {
      T d = Sm[c * ld + c * MP];
      if (!(d > T(0))) {
        if (act && q == 0) atomicMin(status + mat, (long long)(sj.first + c));
        d = T(1);
      }
      x = rsqrt_of(d);
      lcc = d * x;
    }
    const T dinv = T(1) / lcc;  // k_trsm_w's 1 / L_cc
    if (q == 0) dv[c * MW + m] = F64PIV ? 1.0 / (double)lcc : (double)dinv;  // k_trtri_w's FP64 1 / L_cc
    // column c: rows of the diagonal block times x (POTRF), rows below it times 1 / L_cc (TRSM)
    const int r1 = q > c ? q : q + ((c + 1 - q + G - 1) / G) * G;  // first own row > c
    T *const colc = Sm + c * ld;
    for (int rr = r1; rr < nr; rr += G) colc[rr * MP] *= rr < nc ? x : dinv;
    __syncwarp();
    if (c % G == q) colc[c * MP] = lcc;
    for (int rr = r1; rr < nr; rr += G) {
      T *const row = Sm + rr * MP;
      const T lrc = row[c * ld];
      if (F64PIV && rr < nc) dd[rr * MW + m] = fma(-(double)lrc, (double)lrc, dd[rr * MW + m]);
      const int cend = rr < nc ? (F64PIV ? rr - 1 : rr) : nc - 1;  // FP32: the FP64 chain holds the diagonal
#pragma unroll 4
      for (int cc = c + 1; cc <= cend; ++cc) row[cc * ld] = fma(-lrc, colc[cc * MP], row[cc * ld]);
    }
    __syncwarp();
  }
  // zeros above the diagonal (in the FP64 arm also the start of the inverse's rows there)
  for (int rr = q; rr < nc; rr += G)
    for (int j = 0; j < rr; ++j) {
      Sm[rr * ld + j * MP] = T(0);
      if constexpr (F64PIV) xd[(size_t)(rr * (rr - 1) / 2 + j) * MW + m] = 0.0;
    }
  __syncwarp();
  stage_out<T, G>(Lx + (int64_t)mat0 * bt.lx + sj.lx, bt.lx, S, np, nm);
  __syncwarp();
  // inverse of the diagonal block in FP64: x(r, j) for r > j in the FP64 arm at position (j, r)
  // of the panel (above the diagonal, already written out), in the FP32 arm in xd
  auto xr = [&](int rr, int j, int mm) -> double & {
    if constexpr (F64PIV) return xd[(size_t)(rr * (rr - 1) / 2 + j) * MW + mm];
    else return S[(rr * nr + j) * MP + mm];
  };
  for (int c = 0; c + 1 < nc; ++c) {
    const int r1 = q > c ? q : q + ((c + 1 - q + G - 1) / G) * G;
    for (int rr = r1; rr < nc; rr += G) {
      const double a = (double)Sm[c * ld + rr * MP];  // L(rr, c)
      const double dr = dv[rr * MW + m];
#pragma unroll 4
      for (int j = 0; j <= c; ++j) {
        const double xcj = j == c ? dv[c * MW + m] : xr(c, j, m);
        const double v = fma(-a, xcj, xr(rr, j, m));
        xr(rr, j, m) = rr == c + 1 ? v * dr : v;
      }
    }
    __syncwarp();
  }
  const int ts = nc;
  const float rts = 1.0f / (float)ts;  // e / ts for e < ts^2 <= 1024: exact through FP32
  T *out = Linv + (int64_t)mat0 * bt.dinv + sj.dx;
  for (int i = lane; i < ts * ts * MW; i += 32) {  // matrices fastest (as stage_out with G > 1)
    const int mm = i & (MW - 1), e = i / MW;
    const int c = (int)(((float)e + 0.5f) * rts), rr = e - c * ts;
    if (mm < nm) out[mm * bt.dinv + e] = rr > c ? (T)xr(rr, c, mm) : rr == c ? (T)dv[c * MW + mm] : T(0);
  }
}

template <typename T, int G>
size_t panel_b_smem(int32_t pmax, int32_t ncmax) {
  return (size_t)panel_smem_bytes(pmax, ncmax, std::is_same<T, float>::value, G);
}

// (f) Warp forms of the solve kernels for batches, on launches whose supernodes all have at most
// SMALL_TILE columns (the schedule marks them tb = SMALL_TILE): one warp per (task, matrix), the
// same task of WT_WARPS consecutive matrices per CTA. A batch's leaf levels hold ~10^3 tasks of a
// few dozen values each per matrix; one CTA per (task, matrix) spends its time being scheduled.
// Each keeps its CTA form's order of operations (bit-identical results).

// S_FSUM (k_fsum): lane c subtracts column c's contributions.
template <typename V, int NR>
__global__ void __launch_bounds__(32 * WT_WARPS) k_fsum_w(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                          const int64_t *__restrict__ cptr,
                                                          const int32_t *__restrict__ contrib,
                                                          const V *__restrict__ t, int64_t tsize, V *__restrict__ y,
                                                          int64_t n, int r0, int64_t toff, int32_t nmat,
                                                          const Batch bt) {
  pdl_trigger_early<V>();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t mat = blockIdx.y * WT_WARPS + w;
  if (mat >= nmat) return;
  y += (int64_t)mat * bt.y;
  t += (int64_t)mat * bt.t;
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  pdl_wait_then_trigger<V>();  // t and y are the predecessors' output
  for (int c = lane; c < sj.ncols; c += 32) {
    const int64_t gcol = sj.first + c;
    V acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = V(0);
    for (int64_t p = cptr[gcol]; p < cptr[gcol + 1]; ++p) {
      const int64_t e = contrib[p];
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] += t[(int64_t)q * tsize + e];
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) y[(int64_t)(r0 + q) * n + gcol] -= acc[q];
  }
}

// S_FPUSH (k_fpush): lane r owns rows r and r + 32 of the row tile; each row's product is summed
// over the columns g, g + 4, ... in four partial sums added as ((g0 + g1) + (g2 + g3)).
template <typename T, typename V, int NR>
__global__ void __launch_bounds__(32 * WT_WARPS) k_fpush_w(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                           const T *__restrict__ Lx, const V *__restrict__ y,
                                                           V *__restrict__ t, int64_t tsize, int64_t n, int r0,
                                                           int64_t toff, int32_t nmat, const Batch bt) {
  pdl_trigger_early<V>();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t mat = blockIdx.y * WT_WARPS + w;
  if (mat >= nmat) return;
  Lx += (int64_t)mat * bt.lx;
  y += (int64_t)mat * bt.y;
  t += (int64_t)mat * bt.t;
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  const int64_t rb = d_row_tile_base(tk.b, sj.ncols, sj.ncb);
  const int tm = d_row_tile_rows(tk.b, sj.ncols, sj.nrows, sj.ncb);
  const int c0 = tk.c * SOLVE_CW, cw = min(SOLVE_CW, sj.ncols - c0);
  const int64_t base = sj.tx + (int64_t)tk.c * (sj.nrows - sj.ncols) + (rb - sj.ncols);
  pdl_wait_then_trigger<V>();  // y_J is the predecessor's output
  const V *yj = y + (int64_t)r0 * n + sj.first + c0;
  for (int r = lane; r < tm; r += 32) {
    const T *row = Lx + sj.lx + (int64_t)c0 * sj.nrows + rb + r;
    V acc[4][NR];
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[g][q] = V(0);
    for (int c = 0; c < cw; ++c) {
      const V l = (V)row[(int64_t)c * sj.nrows];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        switch (c & 3) {  // (a register array cannot be indexed by a run-time value)
          case 0: acc[0][q] = fma(l, yj[(int64_t)q * n + c], acc[0][q]); break;
          case 1: acc[1][q] = fma(l, yj[(int64_t)q * n + c], acc[1][q]); break;
          case 2: acc[2][q] = fma(l, yj[(int64_t)q * n + c], acc[2][q]); break;
          default: acc[3][q] = fma(l, yj[(int64_t)q * n + c], acc[3][q]); break;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) t[(int64_t)q * tsize + base + r] = (acc[0][q] + acc[1][q]) + (acc[2][q] + acc[3][q]);
  }
}

// S_BGATHER (k_bgather): per column of the slice, lane l sums the rows below the diagonal block
// with index = l (mod 32) in ascending order, then the warp adds the lanes' sums by butterfly.
template <typename T, typename V, int NR>
__global__ void __launch_bounds__(32 * WT_WARPS) k_bgather_w(const SNode *__restrict__ sn,
                                                             const int32_t *__restrict__ rows,
                                                             const Int4 *__restrict__ tasks, const T *__restrict__ Lx,
                                                             V *__restrict__ y, int64_t n, int r0, int64_t toff,
                                                             int32_t nmat, const Batch bt) {
  pdl_trigger_early<V>();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t mat = blockIdx.y * WT_WARPS + w;
  if (mat >= nmat) return;
  Lx += (int64_t)mat * bt.lx;
  y += (int64_t)mat * bt.y;
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  const int c0 = tk.b * BG;
  const int tn = min(BG, sj.ncols - c0);
  const int32_t *R = rows + sj.rowp;
  pdl_wait_then_trigger<V>();  // z is the predecessor's output
  for (int c = 0; c < tn; ++c) {
    const T *col = Lx + sj.lx + (int64_t)(c0 + c) * sj.nrows;
    V sa[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) sa[q] = V(0);
    for (int rr = sj.ncols + lane; rr < sj.nrows; rr += 32) {
      const V la = (V)col[rr];
      const int64_t g = R[rr];
#pragma unroll
      for (int q = 0; q < NR; ++q) sa[q] = fma(la, y[(int64_t)(r0 + q) * n + g], sa[q]);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      V v = sa[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      sa[q] = v;
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < NR; ++q) y[(int64_t)(r0 + q) * n + sj.first + c0 + c] -= sa[q];
    }
  }
}

// S_FSTEP / S_BSTEP of a supernode of at most SMALL_TILE columns (one column tile, task
// {J, 0, 0, 0}): y_J <- L_JJ^{-1} y_J (forward) or L_JJ^{-T} y_J (backward) with the precomputed
// inverse; lane r forms row r in two partial sums as write_solved_tile does.
template <typename T, typename V, int NR, bool TRANS>
__global__ void __launch_bounds__(32 * WT_WARPS) k_dstep_w(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                                           const T *__restrict__ Linv, V *__restrict__ y, int64_t n,
                                                           int r0, int64_t toff, int32_t nmat, const Batch bt) {
  __shared__ V vs[WT_WARPS][NR][SMALL_TILE];
  pdl_trigger_early<V>();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t mat = blockIdx.y * WT_WARPS + w;
  if (mat >= nmat) return;
  Linv += (int64_t)mat * bt.dinv;
  y += (int64_t)mat * bt.y;
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  const int tu = min(SMALL_TILE, sj.ncols);
  const T *Li = Linv + sj.dx;  // tu x tu, column-major, lower
  pdl_wait_then_trigger<V>();  // y is the predecessor's output
#pragma unroll
  for (int q = 0; q < NR; ++q)
    if (lane < tu) vs[w][q][lane] = y[(int64_t)(r0 + q) * n + sj.first + lane];
  __syncwarp();
  if (lane < tu) {
    const int r = lane;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      V a0 = V(0), a1 = V(0);
      if (!TRANS) {  // (L^-1)(r, k) for k <= r
        int k = 0;
        for (; k + 1 <= r; k += 2) {
          a0 = fma((V)Li[(int64_t)k * tu + r], vs[w][q][k], a0);
          a1 = fma((V)Li[(int64_t)(k + 1) * tu + r], vs[w][q][k + 1], a1);
        }
        if (k <= r) a0 = fma((V)Li[(int64_t)k * tu + r], vs[w][q][k], a0);
      } else {  // (L^-1)(k, r) for k >= r
        int k = r;
        for (; k + 1 < tu; k += 2) {
          a0 = fma((V)Li[(int64_t)r * tu + k], vs[w][q][k], a0);
          a1 = fma((V)Li[(int64_t)r * tu + k + 1], vs[w][q][k + 1], a1);
        }
        if (k < tu) a0 = fma((V)Li[(int64_t)r * tu + k], vs[w][q][k], a0);
      }
      y[(int64_t)(r0 + q) * n + sj.first + r] = a0 + a1;
    }
  }
}

// FP64 solve of a batch's narrow levels in one launch per level and direction (the schedule
// marks them, Plan::fwd_panel / bwd_panel): one warp per (supernode, MW = 32 / G matrices) as in
// k_panel_b, lane q * MW + m on matrix m, the warp's panels and diagonal-block inverses staged in
// shared memory (element e of matrix m at e * MP + m) before the kernel waits for its predecessor.
// Forward, per right-hand side: each column subtracts the products its contribution list names
// (S_FSUM), the diagonal block is solved with its inverse (S_FSTEP), and the rows below it push
// their products (S_FPUSH); lanes of a matrix split the columns, then the rows. Backward: each
// column subtracts the products of the rows below the diagonal block with the solved values
// there (S_BGATHER; per column in ascending row order), then the diagonal block is solved with
// the transposed inverse (S_BSTEP). The steps and pushes keep their warp forms' order; the
// gather's sum runs in plain row order (the warp form adds 32 interleaved partial sums).
template <typename T, int G>
__device__ __forceinline__ void stage_panel_inverse(T *S, T *Si, const SNode &sj, const T *Lx, const T *Linv,
                                                    int32_t mat0, int nm, const Batch &bt) {
  stage_in<T, G>(S, Lx + (int64_t)mat0 * bt.lx + sj.lx, bt.lx, sj.ncols * sj.nrows, nm);
  stage_in<T, G>(Si, Linv + (int64_t)mat0 * bt.dinv + sj.dx, bt.dinv, sj.ncols * sj.ncols, nm);
  cp_async_wait_all();
  __syncwarp();
}

template <typename T, typename V, int G, int NR>
__global__ void __launch_bounds__(32) k_fwd_b(const SNode *__restrict__ sn, const Int4 *__restrict__ tasks,
                                              const int64_t *__restrict__ cptr, const int32_t *__restrict__ contrib,
                                              const T *__restrict__ Lx, const T *__restrict__ Linv,
                                              V *__restrict__ y, V *__restrict__ t, int64_t tsize, int64_t n, int r0,
                                              int nrhs, int64_t toff, int32_t nmat, int32_t pmax, int32_t ncmax,
                                              const Batch bt) {
  constexpr int MW = 32 / G, MP = G == 1 ? 33 : MW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *vb = reinterpret_cast<V *>(smem_raw);  // NR x ncmax x MW: y_J after the sums
  V *ob = vb + (size_t)NR * ncmax * MW;     // NR x ncmax x MW: y_J solved
  T *S = reinterpret_cast<T *>(ob + (size_t)NR * ncmax * MW);
  T *Si = S + (size_t)pmax * MP;
  const int lane = threadIdx.x, m = lane & (MW - 1), q = lane / MW;
  const int32_t mat0 = blockIdx.y * MW, mat = mat0 + m;
  const bool act = mat < nmat;
  const int nm = min(MW, nmat - mat0);
  pdl_trigger_early<V>();
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  const int nc = sj.ncols, nr = sj.nrows;
  stage_panel_inverse<T, G>(S, Si, sj, Lx, Linv, mat0, nm, bt);
  pdl_wait_then_trigger<V>();  // y and t are the predecessors' output
  if (!act) return;  // lanes of absent matrices leave; the warp barriers below name the others
  const unsigned mask = present_lanes(MW, nm);
  y += (int64_t)mat * bt.y;
  t += (int64_t)mat * bt.t;
  const T *Sm = S + m, *Sim = Si + m;
  auto vs = [&](V *b, int u, int c) -> V & { return b[((size_t)u * ncmax + c) * MW + m]; };
  for (int rh0 = 0; rh0 < nrhs; rh0 += NR) {  // NR right-hand sides at a time, in registers
    const int cnt = min(NR, nrhs - rh0);
    V *yq = y + (int64_t)(r0 + rh0) * n + sj.first;  // right-hand side u at yq + u * n
    V *tq = t + (int64_t)rh0 * tsize;                 // and tq + u * tsize
    for (int c = q; c < nc; c += G) {  // S_FSUM: y_g minus the sum of its listed products
      const int64_t g = sj.first + c;
      V acc[NR];
#pragma unroll
      for (int u = 0; u < NR; ++u) acc[u] = V(0);
      for (int64_t p = cptr[g]; p < cptr[g + 1]; ++p) {
        const int64_t e = contrib[p];
#pragma unroll
        for (int u = 0; u < NR; ++u)
          if (u < cnt) acc[u] += tq[u * tsize + e];
      }
#pragma unroll
      for (int u = 0; u < NR; ++u)
        if (u < cnt) vs(vb, u, c) = yq[u * n + c] - acc[u];
    }
    __syncwarp(mask);
    for (int r = q; r < nc; r += G) {  // S_FSTEP: row r of L_JJ^-1 y_J, two partial sums
      V a0[NR], a1[NR];
#pragma unroll
      for (int u = 0; u < NR; ++u) a0[u] = a1[u] = V(0);
      int k = 0;
      for (; k + 1 <= r; k += 2) {
        const V l0 = (V)Sim[(k * nc + r) * MP], l1 = (V)Sim[((k + 1) * nc + r) * MP];
#pragma unroll
        for (int u = 0; u < NR; ++u) {
          a0[u] = fma(l0, vs(vb, u, k), a0[u]);
          a1[u] = fma(l1, vs(vb, u, k + 1), a1[u]);
        }
      }
      if (k <= r) {
        const V l0 = (V)Sim[(k * nc + r) * MP];
#pragma unroll
        for (int u = 0; u < NR; ++u) a0[u] = fma(l0, vs(vb, u, k), a0[u]);
      }
#pragma unroll
      for (int u = 0; u < NR; ++u)
        if (u < cnt) {
          const V o = a0[u] + a1[u];
          yq[u * n + r] = o;
          vs(ob, u, r) = o;
        }
    }
    __syncwarp(mask);
    for (int rr = nc + q; rr < nr; rr += G) {  // S_FPUSH: four partial sums over the columns
      V a[4][NR];  // columns c with c % 4 = 0, 1, 2, 3
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int u = 0; u < NR; ++u) a[j][u] = V(0);
      const T *lr = Sm + rr * MP;
      int c = 0;
      for (; c + 3 < nc; c += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const V l = (V)lr[(c + j) * nr * MP];
#pragma unroll
          for (int u = 0; u < NR; ++u) a[j][u] = fma(l, vs(ob, u, c + j), a[j][u]);
        }
      }
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (c + j < nc) {
          const V l = (V)lr[(c + j) * nr * MP];
#pragma unroll
          for (int u = 0; u < NR; ++u) a[j][u] = fma(l, vs(ob, u, c + j), a[j][u]);
        }
#pragma unroll
      for (int u = 0; u < NR; ++u)
        if (u < cnt) tq[u * tsize + sj.tx + (rr - nc)] = (a[0][u] + a[1][u]) + (a[2][u] + a[3][u]);
    }
    __syncwarp(mask);
  }
}

template <typename T, typename V, int G, int NR>
__global__ void __launch_bounds__(32) k_bwd_b(const SNode *__restrict__ sn, const int32_t *__restrict__ rows,
                                              const Int4 *__restrict__ tasks, const T *__restrict__ Lx,
                                              const T *__restrict__ Linv, V *__restrict__ y, int64_t n, int r0,
                                              int nrhs, int64_t toff, int32_t nmat, int32_t pmax, int32_t ncmax,
                                              const Batch bt) {
  constexpr int MW = 32 / G, MP = G == 1 ? 33 : MW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *zb = reinterpret_cast<V *>(smem_raw);  // NR x ncmax x MW: z_J after the gather
  T *S = reinterpret_cast<T *>(zb + (size_t)2 * NR * ncmax * MW);
  T *Si = S + (size_t)pmax * MP;
  const int lane = threadIdx.x, m = lane & (MW - 1), q = lane / MW;
  const int32_t mat0 = blockIdx.y * MW, mat = mat0 + m;
  const bool act = mat < nmat;
  const int nm = min(MW, nmat - mat0);
  pdl_trigger_early<V>();
  const Int4 tk = tasks[toff + blockIdx.x];
  const SNode sj = sn[tk.a];
  const int nc = sj.ncols, nr = sj.nrows;
  const int32_t *R = rows + sj.rowp;
  stage_panel_inverse<T, G>(S, Si, sj, Lx, Linv, mat0, nm, bt);
  pdl_wait_then_trigger<V>();  // z is the predecessors' output
  if (!act) return;
  const unsigned mask = present_lanes(MW, nm);
  y += (int64_t)mat * bt.y;
  const T *Sm = S + m, *Sim = Si + m;
  auto zs = [&](int u, int c) -> V & { return zb[((size_t)u * ncmax + c) * MW + m]; };
  for (int rh0 = 0; rh0 < nrhs; rh0 += NR) {
    const int cnt = min(NR, nrhs - rh0);
    V *yq = y + (int64_t)(r0 + rh0) * n;  // right-hand side u at yq + u * n
    for (int c = q; c < nc; c += G) {  // S_BGATHER
      V sa[NR];
#pragma unroll
      for (int u = 0; u < NR; ++u) sa[u] = V(0);
      for (int rr = nc; rr < nr; ++rr) {
        const V l = (V)Sm[(c * nr + rr) * MP];
        const int64_t g = R[rr];
#pragma unroll
        for (int u = 0; u < NR; ++u)
          if (u < cnt) sa[u] = fma(l, yq[u * n + g], sa[u]);
      }
#pragma unroll
      for (int u = 0; u < NR; ++u)
        if (u < cnt) zs(u, c) = yq[u * n + sj.first + c] - sa[u];
    }
    __syncwarp(mask);
    for (int r = q; r < nc; r += G) {  // S_BSTEP: row r of L_JJ^-T z_J, two partial sums
      V a0[NR], a1[NR];
#pragma unroll
      for (int u = 0; u < NR; ++u) a0[u] = a1[u] = V(0);
      int k = r;
      for (; k + 1 < nc; k += 2) {
        const V l0 = (V)Sim[(r * nc + k) * MP], l1 = (V)Sim[(r * nc + k + 1) * MP];
#pragma unroll
        for (int u = 0; u < NR; ++u) {
          a0[u] = fma(l0, zs(u, k), a0[u]);
          a1[u] = fma(l1, zs(u, k + 1), a1[u]);
        }
      }
      if (k < nc) {
        const V l0 = (V)Sim[(r * nc + k) * MP];
#pragma unroll
        for (int u = 0; u < NR; ++u) a0[u] = fma(l0, zs(u, k), a0[u]);
      }
#pragma unroll
      for (int u = 0; u < NR; ++u)
        if (u < cnt) yq[u * n + sj.first + r] = a0[u] + a1[u];
    }
    __syncwarp(mask);
  }
}

template <typename T, int TB>
constexpr size_t trsm_smem() { return sizeof(T) * (TB * (TB + 1) + TB * (NB + 1) + TB); }
template <int TB>
constexpr size_t trtri_smem() { return sizeof(double) * (2 * TB * (TB + 1) + TB); }

inline int grid_for(int64_t count, int per) {
  int64_t g = (count + per - 1) / per;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

// Launch with a stream priority attribute (kept by CUDA-graph capture as a node priority).
template <typename... KArgs, typename... Args>
cudaError_t launch_prio(void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t st, int prio,
                        Args... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch that may start before the previous kernel of the stream completes (see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch of a cluster-form solve step: clusters of four CTAs along x, programmatic dependent
// launch (see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_step_c(void (*kernel)(KArgs...), dim3 grid, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  cfg.gridDim = grid;
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 4;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch of thread-block clusters of cs CTAs along x, with a stream priority.
template <typename... KArgs, typename... Args>
cudaError_t launch_cluster_prio(void (*kernel)(KArgs...), dim3 grid, int threads, int cs, cudaStream_t st, int prio,
                                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  cfg.gridDim = dim3(grid.x * (unsigned)cs, grid.y, grid.z);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)cs;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cs > 1 ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline void trace_mark(LaunchTrace *tr, int32_t kind, cudaStream_t st) {
  if (!tr) return;
  cudaEventRecord((*tr->events)[tr->used++], st);
  if (kind >= 0) tr->kinds.push_back(kind);
}

template <typename T>
cudaError_t prepare_factor() {
  cudaError_t e = cudaFuncSetAttribute(k_trsm_r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)trsm_smem<T, NB>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_trsm<T, SMALL_TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsm_smem<T, SMALL_TB>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_trsm_w<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_w_smem<T>());
  if (e != cudaSuccess) return e;
  {
    void (*panel[5])(const SNode *, const Int4 *, T *, T *, long long *, double *, const double *, const int64_t *,
                     int64_t, int32_t, int32_t, const Batch) = {k_panel_b<T, 1>, k_panel_b<T, 2>, k_panel_b<T, 4>,
                                                                 k_panel_b<T, 8>, k_panel_b<T, 32>};
    for (auto *k : panel) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, PANEL_SMEM_HARD);
      if (e != cudaSuccess) return e;
    }
  }
  e = cudaFuncSetAttribute(k_trtri<T, SMALL_TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trtri_smem<SMALL_TB>());
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<T, float>::value) {
    e = prepare_update_tc();
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_trtri<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trtri_smem<NB>());
}

// Sparse right-hand side: zero the columns of the reached supernodes, scatter b, gather x.
__global__ void k_reach_zero(const SNode *__restrict__ sn, const int32_t *__restrict__ snodes,
                             double *__restrict__ y) {
  const SNode s = sn[snodes[blockIdx.x]];
  for (int c = threadIdx.x; c < s.ncols; c += blockDim.x) y[s.first + c] = 0.0;
}
__global__ void k_reach_scatter(const int32_t *__restrict__ pbeta, const double *__restrict__ bvals, int64_t nb,
                                double *__restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nb) y[pbeta[t]] = bvals[t];
}
__global__ void k_reach_gather(const int32_t *__restrict__ cols, int64_t nr, const double *__restrict__ y,
                               double *__restrict__ x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nr) x[t] = y[cols[t]];
}

// Breakdown measure of an FP32 factor: one CTA per matrix scans the pivots in a fixed order and
// reduces (ratio, column) pairs in shared memory (smallest ratio, then smallest column).
__global__ void __launch_bounds__(1024) k_pivot_ratio(const double *__restrict__ piv, int64_t n,
                                                      const double *__restrict__ Ax, int64_t axstride,
                                                      const int64_t *__restrict__ dpos, PivotInfo *out) {
  __shared__ double rs[1024];
  __shared__ int64_t ks[1024];
  piv += blockIdx.x * n;
  Ax += blockIdx.x * axstride;
  double best = INFINITY;
  int64_t bk = -1;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double akk = Ax[dpos[k]];
    const double r = akk > 0.0 ? piv[k] / akk : 0.0;
    if (r < best) {  // k ascends within a thread: ties keep the smaller column
      best = r;
      bk = k;
    }
  }
  rs[threadIdx.x] = best;
  ks[threadIdx.x] = bk;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const double r2 = rs[threadIdx.x + h];
      const int64_t k2 = ks[threadIdx.x + h];
      if (r2 < rs[threadIdx.x] || (r2 == rs[threadIdx.x] && k2 >= 0 && (ks[threadIdx.x] < 0 || k2 < ks[threadIdx.x]))) {
        rs[threadIdx.x] = r2;
        ks[threadIdx.x] = k2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[blockIdx.x].min_ratio = rs[0];
    out[blockIdx.x].column = ks[0];
  }
}

template <typename T, typename V>
cudaError_t prepare_solve() {
  cudaError_t e = cudaFuncSetAttribute(k_fstep<T, V, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)step_smem<V, NB>());
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<T, V>::value) {
    const void *k[14] = {(const void *)k_fwd_b<T, V, 1, 1>,  (const void *)k_fwd_b<T, V, 2, 1>,
                         (const void *)k_fwd_b<T, V, 4, 1>,  (const void *)k_fwd_b<T, V, 8, 1>,
                         (const void *)k_fwd_b<T, V, 32, 1>, (const void *)k_fwd_b<T, V, 32, 4>,
                         (const void *)k_fwd_b<T, V, 32, 8>, (const void *)k_bwd_b<T, V, 1, 1>,
                         (const void *)k_bwd_b<T, V, 2, 1>,  (const void *)k_bwd_b<T, V, 4, 1>,
                         (const void *)k_bwd_b<T, V, 8, 1>,  (const void *)k_bwd_b<T, V, 32, 1>,
                         (const void *)k_bwd_b<T, V, 32, 4>, (const void *)k_bwd_b<T, V, 32, 8>};
    for (const void *f : k) {
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, PANEL_SMEM_HARD);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaFuncSetAttribute(k_fgather<T, V>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
}

bool factor_launch_has_alternative(const Launch &L, int32_t nbatch, bool fp64) {
  const bool small = L.tb == SMALL_TB;
  if (nbatch > 1)  // one warp per (tile, matrix) against one CTA per tile and matrix
    return (small && (L.kind == K_UPDATE || L.kind == K_POTRF || L.kind == K_TRTRI || L.kind == K_TRSM)) ||
           (fp64 && !small && L.kind == K_UPDATE);
  // one matrix: a clustered FP64 update against one CTA per tile; FP32 full-tile updates on the
  // tensor cores against the SIMT pipes; small-tile POTRF and TRTRI with one CTA per tile against
  // one warp per tile
  return (fp64 && !small && L.kind == K_UPDATE && L.cluster > 1) || (!fp64 && !small && L.kind == K_UPDATE) ||
         (small && (L.kind == K_POTRF || L.kind == K_TRTRI));
}

// A batch's small-tile update with lanes mapped to matrices (k_update_mb, G lanes per matrix).
template <typename T>
cudaError_t launch_update_mb(int lanes, unsigned g, unsigned nb, cudaStream_t s, int prio, const DevPlan &d, T *Lx,
                             int64_t off, const Batch &bt) {
#define SYM_UPD_MB(G)                                                                                           \
  case G:                                                                                                       \
    return launch_prio(k_update_mb<T, G>, dim3(g, (nb + WT_WARPS * (32 / G) - 1) / (WT_WARPS * (32 / G))),      \
                       32 * WT_WARPS, 0, s, prio, d.sn, d.upd_tasks, d.upd_entries, d.rel, Lx, off, (int32_t)nb, \
                       bt);
  switch (lanes) {
    SYM_UPD_MB(1)
    SYM_UPD_MB(2)
    SYM_UPD_MB(4)
    SYM_UPD_MB(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef SYM_UPD_MB
}

// One fused narrow-level launch (k_panel_b with the level's lanes per matrix).
template <typename T>
cudaError_t launch_panel_b(const DevPlan &d, const PanelForm &pf, unsigned g, unsigned nb, cudaStream_t s, int prio,
                           T *Lx, T *Linv, long long *status, int64_t off, const Batch &bt) {
  const int lanes = panel_lanes_for(pf, nb, std::is_same<T, float>::value);
#define SYM_PANEL(G)                                                                                         \
  case G:                                                                                                    \
    return launch_prio(k_panel_b<T, G>, dim3(g, (nb + 32 / G - 1) / (32 / G)), 32,                           \
                       panel_b_smem<T, G>(pf.pmax, pf.ncmax), s, prio, d.sn, d.tasks, Lx, Linv, status, d.piv, \
                       d.axc, d.dpos, off, (int32_t)nb, pf.ncmax, bt);
  switch (lanes) {
    SYM_PANEL(1)
    SYM_PANEL(2)
    SYM_PANEL(4)
    SYM_PANEL(8)
    SYM_PANEL(32)
    default:
      return cudaErrorInvalidValue;
  }
#undef SYM_PANEL
}

template <typename T>
cudaError_t run_factor(const DevPlan &d, const std::vector<Launch> &launches, const double *Ax,
                       T *Lx, T *Linv, long long *status, cudaStream_t st, LaunchTrace *trace, const Batch &bt,
                       const TwoStreams *two) {
  const unsigned nb = (unsigned)bt.count;
  // With two streams the schedule's stream/wait fields are honoured (lookahead); otherwise (and
  // when tracing) every launch goes to st in list order, which satisfies every wait.
  const bool dual = two && two->aux && two->events && !trace;
  trace_mark(trace, -1, st);
  k_zero<T><<<dim3(grid_for(d.storage, THREADS * 4), nb), THREADS, 0, st>>>(Lx, d.storage, bt);
  if (d.nnz_a > 0)
    k_scatter<T><<<dim3(grid_for(d.nnz_a, THREADS * 4), nb), THREADS, 0, st>>>(Ax, d.amap, Lx, d.nnz_a, bt);
  trace_mark(trace, K_SCATTER, st);
  if (dual) {  // the auxiliary stream starts after the panels hold A
    cudaEventRecord(two->fork, st);
    cudaStreamWaitEvent(two->aux, two->fork, 0);
  }
  for (size_t li = 0; li < launches.size(); ++li) {
    const Launch &L = launches[li];
    const unsigned g = (unsigned)L.count;
    cudaStream_t s = (dual && L.stream == 1) ? two->aux : st;
    const int prio = (dual && L.stream == 1) ? two->prio_low : two ? two->prio_high : 0;
    if (dual && L.wait >= 0) cudaStreamWaitEvent(s, (*two->events)[L.wait], 0);
    // a fused narrow level: its POTRF launch factors and inverts the whole panels, its TRSM and
    // TRTRI launches have nothing left to do
    int32_t panel = d.batch_panel ? d.batch_panel[li].role : PANEL_NONE;
    if (panel != PANEL_NONE) {  // unless the autotuner keeps the level apart or a batch's panels do not fit
      const int32_t head = d.batch_panel[li].head;
      const int8_t *apart = d.panel_apart[nb > 1 ? 1 : 0];
      if ((apart && apart[head]) || panel_lanes_for(d.batch_panel[head], nb, std::is_same<T, float>::value) == 0)
        panel = PANEL_NONE;
    }
    if (panel == PANEL_COVERED) {
      if (dual) cudaEventRecord((*two->events)[li], s);
      trace_mark(trace, L.kind, st);
      continue;
    }
    cudaError_t e = cudaSuccess;
    const bool small = L.tb == SMALL_TB;  // every tile of the launch fits the small variant
    // the autotuner's choice for this launch: false keeps the default form of a batch
    const int8_t *var = d.variant[nb > 1 ? 1 : 0];
    const bool alt = var && var[li] != 0 &&
                     factor_launch_has_alternative(L, (int32_t)nb, std::is_same<T, double>::value);
    constexpr int TS = TileCfg<SMALL_TB>::threads;
    switch (L.kind) {
      case K_UPDATE:
        // FP64: flat element map (the FP64 pipe is the bound and every issued DFMA should be
        // useful); FP32: 4 x 8 register tiles (operand reuse matters at the FP32 rate)
        if constexpr (!std::is_same<T, double>::value) {
          if (d.tensor_cores && !small && !alt)  // (alt: the SIMT form, the autotuner's choice)
            e = launch_update_tc(dim3(g, nb), s, prio, d, Lx, L.off, bt, status);
          else if (alt && small)  // a batch's small tiles: one warp per (tile, matrix)
            e = launch_prio(k_update_wb<T>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS), 32 * WT_WARPS, 0, s, prio,
                            d.sn, d.upd_tasks, d.upd_entries, d.rel, Lx, L.off, (int32_t)nb, bt);
          else
            e = launch_prio(k_update_f32, dim3(g, nb), F32_THREADS, 0, s, prio, d.sn, d.upd_tasks, d.upd_entries,
                            d.rel, Lx, L.off, bt);
        }
        // a batch, lanes = matrices: the default of small tiles and of full tiles with small entries
        // (alternatives: a warp per (tile, matrix) on the tile in shared or global memory), the
        // alternative of full tiles with large entries (default: one CTA per tile and matrix)
        else if (nb > 1 && d.batch_lanes && d.batch_lanes[li] > 0 &&
                 (small || (d.batch_warp && d.batch_warp[li])) != alt)
          e = launch_update_mb<T>(d.batch_lanes[li], g, nb, s, prio, d, Lx, L.off, bt);
        else if (small && nb > 1)  // a batch: one warp per (tile, matrix)
          e = launch_prio(k_update_wb<T>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS), 32 * WT_WARPS, 0, s, prio,
                          d.sn, d.upd_tasks, d.upd_entries, d.rel, Lx, L.off, (int32_t)nb, bt);
        else if (!small && nb > 1 && d.batch_warp && d.batch_warp[li])  // small entries of a batch
          e = launch_prio(k_update_wg<T>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS), 32 * WT_WARPS, 0, s, prio,
                          d.sn, d.upd_tasks, d.upd_entries, d.rel, Lx, L.off, (int32_t)nb, bt);
        else if (small)
          e = launch_prio(k_update_flat<T, SMALL_TB, false>, dim3(g, nb), TS, 0, s, prio, d.sn, d.upd_tasks,
                          d.upd_entries, d.rel, Lx, L.off, bt);
        else if (L.cluster > 1 && nb == 1 && !alt)  // (a batch already fills the GPU through blockIdx.y)
          e = launch_cluster_prio(k_update_flat<T, NB, true>, dim3(g, nb), THREADS, L.cluster, s, prio, d.sn,
                                  d.upd_tasks, d.upd_entries, d.rel, Lx, L.off, bt);
        else
          e = launch_prio(k_update_flat<T, NB, false>, dim3(g, nb), THREADS, 0, s, prio, d.sn, d.upd_tasks,
                          d.upd_entries, d.rel, Lx, L.off, bt);
        break;
      case K_POTRF:
        // small tiles of a batch: a warp per tile (throughput); of one matrix: a CTA per tile, whose
        // four warps shorten each column step of the tile (latency; 64^2 factor 0.96 -> 0.83 ms);
        // the autotuner's choice (alt) swaps the two
        if (panel == PANEL_FUSED)
          e = launch_panel_b<T>(d, d.batch_panel[li], g, nb, s, prio, Lx, Linv, status, L.off, bt);
        else if (small && (nb > 1) != alt)
          e = launch_prio(k_potrf_w<T>, dim3((g + WT_WARPS - 1) / WT_WARPS, nb), 32 * WT_WARPS, 0, s, prio, d.sn,
                          d.tasks, (int64_t)g, Lx, status, d.piv, d.axc, d.dpos, L.off, bt);
        else if (small)
          e = launch_prio(k_potrf<T, SMALL_TB>, dim3(g, nb), TS, 0, s, prio, d.sn, d.tasks, Lx, status, d.piv, d.axc,
                          d.dpos, L.off, bt);
        else if constexpr (std::is_same<T, float>::value)  // the column chain in registers
          e = launch_prio(k_potrf_r, dim3(g, nb), PR_THREADS, 0, s, prio, d.sn, d.tasks, Lx, status, d.piv, d.axc,
                          d.dpos, L.off, bt);
        else
          e = launch_prio(k_potrf<T, NB>, dim3(g, nb), THREADS, 0, s, prio, d.sn, d.tasks, Lx, status, d.piv, d.axc,
                          d.dpos, L.off, bt);
        break;
      case K_TRSM:
        // (a warp-per-tile form with the column pairs mapped flat onto the lanes made the
        // 512 x 128^2 batch's TRSM slower, 11.0 -> 16.3 ms: its tiles have enough rows; the
        // warp-per-(tile, matrix) form is the autotuner's alternative)
        if (small && nb > 1 && alt)
          e = launch_prio(k_trsm_w<T>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS), 32 * WT_WARPS, trsm_w_smem<T>(), s,
                          prio, d.sn, d.tasks, Lx, L.off, (int32_t)nb, bt);
        else if (small)
          e = launch_prio(k_trsm<T, SMALL_TB>, dim3(g, nb), TS, trsm_smem<T, SMALL_TB>(), s, prio, d.sn, d.tasks, Lx,
                          L.off, bt);
        else  // the tile in registers
          e = launch_prio(k_trsm_r<T>, dim3(g, nb), THREADS, trsm_smem<T, NB>(), s, prio, d.sn, d.tasks, Lx, L.off,
                          bt);
        break;
      case K_GEMM:
        if constexpr (std::is_same<T, double>::value)
          e = launch_prio(k_gemm<T>, dim3(g, nb), THREADS, 0, s, prio, d.sn, d.tasks, Lx, L.off, bt);
        else
          e = launch_prio(k_gemm_f32, dim3(g, nb), F32_THREADS, 0, s, prio, d.sn, d.tasks, Lx, L.off, bt);
        break;
      case K_TRTRI:
        if (small && (nb > 1) != alt)  // (as for POTRF)
          e = launch_prio(k_trtri_w<T>, dim3((g + WT_WARPS - 1) / WT_WARPS, nb), 32 * WT_WARPS, 0, s, prio, d.sn,
                          d.tasks, (int64_t)g, (const T *)Lx, Linv, L.off, bt);
        else
          e = small ? launch_prio(k_trtri<T, SMALL_TB>, dim3(g, nb), TS, trtri_smem<SMALL_TB>(), s, prio, d.sn, d.tasks,
                                  (const T *)Lx, Linv, L.off, bt)
                  : launch_prio(k_trtri<T, NB>, dim3(g, nb), THREADS, trtri_smem<NB>(), s, prio, d.sn, d.tasks,
                                (const T *)Lx, Linv, L.off, bt);
        break;
      default:
        return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (dual) cudaEventRecord((*two->events)[li], s);
    trace_mark(trace, L.kind, st);
  }
  if (dual) {
    cudaEventRecord(two->join, two->aux);
    cudaStreamWaitEvent(st, two->join, 0);
  }
  return cudaGetLastError();
}

// The fused narrow solve levels: the form of launch li of a solve list (forms: the plan's marks
// for that list, nform entries; a pruned list never matches them), or null when the launch runs
// as scheduled. A single FP32 matrix solving more than two right-hand sides per pass keeps the
// separate launches (the 64^3 refined solve with four: 13.9 ms fused against 13.7 ms; FP64 with
// four 8.74 against 8.96 ms; with one, FP64 and FP32 alike, 64^2 0.14 against 0.17 ms and the
// uneven 256-grid union 4.9 against 11.4 ms).
inline const PanelForm *solve_panel(const PanelForm *forms, int64_t nform, size_t nlist, size_t li, unsigned nb,
                                    bool fp64, int nr) {
  if (!forms || (int64_t)nlist != nform || forms[li].role == PANEL_NONE) return nullptr;
  if (nb == 1 && !fp64 && nr > 2) return nullptr;
  return solve_lanes_for(forms[forms[li].head], nb, fp64) > 0 ? &forms[li] : nullptr;
}

template <typename T, typename V>
cudaError_t launch_solve_b(bool forward, const DevPlan &d, const PanelForm &pf, unsigned g, unsigned nb,
                           cudaStream_t st, const T *Lx, const T *Linv, V *y, V *tbuf, int r0, int nr, int64_t off,
                           const Batch &bt) {
  if constexpr (std::is_same<T, V>::value) {
    const int lanes = solve_lanes_for(pf, nb, std::is_same<T, double>::value);
    // right-hand sides per pass of the kernel: batches one at a time, a single matrix 1, 4 or 8
    const int nrb = nb > 1 || nr <= 2 ? 1 : nr <= 4 ? 4 : 8;
    const size_t smem = (size_t)solve_panel_bytes(pf.pmax, pf.ncmax, lanes, nrb);
#define SYM_SOLVE_B(G, NRB)                                                                                      \
  if (lanes == G && nrb == NRB)                                                                                  \
    return forward ? launch_pdl(k_fwd_b<T, V, G, NRB>, dim3(g, (nb + 32 / G - 1) / (32 / G)), 32, smem, st,     \
                                d.sn, d.tasks, d.cptr, d.contrib, Lx, Linv, y, tbuf, d.tsize, d.n, r0, nr, off,  \
                                (int32_t)nb, pf.pmax, pf.ncmax, bt)                                              \
                   : launch_pdl(k_bwd_b<T, V, G, NRB>, dim3(g, (nb + 32 / G - 1) / (32 / G)), 32, smem, st,     \
                                d.sn, d.rows, d.tasks, Lx, Linv, y, d.n, r0, nr, off, (int32_t)nb, pf.pmax,       \
                                pf.ncmax, bt);
    SYM_SOLVE_B(1, 1)
    SYM_SOLVE_B(2, 1)
    SYM_SOLVE_B(4, 1)
    SYM_SOLVE_B(8, 1)
    SYM_SOLVE_B(32, 1)
    SYM_SOLVE_B(32, 4)
    SYM_SOLVE_B(32, 8)
#undef SYM_SOLVE_B
  }
  return cudaErrorInvalidValue;
}

template <typename T, typename V>
cudaError_t run_sweeps(const DevPlan &d, const std::vector<Launch> &fwd, const std::vector<Launch> &bwd,
                       const T *Lx, const T *Linv, int nrhs, V *y, cudaStream_t st, LaunchTrace *trace,
                       const Batch &bt) {
  const int64_t n = d.n;
  const unsigned nb = (unsigned)bt.count;
  V *tbuf = reinterpret_cast<V *>(d.t);
  for (int r0 = 0; r0 < nrhs; r0 += MAXRHS) {
    const int nr = nrhs - r0 < MAXRHS ? nrhs - r0 : MAXRHS;
    constexpr bool fp64 = std::is_same<T, double>::value && std::is_same<V, double>::value;
    for (size_t li = 0; li < fwd.size(); ++li) {
      const Launch &L = fwd[li];
      const unsigned g = (unsigned)L.count;
      cudaError_t e = cudaSuccess;
      // a fused narrow level: its step launch runs the sums, steps and pushes
      if (const PanelForm *pf = solve_panel(d.fwd_panel, d.nfwd_panel, fwd.size(), li, nb, fp64, nr)) {
        if (pf->role == PANEL_FUSED)
          e = launch_solve_b<T, V>(true, d, *pf, g, nb, st, Lx, Linv, y, tbuf, r0, nr, L.off, bt);
        if (e != cudaSuccess) return e;
        trace_mark(trace, L.kind, st);
        continue;
      }
      switch (L.kind) {
        case S_FGATHER: {
          cudaLaunchConfig_t cfg = {};
          cudaLaunchAttribute attr[1];
          cfg.gridDim = dim3(g * (unsigned)L.cluster, nb, 1);
          cfg.blockDim = dim3(THREADS, 1, 1);
          cfg.dynamicSmemBytes = 0;
          cfg.stream = st;
          attr[0].id = cudaLaunchAttributeClusterDimension;
          attr[0].val.clusterDim.x = (unsigned)L.cluster;
          attr[0].val.clusterDim.y = 1;
          attr[0].val.clusterDim.z = 1;
          cfg.attrs = attr;
          cfg.numAttrs = 1;
          e = cudaLaunchKernelEx(&cfg, k_fgather<T, V>, d.sn, d.tasks, d.upd_tasks, d.upd_entries,
                                             d.rel, Lx, y, n, r0, nr, L.off, bt);
          if (e != cudaSuccess) return e;
          break;
        }
        case S_FSTEP:
          if (nb > 1 && L.tb == SMALL_TB) {  // a batch's supernodes of <= SMALL_TILE columns
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_dstep_w<T, V, NR, false>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS),
                                                32 * WT_WARPS, 0, st, d.sn, d.tasks, Linv, y, n, r0, L.off,
                                                (int32_t)nb, bt)));
            break;
          }
          if (L.cluster == 4) {
            SYM_NR_DISPATCH(nr, (e = launch_step_c(k_step_c<T, V, NR, true>, dim3(4 * g, nb), st, d.sn, d.tasks, Lx,
                                                   Linv, y, n, r0, L.off, bt)));
            break;
          }
          e = L.tb == SMALL_TB
                  ? launch_pdl(k_fstep<T, V, SMALL_TB>, dim3(g, nb), TileCfg<SMALL_TB>::threads,
                               step_smem<V, SMALL_TB>(), st, d.sn, d.tasks, Lx, Linv, y, n, r0, nr, L.off, bt)
                  : launch_pdl(k_fstep<T, V, NB>, dim3(g, nb), THREADS, step_smem<V, NB>(), st, d.sn, d.tasks, Lx,
                               Linv, y, n, r0, nr, L.off, bt);
          break;
        case S_FPUSH:
          if (nb > 1 && L.tb == SMALL_TB) {
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_fpush_w<T, V, NR>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS),
                                                32 * WT_WARPS, 0, st, d.sn, d.tasks, Lx, (const V *)y, tbuf, d.tsize,
                                                n, r0, L.off, (int32_t)nb, bt)));
          } else {
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_fpush<T, V, NR>, dim3(g, nb), THREADS, 0, st, d.sn, d.tasks, Lx,
                                                (const V *)y, tbuf, d.tsize, n, r0, L.off, bt)));
          }
          break;
        case S_FSUM:
          if (nb > 1 && L.tb == SMALL_TB) {
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_fsum_w<V, NR>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS),
                                                32 * WT_WARPS, 0, st, d.sn, d.tasks, d.cptr, d.contrib,
                                                (const V *)tbuf, d.tsize, y, n, r0, L.off, (int32_t)nb, bt)));
          } else {
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_fsum<V, NR>, dim3(g, nb), THREADS, 0, st, d.sn, d.tasks, d.cptr,
                                                d.contrib, (const V *)tbuf, d.tsize, y, n, r0, L.off, bt)));
          }
          break;
        default:
          return cudaErrorInvalidValue;
      }
      if (e != cudaSuccess) return e;
      trace_mark(trace, L.kind, st);
    }
    for (size_t li = 0; li < bwd.size(); ++li) {
      const Launch &L = bwd[li];
      const unsigned g = (unsigned)L.count;
      cudaError_t e = cudaSuccess;
      if (const PanelForm *pf = solve_panel(d.bwd_panel, d.nbwd_panel, bwd.size(), li, nb, fp64, nr)) {
        if (pf->role == PANEL_FUSED)
          e = launch_solve_b<T, V>(false, d, *pf, g, nb, st, Lx, Linv, y, tbuf, r0, nr, L.off, bt);
        if (e != cudaSuccess) return e;
        trace_mark(trace, L.kind, st);
        continue;
      }
      switch (L.kind) {
        case S_BGATHER:
          if (nb > 1 && L.tb == SMALL_TB) {
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_bgather_w<T, V, NR>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS),
                                                32 * WT_WARPS, 0, st, d.sn, d.rows, d.tasks, Lx, y, n, r0, L.off,
                                                (int32_t)nb, bt)));
          } else {
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_bgather<T, V, NR>, dim3(g, nb), THREADS, 0, st, d.sn, d.rows,
                                                d.tasks, Lx, y, n, r0, L.off, bt)));
          }
          break;
        case S_BSTEP:
          if (nb > 1 && L.tb == SMALL_TB) {  // a batch's supernodes of <= SMALL_TILE columns
            SYM_NR_DISPATCH(nr, (e = launch_pdl(k_dstep_w<T, V, NR, true>, dim3(g, (nb + WT_WARPS - 1) / WT_WARPS),
                                                32 * WT_WARPS, 0, st, d.sn, d.tasks, Linv, y, n, r0, L.off,
                                                (int32_t)nb, bt)));
            break;
          }
          if (L.cluster == 4) {
            SYM_NR_DISPATCH(nr, (e = launch_step_c(k_step_c<T, V, NR, false>, dim3(4 * g, nb), st, d.sn, d.tasks, Lx,
                                                   Linv, y, n, r0, L.off, bt)));
            break;
          }
          if (L.tb != SMALL_TB) return cudaErrorInvalidValue;  // (wider supernodes: the cluster form)
          e = launch_pdl(k_bstep<T, V, SMALL_TB>, dim3(g, nb), TileCfg<SMALL_TB>::threads, step_smem<V, SMALL_TB>(),
                         st, d.sn, d.tasks, Lx, Linv, y, n, r0, nr, L.off, bt);
          break;
        default:
          return cudaErrorInvalidValue;
      }
      if (e != cudaSuccess) return e;
      trace_mark(trace, L.kind, st);
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_solve(const DevPlan &d, const std::vector<Launch> &fwd, const std::vector<Launch> &bwd,
                      const T *Lx, const T *Linv, int nrhs, const double *B, int64_t ldb, double *X,
                      int64_t ldx, double *y, cudaStream_t st, LaunchTrace *trace, const Batch &bt) {
  const int64_t n = d.n;
  const unsigned nb = (unsigned)bt.count;
  if (n == 0 || nrhs == 0) return cudaSuccess;
  trace_mark(trace, -1, st);
  k_perm_in<double><<<dim3(grid_for(n * nrhs, THREADS), nb), THREADS, 0, st>>>(d.perm, B, ldb, y, n, nrhs, bt);
  trace_mark(trace, S_PERM, st);
  cudaError_t e = run_sweeps<T, double>(d, fwd, bwd, Lx, Linv, nrhs, y, st, trace, bt);
  if (e != cudaSuccess) return e;
  k_perm_out<double><<<dim3(grid_for(n * nrhs, THREADS), nb), THREADS, 0, st>>>(d.perm, y, X, ldx, n, nrhs, bt);
  trace_mark(trace, S_PERM, st);
  return cudaGetLastError();
}

cudaError_t run_sparse_lower(const DevPlan &d, const std::vector<Launch> &fwd, const double *Lx,
                             const double *Linv, const int32_t *snodes, int64_t nsn, const int32_t *pbeta,
                             const double *bvals, int64_t nb, const int32_t *cols, int64_t nr, double *y,
                             double *x, cudaStream_t st) {
  if (nsn > 0) k_reach_zero<<<(unsigned)nsn, 128, 0, st>>>(d.sn, snodes, y);
  if (nb > 0) k_reach_scatter<<<(unsigned)((nb + THREADS - 1) / THREADS), THREADS, 0, st>>>(pbeta, bvals, nb, y);
  static const std::vector<Launch> none;
  cudaError_t e = run_sweeps<double, double>(d, fwd, none, Lx, Linv, 1, y, st, nullptr, Batch());
  if (e != cudaSuccess) return e;
  if (nr > 0) k_reach_gather<<<(unsigned)((nr + THREADS - 1) / THREADS), THREADS, 0, st>>>(cols, nr, y, x);
  return cudaGetLastError();
}

cudaError_t pivot_ratio(const double *piv, int64_t n, const double *Ax, int64_t axstride, const int64_t *dpos,
                        int32_t nbatch, PivotInfo *out, cudaStream_t st) {
  if (n == 0 || nbatch < 1) return cudaSuccess;
  k_pivot_ratio<<<(unsigned)nbatch, 1024, 0, st>>>(piv, n, Ax, axstride, dpos, out);
  return cudaGetLastError();
}

template <typename V>
cudaError_t permute_in(const DevPlan &d, int nrhs, const double *B, int64_t ldb, V *y, cudaStream_t st) {
  if (d.n == 0 || nrhs == 0) return cudaSuccess;
  k_perm_in<V><<<grid_for(d.n * nrhs, THREADS), THREADS, 0, st>>>(d.perm, B, ldb, y, d.n, nrhs, Batch());
  return cudaGetLastError();
}

template <typename V>
cudaError_t permute_out(const DevPlan &d, int nrhs, const V *y, double *X, int64_t ldx, cudaStream_t st) {
  if (d.n == 0 || nrhs == 0) return cudaSuccess;
  k_perm_out<V><<<grid_for(d.n * nrhs, THREADS), THREADS, 0, st>>>(d.perm, y, X, ldx, d.n, nrhs, Batch());
  return cudaGetLastError();
}

template cudaError_t prepare_solve<double, double>();
template cudaError_t prepare_solve<float, float>();
template cudaError_t prepare_factor<double>();
template cudaError_t prepare_factor<float>();
template cudaError_t run_factor<double>(const DevPlan &, const std::vector<Launch> &, const double *,
                                        double *, double *, long long *, cudaStream_t, LaunchTrace *,
                                        const Batch &, const TwoStreams *);
template cudaError_t run_factor<float>(const DevPlan &, const std::vector<Launch> &, const double *,
                                       float *, float *, long long *, cudaStream_t, LaunchTrace *,
                                       const Batch &, const TwoStreams *);
template cudaError_t run_solve<double>(const DevPlan &, const std::vector<Launch> &,
                                       const std::vector<Launch> &, const double *, const double *, int,
                                       const double *, int64_t, double *, int64_t, double *,
                                       cudaStream_t, LaunchTrace *, const Batch &);
template cudaError_t run_sweeps<float, float>(const DevPlan &, const std::vector<Launch> &,
                                              const std::vector<Launch> &, const float *, const float *, int,
                                              float *, cudaStream_t, LaunchTrace *, const Batch &);
template cudaError_t run_sweeps<double, double>(const DevPlan &, const std::vector<Launch> &,
                                                const std::vector<Launch> &, const double *, const double *,
                                                int, double *, cudaStream_t, LaunchTrace *, const Batch &);
template cudaError_t permute_in<double>(const DevPlan &, int, const double *, int64_t, double *, cudaStream_t);
template cudaError_t permute_out<double>(const DevPlan &, int, const double *, double *, int64_t, cudaStream_t);

}  // namespace sym
