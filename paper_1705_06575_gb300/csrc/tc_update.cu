// tc_update.cu — external update of FP32 factors on the tensor cores (tcgen05, kind::tf32).
//
// The left-looking update of Sec. 3.2 restricted to one 64 x 64 tile (bi, bj) of supernode J:
// for every descendant entry, C -= L_K(R1, :) L_K(R0, :)^T scattered through the relative maps.
// Here each entry's two operands are expanded to the tile's coordinates while they are staged in
// shared memory (row a of the entry lands at tile row rel(a); rows the entry does not touch are
// zero), so every entry of the tile accumulates in the tile's coordinates: in tensor memory for
// a few chunks at a time, then in FP32 registers, and the tile is written once.
//
// Precision. An FP32 value x is split into two TF32 values hi = tf32(x) and lo = tf32(x - hi)
// (|x - hi - lo| <= 2^-22 |x|). The A operand is staged as the 128-row matrix [A_hi; A_lo] and
// multiplied by B_hi and by B_lo (two M = 128, N = 64, K = 8 MMAs per step): rows 0-63 of the
// accumulator receive A_hi B^T, rows 64-127 A_lo B^T, and their sum is A B^T with all four
// partial products, each formed exactly.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "tc.cuh"

namespace sym {
namespace {

constexpr int TC_THREADS = 128;
constexpr uint32_t A_BYTES = 128 * tc::KC * 4;  // [A_hi; A_lo]: 16 KB
constexpr uint32_t B_BYTES = 64 * tc::KC * 4;   // B_hi or B_lo: 8 KB
constexpr uint32_t STAGE_BYTES = A_BYTES + 2 * B_BYTES;
constexpr int NSTAGE = 2;
constexpr size_t SMEM_BYTES = NSTAGE * STAGE_BYTES + 128;  // + room to align the stages to 128 B
constexpr uint32_t TMEM_COLS = 2 * NB;  // two FP32 accumulators of 128 x 64
constexpr uint32_t IDESC = tc::idesc_tf32<128, 64>();

__device__ __forceinline__ int64_t tile_base(int32_t i, int32_t ncols, int32_t ncb) {
  return i < ncb ? (int64_t)i * NB : (int64_t)ncols + (int64_t)(i - ncb) * NB;
}
__device__ __forceinline__ int tile_rows(int32_t i, int32_t ncols, int32_t nrows, int32_t ncb) {
  const int64_t base = tile_base(i, ncols, ncb);
  const int64_t r = (i < ncb ? ncols : nrows) - base;
  return (int)(r < NB ? r : NB);
}

// Four consecutive k values (k0 + 4 kq ..) of panel row `row` of K (column-major, ld nrows),
// zero past kc or when the tile position has no row of the entry (row < 0).
__device__ __forceinline__ float4 load4(const float *Kp, int64_t ld, int row, int k0, int k, int kc) {
  float v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = (row >= 0 && k + i < kc) ? Kp[(int64_t)(k0 + k + i) * ld + row] : 0.f;
  return make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void split_store(uint8_t *hi_buf, uint8_t *lo_buf, uint32_t o, float4 x) {
  const float4 h = make_float4(tc::to_tf32(x.x), tc::to_tf32(x.y), tc::to_tf32(x.z), tc::to_tf32(x.w));
  const float4 l = make_float4(tc::to_tf32(x.x - h.x), tc::to_tf32(x.y - h.y), tc::to_tf32(x.z - h.z),
                               tc::to_tf32(x.w - h.w));
  *reinterpret_cast<float4 *>(hi_buf + o) = h;
  *reinterpret_cast<float4 *>(lo_buf + o) = l;
}

// Entries are taken in batches of EB: their descriptors and inverse row maps (tile position ->
// entry row, or -1) are loaded into shared memory first, so that the operand loads of the next
// chunk depend on shared memory only and can be issued while the current chunk is staged.
constexpr int EB = 32;

struct EntryBatch {
  int64_t kp[EB];                       // offset of K's panel in Lx
  int32_t ld[EB], kc[EB], rlo[EB], clo[EB];
  int8_t inv_r[EB][NB], inv_c[EB][NB];  // tile row / column position -> entry row, or -1
};

// Operand values of one chunk for this thread: tile position p, k = 4 (kq0 + 2 j) + i.
struct Prefetch {
  float a[4][4], b[4][4];
};
__device__ __forceinline__ void fetch(Prefetch &f, const float *__restrict__ Lx, const EntryBatch &eb, int i, int k0,
                                      int p, int kq0) {
  const int ar = eb.inv_r[i][p], bc = eb.inv_c[i][p];
  const int64_t ld = eb.ld[i];
  const int rem = eb.kc[i] - k0;
  const float *pa = Lx + eb.kp[i] + (int64_t)k0 * ld + eb.rlo[i] + max(ar, 0);
  const float *pb = Lx + eb.kp[i] + (int64_t)k0 * ld + eb.clo[i] + max(bc, 0);
  if (rem >= tc::KC) {  // a whole chunk: only the row predicates
#pragma unroll
    for (int j = 0; j < tc::KC / 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 4 * (kq0 + 2 * j) + q;
        f.a[j][q] = ar >= 0 ? pa[k * ld] : 0.f;
        f.b[j][q] = bc >= 0 ? pb[k * ld] : 0.f;
      }
  } else {
#pragma unroll
    for (int j = 0; j < tc::KC / 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 4 * (kq0 + 2 * j) + q;
        f.a[j][q] = (ar >= 0 && k < rem) ? pa[k * ld] : 0.f;
        f.b[j][q] = (bc >= 0 && k < rem) ? pb[k * ld] : 0.f;
      }
  }
}

// One CTA (4 warps) per tile, three CTAs per SM. Thread 0 issues the MMAs; all threads stage
// operands, two stages deep: the loads of chunk c + 1 are in flight while chunk c is converted
// and stored, and the MMAs of chunk c run while chunk c + 1 is staged.
//
// Accumulation. The tensor core accumulates into tensor memory; the MMAs of SEG consecutive
// chunks (one segment, across entry boundaries: every entry lands in the tile's coordinates) go
// to one of two accumulators, which is then read back and added to FP32 registers (each thread
// owns one accumulator row: warps 0-1 the A_hi rows, warps 2-3 the A_lo rows) while the next
// segment runs on the other accumulator. Long sums are thus rounded to nearest in FP32 as in the
// SIMT form; inside the tensor core a sum runs over at most 8 SEG K = 8 steps.
// A wait that runs out (wait_ns, about a second by default) records -1 in *status and leaves the
// tile unwritten. withhold != 0 (a failure-path test) issues no MMA and no commit, so the first
// wait runs out; nothing is then in flight when the tensor memory is freed.
constexpr int SEG = 8;

__global__ void __launch_bounds__(TC_THREADS, 3) k_update_tc(const SNode *__restrict__ sn,
                                                             const UpdTask *__restrict__ tasks,
                                                             const UpdEntry *__restrict__ ents,
                                                             const int32_t *__restrict__ rel, float *__restrict__ Lx,
                                                             int64_t toff, const Batch bt, long long *status,
                                                             uint64_t wait_ns, int withhold) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ EntryBatch eb;
  __shared__ __align__(8) uint64_t mbar[NSTAGE];
  __shared__ uint32_t tmem_slot;
  Lx += blockIdx.y * bt.lx;
  status += blockIdx.y;
  uint8_t *stage0 = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const UpdTask t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.J];
  const int64_t rb = tile_base(t.bi, sj.ncols, sj.ncb);
  const int tm = tile_rows(t.bi, sj.ncols, sj.nrows, sj.ncb);
  const int cb = t.bj * NB;
  const int tn = min(NB, sj.ncols - cb);

  if (warp == 0) tc::tmem_alloc(&tmem_slot, TMEM_COLS);
  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) tc::mbar_init(&mbar[b], 1);
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t row_addr = (uint32_t)(32 * warp) << 16;

  float acc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) acc[q] = 0.f;
  // Read back accumulator `which` (the MMAs of chunk `last` and all before it complete) and add
  // it to acc. Uniform across the CTA; false when the wait ran out.
  auto drain = [&](int which, int last) -> bool {
    const bool ok = tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u, wait_ns);
    if (__syncthreads_or(!ok)) return false;
    tc::fence_after_sync();
    float v[32];
    tc::ld32(tmem + row_addr + which * NB, v);
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] += v[q];
    tc::ld32(tmem + row_addr + which * NB + 32, v);
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[32 + q] += v[q];
    tc::fence_before_sync();
    return true;
  };

  int it = 0;          // chunks issued (chunk it uses stage it % 2, accumulator (it / SEG) % 2)
  bool failed = false;
  const int p = tid & (NB - 1), kq0 = tid >> 6;
  Prefetch f;
  for (int64_t e0 = t.e0; e0 < t.e1 && !failed; e0 += EB) {
    const int ne = (int)min((int64_t)EB, t.e1 - e0);
    // (every thread has finished staging from the previous batch: a barrier follows each store)
    for (int idx = tid; idx < ne * NB; idx += TC_THREADS) {
      (&eb.inv_r[0][0])[idx] = -1;
      (&eb.inv_c[0][0])[idx] = -1;
    }
    if (tid < ne) {
      const UpdEntry E = ents[e0 + tid];
      const SNode sk = sn[E.K];
      eb.kp[tid] = sk.lx;
      eb.ld[tid] = sk.nrows;
      eb.kc[tid] = sk.ncols;
      eb.rlo[tid] = E.r_lo;
      eb.clo[tid] = E.c_lo;
    }
    __syncthreads();
    for (int idx = tid; idx < ne * NB; idx += TC_THREADS) {
      const int i = idx / NB, a = idx % NB;
      const UpdEntry &E = ents[e0 + i];
      if (a < E.m) eb.inv_r[i][rel[E.relr + a] - (int)rb] = (int8_t)a;
      if (a < E.n) eb.inv_c[i][rel[E.relc + a] - cb] = (int8_t)a;
    }
    __syncthreads();
    int i = 0, k0 = 0;
    fetch(f, Lx, eb, i, k0, p, kq0);
    while (i < ne) {
      const int st = it & 1;
      if (it >= NSTAGE) {  // the MMAs of chunk it - 2 read this stage
        const bool ok = tc::mbar_wait(&mbar[st], (uint32_t)((it >> 1) - 1) & 1u, wait_ns);
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
      }
      uint8_t *A = stage0 + st * STAGE_BYTES, *Bh = A + A_BYTES, *Bl = Bh + B_BYTES;
#pragma unroll
      for (int j = 0; j < tc::KC / 8; ++j) {
        const uint32_t o = tc::off(p, 4 * (kq0 + 2 * j));
        split_store(A, A + tc::off(NB, 0), o, make_float4(f.a[j][0], f.a[j][1], f.a[j][2], f.a[j][3]));
        split_store(Bh, Bl, o, make_float4(f.b[j][0], f.b[j][1], f.b[j][2], f.b[j][3]));
      }
      tc::fence_smem_to_async();
      const int kc_now = min(tc::KC, eb.kc[i] - k0);
      // advance to the next chunk of this batch and start its loads
      k0 += tc::KC;
      if (k0 >= eb.kc[i]) {
        ++i;
        k0 = 0;
      }
      if (i < ne) fetch(f, Lx, eb, i, k0, p, kq0);
      __syncthreads();
      const int seg = it / SEG;
      if (tid == 0 && !withhold) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_addr(A), bh0 = tc::smem_addr(Bh), bl0 = tc::smem_addr(Bl);
        const uint32_t d = tmem + (uint32_t)(seg & 1) * NB;
        uint32_t accumulate = it % SEG != 0;
        for (int ks = 0; ks < (kc_now + 7) / 8; ++ks) {
          const uint32_t o = ks * tc::KSTEP;
          tc::mma_tf32(d, tc::desc(a0 + o), tc::desc(bh0 + o), IDESC, accumulate);
          tc::mma_tf32(d, tc::desc(a0 + o), tc::desc(bl0 + o), IDESC, 1u);
          accumulate = 1u;
        }
        tc::commit(&mbar[st]);
      }
      ++it;
      // a new segment just started on the other accumulator: add up the finished one
      if ((it - 1) % SEG == 0 && it > 1 && !drain((seg - 1) & 1, it - 2)) {
        failed = true;
        break;
      }
    }
  }
  // (it and failed are uniform across the CTA.) The open segment ends with the last chunk.
  if (!failed && it > 0 && !drain(((it - 1) / SEG) & 1, it - 1)) failed = true;
  if (failed && it > 0) {  // let the MMAs in flight finish (bounded) before the memory is freed
    const int last = it - 1;
    tc::mbar_wait(&mbar[last & 1], (uint32_t)(last >> 1) & 1u, wait_ns);
    __syncthreads();
    if (tid == 0) atomicMin(status, -1ll);
  } else if (it > 0) {
    float *red = reinterpret_cast<float *>(stage0);  // [col][row]: the A_lo rows' sums
    if (warp >= 2) {
      const int r = 32 * (warp - 2) + lane;
#pragma unroll
      for (int q = 0; q < NB; ++q) red[q * (NB + 1) + r] = acc[q];
    }
    __syncthreads();
    if (warp < 2) {
      const int r = 32 * warp + lane;
      if (r < tm) {
        float *C = Lx + sj.lx + (int64_t)cb * sj.nrows + rb + r;
#pragma unroll
        for (int q = 0; q < NB; ++q)
          if (q < tn) C[(int64_t)q * sj.nrows] -= acc[q] + red[q * (NB + 1) + r];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, TMEM_COLS);
  }
}

}  // namespace

cudaError_t prepare_update_tc() {
  return cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
}

cudaError_t launch_update_tc(dim3 grid, cudaStream_t st, int prio, const DevPlan &d, float *Lx, int64_t toff,
                             const Batch &bt, long long *status) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = grid;
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_update_tc, d.sn, d.upd_tasks, d.upd_entries, d.rel, Lx, toff, bt, status,
                            d.tc_wait_ns, (int)d.tc_withhold);
}

}  // namespace sym
