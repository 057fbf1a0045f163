// tc_update.cu — external update of FP32 factors on the tensor cores (tcgen05, kind::tf32).
//
// The left-looking update of Sec. 3.2 restricted to one 64 x 64 tile (bi, bj) of supernode J:
// for every descendant entry, C -= L_K(R1, :) L_K(R0, :)^T scattered through the relative maps.
// Each entry is a compact GEMM: its m rows R1 and n rows R0 are contiguous rows of K's panel, so
// they are staged as they are (rows 0..m-1 and 0..n-1 of the operands) from K's TF32 split copy,
// which the TRSM kernels wrote once, transposed (each row's k values contiguous) and already
// split, when K's panel became final. The tensor core forms the m x n product in tensor memory;
// the relative maps are applied only on the way out, when the product is subtracted from the
// tile, which sits in shared memory for the whole CTA and is written back once.
//
// Precision. An FP32 value x is split into two TF32 values hi = tf32(x) and lo = tf32(x - hi)
// (|x - hi - lo| <= 2^-22 |x|). The A operand is staged as the 128-row matrix [A_hi; A_lo] and
// multiplied by B_hi and by B_lo (two M = 128, K = 8 MMAs per step, N = n rounded up to 16):
// accumulator rows 0-63 receive A_hi B^T, rows 64-127 A_lo B^T, all four partial products formed
// exactly. Sums run in tensor memory over at most SEG chunks (256 values of k) and are then
// added in FP32 registers (a long sum inside the tensor core loses accuracy), as in the SIMT form.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "tc.cuh"

namespace sym {
namespace {

constexpr int TC_THREADS = 128;
// Operand chunks of KC = 16 values of k, K-major core matrices without swizzle (8 rows x 16 bytes
// each; the next 4 values of k LBO = 128 bytes on, the next 8 rows SBO = 512 bytes on), in
// NSTAGE = 4 stages: the copies of three chunks are in flight while one chunk's MMAs run.
constexpr int KC = 16;
constexpr uint32_t LBO = 128, SBO = (KC / 4) * 128;
constexpr uint32_t A_BYTES = 128 * KC * 4;      // [A_hi; A_lo]: 8 KB
constexpr uint32_t B_BYTES = 64 * KC * 4;       // B_hi or B_lo: 4 KB
constexpr uint32_t STAGE_BYTES = A_BYTES + 2 * B_BYTES;
constexpr int NSTAGE = 4;
constexpr int TILE_LD = NB + 1;                 // the tile in shared memory, [col][row]
constexpr size_t SMEM_BYTES = NSTAGE * STAGE_BYTES + 128 + sizeof(float) * NB * TILE_LD;
constexpr uint32_t TMEM_COLS = 2 * NB;          // two FP32 accumulators of 128 x 64
constexpr int SEG = 16;                         // chunks per tensor-memory sum (256 values of k)

// Byte offset of element (row r, k) of an operand chunk.
__device__ __forceinline__ uint32_t off(int r, int k) {
  return (uint32_t)(r >> 3) * SBO + (uint32_t)(k >> 2) * LBO + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ int64_t tile_base(int32_t i, int32_t ncols, int32_t ncb) {
  return i < ncb ? (int64_t)i * NB : (int64_t)ncols + (int64_t)(i - ncb) * NB;
}
__device__ __forceinline__ int tile_rows(int32_t i, int32_t ncols, int32_t nrows, int32_t ncb) {
  const int64_t base = tile_base(i, ncols, ncb);
  const int64_t r = (i < ncb ? ncols : nrows) - base;
  return (int)(r < NB ? r : NB);
}

// kind::tf32 instruction descriptor with M = 128 and n rounded up to a multiple of 16.
__device__ __forceinline__ uint32_t idesc_for(int n) {
  const uint32_t N = (uint32_t)((n + 15) & ~15);
  return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Entries are taken in batches of EB: their descriptors and relative maps are loaded into shared
// memory first, so that staging and the output side depend on shared memory only.
constexpr int EB = 32;
struct EntryBatch {
  int64_t a_off[EB];   // offset of the entry's first R1 row in K's split copies
  int64_t b_off[EB];   // offset of its first R0 row
  int32_t pitch[EB];   // row length of K's split copies
  int32_t nch[EB];     // chunks of KC values of k
  int32_t m[EB], n[EB];
  int8_t prow[EB][NB], pcol[EB][NB];  // tile row / column of the entry's row a / column b
};

// Issue the copies of chunk c of entry i into a stage: rows of [A_hi; A_lo] and B_hi, B_lo, in
// 16-byte units (4 values of k), each landing in its K-major core-matrix position. Thread t copies
// unit q = t % 4 of rows t / 4 and t / 4 + 32 of each of the four operands.
__device__ __forceinline__ void stage_chunk(uint8_t *stage, const float *__restrict__ shi,
                                            const float *__restrict__ slo, const EntryBatch &eb, int i, int c,
                                            int tid) {
  const uint32_t A = tc::smem_addr(stage), Bh = A + A_BYTES, Bl = Bh + B_BYTES;
  const int m = eb.m[i], n = eb.n[i], q = tid & 3, r0 = tid >> 2;
  const int64_t pitch = eb.pitch[i], k = (int64_t)c * KC + 4 * q;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = r0 + 32 * h;
    if (r < m) {
      const int64_t o = eb.a_off[i] + r * pitch + k;
      cp_async16(A + off(r, 4 * q), shi + o);
      cp_async16(A + off(r + 64, 4 * q), slo + o);
    }
    if (r < n) {
      const int64_t o = eb.b_off[i] + r * pitch + k;
      cp_async16(Bh + off(r, 4 * q), shi + o);
      cp_async16(Bl + off(r, 4 * q), slo + o);
    }
  }
}

// One CTA (4 warps) per tile, two CTAs per SM. Every thread stages, thread 0 issues the MMAs, all
// threads read the accumulators back. The tile's chunks (every entry's chunks in entry order)
// form one sequence: the copies of the next NSTAGE - 1 chunks are in flight while the MMAs of a
// chunk run.
// A segment (at most SEG chunks of one entry) accumulates in one of two tensor-memory
// accumulators; once the MMAs of the next segment are issued, the finished segment is read back
// into FP32 registers (each thread one accumulator row: warps 0-1 the A_hi rows, warps 2-3 the
// A_lo rows), and an entry's last segment is then subtracted from the tile through the entry's
// relative maps (hi rows first, then lo rows, so no two threads write one element at once).
// Waits are bounded (wait_ns, about a second by default): one that runs out records -1 in *status
// and leaves the tile unwritten. withhold != 0 (a failure-path test) issues no MMA and no commit,
// so the first wait runs out; nothing is then in flight when the tensor memory is freed.
__global__ void __launch_bounds__(TC_THREADS, 2) k_update_tc(const SNode *__restrict__ sn,
                                                             const UpdTask *__restrict__ tasks,
                                                             const UpdEntry *__restrict__ ents,
                                                             const int32_t *__restrict__ rel, float *__restrict__ Lx,
                                                             const float *__restrict__ shi,
                                                             const float *__restrict__ slo, int64_t toff,
                                                             const Batch bt, long long *status, uint64_t wait_ns,
                                                             int withhold) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ EntryBatch eb;
  __shared__ __align__(8) uint64_t mbar[NSTAGE];
  __shared__ uint32_t tmem_slot;
  Lx += blockIdx.y * bt.lx;
  shi += blockIdx.y * bt.sx;
  slo += blockIdx.y * bt.sx;
  status += blockIdx.y;
  uint8_t *stage0 = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *tile = reinterpret_cast<float *>(stage0 + NSTAGE * STAGE_BYTES);  // [col][row], TILE_LD
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const UpdTask t = tasks[toff + blockIdx.x];
  const SNode sj = sn[t.J];
  const int64_t rb = tile_base(t.bi, sj.ncols, sj.ncb);
  const int tm = tile_rows(t.bi, sj.ncols, sj.nrows, sj.ncb);
  const int cb = t.bj * NB;
  const int tn = min(NB, sj.ncols - cb);
  float *C = Lx + sj.lx + (int64_t)cb * sj.nrows + rb;

  if (warp == 0) tc::tmem_alloc(&tmem_slot, TMEM_COLS);
  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) tc::mbar_init(&mbar[b], 1);
    tc::mbar_init_fence();
  }
  for (int idx = tid; idx < tm * tn; idx += TC_THREADS) {
    const int r = idx % tm, c = idx / tm;
    tile[c * TILE_LD + r] = C[(int64_t)c * sj.nrows + r];
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t row_addr = (uint32_t)(32 * warp) << 16;
  const int arow = 32 * (warp & 1) + lane;  // this thread's accumulator row within A_hi or A_lo

  float racc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) racc[q] = 0.f;

  // Chunk j of the tile uses stage j % NSTAGE and commits to mbar[j % NSTAGE], whose phase j / NSTAGE
  // completes with it. Wait (bounded, uniform across the CTA) until chunk j's MMAs completed.
  auto wait_chunk = [&](int j) -> bool {
    const bool ok = tc::mbar_wait(&mbar[j % NSTAGE], (uint32_t)(j / NSTAGE) & 1u, wait_ns);
    return !__syncthreads_or(!ok);
  };
  // Read back accumulator `which` once the MMAs of chunk `last` (and all before) completed, and
  // add its first n columns to racc; with `scatter`, subtract racc from the tile through the
  // entry's maps and clear it. Uniform across the CTA; false when the wait ran out.
  auto drain = [&](int which, int last, int ei, bool scatter) -> bool {
    if (!wait_chunk(last)) return false;
    tc::fence_after_sync();
    const int n = eb.n[ei];
    float v[32];
    tc::ld32(tmem + row_addr + which * NB, v);
#pragma unroll
    for (int q = 0; q < 32; ++q) racc[q] += v[q];
    if (n > 32) {
      tc::ld32(tmem + row_addr + which * NB + 32, v);
#pragma unroll
      for (int q = 0; q < 32; ++q) racc[32 + q] += v[q];
    }
    tc::fence_before_sync();
    if (scatter) {
      const int m = eb.m[ei];
      for (int phase = 0; phase < 2; ++phase) {
        if ((warp >> 1) == phase && arow < m) {
          const int r = eb.prow[ei][arow];
#pragma unroll
          for (int q = 0; q < NB; ++q)
            if (q < n) tile[eb.pcol[ei][q] * TILE_LD + r] -= racc[q];
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) racc[q] = 0.f;
    }
    return true;
  };

  int it = 0;   // chunks issued over the whole tile
  int sg = -1;  // segments started (segment sg uses accumulator sg & 1)
  bool failed = false;
  // the open segment: its entry (batch slot) and last chunk
  int seg_entry = -1, seg_last = -1;
  for (int64_t e0 = t.e0; e0 < t.e1 && !failed; e0 += EB) {
    const int ne = (int)min((int64_t)EB, t.e1 - e0);
    // (the previous batch's chunks have all completed: its maps and stages are free)
    if (tid < ne) {
      const UpdEntry E = ents[e0 + tid];
      const SNode sk = sn[E.K];
      const int64_t pitch = split_pitch(sk.ncols);
      eb.a_off[tid] = sk.sx + (int64_t)E.r_lo * pitch;
      eb.b_off[tid] = sk.sx + (int64_t)E.c_lo * pitch;
      eb.pitch[tid] = (int32_t)pitch;
      eb.nch[tid] = (sk.ncols + KC - 1) / KC;
      eb.m[tid] = E.m;
      eb.n[tid] = E.n;
    }
    for (int idx = tid; idx < ne * NB; idx += TC_THREADS) {
      const int i = idx / NB, a = idx % NB;
      const UpdEntry &E = ents[e0 + i];
      if (a < E.m) eb.prow[i][a] = (int8_t)(rel[E.relr + a] - (int)rb);
      if (a < E.n) eb.pcol[i][a] = (int8_t)(rel[E.relc + a] - cb);
    }
    __syncthreads();
    // The copies run NSTAGE - 1 chunks ahead of the MMAs: (si, sc) is the next chunk to stage,
    // `staged` its index in the tile's sequence. Every call commits one copy group (an empty one
    // once the batch is exhausted), so chunk it's group is complete when at most NSTAGE - 2
    // newer ones are pending.
    int si = 0, sc = 0, staged = it;
    auto stage_next = [&]() {
      if (si < ne) {
        stage_chunk(stage0 + (staged % NSTAGE) * STAGE_BYTES, shi, slo, eb, si, sc, tid);
        if (++sc >= eb.nch[si]) {
          ++si;
          sc = 0;
        }
        ++staged;
      }
      cp_async_commit();
    };
    for (int p = 0; p < NSTAGE - 1; ++p) stage_next();
    int i = 0, c = 0;
    while (i < ne) {
      int ni = i, nc = c + 1;
      if (nc >= eb.nch[i]) {
        ++ni;
        nc = 0;
      }
      cp_async_wait<NSTAGE - 2>();
      tc::fence_smem_to_async();
      __syncthreads();
      const bool new_seg = c % SEG == 0;
      if (new_seg) ++sg;
      if (tid == 0 && !withhold) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_addr(stage0 + (it % NSTAGE) * STAGE_BYTES);
        const uint32_t bh0 = a0 + A_BYTES, bl0 = bh0 + B_BYTES;
        const uint32_t d = tmem + (uint32_t)(sg & 1) * NB;
        const uint32_t idesc = idesc_for(eb.n[i]);
        uint32_t accumulate = new_seg ? 0u : 1u;
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t o = ks * 2 * LBO;  // K = 8: two core matrices along k
          tc::mma_tf32(d, tc::desc(a0 + o, LBO, SBO), tc::desc(bh0 + o, LBO, SBO), idesc, accumulate);
          tc::mma_tf32(d, tc::desc(a0 + o, LBO, SBO), tc::desc(bl0 + o, LBO, SBO), idesc, 1u);
          accumulate = 1u;
        }
        tc::commit(&mbar[it % NSTAGE]);
      }
      const bool drain_prev = new_seg && seg_entry >= 0;
      // the stage of chunk it - 1 takes the chunk NSTAGE - 1 ahead once its MMAs completed
      if (it >= 1 && (si < ne || drain_prev) && !wait_chunk(it - 1)) {
        failed = true;
        break;
      }
      stage_next();
      // a new segment started on the other accumulator: read the finished one back (and
      // subtract it from the tile when it closed its entry)
      if (drain_prev && !drain((sg - 1) & 1, seg_last, seg_entry, seg_entry != i)) {
        failed = true;
        break;
      }
      seg_entry = i;
      seg_last = it;
      ++it;
      i = ni;
      c = nc;
    }
    // the batch's last segment closes its entry: drain it before the batch's maps are replaced
    if (!failed && seg_entry >= 0) {
      if (!drain(sg & 1, seg_last, seg_entry, true)) failed = true;
      seg_entry = -1;
    }
    cp_async_wait<0>();
    __syncthreads();
  }
  if (failed && it > 0) {  // let the MMAs in flight finish (bounded) before the memory is freed
    const int last = it - 1;
    tc::mbar_wait(&mbar[last % NSTAGE], (uint32_t)(last / NSTAGE) & 1u, wait_ns);
    cp_async_wait<0>();
    __syncthreads();
    if (tid == 0) atomicMin(status, -1ll);
  } else {
    for (int idx = tid; idx < tm * tn; idx += TC_THREADS) {
      const int r = idx % tm, c = idx / tm;
      C[(int64_t)c * sj.nrows + r] = tile[c * TILE_LD + r];
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
  return cudaLaunchKernelEx(&cfg, k_update_tc, d.sn, d.upd_tasks, d.upd_entries, d.rel, Lx, (const float *)d.shi,
                            (const float *)d.slo, toff, bt, status, d.tc_wait_ns, (int)d.tc_withhold);
}

}  // namespace sym
