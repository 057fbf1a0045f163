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
// (|x - hi - lo| <= 2^-22 |x|). The A operand is staged as the 128-row matrix [A_hi; A_lo]; per
// K = 8 step three MMAs (M = 128, N = n rounded up to 16) add A_hi B_hi^T, A_hi B_lo^T and
// A_lo B_hi^T, each formed exactly, to accumulator rows 0-63 (A_lo B_lo^T, below 2^-22 |A| |B|,
// is left out). Sums run in tensor memory over at most SEG chunks (256 values of k) and are then
// added in FP32 registers (a long sum inside the tensor core loses accuracy), as in the SIMT form.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "tc.cuh"

namespace sym {
namespace {

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

// Copies of chunk c (KC values of k from c KC on) of one entry into a stage, issued by the 32 lanes
// of the producer warp: 16-byte units (4 values of k) of the rows of [A_hi; A_lo] and B_hi, B_lo,
// each landing in its K-major core-matrix position. Unit u of an operand: row u / 4, 4 (u % 4) on.
__device__ __forceinline__ void stage_chunk(uint8_t *stage, const float *__restrict__ shi,
                                            const float *__restrict__ slo, int64_t a_off, int64_t b_off,
                                            int64_t pitch, int m, int n, int c, int lane) {
  const uint32_t A = tc::smem_addr(stage), Bh = A + A_BYTES, Bl = Bh + B_BYTES;
  const int64_t k0 = (int64_t)c * KC;
  for (int u = lane; u < 4 * m; u += 32) {
    const int r = u >> 2, q = u & 3;
    const int64_t o = a_off + r * pitch + k0 + 4 * q;
    cp_async16(A + off(r, 4 * q), shi + o);
    cp_async16(A + off(r + 64, 4 * q), slo + o);
  }
  for (int u = lane; u < 4 * n; u += 32) {
    const int r = u >> 2, q = u & 3;
    const int64_t o = b_off + r * pitch + k0 + 4 * q;
    cp_async16(Bh + off(r, 4 * q), shi + o);
    cp_async16(Bl + off(r, 4 * q), slo + o);
  }
}

// One CTA per tile, two CTAs per SM, with warp roles (no CTA-wide barrier inside the loop):
//   warp 2 (producer): copies each chunk into the next free stage; a stage is free once the MMAs
//     of the chunk it held completed (empty[st], committed by the MMA thread); its lanes arrive on
//     full[st] when their copies have landed;
//   warp 3, lane 0 (MMA): per chunk, waits for full[st], issues 3 x (KC / 8) MMAs into the
//     segment's accumulator (two alternate; it waits for the epilogue to have read one before
//     reusing it, acc_empty) and commits to empty[st], and at a segment's end to acc_full;
//   warps 0-1 (epilogue; warp w reads tensor-memory lanes 32 w .. 32 w + 31, one accumulator row
//     per thread): per segment, add the accumulator to FP32 registers and release it; after an
//     entry's last segment, subtract the sum from the tile through the entry's relative maps, then
//     meet at a barrier of the two warps (the next entry may write the same tile elements).
// Per K = 8 step the accumulator rows 0-63 receive A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T: the
// third MMA takes its A operand from the A_lo rows (rows 64.. of the staged [A_hi; A_lo], its rows
// beyond 64 then read the B operands and land in accumulator rows 64-127, which nobody reads). The
// dropped A_lo B_lo^T is below 2^-22 |A| |B|, the size of the split's own error.
// A segment is at most SEG chunks of one entry. Every wait is bounded (wait_ns; about a second by
// default) and also ends when another warp has given up; then -1 goes to *status, the tile is left
// unwritten, and the tensor memory is freed once every issued MMA has completed. withhold != 0 (a
// failure-path test) issues no MMA and no commit, so the first waits run out.
constexpr int EPI_WARPS = 2, PRODUCER = 2, MMA_WARP = 3;
constexpr int TC_BLOCK = 32 * 4;
constexpr uint32_t LO_ROWS = 8 * SBO;  // byte offset of row 64 (the A_lo rows) in an A operand

__global__ void __launch_bounds__(TC_BLOCK, 2) k_update_tc(const SNode *__restrict__ sn,
                                                           const UpdTask *__restrict__ tasks,
                                                           const UpdEntry *__restrict__ ents,
                                                           const int32_t *__restrict__ rel, float *__restrict__ Lx,
                                                           const float *__restrict__ shi,
                                                           const float *__restrict__ slo, int64_t toff,
                                                           const Batch bt, long long *status, uint64_t wait_ns,
                                                           int withhold) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], acc_full[2], acc_empty[2], done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int fail;
  __shared__ int8_t pcol[2][NB];  // tile column of each column of an entry (by entry parity)
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
  if (tid == 32) {
    for (int b = 0; b < NSTAGE; ++b) {
      tc::mbar_init(&full[b], 32);
      tc::mbar_init(&empty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], EPI_WARPS);
    }
    tc::mbar_init(&done, 1);
    fail = 0;
    tc::mbar_init_fence();
  }
  for (int idx = tid; idx < tm * tn; idx += TC_BLOCK) {
    const int r = idx % tm, c = idx / tm;
    tile[c * TILE_LD + r] = C[(int64_t)c * sj.nrows + r];
  }
  if (t.e0 < t.e1 && tid < NB) {  // the first entry's column map
    const UpdEntry E0 = ents[t.e0];
    if (tid < E0.n) pcol[0][tid] = (int8_t)(rel[E0.relc + tid] - cb);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  auto give_up = [&]() { fail = 1; };

  if (warp == PRODUCER) {
    int j = 0;  // chunk index over the tile's sequence
    UpdEntry En = t.e0 < t.e1 ? ents[t.e0] : UpdEntry{};  // the next entry, loaded one ahead
    for (int64_t e = t.e0; e < t.e1 && !fail; ++e) {
      const UpdEntry E = En;
      const SNode sk = sn[E.K];
      if (e + 1 < t.e1) En = ents[e + 1];
      const int64_t pitch = split_pitch(sk.ncols);
      const int nch = (sk.ncols + KC - 1) / KC;
      for (int c = 0; c < nch; ++c, ++j) {
        const int st = j % NSTAGE;
        const bool free_st =
            j < NSTAGE || tc::mbar_wait_or_abort(&empty[st], (uint32_t)(j / NSTAGE - 1) & 1u, wait_ns, &fail);
        if (!__all_sync(0xffffffffu, free_st)) {  // the lanes agree
          give_up();
          break;
        }
        stage_chunk(stage0 + st * STAGE_BYTES, shi, slo, sk.sx + (int64_t)E.r_lo * pitch,
                    sk.sx + (int64_t)E.c_lo * pitch, pitch, E.m, E.n, c, lane);
        tc::cp_async_arrive(&full[st]);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      int j = 0, seg = 0;
      bool issued = false;
      // the next entry's column count and width, loaded one entry ahead
      int nxt_n = 0, nxt_k = 0;
      if (t.e0 < t.e1) {
        const UpdEntry E0 = ents[t.e0];
        nxt_n = E0.n;
        nxt_k = sn[E0.K].ncols;
      }
      for (int64_t e = t.e0; e < t.e1 && !fail; ++e) {
        const int nch = (nxt_k + KC - 1) / KC;
        const uint32_t idesc = idesc_for(nxt_n);
        if (e + 1 < t.e1) {
          const UpdEntry E1 = ents[e + 1];
          nxt_n = E1.n;
          nxt_k = sn[E1.K].ncols;
        }
        for (int c = 0; c < nch; ++c, ++j) {
          const int st = j % NSTAGE, acc = seg & 1;
          if (!tc::mbar_wait_or_abort(&full[st], (uint32_t)(j / NSTAGE) & 1u, wait_ns, &fail)) {
            give_up();
            break;
          }
          const bool first = c % SEG == 0;  // a segment starts: its accumulator must be free
          if (first && seg >= 2 &&
              !tc::mbar_wait_or_abort(&acc_empty[acc], (uint32_t)(seg / 2 - 1) & 1u, wait_ns, &fail)) {
            give_up();
            break;
          }
          tc::fence_smem_to_async();
          tc::fence_after_sync();
          if (!withhold) {
            const uint32_t a0 = tc::smem_addr(stage0 + st * STAGE_BYTES);
            const uint32_t bh0 = a0 + A_BYTES, bl0 = bh0 + B_BYTES;
            const uint32_t d = tmem + (uint32_t)acc * NB;
            uint32_t accumulate = first ? 0u : 1u;
            for (int ks = 0; ks < KC / 8; ++ks) {
              const uint32_t o = ks * 2 * LBO;  // K = 8: two core matrices along k
              tc::mma_tf32(d, tc::desc(a0 + o, LBO, SBO), tc::desc(bh0 + o, LBO, SBO), idesc, accumulate);
              tc::mma_tf32(d, tc::desc(a0 + o, LBO, SBO), tc::desc(bl0 + o, LBO, SBO), idesc, 1u);
              tc::mma_tf32(d, tc::desc(a0 + LO_ROWS + o, LBO, SBO), tc::desc(bh0 + o, LBO, SBO), idesc, 1u);
              accumulate = 1u;
            }
            tc::commit(&empty[st]);
            if (c % SEG == SEG - 1 || c == nch - 1) tc::commit(&acc_full[acc]);
            issued = true;
          }
          if (c % SEG == SEG - 1 || c == nch - 1) ++seg;
        }
      }
      if (issued) {  // every issued MMA completes before the tensor memory can be freed
        tc::commit(&done);
        if (!tc::mbar_wait(&done, 0u, wait_ns)) give_up();
      }
    }
  } else {  // epilogue warps 0-1: accumulator row tid
    float racc[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) racc[q] = 0.f;
    const uint32_t row_addr = (uint32_t)(32 * warp) << 16;
    int seg = 0, par = 0;
    bool go = true;  // uniform across the two epilogue warps
    UpdEntry E = t.e0 < t.e1 ? ents[t.e0] : UpdEntry{};
    int r = (t.e0 < t.e1 && tid < E.m) ? rel[E.relr + tid] - (int)rb : -1;
    for (int64_t e = t.e0; e < t.e1 && go; ++e, par ^= 1) {
      const int nch = (sn[E.K].ncols + KC - 1) / KC;
      const int nseg = (nch + SEG - 1) / SEG;
      // the next entry's maps, loaded while this one's MMAs run (its column map into the other
      // buffer, which the barrier closing this entry publishes)
      UpdEntry En = E;
      int rn = -1;
      if (e + 1 < t.e1) {
        En = ents[e + 1];
        if (tid < En.n) pcol[par ^ 1][tid] = (int8_t)(rel[En.relc + tid] - cb);
        if (tid < En.m) rn = rel[En.relr + tid] - (int)rb;
      }
      bool ok = true;
      for (int g = 0; g < nseg; ++g, ++seg) {
        const int acc = seg & 1;
        // the lanes agree before the warp-wide tensor-memory loads
        if (!__all_sync(0xffffffffu, tc::mbar_wait_or_abort(&acc_full[acc], (uint32_t)(seg / 2) & 1u, wait_ns,
                                                            &fail))) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        float v[32];
        tc::ld32(tmem + row_addr + acc * NB, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) racc[q] += v[q];
        if (E.n > 32) {
          tc::ld32(tmem + row_addr + acc * NB + 32, v);
#pragma unroll
          for (int q = 0; q < 32; ++q) racc[32 + q] += v[q];
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
      }
      if (!ok) give_up();
      if (ok && r >= 0) {
#pragma unroll
        for (int q = 0; q < NB; ++q)
          if (q < E.n) tile[pcol[par][q] * TILE_LD + r] -= racc[q];
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) racc[q] = 0.f;
      // the two warps continue together, unless either has seen a failure
      uint32_t stop;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\t"
          "setp.ne.u32 p, %1, 0;\n\t"
          "barrier.cta.red.or.pred q, 1, %2, p;\n\t"
          "selp.u32 %0, 1, 0, q;\n\t}"
          : "=r"(stop)
          : "r"((uint32_t)(fail != 0 || !ok)), "n"(32 * EPI_WARPS)
          : "memory");
      go = stop == 0;
      E = En;
      r = rn;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (fail) {
    if (tid == 0) atomicMin(status, -1ll);
  } else {
    for (int idx = tid; idx < tm * tn; idx += TC_BLOCK) {
      const int r = idx % tm, c = idx / tm;
      C[(int64_t)c * sj.nrows + r] = tile[c * TILE_LD + r];
    }
  }
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
  cfg.blockDim = dim3(TC_BLOCK, 1, 1);
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
