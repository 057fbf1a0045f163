// plan.h — the symbolic plan that the host inspector builds once per sparsity pattern and the
// CUDA kernels consume. Internal to the library (the public interface is include/sym.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "sym.h"

namespace sym {

// Edge of the square tiles that the numeric kernels work on (rows and columns of a supernode's
// panel are cut into tiles of NB; see row_tile_base below).
constexpr int NB = 64;
// Columns per CTA of the backward solve's gather from the rows below a diagonal block.
constexpr int SOLVE_BG = 16;
// Columns per CTA of the forward solve's push from a solved supernode to the rows below its
// diagonal block (a supernode with more columns writes one partial result per chunk).
constexpr int SOLVE_CW = 512;
// Right-hand sides per pass of the solve kernels (the buffer t holds this many).
constexpr int SOLVE_MAXRHS = 8;
// Order bound of the tiles that the small-tile kernel variants take.
constexpr int SMALL_TILE = 32;
// Batches: full-tile update launches whose entries have at most this many output elements on
// average default to the warp-per-(tile, matrix) form (measured on a 512 x 128^2 9-point batch:
// 1.35-4.7x faster than one CTA per tile at 34-134 elements, about equal at 175-230).
constexpr int BATCH_WARP_ELEMS = 160;
// Narrow levels in one launch (k_panel_b): a level whose supernodes all have at most SMALL_TILE
// columns factors each panel (POTRF of the diagonal block, TRSM of the rows below it, TRTRI of
// the diagonal block) in one warp per (supernode, 32 / G matrices), G lanes per matrix, the
// warp's panels in shared memory; a single matrix takes G = 32. panel_lanes gives a batch's G for
// a level's largest panel (pmax elements) and widest supernode (ncmax columns): the smallest of
// 1, 2, 4, 8 whose shared memory per warp is at most PANEL_SMEM_SOFT (six warps per SM), else 8
// if that fits PANEL_SMEM_HARD (four warps per SM, one per scheduler), else 0 (the batch keeps
// the level's separate launches). f32: FP32 panels (the FP64 pivot chain and the FP64 inverse
// need their own arrays).
constexpr int PANEL_SMEM_SOFT = 36 * 1024;
constexpr int PANEL_ONE_MIN = 8 * 152;  // see symbolic.cpp (fused factor levels of one matrix)
constexpr int PANEL_SMEM_HARD = 56 * 1024;
inline int64_t panel_smem_bytes(int64_t pmax, int64_t ncmax, bool f32, int g) {
  const int64_t stride = g == 1 ? 33 : 32 / g;  // panel element stride (padded with one matrix per lane)
  return stride * pmax * (f32 ? 4 : 8) + (32 / g) * (ncmax * 8 + (f32 ? ncmax * 8 + ncmax * (ncmax - 1) / 2 * 8 : 0));
}
inline int panel_lanes(int64_t pmax, int64_t ncmax, bool f32) {
  for (int g = 1; g <= 8; g *= 2)
    if (panel_smem_bytes(pmax, ncmax, f32, g) <= PANEL_SMEM_SOFT) return g;
  return panel_smem_bytes(pmax, ncmax, f32, 8) <= PANEL_SMEM_HARD ? 8 : 0;
}
// The same for the solve on such levels (k_fwd_b, k_bwd_b; batches in FP64): each warp holds its
// matrices' panels and diagonal-block inverses (pmax + ncmax^2 elements per matrix) and two
// vectors of ncmax values per matrix and right-hand side of a pass.
inline int64_t solve_panel_bytes(int64_t pmax, int64_t ncmax, int g, int nrb = 1) {
  const int64_t stride = g == 1 ? 33 : 32 / g;  // nrb: right-hand sides per pass of the kernel
  return stride * (pmax + ncmax * ncmax) * 8 + (32 / g) * 2 * nrb * ncmax * 8;
}
inline int solve_panel_lanes(int64_t pmax, int64_t ncmax) {
  for (int g = 1; g <= 8; g *= 2)
    if (solve_panel_bytes(pmax, ncmax, g) <= PANEL_SMEM_SOFT) return g;
  return solve_panel_bytes(pmax, ncmax, 8) <= PANEL_SMEM_HARD ? 8 : 0;
}
// Role of a factor launch in the fused narrow levels (PanelForm::role).
constexpr int32_t PANEL_NONE = 0, PANEL_FUSED = 1, PANEL_COVERED = 2;
struct PanelForm {
  int32_t role;   // PANEL_FUSED: the level's POTRF launch runs k_panel_b for batches;
                  // PANEL_COVERED: its TRSM and TRTRI launches, which batches then skip
  int32_t pmax;   // PANEL_FUSED: the level's largest panel, nrows x ncols elements
  int32_t ncmax;  // PANEL_FUSED: the level's widest supernode
  int32_t head;   // PANEL_FUSED and PANEL_COVERED: index of the level's PANEL_FUSED launch
};
// Lanes per matrix of a fused narrow level (pf: its PANEL_FUSED form) for nb matrices, 0 when the
// level runs as separate launches: a batch's factor by panel_lanes, its solve by
// solve_panel_lanes (FP64 only); one matrix 32 (one warp per supernode, rows spread over the
// lanes) where the panels fit.
inline int panel_lanes_for(const PanelForm &pf, unsigned nb, bool f32) {
  if (nb > 1) return panel_lanes(pf.pmax, pf.ncmax, f32);
  return panel_smem_bytes(pf.pmax, pf.ncmax, f32, 32) <= PANEL_SMEM_HARD ? 32 : 0;
}
inline int solve_lanes_for(const PanelForm &pf, unsigned nb, bool fp64) {
  if (nb > 1) return fp64 ? solve_panel_lanes(pf.pmax, pf.ncmax) : 0;
  return solve_panel_bytes(pf.pmax, pf.ncmax, 32, 8) <= PANEL_SMEM_HARD ? 32 : 0;
}
// Trailing-update GEMM CTAs resident on the whole GPU at once (3 per SM on 152 SMs): the size of
// one wave, used to split the last wave of a long launch into finer work.
constexpr int GEMM_SLOTS = 3 * 152;

// One supernode as the kernels see it. Its panel is column-major, nrows x ncols, leading
// dimension nrows, at Lx + lx. Row r of the panel is global row rows[rowp + r]; the first ncols
// rows are the supernode's own columns (the dense diagonal block).
struct SNode {
  int32_t first;  // first column
  int32_t ncols;
  int32_t nrows;
  int32_t ncb;    // column tiles = ceil(ncols / NB)
  int64_t rowp;   // offset into rows[]
  int64_t lx;     // offset into Lx
  int64_t dx;     // offset of the inverses of its diagonal tiles: tile s (order ts) is a
                  // column-major ts x ts block at dx + s * NB * NB
  int64_t tx;     // offset of its pushed products in the forward solve's buffer t: chunk ch of
                  // its columns gives t[tx + ch * (nrows - ncols) + (r - ncols)] for each row r
                  // below the diagonal block
};

// Row tiling of a panel: the diagonal block is cut at multiples of NB, and the rows below it
// (the off-diagonal block) again from row ncols, so that tile (s, s) is exactly the square
// diagonal tile of column tile s.
inline int64_t row_tile_base(int32_t i, int32_t ncols, int32_t ncb) {
  return i < ncb ? (int64_t)i * NB : (int64_t)ncols + (int64_t)(i - ncb) * NB;
}
inline int32_t row_tile_of(int64_t pos, int32_t ncols, int32_t ncb) {
  return pos < ncols ? (int32_t)(pos / NB) : ncb + (int32_t)((pos - ncols) / NB);
}
inline int32_t num_row_tiles(int32_t nrows, int32_t ncols, int32_t ncb) {
  return ncb + (int32_t)((nrows - ncols + NB - 1) / NB);
}

// One descendant contribution to one tile of an ancestor J (the left-looking update of
// Sec. 3.2 restricted to a tile): rows r_lo..r_lo+m-1 of K's panel land in the tile's rows at
// positions rel[relr + a] (positions within rows(J)), and rows c_lo..c_lo+n-1 of K's panel give
// the tile's columns at positions rel[relc + b]. Inner dimension: ncols(K).
struct UpdEntry {
  int32_t K;
  int32_t r_lo;
  int32_t c_lo;
  int32_t m;
  int32_t n;
  int32_t pad;
  int64_t relr;
  int64_t relc;
};

// A tile (bi, bj) of supernode J and the range of its UpdEntry list.
struct UpdTask {
  int32_t J;
  int32_t bi;
  int32_t bj;
  int32_t pad;
  int64_t e0;
  int64_t e1;
};

// Kernel kinds of the launch schedule.
enum Kind : int32_t {
  K_SCATTER = 0,  // zero the panels and scatter A into them (two launches)
  K_UPDATE = 1,   // external updates of tiles (UpdTask list)
  K_POTRF = 2,    // dense Cholesky of diagonal tile s (int4 {J, s, s, s})
  K_TRSM = 3,     // tile (i, s) <- tile * L_ss^-T (int4 {J, i, s, s})
  K_GEMM = 4,     // tile (i, j) -= L_is L_js^T (int4 {J, i, j, s})
  K_TRTRI = 5,    // inverse of every diagonal tile, for the solve (int4 {J, s, s, s})
  S_FGATHER = 11, // y_J(tile bj) -= sum_K L_K(rows in tile) y_K (int4 {J, bj, task, 0})
  S_FSTEP = 12,   // column tile s of J: y_i -= L_is L_ss^-1 y_s (CTAs i > s); CTA i = s writes
                  // the solved tiles s-1 (and s if last) (int4 {J, i, s, s}). A launch with
                  // cluster = 4 holds cluster tasks instead (int4 {J, i, s, 0}, s = -1 .. ncb-2):
                  // y_i -= L_is y_s with y_s already solved (s >= 0), and for i = s + 1 the
                  // solve y_i <- L_ii^-1 y_i in place
  S_FPUSH = 13,   // t_J(rows of row tile i, chunk ch) = L_J(tile rows, chunk cols) y_J(chunk cols)
                  // for the row tiles below J's diagonal block (int4 {J, i, ch, 0})
  S_BGATHER = 14, // z_J(slice) -= L_J(off rows, slice)^T z(off rows) (int4 {J, slice, 0, 0}),
                  // slices of SOLVE_BG columns
  S_BSTEP = 15,   // column tile s of J: z_i -= L_si^T L_ss^-T z_s (CTAs i < s); CTA i = s writes
                  // the solved tiles s+1 (and 0 if s = 0) (int4 {J, i, s, s}). With cluster = 4:
                  // cluster tasks {J, i, s, 0}, s = ncb .. 1: z_i -= L_si^T z_s with z_s solved
                  // (s < ncb), and for i = s - 1 the solve z_i <- L_ii^-T z_i in place
  S_FSUM = 16,    // y_g -= sum of t over the contribution list of column g, for the columns
                  // of J in block cb of 256 (int4 {J, cb, 0, 0})
  S_PERM = 17,    // y = P b and x = P^T y
  NUM_KINDS = 18,
};

struct Launch {
  int32_t kind;
  int32_t level;
  int64_t off;          // offset into the task array of this kind
  int64_t count;        // number of tasks
  int32_t cluster = 1;  // CTAs per task (a thread-block cluster) where the kernel supports it
  int32_t stream = 0;   // 0: the main (high-priority) stream, 1: the auxiliary (low-priority) one
  int32_t wait = -1;    // index of an earlier launch of this list to wait for (other stream), or -1
  int32_t tb = 0;       // SMALL_TILE: every tile of the launch has at most SMALL_TILE columns
                        // (update: rows and columns), run by the small-tile kernel variant; else 0
};

struct Int4 {
  int32_t a, b, c, d;
};

struct Plan {
  int64_t n = 0;
  int64_t nnz_a = 0;
  int64_t nnz_l = 0;
  double flops = 0.0;
  double analyze_seconds = 0.0;
  std::vector<int32_t> perm, iperm;   // final ordering
  std::vector<int32_t> parent;        // etree of P A P^T
  std::vector<int64_t> colcount;      // |L_j|
  std::vector<int32_t> fsuper;        // fundamental supernodes (first columns, +n)
  std::vector<int32_t> super;         // supernodes after amalgamation (first columns, +n)
  std::vector<int64_t> rowptr;        // nsuper+1
  std::vector<int32_t> rows;          // rows(J)
  std::vector<int32_t> sparent;       // supernodal tree
  std::vector<int64_t> descptr;       // nsuper+1
  std::vector<int32_t> desc;          // K of each pair
  std::vector<int64_t> descr0;        // first position of rows(K) >= first(J)
  std::vector<int32_t> descnin;       // rows of K inside cols(J)
  std::vector<int64_t> relptr;        // npairs+1
  std::vector<int32_t> rel;           // relative row maps
  std::vector<int32_t> level, levelptr, levellist;
  std::vector<int64_t> lxptr;         // nsuper+1; lxptr[nsuper] = storage
  int64_t dinv_storage = 0;           // entries of all diagonal-tile inverses
  std::vector<int64_t> amap;          // nnz_a: panel position of each entry of A
  // Full CSR of C = P A P^T (both triangles) for FP64 residuals of the mixed-precision path;
  // built only when requested. cmap[p] is the index of the entry of A that gives C's entry p.
  std::vector<int64_t> csr_p, csr_map;
  std::vector<int32_t> csr_i;
  std::vector<SNode> snodes;
  std::vector<UpdEntry> upd_entries;
  std::vector<UpdTask> upd_tasks;
  std::vector<Int4> tasks;            // every other kind of task
  std::vector<Launch> factor_launches;
  std::vector<int8_t> variant[2];     // per factor launch: the autotuner's kernel form (0 default),
                                      // [0] for one matrix, [1] for batches
  std::vector<int8_t> batch_warp;     // per factor launch: 1 if a batch's default form of this
                                      // full-tile update is one warp per (tile, matrix)
  std::vector<int8_t> batch_lanes;     // per factor launch: for a small-tile update, a batch's
                                      // lanes per matrix in the lanes-to-matrices form (1, 2, 4
                                      // or 8), else 0
  std::vector<PanelForm> batch_panel;  // per factor launch: fused narrow levels (batches and,
                                       // where panel_apart[0] allows, single matrices)
  std::vector<int8_t> panel_apart[2];  // per factor launch, on PANEL_FUSED ones: 1 if the
                                       // autotuner found the level faster as separate launches;
                                       // [0] one matrix, [1] batches
  std::vector<Launch> fwd_launches;
  std::vector<Launch> bwd_launches;
  // Per forward / backward solve launch, the fused narrow levels (single matrices, and batches in
  // FP64): the level's S_FSTEP (forward) or S_BSTEP (backward) launch is PANEL_FUSED and runs the
  // level's sums, steps and pushes (forward) or gathers and steps (backward) in one launch; its
  // other launches are PANEL_COVERED.
  std::vector<PanelForm> fwd_panel, bwd_panel;
  // Forward solve by pushes: t holds tsize entries per right-hand side; the contribution list of
  // column g, contrib[contrib_ptr[g] .. contrib_ptr[g+1]), names the entries of t that column g
  // subtracts (every row g below the diagonal block of a supernode, once per column chunk), in
  // ascending supernode and chunk order.
  int64_t tsize = 0;
  std::vector<int64_t> contrib_ptr;
  std::vector<int32_t> contrib;
  int32_t max_ncols = 0;
  // Algorithmic flops per kind for one factorization (solve kinds: per right-hand side): the
  // useful multiply-adds (x2), square roots and divisions, excluding the strict upper part of
  // diagonal tiles; explicit zeros of amalgamated panels are included.
  double kind_flops[NUM_KINDS] = {};
  // Useful flops of the external updates (K_UPDATE) on the exact pattern of L: the share of the
  // factor's sum of c_j^2 that descendant updates carry (no explicit zeros of amalgamation).
  double update_flops = 0.0;
  // How the ordering was obtained (SYM_ORDER_NATURAL, SYM_ORDER_GIVEN, SYM_ORDER_METHOD_MD or
  // SYM_ORDER_METHOD_ND) and, for SYM_ORDER_AUTO, the flops of both candidates.
  int32_t ordering_method = SYM_ORDER_NATURAL;
  double ordering_flops[2] = {0.0, 0.0};

  int32_t nsuper() const { return (int32_t)super.size() - 1; }
  int64_t storage() const { return lxptr.empty() ? 0 : lxptr.back(); }
};

// Build P.csr_* from the pattern (after analyze).
void build_permuted_csr(const int64_t *Ap, const int32_t *Ai, Plan &P);

// One amalgamation rule: amalgamate (0: never merge), nrelax[3], zrelax_permille[3].
struct AmalgamationRule {
  int32_t amalgamate, nrelax[3], zrelax_permille[3];
};

// Run the inspector. Returns SYM_OK or an error code with a message in err. With fund_rule
// (one rule index per fundamental supernode, nfund of them), a candidate merge of S into the
// next supernode follows rules[fund_rule[f]], f the fundamental supernode holding last(S);
// otherwise every merge follows opt's rule.
int analyze(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm,
            const sym_options &opt, Plan &P, std::string &err,
            const std::vector<AmalgamationRule> *rules = nullptr, const std::vector<int32_t> *fund_rule = nullptr);

}  // namespace sym
