// symbolic.cpp — host symbolic inspector (runs once per sparsity pattern).
//
// The paper's inspector for Cholesky (Sec. 3.2) computes the elimination tree, the row patterns
// of L (the prune-set of VI-Prune) and the supernodes (the block-set of VS-Block). This file
// computes the same objects with near-linear algorithms and adds what the GPU needs on top:
// relaxed amalgamation, the supernodal row structure, descendant lists, relative row maps, a
// level schedule of the supernodal tree, the scatter map of A into the panels and the kernel
// task lists. No numeric work happens here (Sec. 4.2: the numeric code does no symbolic work).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <functional>
#include <numeric>

#include "ordering.h"
#include "plan.h"

namespace sym {
namespace {

// Validation of the input format (lower CSC, rows strictly increasing, diagonal first).
bool valid_pattern(int64_t n, const int64_t *Ap, const int32_t *Ai, std::string &err) {
  if (n < 0 || n > INT32_MAX - 1) { err = "n out of range"; return false; }
  if (!Ap || (n > 0 && !Ai)) { err = "null pattern pointer"; return false; }
  if (Ap[0] != 0) { err = "Ap[0] != 0"; return false; }
  for (int64_t j = 0; j < n; ++j) {
    if (Ap[j + 1] <= Ap[j]) { err = "column " + std::to_string(j) + " has no diagonal"; return false; }
    if (Ai[Ap[j]] != j) { err = "column " + std::to_string(j) + " does not start with its diagonal"; return false; }
    for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p)
      if (Ai[p] <= Ai[p - 1] || Ai[p] >= n) {
        err = "column " + std::to_string(j) + " has unsorted or out-of-range rows";
        return false;
      }
  }
  return true;
}

// Strictly-lower entries of P A P^T grouped by row: for row i, the columns j < i.
void rows_of_permuted(int64_t n, const int64_t *Ap, const int32_t *Ai,
                      const std::vector<int32_t> &iperm, std::vector<int64_t> &rp,
                      std::vector<int32_t> &rj) {
  rp.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p) {
      int32_t a = iperm[Ai[p]], b = iperm[j];
      rp[std::max(a, b) + 1]++;
    }
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  rj.resize(rp[n]);
  std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p) {
      int32_t a = iperm[Ai[p]], b = iperm[j];
      rj[fill[std::max(a, b)]++] = std::min(a, b);
    }
}

// Elimination tree by Liu's algorithm with path compression: row i of the strictly-lower part
// links every tree root reachable from its columns to i.
void etree_liu(int64_t n, const std::vector<int64_t> &rp, const std::vector<int32_t> &rj,
               std::vector<int32_t> &parent) {
  parent.assign(n, -1);
  std::vector<int32_t> anc(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t j = rj[p];
      while (j != -1 && j < i) {
        int32_t next = anc[j];
        anc[j] = (int32_t)i;
        if (next == -1) { parent[j] = (int32_t)i; break; }
        j = next;
      }
    }
  }
}

// Postorder with children (and roots) taken in increasing order. post[k] = node at position k.
void postorder(int64_t n, const std::vector<int32_t> &parent, std::vector<int32_t> &post) {
  std::vector<int32_t> first_child(n, -1), sibling(n, -1);
  for (int64_t j = n - 1; j >= 0; --j) {
    int32_t p = parent[j];
    if (p >= 0) { sibling[j] = first_child[p]; first_child[p] = (int32_t)j; }
  }
  post.clear();
  post.reserve(n);
  std::vector<int32_t> stack;
  for (int64_t r = 0; r < n; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back((int32_t)r);
    while (!stack.empty()) {
      int32_t v = stack.back();
      int32_t c = first_child[v];
      if (c != -1) {
        first_child[v] = sibling[c];
        stack.push_back(c);
      } else {
        stack.pop_back();
        post.push_back(v);
      }
    }
  }
}

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double seconds() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

}  // namespace

void build_permuted_csr(const int64_t *Ap, const int32_t *Ai, Plan &P) {
  const int64_t n = P.n;
  P.csr_p.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
      const int32_t a = P.iperm[Ai[p]], b = P.iperm[j];
      P.csr_p[a + 1]++;
      if (a != b) P.csr_p[b + 1]++;
    }
  for (int64_t i = 0; i < n; ++i) P.csr_p[i + 1] += P.csr_p[i];
  P.csr_i.resize(P.csr_p[n]);
  P.csr_map.resize(P.csr_p[n]);
  std::vector<int64_t> fill(P.csr_p.begin(), P.csr_p.end() - 1);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
      const int32_t a = P.iperm[Ai[p]], b = P.iperm[j];
      int64_t q = fill[a]++;
      P.csr_i[q] = b;
      P.csr_map[q] = p;
      if (a != b) {
        q = fill[b]++;
        P.csr_i[q] = a;
        P.csr_map[q] = p;
      }
    }
}

namespace {
// Flops sum_j c_j^2 of the factor of A permuted by p0 (etree of that ordering, then column counts
// by row subtrees; the fill does not depend on the etree postorder applied later).
double ordering_flops(int64_t n, const int64_t *Ap, const int32_t *Ai, const std::vector<int32_t> &p0) {
  std::vector<int32_t> ip(n);
  for (int64_t k = 0; k < n; ++k) ip[p0[k]] = (int32_t)k;
  std::vector<int64_t> rp;
  std::vector<int32_t> rj, parent;
  rows_of_permuted(n, Ap, Ai, ip, rp, rj);
  etree_liu(n, rp, rj, parent);
  std::vector<int64_t> cc(n, 1);
  std::vector<int32_t> mark(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    mark[i] = (int32_t)i;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      for (int32_t j = rj[p]; mark[j] != i; j = parent[j]) {
        mark[j] = (int32_t)i;
        cc[j]++;
      }
  }
  double f = 0.0;
  for (int64_t j = 0; j < n; ++j) f += (double)cc[j] * (double)cc[j];
  return f;
}
}  // namespace

int analyze(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm_in,
            const sym_options &opt, Plan &P, std::string &err, const std::vector<AmalgamationRule> *rules,
            const std::vector<int32_t> *fund_rule) {
  Timer timer;
  if (!valid_pattern(n, Ap, Ai, err)) return SYM_ERR_INVALID;
  P = Plan();
  P.n = n;
  P.nnz_a = Ap[n];

  // 1. Given ordering, or (SYM_ORDER_AUTO) the better of minimum degree and nested dissection
  //    by the flops of the factor each produces.
  std::vector<int32_t> p0(n), ip0(n, -1);
  std::vector<int32_t> automatic;
  P.ordering_method = opt.ordering == SYM_ORDER_GIVEN && perm_in ? SYM_ORDER_GIVEN : SYM_ORDER_NATURAL;
  if (opt.ordering == SYM_ORDER_AUTO && n > 0) {
    std::vector<int64_t> xadj;
    std::vector<int32_t> adj, pmd, pnd;
    pattern_graph(n, Ap, Ai, xadj, adj);
    order_min_degree(n, xadj, adj, pmd);
    order_nested_dissection(n, xadj, adj, pnd);
    const double fmd = ordering_flops(n, Ap, Ai, pmd), fnd = ordering_flops(n, Ap, Ai, pnd);
    P.ordering_flops[0] = fmd;
    P.ordering_flops[1] = fnd;
    const bool nd = fnd < fmd;
    automatic.swap(nd ? pnd : pmd);
    P.ordering_method = nd ? SYM_ORDER_METHOD_ND : SYM_ORDER_METHOD_MD;
  }
  for (int64_t k = 0; k < n; ++k) {
    int32_t v = !automatic.empty() ? automatic[k]
                : (opt.ordering == SYM_ORDER_GIVEN && perm_in) ? perm_in[k] : (int32_t)k;
    if (v < 0 || v >= n || ip0[v] != -1) { err = "perm is not a permutation"; return SYM_ERR_INVALID; }
    p0[k] = v;
    ip0[v] = (int32_t)k;
  }
  // 2. Etree of the given ordering, its postorder, and the final ordering perm0 o post.
  std::vector<int64_t> rp;
  std::vector<int32_t> rj, parent0, post;
  rows_of_permuted(n, Ap, Ai, ip0, rp, rj);
  etree_liu(n, rp, rj, parent0);
  postorder(n, parent0, post);
  std::vector<int32_t> ipost(n);
  for (int64_t k = 0; k < n; ++k) ipost[post[k]] = (int32_t)k;
  P.perm.resize(n);
  P.iperm.resize(n);
  for (int64_t k = 0; k < n; ++k) P.perm[k] = p0[post[k]];
  for (int64_t k = 0; k < n; ++k) P.iperm[P.perm[k]] = (int32_t)k;
  // The etree relabels with the postorder.
  P.parent.resize(n);
  for (int64_t k = 0; k < n; ++k) {
    int32_t q = parent0[post[k]];
    P.parent[k] = q < 0 ? -1 : ipost[q];
  }
  // 3. Column counts by row subtrees: row i of L is the union of the etree paths from each
  //    column j of row i of C up to i; every node on them gains one entry.
  rows_of_permuted(n, Ap, Ai, P.iperm, rp, rj);
  P.colcount.assign(n, 1);
  {
    std::vector<int32_t> mark(n, -1);
    for (int64_t i = 0; i < n; ++i) {
      mark[i] = (int32_t)i;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
        for (int32_t j = rj[p]; mark[j] != i; j = P.parent[j]) {
          mark[j] = (int32_t)i;
          P.colcount[j]++;
        }
    }
  }
  P.nnz_l = 0;
  P.flops = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    P.nnz_l += P.colcount[j];
    P.flops += (double)P.colcount[j] * (double)P.colcount[j];
  }
  // 4. Fundamental supernodes: j-1 joins j when j-1 is j's only child and |L_{j-1}| = |L_j|+1.
  {
    std::vector<int32_t> nchild(n, 0);
    for (int64_t j = 0; j < n; ++j)
      if (P.parent[j] >= 0) nchild[P.parent[j]]++;
    for (int64_t j = 0; j < n; ++j) {
      bool joins = j > 0 && P.parent[j - 1] == j && nchild[j] == 1 &&
                   P.colcount[j - 1] == P.colcount[j] + 1;
      if (!joins) P.fsuper.push_back((int32_t)j);
    }
    P.fsuper.push_back((int32_t)n);
  }
  const int32_t nf = (int32_t)P.fsuper.size() - 1;
  // 5. Row structure of each fundamental supernode: its columns, the entries of C below it,
  //    and the rows of its child supernodes below it (Eq. (1) applied per supernode).
  //    Columns of C: the transpose of the row lists.
  std::vector<int64_t> cp(n + 1, 0);
  std::vector<int32_t> ci;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) cp[rj[p] + 1]++;
  for (int64_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
  ci.resize(cp[n]);
  {
    std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) ci[fill[rj[p]]++] = (int32_t)i;
  }
  std::vector<int32_t> col2f(n);
  for (int32_t s = 0; s < nf; ++s)
    for (int32_t j = P.fsuper[s]; j < P.fsuper[s + 1]; ++j) col2f[j] = s;
  std::vector<std::vector<int32_t>> srows(nf);
  std::vector<std::vector<int32_t>> fchildren(nf);
  for (int32_t s = 0; s < nf; ++s) {
    int32_t pl = P.parent[P.fsuper[s + 1] - 1];
    if (pl >= 0) fchildren[col2f[pl]].push_back(s);
  }
  {
    std::vector<int32_t> mark(n, -1);
    for (int32_t s = 0; s < nf; ++s) {
      int32_t f = P.fsuper[s], l = P.fsuper[s + 1] - 1;
      std::vector<int32_t> &R = srows[s];
      for (int32_t j = f; j <= l; ++j) { R.push_back(j); mark[j] = s; }
      for (int32_t j = f; j <= l; ++j)
        for (int64_t p = cp[j]; p < cp[j + 1]; ++p)
          if (ci[p] > l && mark[ci[p]] != s) { mark[ci[p]] = s; R.push_back(ci[p]); }
      for (int32_t c : fchildren[s])
        for (int32_t r : srows[c])
          if (r > l && mark[r] != s) { mark[r] = s; R.push_back(r); }
      std::sort(R.begin() + (l - f + 1), R.end());
    }
  }
  // The exact pattern of column k of fundamental supernode F is the suffix of rows(F) from k;
  // keep the rows below each F to split the useful flops by kernel once the final supernodes
  // are known.
  std::vector<std::vector<int32_t>> fbelow(nf);
  for (int32_t s = 0; s < nf; ++s)
    fbelow[s].assign(srows[s].begin() + (P.fsuper[s + 1] - P.fsuper[s]), srows[s].end());
  // 6. Relaxed amalgamation (this library's rule; the paper runs without it, Sec. 4.1).
  std::vector<int64_t> ccum(n + 1, 0);
  for (int64_t j = 0; j < n; ++j) ccum[j + 1] = ccum[j] + P.colcount[j];
  std::vector<int32_t> sf(P.fsuper.begin(), P.fsuper.end() - 1);  // first column of each slot
  std::vector<int32_t> sl(nf);                                    // last column of each slot
  std::vector<int32_t> nxt(nf);
  for (int32_t s = 0; s < nf; ++s) { sl[s] = P.fsuper[s + 1] - 1; nxt[s] = s + 1; }
  int32_t head = nf > 0 ? 0 : nf;
  if (fund_rule && (int64_t)fund_rule->size() != nf) {
    err = "one amalgamation rule per fundamental supernode expected (" + std::to_string(nf) + ")";
    return SYM_ERR_INVALID;
  }
  if (opt.amalgamate || fund_rule) {
    std::vector<int32_t> merged;
    for (bool changed = true; changed;) {
      changed = false;
      int32_t prev = -1;
      for (int32_t s = head; s < nf && nxt[s] < nf;) {
        int32_t t = nxt[s];
        if (P.parent[sl[s]] == sl[s] + 1) {
          merged.clear();
          std::set_union(srows[s].begin(), srows[s].end(), srows[t].begin(), srows[t].end(),
                         std::back_inserter(merged));
          const int64_t m = (int64_t)merged.size();
          const int64_t nc = (int64_t)sl[t] - sf[s] + 1;
          const int64_t total = nc * m - nc * (nc - 1) / 2;
          const int64_t z = total - (ccum[sl[t] + 1] - ccum[sf[s]]);
          // the rule of the fundamental supernode holding last(S): slot s is that supernode
          AmalgamationRule R{1, {opt.nrelax[0], opt.nrelax[1], opt.nrelax[2]},
                             {opt.zrelax_permille[0], opt.zrelax_permille[1], opt.zrelax_permille[2]}};
          if (fund_rule) R = (*rules)[(*fund_rule)[s]];
          const bool ok = R.amalgamate &&
                          (nc <= R.nrelax[0] ||
                           (nc <= R.nrelax[1] && z * 1000 <= (int64_t)R.zrelax_permille[0] * total) ||
                           (nc <= R.nrelax[2] && z * 1000 <= (int64_t)R.zrelax_permille[1] * total) ||
                           z * 1000 <= (int64_t)R.zrelax_permille[2] * total);
          if (ok) {
            srows[t].swap(merged);
            std::vector<int32_t>().swap(srows[s]);
            sf[t] = sf[s];
            if (prev < 0) head = t; else nxt[prev] = t;
            s = t;  // the merged supernode is next in order of last column
            changed = true;
            continue;
          }
        }
        prev = s;
        s = t;
      }
    }
  }
  // Final supernodes.
  std::vector<int32_t> slots;
  for (int32_t s = head; s < nf; s = nxt[s]) slots.push_back(s);
  const int32_t ns = (int32_t)slots.size();
  P.super.resize(ns + 1);
  P.rowptr.assign(ns + 1, 0);
  for (int32_t J = 0; J < ns; ++J) {
    P.super[J] = sf[slots[J]];
    P.rowptr[J + 1] = P.rowptr[J] + (int64_t)srows[slots[J]].size();
  }
  P.super[ns] = (int32_t)n;
  P.rows.resize(P.rowptr[ns]);
  for (int32_t J = 0; J < ns; ++J) {
    std::copy(srows[slots[J]].begin(), srows[slots[J]].end(), P.rows.begin() + P.rowptr[J]);
    std::vector<int32_t>().swap(srows[slots[J]]);
  }
  std::vector<int32_t> col2s(n);
  for (int32_t J = 0; J < ns; ++J)
    for (int32_t j = P.super[J]; j < P.super[J + 1]; ++j) col2s[j] = J;
  P.sparent.resize(ns);
  for (int32_t J = 0; J < ns; ++J) {
    int32_t pl = P.parent[P.super[J + 1] - 1];
    P.sparent[J] = pl < 0 ? -1 : col2s[pl];
  }
  // Useful flops of the external updates: column k of F (pattern rows(F) from k, c_k entries)
  // updates column j = its t-th row with the c_k - t entries at or below j, 2 (c_k - t) flops;
  // for a row at position q of rows(F) this is 2 (|rows(F)| - q) for each of F's columns, and
  // it is an external update when j lies in another final supernode.
  P.update_flops = 0.0;
  for (int32_t s = 0; s < nf; ++s) {
    const int64_t nc = P.fsuper[s + 1] - P.fsuper[s];
    const int64_t m = nc + (int64_t)fbelow[s].size();
    const int32_t home = col2s[P.fsuper[s]];
    for (size_t t = 0; t < fbelow[s].size(); ++t)
      if (col2s[fbelow[s][t]] != home) P.update_flops += 2.0 * (double)(m - (nc + (int64_t)t)) * (double)nc;
  }
  std::vector<std::vector<int32_t>>().swap(fbelow);
  // 7. Descendant lists: every K whose rows reach into the columns of J (the block-level
  //    prune-set), with the first row position r0 at or after first(J) and the count nin of
  //    K's rows inside cols(J). Scanning K in increasing order keeps each list sorted.
  {
    std::vector<int64_t> cnt(ns + 1, 0);
    for (int32_t K = 0; K < ns; ++K) {
      int32_t lastJ = -1;
      for (int64_t p = P.rowptr[K] + (P.super[K + 1] - P.super[K]); p < P.rowptr[K + 1]; ++p) {
        int32_t J = col2s[P.rows[p]];
        if (J != lastJ) { cnt[J + 1]++; lastJ = J; }
      }
    }
    P.descptr.assign(ns + 1, 0);
    for (int32_t J = 0; J < ns; ++J) P.descptr[J + 1] = P.descptr[J] + cnt[J + 1];
    const int64_t np = P.descptr[ns];
    P.desc.resize(np);
    P.descr0.resize(np);
    P.descnin.resize(np);
    std::vector<int64_t> fill(P.descptr.begin(), P.descptr.end() - 1);
    for (int32_t K = 0; K < ns; ++K) {
      int32_t lastJ = -1;
      int64_t q = -1;
      for (int64_t p = P.rowptr[K] + (P.super[K + 1] - P.super[K]); p < P.rowptr[K + 1]; ++p) {
        int32_t J = col2s[P.rows[p]];
        if (J != lastJ) {
          q = fill[J]++;
          P.desc[q] = K;
          P.descr0[q] = p - P.rowptr[K];
          P.descnin[q] = 0;
          lastJ = J;
        }
        P.descnin[q]++;
      }
    }
  }
  // 8. Relative row maps through a position table of rows(J).
  {
    const int64_t np = P.descptr[ns];
    P.relptr.assign(np + 1, 0);
    for (int32_t J = 0; J < ns; ++J)
      for (int64_t q = P.descptr[J]; q < P.descptr[J + 1]; ++q) {
        int32_t K = P.desc[q];
        P.relptr[q + 1] = P.relptr[q] + (P.rowptr[K + 1] - P.rowptr[K] - P.descr0[q]);
      }
    P.rel.resize(P.relptr[np]);
    std::vector<int32_t> pos(n, -1);
    for (int32_t J = 0; J < ns; ++J) {
      for (int64_t p = P.rowptr[J]; p < P.rowptr[J + 1]; ++p) pos[P.rows[p]] = (int32_t)(p - P.rowptr[J]);
      for (int64_t q = P.descptr[J]; q < P.descptr[J + 1]; ++q) {
        int32_t K = P.desc[q];
        int64_t t = P.relptr[q];
        for (int64_t p = P.rowptr[K] + P.descr0[q]; p < P.rowptr[K + 1]; ++p) P.rel[t++] = pos[P.rows[p]];
      }
      for (int64_t p = P.rowptr[J]; p < P.rowptr[J + 1]; ++p) pos[P.rows[p]] = -1;
    }
  }
  // 9. Level schedule: leaves at 0, a parent one above its highest child.
  P.level.assign(ns, 0);
  for (int32_t J = 0; J < ns; ++J)
    if (P.sparent[J] >= 0) P.level[P.sparent[J]] = std::max(P.level[P.sparent[J]], P.level[J] + 1);
  int32_t nlev = 0;
  for (int32_t J = 0; J < ns; ++J) nlev = std::max(nlev, P.level[J] + 1);
  P.levelptr.assign(nlev + 1, 0);
  for (int32_t J = 0; J < ns; ++J) P.levelptr[P.level[J] + 1]++;
  for (int32_t l = 0; l < nlev; ++l) P.levelptr[l + 1] += P.levelptr[l];
  P.levellist.resize(ns);
  {
    std::vector<int32_t> fill(P.levelptr.begin(), P.levelptr.end() - 1);
    for (int32_t J = 0; J < ns; ++J) P.levellist[fill[P.level[J]]++] = J;
  }
  // 10. Panel layout and the scatter map of A's entries (caller's order) into the panels.
  P.lxptr.assign(ns + 1, 0);
  P.snodes.resize(ns);
  for (int32_t J = 0; J < ns; ++J) {
    SNode &s = P.snodes[J];
    s.first = P.super[J];
    s.ncols = P.super[J + 1] - P.super[J];
    s.nrows = (int32_t)(P.rowptr[J + 1] - P.rowptr[J]);
    s.ncb = (s.ncols + NB - 1) / NB;
    s.rowp = P.rowptr[J];
    s.lx = P.lxptr[J];
    P.lxptr[J + 1] = P.lxptr[J] + (int64_t)s.nrows * s.ncols;
    s.dx = P.dinv_storage;
    if (s.ncb > 0) {
      const int64_t last = s.ncols - (int64_t)(s.ncb - 1) * NB;
      P.dinv_storage += (int64_t)(s.ncb - 1) * NB * NB + last * last;
    }
    P.max_ncols = std::max(P.max_ncols, s.ncols);
    s.tx = P.tsize;
    P.tsize += (int64_t)(s.nrows - s.ncols) * ((s.ncols + SOLVE_CW - 1) / SOLVE_CW);
  }
  // Contribution lists of the forward solve: row g below the diagonal block of J receives
  // L_J(g, :) y_J, pushed as one partial product per column chunk of J.
  if (P.tsize >= INT32_MAX) {
    err = "forward-solve buffer exceeds 2^31 entries";
    return SYM_ERR_LIMIT;
  }
  P.contrib_ptr.assign(n + 1, 0);
  for (int32_t J = 0; J < ns; ++J) {
    const SNode &sj = P.snodes[J];
    const int32_t nch = (sj.ncols + SOLVE_CW - 1) / SOLVE_CW;
    for (int32_t r = sj.ncols; r < sj.nrows; ++r) P.contrib_ptr[P.rows[sj.rowp + r] + 1] += nch;
  }
  for (int64_t g = 0; g < n; ++g) P.contrib_ptr[g + 1] += P.contrib_ptr[g];
  P.contrib.resize(P.contrib_ptr[n]);
  {
    std::vector<int64_t> fill(P.contrib_ptr.begin(), P.contrib_ptr.end() - 1);
    for (int32_t J = 0; J < ns; ++J) {
      const SNode &sj = P.snodes[J];
      const int32_t nch = (sj.ncols + SOLVE_CW - 1) / SOLVE_CW, off = sj.nrows - sj.ncols;
      for (int32_t ch = 0; ch < nch; ++ch)
        for (int32_t r = sj.ncols; r < sj.nrows; ++r)
          P.contrib[fill[P.rows[sj.rowp + r]]++] = (int32_t)(sj.tx + (int64_t)ch * off + (r - sj.ncols));
    }
  }
  P.amap.resize(P.nnz_a);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
      int32_t a = P.iperm[Ai[p]], b = P.iperm[j];
      int32_t row = std::max(a, b), col = std::min(a, b);
      const SNode &s = P.snodes[col2s[col]];
      const int32_t *R = P.rows.data() + s.rowp;
      int64_t r = std::lower_bound(R, R + s.nrows, row) - R;
      P.amap[p] = s.lx + (int64_t)(col - s.first) * s.nrows + r;
    }

  // 11. Task lists and the launch schedule.
  //   Factor, per level: K_UPDATE over all tiles that receive descendant updates, then for each
  //   column tile s of the level's widest supernode: K_POTRF (diagonal tile s), K_TRSM (row
  //   tiles below it) and K_GEMM (trailing tiles of the same supernode).
  //   Forward solve, per level ascending: S_FSUM, S_FSTEP per column tile, S_FPUSH.
  //   Backward solve, per level descending: S_BGATHER, then S_BSTEP per column tile, last tile
  //   first.
  {
    struct Pending {
      int32_t bi, bj;
      double work;
      std::vector<UpdEntry> ents;
    };
    std::vector<int32_t> tile_slot;
    int32_t pending_join = -1;  // auxiliary launch the next main-stream launch must wait for
    for (int32_t l = 0; l < nlev; ++l) {
      // Gather the level's tasks, then order them by decreasing work (longest first) so that
      // the longest tiles start early; ties keep (J, bi, bj) order.
      struct LTask { int32_t J, bi, bj; double work; std::vector<UpdEntry> ents; };
      std::vector<LTask> lt;
      for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
        const int32_t J = P.levellist[t];
        const SNode &sj = P.snodes[J];
        const int32_t nrb = num_row_tiles(sj.nrows, sj.ncols, sj.ncb);
        std::vector<Pending> pend;
        tile_slot.assign((size_t)nrb * sj.ncb, -1);
        for (int64_t q = P.descptr[J]; q < P.descptr[J + 1]; ++q) {
          const int32_t K = P.desc[q];
          const SNode &sk = P.snodes[K];
          const int32_t *rel = P.rel.data() + P.relptr[q];
          const int32_t cnt = sk.nrows - (int32_t)P.descr0[q];
          const int32_t nin = P.descnin[q];
          // runs of rows with the same row tile (rel is increasing)
          struct Run { int32_t tile, start, len; };
          std::vector<Run> rr, cr;
          for (int32_t a = 0; a < cnt;) {
            int32_t ti = row_tile_of(rel[a], sj.ncols, sj.ncb);
            int32_t b = a + 1;
            while (b < cnt && row_tile_of(rel[b], sj.ncols, sj.ncb) == ti) ++b;
            rr.push_back({ti, a, b - a});
            if (a < nin) cr.push_back({ti, a, std::min(b, nin) - a});  // tiles of cols(J)
            a = b;
          }
          for (const Run &c : cr)
            for (const Run &r : rr) {
              if (r.tile < c.tile) continue;
              size_t key = (size_t)r.tile * sj.ncb + c.tile;
              if (tile_slot[key] < 0) {
                tile_slot[key] = (int32_t)pend.size();
                pend.push_back({r.tile, c.tile, 0.0, {}});
              }
              Pending &pd = pend[tile_slot[key]];
              UpdEntry e;
              e.K = K;
              e.r_lo = (int32_t)P.descr0[q] + r.start;
              e.c_lo = (int32_t)P.descr0[q] + c.start;
              e.m = r.len;
              e.n = c.len;
              e.pad = 0;
              e.relr = P.relptr[q] + r.start;
              e.relc = P.relptr[q] + c.start;
              pd.ents.push_back(e);
              pd.work += (double)r.len * c.len * sk.ncols;
            }
        }
        for (Pending &pd : pend) lt.push_back({J, pd.bi, pd.bj, pd.work, std::move(pd.ents)});
      }
      std::stable_sort(lt.begin(), lt.end(), [](const LTask &x, const LTask &y) { return x.work > y.work; });
      // A level whose update tiles all have at most SMALL_TILE rows and columns runs the
      // small-tile kernel variant. (Splitting a mixed level into two launches, the small tiles
      // beside the others on the auxiliary stream, measured slower at 64^3: in one launch the
      // small tiles, sorted last, fill the tail of the large ones.)
      auto small_tile = [&](const LTask &x) {
        const SNode &sj = P.snodes[x.J];
        const int64_t rb = row_tile_base(x.bi, sj.ncols, sj.ncb);
        const int64_t tm = std::min<int64_t>(NB, (x.bi < sj.ncb ? sj.ncols : sj.nrows) - rb);
        const int64_t tn = std::min<int32_t>(NB, sj.ncols - x.bj * NB);
        return tm <= SMALL_TILE && tn <= SMALL_TILE;
      };
      const bool all_small = std::all_of(lt.begin(), lt.end(), small_tile);
      {
        Launch U{K_UPDATE, l, (int64_t)P.upd_tasks.size(), 0};
        for (LTask &x : lt) {
          UpdTask u;
          u.J = x.J;
          u.bi = x.bi;
          u.bj = x.bj;
          u.pad = 0;
          u.e0 = (int64_t)P.upd_entries.size();
          P.upd_entries.insert(P.upd_entries.end(), x.ents.begin(), x.ents.end());
          u.e1 = (int64_t)P.upd_entries.size();
          P.upd_tasks.push_back(u);
        }
        U.count = (int64_t)P.upd_tasks.size() - U.off;
        if (U.count > 0) {
          U.tb = all_small ? SMALL_TILE : 0;
          // Few tiles (the top of the tree, small matrices): spread each tile's descendant entries
          // over a thread-block cluster of up to 8 CTAs while the launch still fits one wave.
          U.cluster = 1;
          if (!all_small)
            while (U.cluster < 8 && U.count * U.cluster * 2 <= GEMM_SLOTS) U.cluster *= 2;
          U.wait = pending_join;
          pending_join = -1;
          P.factor_launches.push_back(U);
        }
      }
      // Dense part of each supernode of this level: right-looking over column tiles s with
      // lookahead 1. After TRSM(s), the trailing update of column tile s+1 (NEXT) runs on the
      // main stream, followed at once by POTRF(s+1) and TRSM(s+1), while the update of the
      // tiles right of it (REST) runs on the auxiliary stream. NEXT(s) waits for REST(s-1),
      // the last earlier update of column s+1; REST(s) waits for TRSM(s).
      int32_t maxcb = 0;
      for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t)
        maxcb = std::max(maxcb, P.snodes[P.levellist[t]].ncb);
      auto emit = [&](int kind, int32_t s, int stream, int32_t wait,
                      const std::function<void(int32_t J, const SNode &, int32_t nrb)> &gen) -> int32_t {
        const int64_t off = (int64_t)P.tasks.size();
        for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
          const int32_t J = P.levellist[t];
          const SNode &sj = P.snodes[J];
          gen(J, sj, num_row_tiles(sj.nrows, sj.ncols, sj.ncb));
        }
        if ((int64_t)P.tasks.size() == off) return -1;
        // POTRF and TRSM tasks whose diagonal tile has at most SMALL_TILE columns form a second
        // launch of the small-tile kernel variant, after the full-size one on the same stream.
        std::vector<Int4> parts[2];
        for (int64_t q = off; q < (int64_t)P.tasks.size(); ++q) {
          const Int4 a = P.tasks[q];
          const bool small = (kind == K_POTRF || kind == K_TRSM) &&
                             std::min<int32_t>(NB, P.snodes[a.a].ncols - a.c * NB) <= SMALL_TILE;
          parts[small ? 1 : 0].push_back(a);
        }
        P.tasks.resize(off);
        int32_t last = -1;
        for (int part = 0; part < 2; ++part) {
          if (parts[part].empty()) continue;
          const int64_t o = (int64_t)P.tasks.size();
          // A short launch on the main stream (the lookahead chain) splits its tiles into row
          // halves so that twice as many SMs share the work of this latency-critical step. A
          // trailing-update launch on the auxiliary stream splits its last wave's worth of tiles
          // (GEMM_SLOTS: 3 CTAs on each of the 152 SMs) into halves, so its final wave ends
          // within half a tile's time instead of leaving most SMs idle for up to a whole one.
          const int64_t c0 = (int64_t)parts[part].size();
          int64_t split_from = c0;  // tasks from this index on are split into row halves
          if (stream == 0 && (kind == K_TRSM || kind == K_GEMM) && 2 * c0 <= 152) split_from = 0;
          if (stream == 1 && kind == K_GEMM) split_from = std::max<int64_t>(0, c0 - GEMM_SLOTS);
          for (int64_t q = 0; q < c0; ++q) {
            const Int4 &a = parts[part][q];
            if (q < split_from) {
              P.tasks.push_back(a);
            } else {
              P.tasks.push_back({a.a, a.b, a.c, a.d | (1 << 16)});
              P.tasks.push_back({a.a, a.b, a.c, a.d | (2 << 16)});
            }
          }
          Launch L{kind, l, o, (int64_t)P.tasks.size() - o};
          L.stream = stream;
          L.wait = last < 0 ? wait : -1;  // the second part follows the first on its stream
          L.tb = part == 1 ? SMALL_TILE : 0;
          P.factor_launches.push_back(L);
          last = (int32_t)P.factor_launches.size() - 1;
        }
        (void)s;
        return last;
      };
      auto potrf = [&](int32_t s) {
        return emit(K_POTRF, s, 0, -1, [&](int32_t J, const SNode &sj, int32_t) {
          if (s < sj.ncb) P.tasks.push_back({J, s, s, s});
        });
      };
      // Inverses of diagonal tiles (the solve uses them) on the auxiliary stream, after launch
      // `wait` of the main stream: column tiles c0 <= c < c1 of the level's supernodes, full-size
      // tiles then tiles of <= SMALL_TILE columns. The next level does not wait for them; the
      // factorization ends with both streams joined.
      auto trtri = [&](int32_t c0, int32_t c1, int32_t wait) {
        int32_t first = -1;
        for (int part = 0; part < 2; ++part) {
          const int64_t o = (int64_t)P.tasks.size();
          for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
            const int32_t J = P.levellist[t];
            for (int32_t c = c0; c < std::min(c1, P.snodes[J].ncb); ++c)
              if ((std::min<int32_t>(NB, P.snodes[J].ncols - c * NB) <= SMALL_TILE) == (part == 1))
                P.tasks.push_back({J, c, c, c});
          }
          if ((int64_t)P.tasks.size() > o) {
            Launch T{K_TRTRI, l, o, (int64_t)P.tasks.size() - o};
            T.stream = 1;
            T.wait = first < 0 ? wait : -1;
            T.tb = part == 1 ? SMALL_TILE : 0;
            P.factor_launches.push_back(T);
            first = (int32_t)P.factor_launches.size() - 1;
          }
        }
      };
      auto trsm = [&](int32_t s) {
        return emit(K_TRSM, s, 0, -1, [&](int32_t J, const SNode &sj, int32_t nrb) {
          if (s < sj.ncb)
            for (int32_t i = s + 1; i < nrb; ++i) P.tasks.push_back({J, i, s, s});
        });
      };
      if (maxcb > 0) {
        int32_t last_main = -1;  // latest main-stream launch (panel s is final after it)
        auto note = [&](int32_t idx) {
          if (idx >= 0) last_main = idx;
        };
        {
          // the first dense launch of the level also joins any pending auxiliary work
          const int32_t idx = potrf(0);
          if (idx >= 0 && pending_join >= 0) {
            P.factor_launches[idx].wait = pending_join;
            pending_join = -1;
          }
          note(idx);
          // the last two column tiles' inverses start as soon as their POTRF is done (no
          // trailing-update launch of this level follows them on the auxiliary stream)
          if (maxcb <= 2) trtri(0, 1, idx);
        }
        note(trsm(0));
        int32_t rest_prev = -1;
        for (int32_t s = 0; s + 1 < maxcb; ++s) {
          const int32_t rest_idx = emit(K_GEMM, s, 1, last_main, [&](int32_t J, const SNode &sj, int32_t nrb) {
            for (int32_t j = s + 2; j < sj.ncb; ++j)
              for (int32_t i = j; i < nrb; ++i) P.tasks.push_back({J, i, j, s});
          });
          note(emit(K_GEMM, s, 0, rest_prev, [&](int32_t J, const SNode &sj, int32_t nrb) {
            if (s + 1 < sj.ncb)
              for (int32_t i = s + 1; i < nrb; ++i) P.tasks.push_back({J, i, s + 1, s});
          }));
          const int32_t pidx = potrf(s + 1);
          note(pidx);
          if (s + 3 >= maxcb) trtri(s + 1, s + 2, pidx);
          note(trsm(s + 1));
          if (rest_idx >= 0) rest_prev = rest_idx;
        }
        // join: the next launch on the main stream waits for the last auxiliary launch
        pending_join = rest_prev;
        // the other column tiles' inverses once the level's panels are final
        if (maxcb > 2) trtri(0, maxcb - 2, last_main);
      }
    }
  }
  // Solve schedules. Forward, per level: S_FSUM (columns subtract what their descendants
  // pushed), S_FSTEP per column tile, S_FPUSH (the level's solved supernodes push their products
  // to the rows below their diagonal blocks).
  // A level whose supernodes all have at most SMALL_TILE columns marks its sum, push and gather
  // launches tb = SMALL_TILE: batches run them one warp per (task, matrix).
  auto small_level = [&](int32_t l) {
    for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t)
      if (P.snodes[P.levellist[t]].ncols > SMALL_TILE) return false;
    return true;
  };
  auto push_solve = [&](std::vector<Launch> &list, int32_t kind, int32_t l, int64_t off) {
    if ((int64_t)P.tasks.size() <= off) return;
    Launch L{kind, l, off, (int64_t)P.tasks.size() - off};
    if (small_level(l)) L.tb = SMALL_TILE;
    list.push_back(L);
  };
  for (int32_t l = 0; l < nlev; ++l) {
    int64_t off = (int64_t)P.tasks.size();
    int32_t maxcb = 0;
    for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
      const int32_t J = P.levellist[t];
      const SNode &sj = P.snodes[J];
      maxcb = std::max(maxcb, sj.ncb);
      if (P.contrib_ptr[sj.first + sj.ncols] > P.contrib_ptr[sj.first])
        for (int32_t cb = 0; cb * 256 < sj.ncols; ++cb) P.tasks.push_back({J, cb, 0, 0});
    }
    push_solve(P.fwd_launches, S_FSUM, l, off);
    // Supernodes of more than SMALL_TILE columns: cluster steps s = -1 .. ncb - 2, tasks {J, i, s}
    // (cluster = 4): i = s + 1 applies the solved tile s and solves tile i, i > s + 1 applies it.
    for (int32_t s = -1; s + 1 < maxcb; ++s) {
      off = (int64_t)P.tasks.size();
      for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
        const int32_t J = P.levellist[t];
        if (P.snodes[J].ncols <= SMALL_TILE) continue;
        const int32_t ncb = P.snodes[J].ncb;
        if (s + 1 >= ncb) continue;
        for (int32_t i = s + 1; i < (s >= 0 ? ncb : 1); ++i) P.tasks.push_back({J, i, s, 0});
      }
      if ((int64_t)P.tasks.size() > off) {
        Launch L{S_FSTEP, l, off, (int64_t)P.tasks.size() - off};
        L.cluster = 4;
        P.fwd_launches.push_back(L);
      }
    }
    // The others (one tile each): the one-CTA form, tasks {J, i, s, s}.
    for (int32_t s = 0; s < maxcb; ++s) {
      off = (int64_t)P.tasks.size();
      for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
        const int32_t J = P.levellist[t];
        if (P.snodes[J].ncols > SMALL_TILE) continue;
        const int32_t ncb = P.snodes[J].ncb;
        for (int32_t i = s; i < ncb; ++i) P.tasks.push_back({J, i, s, s});
      }
      if ((int64_t)P.tasks.size() > off) {
        Launch L{S_FSTEP, l, off, (int64_t)P.tasks.size() - off};
        L.tb = SMALL_TILE;
        P.fwd_launches.push_back(L);
      }
    }
    off = (int64_t)P.tasks.size();
    for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
      const int32_t J = P.levellist[t];
      const SNode &sj = P.snodes[J];
      const int32_t nrb = num_row_tiles(sj.nrows, sj.ncols, sj.ncb);
      for (int32_t ch = 0; ch * SOLVE_CW < sj.ncols; ++ch)
        for (int32_t i = sj.ncb; i < nrb; ++i) P.tasks.push_back({J, i, ch, 0});
    }
    push_solve(P.fwd_launches, S_FPUSH, l, off);
  }
  for (int32_t l = nlev - 1; l >= 0; --l) {
    int64_t off = (int64_t)P.tasks.size();
    int32_t maxcb = 0;
    for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
      const int32_t J = P.levellist[t];
      const SNode &sj = P.snodes[J];
      maxcb = std::max(maxcb, sj.ncb);
      if (sj.nrows > sj.ncols)
        for (int32_t sl = 0; sl * SOLVE_BG < sj.ncols; ++sl) P.tasks.push_back({J, sl, 0, 0});
    }
    push_solve(P.bwd_launches, S_BGATHER, l, off);
    // Supernodes of more than SMALL_TILE columns: cluster steps s = ncb .. 1, tasks {J, i, s}
    // (cluster = 4): i = s - 1 applies the solved tile s (s < ncb) and solves tile i, i < s - 1
    // applies it.
    for (int32_t s = maxcb; s >= 1; --s) {
      off = (int64_t)P.tasks.size();
      for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
        const int32_t J = P.levellist[t];
        if (P.snodes[J].ncols <= SMALL_TILE) continue;
        const int32_t ncb = P.snodes[J].ncb;
        if (s > ncb) continue;
        for (int32_t i = s - 1; i >= (s < ncb ? 0 : s - 1); --i) P.tasks.push_back({J, i, s, 0});
      }
      if ((int64_t)P.tasks.size() > off) {
        Launch L{S_BSTEP, l, off, (int64_t)P.tasks.size() - off};
        L.cluster = 4;
        P.bwd_launches.push_back(L);
      }
    }
    for (int32_t s = maxcb - 1; s >= 0; --s) {
      off = (int64_t)P.tasks.size();
      for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
        const int32_t J = P.levellist[t];
        if (P.snodes[J].ncols > SMALL_TILE) continue;
        const int32_t ncb = P.snodes[J].ncb;
        if (s >= ncb) continue;
        for (int32_t i = s; i >= 0; --i) P.tasks.push_back({J, i, s, s});
      }
      if ((int64_t)P.tasks.size() > off) {
        Launch L{S_BSTEP, l, off, (int64_t)P.tasks.size() - off};
        L.tb = SMALL_TILE;
        P.bwd_launches.push_back(L);
      }
    }
  }
  // The solve launches of levels of narrow supernodes become one launch per level and direction
  // (k_fwd_b, k_bwd_b; a batch only where the panels fit, see solve_panel_lanes).
  {
    auto mark = [&](const std::vector<Launch> &list, std::vector<PanelForm> &form, int32_t step_kind) {
      form.assign(list.size(), PanelForm{PANEL_NONE, 0, 0, -1});
      for (int32_t l = 0; l < nlev; ++l) {
        int64_t pmax = 0, ncmax = 0;
        for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
          const SNode &sj = P.snodes[P.levellist[t]];
          pmax = std::max<int64_t>(pmax, (int64_t)sj.nrows * sj.ncols);
          ncmax = std::max<int64_t>(ncmax, sj.ncols);
        }
        if (P.levelptr[l + 1] == P.levelptr[l] || !small_level(l)) continue;
        std::vector<size_t> step, other;
        for (size_t li = 0; li < list.size(); ++li)
          if (list[li].level == l) (list[li].kind == step_kind ? step : other).push_back(li);
        if (step.size() != 1) continue;
        const int32_t head = (int32_t)step[0];
        form[head] = PanelForm{PANEL_FUSED, (int32_t)pmax, (int32_t)ncmax, head};
        for (size_t li : other) form[li] = PanelForm{PANEL_COVERED, 0, 0, head};
      }
    };
    mark(P.fwd_launches, P.fwd_panel, S_FSTEP);
    mark(P.bwd_launches, P.bwd_panel, S_BSTEP);
  }
  for (auto &v : P.variant) v.assign(P.factor_launches.size(), 0);
  // Default form of a batch's full-tile FP64 update launches: one warp per (tile, matrix) when
  // the launch's entries are small (at most BATCH_WARP_ELEMS output elements on average: the
  // one-CTA form then spends its time staging and waiting at barriers), else one CTA per tile.
  // Small-tile update launches of a batch run with lanes mapped to matrices (k_update_mb), about
  // three elements of an average entry per lane: G = the largest power of two <= mean / 3, 1..8.
  P.batch_warp.assign(P.factor_launches.size(), 0);
  P.batch_lanes.assign(P.factor_launches.size(), 0);
  for (size_t li = 0; li < P.factor_launches.size(); ++li) {
    const Launch &L = P.factor_launches[li];
    if (L.kind != K_UPDATE) continue;
    double elems = 0.0, cnt = 0.0;
    for (int64_t t = L.off; t < L.off + L.count; ++t) {
      const UpdTask &u = P.upd_tasks[t];
      for (int64_t e = u.e0; e < u.e1; ++e) {
        const UpdEntry &E = P.upd_entries[e];
        elems += u.bi == u.bj ? 0.5 * E.m * (E.m + 1) : (double)E.m * E.n;
        cnt += 1.0;
      }
    }
    int g = 1;
    while (g < 8 && cnt > 0.0 && 2 * g * 3.0 * cnt <= elems) g *= 2;
    P.batch_lanes[li] = (int8_t)g;
  }
  for (size_t li = 0; li < P.factor_launches.size(); ++li) {
    const Launch &L = P.factor_launches[li];
    if (L.kind != K_UPDATE || L.tb == SMALL_TILE) continue;
    double elems = 0.0, cnt = 0.0;
    for (int64_t t = L.off; t < L.off + L.count; ++t) {
      const UpdTask &u = P.upd_tasks[t];
      for (int64_t e = u.e0; e < u.e1; ++e) {
        const UpdEntry &E = P.upd_entries[e];
        elems += u.bi == u.bj ? 0.5 * E.m * (E.m + 1) : (double)E.m * E.n;
        cnt += 1.0;
      }
    }
    P.batch_warp[li] = cnt > 0.0 && elems <= BATCH_WARP_ELEMS * cnt;
  }
  // Levels of supernodes with at most SMALL_TILE columns run their POTRF, TRSM and TRTRI as one
  // launch (k_panel_b; a batch only where the panels fit, see panel_lanes). Such a level has one
  // launch of each (one column tile, all of it small-tile).
  P.batch_panel.assign(P.factor_launches.size(), PanelForm{PANEL_NONE, 0, 0, -1});
  for (auto &v : P.panel_apart) v.assign(P.factor_launches.size(), 0);
  for (int32_t l = 0; l < nlev; ++l) {
    int64_t pmax = 0, ncmax = 0;
    bool narrow = P.levelptr[l + 1] > P.levelptr[l];
    for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
      const SNode &sj = P.snodes[P.levellist[t]];
      narrow = narrow && sj.ncols <= SMALL_TILE;
      pmax = std::max<int64_t>(pmax, (int64_t)sj.nrows * sj.ncols);
      ncmax = std::max<int64_t>(ncmax, sj.ncols);
    }
    if (!narrow) continue;
    std::vector<size_t> potrf, other;
    for (size_t li = 0; li < P.factor_launches.size(); ++li) {
      const Launch &L = P.factor_launches[li];
      if (L.level != l) continue;
      if (L.kind == K_POTRF) potrf.push_back(li);
      if (L.kind == K_TRSM || L.kind == K_TRTRI) other.push_back(li);
    }
    if (potrf.size() != 1) continue;
    const int32_t head = (int32_t)potrf[0];
    P.batch_panel[head] = PanelForm{PANEL_FUSED, (int32_t)pmax, (int32_t)ncmax, head};
    // A single matrix runs the fused launch (one warp per supernode) by default only on levels of
    // at least PANEL_ONE_MIN supernodes, where many warps per SM hide each one's column chain; on
    // the 64^2 5-point grid's levels of 1-64 supernodes of 16-32 columns it was 1.7-4.3x slower
    // than the separate launches, whose CTAs spread the column steps over more schedulers. The
    // autotuner decides either way.
    P.panel_apart[0][head] = P.levelptr[l + 1] - P.levelptr[l] < PANEL_ONE_MIN;
    for (size_t li : other) P.batch_panel[li] = PanelForm{PANEL_COVERED, 0, 0, head};
  }
  // 12. Algorithmic flops of each kernel kind (see Plan::kind_flops).
  {
    auto sq = [](double x) { return x * x; };
    for (const UpdTask &u : P.upd_tasks) {
      for (int64_t e = u.e0; e < u.e1; ++e) {
        const UpdEntry &E = P.upd_entries[e];
        const double k = P.snodes[E.K].ncols;
        if (u.bi != u.bj) {
          P.kind_flops[K_UPDATE] += 2.0 * E.m * E.n * k;
        } else {
          const int32_t *rr = P.rel.data() + E.relr;
          const int32_t *rc = P.rel.data() + E.relc;
          double pairs = 0;
          for (int32_t b = 0; b < E.n; ++b)
            pairs += (double)(E.m - (std::lower_bound(rr, rr + E.m, rc[b]) - rr));
          P.kind_flops[K_UPDATE] += 2.0 * k * pairs;
        }
      }
    }
    auto cols_of_tile = [](const SNode &s, int32_t t) { return std::min<int32_t>(NB, s.ncols - t * NB); };
    // rows of the row tile q.b of a TRSM or GEMM task, or of its row half (bits 16+ of q.d)
    auto task_rows = [](const SNode &s, const Int4 &q) {
      const int64_t rb = row_tile_base(q.b, s.ncols, s.ncb);
      int64_t tm = std::min<int64_t>(NB, (q.b < s.ncb ? s.ncols : s.nrows) - rb);
      const int half = q.d >> 16;
      if (half) tm = std::max<int64_t>(0, std::min<int64_t>(NB / 2, tm - (half - 1) * (NB / 2)));
      return (double)tm;
    };
    for (const Launch &L : P.factor_launches) {
      if (L.kind == K_UPDATE) continue;
      for (int64_t t = L.off; t < L.off + L.count; ++t) {
        const Int4 &q = P.tasks[t];
        const SNode &s = P.snodes[q.a];
        if (L.kind == K_POTRF) {
          const double ts = cols_of_tile(s, q.b);
          P.kind_flops[K_POTRF] += ts * (ts + 1) * (2 * ts + 1) / 6.0;
        } else if (L.kind == K_TRSM) {
          const double ts = cols_of_tile(s, q.c);
          P.kind_flops[K_TRSM] += task_rows(s, q) * sq(ts);
        } else if (L.kind == K_TRTRI) {
          const double ts = cols_of_tile(s, q.b);
          P.kind_flops[K_TRTRI] += ts * ts * ts / 3.0;
        } else if (L.kind == K_GEMM) {
          const double ks = cols_of_tile(s, q.d & 0xffff), tn = cols_of_tile(s, q.c);
          const double tm = task_rows(s, q);
          // diagonal tile: only its lower triangle is useful; a row half counts half of it
          P.kind_flops[K_GEMM] += q.b == q.c ? ks * tn * (tn + 1) * ((q.d >> 16) ? 0.5 : 1.0)
                                             : 2.0 * tm * tn * ks;
        }
      }
    }
    for (const std::vector<Launch> *list : {&P.fwd_launches, &P.bwd_launches})
      for (const Launch &L : *list)
        for (int64_t t = L.off; t < L.off + L.count; ++t) {
          const Int4 &q = P.tasks[t];
          const SNode &s = P.snodes[q.a];
          // diagonal tile: ts^2 (solve with L_ss); off-diagonal tile: 2 tm ts
          if ((L.kind == S_FSTEP || L.kind == S_BSTEP) && L.cluster == 4) {
            const bool fwd = L.kind == S_FSTEP;
            const bool has_s = fwd ? q.c >= 0 : q.c < s.ncb;
            const double ti = cols_of_tile(s, q.b);
            P.kind_flops[L.kind] += (has_s ? 2.0 * ti * cols_of_tile(s, q.c) : 0.0) +
                                    (q.b == (fwd ? q.c + 1 : q.c - 1) ? ti * ti : 0.0);
          } else if (L.kind == S_FSTEP || L.kind == S_BSTEP) {
            P.kind_flops[L.kind] += q.b == q.c ? sq(cols_of_tile(s, q.c))
                                                : 2.0 * cols_of_tile(s, q.b) * cols_of_tile(s, q.c);
          }
          if (L.kind == S_BGATHER)
            P.kind_flops[L.kind] += 2.0 * (s.nrows - s.ncols) * std::min<int32_t>(SOLVE_BG, s.ncols - q.b * SOLVE_BG);
          if (L.kind == S_FPUSH)
            P.kind_flops[L.kind] += 2.0 * std::min<int64_t>(NB, s.nrows - row_tile_base(q.b, s.ncols, s.ncb)) *
                                    std::min<int32_t>(SOLVE_CW, s.ncols - q.c * SOLVE_CW);
          if (L.kind == S_FSUM) {
            const int64_t g0 = s.first + (int64_t)q.b * 256, g1 = std::min<int64_t>(s.first + s.ncols, g0 + 256);
            P.kind_flops[L.kind] += (double)(P.contrib_ptr[g1] - P.contrib_ptr[g0]);
          }
        }
  }
  P.analyze_seconds = timer.seconds();
  return SYM_OK;
}

}  // namespace sym
