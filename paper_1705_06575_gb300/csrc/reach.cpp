// reach.cpp — inspector for sparse right-hand sides (the paper's triangular-solve workload).
//
// For L x = b with a sparse b, the nonzeros of x are Reach_L(beta), the nodes reachable from
// beta = {i : b_i != 0} in the dependence graph of L (Sec. 1.1). For a Cholesky factor every edge
// j -> i of that graph joins j to one of its elimination-tree ancestors, and the ancestors of j
// are exactly the nodes its column reaches, so the reach is the union of the etree paths from
// beta up to the roots. The inspector marks those columns once per pattern of b (VI-Prune's
// inspection set) and prunes the forward solve's task lists to the supernodes that hold them and,
// inside each, to the descendant contributions from other reached supernodes (VS-Block keeps the
// dense per-supernode kernels).
#include <algorithm>

#include "reach.h"

namespace sym {

int build_reach(const Plan &P, int64_t nb, const int32_t *beta, Reach &R, std::string &err) {
  R = Reach();
  const int64_t n = P.n;
  const int32_t ns = P.nsuper();
  std::vector<uint8_t> seen(n, 0);
  R.pbeta.resize(nb);
  for (int64_t t = 0; t < nb; ++t) {
    const int32_t b = beta[t];
    if (b < 0 || b >= n) { err = "right-hand side index out of range"; return SYM_ERR_INVALID; }
    const int32_t pb = P.iperm[b];
    if (seen[pb]) { err = "duplicate right-hand side index"; return SYM_ERR_INVALID; }
    seen[pb] = 1;
    R.pbeta[t] = pb;
  }
  // Column reach: walk up the elimination tree from every nonzero until a marked node.
  std::vector<uint8_t> mark(n, 0);
  for (int32_t pb : R.pbeta)
    for (int32_t j = pb; j >= 0 && !mark[j]; j = P.parent[j]) mark[j] = 1;
  for (int64_t j = 0; j < n; ++j)
    if (mark[j]) R.cols.push_back((int32_t)j);  // increasing order is topological
  // Reached supernodes, and the first reached column tile of each: a path enters a supernode at
  // some column and then runs through all later ones (its columns form an etree chain), so the
  // tiles before the entry hold zeros only and their steps are skipped.
  std::vector<uint8_t> sr(ns, 0);
  std::vector<int32_t> s0(ns, 0);
  {
    int32_t J = 0;
    for (int32_t j : R.cols) {
      while (P.super[J + 1] <= j) ++J;
      if (!sr[J]) s0[J] = (j - P.super[J]) / NB;
      sr[J] = 1;
    }
  }
  for (int32_t J = 0; J < ns; ++J)
    if (sr[J]) R.snodes.push_back(J);
  // Pruned forward schedule, level by level.
  const int32_t nlev = (int32_t)P.levelptr.size() - 1;
  // index of the update task of each diagonal tile (J, s): scan the update tasks once
  std::vector<int64_t> diag_first(ns + 1, 0);
  for (int32_t J = 0; J < ns; ++J) diag_first[J + 1] = diag_first[J] + P.snodes[J].ncb;
  std::vector<int64_t> diag_task(diag_first[ns], -1);
  for (size_t q = 0; q < P.upd_tasks.size(); ++q) {
    const UpdTask &u = P.upd_tasks[q];
    if (u.bi == u.bj) diag_task[diag_first[u.J] + u.bj] = (int64_t)q;
  }
  for (int32_t l = 0; l < nlev; ++l) {
    int32_t maxcb = 0;
    int64_t off = (int64_t)R.tasks.size();
    for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
      const int32_t J = P.levellist[t];
      if (!sr[J]) continue;
      maxcb = std::max(maxcb, P.snodes[J].ncb);
      for (int32_t bj = 0; bj < P.snodes[J].ncb; ++bj) {
        const int64_t q = diag_task[diag_first[J] + bj];
        if (q < 0) continue;
        const UpdTask &u = P.upd_tasks[q];
        UpdTask v = u;
        v.e0 = (int64_t)R.upd_entries.size();
        for (int64_t e = u.e0; e < u.e1; ++e)
          if (sr[P.upd_entries[e].K]) R.upd_entries.push_back(P.upd_entries[e]);
        v.e1 = (int64_t)R.upd_entries.size();
        if (v.e1 == v.e0) continue;
        R.tasks.push_back({J, bj, (int32_t)R.upd_tasks.size(), 0});
        R.upd_tasks.push_back(v);
      }
    }
    if ((int64_t)R.tasks.size() > off) {
      const int64_t cnt = (int64_t)R.tasks.size() - off;
      Launch L{S_FGATHER, l, off, cnt};
      L.cluster = cnt < 304 ? 8 : (cnt < 1216 ? 2 : 1);
      R.fwd.push_back(L);
    }
    for (int32_t s = 0; s < maxcb; ++s) {
      off = (int64_t)R.tasks.size();
      for (int32_t t = P.levelptr[l]; t < P.levelptr[l + 1]; ++t) {
        const int32_t J = P.levellist[t];
        if (!sr[J] || s < s0[J]) continue;
        for (int32_t i = s; i < P.snodes[J].ncb; ++i) R.tasks.push_back({J, i, s, s});
      }
      if ((int64_t)R.tasks.size() > off) R.fwd.push_back({S_FSTEP, l, off, (int64_t)R.tasks.size() - off});
    }
  }
  return SYM_OK;
}

}  // namespace sym
