// ordering.cpp — fill-reducing orderings computed from the sparsity pattern alone (the inspector's
// SYM_ORDER_AUTO). The paper takes the ordering as given; the library offers two classic
// heuristics, written from their published descriptions, and keeps the one whose factor needs
// fewer flops:
//
//   * approximate minimum degree (Amestoy, Davis and Duff, 1996): eliminate, one supervariable at
//     a time, a variable of least approximate external degree on the quotient graph of variables
//     and elements; elements reached from the pivot are absorbed into the new one, variables with
//     identical adjacency merge into supervariables, and the degree bound
//     d_i <= min(d_i + |L_p \ i|, |A_i \ i| + |L_p \ i| + sum_e |L_e \ L_p|) replaces exact degrees;
//   * nested dissection by level structures (George and Liu): a breadth-first level structure
//     rooted at a pseudo-peripheral node, one level as the vertex separator (the smallest level
//     that leaves both sides a fifth of the nodes), the two sides ordered first, recursively, and
//     the separator last; parts of at most ND_LEAF nodes are ordered by minimum degree.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "ordering.h"

namespace sym {
namespace {

constexpr int32_t ND_LEAF = 96;

// Approximate minimum degree on the graph (xadj, adj) (symmetric, no self loops).
class Amd {
 public:
  Amd(int32_t n, const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj) : n_(n) {
    A_.resize(n);
    E_.resize(n);
    L_.resize(n);
    members_.resize(n);
    nv_.assign(n, 1);
    state_.assign(n, kVar);
    deg_.resize(n);
    esize_.assign(n, 0);
    w_.assign(n, 0);
    wstamp_.assign(n, -1);
    mark_.assign(n, -1);
    head_.assign(n + 1, -1);
    next_.assign(n, -1);
    prev_.assign(n, -1);
    for (int32_t i = 0; i < n; ++i) {
      A_[i].assign(adj.begin() + xadj[i], adj.begin() + xadj[i + 1]);
      deg_[i] = (int32_t)A_[i].size();
      insert(i);
    }
  }

  void run(std::vector<int32_t> &order) {
    order.clear();
    order.reserve(n_);
    int32_t remaining = n_, stamp = 0, mindeg = 0;
    std::vector<int32_t> Lp;
    while (remaining > 0) {
      while (mindeg <= n_ && head_[mindeg] < 0) ++mindeg;
      const int32_t p = head_[mindeg];
      remove(p);
      // The pivot's supervariable is eliminated as a whole (mass elimination).
      order.push_back(p);
      for (int32_t m : members_[p]) order.push_back(m);
      remaining -= nv_[p];
      state_[p] = kElem;
      // L_p: the variables of the elements around p (absorbed into p) and p's variable neighbours.
      ++stamp;
      mark_[p] = stamp;
      Lp.clear();
      int64_t lpw = 0;
      for (int32_t e : E_[p]) {
        if (state_[e] != kElem || e == p) continue;
        for (int32_t i : L_[e])
          if (state_[i] == kVar && mark_[i] != stamp) {
            mark_[i] = stamp;
            Lp.push_back(i);
            lpw += nv_[i];
          }
        state_[e] = kDead;
        std::vector<int32_t>().swap(L_[e]);
      }
      for (int32_t j : A_[p])
        if (state_[j] == kVar && mark_[j] != stamp) {
          mark_[j] = stamp;
          Lp.push_back(j);
          lpw += nv_[j];
        }
      std::vector<int32_t>().swap(A_[p]);
      std::vector<int32_t>().swap(E_[p]);
      L_[p] = Lp;
      esize_[p] = lpw;
      // |L_e \ L_p| for every element e next to a variable of L_p.
      for (int32_t i : Lp)
        for (int32_t e : E_[i]) {
          if (state_[e] != kElem || e == p) continue;
          if (wstamp_[e] != stamp) {
            wstamp_[e] = stamp;
            w_[e] = esize_[e];
          }
          w_[e] -= nv_[i];
        }
      // Update each variable of L_p: prune its lists, absorb elements inside L_p, bound its degree.
      for (int32_t i : Lp) {
        remove(i);
        int64_t ext = 0;
        std::vector<int32_t> &Ei = E_[i];
        size_t o = 0;
        for (int32_t e : Ei) {
          if (state_[e] != kElem || e == p) continue;
          if (w_[e] <= 0) {  // L_e inside L_p: aggressive absorption into p
            state_[e] = kDead;
            std::vector<int32_t>().swap(L_[e]);
            continue;
          }
          ext += w_[e];
          Ei[o++] = e;
        }
        Ei.resize(o);
        Ei.push_back(p);
        std::vector<int32_t> &Ai = A_[i];
        o = 0;
        for (int32_t j : Ai) {
          if (state_[j] != kVar || mark_[j] == stamp) continue;  // j eliminated, merged or in L_p
          ext += nv_[j];
          Ai[o++] = j;
        }
        Ai.resize(o);
        const int64_t own = lpw - nv_[i];
        int64_t d = std::min<int64_t>((int64_t)deg_[i] + own, ext + own);
        d = std::min<int64_t>(d, (int64_t)remaining - nv_[i]);
        deg_[i] = (int32_t)std::max<int64_t>(d, 0);
      }
      // Supervariables: variables of L_p with identical element and variable lists merge.
      merge_indistinguishable(Lp, stamp);
      for (int32_t i : Lp)
        if (state_[i] == kVar) {
          insert(i);
          mindeg = std::min(mindeg, deg_[i]);
        }
    }
  }

 private:
  static constexpr int8_t kVar = 0, kElem = 1, kDead = 2;

  void insert(int32_t i) {
    const int32_t d = deg_[i];
    next_[i] = head_[d];
    prev_[i] = -1;
    if (head_[d] >= 0) prev_[head_[d]] = i;
    head_[d] = i;
  }
  void remove(int32_t i) {
    if (prev_[i] >= 0) next_[prev_[i]] = next_[i];
    else if (head_[deg_[i]] == i) head_[deg_[i]] = next_[i];
    else return;  // not in a bucket
    if (next_[i] >= 0) prev_[next_[i]] = prev_[i];
    next_[i] = prev_[i] = -1;
  }

  void merge_indistinguishable(const std::vector<int32_t> &Lp, int32_t stamp) {
    std::vector<std::pair<uint64_t, int32_t>> keyed;
    keyed.reserve(Lp.size());
    for (int32_t i : Lp) {
      uint64_t h = (uint64_t)A_[i].size() * 1000003ull + (uint64_t)E_[i].size();
      for (int32_t j : A_[i]) h += (uint64_t)j * 2654435761ull;
      for (int32_t e : E_[i]) h += (uint64_t)e * 40503ull + 7;
      keyed.emplace_back(h, i);
    }
    std::sort(keyed.begin(), keyed.end());
    std::vector<int32_t> sa, sb;
    for (size_t a = 0; a < keyed.size(); ++a) {
      const int32_t i = keyed[a].second;
      if (state_[i] != kVar) continue;
      for (size_t b = a + 1; b < keyed.size() && keyed[b].first == keyed[a].first; ++b) {
        const int32_t j = keyed[b].second;
        if (state_[j] != kVar || A_[i].size() != A_[j].size() || E_[i].size() != E_[j].size()) continue;
        sa = A_[i];
        sb = A_[j];
        std::sort(sa.begin(), sa.end());
        std::sort(sb.begin(), sb.end());
        if (sa != sb) continue;
        sa = E_[i];
        sb = E_[j];
        std::sort(sa.begin(), sa.end());
        std::sort(sb.begin(), sb.end());
        if (sa != sb) continue;
        // j joins i: same neighbourhood, so i's degree loses j's weight
        nv_[i] += nv_[j];
        deg_[i] = std::max(0, deg_[i] - nv_[j]);
        members_[i].push_back(j);
        members_[i].insert(members_[i].end(), members_[j].begin(), members_[j].end());
        std::vector<int32_t>().swap(members_[j]);
        nv_[j] = 0;
        state_[j] = kDead;
        std::vector<int32_t>().swap(A_[j]);
        std::vector<int32_t>().swap(E_[j]);
      }
    }
    (void)stamp;
  }

  int32_t n_;
  std::vector<std::vector<int32_t>> A_, E_, L_, members_;
  std::vector<int32_t> nv_, deg_, w_, wstamp_, mark_, head_, next_, prev_;
  std::vector<int64_t> esize_;
  std::vector<int8_t> state_;
};

// Induced subgraph on `nodes` (local numbering by position).
void induced(const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj, const std::vector<int32_t> &nodes,
             std::vector<int32_t> &local, std::vector<int64_t> &sx, std::vector<int32_t> &sa) {
  sx.assign(nodes.size() + 1, 0);
  sa.clear();
  for (size_t t = 0; t < nodes.size(); ++t) local[nodes[t]] = (int32_t)t;
  for (size_t t = 0; t < nodes.size(); ++t) {
    const int32_t v = nodes[t];
    for (int64_t q = xadj[v]; q < xadj[v + 1]; ++q)
      if (local[adj[q]] >= 0) sa.push_back(local[adj[q]]);
    sx[t + 1] = (int64_t)sa.size();
  }
  for (int32_t v : nodes) local[v] = -1;
}

class NestedDissection {
 public:
  NestedDissection(const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj)
      : xadj_(xadj), adj_(adj), n_((int32_t)xadj.size() - 1) {
    part_.assign(n_, -1);
    level_.assign(n_, -1);
    local_.assign(n_, -1);
  }

  void run(std::vector<int32_t> &order) {
    order.clear();
    std::vector<int32_t> all(n_);
    std::iota(all.begin(), all.end(), 0);
    int32_t label = 0;
    for (int32_t v : all) part_[v] = label;
    dissect(all, label, order);
  }

 private:
  // Nodes of `nodes` (all labelled `label`) reachable from s, with their BFS levels; returns the
  // visit order.
  void bfs(int32_t s, int32_t label, std::vector<int32_t> &visit) {
    visit.clear();
    visit.push_back(s);
    level_[s] = 0;
    for (size_t h = 0; h < visit.size(); ++h) {
      const int32_t v = visit[h];
      for (int64_t q = xadj_[v]; q < xadj_[v + 1]; ++q) {
        const int32_t u = adj_[q];
        if (part_[u] == label && level_[u] < 0) {
          level_[u] = level_[v] + 1;
          visit.push_back(u);
        }
      }
    }
  }
  void clear_levels(const std::vector<int32_t> &visit) {
    for (int32_t v : visit) level_[v] = -1;
  }

  void leaf(const std::vector<int32_t> &nodes, std::vector<int32_t> &order) {
    std::vector<int64_t> sx;
    std::vector<int32_t> sa, lo;
    induced(xadj_, adj_, nodes, local_, sx, sa);
    Amd amd((int32_t)nodes.size(), sx, sa);
    amd.run(lo);
    for (int32_t t : lo) order.push_back(nodes[t]);
  }

  void dissect(const std::vector<int32_t> &nodes, int32_t label, std::vector<int32_t> &order) {
    if ((int32_t)nodes.size() <= ND_LEAF) {
      leaf(nodes, order);
      return;
    }
    // connected components of the part, each dissected on its own
    std::vector<int32_t> visit;
    bfs(nodes[0], label, visit);
    if (visit.size() < nodes.size()) {
      std::vector<std::vector<int32_t>> comps;
      comps.push_back(visit);
      for (int32_t v : nodes)
        if (level_[v] < 0) {
          std::vector<int32_t> c;
          bfs(v, label, c);
          comps.push_back(c);
        }
      for (int32_t v : nodes) level_[v] = -1;
      for (auto &c : comps) {
        const int32_t lab = ++next_label_;
        for (int32_t v : c) part_[v] = lab;
        dissect(c, lab, order);
      }
      return;
    }
    // pseudo-peripheral root: restart from a least-degree node of the last level while the
    // eccentricity grows
    int32_t root = nodes[0], ecc = level_[visit.back()];
    for (int it = 0; it < 6; ++it) {
      int32_t cand = -1, cd = 0;
      for (size_t h = visit.size(); h-- > 0 && level_[visit[h]] == ecc;) {
        const int32_t v = visit[h];
        const int32_t d = (int32_t)(xadj_[v + 1] - xadj_[v]);
        if (cand < 0 || d < cd) {
          cand = v;
          cd = d;
        }
      }
      clear_levels(visit);
      bfs(cand, label, visit);
      const int32_t e2 = level_[visit.back()];
      if (e2 <= ecc) {
        if (e2 < ecc) {  // keep the deeper structure
          clear_levels(visit);
          bfs(root, label, visit);
        }
        break;
      }
      root = cand;
      ecc = e2;
    }
    const int32_t h = level_[visit.back()];
    const int64_t N = (int64_t)nodes.size();
    if (h < 2) {
      clear_levels(visit);
      leaf(nodes, order);
      return;
    }
    std::vector<int64_t> cnt(h + 1, 0);
    for (int32_t v : visit) cnt[level_[v]]++;
    int32_t best = -1;
    int64_t below = 0;
    for (int32_t l = 0; l <= h; ++l) {
      const int64_t above = N - below - cnt[l];
      if (l > 0 && l < h && 5 * below >= N && 5 * above >= N && (best < 0 || cnt[l] < cnt[best])) best = l;
      below += cnt[l];
    }
    if (best < 0) {  // no balanced level: the median level
      below = 0;
      for (int32_t l = 0; l <= h; ++l) {
        if (2 * (below + cnt[l]) >= N) {
          best = std::min(std::max(l, 1), h - 1);
          break;
        }
        below += cnt[l];
      }
    }
    std::vector<int32_t> left, right, sep;
    for (int32_t v : visit) {
      const int32_t l = level_[v];
      if (l < best) left.push_back(v);
      else if (l > best) right.push_back(v);
      else {
        // a separator node with no neighbour beyond the separator joins the near side
        bool far = false;
        for (int64_t q = xadj_[v]; q < xadj_[v + 1] && !far; ++q) far = level_[adj_[q]] > best;
        (far ? sep : left).push_back(v);
      }
    }
    clear_levels(visit);
    const int32_t la = ++next_label_, lb = ++next_label_, ls = ++next_label_;
    for (int32_t v : left) part_[v] = la;
    for (int32_t v : right) part_[v] = lb;
    for (int32_t v : sep) part_[v] = ls;
    if (!left.empty()) dissect(left, la, order);
    if (!right.empty()) dissect(right, lb, order);
    order.insert(order.end(), sep.begin(), sep.end());
  }

  const std::vector<int64_t> &xadj_;
  const std::vector<int32_t> &adj_;
  int32_t n_;
  int32_t next_label_ = 0;
  std::vector<int32_t> part_, level_, local_;
};

}  // namespace

void pattern_graph(int64_t n, const int64_t *Ap, const int32_t *Ai, std::vector<int64_t> &xadj,
                   std::vector<int32_t> &adj) {
  xadj.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p)
      if (Ai[p] != j) {
        xadj[Ai[p] + 1]++;
        xadj[j + 1]++;
      }
  for (int64_t i = 0; i < n; ++i) xadj[i + 1] += xadj[i];
  adj.resize(xadj[n]);
  std::vector<int64_t> fill(xadj.begin(), xadj.end() - 1);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p)
      if (Ai[p] != j) {
        adj[fill[Ai[p]]++] = (int32_t)j;
        adj[fill[j]++] = Ai[p];
      }
}

void order_min_degree(int64_t n, const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj,
                      std::vector<int32_t> &perm) {
  Amd amd((int32_t)n, xadj, adj);
  amd.run(perm);
}

void order_nested_dissection(int64_t n, const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj,
                             std::vector<int32_t> &perm) {
  (void)n;
  NestedDissection nd(xadj, adj);
  nd.run(perm);
}

}  // namespace sym
