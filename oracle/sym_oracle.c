/*
 * CPU FP64 oracle for decoupled supernodal Cholesky (Sympiler, arXiv 1705.06575).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. It shares no code, header, helper or table with the CUDA path. Every
 * step is written for plain correctness, in the order the paper defines it, not for speed.
 *
 * What it computes, by section of the paper:
 *   - permuted matrix C = P A P^T (lower triangle kept; entries flipped across the diagonal are
 *     mirrored);
 *   - elimination tree: parent[j] = min{ i > j : L_ij != 0 } (Sec. 3.2, "Theory");
 *   - column patterns of L by Eq. (1): L_j = A_j U {j} U (union over children s of L_s \ {s});
 *   - row patterns of L by walking the etree up from each A_ij until i or a marked node
 *     (Sec. 3.2), cross-checked against the transpose of the column patterns;
 *   - fundamental supernodes: column j-1 joins j when parent[j-1] = j, j-1 is the only child of
 *     j and |L_{j-1}| = |L_j| + 1 (Sec. 3.2, supernode rule);
 *   - relaxed amalgamation (not in the paper, which disables it, Sec. 4.1): a stated rule;
 *   - supernodal row structure, descendant lists (the prune-set of Sec. 3.2 at block level) and
 *     relative row maps;
 *   - a level schedule over the supernodal tree;
 *   - numeric L by an up-looking sparse Cholesky: row k of L is the solution of a sparse lower
 *     triangular system whose nonzero pattern is the reach of row k of C in the etree (Sec. 1.1
 *     reach-set idea, Sec. 3.2 row patterns); then L_kk = sqrt(C_kk - sum_j L_kj^2);
 *   - forward and backward substitution with L (Sec. 3.1 for the forward sweep; the backward
 *     sweep with L^T is the textbook one, the paper does not describe it);
 *   - checks: ||L L^T - C||_F / ||C||_F and the normwise backward error of a solve.
 *
 * The amalgamation keeps a log of its merges (which supernode was absorbed into which, in
 * order), so that a test can replay them and re-derive each merge's zero count from the dense
 * filled pattern.
 *
 * Where the paper is silent the oracle follows these readings:
 *   - postorder of the etree: children in increasing index order, roots in increasing order;
 *   - a non-positive or NaN pivot stops the factorization and reports the column;
 *   - amalgamation: supernode S merges into the next supernode P iff parent[last(S)] = last(S)+1
 *     and, with the merged column count m and the fraction z of explicit zeros in the merged
 *     trapezoid, m <= nrelax0, or (m <= nrelax1 and z <= zrelax0), or (m <= nrelax2 and
 *     z <= zrelax1), or z <= zrelax2; passes repeat until none merges. Fractions are compared in
 *     integers: z_count * 1000 <= zrelax_permille * total.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID -1
#define ORC_ERR_NOT_SPD -2
#define ORC_ERR_NOMEM -5

typedef struct {
  int64_t n;
  /* final ordering and permuted matrix C (lower CSC); Cmap[q] = index into the user's Ax */
  int32_t *perm, *iperm;
  int64_t *Cp;
  int32_t *Ci;
  int64_t *Cmap;
  /* etree and column patterns of L (Eq. 1), column j sorted with j first */
  int32_t *parent;
  int64_t *Lp;
  int32_t *Li;
  /* fundamental supernodes: first columns, nfsn+1 entries */
  int32_t nfsn;
  int32_t *fsn;
  /* amalgamated supernodes */
  int32_t nsn;
  int32_t *sn;      /* first column of each, nsn+1 entries */
  int64_t *srp;     /* row-structure pointers, nsn+1 */
  int32_t *sri;     /* rows(J), sorted */
  int32_t *sparent; /* supernodal tree parent or -1 */
  int64_t *dp;      /* descendant-list pointers, nsn+1 */
  int32_t *dk;      /* descendant K of each pair */
  int64_t *dr0;     /* first position in rows(K) at or after first(J) */
  int32_t *dnin;    /* number of rows of K inside cols(J) */
  int64_t *relp;    /* relative-map pointers, one per pair + 1 */
  int32_t *rel;     /* rel[relp[q] + t] = position of rows(K)[r0 + t] in rows(J) */
  int32_t *level;   /* per supernode */
  int32_t nlev;
  int32_t *lvp, *lvl; /* level pointers (nlev+1) and supernodes by level, ascending */
  /* amalgamation log: merge t absorbed the supernode starting at column merges[2t] into the
   * next one, which started at column merges[2t+1] when the merge was made */
  int64_t nmerge;
  int32_t *merges;
  /* numeric factor on the pattern Lp/Li */
  double *Lx;
  int64_t err_col;
} orc_t;

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Input rules: 0-based lower-triangular CSC, rows strictly increasing in a column, the diagonal
 * present and first. */
int orc_validate(int64_t n, const int64_t *Ap, const int32_t *Ai) {
  if (n < 0 || !Ap || (n > 0 && !Ai)) return ORC_ERR_INVALID;
  if (Ap[0] != 0) return ORC_ERR_INVALID;
  for (int64_t j = 0; j < n; ++j) {
    if (Ap[j + 1] <= Ap[j]) return ORC_ERR_INVALID; /* a diagonal is required */
    if (Ai[Ap[j]] != j) return ORC_ERR_INVALID;
    for (int64_t p = Ap[j] + 1; p < Ap[j + 1]; ++p) {
      if (Ai[p] <= Ai[p - 1] || Ai[p] >= n) return ORC_ERR_INVALID;
    }
  }
  return ORC_OK;
}

/* C = P A P^T, lower triangle. perm[k] = original index at position k. C_ij = A_{perm i, perm j}.
 * Cmap[q] is the index of the user's entry that lands at C's entry q. */
static int permute(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *iperm,
                   int64_t **Cp_out, int32_t **Ci_out, int64_t **Cmap_out) {
  int64_t nnz = Ap[n];
  int64_t *Cp = xcalloc(n + 1, sizeof(int64_t));
  int32_t *Ci = xcalloc(nnz, sizeof(int32_t));
  int64_t *Cm = xcalloc(nnz, sizeof(int64_t));
  int64_t *fill = xcalloc(n + 1, sizeof(int64_t));
  if (!Cp || !Ci || !Cm || !fill) return ORC_ERR_NOMEM;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
      int32_t a = iperm[Ai[p]], b = iperm[j];
      int32_t col = a < b ? a : b;
      Cp[col + 1]++;
    }
  for (int64_t j = 0; j < n; ++j) Cp[j + 1] += Cp[j];
  memcpy(fill, Cp, sizeof(int64_t) * (n + 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
      int32_t a = iperm[Ai[p]], b = iperm[j];
      int32_t row = a > b ? a : b, col = a < b ? a : b;
      int64_t q = fill[col]++;
      Ci[q] = row;
      Cm[q] = p;
    }
  /* sort each column by row (insertion sort keeps it simple; columns are short) */
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t p = Cp[j] + 1; p < Cp[j + 1]; ++p) {
      int32_t r = Ci[p];
      int64_t m = Cm[p];
      int64_t q = p - 1;
      while (q >= Cp[j] && Ci[q] > r) {
        Ci[q + 1] = Ci[q];
        Cm[q + 1] = Cm[q];
        --q;
      }
      Ci[q + 1] = r;
      Cm[q + 1] = m;
    }
  }
  free(fill);
  *Cp_out = Cp;
  *Ci_out = Ci;
  *Cmap_out = Cm;
  return ORC_OK;
}

/* Column patterns of L by Eq. (1) and the etree by its definition parent[j] = min(L_j \ {j}).
 * Columns are visited in increasing order, so every child s of j (parent[s] = j < ... ) is
 * complete before j. */
static int column_patterns(int64_t n, const int64_t *Cp, const int32_t *Ci, int32_t **parent_out,
                           int64_t **Lp_out, int32_t **Li_out) {
  int32_t *parent = xcalloc(n, sizeof(int32_t));
  int64_t *Lp = xcalloc(n + 1, sizeof(int64_t));
  int32_t *mark = xcalloc(n, sizeof(int32_t));
  int32_t *buf = xcalloc(n, sizeof(int32_t));
  /* children lists: head/next */
  int32_t *head = xcalloc(n, sizeof(int32_t)), *next = xcalloc(n, sizeof(int32_t));
  int64_t cap = Cp[n] * 2 + 16, used = 0;
  int32_t *Li = malloc(sizeof(int32_t) * cap);
  if (!parent || !Lp || !mark || !buf || !head || !next || !Li) return ORC_ERR_NOMEM;
  for (int64_t j = 0; j < n; ++j) { mark[j] = -1; head[j] = -1; }
  for (int64_t j = 0; j < n; ++j) {
    int64_t len = 0;
    mark[j] = (int32_t)j;
    buf[len++] = (int32_t)j;
    for (int64_t p = Cp[j]; p < Cp[j + 1]; ++p) { /* A_j */
      int32_t i = Ci[p];
      if (mark[i] != j) { mark[i] = (int32_t)j; buf[len++] = i; }
    }
    for (int32_t s = head[j]; s != -1; s = next[s]) { /* children: L_s \ {s} */
      for (int64_t p = Lp[s]; p < Lp[s + 1]; ++p) {
        int32_t i = Li[p];
        if (i == s) continue;
        if (mark[i] != j) { mark[i] = (int32_t)j; buf[len++] = i; }
      }
    }
    qsort(buf, len, sizeof(int32_t), cmp_i32);
    if (used + len > cap) {
      while (used + len > cap) cap *= 2;
      int32_t *t = realloc(Li, sizeof(int32_t) * cap);
      if (!t) return ORC_ERR_NOMEM;
      Li = t;
    }
    memcpy(Li + used, buf, sizeof(int32_t) * len);
    used += len;
    Lp[j + 1] = used;
    parent[j] = len > 1 ? buf[1] : -1; /* buf[0] == j */
    if (parent[j] >= 0) {
      /* append j at the tail of parent's child list, keeping children in increasing order */
      int32_t pj = parent[j];
      next[j] = -1;
      if (head[pj] == -1) head[pj] = (int32_t)j;
      else {
        int32_t t = head[pj];
        while (next[t] != -1) t = next[t];
        next[t] = (int32_t)j;
      }
    }
  }
  free(mark); free(buf); free(head); free(next);
  *parent_out = parent;
  *Lp_out = Lp;
  *Li_out = Li;
  return ORC_OK;
}

/* Postorder of a forest: roots and children in increasing index order. post[k] = node. */
static void postorder(int64_t n, const int32_t *parent, int32_t *post) {
  int32_t *head = xcalloc(n, sizeof(int32_t)), *next = xcalloc(n, sizeof(int32_t));
  int32_t *stack = xcalloc(n, sizeof(int32_t));
  for (int64_t j = 0; j < n; ++j) head[j] = -1;
  /* insert in decreasing order so each list comes out increasing */
  for (int64_t j = n - 1; j >= 0; --j)
    if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = (int32_t)j; }
  int64_t k = 0;
  for (int64_t r = 0; r < n; ++r) {
    if (parent[r] != -1) continue;
    int64_t top = 0;
    stack[top++] = (int32_t)r;
    while (top > 0) {
      int32_t v = stack[top - 1];
      int32_t c = head[v];
      if (c == -1) {
        --top;
        post[k++] = v;
      } else {
        head[v] = next[c]; /* consume the child */
        stack[top++] = c;
      }
    }
  }
  free(head); free(next); free(stack);
}

void orc_free(orc_t *o) {
  if (!o) return;
  free(o->perm); free(o->iperm); free(o->Cp); free(o->Ci); free(o->Cmap);
  free(o->parent); free(o->Lp); free(o->Li); free(o->fsn); free(o->sn); free(o->srp);
  free(o->sri); free(o->sparent); free(o->dp); free(o->dk); free(o->dr0); free(o->dnin);
  free(o->relp); free(o->rel); free(o->level); free(o->lvp); free(o->lvl); free(o->Lx);
  free(o->merges);
  free(o);
}

/* sorted union of two sorted int arrays; returns length */
static int64_t merge_union(const int32_t *a, int64_t na, const int32_t *b, int64_t nb, int32_t *out) {
  int64_t i = 0, j = 0, k = 0;
  while (i < na || j < nb) {
    if (j >= nb || (i < na && a[i] < b[j])) out[k++] = a[i++];
    else if (i >= na || b[j] < a[i]) out[k++] = b[j++];
    else { out[k++] = a[i++]; ++j; }
  }
  return k;
}

static int analyze_impl(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm0,
                        const int32_t *relax, const int32_t *rules, int32_t nrules, const int32_t *fund_rule,
                        int64_t nfund, int want_rel, orc_t **out);

/* Run every symbolic step. perm0 may be NULL (natural order). relax = {nrelax0..2, zrelax0..2
 * per mille}, or NULL for no amalgamation. want_rel != 0 also builds the relative row maps. */
int orc_analyze(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm0,
                const int32_t *relax, int want_rel, orc_t **out) {
  return analyze_impl(n, Ap, Ai, perm0, relax, NULL, 0, NULL, 0, want_rel, out);
}

/* The same with one amalgamation rule per fundamental supernode: rules holds nrules records
 * {amalgamate, nrelax0..2, zrelax0..2 per mille}; the merge of supernode i into the next one
 * follows rules[fund_rule[f]] with f the fundamental supernode that holds the last column of i.
 * Returns ORC_ERR_INVALID when nfund is not the number of fundamental supernodes. */
int orc_analyze_rules(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm0,
                      const int32_t *rules, int32_t nrules, const int32_t *fund_rule, int64_t nfund,
                      int want_rel, orc_t **out) {
  return analyze_impl(n, Ap, Ai, perm0, NULL, rules, nrules, fund_rule, nfund, want_rel, out);
}

static int analyze_impl(int64_t n, const int64_t *Ap, const int32_t *Ai, const int32_t *perm0,
                        const int32_t *relax, const int32_t *rules, int32_t nrules, const int32_t *fund_rule,
                        int64_t nfund, int want_rel, orc_t **out) {
  *out = NULL;
  int rc = orc_validate(n, Ap, Ai);
  if (rc) return rc;
  orc_t *o = xcalloc(1, sizeof(orc_t));
  o->n = n;
  o->err_col = -1;
  int32_t *p0 = xcalloc(n, sizeof(int32_t)), *ip0 = xcalloc(n, sizeof(int32_t));
  for (int64_t k = 0; k < n; ++k) p0[k] = perm0 ? perm0[k] : (int32_t)k;
  for (int64_t k = 0; k < n; ++k) {
    if (p0[k] < 0 || p0[k] >= n) { free(p0); free(ip0); orc_free(o); return ORC_ERR_INVALID; }
    ip0[k] = -1;
  }
  for (int64_t k = 0; k < n; ++k) {
    if (ip0[p0[k]] != -1) { free(p0); free(ip0); orc_free(o); return ORC_ERR_INVALID; }
    ip0[p0[k]] = (int32_t)k;
  }
  /* Pass 1: etree of the given ordering, then its postorder. */
  int64_t *Cp0; int32_t *Ci0; int64_t *Cm0; int32_t *par0; int64_t *Lp0; int32_t *Li0;
  if ((rc = permute(n, Ap, Ai, ip0, &Cp0, &Ci0, &Cm0))) return rc;
  if ((rc = column_patterns(n, Cp0, Ci0, &par0, &Lp0, &Li0))) return rc;
  int32_t *post = xcalloc(n, sizeof(int32_t));
  postorder(n, par0, post);
  free(Cp0); free(Ci0); free(Cm0); free(Lp0); free(Li0); free(par0);
  /* Final ordering: perm[k] = perm0[post[k]]. */
  o->perm = xcalloc(n, sizeof(int32_t));
  o->iperm = xcalloc(n, sizeof(int32_t));
  for (int64_t k = 0; k < n; ++k) o->perm[k] = p0[post[k]];
  for (int64_t k = 0; k < n; ++k) o->iperm[o->perm[k]] = (int32_t)k;
  free(p0); free(ip0); free(post);
  /* Pass 2: C = P A P^T in the final order, its etree and L's column patterns (Eq. 1). */
  if ((rc = permute(n, Ap, Ai, o->iperm, &o->Cp, &o->Ci, &o->Cmap))) return rc;
  if ((rc = column_patterns(n, o->Cp, o->Ci, &o->parent, &o->Lp, &o->Li))) return rc;

  /* Fundamental supernodes (Sec. 3.2 rule). */
  int32_t *nchild = xcalloc(n, sizeof(int32_t));
  for (int64_t j = 0; j < n; ++j) if (o->parent[j] >= 0) nchild[o->parent[j]]++;
  o->fsn = xcalloc(n + 1, sizeof(int32_t));
  o->nfsn = 0;
  for (int64_t j = 0; j < n; ++j) {
    int joins = 0;
    if (j > 0) {
      int64_t cprev = o->Lp[j] - o->Lp[j - 1], cj = o->Lp[j + 1] - o->Lp[j];
      joins = o->parent[j - 1] == j && nchild[j] == 1 && cprev == cj + 1;
    }
    if (!joins) o->fsn[o->nfsn++] = (int32_t)j;
  }
  o->fsn[o->nfsn] = (int32_t)n;
  free(nchild);

  /* Relaxed amalgamation over a linked list of supernodes (fundamental ones to start), each
   * with its row set (the sorted union of its columns' patterns) and its count of true
   * nonzeros. relax = {nrelax0, nrelax1, nrelax2, zrelax0, zrelax1, zrelax2 (per mille)}. */
  int32_t ns = o->nfsn;
  int32_t *first = xcalloc(ns + 1, sizeof(int32_t)), *last = xcalloc(ns + 1, sizeof(int32_t));
  int32_t *nxt = xcalloc(ns + 1, sizeof(int32_t));
  int32_t **rows = xcalloc(ns + 1, sizeof(int32_t *));
  int64_t *nrows = xcalloc(ns + 1, sizeof(int64_t)), *truennz = xcalloc(ns + 1, sizeof(int64_t));
  int32_t *tmp = xcalloc(n + 1, sizeof(int32_t));
  for (int32_t s = 0; s < ns; ++s) {
    first[s] = o->fsn[s];
    last[s] = o->fsn[s + 1] - 1;
    nxt[s] = s + 1;
    int64_t len = 0;
    rows[s] = xcalloc(1, sizeof(int32_t));
    for (int32_t j = first[s]; j <= last[s]; ++j) {
      int64_t cj = o->Lp[j + 1] - o->Lp[j];
      int64_t m = merge_union(rows[s], len, o->Li + o->Lp[j], cj, tmp);
      free(rows[s]);
      rows[s] = xcalloc(m, sizeof(int32_t));
      memcpy(rows[s], tmp, sizeof(int32_t) * m);
      len = m;
      truennz[s] += cj;
    }
    nrows[s] = len;
  }
  int32_t head = 0;
  /* at most ns - 1 merges: each one removes a supernode */
  o->merges = xcalloc(2 * (size_t)(ns > 0 ? ns : 1), sizeof(int32_t));
  o->nmerge = 0;
  int bad_rule = 0;
  for (int64_t f = 0; fund_rule && f < nfund; ++f) bad_rule |= fund_rule[f] < 0 || fund_rule[f] >= nrules;
  if (fund_rule && (nfund != ns || bad_rule)) {
    for (int32_t s = 0; s < ns; ++s) free(rows[s]);
    free(rows); free(first); free(last); free(nxt); free(nrows); free(truennz); free(tmp);
    orc_free(o);
    return ORC_ERR_INVALID;
  }
  if (relax || fund_rule) {
    int changed = 1;
    while (changed) {
      changed = 0;
      int32_t i = head, prev = -1;
      while (i < ns && nxt[i] < ns) {
        int32_t P = nxt[i];
        int32_t ls = last[i];
        if (o->parent[ls] == ls + 1) { /* i is the child whose last column's parent starts P */
          int64_t m = merge_union(rows[i], nrows[i], rows[P], nrows[P], tmp);
          int64_t nc = (int64_t)last[P] - first[i] + 1;
          int64_t total = nc * m - nc * (nc - 1) / 2;
          int64_t z = total - (truennz[i] + truennz[P]);
          /* slot i is the fundamental supernode holding the last column of supernode i */
          int32_t rule_buf[6];
          if (fund_rule) {
            const int32_t *q = rules + 7 * fund_rule[i];
            if (!q[0]) { prev = i; i = P; continue; } /* this rule never merges */
            for (int t = 0; t < 6; ++t) rule_buf[t] = q[1 + t];
            relax = rule_buf;
          }
#if defined(ORC_PLANT_DROP_Z_CLAUSE)
          /* deliberately wrong rules, compiled only into the copies the tests use to show that
           * the amalgamation pin catches over-merging: the zero-fraction clause of the third
           * size class dropped, or || written for && in the second */
          int accept = nc <= relax[0] || (nc <= relax[1] && z * 1000 <= (int64_t)relax[3] * total) ||
                       nc <= relax[2] || z * 1000 <= (int64_t)relax[5] * total;
#elif defined(ORC_PLANT_OR_FOR_AND)
          int accept = nc <= relax[0] || (nc <= relax[1] || z * 1000 <= (int64_t)relax[3] * total) ||
                       (nc <= relax[2] && z * 1000 <= (int64_t)relax[4] * total) ||
                       z * 1000 <= (int64_t)relax[5] * total;
#else
          int accept = nc <= relax[0] || (nc <= relax[1] && z * 1000 <= (int64_t)relax[3] * total) ||
                       (nc <= relax[2] && z * 1000 <= (int64_t)relax[4] * total) ||
                       z * 1000 <= (int64_t)relax[5] * total;
#endif
          if (accept) {
            o->merges[2 * o->nmerge] = first[i];
            o->merges[2 * o->nmerge + 1] = first[P];
            o->nmerge++;
            free(rows[P]);
            rows[P] = xcalloc(m, sizeof(int32_t));
            memcpy(rows[P], tmp, sizeof(int32_t) * m);
            nrows[P] = m;
            first[P] = first[i];
            truennz[P] += truennz[i];
            free(rows[i]);
            rows[i] = NULL;
            if (prev < 0) head = P; else nxt[prev] = P;
            i = P; /* the merged supernode is the next one in order of last column */
            changed = 1;
            continue;
          }
        }
        prev = i;
        i = P;
      }
    }
  }
  int32_t nsn = 0;
  for (int32_t s = head; s < ns; s = nxt[s]) ++nsn;
  o->nsn = nsn;
  o->sn = xcalloc(nsn + 1, sizeof(int32_t));
  o->srp = xcalloc(nsn + 1, sizeof(int64_t));
  {
    int32_t t = 0;
    for (int32_t s = head; s < ns; s = nxt[s], ++t) { o->sn[t] = first[s]; o->srp[t + 1] = o->srp[t] + nrows[s]; }
  }
  o->sn[nsn] = (int32_t)n;
  o->sri = xcalloc(o->srp[nsn], sizeof(int32_t));
  {
    int32_t t = 0;
    for (int32_t s = head; s < ns; s = nxt[s], ++t) memcpy(o->sri + o->srp[t], rows[s], sizeof(int32_t) * nrows[s]);
  }
  for (int32_t s = 0; s < ns; ++s) free(rows[s]);
  free(rows); free(first); free(last); free(nxt); free(nrows); free(truennz); free(tmp);
  ns = nsn;

  /* column -> supernode */
  int32_t *col2sn = xcalloc(n, sizeof(int32_t));
  for (int32_t s = 0; s < ns; ++s)
    for (int32_t j = o->sn[s]; j < o->sn[s + 1]; ++j) col2sn[j] = s;
  /* supernodal tree: parent of J = supernode holding the etree parent of J's last column */
  o->sparent = xcalloc(ns, sizeof(int32_t));
  for (int32_t s = 0; s < ns; ++s) {
    int32_t pl = o->parent[o->sn[s + 1] - 1];
    o->sparent[s] = pl < 0 ? -1 : col2sn[pl];
  }
  /* descendant lists: J collects every K < J that has a row inside cols(J) */
  int64_t *cnt = xcalloc(ns + 1, sizeof(int64_t));
  int32_t *seen = xcalloc(ns, sizeof(int32_t));
  for (int32_t s = 0; s < ns; ++s) seen[s] = -1;
  for (int32_t k = 0; k < ns; ++k)
    for (int64_t p = o->srp[k]; p < o->srp[k + 1]; ++p) {
      int32_t J = col2sn[o->sri[p]];
      if (J != k && seen[J] != k) { seen[J] = k; cnt[J + 1]++; }
    }
  o->dp = xcalloc(ns + 1, sizeof(int64_t));
  for (int32_t s = 0; s < ns; ++s) o->dp[s + 1] = o->dp[s] + cnt[s + 1];
  int64_t npair = o->dp[ns];
  o->dk = xcalloc(npair, sizeof(int32_t));
  o->dr0 = xcalloc(npair, sizeof(int64_t));
  o->dnin = xcalloc(npair, sizeof(int32_t));
  int64_t *fillp = xcalloc(ns, sizeof(int64_t));
  for (int32_t s = 0; s < ns; ++s) { fillp[s] = o->dp[s]; seen[s] = -1; }
  for (int32_t k = 0; k < ns; ++k) /* increasing K keeps every list sorted */
    for (int64_t p = o->srp[k]; p < o->srp[k + 1]; ++p) {
      int32_t J = col2sn[o->sri[p]];
      if (J == k) continue;
      if (seen[J] != k) {
        seen[J] = k;
        int64_t q = fillp[J]++;
        o->dk[q] = k;
        o->dr0[q] = p - o->srp[k];
        o->dnin[q] = 0;
      }
      o->dnin[fillp[J] - 1]++;
    }
  free(cnt); free(seen); free(fillp);
  /* relative maps by binary search of rows(J) (optional: they can be large) */
  o->relp = xcalloc(npair + 1, sizeof(int64_t));
  if (want_rel) {
    for (int32_t J = 0; J < ns; ++J)
      for (int64_t q = o->dp[J]; q < o->dp[J + 1]; ++q) {
        int32_t K = o->dk[q];
        o->relp[q + 1] = o->relp[q] + (o->srp[K + 1] - o->srp[K] - o->dr0[q]);
      }
    o->rel = xcalloc(o->relp[npair], sizeof(int32_t));
    for (int32_t J = 0; J < ns; ++J)
      for (int64_t q = o->dp[J]; q < o->dp[J + 1]; ++q) {
        int32_t K = o->dk[q];
        int64_t t = 0;
        for (int64_t p = o->srp[K] + o->dr0[q]; p < o->srp[K + 1]; ++p, ++t) {
          int32_t r = o->sri[p];
          const int32_t *base = o->sri + o->srp[J];
          const int32_t *hit = bsearch(&r, base, o->srp[J + 1] - o->srp[J], sizeof(int32_t), cmp_i32);
          o->rel[o->relp[q] + t] = hit ? (int32_t)(hit - base) : -1; /* -1: a structure bug */
        }
      }
  }
  /* levels: leaves 0, else 1 + max over children; within a level, ascending J */
  o->level = xcalloc(ns, sizeof(int32_t));
  o->nlev = 0;
  for (int32_t s = 0; s < ns; ++s) { /* children precede parents */
    if (o->sparent[s] >= 0 && o->level[o->sparent[s]] < o->level[s] + 1)
      o->level[o->sparent[s]] = o->level[s] + 1;
  }
  for (int32_t s = 0; s < ns; ++s) if (o->level[s] + 1 > o->nlev) o->nlev = o->level[s] + 1;
  o->lvp = xcalloc(o->nlev + 1, sizeof(int32_t));
  o->lvl = xcalloc(ns, sizeof(int32_t));
  for (int32_t s = 0; s < ns; ++s) o->lvp[o->level[s] + 1]++;
  for (int32_t l = 0; l < o->nlev; ++l) o->lvp[l + 1] += o->lvp[l];
  {
    int32_t *f = xcalloc(o->nlev + 1, sizeof(int32_t));
    for (int32_t l = 0; l < o->nlev; ++l) f[l] = o->lvp[l];
    for (int32_t s = 0; s < ns; ++s) o->lvl[f[o->level[s]]++] = s;
    free(f);
  }
  free(col2sn);
  *out = o;
  return ORC_OK;
}

/* Row patterns of L by the etree walk of Sec. 3.2: for each C_ij (j < i) walk up from j until
 * i or a node already marked for row i. Row i's pattern (without i) is written to rp/ri,
 * sorted. Returns 0, or 1 when it disagrees with the transpose of the column patterns. */
int orc_row_patterns_check(const orc_t *o) {
  int64_t n = o->n;
  int32_t *mark = xcalloc(n, sizeof(int32_t));
  int32_t *buf = xcalloc(n, sizeof(int32_t));
  int64_t *cnt = xcalloc(n + 1, sizeof(int64_t));
  /* row counts of L from the column patterns (transpose) */
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = o->Lp[j] + 1; p < o->Lp[j + 1]; ++p) cnt[o->Li[p]]++;
  /* rows of C: build the transpose of C's strictly-lower part */
  int64_t *Rp = xcalloc(n + 1, sizeof(int64_t));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = o->Cp[j] + 1; p < o->Cp[j + 1]; ++p) Rp[o->Ci[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) Rp[i + 1] += Rp[i];
  int32_t *Rj = xcalloc(Rp[n], sizeof(int32_t));
  int64_t *f = xcalloc(n + 1, sizeof(int64_t));
  memcpy(f, Rp, sizeof(int64_t) * (n + 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = o->Cp[j] + 1; p < o->Cp[j + 1]; ++p) Rj[f[o->Ci[p]]++] = (int32_t)j;
  /* position cursors into each column pattern for the transpose comparison */
  int64_t *cur = xcalloc(n, sizeof(int64_t));
  for (int64_t j = 0; j < n; ++j) { cur[j] = o->Lp[j] + 1; mark[j] = -1; }
  int bad = 0;
  for (int64_t i = 0; i < n && !bad; ++i) {
    int64_t len = 0;
    mark[i] = (int32_t)i;
    for (int64_t p = Rp[i]; p < Rp[i + 1]; ++p) {
      int32_t j = Rj[p];
      while (j != -1 && mark[j] != i) {
        mark[j] = (int32_t)i;
        buf[len++] = j;
        j = o->parent[j];
      }
      if (j == -1) { bad = 1; break; } /* never reached i: not an ancestor */
    }
    if (len != cnt[i]) { bad = 1; break; }
    qsort(buf, len, sizeof(int32_t), cmp_i32);
    for (int64_t t = 0; t < len; ++t) {
      int32_t j = buf[t];
      /* column j's next pattern entry must be row i (rows are visited in increasing i) */
      if (cur[j] >= o->Lp[j + 1] || o->Li[cur[j]] != i) { bad = 1; break; }
      cur[j]++;
    }
  }
  free(mark); free(buf); free(cnt); free(Rp); free(Rj); free(f); free(cur);
  return bad;
}

/* Numeric up-looking Cholesky of C with values Ax (the user's order). Rows 0..kmax-1 are
 * computed (kmax < 0: all); this is the exact leading kmax x kmax factor. For row k:
 *   x = C_{0:k-1,k} scattered; for j in the reach of row k in the etree, increasing:
 *   L_kj = x_j / L_jj; x_i -= L_ij * L_kj for the rows i < k of column j; then
 *   d = C_kk - sum_j L_kj^2 and L_kk = sqrt(d). */
int orc_factor(orc_t *o, const double *Ax, int64_t kmax) {
  int64_t n = o->n;
  if (kmax < 0 || kmax > n) kmax = n;
  free(o->Lx);
  o->Lx = xcalloc(o->Lp[n], sizeof(double));
  o->err_col = -1;
  int64_t *Rp = xcalloc(n + 1, sizeof(int64_t));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = o->Cp[j] + 1; p < o->Cp[j + 1]; ++p) Rp[o->Ci[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) Rp[i + 1] += Rp[i];
  int32_t *Rj = xcalloc(Rp[n], sizeof(int32_t));
  double *Rx = xcalloc(Rp[n], sizeof(double));
  int64_t *f = xcalloc(n + 1, sizeof(int64_t));
  memcpy(f, Rp, sizeof(int64_t) * (n + 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = o->Cp[j] + 1; p < o->Cp[j + 1]; ++p) {
      int64_t q = f[o->Ci[p]]++;
      Rj[q] = (int32_t)j;
      Rx[q] = Ax[o->Cmap[p]];
    }
  int64_t *len = xcalloc(n, sizeof(int64_t)); /* entries filled so far in each column */
  double *x = xcalloc(n, sizeof(double));
  int32_t *mark = xcalloc(n, sizeof(int32_t)), *reach = xcalloc(n, sizeof(int32_t));
  for (int64_t j = 0; j < n; ++j) mark[j] = -1;
  int rc = ORC_OK;
  for (int64_t k = 0; k < kmax; ++k) {
    int64_t nr = 0;
    mark[k] = (int32_t)k;
    for (int64_t p = Rp[k]; p < Rp[k + 1]; ++p) {
      int32_t j = Rj[p];
      x[j] = Rx[p];
      while (mark[j] != k) {
        mark[j] = (int32_t)k;
        reach[nr++] = j;
        j = o->parent[j];
      }
    }
    qsort(reach, nr, sizeof(int32_t), cmp_i32); /* increasing = a topological order */
    double d = Ax[o->Cmap[o->Cp[k]]];           /* C_kk: the diagonal is first */
    for (int64_t t = 0; t < nr; ++t) {
      int32_t j = reach[t];
      double ljj = o->Lx[o->Lp[j]];
      double y = x[j] / ljj;
      x[j] = 0.0;
      for (int64_t p = o->Lp[j] + 1; p < o->Lp[j] + len[j]; ++p) x[o->Li[p]] -= o->Lx[p] * y;
      int64_t q = o->Lp[j] + len[j];
      if (o->Li[q] != k) { rc = ORC_ERR_INVALID; goto done; } /* pattern disagrees with Eq. (1) */
      o->Lx[q] = y;
      len[j]++;
      d -= y * y;
    }
    if (!(d > 0.0)) { o->err_col = k; rc = ORC_ERR_NOT_SPD; goto done; }
    o->Lx[o->Lp[k]] = sqrt(d);
    len[k] = 1;
  }
done:
  free(Rp); free(Rj); free(Rx); free(f); free(len); free(x); free(mark); free(reach);
  return rc;
}

/* Solve A X = B for nrhs column-major right-hand sides (ld = n): y = P b; L y' = y (forward,
 * column oriented); L^T z = y' (backward); x = P^T z. */
int orc_solve(const orc_t *o, int64_t nrhs, const double *B, double *X) {
  int64_t n = o->n;
  double *y = xcalloc(n, sizeof(double));
  for (int64_t c = 0; c < nrhs; ++c) {
    const double *b = B + c * n;
    for (int64_t k = 0; k < n; ++k) y[k] = b[o->perm[k]];
    for (int64_t j = 0; j < n; ++j) {
      y[j] /= o->Lx[o->Lp[j]];
      for (int64_t p = o->Lp[j] + 1; p < o->Lp[j + 1]; ++p) y[o->Li[p]] -= o->Lx[p] * y[j];
    }
    for (int64_t j = n - 1; j >= 0; --j) {
      double s = y[j];
      for (int64_t p = o->Lp[j] + 1; p < o->Lp[j + 1]; ++p) s -= o->Lx[p] * y[o->Li[p]];
      y[j] = s / o->Lx[o->Lp[j]];
    }
    for (int64_t k = 0; k < n; ++k) X[c * n + o->perm[k]] = y[k];
  }
  free(y);
  return ORC_OK;
}

/* ||L L^T - C||_F / ||C||_F over the full symmetric matrices, for the leading kmax columns
 * (kmax <= 0: all). Column b of L L^T (rows a >= b) = sum over j in row b's pattern of
 * L_{:,j} L_bj. */
double orc_factor_residual_with(const orc_t *o, const double *Ax, const double *Lx, int64_t kmax);
double orc_factor_residual(const orc_t *o, const double *Ax, int64_t kmax) {
  return orc_factor_residual_with(o, Ax, o->Lx, kmax);
}

/* The same check for a factor Lx given on the oracle's pattern Lp/Li (for example one computed
 * elsewhere and mapped onto this pattern). */
double orc_factor_residual_with(const orc_t *o, const double *Ax, const double *Lx, int64_t kmax) {
  int64_t n = o->n;
  if (kmax <= 0 || kmax > n) kmax = n;
  /* row patterns of L (transpose) with the value positions */
  int64_t *Rp = xcalloc(n + 1, sizeof(int64_t));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = o->Lp[j]; p < o->Lp[j + 1]; ++p) Rp[o->Li[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) Rp[i + 1] += Rp[i];
  int32_t *Rj = xcalloc(Rp[n], sizeof(int32_t));
  int64_t *Rq = xcalloc(Rp[n], sizeof(int64_t));
  int64_t *f = xcalloc(n + 1, sizeof(int64_t));
  memcpy(f, Rp, sizeof(int64_t) * (n + 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = o->Lp[j]; p < o->Lp[j + 1]; ++p) {
      int64_t q = f[o->Li[p]]++;
      Rj[q] = (int32_t)j;
      Rq[q] = p;
    }
  double *acc = xcalloc(n, sizeof(double));
  double num = 0.0, den = 0.0;
  for (int64_t b = 0; b < kmax; ++b) {
    for (int64_t t = Rp[b]; t < Rp[b + 1]; ++t) {
      int32_t j = Rj[t];
      double lbj = Lx[Rq[t]];
      for (int64_t p = Rq[t]; p < o->Lp[j + 1]; ++p) acc[o->Li[p]] += Lx[p] * lbj;
    }
    for (int64_t p = o->Cp[b]; p < o->Cp[b + 1]; ++p) {
      int32_t a = o->Ci[p];
      double c = Ax[o->Cmap[p]];
      if (a < kmax) {
        double w = (a == b) ? 1.0 : 2.0;
        den += w * c * c;
        acc[a] -= c;
      }
    }
    /* every position touched lies in the pattern of L's column b */
    for (int64_t p = o->Lp[b]; p < o->Lp[b + 1]; ++p) {
      int32_t a = o->Li[p];
      if (a < kmax) {
        double w = (a == b) ? 1.0 : 2.0;
        num += w * acc[a] * acc[a];
      }
      acc[a] = 0.0;
    }
  }
  free(Rp); free(Rj); free(Rq); free(f); free(acc);
  return den > 0 ? sqrt(num / den) : 0.0;
}

/* Normwise backward error max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
 * with A given as its lower triangle in the user's order. */
double orc_backward_error(int64_t n, const int64_t *Ap, const int32_t *Ai, const double *Ax,
                          int64_t nrhs, const double *B, const double *X) {
  double *r = xcalloc(n, sizeof(double)), *rs = xcalloc(n, sizeof(double));
  double anorm = 0.0, worst = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
      int32_t i = Ai[p];
      rs[i] += fabs(Ax[p]);
      if (i != j) rs[j] += fabs(Ax[p]);
    }
  for (int64_t i = 0; i < n; ++i) if (rs[i] > anorm) anorm = rs[i];
  for (int64_t c = 0; c < nrhs; ++c) {
    const double *b = B + c * n, *x = X + c * n;
    for (int64_t i = 0; i < n; ++i) r[i] = b[i];
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = Ap[j]; p < Ap[j + 1]; ++p) {
        int32_t i = Ai[p];
        r[i] -= Ax[p] * x[j];
        if (i != j) r[j] -= Ax[p] * x[i];
      }
    double rn = 0, xn = 0, bn = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (fabs(r[i]) > rn) rn = fabs(r[i]);
      if (fabs(x[i]) > xn) xn = fabs(x[i]);
      if (fabs(b[i]) > bn) bn = fabs(b[i]);
    }
    double eta = rn / (anorm * xn + bn);
    if (eta > worst) worst = eta;
  }
  free(r); free(rs);
  return worst;
}

/* Sparse right-hand side (Sec. 1.1, Sec. 3.1): the nonzero pattern of the solution of L x = b is
 * Reach_L(beta), the nodes reachable in the dependence graph DG_L (edge j -> i for L_ij != 0)
 * from beta = {i : b_i != 0}. Depth-first search from every node of beta; the reverse of the
 * finishing order is a topological order. beta and the result are in the permuted numbering.
 * Returns the reach size; reach must hold n entries. */
int64_t orc_reach(const orc_t *o, int64_t nb, const int32_t *beta, int32_t *reach) {
  int64_t n = o->n;
  uint8_t *mark = xcalloc(n, 1);
  int32_t *stack = xcalloc(n, sizeof(int32_t));
  int64_t *next = xcalloc(n, sizeof(int64_t)); /* next pattern position to explore per node */
  int32_t *finish = xcalloc(n, sizeof(int32_t));
  int64_t nf = 0;
  for (int64_t t = 0; t < nb; ++t) {
    int32_t s = beta[t];
    if (mark[s]) continue;
    int64_t top = 0;
    stack[top++] = s;
    mark[s] = 1;
    next[s] = o->Lp[s] + 1; /* skip the diagonal */
    while (top > 0) {
      int32_t j = stack[top - 1];
      if (next[j] < o->Lp[j + 1]) {
        int32_t i = o->Li[next[j]++];
        if (!mark[i]) {
          mark[i] = 1;
          next[i] = o->Lp[i] + 1;
          stack[top++] = i;
        }
      } else {
        --top;
        finish[nf++] = j;
      }
    }
  }
  for (int64_t t = 0; t < nf; ++t) reach[t] = finish[nf - 1 - t];
  free(mark); free(stack); free(next); free(finish);
  return nf;
}

/* Numeric sparse lower solve over a reach set in topological order (the decoupled code of
 * Sec. 1.1): x = b on beta, zero elsewhere; for j in reach: x_j /= L_jj; x_i -= L_ij x_j for the
 * rows i of column j. x is a dense work vector of n entries (permuted numbering). */
void orc_sparse_lsolve(const orc_t *o, int64_t nr, const int32_t *reach, int64_t nb, const int32_t *beta,
                       const double *bvals, double *x) {
  for (int64_t t = 0; t < nr; ++t) x[reach[t]] = 0.0;
  for (int64_t t = 0; t < nb; ++t) x[beta[t]] = bvals[t];
  for (int64_t t = 0; t < nr; ++t) {
    int32_t j = reach[t];
    x[j] /= o->Lx[o->Lp[j]];
    for (int64_t p = o->Lp[j] + 1; p < o->Lp[j + 1]; ++p) x[o->Li[p]] -= o->Lx[p] * x[j];
  }
}

/* Sizes and read-only views for the Python wrapper. */
int64_t orc_n(const orc_t *o) { return o->n; }
int64_t orc_nnzL(const orc_t *o) { return o->Lp[o->n]; }
int32_t orc_nfsn(const orc_t *o) { return o->nfsn; }
int32_t orc_nsn(const orc_t *o) { return o->nsn; }
int64_t orc_nsrows(const orc_t *o) { return o->srp[o->nsn]; }
int64_t orc_npairs(const orc_t *o) { return o->dp[o->nsn]; }
int64_t orc_nrel(const orc_t *o) { return o->rel ? o->relp[o->dp[o->nsn]] : 0; }
int32_t orc_nlev(const orc_t *o) { return o->nlev; }
int64_t orc_nmerge(const orc_t *o) { return o->nmerge; }
const int32_t *orc_merges(const orc_t *o) { return o->merges; }
int64_t orc_err_col(const orc_t *o) { return o->err_col; }
const int32_t *orc_perm(const orc_t *o) { return o->perm; }
const int32_t *orc_parent(const orc_t *o) { return o->parent; }
const int64_t *orc_Lp(const orc_t *o) { return o->Lp; }
const int32_t *orc_Li(const orc_t *o) { return o->Li; }
const double *orc_Lx(const orc_t *o) { return o->Lx; }
const int64_t *orc_Cp(const orc_t *o) { return o->Cp; }
const int32_t *orc_Ci(const orc_t *o) { return o->Ci; }
const int64_t *orc_Cmap(const orc_t *o) { return o->Cmap; }
const int32_t *orc_fsn(const orc_t *o) { return o->fsn; }
const int32_t *orc_sn(const orc_t *o) { return o->sn; }
const int64_t *orc_srp(const orc_t *o) { return o->srp; }
const int32_t *orc_sri(const orc_t *o) { return o->sri; }
const int32_t *orc_sparent(const orc_t *o) { return o->sparent; }
const int64_t *orc_dp(const orc_t *o) { return o->dp; }
const int32_t *orc_dk(const orc_t *o) { return o->dk; }
const int64_t *orc_dr0(const orc_t *o) { return o->dr0; }
const int32_t *orc_dnin(const orc_t *o) { return o->dnin; }
const int64_t *orc_relp(const orc_t *o) { return o->relp; }
const int32_t *orc_rel(const orc_t *o) { return o->rel; }
const int32_t *orc_level(const orc_t *o) { return o->level; }
const int32_t *orc_lvp(const orc_t *o) { return o->lvp; }
const int32_t *orc_lvl(const orc_t *o) { return o->lvl; }
