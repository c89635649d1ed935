/*
 * Plain CPU oracle for supernodal selected inversion (PSelInv, arXiv
 * 1404.0447).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it; the GPU library never links or calls
 * it, and it shares no code with the GPU library.
 *
 * Everything here is deliberately scalar and column-by-column:
 *
 *  - symbolic analysis: elimination tree (Section 2.2's parent rule applied
 *    to single columns), column structures of L, a supernode partition
 *    (Section 2.1: contiguous columns with a dense diagonal block and a shared
 *    structure below, relaxed to a maximum width), the supernodal tree, the
 *    priority numbers of Algorithm 2 and the relative-index map that places
 *    the rows of each supernode's set C inside the ancestor supernodes;
 *  - numeric: a left-looking, pivot-free LDL^T (Section 2.1's symmetric
 *    simplification; no pivoting, symmetric permutation only, Section 4) and
 *    the column form of the selected-inversion recurrence of Eqs. (7)-(13)
 *    applied one column at a time (Algorithm 1 with one-column supernodes,
 *    U = D L^T so that Uhat = Lhat^T, Eq. 14);
 *  - helpers: log-determinant from D, and a solve with L and D (the direct
 *    inversion of Eq. 6, used to check columns of the inverse).
 *
 * Complex matrices are complex *symmetric*: every transpose is a plain
 * transpose, never a conjugate transpose.
 *
 * Index conventions: lower-triangular CSC with the diagonal first in each
 * column and rows sorted; colptr int64, row indices int32.  The L pattern
 * is stored strictly below the diagonal ("struct(j)"), D separately.
 *
 * Parity pins: every function here is checked against values fixed
 * independently of this file.  Per function, the test that a plausible
 * mistake in it (a dropped term, a wrong sign or index, an off-by-one in a
 * threshold) would fail:
 *   orc_etree, orc_sym_*      brute-force boolean elimination on random
 *                             patterns (test_oracle_pins::test_symbolic_vs_brute_force),
 *                             Figure 1's tree (test_figure1_worked_example)
 *   orc_postorder             random forests: children before parents, subtrees
 *                             contiguous (test_postorder_of_random_forest)
 *   orc_supernodes            hand-derived partitions of chains, a 5 x 5 grid and
 *                             cases on both sides of the 5% zero threshold
 *                             (tests/golden/relaxed_supernodes.txt,
 *                             test_supernode_golden); width caps and the
 *                             zero bound (test_supernode_rule_properties)
 *   orc_sn_struct, orc_relidx the definition ancestor-row by ancestor-row on
 *                             random patterns (test_relative_indices_definition),
 *                             Figure 1 (test_figure1_worked_example)
 *   orc_ldlt_*, orc_selinv_*  dense inverses of random SPD and complex symmetric
 *                             matrices (test_tiny_random_vs_dense_inverse), exact
 *                             rational inverses (test_exact_rational_inverse), the
 *                             closed form of tridiag(-1,2,-1) and of grid
 *                             Laplacians (test_laplacian_1d_closed_form_and_linear_work,
 *                             test_oracle_vs_grid_closed_form_nd_order), the trace
 *                             identity (test_trace_identity_grid2d_31)
 *   orc_selinv_omp            bitwise equal to the one-thread sweep
 *                             (test_oracle_omp)
 *   orc_solve_*               numpy.linalg.solve (test_solve_vs_numpy)
 *   orc_logdet_*              numpy.linalg.slogdet (test_logdet_vs_slogdet)
 *   orc_ldu_*, orc_selinv_lu_*, orc_solve_lu_*
 *                             tests/test_oracle_lu_pins.py: dense and exact
 *                             rational inverses, Usmani's closed form for
 *                             tridiagonal inverses, L D U' reproducing A, the
 *                             convection-diffusion closed form, bitwise reduction
 *                             to the symmetric sweep when A is symmetric
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Symbolic analysis                                                         */
/* ------------------------------------------------------------------------ */

/* Check the input is lower CSC, diagonal first, rows strictly increasing. */
static int check_lower(int32_t n, const int64_t* cp, const int32_t* ri) {
  for (int32_t j = 0; j < n; ++j) {
    if (cp[j + 1] < cp[j] + 1) return -1;
    if (ri[cp[j]] != j) return -1;
    for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p)
      if (ri[p] <= ri[p - 1] || ri[p] >= n) return -1;
  }
  return 0;
}

/*
 * Elimination tree: parent(j) = min{ i > j : L_ij != 0 } (Section 2.2, for
 * single columns).  Computed from the pattern of A by the usual ancestor
 * walk with path compression: for every A_ij (i > j) follow j's current
 * ancestor chain up to a root r < i and link r under i.  Roots get -1.
 */
int orc_etree(int32_t n, const int64_t* cp, const int32_t* ri, int32_t* parent) {
  if (check_lower(n, cp, ri)) return -1;
  int32_t* anc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  /* visit the entries row by row: A_ij with i > j is seen when i is reached,
     so build the row-wise (transposed) lists first */
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int32_t j = 0; j < n; ++j)
    for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p) rp[ri[p] + 1]++;
  for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  int32_t* cj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) fill[i] = rp[i];
  for (int32_t j = 0; j < n; ++j)
    for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p) cj[fill[ri[p]]++] = j;
  for (int32_t i = 0; i < n; ++i) {
    parent[i] = -1;
    anc[i] = -1;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
      int32_t k = cj[q];
      while (k != -1 && k < i) {
        int32_t next = anc[k];
        anc[k] = i;               /* path compression */
        if (next == -1) { parent[k] = i; break; }
        k = next;
      }
    }
  }
  free(anc); free(rp); free(cj); free(fill);
  return 0;
}

/*
 * Postorder of a forest given by parent[] (parent > child, roots = -1):
 * a depth-first walk, roots taken in increasing order and the children of
 * every node in increasing order; post[k] = the node finished k-th.
 */
int orc_postorder(int32_t n, const int32_t* parent, int32_t* post) {
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i <= n; ++i) head[i] = -1;
  /* push children in decreasing order so each list reads increasing;
     the virtual node n is the parent of every root */
  for (int32_t j = n - 1; j >= 0; --j) {
    int32_t p = parent[j] < 0 ? n : parent[j];
    next[j] = head[p];
    head[p] = j;
  }
  int32_t k = 0, top = 0;
  /* iterative DFS: stack holds nodes whose children are being visited */
  for (int32_t root = head[n]; root != -1; root = next[root]) {
    stack[top++] = root;
    while (top > 0) {
      int32_t v = stack[top - 1];
      int32_t c = head[v];
      if (c == -1) {
        post[k++] = v;
        --top;
      } else {
        head[v] = next[c];        /* consume the first unvisited child */
        stack[top++] = c;
      }
    }
  }
  free(head); free(next); free(stack);
  return k == n ? 0 : -1;
}

/*
 * Column structures of L (strictly below the diagonal):
 *   struct(j) = ( { i > j : A_ij != 0 }  U  union over children c of struct(c) ) \ {j}
 * computed column by column in increasing j with a marker array, then sorted.
 * Returned through an opaque object because nnz(L) is not known in advance.
 */
typedef struct {
  int32_t n;
  int32_t* parent;
  int64_t* lcp;
  int32_t* lri;
} orc_sym;

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

void* orc_sym_new(int32_t n, const int64_t* cp, const int32_t* ri) {
  orc_sym* s = (orc_sym*)calloc(1, sizeof(orc_sym));
  s->n = n;
  s->parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (orc_etree(n, cp, ri, s->parent)) { free(s->parent); free(s); return NULL; }
  /* children lists */
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) head[i] = -1;
  for (int32_t j = n - 1; j >= 0; --j)
    if (s->parent[j] >= 0) { next[j] = head[s->parent[j]]; head[s->parent[j]] = j; }
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) mark[i] = -1;
  int64_t cap = 1024;
  for (int32_t j = 0; j < n; ++j) cap += cp[j + 1] - cp[j];
  s->lcp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  s->lri = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  s->lcp[0] = 0;
  int64_t len = 0;
  for (int32_t j = 0; j < n; ++j) {
    int64_t start = len;
    mark[j] = j;                                  /* exclude j itself */
#define PUSH(row)                                                        \
    do {                                                                 \
      int32_t r_ = (row);                                                \
      if (mark[r_] != j) {                                               \
        mark[r_] = j;                                                    \
        if (len == cap) {                                                \
          cap *= 2;                                                      \
          s->lri = (int32_t*)realloc(s->lri, sizeof(int32_t) * (size_t)cap); \
        }                                                                \
        s->lri[len++] = r_;                                              \
      }                                                                  \
    } while (0)
    for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p) PUSH(ri[p]);
    for (int32_t c = head[j]; c != -1; c = next[c])
      for (int64_t p = s->lcp[c]; p < s->lcp[c + 1]; ++p) PUSH(s->lri[p]);
#undef PUSH
    qsort(s->lri + start, (size_t)(len - start), sizeof(int32_t), cmp_i32);
    s->lcp[j + 1] = len;
  }
  free(head); free(next); free(mark);
  return s;
}

int64_t orc_sym_nnzl(void* h) { return ((orc_sym*)h)->lcp[((orc_sym*)h)->n]; }

void orc_sym_get(void* h, int32_t* parent, int64_t* lcp, int32_t* lri) {
  orc_sym* s = (orc_sym*)h;
  if (parent) memcpy(parent, s->parent, sizeof(int32_t) * (size_t)s->n);
  if (lcp) memcpy(lcp, s->lcp, sizeof(int64_t) * (size_t)(s->n + 1));
  if (lri) memcpy(lri, s->lri, sizeof(int32_t) * (size_t)s->lcp[s->n]);
}

void orc_sym_free(void* h) {
  orc_sym* s = (orc_sym*)h;
  if (!s) return;
  free(s->parent); free(s->lcp); free(s->lri); free(s);
}

/*
 * Supernode partition (Section 2.1).  The paper relaxes "maximal columns
 * with identical structure" by a width cap and by merging nearly identical
 * patterns without giving the rule; the rule used here is:
 *   (1) fundamental supernodes: column j+1 joins j's supernode iff
 *       parent(j) = j+1, j is the only child of j+1 and
 *       |struct(j)| = |struct(j+1)| + 1;
 *   (2) if relax != 0: walk the supernodes in increasing order; the current
 *       (possibly already merged) node K merges into the next node P when
 *       P contains parent(last(K)), first(P) = last(K)+1,
 *       width(K)+width(P) <= wmax, and either the merged width is <= 8 or
 *       the merged panel's explicit zeros are <= 5% of its stored entries;
 *       stored entries of a node of width s with r rows below are
 *       s(s+1)/2 + s*r, true entries are sum over its columns of
 *       1 + |struct(j)|, and the merged node has the rows below of P;
 *   (3) if wmax > 0: split every node wider than wmax into chunks of wmax
 *       columns from its first column (the last chunk is narrower).
 * Returns the number of supernodes; sn_start gets nsn+1 entries.
 */
int32_t orc_supernodes(int32_t n, const int32_t* parent, const int64_t* lcp,
                       int32_t wmax, int32_t relax, int32_t* sn_start) {
  if (n <= 0) { sn_start[0] = 0; return 0; }
  int32_t* nchild = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  for (int32_t j = 0; j < n; ++j) if (parent[j] >= 0) nchild[parent[j]]++;
  /* (1) fundamental */
  int32_t* fs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t nf = 0;
  for (int32_t j = 0; j < n; ++j) {
    int join = 0;
    if (j > 0) {
      int64_t c_prev = lcp[j] - lcp[j - 1];      /* |struct(j-1)| */
      int64_t c_this = lcp[j + 1] - lcp[j];      /* |struct(j)|   */
      join = parent[j - 1] == j && nchild[j] == 1 && c_prev == c_this + 1;
    }
    if (!join) fs[nf++] = j;
  }
  fs[nf] = n;
  /* (2) relaxed merging */
  int32_t* ms = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t nm = 0;
  if (relax && wmax > 0) {
    int32_t cur_first = fs[0];
    int64_t cur_true = 0;
    for (int32_t j = fs[0]; j < fs[1]; ++j) cur_true += 1 + (lcp[j + 1] - lcp[j]);
    for (int32_t k = 0; k < nf; ++k) {
      int32_t cur_last = fs[k + 1] - 1;
      int merged = 0;
      if (k + 1 < nf) {
        int32_t pf = fs[k + 1], pl = fs[k + 2] - 1;
        int32_t par = parent[cur_last];
        if (par >= pf && par <= pl) {             /* P contains parent(last(K)) */
          int64_t sK = cur_last - cur_first + 1, sP = pl - pf + 1;
          int64_t s = sK + sP;
          int64_t rP = lcp[pl + 1] - lcp[pl];     /* rows below P = struct(last(P)) */
          int64_t ptrue = 0;
          for (int32_t j = pf; j <= pl; ++j) ptrue += 1 + (lcp[j + 1] - lcp[j]);
          int64_t stored = s * (s + 1) / 2 + s * rP;
          int64_t zeros = stored - cur_true - ptrue;
          if (s <= wmax && (s <= 8 || 20 * zeros <= stored)) {
            merged = 1;
            cur_true += ptrue;                    /* cur_first unchanged */
          }
        }
      }
      if (!merged) {
        ms[nm++] = cur_first;
        if (k + 1 < nf) {
          cur_first = fs[k + 1];
          cur_true = 0;
          for (int32_t j = fs[k + 1]; j < fs[k + 2]; ++j) cur_true += 1 + (lcp[j + 1] - lcp[j]);
        }
      }
    }
  } else {
    for (int32_t k = 0; k < nf; ++k) ms[nm++] = fs[k];
  }
  ms[nm] = n;
  /* (3) split */
  int32_t ns = 0;
  for (int32_t k = 0; k < nm; ++k) {
    int32_t f = ms[k], l = ms[k + 1];
    if (wmax > 0) {
      for (int32_t c = f; c < l; c += wmax) sn_start[ns++] = c;
    } else {
      sn_start[ns++] = f;
    }
  }
  sn_start[ns] = n;
  free(nchild); free(fs); free(ms);
  return ns;
}

/*
 * Supernodal structure for a given partition sn_start[0..nsn]:
 *   R(K) = ( union over j in K of struct(j) ) \ cols(K), sorted  (rows below K,
 *          the set C of Algorithm 1 step 0 in the symmetric case);
 *   parent(K) = the supernode containing min R(K) (Section 2.2), -1 if empty;
 *   sigma(K) by Algorithm 2: sigma(root) = 1, sigma(K) = sigma(parent(K)) + 1,
 *          assigned from the last supernode down to the first.
 * Outputs: sn_parent[nsn], sigma[nsn], rcount[nsn] (=|R(K)|); if rrows is
 * non-NULL, the R(K) lists concatenated in supernode order.
 */
int orc_sn_struct(int32_t n, const int64_t* lcp, const int32_t* lri, int32_t nsn,
                  const int32_t* sn_start, int32_t* sn_parent, int32_t* sigma,
                  int64_t* rcount, int32_t* rrows) {
  int32_t* col2sn = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t k = 0; k < nsn; ++k)
    for (int32_t j = sn_start[k]; j < sn_start[k + 1]; ++j) col2sn[j] = k;
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) mark[i] = -1;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t out = 0;
  for (int32_t k = 0; k < nsn; ++k) {
    int32_t f = sn_start[k], l = sn_start[k + 1] - 1;
    int32_t m = 0;
    for (int32_t j = f; j <= l; ++j)
      for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) {
        int32_t i = lri[p];
        if (i > l && mark[i] != k) { mark[i] = k; buf[m++] = i; }
      }
    qsort(buf, (size_t)m, sizeof(int32_t), cmp_i32);
    rcount[k] = m;
    sn_parent[k] = m > 0 ? col2sn[buf[0]] : -1;
    if (rrows) { memcpy(rrows + out, buf, sizeof(int32_t) * (size_t)m); }
    out += m;
  }
  for (int32_t k = nsn - 1; k >= 0; --k)
    sigma[k] = sn_parent[k] < 0 ? 1 : sigma[sn_parent[k]] + 1;
  free(col2sn); free(mark); free(buf);
  return 0;
}

/*
 * Relative indices (how the rows of C are found inside the ancestors'
 * storage, Section 3.1's non-contiguous row-index lists).  For supernode K
 * with rows below C = R(K) (length r), split C into maximal runs of rows
 * lying in one supernode J ("blocks", in increasing order).  For a block
 * starting at position p of C and every i in [p, r), the entry is the
 * position of C[i] in J's panel row list  cols(J) followed by R(J).
 * Entries are concatenated block by block and supernode by supernode.
 * Pass relidx = NULL to get only the total count (returned).
 * nblk[K] gets the number of blocks of K.
 */
int64_t orc_relidx(int32_t n, int32_t nsn, const int32_t* sn_start, const int64_t* rcount,
                   const int32_t* rrows, int32_t* nblk, int32_t* relidx) {
  int32_t* col2sn = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t k = 0; k < nsn; ++k)
    for (int32_t j = sn_start[k]; j < sn_start[k + 1]; ++j) col2sn[j] = k;
  int64_t* roff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nsn + 1));
  roff[0] = 0;
  for (int32_t k = 0; k < nsn; ++k) roff[k + 1] = roff[k] + rcount[k];
  int64_t total = 0;
  for (int32_t k = 0; k < nsn; ++k) {
    const int32_t* C = rrows + roff[k];
    int64_t r = rcount[k];
    int32_t nb = 0;
    int64_t p = 0;
    while (p < r) {
      int32_t J = col2sn[C[p]];
      int64_t q = p;
      while (q < r && col2sn[C[q]] == J) ++q;
      nb++;
      if (relidx) {
        int32_t fJ = sn_start[J], sJ = sn_start[J + 1] - sn_start[J];
        const int32_t* RJ = rrows + roff[J];
        int64_t rJ = rcount[J];
        for (int64_t i = p; i < r; ++i) {
          int32_t row = C[i];
          int32_t pos = -1;
          if (row < fJ + sJ) {
            pos = row - fJ;                       /* one of J's own columns */
          } else {                                /* binary search in R(J) */
            int64_t lo = 0, hi = rJ;
            while (lo < hi) {
              int64_t mid = (lo + hi) / 2;
              if (RJ[mid] < row) lo = mid + 1; else hi = mid;
            }
            if (lo < rJ && RJ[lo] == row) pos = sJ + (int32_t)lo;
          }
          relidx[total + (i - p)] = pos;          /* -1 would mean "not closed" */
        }
      }
      total += r - p;
      p = q;
    }
    if (nblk) nblk[k] = nb;
  }
  free(col2sn); free(roff);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Numeric part, instantiated for double and double complex                 */
/* ------------------------------------------------------------------------ */

#define ORC_T double
#define ORC_SFX(name) name##_d
#define ORC_ISBAD(x) (!isfinite(x) || (x) == 0.0)
#include "oracle_num.h"
#undef ORC_T
#undef ORC_SFX
#undef ORC_ISBAD

#define ORC_T double complex
#define ORC_SFX(name) name##_z
#define ORC_ISBAD(x) (!isfinite(creal(x)) || !isfinite(cimag(x)) || ((x) == 0.0))
#include "oracle_num.h"
#undef ORC_T
#undef ORC_SFX
#undef ORC_ISBAD

/* log det A = sum_j log d_j.  Real: sum of log|d_j| plus the number of
   negative pivots (sign = (-1)^neg).  Complex: sum of principal logs. */
int orc_logdet_d(int32_t n, const double* d, double* out) {
  double s = 0.0;
  int neg = 0;
  for (int32_t j = 0; j < n; ++j) { s += log(fabs(d[j])); neg += d[j] < 0; }
  out[0] = s;
  out[1] = (double)neg;
  return 0;
}

int orc_logdet_z(int32_t n, const double* dz, double* out) {
  const double complex* d = (const double complex*)dz;
  double re = 0.0, im = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    re += log(cabs(d[j]));
    im += carg(d[j]);
  }
  out[0] = re;
  out[1] = im;
  return 0;
}
