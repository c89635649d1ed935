/*
 * Numeric oracle kernels, instantiated by oracle.c for ORC_T = double and
 * ORC_T = double complex (complex symmetric: plain transposes only).
 * TEST INFRASTRUCTURE ONLY (see oracle.c).
 */

/*
 * Left-looking pivot-free LDL^T on a given elimination-closed pattern
 * (Section 2.1's LDL^T simplification of the LU form; Section 4: no
 * pivoting, symmetric permutation only).  L is unit lower triangular,
 * stored strictly below the diagonal on lcp/lri; D on the diagonal.
 *
 *   for j = 0..n-1:
 *     w = A(j:n, j)                                  (rows {j} U struct(j))
 *     for every k < j with L_jk != 0:  w(i) -= L_ik d_k L_jk,  i in {j} U struct(k), i >= j
 *     d_j = w(j);   L_ij = w(i) / d_j  for i in struct(j)
 *
 * Returns 0, or -(j+1) if d_j is zero or not finite (first such column), or
 * -(n+1) if A has an entry outside {j} U struct(j).
 */
int ORC_SFX(orc_ldlt)(int32_t n, const int64_t* cp, const int32_t* ri, const ORC_T* av,
                      const int64_t* lcp, const int32_t* lri, ORC_T* lv, ORC_T* d) {
  /* row lists of L: for each row j the (column k, position p) with lri[p] == j */
  int64_t nnzl = lcp[n];
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t p = 0; p < nnzl; ++p) rp[lri[p] + 1]++;
  for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  int32_t* rk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnzl > 0 ? nnzl : 1));
  int64_t* rpos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnzl > 0 ? nnzl : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) fill[i] = rp[i];
  for (int32_t k = 0; k < n; ++k)
    for (int64_t p = lcp[k]; p < lcp[k + 1]; ++p) {
      rk[fill[lri[p]]] = k;
      rpos[fill[lri[p]]++] = p;
    }
  ORC_T* w = (ORC_T*)calloc((size_t)(n > 0 ? n : 1), sizeof(ORC_T));
  char* in = (char*)calloc((size_t)(n > 0 ? n : 1), 1);      /* membership of {j} U struct(j) */
  int status = 0;
  for (int32_t j = 0; j < n && status == 0; ++j) {
    in[j] = 1;
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) in[lri[p]] = 1;
    for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
      if (!in[ri[p]]) { status = -(n + 1); break; }
      w[ri[p]] = av[p];
    }
    if (status) break;
    for (int64_t q = rp[j]; q < rp[j + 1]; ++q) {
      int32_t k = rk[q];
      int64_t pj = rpos[q];                   /* position of L_jk in column k */
      ORC_T f = lv[pj] * d[k];
      for (int64_t p = pj; p < lcp[k + 1]; ++p) w[lri[p]] -= lv[p] * f;
    }
    d[j] = w[j];
    w[j] = 0;
    in[j] = 0;
    if (ORC_ISBAD(d[j])) status = -(j + 1);
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) {
      lv[p] = w[lri[p]] / d[j];
      w[lri[p]] = 0;
      in[lri[p]] = 0;
    }
  }
  free(rp); free(rk); free(rpos); free(fill); free(w); free(in);
  return status;
}

/*
 * Selected inversion, column form of Eqs. (11)-(13) (Algorithm 1 with
 * one-column supernodes; Lhat = L because L_jj = 1; Uhat = Lhat^T by Eq. 14;
 * U_jj^{-1} L_jj^{-1} = 1/d_j).  For j = n-1 down to 0 with C = struct(j):
 *
 *   X_ij = - sum_{k in C} X_{max(i,k), min(i,k)} L_kj      (i in C)    step 2
 *   X_jj = 1/d_j - sum_{i in C} L_ij X_ij                               step 3
 *
 * X is stored on the same pattern as L (xv) plus its diagonal (xd).  The
 * entries X_{a,b} (a > b, both in C) are found by a merge walk of C against
 * struct(b): C ∩ (b, n) ⊆ struct(b) holds for elimination-closed patterns.
 * The double sum is visited once per unordered pair {a, b} and credited to
 * both rows (X is symmetric).  Returns 0, or -(j+1) if the walk for column j
 * fails (pattern not closed).
 */
int ORC_SFX(orc_selinv)(int32_t n, const int64_t* lcp, const int32_t* lri, const ORC_T* lv,
                        const ORC_T* d, ORC_T* xv, ORC_T* xd) {
  ORC_T* y = (ORC_T*)calloc((size_t)(n > 0 ? n : 1), sizeof(ORC_T));
  int status = 0;
  for (int32_t j = n - 1; j >= 0 && status == 0; --j) {
    int64_t p0 = lcp[j], r = lcp[j + 1] - lcp[j];
    const int32_t* C = lri + p0;
    const ORC_T* Lj = lv + p0;
    for (int64_t a = 0; a < r; ++a) y[a] = 0;
    for (int64_t b = 0; b < r && status == 0; ++b) {
      int32_t k = C[b];
      ORC_T lkj = Lj[b];
      y[b] += xd[k] * lkj;                    /* pair (k, k) */
      int64_t q = lcp[k], qend = lcp[k + 1];
      for (int64_t a = b + 1; a < r; ++a) {   /* pairs (C[a], k), C[a] > k */
        while (q < qend && lri[q] != C[a]) ++q;
        if (q == qend) { status = -(j + 1); break; }
        ORC_T x = xv[q];
        y[a] += x * lkj;
        y[b] += x * Lj[a];
      }
    }
    ORC_T acc = 0;
    for (int64_t a = 0; a < r; ++a) {
      xv[p0 + a] = -y[a];
      acc += Lj[a] * xv[p0 + a];
    }
    xd[j] = 1.0 / d[j] - acc;
  }
  free(y);
  return status;
}

/*
 * The same recurrence on `nthreads` OpenMP threads (timing at scale only),
 * with every X entry formed by one thread by the scalar operations of
 * orc_selinv in the same order, so the result is bitwise that of
 * orc_selinv.  Column j needs only the columns of its ancestors in the
 * elimination tree (C = struct(j) lies on its path to the root), so the
 * columns of one depth of the tree are independent:
 *  - a depth holding many columns: one column per thread, each by the
 *    orc_selinv column step;
 *  - otherwise column by column, the rows of C cut into one contiguous
 *    block [a0, a1) per thread: the thread runs the loop of orc_selinv over
 *    b restricted to its own y entries -- for b < a0 the walk of struct(C[b])
 *    over the rows C[a0..a1) only (started by a binary search), for b in
 *    [a0, a1) the whole walk -- so every y entry receives the same terms in
 *    the same order as there; X_jj by one thread.
 */
static int ORC_SFX(orc_selinv_column)(int32_t j, const int64_t* lcp, const int32_t* lri, const ORC_T* lv,
                                      const ORC_T* d, ORC_T* xv, ORC_T* xd, ORC_T* y) {
  const int64_t p0 = lcp[j], r = lcp[j + 1] - lcp[j];
  const int32_t* C = lri + p0;
  const ORC_T* Lj = lv + p0;
  for (int64_t a = 0; a < r; ++a) y[a] = 0;
  for (int64_t b = 0; b < r; ++b) {
    int32_t k = C[b];
    ORC_T lkj = Lj[b];
    y[b] += xd[k] * lkj;
    int64_t q = lcp[k], qend = lcp[k + 1];
    for (int64_t a = b + 1; a < r; ++a) {
      while (q < qend && lri[q] != C[a]) ++q;
      if (q == qend) return -(j + 1);
      ORC_T x = xv[q];
      y[a] += x * lkj;
      y[b] += x * Lj[a];
    }
  }
  ORC_T acc = 0;
  for (int64_t a = 0; a < r; ++a) {
    xv[p0 + a] = -y[a];
    acc += Lj[a] * xv[p0 + a];
  }
  xd[j] = 1.0 / d[j] - acc;
  return 0;
}

int ORC_SFX(orc_selinv_omp)(int32_t n, const int64_t* lcp, const int32_t* lri, const ORC_T* lv,
                            const ORC_T* d, ORC_T* xv, ORC_T* xd, int32_t nthreads) {
  int status = 0;
  if (nthreads < 1) nthreads = 1;
  if (n <= 0) return 0;
  /* depth of each column below its root (parent(j) = min struct(j)), columns grouped by depth */
  int32_t* depth = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t maxd = 0;
  int64_t maxr = 0;
  for (int32_t j = n - 1; j >= 0; --j) {
    const int64_t r = lcp[j + 1] - lcp[j];
    depth[j] = r > 0 ? depth[lri[lcp[j]]] + 1 : 0;
    if (depth[j] > maxd) maxd = depth[j];
    if (r > maxr) maxr = r;
  }
  int64_t* dptr = (int64_t*)calloc((size_t)maxd + 2, sizeof(int64_t));
  int32_t* dcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t j = 0; j < n; ++j) dptr[depth[j] + 1]++;
  for (int32_t t = 0; t <= maxd; ++t) dptr[t + 1] += dptr[t];
  for (int32_t j = 0; j < n; ++j) dcol[dptr[depth[j]]++] = j;
  for (int32_t t = maxd; t > 0; --t) dptr[t] = dptr[t - 1];
  dptr[0] = 0;
  ORC_T* ybuf = (ORC_T*)calloc((size_t)nthreads * (size_t)(maxr > 0 ? maxr : 1), sizeof(ORC_T));
#pragma omp parallel num_threads(nthreads)
  {
    int tid = 0, nt = 1;
#ifdef _OPENMP
    tid = omp_get_thread_num();
    nt = omp_get_num_threads();
#endif
    ORC_T* y = ybuf + (size_t)tid * (size_t)(maxr > 0 ? maxr : 1);
    for (int32_t t = 0; t <= maxd; ++t) {
      const int64_t c0 = dptr[t], c1 = dptr[t + 1];
      if (c1 - c0 >= 4 * (int64_t)nt) {
#pragma omp for schedule(dynamic, 4)
        for (int64_t c = c0; c < c1; ++c) {
          const int st = ORC_SFX(orc_selinv_column)(dcol[c], lcp, lri, lv, d, xv, xd, y);
          if (st) {
#pragma omp atomic write
            status = st;
          }
        }
        continue;
      }
      for (int64_t c = c0; c < c1; ++c) {
        const int32_t j = dcol[c];
        const int64_t p0 = lcp[j], r = lcp[j + 1] - lcp[j];
        const int32_t* C = lri + p0;
        const ORC_T* Lj = lv + p0;
        const int64_t a0 = r * tid / nt, a1 = r * (tid + 1) / nt;
        for (int64_t a = a0; a < a1; ++a) y[a - a0] = 0;
        int bad = 0;
        for (int64_t b = 0; b < a1 && !bad; ++b) {
          const int32_t k = C[b];
          const ORC_T lkj = Lj[b];
          int64_t q = lcp[k], qend = lcp[k + 1];
          if (b < a0) {                       /* rows C[a0..a1) of column k */
            int64_t lo = q, hi = qend;
            while (lo < hi) {
              const int64_t mid = lo + (hi - lo) / 2;
              if (lri[mid] < C[a0]) lo = mid + 1; else hi = mid;
            }
            q = lo;
            for (int64_t a = a0; a < a1; ++a) {
              while (q < qend && lri[q] != C[a]) ++q;
              if (q == qend) { bad = 1; break; }
              y[a - a0] += xv[q] * lkj;
            }
            continue;
          }
          y[b - a0] += xd[k] * lkj;           /* b in [a0, a1): the loop of orc_selinv */
          for (int64_t a = b + 1; a < r; ++a) {
            while (q < qend && lri[q] != C[a]) ++q;
            if (q == qend) { bad = 1; break; }
            const ORC_T x = xv[q];
            if (a < a1) y[a - a0] += x * lkj;
            y[b - a0] += x * Lj[a];
          }
        }
        if (bad) {
#pragma omp atomic write
          status = -(j + 1);
        }
        for (int64_t a = a0; a < a1; ++a) xv[p0 + a] = -y[a - a0];
#pragma omp barrier
#pragma omp single
        {
          ORC_T acc = 0;
          for (int64_t a = 0; a < r; ++a) acc += Lj[a] * xv[p0 + a];
          xd[j] = 1.0 / d[j] - acc;
        }
      }
    }
  }
  free(ybuf);
  free(depth);
  free(dptr);
  free(dcol);
  return status;
}

/*
 * Solve A x = b with A = L D L^T (in place on b): L z = b, z /= d, L^T x = z.
 * This is the direct inversion of Eq. (6) one right-hand side at a time,
 * used to check columns of the inverse.
 */
int ORC_SFX(orc_solve)(int32_t n, const int64_t* lcp, const int32_t* lri, const ORC_T* lv,
                       const ORC_T* d, ORC_T* b) {
  for (int32_t j = 0; j < n; ++j)
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) b[lri[p]] -= lv[p] * b[j];
  for (int32_t j = 0; j < n; ++j) b[j] /= d[j];
  for (int32_t j = n - 1; j >= 0; --j) {
    ORC_T acc = b[j];
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) acc -= lv[p] * b[lri[p]];
    b[j] = acc;
  }
  return 0;
}

/*
 * Non-symmetric A with a symmetric pattern: left-looking pivot-free
 * A = L D U' with L unit lower, U' unit upper and D diagonal -- the LU
 * factorisation Algorithm 1 takes as input, with U = D U' (so the pivots
 * of U are D and U_KK^{-1} L_KK^{-1} = U'_KK^{-1} D_K^{-1} L_KK^{-1}).
 * Input: av = A_ij and au = A_ji at every stored lower position (i, j),
 * i >= j, of the same CSC pattern (au's diagonal entries are not read).
 * Output on the L pattern: lv = L_ij and uv = U'_ji (the upper factor held
 * transposed, at the position of L_ij), plus d.
 *
 *   for j = 0..n-1:
 *     w(i) = A_ij, v(i) = A_ji                        (i in {j} U struct(j))
 *     for every k < j with j in struct(k):
 *       w(i) -= L_ik d_k U'_kj,  v(i) -= L_jk d_k U'_ki  (i in {j} U struct(k), i >= j)
 *     d_j = w(j);  L_ij = w(i) / d_j;  U'_ji = v(i) / d_j   (i in struct(j))
 *
 * Returns 0, -(j+1) for a zero or non-finite pivot, -(n+1) for an entry
 * outside the pattern.
 */
int ORC_SFX(orc_ldu)(int32_t n, const int64_t* cp, const int32_t* ri, const ORC_T* av, const ORC_T* au,
                     const int64_t* lcp, const int32_t* lri, ORC_T* lv, ORC_T* uv, ORC_T* d) {
  int64_t nnzl = lcp[n];
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t p = 0; p < nnzl; ++p) rp[lri[p] + 1]++;
  for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  int32_t* rk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnzl > 0 ? nnzl : 1));
  int64_t* rpos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnzl > 0 ? nnzl : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) fill[i] = rp[i];
  for (int32_t k = 0; k < n; ++k)
    for (int64_t p = lcp[k]; p < lcp[k + 1]; ++p) {
      rk[fill[lri[p]]] = k;
      rpos[fill[lri[p]]++] = p;
    }
  ORC_T* w = (ORC_T*)calloc((size_t)(n > 0 ? n : 1), sizeof(ORC_T));
  ORC_T* v = (ORC_T*)calloc((size_t)(n > 0 ? n : 1), sizeof(ORC_T));
  char* in = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  int status = 0;
  for (int32_t j = 0; j < n && status == 0; ++j) {
    in[j] = 1;
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) in[lri[p]] = 1;
    for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
      if (!in[ri[p]]) { status = -(n + 1); break; }
      w[ri[p]] = av[p];
      if (ri[p] != j) v[ri[p]] = au[p];
    }
    if (status) break;
    for (int64_t q = rp[j]; q < rp[j + 1]; ++q) {
      int32_t k = rk[q];
      int64_t pj = rpos[q];                   /* position of (j, k) in column k */
      ORC_T fl = uv[pj] * d[k];               /* d_k U'_kj */
      ORC_T fu = lv[pj] * d[k];               /* L_jk d_k */
      w[j] -= lv[pj] * fl;                    /* i = j: L_jk d_k U'_kj */
      for (int64_t p = pj + 1; p < lcp[k + 1]; ++p) {
        w[lri[p]] -= lv[p] * fl;
        v[lri[p]] -= uv[p] * fu;
      }
    }
    d[j] = w[j];
    w[j] = 0;
    in[j] = 0;
    if (ORC_ISBAD(d[j])) status = -(j + 1);
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) {
      lv[p] = w[lri[p]] / d[j];
      uv[p] = v[lri[p]] / d[j];
      w[lri[p]] = 0;
      v[lri[p]] = 0;
      in[lri[p]] = 0;
    }
  }
  free(rp); free(rk); free(rpos); free(fill); free(w); free(v); free(in);
  return status;
}

/*
 * Non-symmetric selected inversion, column form of Algorithm 1 (one-column
 * supernodes: Lhat = L and Uhat = U' because L_jj = U'_jj = 1, and
 * U_jj^{-1} L_jj^{-1} = 1/d_j).  For j = n-1 down to 0 with C = struct(j):
 *
 *   X_ij = - sum_{k in C} X_ik L_kj            (i in C)    step 2
 *   X_jj = 1/d_j - sum_{k in C} U'_jk X_kj                 step 3
 *   X_ji = - sum_{k in C} U'_jk X_ki           (i in C)    step 4
 *
 * X is held as xv (X_ij at the L position (i, j), i > j), xu (X_ji at the
 * same position) and xd.  For a, b in C with a > b, X_ab is xv and X_ba is
 * xu at the position of a in struct(b), found by the same merge walk as the
 * symmetric form.  Returns 0, or -(j+1) if the walk for column j fails.
 */
int ORC_SFX(orc_selinv_lu)(int32_t n, const int64_t* lcp, const int32_t* lri, const ORC_T* lv, const ORC_T* uv,
                           const ORC_T* d, ORC_T* xv, ORC_T* xu, ORC_T* xd) {
  ORC_T* y = (ORC_T*)calloc((size_t)(n > 0 ? n : 1), sizeof(ORC_T));   /* sum_k X_{C[a],k} L_kj */
  ORC_T* z = (ORC_T*)calloc((size_t)(n > 0 ? n : 1), sizeof(ORC_T));   /* sum_k U'_jk X_{k,C[a]} */
  int status = 0;
  for (int32_t j = n - 1; j >= 0 && status == 0; --j) {
    int64_t p0 = lcp[j], r = lcp[j + 1] - lcp[j];
    const int32_t* C = lri + p0;
    const ORC_T* Lj = lv + p0;                /* L_{C[a], j} */
    const ORC_T* Uj = uv + p0;                /* U'_{j, C[a]} */
    for (int64_t a = 0; a < r; ++a) y[a] = z[a] = 0;
    for (int64_t b = 0; b < r && status == 0; ++b) {
      int32_t k = C[b];
      y[b] += xd[k] * Lj[b];                  /* X_kk L_kj */
      z[b] += Uj[b] * xd[k];                  /* U'_jk X_kk */
      int64_t q = lcp[k], qend = lcp[k + 1];
      for (int64_t a = b + 1; a < r; ++a) {   /* C[a] > k */
        while (q < qend && lri[q] != C[a]) ++q;
        if (q == qend) { status = -(j + 1); break; }
        ORC_T xlo = xv[q];                    /* X_{C[a], k} */
        ORC_T xup = xu[q];                    /* X_{k, C[a]} */
        y[a] += xlo * Lj[b];
        y[b] += xup * Lj[a];
        z[a] += Uj[b] * xup;
        z[b] += Uj[a] * xlo;
      }
    }
    ORC_T acc = 0;
    for (int64_t a = 0; a < r; ++a) {
      xv[p0 + a] = -y[a];
      xu[p0 + a] = -z[a];
      acc += Uj[a] * xv[p0 + a];
    }
    xd[j] = 1.0 / d[j] - acc;
  }
  free(y); free(z);
  return status;
}

/* Solve A x = b with A = L D U' (in place): L w = b, w /= d, U' x = w. */
int ORC_SFX(orc_solve_lu)(int32_t n, const int64_t* lcp, const int32_t* lri, const ORC_T* lv, const ORC_T* uv,
                          const ORC_T* d, ORC_T* b) {
  for (int32_t j = 0; j < n; ++j)
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) b[lri[p]] -= lv[p] * b[j];
  for (int32_t j = 0; j < n; ++j) b[j] /= d[j];
  for (int32_t j = n - 1; j >= 0; --j) {
    ORC_T acc = b[j];
    for (int64_t p = lcp[j]; p < lcp[j + 1]; ++p) acc -= uv[p] * b[lri[p]];
    b[j] = acc;
  }
  return 0;
}
