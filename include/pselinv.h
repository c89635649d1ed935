/*
 * pselinv -- supernodal selected inversion of sparse symmetric matrices on
 * one NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Method: L. Lin, M. Jacquelin, C. Yang, "PSelInv -- A Distributed Memory
 * Parallel Algorithm for Selected Inversion: the Symmetric Case"
 * (arXiv 1404.0447).  Given A = L D L^T (pivot-free, symmetric permutation
 * only; Section 4), the library computes every entry of A^{-1} on the
 * pattern of L + L^T (Section 1, Eq. 1 and the superset remark that
 * follows it) by the supernodal recurrence of Algorithm 1 in the symmetric
 * form of Eq. 14:
 *
 *   step 1  Lhat_{C,K} = L_{C,K} (L_{K,K})^{-1}
 *   step 2  X_{C,K}    = - X_{C,C} Lhat_{C,K}
 *   step 3  X_{K,K}    = L_{K,K}^{-T} D_K^{-1} L_{K,K}^{-1} - Lhat_{C,K}^T X_{C,K},
 *           then X_{K,K} <- (X_{K,K} + X_{K,K}^T) / 2   (end of Section 2.1)
 *   step 4  X_{K,C} = X_{C,K}^T (not stored: lower triangle only)
 *
 * supernodes taken level by level in the priority order of Algorithm 2.
 * Complex matrices are complex symmetric: all transposes are plain.
 *
 * Non-symmetric matrices with a symmetric pattern (opts.unsym = 1) use
 * Algorithm 1 in its general form on the pivot-free A = L D U' (L unit
 * lower, U' unit upper, U = D U'):
 *
 *   step 1  Lhat_{C,K} = L_{C,K} (L_{K,K})^{-1},  Uhat_{K,C} = (U'_{K,K})^{-1} U'_{K,C}
 *   step 2  X_{C,K} = - X_{C,C} Lhat_{C,K}
 *   step 3  X_{K,K} = U'_{K,K}^{-1} D_K^{-1} L_{K,K}^{-1} - Uhat_{K,C} X_{C,K}   (no symmetrisation)
 *   step 4  X_{K,C} = - Uhat_{K,C} X_{C,C}
 *
 * The upper factor and the upper triangle of X are stored transposed in
 * panels of the lower layout ("U panels", "XU panels"): panel position
 * (i, j), i >= j, holds U'_{j,i} and X_{j,i}.
 *
 * Conventions for every entry point:
 *  - Status: 0 = PSELINV_OK, < 0 = error (PSELINV_ERR_*).  After an error,
 *    pselinv_last_error(handle) returns a message (and, for a bad pivot,
 *    the column).  No entry point aborts or traps.
 *  - Host pointers ("h_") are read during the call and may be freed after
 *    it returns; device pointers ("d_") must stay valid until the work
 *    enqueued on the given stream has completed.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default).
 *  - Values are laid out batch-major: member b of a batch of B matrices
 *    sharing one pattern starts at b * nnz (elements of the dtype).
 *  - complex128 values are interleaved (re, im) pairs of doubles.
 *  - There is no CPU fallback: without a usable GPU the numeric entry
 *    points return PSELINV_ERR_CUDA.
 *  - A handle may be used by one host thread at a time.
 */
#ifndef PSELINV_H
#define PSELINV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PSELINV_OK 0
#define PSELINV_ERR_ARG (-1)        /* bad argument (null pointer, size, option) */
#define PSELINV_ERR_NOT_LOWER (-2)  /* pattern is not lower CSC, sorted, diagonal first */
#define PSELINV_ERR_ZERO_PIVOT (-3) /* a pivot d_j is exactly zero */
#define PSELINV_ERR_NONFINITE (-4)  /* a pivot d_j is Inf or NaN */
#define PSELINV_ERR_OOM (-5)        /* device allocation failed */
#define PSELINV_ERR_CUDA (-6)       /* CUDA runtime error or no device */
#define PSELINV_ERR_TIMEOUT (-7)    /* a bounded device wait ran out */
#define PSELINV_ERR_STATE (-8)      /* call out of order (e.g. selinv before factor) */
#define PSELINV_ERR_RANGE (-9)      /* FP64 emulation: X is not positive definite (a diagonal entry
                                       <= 0, or a scaled entry out of its slice range) */

/* value types */
#define PSELINV_F64 0
#define PSELINV_C128 1

/* supernode relaxation (Section 2.1: width cap plus merging of nearly
   identical patterns) */
#define PSELINV_RELAX_NONE 0  /* fundamental supernodes, split at the width cap */
#define PSELINV_RELAX_AMALG 1 /* merge child into parent (rule in pselinv_analyze) */

/* selected-inversion schedules (Algorithm 3 and Section 3.3) */
#define PSELINV_PLAIN 0 /* one supernode per launch, reverse postorder */
#define PSELINV_LEVEL 1 /* one grouped launch per kernel per level of Algorithm 2 */
#define PSELINV_GRAPH 2 /* the LEVEL sequence captured once into a CUDA graph and replayed */
#define PSELINV_PERSISTENT 3 /* one persistent launch for the whole sweep running every level's work
                                from one task list with bounded dependency waits and no barrier
                                between levels; captured once into a CUDA graph and replayed */

typedef struct pselinv_handle pselinv_handle;

typedef struct {
  int32_t dtype;          /* PSELINV_F64 or PSELINV_C128 */
  int32_t batch;          /* B >= 1 matrices sharing the pattern (e.g. poles H - z_l I) */
  int32_t max_sn_width;   /* width cap w_max, 1..128; 0 means 128 */
  int32_t relax;          /* PSELINV_RELAX_NONE or PSELINV_RELAX_AMALG */
  int32_t small_cutoff;   /* supernodes narrower than this use the narrowest padding-minimal tiles,
                             wider ones prefer 64-column tiles; < 0 = padding-minimal everywhere */
  int32_t split_k_rows;   /* step 2 of a supernode with |C| = r is split into ceil(r / split_k_rows)
                             partial products summed in slice order (by the CTA that finishes a
                             tile's last slice); <= 0 = no split */
  int32_t debug_checks;   /* nonzero: kernels bounds-check every index and report */
  int32_t unsym;          /* 0: symmetric A = L D L^T.  1: non-symmetric A with a symmetric pattern,
                             A = L D U' (pselinv_factor_unsym; Algorithm 1 with step 4); complex
                             non-symmetric handles cap w_max at 112 (shared-memory budget of the
                             diagonal-block factorisation) */
  int64_t spin_limit_ns;  /* limit for bounded device waits; <= 0 = 1e9 */
  int32_t level_tiles;    /* a level whose step-2 (step-3) tiles number fewer than this gets its slices
                             (row chunks) of C shrunk until it has about this many; 0 = 128 per SM (19456) */
  int32_t min_slice_rows; /* smallest step-2 slice that shrinking makes; 0 = 128 (step-3 chunks: a quarter) */
  int32_t fp64_emulation; /* 0: steps 2 and 3 in FP64 (mma.sync f64).  1 (mma.sync bf16, opt-in, outside
                             the FP64 hot path): step 2, X_{C,K} = -X_{C,C} Lhat_{C,K}, and step 3's
                             Lhat_{C,K}^T X_{C,K} (Algorithm 1),
                             in FP64 accuracy on the bf16 tensor cores, for real symmetric
                             positive definite A (dtype F64, unsym 0, pivot-free factor; PLAIN, LEVEL and
                             GRAPH schedules).  With e_p = ceil(log2 sqrt(X_pp)), every entry of
                             2^-(e_p+e_q) X has modulus < 1 (Cauchy-Schwarz for SPD X); the scaled X and
                             the row-scaled Lhat are cut into 7 signed 8-bit slices each, the 28 slice
                             products of weight >= 2^-48 are formed with exact FP32 sums over 32-row
                             chunks and accumulated in 64-bit integers; the error per term is below
                             2^-53 of 2^(e_i + F_j) (F_j: exponent of column j of the scaled Lhat).
                             Costs 16 bytes per X panel entry and per Lhat entry of device memory.
                             A matrix whose X is not positive definite is detected (X_pp <= 0 or a
                             scaled entry >= 2) and reported as PSELINV_ERR_RANGE by
                             pselinv_sync_status; that selinv's X is then invalid. */
} pselinv_opts;

/* Sizes and work counts of an analysed handle. */
typedef struct {
  int64_t n;              /* matrix order */
  int64_t nnz_a;          /* entries of A's lower triangle (diagonal included) */
  int64_t nnz_l;          /* entries of the supernodal L pattern, lower, diagonal included */
  int64_t panel_entries;  /* sum over supernodes of (s + r) * s: one panel array */
  int64_t relidx_len;     /* relative-index entries */
  int32_t nsn;            /* supernodes */
  int32_t nlevels;        /* priority lists of Algorithm 2 */
  int32_t max_width;      /* widest supernode */
  int32_t batch;
  int64_t max_r;          /* largest |C| */
  double flops_selinv;    /* sum_K 2 r^2 s + 3 r s^2 + 2/3 s^3 (real flops per matrix; x4 for complex);
                             non-symmetric: sum_K 4 r^2 s + 4 r s^2 + 4/3 s^3 */
  double flops_gemm1;     /* sum_K 2 r^2 s (non-symmetric: 4 r^2 s, steps 2 and 4) */
  double bytes_selinv;    /* algorithmic HBM bytes of one selinv (per matrix) */
  int64_t device_bytes;   /* device memory the handle holds (after factor) */
} pselinv_info;

/* Read-only view of the symbolic analysis, owned by the handle (valid until
   pselinv_destroy).  Supernodes are numbered in column order; all arrays
   are host memory. */
typedef struct {
  int64_t n;
  int32_t nsn;
  int32_t nlevels;
  const int32_t* perm;      /* [n] internal index k is user index perm[k] (user perm then postorder) */
  const int32_t* parent;    /* [n] column elimination tree (Section 2.2), -1 = root */
  const int32_t* sn_start;  /* [nsn+1] first column of each supernode */
  const int32_t* sn_parent; /* [nsn] supernodal tree, -1 = root */
  const int32_t* sigma;     /* [nsn] priority numbers of Algorithm 2 (1 = root) */
  const int64_t* rowptr;    /* [nsn+1] offsets into rows */
  const int32_t* rows;      /* R(K): sorted rows below supernode K (the set C of Alg. 1) */
  const int64_t* panel_off; /* [nsn+1] element offset of each (s+r) x s column-major panel */
  const int64_t* relptr;    /* [nsn+1] offsets into relidx */
  const int32_t* relidx;    /* relative indices, see pselinv_analyze */
  const int32_t* nblk;      /* [nsn] ancestor blocks of each C */
  const int32_t* level_ptr; /* [nlevels+1] offsets into level_sn */
  const int32_t* level_sn;  /* [nsn] supernodes of level k (k = 0 is sigma 1), costliest first */
  /* Schur groups of the factorisation (the supernodes of a level whose sets
     C are pairwise disjoint, so their updates hit disjoint entries and run in
     one launch without atomics): level k's groups are
     group_ptr[k] .. group_ptr[k+1]-1, group g's supernodes
     group_sn[group_sn_ptr[g] .. group_sn_ptr[g+1]-1]; supernodes with an
     empty C may be absent */
  int32_t ngroups;
  const int32_t* group_ptr;     /* [nlevels+1] */
  const int32_t* group_sn_ptr;  /* [ngroups+1] */
  const int32_t* group_sn;
} pselinv_symbolic;

/* Fill *o with defaults: F64, batch 1, w_max 128, RELAX_AMALG, padding-minimal
   tiles, split_k_rows 1024, no debug checks, 1 s spin limit, level_tiles and
   min_slice_rows 0 (19456 and 128), fp64_emulation 0. */
void pselinv_default_opts(pselinv_opts* o);

/*
 * Symbolic analysis (host only; no device work until pselinv_factor).
 * Section 2.1 (supernodes), Section 2.2 (elimination tree), Algorithm 1
 * step 0 (the sets C), Algorithm 2 (priority lists).
 *
 * n                order of A (1 <= n < 2^31)
 * h_colptr[n+1]    lower-CSC column pointers of A (int64)
 * h_rowind[nnz]    row indices, sorted inside each column, diagonal first
 * h_perm[n]        optional symmetric ordering (internal k = user h_perm[k]);
 *                  NULL = identity.  The elimination tree is then postordered
 *                  (children in increasing order) and that postorder is
 *                  composed into the ordering.
 * opts             NULL = defaults
 * out              receives the handle (caller destroys it)
 *
 * Supernode rule: (1) fundamental supernodes: column j+1 joins j's
 * supernode iff parent(j) = j+1, j is j+1's only child and
 * |struct(j)| = |struct(j+1)| + 1; (2) with RELAX_AMALG, walking the
 * supernodes in column order, the current node K merges into the next node
 * P if P contains parent(last(K)), width(K)+width(P) <= w_max and either
 * the merged width is <= 8 or its explicit zeros are <= 5% of its stored
 * entries (a node of width s with r rows below stores s(s+1)/2 + s r);
 * (3) nodes wider than w_max are split into chunks of w_max from the left.
 *
 * Relative indices: for supernode K with rows below C (|C| = r), split C
 * into maximal runs lying in one supernode J ("blocks"); for a block
 * starting at position p and every i in [p, r) the entry is the position of
 * C[i] in J's panel rows (J's columns, then R(J)); blocks and supernodes
 * are concatenated in order.
 *
 * Errors: ERR_ARG (null pointers, n out of range, bad options),
 * ERR_NOT_LOWER (pattern not lower CSC / unsorted / missing diagonal /
 * perm not a permutation).
 */
int pselinv_analyze(int64_t n, const int64_t* h_colptr, const int32_t* h_rowind,
                    const int32_t* h_perm, const pselinv_opts* opts, pselinv_handle** out);

/*
 * Symbolic analysis of an uneven batch: k independent symmetric matrices,
 * each with its own pattern and optional ordering, analysed as the one
 * block-diagonal matrix diag(A_0, ..., A_{k-1}).  Its elimination forest has
 * one tree per member, so the priority lists of Algorithm 2 (roots at 1)
 * merge the members level by level and every level runs as one grouped
 * launch over all members.  Member b's unknowns are n_0 + ... + n_{b-1} + [0, n_b)
 * and its stored values follow those of members 0..b-1 (values of
 * pselinv_factor, outputs of pselinv_get_selected / pselinv_logdet_grad /
 * pselinv_selinv_adjoint).  h_perm may be NULL, or hold NULL entries.
 * Errors as pselinv_analyze (a member's failure names the member).
 */
int pselinv_analyze_batch(int32_t k, const int64_t* h_n, const int64_t* const* h_colptr,
                          const int32_t* const* h_rowind, const int32_t* const* h_perm, const pselinv_opts* opts,
                          pselinv_handle** out);

/*
 * Numeric factorisation A = L D L^T on the device (supernodal, level by
 * level from the leaves; no pivoting, Section 4); it produces the input of
 * the selected inversion.  Per level: the diagonal blocks, the panel solves,
 * then the Schur updates of the ancestors in groups of supernodes whose
 * update targets are disjoint (fixed order, no atomics): L and D, and so X,
 * are bitwise reproducible from run to run.  The handle's X panels serve as
 * scratch (the panel solve's L_{C,K} D_K): a selected inverse computed before
 * is gone.
 *
 * d_values   device, batch x nnz_a values of A's lower CSC in the user's
 *            order (dtype of the handle)
 * Enqueues the work on stream and returns without synchronising.  A zero
 * or non-finite pivot is recorded on the device (first bad column, internal
 * order) and reported by the next pselinv_sync_status or pselinv_logdet as
 * ERR_ZERO_PIVOT / ERR_NONFINITE (message via pselinv_last_error), which
 * also returns the handle to the unfactored state; a selinv enqueued before
 * that check computes with the bad factor.  Errors returned directly:
 * ERR_ARG, ERR_STATE, ERR_OOM, ERR_CUDA.
 */
int pselinv_factor(pselinv_handle* h, const void* d_values, void* stream);

/*
 * Numeric factorisation A = P L D L^T P^T of a symmetric indefinite A with
 * Bunch-Kaufman 1x1/2x2 pivots (Bunch and Kaufman 1977, the accuracy remedy
 * of Section 4 and the conclusions) restricted to each supernode's diagonal
 * block: P only permutes the columns of a supernode among themselves, so the
 * symbolic analysis, the panels and every schedule stay as they are.  Per
 * supernode, at pivot position k of the reduced diagonal block: a = |T_kk|,
 * colmax = max_{i>k} |T_ik| at imax (|re| + |im| for complex); a >= alpha
 * colmax -> 1x1; else, rowmax = the largest off-diagonal magnitude of
 * row/column imax: a rowmax >= alpha colmax^2 -> 1x1; |T_imax,imax| >= alpha
 * rowmax -> 1x1 after a symmetric interchange of k and imax; else a 2x2 pivot
 * on (k, k+1) after interchanging k+1 and imax; alpha = (1 + sqrt 17) / 8
 * (LAPACK xSYTF2's rule, applied inside the block).  The L panels then hold
 * each supernode's columns in pivot order (L zero beside a 2x2 block, D's
 * diagonal on the diagonal slots); the selected inversion undoes the order,
 * so X, pselinv_get_selected, pselinv_logdet and pselinv_logdet_grad are as
 * for pselinv_factor.  pselinv_selinv_adjoint needs the pivot-free factor.
 * d_values as for pselinv_factor (the X panels serve as scratch here too).
 * Errors: ERR_ZERO_PIVOT for a reduced
 * column that is entirely zero or a singular 2x2 block (first column, internal
 * order) and ERR_NONFINITE, both reported as for pselinv_factor (no
 * synchronisation here), ERR_STATE on non-symmetric handles.
 */
int pselinv_factor_bk(pselinv_handle* h, const void* d_values, void* stream);

/*
 * Pivots of the last pselinv_factor_bk, host arrays of batch x n (internal
 * column order, member-major): h_piv[b * n + j] = the supernode-local
 * original column at pivot position j - first(K) of its supernode K;
 * h_type = 0 for a 1x1 pivot, 1 and 2 for the first and second column of a
 * 2x2 pivot.  Synchronises.  ERR_STATE without a pivoted factor.
 */
int pselinv_get_pivots(pselinv_handle* h, int32_t* h_piv, int8_t* h_type, void* stream);

/*
 * Numeric factorisation of a non-symmetric A with a symmetric pattern
 * (handle analysed with opts.unsym = 1): A = L D U', supernodal, level by
 * level from the leaves, no pivoting.  Per supernode K: the diagonal block
 * A_KK = L_KK D_K U'_KK by Gaussian elimination, L_{C,K} = A_{C,K}
 * U'_KK^{-1} D_K^{-1}, U'_{K,C} = D_K^{-1} L_KK^{-1} A_{K,C}, and the Schur
 * update A_{C,C} -= L_{C,K} D_K U'_{K,C} into the ancestors (both triangles).
 *
 * d_lower  device, batch x nnz_a: A_ij at every stored lower position (i, j),
 *          i >= j, of the pattern given to pselinv_analyze (user order)
 * d_upper  device, batch x nnz_a: A_ji at the same positions (the entries
 *          at diagonal positions are not read)
 * The X and XU panels serve as scratch, as in pselinv_factor.
 * Errors as pselinv_factor; ERR_STATE on a symmetric handle.
 */
int pselinv_factor_unsym(pselinv_handle* h, const void* d_lower, const void* d_upper, void* stream);

/*
 * Selected inversion (Algorithm 3's normalisation pass, then steps 2-3 of
 * Algorithm 1 for every supernode, top-down in the priority order of
 * Algorithm 2).  The result stays in the handle's X panels (same layout as
 * the L panels: per supernode an (s + r) x s column-major block, rows = the
 * supernode's columns then R(K); the s x s diagonal block is full and
 * symmetric).  mode: PSELINV_PLAIN, PSELINV_LEVEL, PSELINV_GRAPH or
 * PSELINV_PERSISTENT.  Non-symmetric handles: steps 2, 3 and 4 per level
 * (the diagonal block is full and not symmetric; the upper triangle goes to
 * the XU panels); PLAIN, LEVEL and GRAPH only (ERR_ARG for PERSISTENT).
 * Enqueues work only; no host synchronisation.  ERR_STATE before factor.
 */
int pselinv_selinv(pselinv_handle* h, int32_t mode, void* stream);

/*
 * Selected inversion with the result streamed to host memory: the LEVEL
 * schedule of pselinv_selinv, and on an internal copy stream the X panels of
 * every level copied to h_x as soon as that level of Algorithm 2 has
 * finished (its supernodes' panels are final then), so the device-to-host
 * transfer overlaps the rest of the sweep; the deepest levels, whose many
 * small supernodes are scattered through the panel array, are copied after
 * the last level.  The paper keeps X distributed and has no counterpart.
 *
 * h_x   host, batch x panel_entries elements (the layout of
 *       pselinv_get_panels(which = 0)); pinned memory gives the overlap,
 *       pageable memory works but serialises the copies with the sweep
 * h_xu  non-symmetric handles: the XU panels likewise (NULL = not copied);
 *       must be NULL on symmetric handles
 * When `stream` completes, both the device panels and the host copies are
 * complete.  Enqueues work only.  ERR_STATE before factor.
 */
int pselinv_selinv_to_host(pselinv_handle* h, void* h_x, void* h_xu, void* stream);

/*
 * Copy panels to caller memory: which = 0 for X (after selinv), 1 for L
 * (after factor; unit diagonal not stored, D on the diagonal positions);
 * non-symmetric handles also 2 for the XU panels (X_{j,i} at position
 * (i, j)) and 3 for the U panels (U'_{j,i} at (i, j), diagonal slots unused).
 * out: batch x panel_entries elements of the dtype, in device memory or in
 * host memory the CUDA runtime can address (pinned host memory gives an
 * asynchronous copy on `stream`; pageable host memory a synchronous one).
 */
int pselinv_get_panels(pselinv_handle* h, int32_t which, void* out, void* stream);

/*
 * Synchronise `stream` and report device-side failures of earlier enqueued
 * work on h: PSELINV_ERR_ZERO_PIVOT / PSELINV_ERR_NONFINITE if the last
 * factorisation met a bad pivot (first column, internal order; reported
 * until the next factorisation, the handle is back to "not factored"),
 * PSELINV_ERR_TIMEOUT if a bounded wait of the PERSISTENT schedule ran out
 * (that call's results are invalid; the flag is cleared and the handle stays
 * usable), PSELINV_ERR_RANGE if a selinv with opts.fp64_emulation met an X
 * that is not positive definite (same treatment).  Returns PSELINV_OK
 * otherwise.
 */
int pselinv_sync_status(pselinv_handle* h, void* stream);

/*
 * Debug switches (failure-detection tests; no paper counterpart).  Bit 1
 * (value 2): the next PERSISTENT pselinv_selinv arms one dependency wait
 * that is never satisfied, so it must end by the spin limit with
 * PSELINV_ERR_TIMEOUT from pselinv_sync_status instead of hanging.
 */
int pselinv_set_debug(pselinv_handle* h, int32_t flags);

/*
 * Gather the selected inverse at the positions of A's lower CSC in the
 * user's order (the requested set of Eq. 1): d_out[b * nnz_a + q] =
 * (A_b^{-1})_{i,j} for the q-th stored entry (i, j).  Device pointer,
 * batch x nnz_a elements.  This is also the gradient of log det A with
 * respect to each stored entry read as a full-matrix entry.
 */
int pselinv_get_selected(pselinv_handle* h, void* d_out, void* stream);

/*
 * Non-symmetric handles: the upper triangle of the selected inverse at the
 * stored lower positions, d_out[b * nnz_a + q] = (A_b^{-1})_{j,i} for the
 * q-th stored entry (i, j) (the diagonal repeats pselinv_get_selected's).
 * ERR_STATE on a symmetric handle.
 */
int pselinv_get_selected_upper(pselinv_handle* h, void* d_out, void* stream);

/*
 * Gradient of log det A with respect to the stored values of A's lower CSC
 * in the user's order: d log det A = tr(A^{-1} dA), and a stored
 * off-diagonal value stands for both A_ij and A_ji, so
 * d_out[b * nnz_a + q] = X_jj for a diagonal entry and 2 X_ij for an
 * off-diagonal one (X = A_b^{-1} from the last pselinv_selinv; plain
 * transpose for complex symmetric A).  Device pointer, batch x nnz_a.
 * Symmetric handles only (ERR_STATE otherwise).
 */
int pselinv_logdet_grad(pselinv_handle* h, void* d_out, void* stream);

/*
 * Pole sum of a batch (the expansion of Section 4.4, Gamma = sum_l w_l
 * (H - z_l S)^{-1}, on the selected pattern): d_out = sum_b w_b X_b in the
 * X panel layout (one panel array, dtype of the handle).  h_weights: host,
 * batch complex weights as (re, im) pairs for C128 handles, batch real
 * weights for F64 handles.  Requires selinv.  HBM-bound pass over the batch.
 * Symmetric handles only (ERR_STATE otherwise).
 */
int pselinv_pole_sum(pselinv_handle* h, const double* h_weights, void* d_out, void* stream);

/*
 * The selected inversion of the batch (LEVEL schedule, as pselinv_selinv)
 * with the pole sum of Section 4.4 accumulated in its write step:
 * d_out = sum_b w_b X_b in the X panel layout, formed while the sweep runs.
 * The step-3 finish writes each panel entry last, so the CTA that finishes a
 * supernode's share for the last member of the batch sums that share over
 * the members in order b = 0, 1, ... (no value atomics; bitwise
 * reproducible, the same arithmetic as pselinv_pole_sum).  The X panels of
 * every member are kept as by pselinv_selinv.  h_weights as for
 * pselinv_pole_sum.  Errors: ERR_ARG (NULL argument, fp64_emulation set),
 * ERR_STATE (non-symmetric handle, no factor, a pivoted factor), ERR_OOM,
 * ERR_CUDA.  Allocates nsn x 32 counters on first use.
 */
int pselinv_selinv_pole_sum(pselinv_handle* h, const double* h_weights, void* d_out, void* stream);

/*
 * Trace pairing of Section 4.3, Eq. (16): for every batch member b,
 * S_b = sum over the nonzeros of A_b (both triangles) of X_ij A_ji, so that
 * E_b = |1 - S_b / n|.  d_values: the batch's values of A (as passed to
 * pselinv_factor).  h_out: host, batch x 2 doubles (re, im; im = 0 for F64).
 * Requires selinv.  Synchronises the stream.  Symmetric handles only.
 */
int pselinv_trace_sum(pselinv_handle* h, const void* d_values, double* h_out, void* stream);

/*
 * log det A = sum_j log d_j (Section 2.1's LDL^T, or the pivots of
 * A = L D U' for non-symmetric handles).  h_out (host) receives
 * per batch member two doubles: F64 -> (sum log|d_j|, number of negative
 * pivots); C128 -> (real, imaginary) of the sum of principal logs.
 * Synchronises the stream.
 */
int pselinv_logdet(pselinv_handle* h, double* h_out, void* stream);

/*
 * Adjoint of the selected inversion.  For J = <G, X> = sum over the full
 * symmetric selected pattern of G_ij X_ij (bilinear: no conjugation for
 * complex symmetric A), returns dJ/d(stored values of A's lower CSC), user
 * order: -(X G X)_jj on the diagonal and -2 (X G X)_ij off it (a stored
 * off-diagonal value stands for A_ij and A_ji), the same convention as
 * pselinv_logdet_grad.
 *
 * d_G      device, batch x panel_entries in the X panel layout, read
 *          according to g_kind:
 *          PSELINV_G_SYMMETRIC: G symmetric on the selected pattern; only
 *            the lower triangle of each diagonal block and the rows below
 *            are read (J as above);
 *          PSELINV_G_PANEL: d_G holds dJ/d(panel entries of X) for any J
 *            (every panel entry read; the diagonal block's two triangles are
 *            separate entries), e.g. the incoming gradient of an autograd
 *            function whose output is the X panels
 * d_gradA  device, batch x nnz_a
 * Requires a prior pselinv_selinv on the same factor (uses X, L, D;
 * recomputes Lhat and (L_KK)^{-1}).  Reverse sweep leaves -> root of the
 * recurrence of Algorithm 1 (steps 3, 2, 1 in that order per supernode,
 * scattering into the ancestors' adjoints through the relative indices, in
 * the factorisation's groups of supernodes with disjoint targets: no
 * atomics, bitwise reproducible), then the adjoint of the supernodal LDL^T
 * root -> leaves.  Allocates its work buffers on first use.  Symmetric
 * handles only (ERR_STATE otherwise).
 */
#define PSELINV_G_SYMMETRIC 0
#define PSELINV_G_PANEL 1
int pselinv_selinv_adjoint(pselinv_handle* h, const void* d_G, int32_t g_kind, void* d_gradA, void* stream);

/*
 * Kernel timing of the selected inversion (measurement support, no paper
 * counterpart beyond Section 4.2's per-phase timings).  enable != 0 makes
 * every later pselinv_selinv in PLAIN or LEVEL mode record CUDA events on
 * its stream around each kernel class; pselinv_get_timing waits for them
 * and returns in h_ms[PSELINV_NTIMERS] the summed milliseconds since the
 * previous pselinv_get_timing (or enable), in h_launches[PSELINV_NTIMERS]
 * the kernel launches per class, and resets both.  GRAPH mode does not
 * record.  Classes:
 *   0 normalisation (diagonal inverses, Lhat)   1 step 2 (X_{C,K})
 *   2 step 3 partial products                    3 step 3 finish (symmetrise)
 */
#define PSELINV_NTIMERS 4
int pselinv_set_timing(pselinv_handle* h, int32_t enable);
int pselinv_get_timing(pselinv_handle* h, double* h_ms, int64_t* h_launches);

/*
 * Autotuner (measurement-driven choice of the schedule; no paper
 * counterpart beyond Section 3.3's remark that task order matters).  On a
 * factored handle, times pselinv_selinv (LEVEL schedule, CUDA events on
 * `stream`, best of two after a warm-up) for each candidate schedule --
 * first split_k_rows over {0, 512, 1024, 2048, 4096} with the current
 * small_cutoff, then small_cutoff over {-1, 32, 64} with the best split,
 * then level_tiles over {4864, 9728, 19456} -- keeps the fastest in the
 * handle, then times the GRAPH and PERSISTENT modes on it, and returns
 * h_best[0] = split_k_rows, h_best[1] = small_cutoff, h_best[2] =
 * level_tiles, h_best[3] = the fastest mode (h_best holds 4 entries) and
 * that mode's time in *h_best_ms.
 * Overwrites the X panels; drops a captured GRAPH schedule.  Synchronises.
 */
int pselinv_autotune(pselinv_handle* h, int32_t* h_best, double* h_best_ms, void* stream);

int pselinv_get_info(const pselinv_handle* h, pselinv_info* info);
int pselinv_export_symbolic(const pselinv_handle* h, pselinv_symbolic* view);

/*
 * Allocation-free inverse of a batch of small dense blocks from their LDL^T
 * factors: d_M[b] = L_b^{-T} D_b^{-1} L_b^{-1}, which equals A_b^{-1} when
 * A_b = L_b D_b L_b^T.  The paper has no counterpart: this exists for callers that may not call cudaMalloc or
 * cudaFree (cudaFree synchronises the device and cudaMalloc can stall) --
 * code running inside another framework's memory pool or under a fixed
 * memory budget, loops that must never block on the allocator.  It calls no
 * allocating routine; its only scratch (the L^{-1} blocks) is a file-scope
 * device array of 2^21 doubles (16 MiB) that every GPU loading this library
 * holds until the process exits.
 *
 * s         block order, 1..128
 * count     number of blocks; count * s * s must be <= 2^21, else ERR_ARG
 * d_L       device, count blocks of s x s column-major (ld s); only the
 *           strictly lower triangle is read (unit diagonal implied), so the
 *           L panel of pselinv_get_panels(which = 1) of a single-supernode
 *           matrix can be passed as is
 * d_d       device, count x s pivots
 * d_M       device, count x s x s output, full symmetric, column-major
 * The first call on each device looks up the scratch array's device address
 * and sets a kernel attribute for that device; make that first call before
 * any stream capture.  All calls share the one scratch array: calls that can
 * overlap on the GPU (different streams, or different host threads) race on
 * it and must be serialised by the caller.  Every call writes all scratch
 * it reads, so nothing needs clearing between calls.  Enqueues work on
 * stream; no synchronisation.  Errors: ERR_ARG (sizes, NULL), ERR_CUDA;
 * message via pselinv_last_error(NULL).
 */
int pselinv_block_inverse_static(int32_t s, int32_t count, const double* d_L, const double* d_d, double* d_M,
                                 void* stream);

/* Frees everything the handle owns; NULL is allowed. */
void pselinv_destroy(pselinv_handle* h);

/* Message for the last error on h (or on the last failed analyze if h is
   NULL); never NULL. */
const char* pselinv_last_error(const pselinv_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* PSELINV_H */
