// Launch wrappers of the device kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace psi {

// Per-batch-member sizes (elements of the scalar) of every batched array.
struct Sizes {
  int64_t panel;  // L and X panels
  int64_t lhat;   // normalised factor / factor scratch
  int64_t linv;   // diagonal-block inverses
  int64_t n;      // pivots
  int64_t part;   // step-3 partial products
  int64_t ypart;  // step-2 partial products
  int batch;
};

enum class Kern {
  Trsm, Schur, Lhat, Gemm1, Gemm2, FactorDiag, CopyBack, NormDiag, DiagFinal, Gemm1Reduce,
  FactorDiagLU, NormDiagLU,  // non-symmetric diagonal blocks
  FactorDiagBK, CopyBackBK   // Bunch-Kaufman pivoted factor
};

// Everything a kernel may need; device pointers typed by dtype inside.
struct KArgs {
  int dtype;  // PSELINV_F64 / PSELINV_C128
  int maxw;   // widest supernode (shared-memory size of the diagonal kernels)
  const SnMeta* meta;
  const ColDesc* desc;
  const int32_t* relidx;
  void* L;
  void* D;
  void* Linv;
  void* Lhat;
  void* X;
  void* part;
  void* ypart;
  int* status;
  // split step 2: per-output-tile counters (batch x tctr_total, zero between
  // launches); set: the last slice CTA of a tile sums the slices in slice
  // order and writes X_{C,K} (no separate reduction); nullptr: partials only
  int* tctr;
  int64_t tctr_n;  // counters per batch member
  Sizes sz;
  // non-symmetric handles (nullptr / 0 for symmetric ones)
  void* U;     // U panels: U'_{j,i} at panel position (i, j)
  void* Uinv;  // (U'_KK^T)^{-1}, linv layout
  void* Uhat;  // Uhat_{K,C}^T, lhat layout; Schur: second operand (nullptr = Lhat)
  void* XU;    // XU panels: X_{j,i} at panel position (i, j); step 2 reads X_{C,C} above the
               // diagonal from here, step 3 finish writes X_KK^T here
  int strict;  // Schur: skip the diagonal entries of the updated blocks
  // Bunch-Kaufman pivoted factor (nullptr when not pivoted), batch x n each:
  const int32_t* piv;  // supernode-local original column at each pivot position
  const int8_t* ptype; // 0 = 1x1 pivot, 1 / 2 = first / second column of a 2x2 pivot
  const void* E;       // D_{k+1,k} of a 2x2 pivot, at its first column
  // pole sum accumulated in the step-3 finish (pselinv_selinv_pole_sum):
  // weights w_b (batch), Gamma = sum_b w_b X_b (one panel array), counters
  // (nsn x kFinishCtas, zero between launches); nullptr otherwise
  const void* gw;
  void* gam;
  int* gctr;
  // factor: W_{C,K} = L_{C,K} D_K (U side: U'_{K,C}^T D_K; pivoted: D_K's
  // 1 x 1 and 2 x 2 blocks, columns in pivot order), the panel solve's
  // product before the D^{-1} scaling, kept for the Schur update; r x s
  // column-major at each supernode's panel offset of this array (the X or XU
  // panels, free during the factorisation); nullptr elsewhere
  void* W;
};

// CTAs of the per-level step-3 finish per supernode (blockIdx.z of k_diag_final).
constexpr int kFinishCtas = 32;

// Original local column of pivot position k of the supernode starting at f.
__device__ __forceinline__ int pcol(const KArgs& a, int b, int f, int k) {
  return a.piv ? a.piv[(int64_t)b * a.sz.n + f + k] : k;
}

cudaError_t setup_kernels();
cudaError_t launch_scatter_values(int dtype, const void* vals, const int64_t* vmap, int64_t nnz, void* L,
                                  const Sizes& sz, cudaStream_t st);
// Non-symmetric values: lower (A_ij) to the L panels, upper (A_ji) to the U
// panels, swapped where flip[q] (the ordering transposed entry q).
cudaError_t launch_scatter_values_lu(int dtype, const void* lower, const void* upper, const int64_t* vmap,
                                     const uint8_t* flip, int64_t nnz, void* L, void* U, const Sizes& sz,
                                     cudaStream_t st);
// Non-symmetric gather: X_ij (upper = 0) or X_ji (upper = 1) at stored entry q.
cudaError_t launch_gather_values_lu(int dtype, const void* XL, const void* XU, const int64_t* vmap,
                                    const uint8_t* flip, int64_t nnz, int upper, void* out, const Sizes& sz,
                                    cudaStream_t st);
// diagmask == nullptr: plain gather; else off-diagonal entries doubled.
cudaError_t launch_gather_values(int dtype, const void* X, const int64_t* vmap, const uint8_t* diagmask, int64_t nnz,
                                 void* out, const Sizes& sz, cudaStream_t st);
// Tile kernels (Trsm, Schur, Lhat, Gemm1, Gemm2) over n tasks of one tile
// width variant (BN = 8 << var).
cudaError_t launch_tiles(Kern k, int var, const KArgs& a, const Task* tasks, int64_t n, cudaStream_t st);
// Per-supernode kernels (FactorDiag, CopyBack, NormDiag, DiagFinal, Gemm1Reduce) over the
// nsn supernodes listed in sns (NormDiag: supernodes 0..nsn-1, sns unused).
// threads: block size of the diagonal-factorisation kernels (FactorDiag,
// FactorDiagLU, FactorDiagBK -- the last capped at 512); the others use 256.
cudaError_t launch_per_sn(Kern k, const KArgs& a, const int32_t* sns, int nsn, cudaStream_t st, int threads = 256);
cudaError_t launch_logdet(int dtype, const void* D, int64_t n, double* out, int batch, cudaStream_t st,
                          const int8_t* ptype = nullptr, const void* E = nullptr);
cudaError_t launch_pole_sum(int dtype, const void* X, int64_t panel_total, int batch, const void* w, void* out,
                            cudaStream_t st);
cudaError_t launch_trace_sum(int dtype, const void* X, int64_t panel_total, const int64_t* vmap,
                             const uint8_t* diagmask, const void* vals, int64_t nnz, int batch, void* out,
                             cudaStream_t st);

// ---- step 2 with FP64 arithmetic emulated on the bf16 tensor cores (emulate.cu) ----
// Real symmetric positive definite X only: |X_pq| <= sqrt(X_pp X_qq), so with
// e_p = ceil(log2 sqrt(X_pp)) every entry of Xt = 2^-(e_p + e_q) X has |Xt| < 1.
// Each entry of Xt (and of B' = diag(2^e_C) Lhat over a per-column exponent)
// is cut once into 7 signed 8-bit slices held as bf16; step 2 forms the 28
// slice products of weight >= 2^-48 with exact FP32 sums over 32-row chunks
// folded into 64-bit integers.
struct EmArgs {
  void* xs;              // [batch][panel_total] uint4: 7 bf16 slices of Xt per X panel entry
  void* ls;              // [batch][lhat_total] uint4: 7 bf16 slices of B' per Lhat entry
  int32_t* sig;          // [batch][n] e_p of every column (written when its level finishes)
  int32_t* lexp;         // [batch][n] column exponent F of B' (|B'_{:,j}| < 2^F), per global column
  int32_t* gexp;         // [batch][n] column exponent G of X'' = diag(2^-e_C) X_{C,K} (step 3)
  const int32_t* crow;   // [sum r] global row of C[i] of supernode K at desc offset of K
  int64_t n;
};
// Emulation status word: kEmRange after an X diagonal <= 0 / not finite or a
// scaled entry outside its slice range (X not positive definite).
constexpr int kEmStatusWord = 4;
constexpr int kEmRange = 1;
// After steps 2-3 of a level: e_p of the level's columns and the slices of
// its X panels.  Before step 2 of a level: F and the slices of its B'.
cudaError_t launch_em_split_x(const KArgs& a, const EmArgs& e, const int32_t* sns, int nsn, cudaStream_t st);
// max_r: the largest |C| among the supernodes (sizes the shared memory).
cudaError_t launch_em_split_lhat(const KArgs& a, const EmArgs& e, const int32_t* sns, int nsn, int max_r,
                                 cudaStream_t st);
// After step 2 of a level (step 3 emulated): G and the slices of X'' for its
// supernodes, written over the slice array at the rows of C of their panels.
cudaError_t launch_em_split_xck(const KArgs& a, const EmArgs& e, const int32_t* sns, int nsn, int max_r,
                                cudaStream_t st);
// Step-3 partial products (the Gemm2 task list of tile variant var) on the slices.
cudaError_t launch_em_gemm2(int var, const KArgs& a, const EmArgs& e, const Task* tasks, int64_t n, cudaStream_t st);
// Dynamic shared-memory limits of the step-2 kernels (called by setup_kernels).
cudaError_t setup_em_kernels();
// Step-2 tiles (the Gemm1 task list of tile variant var) on the slices:
// 64 x 8 / 64 x 16 tiles on mma.sync (var 0, 1).
cudaError_t launch_em_gemm1(int var, const KArgs& a, const EmArgs& e, const Task* tasks, int64_t n,
                            cudaStream_t st);

// ---- persistent per-level schedule (persistent.cu) ----
struct PArgs {
  const Task* g1;       // step-2 task array (t_gemm1)
  const Task* g2;       // step-3 task array (t_gemm2)
  int* c1;              // [batch][nsn] finished step-2 tiles
  int* c2;              // [batch][nsn] finished step-3 tiles
  int* cr;              // [batch][nsn] finished slice reductions
  int* cf;              // [batch][nsn] finished step-3 finish parts (X of the supernode final at kFinishParts)
  int* lvl;             // [nlevels] finished finish parts of a level, all batch members
  const int32_t* n1;    // [nsn] step-2 tiles per supernode
  const int32_t* n2;    // [nsn] step-3 tiles per supernode
  const int32_t* snlevel;   // [nsn] level (0 = roots)
  const int32_t* snparent;  // [nsn] supernodal parent, -1 = root
  const int32_t* level_ptr; // [nlevels + 1] supernodes per level (prefix sums)
  int* head;            // dequeue counter
  int nsn;
  int64_t yslot, pslot; // elements of one level slot of the step-2 / step-3 partial buffers
  long long spin_ns;    // bound of every wait
};
// Slots of the partial-product ring: a level starts its step 2 only once the
// level kRing above it has finished, so at most kRing levels hold partials.
constexpr int kRing = 4;
cudaError_t launch_persistent(const KArgs& a, const PArgs& p, const PTask* list, int64_t ntask, int grid,
                              cudaStream_t st);
cudaError_t persistent_grid(int dtype, int* grid);

// ---- adjoint (adjoint.cu) ----
struct AdjArgs {
  KArgs k;
  const void* G;  // seed, X panel layout
  int g_kind;     // PSELINV_G_SYMMETRIC / PSELINV_G_PANEL
  void* Xb;       // adjoint of X panels; later adjoint of the updated factor panels
  void* Lb;       // adjoint of L (panel layout)
  void* Db;       // adjoint of D
  void* Zb;       // s x s per supernode (linv layout): Zbar, then Vbar, then P
  void* W1;       // s x s per supernode scratch
  void* Yb;       // r x s per supernode (lhat layout): Ybar, then T1
  void* Hb;       // r x s per supernode: Lhat-bar
};
enum class AdjKern { Ybar, Lhbar, LbarOff, T1, Q, Vpart, Rpart, Syr2k, Dr1, Dr3, Dr4, Df2, Df3, Df4 };
enum class AdjSn { Seed, Ev, Zbar, Dr2, Df1, Df5, SumParts };
cudaError_t launch_adj_tiles(AdjKern k, int var, const AdjArgs& a, const Task* tasks, int64_t n, cudaStream_t st);
cudaError_t launch_adj_per_sn(AdjSn k, const AdjArgs& a, const int32_t* sns, int nsn, cudaStream_t st);

}  // namespace psi
