// Device kernels of the supernodal LDL^T and the selected inversion.
//
// Storage (per batch member, offsets in SnMeta): L and X panels are
// (s + r) x s column-major blocks with ld = s + r whose rows are the
// supernode's own columns followed by R(K) = C; Lhat_{C,K} is r x s with
// ld = r; (L_KK)^{-1} is s x s with ld = s; D holds the pivots.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"
#include "tile_gemm.cuh"

namespace psi {

// --------------------------------------------------------------------------
// small helpers
// --------------------------------------------------------------------------

// packed lower-triangular index, column-major: (i, j), i >= j, order s
__device__ __forceinline__ int pk(int i, int j, int s) { return j * s - (j * (j - 1)) / 2 + (i - j); }

__device__ __forceinline__ bool bad_pivot(double d) { return !(isfinite(d)) || d == 0.0; }

__device__ void report_pivot(int* status, int col, double d) {
  atomicMin(&status[0], col);
  atomicMax(&status[1], d == 0.0 ? 1 : 2);
}

// --------------------------------------------------------------------------
// value scatter / selected-entry gather (HBM-bound, index driven)
// --------------------------------------------------------------------------

__global__ void k_scatter_values(const double* __restrict__ vals, const int64_t* __restrict__ vmap,
                                 int64_t nnz, double* __restrict__ L, int64_t panel_total) {
  const int b = blockIdx.y;
  const double* v = vals + (int64_t)b * nnz;
  double* Lb = L + (int64_t)b * panel_total;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
    Lb[vmap[q]] = v[q];
}

__global__ void k_gather_values(const double* __restrict__ X, int64_t panel_total, const int64_t* __restrict__ vmap,
                                int64_t nnz, double* __restrict__ out) {
  const int b = blockIdx.y;
  const double* Xb = X + (int64_t)b * panel_total;
  double* o = out + (int64_t)b * nnz;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
    o[q] = Xb[vmap[q]];
}

// --------------------------------------------------------------------------
// factorisation: dense LDL^T of the diagonal block and its inverse
// --------------------------------------------------------------------------

// One CTA per supernode of the level.  The s x s diagonal block (lower part,
// already holding A_KK minus all descendant updates) is factored in shared
// memory by right-looking LDL^T; L_KK (unit diagonal implied, d_j written on
// the diagonal slot) goes back to the panel, d to D, and (L_KK)^{-1} to linv.
__global__ void k_factor_diag(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns, double* __restrict__ L,
                              double* __restrict__ D, double* __restrict__ Linv, Sizes sz, int* status) {
  extern __shared__ double sh[];
  const int k = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, ld = m.s + m.r;
  double* P = L + b * sz.panel + m.panel;
  double* T = sh;                         // packed L_KK, s(s+1)/2
  double* V = sh + s * (s + 1) / 2;       // packed inverse
  const int nt = blockDim.x, t = threadIdx.x;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i >= j) T[pk(i, j, s)] = P[i + (int64_t)j * ld];
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    const double d = T[pk(j, j, s)];
    if (t == 0 && bad_pivot(d)) report_pivot(status, m.f + j, d);
    for (int i = j + 1 + t; i < s; i += nt) T[pk(i, j, s)] /= d;
    __syncthreads();
    const int w = s - j - 1;
    for (int e = t; e < w * w; e += nt) {
      const int ii = j + 1 + e % w, kk = j + 1 + e / w;
      if (ii >= kk) T[pk(ii, kk, s)] -= T[pk(ii, j, s)] * T[pk(kk, j, s)] * d;
    }
    __syncthreads();
  }
  // inverse of the unit lower triangle, one column per thread
  for (int c = t; c < s; c += nt) {
    V[pk(c, c, s)] = 1.0;
    for (int i = c + 1; i < s; ++i) {
      double acc = 0.0;
      for (int q = c; q < i; ++q) acc += T[pk(i, q, s)] * V[pk(q, c, s)];
      V[pk(i, c, s)] = -acc;
    }
  }
  __syncthreads();
  double* Vi = Linv + b * sz.linv + m.linv;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i >= j) {
      P[i + (int64_t)j * ld] = T[pk(i, j, s)];
      Vi[i + j * s] = V[pk(i, j, s)];
    } else {
      Vi[i + j * s] = 0.0;
    }
  }
  for (int j = t; j < s; j += nt) D[b * sz.n + m.f + j] = T[pk(j, j, s)];
}

// Off-diagonal panel solve: Ltmp_{C,K} = A_{C,K} (L_KK)^{-T} D_K^{-1}
// (tiles of r x s), written to the scratch buffer, then copied back.
__global__ void __launch_bounds__(TG_THREADS) k_trsm(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                     const double* __restrict__ L, const double* __restrict__ D,
                                                     const double* __restrict__ Linv, double* __restrict__ Ltmp,
                                                     Sizes sz) {
  __shared__ TileSmem sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const double* A = L + b * sz.panel + m.panel + s;          // rows below the diagonal block
  const double* Vi = Linv + b * sz.linv + m.linv;
  const double* d = D + b * sz.n + m.f;
  double acc[4][4][2] = {};
  auto la = [&](int mm, int kk) { const int row = tk.m0 + mm; return row < r ? A[row + (int64_t)kk * ld] : 0.0; };
  auto lb = [&](int kk, int nn) { const int col = tk.n0 + nn; return col < s ? Vi[col + kk * s] : 0.0; };
  tile_mma(sm, 0, s, [](int) { return false; }, la, lb, acc);
  double* out = Ltmp + b * sz.lhat + m.lhat;
  tile_epilogue(acc, [&](int mm, int nn, double v) {
    const int row = tk.m0 + mm, col = tk.n0 + nn;
    if (row < r && col < s) out[row + (int64_t)col * r] = v / d[col];
  });
}

// Copy Ltmp back into the panels of the level's supernodes.
__global__ void k_copyback(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns, double* __restrict__ L,
                           const double* __restrict__ Ltmp, Sizes sz) {
  const int k = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, r = m.r, ld = s + r;
  double* P = L + b * sz.panel + m.panel + s;
  const double* src = Ltmp + b * sz.lhat + m.lhat;
  const int64_t tot = (int64_t)r * s;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int64_t i = e % r, j = e / r;
    P[i + j * ld] = src[e];
  }
}

// Schur-complement update of the ancestors: for the lower tiles of
// U = L_{C,K} D_K L_{C,K}^T, subtract U[i][k] (i >= k) from the ancestor
// entry located through the column descriptor of k and the relative index
// of i.  Several supernodes of one level can hit the same entry: FP64
// atomics.
__global__ void __launch_bounds__(TG_THREADS) k_schur(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                      const ColDesc* __restrict__ desc,
                                                      const int32_t* __restrict__ relidx, double* __restrict__ L,
                                                      const double* __restrict__ D, const double* __restrict__ Ltmp,
                                                      Sizes sz) {
  __shared__ TileSmem sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r;
  const double* Lc = Ltmp + b * sz.lhat + m.lhat;
  const double* d = D + b * sz.n + m.f;
  double acc[4][4][2] = {};
  auto la = [&](int mm, int kk) { const int row = tk.m0 + mm; return row < r ? Lc[row + (int64_t)kk * r] * d[kk] : 0.0; };
  auto lb = [&](int kk, int nn) { const int col = tk.n0 + nn; return col < r ? Lc[col + (int64_t)kk * r] : 0.0; };
  tile_mma(sm, 0, s, [](int) { return false; }, la, lb, acc);
  double* Lb = L + b * sz.panel;
  const ColDesc* dk = desc + m.desc;
  tile_epilogue(acc, [&](int mm, int nn, double v) {
    const int i = tk.m0 + mm, kc = tk.n0 + nn;
    if (i < r && kc <= i) {
      const ColDesc cd = dk[kc];
      atomicAdd(&Lb[cd.col + relidx[cd.rel + i]], -v);
    }
  });
}

// --------------------------------------------------------------------------
// selected inversion
// --------------------------------------------------------------------------

// Normalisation, diagonal part (all supernodes, one CTA each):
// (L_KK)^{-1} -> linv and M_K = L_KK^{-T} D_K^{-1} L_KK^{-1} -> the diagonal
// block of the X panel (Algorithm 1 step 3's first term; U_KK = D_K L_KK^T).
__global__ void k_norm_diag(const SnMeta* __restrict__ meta, const double* __restrict__ L, const double* __restrict__ D,
                            double* __restrict__ Linv, double* __restrict__ X, Sizes sz) {
  extern __shared__ double sh[];
  const int k = blockIdx.x;
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, ld = m.s + m.r;
  const double* P = L + b * sz.panel + m.panel;
  const double* d = D + b * sz.n + m.f;
  double* T = sh;
  double* V = sh + s * (s + 1) / 2;
  const int nt = blockDim.x, t = threadIdx.x;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i > j) T[pk(i, j, s)] = P[i + (int64_t)j * ld];
  }
  __syncthreads();
  for (int c = t; c < s; c += nt) {
    V[pk(c, c, s)] = 1.0;
    for (int i = c + 1; i < s; ++i) {
      double acc = 0.0;
      for (int q = c; q < i; ++q) acc += T[pk(i, q, s)] * V[pk(q, c, s)];
      V[pk(i, c, s)] = -acc;
    }
  }
  __syncthreads();
  double* Vi = Linv + b * sz.linv + m.linv;
  double* XK = X + b * sz.panel + m.panel;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    Vi[i + j * s] = i >= j ? V[pk(i, j, s)] : 0.0;
    if (i >= j) {
      double acc = 0.0;
      for (int q = i; q < s; ++q) acc += V[pk(q, i, s)] * V[pk(q, j, s)] / d[q];
      XK[i + (int64_t)j * ld] = acc;
      XK[j + (int64_t)i * ld] = acc;
    }
  }
}

// Normalisation, off-diagonal part: Lhat_{C,K} = L_{C,K} (L_KK)^{-1}.
__global__ void __launch_bounds__(TG_THREADS) k_lhat(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                     const double* __restrict__ L, const double* __restrict__ Linv,
                                                     double* __restrict__ Lhat, Sizes sz) {
  __shared__ TileSmem sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const double* A = L + b * sz.panel + m.panel + s;
  const double* Vi = Linv + b * sz.linv + m.linv;
  double acc[4][4][2] = {};
  auto la = [&](int mm, int kk) { const int row = tk.m0 + mm; return row < r ? A[row + (int64_t)kk * ld] : 0.0; };
  auto lb = [&](int kk, int nn) { const int col = tk.n0 + nn; return col < s ? Vi[kk + col * s] : 0.0; };
  tile_mma(sm, 0, s, [](int) { return false; }, la, lb, acc);
  double* out = Lhat + b * sz.lhat + m.lhat;
  tile_epilogue(acc, [&](int mm, int nn, double v) {
    const int row = tk.m0 + mm, col = tk.n0 + nn;
    if (row < r && col < s) out[row + (int64_t)col * r] = v;
  });
}

// Step 2: X_{C,K} = -X_{C,C} Lhat_{C,K}.  X_{C,C} is read straight from the
// ancestors' X panels: entry (i, k) with i >= k (rows of C are sorted) sits
// in column desc[k].col at row relidx[desc[k].rel + i]; entries above the
// diagonal use the symmetric one.  The result is written into rows s.. of
// K's own X panel (Algorithm 3 overwrites Lhat by X_{C,K}; here Lhat stays
// in its own buffer).
__global__ void __launch_bounds__(TG_THREADS) k_gemm1(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                      const ColDesc* __restrict__ desc,
                                                      const int32_t* __restrict__ relidx, const double* __restrict__ Lhat,
                                                      double* __restrict__ X, Sizes sz) {
  __shared__ TileSmem sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const ColDesc* dk = desc + m.desc;
  const double* Xb = X + b * sz.panel;
  const double* Lh = Lhat + b * sz.lhat + m.lhat;
  double acc[4][4][2] = {};
  auto la = [&](int mm, int kk) {
    const int i = tk.m0 + mm;
    if (i >= r) return 0.0;
    const int lo = i < kk ? i : kk, hi = i < kk ? kk : i;
    const ColDesc cd = dk[lo];
    return Xb[cd.col + relidx[cd.rel + hi]];
  };
  auto lb = [&](int kk, int nn) { const int col = tk.n0 + nn; return col < s ? Lh[kk + (int64_t)col * r] : 0.0; };
  // where a k-tile lies wholly above the tile's rows the entries come from
  // the columns of C in the m direction: run the threads along k there so
  // the panel reads stay contiguous
  const int m0 = tk.m0;
  tile_mma(sm, 0, r, [m0](int kt) { return kt >= m0 + TG_BM; }, la, lb, acc);
  double* out = X + b * sz.panel + m.panel + s;
  tile_epilogue(acc, [&](int mm, int nn, double v) {
    const int row = tk.m0 + mm, col = tk.n0 + nn;
    if (row < r && col < s) out[row + (int64_t)col * ld] = -v;
  });
}

// Step 3, partial products: P_c = Lhat_{rows c, K}^T X_{rows c, K} over a
// chunk of kChunkRows rows of C (s x s tiles).
__global__ void __launch_bounds__(TG_THREADS) k_gemm2(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                      const double* __restrict__ Lhat, const double* __restrict__ X,
                                                      double* __restrict__ part, Sizes sz) {
  __shared__ TileSmem sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const double* Lh = Lhat + b * sz.lhat + m.lhat;
  const double* Y = X + b * sz.panel + m.panel + s;
  double acc[4][4][2] = {};
  auto la = [&](int mm, int kk) { const int i = tk.m0 + mm; return i < s ? Lh[kk + (int64_t)i * r] : 0.0; };
  auto lb = [&](int kk, int nn) { const int col = tk.n0 + nn; return col < s ? Y[kk + (int64_t)col * ld] : 0.0; };
  const int kb = tk.c * kChunkRows, ke = min(r, kb + kChunkRows);
  tile_mma(sm, kb, ke, [](int) { return true; }, la, lb, acc);
  double* out = part + b * sz.part + m.part + (int64_t)tk.c * s * s;
  tile_epilogue(acc, [&](int mm, int nn, double v) {
    const int row = tk.m0 + mm, col = tk.n0 + nn;
    if (row < s && col < s) out[row + col * s] = v;
  });
}

// Step 3, finish: X_KK = (Z + Z^T) / 2 with Z = M_K - sum_c P_c (the
// symmetrisation at the end of Section 2.1 / Algorithm 3).  One thread per
// unordered pair {i, j} reads and writes exactly (i, j) and (j, i).
__global__ void k_diag_final(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns,
                             const double* __restrict__ part, double* __restrict__ X, Sizes sz) {
  const int k = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, ld = m.s + m.r;
  double* XK = X + b * sz.panel + m.panel;
  const double* pp = part + b * sz.part + m.part;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    if (i < j) continue;
    double zij = XK[i + (int64_t)j * ld], zji = XK[j + (int64_t)i * ld];
    for (int c = 0; c < m.nchunk; ++c) {
      zij -= pp[(int64_t)c * s * s + i + j * s];
      zji -= pp[(int64_t)c * s * s + j + i * s];
    }
    const double x = 0.5 * (zij + zji);
    XK[i + (int64_t)j * ld] = x;
    XK[j + (int64_t)i * ld] = x;
  }
}

// log det = sum_j log|d_j| and the count of negative pivots, per batch member.
__global__ void k_logdet(const double* __restrict__ D, int64_t n, double* __restrict__ out) {
  __shared__ double s1[256];
  __shared__ double s2[256];
  const int b = blockIdx.x;
  double a = 0.0, neg = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = D[b * n + j];
    a += log(fabs(d));
    neg += d < 0.0 ? 1.0 : 0.0;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = neg;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * b] = s1[0];
    out[2 * b + 1] = s2[0];
  }
}

// --------------------------------------------------------------------------
// launch wrappers
// --------------------------------------------------------------------------

static inline unsigned blocks_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

cudaError_t launch_scatter_values(const double* vals, const int64_t* vmap, int64_t nnz, double* L, const Sizes& sz,
                                  cudaStream_t st) {
  k_scatter_values<<<dim3(blocks_for(nnz, 256), sz.batch), 256, 0, st>>>(vals, vmap, nnz, L, sz.panel);
  return cudaGetLastError();
}
cudaError_t launch_gather_values(const double* X, const int64_t* vmap, int64_t nnz, double* out, const Sizes& sz,
                                 cudaStream_t st) {
  k_gather_values<<<dim3(blocks_for(nnz, 256), sz.batch), 256, 0, st>>>(X, sz.panel, vmap, nnz, out);
  return cudaGetLastError();
}

static size_t diag_smem(int maxw) { return sizeof(double) * (size_t)maxw * (maxw + 1); }

cudaError_t setup_kernels() {
  const size_t sm = diag_smem(kMaxWidth);
  cudaError_t e = cudaFuncSetAttribute(k_factor_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_norm_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

cudaError_t launch_factor_level(const SnMeta* meta, const int32_t* sns, int nsn_level, const Task* trsm,
                                int64_t ntrsm, const Task* schur, int64_t nschur, const ColDesc* desc,
                                const int32_t* relidx, double* L, double* D, double* Linv, double* Ltmp,
                                int maxw, const Sizes& sz, int* status, cudaStream_t st) {
  if (nsn_level <= 0) return cudaSuccess;
  k_factor_diag<<<dim3(nsn_level, sz.batch), 256, diag_smem(maxw), st>>>(meta, sns, L, D, Linv, sz, status);
  if (ntrsm > 0) {
    k_trsm<<<dim3((unsigned)ntrsm, sz.batch), TG_THREADS, 0, st>>>(meta, trsm, L, D, Linv, Ltmp, sz);
    k_copyback<<<dim3(nsn_level, sz.batch), 256, 0, st>>>(meta, sns, L, Ltmp, sz);
  }
  if (nschur > 0)
    k_schur<<<dim3((unsigned)nschur, sz.batch), TG_THREADS, 0, st>>>(meta, schur, desc, relidx, L, D, Ltmp, sz);
  return cudaGetLastError();
}

cudaError_t launch_normalise(const SnMeta* meta, int nsn, const Task* lhat_tasks, int64_t nlhat, const double* L,
                             const double* D, double* Linv, double* Lhat, double* X, int maxw, const Sizes& sz,
                             cudaStream_t st) {
  k_norm_diag<<<dim3(nsn, sz.batch), 256, diag_smem(maxw), st>>>(meta, L, D, Linv, X, sz);
  if (nlhat > 0) k_lhat<<<dim3((unsigned)nlhat, sz.batch), TG_THREADS, 0, st>>>(meta, lhat_tasks, L, Linv, Lhat, sz);
  return cudaGetLastError();
}

cudaError_t launch_gemm1(const SnMeta* meta, const Task* g1, int64_t ng1, const ColDesc* desc, const int32_t* relidx,
                         const double* Lhat, double* X, const Sizes& sz, cudaStream_t st) {
  if (ng1 > 0) k_gemm1<<<dim3((unsigned)ng1, sz.batch), TG_THREADS, 0, st>>>(meta, g1, desc, relidx, Lhat, X, sz);
  return cudaGetLastError();
}

cudaError_t launch_gemm2(const SnMeta* meta, const Task* g2, int64_t ng2, const double* Lhat, const double* X,
                         double* part, const Sizes& sz, cudaStream_t st) {
  if (ng2 > 0) k_gemm2<<<dim3((unsigned)ng2, sz.batch), TG_THREADS, 0, st>>>(meta, g2, Lhat, X, part, sz);
  return cudaGetLastError();
}

cudaError_t launch_diag_final(const SnMeta* meta, const int32_t* sns, int nsn_step, const double* part, double* X,
                              const Sizes& sz, cudaStream_t st) {
  if (nsn_step > 0) k_diag_final<<<dim3(nsn_step, sz.batch), 256, 0, st>>>(meta, sns, part, X, sz);
  return cudaGetLastError();
}

cudaError_t launch_logdet(const double* D, int64_t n, double* out, int batch, cudaStream_t st) {
  k_logdet<<<batch, 256, 0, st>>>(D, n, out);
  return cudaGetLastError();
}

}  // namespace psi
