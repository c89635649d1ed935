// Steps 2 and 3 of the selected inversion as device functions, shared by
// the grouped per-level kernels (kernels.cu) and the persistent per-level
// kernel (persistent.cu).
#pragma once

#include "kernels.h"
#include "tile_gemm.cuh"

namespace psi {

// Loads of data another CTA wrote earlier in the same launch (persistent
// schedule) bypass L1, which is not coherent across SMs.
template <class T>
__device__ __forceinline__ T ld_cg(const T* p);
template <>
__device__ __forceinline__ double ld_cg<double>(const double* p) {
  return __ldcg(p);
}
template <>
__device__ __forceinline__ Cplx ld_cg<Cplx>(const Cplx* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
template <class T>
__device__ __forceinline__ T ld_maybe_cg(const T* p, bool cg) {
  return cg ? ld_cg(p) : *p;
}

// Split tiles (m.ksplit slices of C): every slice CTA has stored its
// partial tile; this counts the CTA on the tile's counter and returns true
// in the one CTA that brings the count to ksplit (it then sums the slices
// and resets the counter).  No CTA waits for another.
template <int BN>
__device__ __forceinline__ bool last_slice(const KArgs& a, const SnMeta& m, const Task& tk, int b) {
  __shared__ int last;
  __threadfence();  // this CTA's partial before the count
  __syncthreads();
  if (threadIdx.x == 0) {
    int* ctr = a.tctr + (int64_t)b * a.tctr_n + m.tctr + (tk.m0 / TG_BM) * ((m.s + BN - 1) / BN) + tk.n0 / BN;
    last = atomicAdd(ctr, 1) == m.ksplit - 1;
    if (last) *ctr = 0;
    __threadfence();
  }
  __syncthreads();
  return last != 0;
}

// Step 2 tile: X_{C,K} = -X_{C,C} Lhat_{C,K} over rows [m0, m0+64), columns
// [n0, n0+BN) and the k-slice tk.c of C.  X_{C,C} is read straight from the
// ancestors' X panels: entry (i, k) with i >= k (rows of C are sorted) sits
// in column desc[k].col at row relidx[desc[k].rel + i]; entries above the
// diagonal use the symmetric one.  Unsplit supernodes write rows s.. of K's
// own X panel (Algorithm 3 overwrites Lhat by X_{C,K}; here Lhat stays in its
// own buffer); split ones write their slice's partial product.
//
// UNSYM (non-symmetric A): entry (i, k) with i < k is X_{C[i],C[k]}, read
// from the XU panels at the same position.  Step 4 of Algorithm 1 in
// transposed form, X_{K,C}^T = -X_{C,C}^T Uhat_{K,C}^T, is this same tile
// with X and XU swapped and Uhat^T in place of Lhat: it then writes the XU
// panel rows.
// yoff / poff (persistent schedule): element offset of the level's slot in
// the step-2 / step-3 partial-product buffers (0 for the per-level launches).
template <class T, int BN, bool UNSYM = false>
__device__ __forceinline__ void step2_tile(const KArgs& a, const Task& tk, int b, TileSmem<T, BN>& sm,
                                           int64_t yoff = 0) {
  const Sizes& sz = a.sz;
  const SnMeta m = a.meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const ColDesc* dk = a.desc + m.desc;
  const int32_t* relidx = a.relidx;
  const T* Xb = (const T*)a.X + b * sz.panel;
  const T* XUb = UNSYM ? (const T*)a.XU + b * sz.panel : Xb;
  const T* Lh = (const T*)a.Lhat + b * sz.lhat + m.lhat;
  Acc<T, BN> acc;
  acc_zero<T, BN>(acc);
  auto la = [&](int mm, int kk) {
    const int i = tk.m0 + mm;
    if (i >= r) return Sc<T>::zero();
    const int lo = i < kk ? i : kk, hi = i < kk ? kk : i;
    const ColDesc cd = dk[lo];
    if constexpr (UNSYM) return (i < kk ? XUb : Xb)[cd.col + relidx[cd.rel + hi]];
    return Xb[cd.col + relidx[cd.rel + hi]];
  };
  auto lb = [&](int kk, int nn) {
    const int col = tk.n0 + nn;
    return col < s ? Lh[kk + (int64_t)col * r] : Sc<T>::zero();
  };
  // where a k-tile lies wholly right of the tile's rows the entries come from
  // the columns of C in the m direction: threads run along k there so the
  // panel reads stay contiguous
  const int m0 = tk.m0;
  const int kb = tk.c * m.kchunk, ke = min(r, kb + m.kchunk);
  tile_mma<T, BN>(sm, kb, ke, [m0](int kt) { return kt >= m0 + TG_BM; }, la, lb, acc,
                  LiveRect{r - tk.m0, s - tk.n0});
  if (m.ksplit == 1) {
    // a pivoted factor computes K's columns in pivot order; X keeps the original order
    T* out = (T*)a.X + b * sz.panel + m.panel + s;
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int row = tk.m0 + mm, col = tk.n0 + nn;
      if (row < r && col < s) out[row + (int64_t)pcol(a, b, m.f, col) * ld] = -v;
    });
  } else {
    T* yp = (T*)a.ypart + b * sz.ypart + yoff + m.ypart;
    T* out = yp + (int64_t)tk.c * r * s;
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int row = tk.m0 + mm, col = tk.n0 + nn;
      if (row < r && col < s) out[row + (int64_t)col * r] = v;
    });
    if (!a.tctr) return;  // a separate kernel sums the slices
    // The CTA that finishes a tile's last slice sums all slices of the tile in
    // slice order, its own from registers, and writes X_{C,K}: the same
    // arithmetic as step2_reduce, without its launch and its pass over HBM.
    if (!last_slice<BN>(a, m, tk, b)) return;
    const int64_t rs = (int64_t)r * s;
    T* xo = (T*)a.X + b * sz.panel + m.panel + s;
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int row = tk.m0 + mm, col = tk.n0 + nn;
      if (row >= r || col >= s) return;
      const int64_t e = row + (int64_t)col * r;
      T sum = tk.c == 0 ? v : ld_cg(yp + e);
      for (int c = 1; c < m.ksplit; ++c) sum += c == tk.c ? v : ld_cg(yp + c * rs + e);
      xo[row + (int64_t)pcol(a, b, m.f, col) * ld] = -sum;
    });
  }
}

// Step 2 finish of a split supernode k: X_{C,K} = -(sum of the slice
// partial products, in slice order), columns col0, col0 + cstride, ...
template <class T>
__device__ __forceinline__ void step2_reduce(const KArgs& a, int k, int b, int col0, int cstride, bool cg,
                                             int64_t yoff = 0) {
  const Sizes& sz = a.sz;
  const SnMeta m = a.meta[k];
  if (m.ksplit == 1) return;
  const int s = m.s, r = m.r, ld = s + r;
  const T* yp = (const T*)a.ypart + b * sz.ypart + yoff + m.ypart;
  T* out = (T*)a.X + b * sz.panel + m.panel + s;
  const int64_t rs = (int64_t)r * s;
  for (int j = col0; j < s; j += cstride) {
    const T* col = yp + (int64_t)j * r;
    T* oc = out + (int64_t)pcol(a, b, m.f, j) * ld;
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      T acc = ld_maybe_cg(col + i, cg);
      for (int c = 1; c < m.ksplit; ++c) acc += ld_maybe_cg(col + c * rs + i, cg);
      oc[i] = -acc;
    }
  }
}

// Step 3 partial product tile: P_c = Lhat_{rows c, K}^T X_{rows c, K} over a
// chunk of kchunk3 rows of C (plain transpose; s x s output tiles).
template <class T, int BN>
__device__ __forceinline__ void step3_tile(const KArgs& a, const Task& tk, int b, TileSmem<T, BN>& sm, bool cg,
                                           int64_t poff = 0) {
  const Sizes& sz = a.sz;
  const SnMeta m = a.meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const T* Lh = (const T*)a.Lhat + b * sz.lhat + m.lhat;
  const T* Y = (const T*)a.X + b * sz.panel + m.panel + s;
  Acc<T, BN> acc;
  acc_zero<T, BN>(acc);
  auto la = [&](int mm, int kk) {
    const int i = tk.m0 + mm;
    return i < s ? Lh[kk + (int64_t)i * r] : Sc<T>::zero();
  };
  auto lb = [&](int kk, int nn) {
    const int col = tk.n0 + nn;
    return col < s ? ld_maybe_cg(Y + kk + (int64_t)pcol(a, b, m.f, col) * ld, cg) : Sc<T>::zero();
  };
  const int kb = tk.c * m.kchunk3, ke = min(r, kb + m.kchunk3);
  tile_mma<T, BN>(sm, kb, ke, [](int) { return true; }, la, lb, acc, LiveRect{s - tk.m0, s - tk.n0});
  T* out = (T*)a.part + b * sz.part + poff + m.part + (int64_t)tk.c * s * s;
  tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
    const int row = tk.m0 + mm, col = tk.n0 + nn;
    if (row < s && col < s) out[row + col * s] = v;
  });
}

// Step 3 finish: X_KK = (Z + Z^T) / 2 with Z = M_K - sum_c P_c (the
// symmetrisation at the end of Section 2.1 / Algorithm 3).  One thread per
// unordered pair {i, j} reads and writes exactly (i, j) and (j, i) -- for a
// pivoted factor at the original columns (P(i), P(j)), where the
// normalisation pass left M_K.
// Non-symmetric handles (a.XU set): X_KK = Z as it is, and Z^T goes to the
// diagonal block of the XU panel.
template <class T>
__device__ __forceinline__ void step3_finish(const KArgs& a, int k, int b, int part, int nparts, bool cg,
                                             int64_t poff = 0) {
  const Sizes& sz = a.sz;
  const SnMeta m = a.meta[k];
  const int s = m.s, ld = m.s + m.r;
  T* XK = (T*)a.X + b * sz.panel + m.panel;
  const T* pp = (const T*)a.part + b * sz.part + poff + m.part;
  if (a.XU) {
    T* XUK = (T*)a.XU + b * sz.panel + m.panel;
    for (int e = threadIdx.x + part * blockDim.x; e < s * s; e += nparts * blockDim.x) {
      const int i = e % s, j = e / s;
      T z = XK[i + (int64_t)j * ld];
      for (int c = 0; c < m.nchunk; ++c) z -= ld_maybe_cg(pp + (int64_t)c * s * s + i + j * s, cg);
      XK[i + (int64_t)j * ld] = z;
      XUK[j + (int64_t)i * ld] = z;
    }
    return;
  }
  // the CTAs part = 0..nparts-1 share the pairs of one supernode
  for (int e = threadIdx.x + part * blockDim.x; e < s * s; e += nparts * blockDim.x) {
    const int i = e % s, j = e / s;
    if (i < j) continue;
    const int pi = pcol(a, b, m.f, i), pj = pcol(a, b, m.f, j);
    T zij = XK[pi + (int64_t)pj * ld], zji = XK[pj + (int64_t)pi * ld];
    for (int c = 0; c < m.nchunk; ++c) {
      zij -= ld_maybe_cg(pp + (int64_t)c * s * s + i + j * s, cg);
      zji -= ld_maybe_cg(pp + (int64_t)c * s * s + j + i * s, cg);
    }
    const T x = 0.5 * (zij + zji);
    XK[pi + (int64_t)pj * ld] = x;
    XK[pj + (int64_t)pi * ld] = x;
  }
}

}  // namespace psi
