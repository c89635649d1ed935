// Adjoint of the selected inversion and of the supernodal LDL^T.
//
// J = <G, X> (bilinear, over the full symmetric selected pattern).  Panel
// variables per supernode K: the full diagonal block X_KK and X_CK = Y.  The
// forward recurrence (Algorithm 1 in the symmetric form of Eq. 14, with
// V = (L_KK)^{-1}, E = D_K^{-1}):
//   M = V^T E V,  Lhat = L_CK V,  Y = -X_CC Lhat,  Z = M - Lhat^T Y,
//   X_KK = (Z + Z^T) / 2,  X_CK = Y.
// Reverse sweep, supernodes leaves -> root (levels deepest first):
//   Zb   = (Xb_KK + Xb_KK^T) / 2                          (= Mbar)
//   Yb   = Xb_CK - Lhat Zb
//   Hb   = -X_CC Yb - Y Zb^T                              (Lhat-bar)
//   ancestors: Xb_CC += -(Yb Lhat^T + Lhat Yb^T) on the stored lower
//              triangle (diagonal halved), through the relative indices
//   Lb_CK = Hb V^T
//   Vb    = L_CK^T Hb + 2 E V Zb,  Db_t = -(V Zb V^T)_tt / d_t^2,
//   Lb_KK = strict_lower(-V^T Vb V^T).
// LDL^T adjoint, supernodes root -> leaves (levels top first), with Fb the
// adjoint of the updated (Schur-complemented) panel values:
//   T1 = (W + W^T) L_CK,  W = Fb gathered at C x C (stored lower triangle)
//   Q  = (Lb_CK E - T1) V                                 -> Fb_CK
//   R  = Q^T L_CK
//   Db_t += -1/2 sum_i L_CK[i,t] T1[i,t] - sum_j L_KK[j,t] R[j,t]
//   Lb_KK -= strict_lower(R D)
//   P = strict_lower(L_KK^T Lb_KK) E + diag(Db),  Ab = V^T P V
//   Fb_KK (stored lower) = Ab_ij + Ab_ji (i > j), Ab_ii.
// dJ/d(stored A values) = Fb at the value map.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"
#include "selinv_steps.cuh"
#include "tile_gemm.cuh"

namespace psi {

enum AdjOp { A_YBAR, A_LHBAR, A_LBAROFF, A_T1, A_Q, A_VPART, A_RPART, A_SYR2K,
             A_DR1, A_DR3, A_DR4, A_DF2, A_DF3, A_DF4 };  // s x s products of the diagonal steps

// The last slice CTA of a split (r x s) tile: out = (-)(sum of the slice
// partials in slice order), its own slice from registers.  Hb = -sum for the
// reverse sweep, T1 = sum for the LDL^T adjoint.
template <class T, int BN>
__device__ __forceinline__ void slice_sum(const Acc<T, BN>& acc, const SnMeta& m, const Task& tk, const T* yp, T* out,
                                          bool negate) {
  const int r = m.r, s = m.s;
  const int64_t rs = (int64_t)r * s;
  tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
    const int i = tk.m0 + mm, n = tk.n0 + nn;
    if (i >= r || n >= s) return;
    const int64_t e = i + (int64_t)n * r;
    T sum = tk.c == 0 ? v : ld_cg(yp + e);
    for (int c = 1; c < m.ksplit; ++c) sum += c == tk.c ? v : ld_cg(yp + c * rs + e);
    out[e] = negate ? -sum : sum;
  });
}

// Occupancy hint per operation: the r^2 s contractions (LHBAR, T1, SYR2K)
// and Q get the step-2 tile's CTAs per SM (one less for 64-wide T1 tiles and
// real Q tiles from 32 wide, whose two products would spill under that
// register cap); the rest keeps the compiler's choice.
template <class T, int BN, int OP>
constexpr int adj_min_ctas() {
  if (OP == A_LHBAR || OP == A_SYR2K) return tile_min_ctas<T, BN>();
  if (OP == A_T1) return BN == 64 ? tile_min_ctas<T, BN>() - 1 : tile_min_ctas<T, BN>();
  if (OP == A_Q) return BN >= 32 && Sc<T>::P == 1 ? tile_min_ctas<T, BN>() - 1 : tile_min_ctas<T, BN>();
  return 1;
}

template <class T, int BN, int OP>
__global__ void __launch_bounds__(TG_THREADS, (adj_min_ctas<T, BN, OP>())) k_adj_tile(AdjArgs a, const Task* __restrict__ tasks) {
  __shared__ TileSmem<T, BN> sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const T* X = (const T*)a.k.X + b * sz.panel;
  const T* L = (const T*)a.k.L + b * sz.panel;
  const T* Lh = (const T*)a.k.Lhat + b * sz.lhat + m.lhat;
  const T* V = (const T*)a.k.Linv + b * sz.linv + m.linv;
  const T* d = (const T*)a.k.D + b * sz.n + m.f;
  T* Xb = (T*)a.Xb + b * sz.panel;
  T* Lb = (T*)a.Lb + b * sz.panel;
  const T* Z = (const T*)a.Zb + b * sz.linv + m.linv;
  T* Yb = (T*)a.Yb + b * sz.lhat + m.lhat;
  T* Hb = (T*)a.Hb + b * sz.lhat + m.lhat;
  const ColDesc* dk = a.k.desc + m.desc;
  const int32_t* rel = a.k.relidx;
  const T zero = Sc<T>::zero();
  const int m0 = tk.m0, n0 = tk.n0;
  auto none = [](int) { return false; };
  auto by_k = [](int) { return true; };
  auto upper_by_k = [m0](int kt) { return kt >= m0 + TG_BM; };
  const LiveRect rect{r - m0, s - n0};  // r x s outputs: fragments inside the output
  Acc<T, BN> acc;
  acc_zero<T, BN>(acc);

  if constexpr (OP == A_YBAR) {  // Yb = Xb_CK - Lhat Zb
    auto la = [&](int mm, int t) { const int i = m0 + mm; return i < r ? Lh[i + (int64_t)t * r] : zero; };
    auto lb = [&](int t, int nn) { const int n = n0 + nn; return n < s ? Z[t + n * s] : zero; };
    tile_mma<T, BN>(sm, 0, s, none, la, lb, acc, rect);
    const T* XbCK = Xb + m.panel + s;
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, n = n0 + nn;
      if (i < r && n < s) Yb[i + (int64_t)n * r] = XbCK[i + (int64_t)n * ld] - v;
    });
  } else if constexpr (OP == A_LHBAR) {  // Hb = -X_CC Yb - Y Zb^T, k-slice tk.c of C (step-2 slices)
    const int kb = tk.c * m.kchunk, ke = min(r, kb + m.kchunk);
    auto la1 = [&](int mm, int kk) {
      const int i = m0 + mm;
      if (i >= r) return zero;
      const int lo = i < kk ? i : kk, hi = i < kk ? kk : i;
      const ColDesc cd = dk[lo];
      return X[cd.col + rel[cd.rel + hi]];
    };
    auto lb1 = [&](int kk, int nn) { const int n = n0 + nn; return n < s ? Yb[kk + (int64_t)n * r] : zero; };
    tile_mma<T, BN>(sm, kb, ke, upper_by_k, la1, lb1, acc, rect);
    if (tk.c == 0) {  // the s-long term rides with the first slice
      const T* Y = X + m.panel + s;
      auto la2 = [&](int mm, int t) { const int i = m0 + mm; return i < r ? Y[i + (int64_t)t * ld] : zero; };
      auto lb2 = [&](int t, int nn) { const int n = n0 + nn; return n < s ? Z[n + t * s] : zero; };
      tile_mma<T, BN>(sm, 0, s, none, la2, lb2, acc, rect);
    }
    T* yp = (T*)a.k.ypart + b * sz.ypart + m.ypart;
    T* out = m.ksplit == 1 ? Hb : yp + (int64_t)tk.c * r * s;
    const T sign = m.ksplit == 1 ? -Sc<T>::one() : Sc<T>::one();
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, n = n0 + nn;
      if (i < r && n < s) out[i + (int64_t)n * r] = sign * v;
    });
    if (m.ksplit > 1 && a.k.tctr && last_slice<BN>(a.k, m, tk, b)) slice_sum<T, BN>(acc, m, tk, yp, Hb, true);
  } else if constexpr (OP == A_LBAROFF) {  // Lb_CK = Hb V^T
    auto la = [&](int mm, int t) { const int i = m0 + mm; return i < r ? Hb[i + (int64_t)t * r] : zero; };
    auto lb = [&](int t, int nn) { const int n = n0 + nn; return n < s ? V[n + t * s] : zero; };
    tile_mma<T, BN>(sm, 0, min(s, n0 + BN), none, la, lb, acc, rect, KUpperB<BN>{n0});
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, n = n0 + nn;
      if (i < r && n < s) Lb[m.panel + s + i + (int64_t)n * ld] = v;
    });
  } else if constexpr (OP == A_T1) {  // T1 = (W + W^T) L_CK, W gathered from Fb (= Xb), k-slice tk.c
    const int kb = tk.c * m.kchunk, ke = min(r, kb + m.kchunk);
    // the product runs on the symmetric W (W_ik on both sides of the diagonal,
    // W_ii once), with no FP64 operation per loaded element; the second W_ii of
    // (W + W^T)'s diagonal is one more product, diag(W_ii) L_CK[i, :], over the
    // rows of the tile on the slice's part of the diagonal (at most 64 k)
    auto la = [&](int mm, int kk) {
      const int i = m0 + mm;
      if (i >= r) return zero;
      const int lo = i < kk ? i : kk, hi = i < kk ? kk : i;
      const ColDesc cd = dk[lo];
      return Xb[cd.col + rel[cd.rel + hi]];
    };
    auto lb = [&](int kk, int nn) { const int n = n0 + nn; return n < s ? L[m.panel + s + kk + (int64_t)n * ld] : zero; };
    tile_mma<T, BN>(sm, kb, ke, upper_by_k, la, lb, acc, rect);
    const int db = max(kb, m0), de = min(min(ke, r), m0 + TG_BM);
    if (db < de) {
      auto ld_ = [&](int mm, int kk) {
        if (m0 + mm != kk) return zero;
        const ColDesc cd = dk[kk];
        return Xb[cd.col + rel[cd.rel + kk]];
      };
      tile_mma<T, BN>(sm, db, de, none, ld_, lb, acc, rect);
    }
    T* yp = (T*)a.k.ypart + b * sz.ypart + m.ypart;
    T* out = m.ksplit == 1 ? Yb : yp + (int64_t)tk.c * r * s;
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, n = n0 + nn;
      if (i < r && n < s) out[i + (int64_t)n * r] = v;
    });
    if (m.ksplit > 1 && a.k.tctr && last_slice<BN>(a.k, m, tk, b)) slice_sum<T, BN>(acc, m, tk, yp, Yb, false);
  } else if constexpr (OP == A_Q) {  // Q = (Lb_CK E - T1) V = Lb_CK (E V) - T1 V -> Fb_CK
    // E V (rows of V divided by d) in W1 from k_adj_ev: no FP64 operation per loaded element
    const T* EV = (const T*)a.W1 + b * sz.linv + m.linv;
    auto la1 = [&](int mm, int t) { const int i = m0 + mm; return i < r ? Yb[i + (int64_t)t * r] : zero; };
    auto lb1 = [&](int t, int nn) { const int n = n0 + nn; return n < s ? V[t + n * s] : zero; };
    tile_mma<T, BN>(sm, n0, s, none, la1, lb1, acc, rect, KLowerB<BN>{n0});
    tile_update<T, BN>(acc, [](int, int, T v) { return -v; });
    auto la2 = [&](int mm, int t) { const int i = m0 + mm; return i < r ? Lb[m.panel + s + i + (int64_t)t * ld] : zero; };
    auto lb2 = [&](int t, int nn) { const int n = n0 + nn; return n < s ? EV[t + n * s] : zero; };
    tile_mma<T, BN>(sm, n0, s, none, la2, lb2, acc, rect, KLowerB<BN>{n0});
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, n = n0 + nn;
      if (i < r && n < s) Xb[m.panel + s + i + (int64_t)n * ld] = v;
    });
  } else if constexpr (OP == A_VPART || OP == A_RPART) {
    // chunk partials of L_CK^T Hb (VPART) or Q^T L_CK with Q = Fb_CK (RPART)
    const int kb = tk.c * m.kchunk3, ke = min(r, kb + m.kchunk3);
    auto la = [&](int mm, int kk) {
      const int i = m0 + mm;
      if (i >= s) return zero;
      return OP == A_VPART ? L[m.panel + s + kk + (int64_t)i * ld] : Xb[m.panel + s + kk + (int64_t)i * ld];
    };
    auto lb = [&](int kk, int nn) {
      const int n = n0 + nn;
      if (n >= s) return zero;
      return OP == A_VPART ? Hb[kk + (int64_t)n * r] : L[m.panel + s + kk + (int64_t)n * ld];
    };
    tile_mma<T, BN>(sm, kb, ke, by_k, la, lb, acc, LiveRect{s - m0, s - n0});
    T* out = (T*)a.k.part + b * sz.part + m.part + (int64_t)tk.c * s * s;
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, n = n0 + nn;
      if (i < s && n < s) out[i + n * s] = v;
    });
  } else if constexpr (OP >= A_DR1) {
    // s x s products of the diagonal-block steps, tile (m0, n0) of K's block:
    //   DR1  W = V Zb            DR3  W = Vb V^T           DR4  Lb_KK = strict_lower(-V^T W)
    //   DF2  P = strict_lower(L_KK^T W) E + diag(Db)       DF3  W = P V      DF4  Ab = V^T W
    T* Zs = (T*)a.Zb + b * sz.linv + m.linv;
    T* W = (T*)a.W1 + b * sz.linv + m.linv;
    const T* Db = (const T*)a.Db + b * sz.n + m.f;
    auto Lkk = [&](int i, int j) {
      return i == j ? Sc<T>::one() : (i > j ? L[m.panel + i + (int64_t)j * ld] : zero);
    };
    auto la = [&](int mm, int q) -> T {
      const int i = m0 + mm;
      if (i >= s) return zero;
      if constexpr (OP == A_DR1) return V[i + q * s];
      if constexpr (OP == A_DR3) return Zs[i + q * s];
      if constexpr (OP == A_DR4 || OP == A_DF4) return V[q + i * s];
      if constexpr (OP == A_DF2) return Lkk(q, i);
      return Zs[i + q * s];  // DF3: P held in Zb
    };
    auto lb = [&](int q, int nn) -> T {
      const int j = n0 + nn;
      if (j >= s) return zero;
      if constexpr (OP == A_DR1) return Zs[q + j * s];
      if constexpr (OP == A_DR3) return V[j + q * s];
      if constexpr (OP == A_DF3) return V[q + j * s];
      return W[q + j * s];  // DR4, DF2, DF4
    };
    constexpr bool by_k_a = OP == A_DR4 || OP == A_DF2 || OP == A_DF4;
    tile_mma<T, BN>(sm, 0, s, [](int) { return by_k_a; }, la, lb, acc, LiveRect{s - m0, s - n0});
    // DR1/DR3/DF3 write W and DF4 writes Zb (its inputs W, V are not written in the same launch)
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, j = n0 + nn;
      if (i >= s || j >= s) return;
      if constexpr (OP == A_DR1 || OP == A_DR3 || OP == A_DF3) W[i + j * s] = v;
      if constexpr (OP == A_DR4) {
        if (i > j) Lb[m.panel + i + (int64_t)j * ld] = -v;
      }
      if constexpr (OP == A_DF2) Zs[i + j * s] = i > j ? v / d[j] : (i == j ? Db[i] : zero);
      if constexpr (OP == A_DF4) Zs[i + j * s] = v;
    });
  } else {  // A_SYR2K: ancestors' Xb += -(Yb Lhat^T + Lhat Yb^T), lower, diagonal halved
    // launched per Schur group (supernodes of a level whose C are disjoint):
    // every target entry is updated by one thread of the launch, no atomics
    auto la1 = [&](int mm, int t) { const int i = m0 + mm; return i < r ? Yb[i + (int64_t)t * r] : zero; };
    auto lb1 = [&](int t, int nn) { const int n = n0 + nn; return n < tk.c ? Lh[n + (int64_t)t * r] : zero; };
    const int dm = m0 - n0;  // fragments with a row inside C, a column below the tile's end, on/below the diagonal
    auto tri = [&](int r0, int c0) { return m0 + r0 < r && n0 + c0 < tk.c && c0 <= dm + r0 + 7; };
    tile_mma<T, BN>(sm, 0, s, none, la1, lb1, acc, tri);
    auto la2 = [&](int mm, int t) { const int i = m0 + mm; return i < r ? Lh[i + (int64_t)t * r] : zero; };
    auto lb2 = [&](int t, int nn) { const int n = n0 + nn; return n < tk.c ? Yb[n + (int64_t)t * r] : zero; };
    tile_mma<T, BN>(sm, 0, s, none, la2, lb2, acc, tri);
    tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
      const int i = m0 + mm, kc = n0 + nn;
      if (i < r && kc < tk.c && kc <= i) {  // tk.c: the Schur tile's column end
        const ColDesc cd = dk[kc];
        T* dst = &Xb[cd.col + rel[cd.rel + i]];
        *dst = *dst + (i == kc ? -0.5 : -1.0) * v;
      }
    });
  }
}

// --------------------------------------------------------------------------
// per-supernode kernels (one CTA each)
// --------------------------------------------------------------------------

// Seed of the reverse sweep (all supernodes; blockIdx.x is the supernode).
// Symmetric G: Xb_KK = G (mirrored from its stored lower triangle) and
// Xb_CK = 2 G_CK (X_CK stands for both X_CK and X_KC).  Panel gradient:
// Xb = G entry for entry.
template <class T>
__global__ void k_adj_seed(AdjArgs a) {
  const int k = blockIdx.x, b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[k];
  const int s = m.s, r = m.r, ld = s + r;
  const T* G = (const T*)a.G + b * sz.panel + m.panel;
  T* Xb = (T*)a.Xb + b * sz.panel + m.panel;
  for (int j = 0; j < s; ++j)
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
      const int64_t e = i + (int64_t)j * ld;
      T v;
      if (a.g_kind == PSELINV_G_PANEL)
        v = G[e];
      else if (i >= s)
        v = 2.0 * G[e];
      else
        v = i >= j ? G[e] : G[j + (int64_t)i * ld];
      Xb[e] = v;
    }
}

// Step-3 chunk partials of a supernode summed in chunk order into chunk 0
// (VPART before the reverse diagonal step, RPART before the factor one);
// blockIdx.z selects one of gridDim.z CTAs sharing the s x s entries.
template <class T>
__global__ void k_adj_sum_parts(AdjArgs a, const int32_t* __restrict__ sns) {
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[k];
  if (m.nchunk < 2) return;
  const int s = m.s;
  T* part = (T*)a.k.part + b * sz.part + m.part;
  const int64_t ss = (int64_t)s * s;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.z * blockDim.x; e < ss; e += (int64_t)gridDim.z * blockDim.x) {
    T acc = part[e];
    for (int c = 1; c < m.nchunk; ++c) acc += part[c * ss + e];
    part[e] = acc;
  }
}

// Zb = (Xb_KK + Xb_KK^T) / 2 for the supernodes of a level.
template <class T>
__global__ void k_adj_zbar(AdjArgs a, const int32_t* __restrict__ sns) {
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[k];
  const int s = m.s, ld = s + m.r;
  const T* Xb = (const T*)a.Xb + b * sz.panel + m.panel;
  T* Z = (T*)a.Zb + b * sz.linv + m.linv;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    Z[e] = 0.5 * (Xb[i + (int64_t)j * ld] + Xb[j + (int64_t)i * ld]);
  }
}

// Sum over a warp (all lanes get it).
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ Cplx warp_sum(Cplx v) { return {warp_sum(v.re), warp_sum(v.im)}; }

// Reverse sweep, elementwise part of the diagonal step, between the DR1 and
// DR3 products: Db_t = -(V Zb V^T)_tt / d_t^2 = -(sum_j G1[t, j] V[t, j]) / d_t^2
// with G1 = V Zb in W1, and Vb = 2 E G1 + (L_CK^T Hb, summed chunk partials) -> Zb.
template <class T>
__global__ void k_adj_dr2(AdjArgs a, const int32_t* __restrict__ sns) {
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[k];
  const int s = m.s;
  const T* V = (const T*)a.k.Linv + b * sz.linv + m.linv;
  const T* d = (const T*)a.k.D + b * sz.n + m.f;
  const T* part = (const T*)a.k.part + b * sz.part + m.part;
  T* Z = (T*)a.Zb + b * sz.linv + m.linv;
  const T* W = (const T*)a.W1 + b * sz.linv + m.linv;
  T* Db = (T*)a.Db + b * sz.n + m.f;
  // blockIdx.z of gridDim.z CTAs: columns t = z (mod gridDim.z), entries e in blocks of blockDim.x
  const int zc = blockIdx.z, nz = gridDim.z;
  for (int t = zc + threadIdx.x * nz; t < s; t += blockDim.x * nz) {
    T acc = Sc<T>::zero();
    for (int j = 0; j < s; ++j) acc += W[t + j * s] * V[t + j * s];
    Db[t] = -(acc / (d[t] * d[t]));
  }
  for (int e = threadIdx.x + zc * blockDim.x; e < s * s; e += blockDim.x * nz) {
    const int t = e % s;
    T vb = 2.0 * W[e] / d[t];
    if (m.nchunk > 0) vb += part[e];  // chunk partials already summed into chunk 0
    Z[e] = vb;
  }
}

// LDL^T adjoint, elementwise part before the DF2 product: Db_t -= 1/2
// sum_i L_CK[i, t] T1[i, t] + sum_j L_KK[j, t] R[j, t] (R = Q^T L_CK, summed
// chunk partials) and W1 = strict_lower(Lb_KK - R D).
template <class T>
__global__ void k_adj_df1(AdjArgs a, const int32_t* __restrict__ sns) {
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[k];
  const int s = m.s, r = m.r, ld = s + r;
  const T* Lp = (const T*)a.k.L + b * sz.panel + m.panel;
  const T* d = (const T*)a.k.D + b * sz.n + m.f;
  const T* part = (const T*)a.k.part + b * sz.part + m.part;
  const T* T1 = (const T*)a.Yb + b * sz.lhat + m.lhat;
  T* Db = (T*)a.Db + b * sz.n + m.f;
  const T* Lb = (const T*)a.Lb + b * sz.panel + m.panel;
  T* W = (T*)a.W1 + b * sz.linv + m.linv;
  __shared__ T colsum[kMaxWidth];
  const T zero = Sc<T>::zero();
  auto R = [&](int i, int j) { return m.nchunk > 0 ? part[i + j * s] : zero; };
  auto Lkk = [&](int i, int j) { return i == j ? Sc<T>::one() : (i > j ? Lp[i + (int64_t)j * ld] : zero); };
  // blockIdx.z of gridDim.z CTAs: columns t = z (mod gridDim.z), one warp per
  // column, lanes along the r rows; entries e of W in blocks of blockDim.x
  const int zc = blockIdx.z, nz = gridDim.z;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int t = zc + warp * nz; t < s; t += nw * nz) {
    T acc = zero;
    for (int i = lane; i < r; i += 32) acc += Lp[s + i + (int64_t)t * ld] * T1[i + (int64_t)t * r];
    acc = warp_sum(acc);
    if (lane == 0) colsum[t] = acc;
  }
  __syncthreads();
  for (int t = zc + threadIdx.x * nz; t < s; t += blockDim.x * nz) {
    T acc2 = zero;
    for (int j = t; j < s; ++j) acc2 += Lkk(j, t) * R(j, t);
    Db[t] = Db[t] - 0.5 * colsum[t] - acc2;
  }
  for (int e = threadIdx.x + zc * blockDim.x; e < s * s; e += blockDim.x * nz) {
    const int i = e % s, j = e / s;
    W[e] = i > j ? Lb[i + (int64_t)j * ld] - R(i, j) * d[j] : zero;
  }
}

// Start of the LDL^T adjoint, every supernode (blockIdx.x): W1 = E V, the
// rows of V = (L_KK)^{-1} divided by d (E = D^{-1}), the second operand of Q.
// W1 is free until the supernode's own DF1.
template <class T>
__global__ void k_adj_ev(AdjArgs a) {
  const int k = blockIdx.x, b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[k];
  const int s = m.s;
  const T* V = (const T*)a.k.Linv + b * sz.linv + m.linv;
  const T* d = (const T*)a.k.D + b * sz.n + m.f;
  T* EV = (T*)a.W1 + b * sz.linv + m.linv;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) EV[e] = V[e] / d[e % s];
}

// LDL^T adjoint, last diagonal part: Fb_KK (stored lower) = Ab_ij + Ab_ji
// (i > j), Ab_ii with Ab = V^T P V (from DF4, in Zb).
template <class T>
__global__ void k_adj_df5(AdjArgs a, const int32_t* __restrict__ sns) {
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const Sizes sz = a.k.sz;
  const SnMeta m = a.k.meta[k];
  const int s = m.s, ld = s + m.r;
  const T* Ab = (const T*)a.Zb + b * sz.linv + m.linv;
  T* Fb = (T*)a.Xb + b * sz.panel + m.panel;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    if (i >= j) Fb[i + (int64_t)j * ld] = i == j ? Ab[e] : Ab[e] + Ab[j + i * s];
  }
}

// --------------------------------------------------------------------------
// launches
// --------------------------------------------------------------------------

template <class T, int BN>
static cudaError_t adj_tile_tb(int op, const AdjArgs& a, const Task* t, int64_t n, cudaStream_t st) {
  const dim3 grid((unsigned)n, a.k.sz.batch);
  switch (op) {
    case A_YBAR: k_adj_tile<T, BN, A_YBAR><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_LHBAR: k_adj_tile<T, BN, A_LHBAR><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_LBAROFF: k_adj_tile<T, BN, A_LBAROFF><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_T1: k_adj_tile<T, BN, A_T1><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_Q: k_adj_tile<T, BN, A_Q><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_VPART: k_adj_tile<T, BN, A_VPART><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_RPART: k_adj_tile<T, BN, A_RPART><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_DR1: k_adj_tile<T, BN, A_DR1><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_DR3: k_adj_tile<T, BN, A_DR3><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_DR4: k_adj_tile<T, BN, A_DR4><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_DF2: k_adj_tile<T, BN, A_DF2><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_DF3: k_adj_tile<T, BN, A_DF3><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    case A_DF4: k_adj_tile<T, BN, A_DF4><<<grid, TG_THREADS, 0, st>>>(a, t); break;
    default: k_adj_tile<T, BN, A_SYR2K><<<grid, TG_THREADS, 0, st>>>(a, t); break;
  }
  return cudaGetLastError();
}

template <class T>
static cudaError_t adj_tile_t(int op, int var, const AdjArgs& a, const Task* t, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  switch (var) {
    case 0: return adj_tile_tb<T, 8>(op, a, t, n, st);
    case 1: return adj_tile_tb<T, 16>(op, a, t, n, st);
    case 2: return adj_tile_tb<T, 32>(op, a, t, n, st);
    default:
      if constexpr (Sc<T>::P == 1) return adj_tile_tb<T, 64>(op, a, t, n, st);
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adj_tiles(AdjKern k, int var, const AdjArgs& a, const Task* t, int64_t n, cudaStream_t st) {
  static const int map[] = {A_YBAR, A_LHBAR, A_LBAROFF, A_T1, A_Q, A_VPART, A_RPART, A_SYR2K,
                            A_DR1, A_DR3, A_DR4, A_DF2, A_DF3, A_DF4};
  const int op = map[(int)k];
  return a.k.dtype == PSELINV_C128 ? adj_tile_t<Cplx>(op, var, a, t, n, st) : adj_tile_t<double>(op, var, a, t, n, st);
}

template <class T>
static cudaError_t adj_sn_t(AdjSn k, const AdjArgs& a, const int32_t* sns, int nsn, cudaStream_t st) {
  if (nsn <= 0) return cudaSuccess;
  const dim3 grid(nsn, a.k.sz.batch);
  switch (k) {
    case AdjSn::Seed: k_adj_seed<T><<<grid, 256, 0, st>>>(a); break;
    case AdjSn::Ev: k_adj_ev<T><<<grid, 256, 0, st>>>(a); break;
    case AdjSn::Zbar: k_adj_zbar<T><<<grid, 256, 0, st>>>(a, sns); break;
    case AdjSn::Dr2: k_adj_dr2<T><<<dim3(nsn, a.k.sz.batch, 8), 256, 0, st>>>(a, sns); break;
    case AdjSn::Df1: k_adj_df1<T><<<dim3(nsn, a.k.sz.batch, 8), 256, 0, st>>>(a, sns); break;
    case AdjSn::Df5: k_adj_df5<T><<<grid, 256, 0, st>>>(a, sns); break;
    case AdjSn::SumParts: k_adj_sum_parts<T><<<dim3(nsn, a.k.sz.batch, 8), 256, 0, st>>>(a, sns); break;
    default: break;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_per_sn(AdjSn k, const AdjArgs& a, const int32_t* sns, int nsn, cudaStream_t st) {
  return a.k.dtype == PSELINV_C128 ? adj_sn_t<Cplx>(k, a, sns, nsn, st) : adj_sn_t<double>(k, a, sns, nsn, st);
}

}  // namespace psi
