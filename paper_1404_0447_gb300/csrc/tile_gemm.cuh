// FP64 tile GEMM core on sm_103a: mma.sync m8n8k4 .f64 (on GB300 these run
// on the FP64 pipe; tcgen05 has no f64 kind).  One CTA of 128 threads
// computes a 64 x BN output tile, BN in {8, 16, 32, 64}; complex128
// operands are split into real and imaginary planes and each complex
// fragment product takes four real MMAs (complex symmetric matrices: no
// conjugation anywhere).
//
// Operands are fetched element by element through loader functors, so the
// same core serves dense panels and the index-driven gather of X_{C,C}
// (relative indices) without a staging copy in global memory.  Global loads
// for k-tile t+1 are issued into registers before the MMAs of tile t and
// stored to the other shared-memory buffer afterwards.
#pragma once

#include <cstdint>

namespace psi {

// ---------------------------------------------------------------------------
// scalar types
// ---------------------------------------------------------------------------

struct Cplx {
  double re, im;
};

__host__ __device__ __forceinline__ Cplx operator+(Cplx a, Cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ Cplx operator-(Cplx a, Cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ Cplx operator-(Cplx a) { return {-a.re, -a.im}; }
__host__ __device__ __forceinline__ Cplx operator*(Cplx a, Cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ Cplx operator*(double a, Cplx b) { return {a * b.re, a * b.im}; }
// a / b = a * conj(b) / |b|^2
__host__ __device__ __forceinline__ Cplx operator/(Cplx a, Cplx b) {
  const double den = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
__host__ __device__ __forceinline__ Cplx& operator+=(Cplx& a, Cplx b) { return a = a + b; }
__host__ __device__ __forceinline__ Cplx& operator-=(Cplx& a, Cplx b) { return a = a - b; }

template <class T>
struct Sc;
template <>
struct Sc<double> {
  static constexpr int P = 1;  // real planes
  __device__ __forceinline__ static double zero() { return 0.0; }
  __device__ __forceinline__ static double one() { return 1.0; }
  __device__ __forceinline__ static double plane(double v, int) { return v; }
  __device__ __forceinline__ static bool bad(double v) { return !isfinite(v) || v == 0.0; }
  __device__ __forceinline__ static bool is_zero(double v) { return v == 0.0; }
};
template <>
struct Sc<Cplx> {
  static constexpr int P = 2;
  __device__ __forceinline__ static Cplx zero() { return {0.0, 0.0}; }
  __device__ __forceinline__ static Cplx one() { return {1.0, 0.0}; }
  __device__ __forceinline__ static double plane(Cplx v, int p) { return p ? v.im : v.re; }
  __device__ __forceinline__ static bool bad(Cplx v) {
    return !isfinite(v.re) || !isfinite(v.im) || (v.re == 0.0 && v.im == 0.0);
  }
  __device__ __forceinline__ static bool is_zero(Cplx v) { return v.re == 0.0 && v.im == 0.0; }
};

// ---------------------------------------------------------------------------
// tile geometry
// ---------------------------------------------------------------------------

constexpr int TG_BM = 64, TG_BK = 16, TG_THREADS = 128;
constexpr int TG_LDA = TG_BM + 4;  // row stride = 4 (mod 16) doubles: conflict-free fragment reads

// Warps: BN >= 32 -> 2 x 2 (warp tile 32 x BN/2); BN <= 16 -> 4 x 1 (16 x BN).
template <int BN>
struct Geo {
  static constexpr int WN = BN >= 32 ? 2 : 1;
  static constexpr int WM = 4 / WN;
  static constexpr int FM = TG_BM / WM / 8;  // 8-row fragments per warp
  static constexpr int FN = BN / WN / 8;     // 8-column fragments per warp
  static constexpr int LDB = BN + 4;         // 4 (mod 16) for every BN
  static constexpr int BREG = TG_BK * BN / TG_THREADS;
};
constexpr int TG_AREG = TG_BM * TG_BK / TG_THREADS;  // 8 A elements per thread per k-tile

// CTAs per SM the tile kernels are compiled for (a register cap of
// 65536 / (128 x this)): the occupancy each tile width had before the
// fragment predicates below raised the compiler's register choice.
template <class T, int BN>
constexpr int tile_min_ctas() {
  return Sc<T>::P == 2 ? (BN >= 32 ? 3 : BN >= 16 ? 4 : 5) : (BN >= 64 ? 4 : BN >= 32 ? 6 : BN >= 16 ? 8 : 9);
}

template <class T, int BN>
struct TileSmem {
  static constexpr int P = Sc<T>::P;
  double a[2][P][TG_BK][TG_LDA];
  double b[2][P][TG_BK][Geo<BN>::LDB];
};

template <class T, int BN>
using Acc = double[Sc<T>::P][Geo<BN>::FM][Geo<BN>::FN][2];

// D(8x8) += A(8x4) B(4x8).  Lane l holds A[l>>2][l&3], B[l&3][l>>2] and
// D[l>>2][2(l&3) + {0,1}].
__device__ __forceinline__ void dmma884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

template <class T, int BN>
__device__ __forceinline__ void acc_zero(Acc<T, BN>& acc) {
  constexpr int P = Sc<T>::P;
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int i = 0; i < Geo<BN>::FM; ++i)
#pragma unroll
      for (int j = 0; j < Geo<BN>::FN; ++j) acc[p][i][j][0] = acc[p][i][j][1] = 0.0;
}

// acc += A[0:64, kbeg:kend] * B[kbeg:kend, 0:BN] of the tile.
// la(m, k) (m tile-local, k global) and lb(k, n) (n tile-local) return the
// operand element (or zero outside the operand); a_by_k_at(kt) picks, per
// k-tile, the thread mapping of the A loads:
//   A: a_by_k: thread t loads k = kt + t % 16, m = t / 16 + 8 j (j < 8);
//      else:   thread t loads m = t % 64,     k = kt + t / 64 + 2 j.
//   B: thread t loads k = kt + t % 16, n = t / 16 + 8 j (j < BN / 8).
// acc[p][i][j][e] is plane p of tile element (wm + 8 i + lane / 4,
// wn + 8 j + 2 (lane % 4) + e), (wm, wn) = the warp's origin.
//
// The FP64 pipe is the bound of every caller, so padding is not computed:
// the MMAs of an 8 x 8 output fragment whose origin (r0, c0) (tile-local)
// fails live(r0, c0) are skipped (ragged edges of the output, fragments
// wholly above the diagonal of a triangular output), and so are the 4-deep
// k-steps at or past kend.  Skipped fragments keep their accumulators (zero
// from acc_zero) and callers store only live entries.  A triangular B
// operand adds klive: klive.frag(kk, c0) is false when B is zero on rows
// kk..kk+3 for the fragment's columns, and klive.all(kt) is true when no
// fragment has such zero rows in the k-tile [kt, kt + 16).
struct KAllLive {
  __device__ __forceinline__ bool all(int) const { return true; }
  __device__ __forceinline__ bool frag(int, int) const { return true; }
};

template <class T, int BN, class MA, class LA, class LB, class LIVE, class KLIVE = KAllLive>
__device__ __forceinline__ void tile_mma(TileSmem<T, BN>& sm, int kbeg, int kend, const MA& a_by_k_at, const LA& la,
                                         const LB& lb, Acc<T, BN>& acc, const LIVE& live,
                                         const KLIVE& klive = KAllLive{}) {
  using G = Geo<BN>;
  constexpr int P = Sc<T>::P;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int wm = (warp % G::WM) * (TG_BM / G::WM), wn = (warp / G::WM) * (BN / G::WN);
  const int g = lane >> 2, q = lane & 3;
  T ra[TG_AREG], rb[G::BREG];
  bool a_by_k = false;
  uint32_t lmask = 0;  // bit i * FN + j: fragment (i, j) of this warp is live (warp-uniform)
#pragma unroll
  for (int i = 0; i < G::FM; ++i)
#pragma unroll
    for (int j = 0; j < G::FN; ++j)
      if (live(wm + 8 * i, wn + 8 * j)) lmask |= 1u << (i * G::FN + j);

  auto fetch = [&](int kt) {
    a_by_k = a_by_k_at(kt);
    if (a_by_k) {
#pragma unroll
      for (int j = 0; j < TG_AREG; ++j) {
        const int kk = kt + (t & 15), mm = (t >> 4) + 8 * j;
        ra[j] = kk < kend ? la(mm, kk) : Sc<T>::zero();
      }
    } else {
#pragma unroll
      for (int j = 0; j < TG_AREG; ++j) {
        const int kk = kt + (t >> 6) + 2 * j, mm = t & 63;
        ra[j] = kk < kend ? la(mm, kk) : Sc<T>::zero();
      }
    }
#pragma unroll
    for (int j = 0; j < G::BREG; ++j) {
      const int kk = kt + (t & 15), nn = (t >> 4) + 8 * j;
      rb[j] = kk < kend ? lb(kk, nn) : Sc<T>::zero();
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      if (a_by_k) {
#pragma unroll
        for (int j = 0; j < TG_AREG; ++j) sm.a[buf][p][t & 15][(t >> 4) + 8 * j] = Sc<T>::plane(ra[j], p);
      } else {
#pragma unroll
        for (int j = 0; j < TG_AREG; ++j) sm.a[buf][p][(t >> 6) + 2 * j][t & 63] = Sc<T>::plane(ra[j], p);
      }
#pragma unroll
      for (int j = 0; j < G::BREG; ++j) sm.b[buf][p][t & 15][(t >> 4) + 8 * j] = Sc<T>::plane(rb[j], p);
    }
  };

  // one 4-deep k-step: the fragments of this warp whose bit is set in mask
  constexpr uint32_t kAll = (1u << (G::FM * G::FN)) - 1u;
  auto kstep = [&](int buf, int ks, uint32_t mask) {
    double fa[P][G::FM], fb[P][G::FN];
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
      for (int i = 0; i < G::FM; ++i) fa[p][i] = sm.a[buf][p][ks + q][wm + 8 * i + g];
#pragma unroll
      for (int j = 0; j < G::FN; ++j) fb[p][j] = sm.b[buf][p][ks + q][wn + 8 * j + g];
    }
#pragma unroll
    for (int i = 0; i < G::FM; ++i)
#pragma unroll
      for (int j = 0; j < G::FN; ++j) {
        if (!(mask & (1u << (i * G::FN + j)))) continue;
        dmma884(acc[0][i][j][0], acc[0][i][j][1], fa[0][i], fb[0][j]);
        if constexpr (P == 2) {
          dmma884(acc[0][i][j][0], acc[0][i][j][1], -fa[1][i], fb[1][j]);
          dmma884(acc[1][i][j][0], acc[1][i][j][1], fa[0][i], fb[1][j]);
          dmma884(acc[1][i][j][0], acc[1][i][j][1], fa[1][i], fb[0][j]);
        }
      }
  };

  const int nk = (kend - kbeg + TG_BK - 1) / TG_BK;
  if (nk <= 0) return;
  fetch(kbeg);
  stash(0);
  __syncthreads();
  for (int it = 0; it < nk; ++it) {
    const int buf = it & 1;
    if (it + 1 < nk) fetch(kbeg + (it + 1) * TG_BK);
    const int kt = kbeg + it * TG_BK;
    const int kleft = kend - kt;  // valid k of this k-tile (> 0)
    if (kleft >= TG_BK && lmask == kAll && klive.all(kt)) {
      // interior k-tile of a tile with every fragment live: no checks
#pragma unroll
      for (int ks = 0; ks < TG_BK; ks += 4) kstep(buf, ks, kAll);
    } else {
#pragma unroll
      for (int ks = 0; ks < TG_BK; ks += 4) {
        if (ks >= kleft) continue;
        uint32_t m = lmask;
#pragma unroll
        for (int j = 0; j < G::FN; ++j)
          if (!klive.frag(kt + ks, wn + 8 * j))
#pragma unroll
            for (int i = 0; i < G::FM; ++i) m &= ~(1u << (i * G::FN + j));
        kstep(buf, ks, m);
      }
    }
    if (it + 1 < nk) stash(buf ^ 1);
    __syncthreads();
  }
}

// Every fragment live.
template <class T, int BN, class MA, class LA, class LB>
__device__ __forceinline__ void tile_mma(TileSmem<T, BN>& sm, int kbeg, int kend, const MA& a_by_k_at, const LA& la,
                                         const LB& lb, Acc<T, BN>& acc) {
  tile_mma<T, BN>(sm, kbeg, kend, a_by_k_at, la, lb, acc, [](int, int) { return true; });
}

// Fragments with a row below mlim and a column below nlim (tile-local): a
// rectangular output's ragged edges.
struct LiveRect {
  int mlim, nlim;
  __device__ __forceinline__ bool operator()(int r0, int c0) const { return r0 < mlim && c0 < nlim; }
};

// B lower triangular in (k, global column): B[k][n] = 0 for k < n; n0 = the
// tile's first column.
template <int BN>
struct KLowerB {
  int n0;
  __device__ __forceinline__ bool all(int kt) const { return kt + 3 >= n0 + BN - 8; }
  __device__ __forceinline__ bool frag(int kk, int c0) const { return kk + 3 >= n0 + c0; }
};

// B upper triangular in (k, global column): B[k][n] = 0 for k > n.
template <int BN>
struct KUpperB {
  int n0;
  __device__ __forceinline__ bool all(int kt) const { return kt + TG_BK - 4 <= n0 + 7; }
  __device__ __forceinline__ bool frag(int kk, int c0) const { return kk <= n0 + c0 + 7; }
};

// Visit every accumulator with its tile coordinates: f(m, n, value).
template <class T, int BN, class F>
__device__ __forceinline__ void tile_epilogue(const Acc<T, BN>& acc, const F& f) {
  using G = Geo<BN>;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int wm = (warp % G::WM) * (TG_BM / G::WM), wn = (warp / G::WM) * (BN / G::WN);
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int i = 0; i < G::FM; ++i)
#pragma unroll
    for (int j = 0; j < G::FN; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        T v;
        if constexpr (Sc<T>::P == 1) {
          v = acc[0][i][j][e];
        } else {
          v = T{acc[0][i][j][e], acc[1][i][j][e]};
        }
        f(wm + 8 * i + g, wn + 8 * j + 2 * q + e, v);
      }
}

// acc(mm, nn) = f(mm, nn, acc(mm, nn)) for every element of the tile
// (tile-local coordinates as in tile_epilogue).
template <class T, int BN, class F>
__device__ __forceinline__ void tile_update(Acc<T, BN>& acc, const F& f) {
  using G = Geo<BN>;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int wm = (warp % G::WM) * (TG_BM / G::WM), wn = (warp / G::WM) * (BN / G::WN);
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int i = 0; i < G::FM; ++i)
#pragma unroll
    for (int j = 0; j < G::FN; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        T v;
        if constexpr (Sc<T>::P == 1) {
          v = acc[0][i][j][e];
        } else {
          v = T{acc[0][i][j][e], acc[1][i][j][e]};
        }
        v = f(wm + 8 * i + g, wn + 8 * j + 2 * q + e, v);
        if constexpr (Sc<T>::P == 1) {
          acc[0][i][j][e] = v;
        } else {
          acc[0][i][j][e] = v.re;
          acc[1][i][j][e] = v.im;
        }
      }
}

}  // namespace psi
