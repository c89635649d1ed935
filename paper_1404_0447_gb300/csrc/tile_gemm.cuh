// FP64 tile GEMM core on the DMMA pipe (mma.sync m8n8k4 .f64; tcgen05 has
// no f64 kind, so this is the tensor-core path for double precision on
// sm_103a).  One CTA of 128 threads computes a 64 x 64 output tile as a
// 2 x 2 grid of warps, each warp 32 x 32 = 4 x 4 fragments of 8 x 8.
//
// Operands are fetched element by element through loader functors, so the
// same core serves dense panels and the index-driven gather of X_{C,C}
// (relative indices) without a staging copy in global memory.  Global
// loads for k-tile t+1 are issued into registers before the MMAs of tile t
// and stored to the other shared-memory buffer afterwards.
#pragma once

#include <cstdint>

namespace psi {

constexpr int TG_BM = 64, TG_BN = 64, TG_BK = 16, TG_THREADS = 128;
constexpr int TG_PAD = 4;  // row stride 68 doubles: conflict-free fragment reads
constexpr int TG_LDA = TG_BM + TG_PAD, TG_LDB = TG_BN + TG_PAD;
constexpr int TG_AREG = TG_BM * TG_BK / TG_THREADS;  // 8 elements per thread
constexpr int TG_BREG = TG_BK * TG_BN / TG_THREADS;  // 8 elements per thread

struct TileSmem {
  double a[2][TG_BK][TG_LDA];
  double b[2][TG_BK][TG_LDB];
};

// D = A(8x4) * B(4x8) + D.  Lane l holds A[l>>2][l&3], B[l&3][l>>2] and
// D[l>>2][2*(l&3) + {0,1}].
__device__ __forceinline__ void dmma884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// Accumulates acc += A[m0:m0+64, kbeg:kend] * B[kbeg:kend, n0:n0+64].
// la(m, k) (m tile-local, k global) and lb(k, n) (n tile-local) return the
// operand element, or 0 outside the operand.  a_by_k_at(kt) picks, per
// k-tile starting at kt, the thread mapping of the A loads:
//   A: if a_by_k, thread t loads k = kt + t % 16, m = t / 16 + 8 j (j < 8);
//      else        thread t loads m = t % 64,     k = t / 64 + 2 j.
//   B: thread t loads k = kt + t % 16, n = t / 16 + 8 j.
// acc[i][j][e] is row wm + 8 i + (lane >> 2), column wn + 8 j + 2 (lane & 3) + e
// of the tile, with (wm, wn) = 32 * (warp % 2, warp / 2).
template <class MA, class LA, class LB>
__device__ __forceinline__ void tile_mma(TileSmem& sm, int kbeg, int kend, const MA& a_by_k_at, const LA& la,
                                         const LB& lb, double (&acc)[4][4][2]) {
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int g = lane >> 2, q = lane & 3;
  double ra[TG_AREG], rb[TG_BREG];
  bool a_by_k = false;  // thread mapping of the A tile held in ra

  auto fetch = [&](int kt) {
    a_by_k = a_by_k_at(kt);
    if (a_by_k) {
#pragma unroll
      for (int j = 0; j < TG_AREG; ++j) {
        const int kk = kt + (t & 15), mm = (t >> 4) + 8 * j;
        ra[j] = kk < kend ? la(mm, kk) : 0.0;
      }
    } else {
#pragma unroll
      for (int j = 0; j < TG_AREG; ++j) {
        const int kk = kt + (t >> 6) + 2 * j, mm = t & 63;
        ra[j] = kk < kend ? la(mm, kk) : 0.0;
      }
    }
#pragma unroll
    for (int j = 0; j < TG_BREG; ++j) {
      const int kk = kt + (t & 15), nn = (t >> 4) + 8 * j;
      rb[j] = kk < kend ? lb(kk, nn) : 0.0;
    }
  };
  auto stash = [&](int buf) {
    if (a_by_k) {
#pragma unroll
      for (int j = 0; j < TG_AREG; ++j) sm.a[buf][t & 15][(t >> 4) + 8 * j] = ra[j];
    } else {
#pragma unroll
      for (int j = 0; j < TG_AREG; ++j) sm.a[buf][(t >> 6) + 2 * j][t & 63] = ra[j];
    }
#pragma unroll
    for (int j = 0; j < TG_BREG; ++j) sm.b[buf][t & 15][(t >> 4) + 8 * j] = rb[j];
  };

  const int nk = (kend - kbeg + TG_BK - 1) / TG_BK;
  if (nk <= 0) return;
  fetch(kbeg);
  stash(0);
  __syncthreads();
  for (int it = 0; it < nk; ++it) {
    const int buf = it & 1;
    if (it + 1 < nk) fetch(kbeg + (it + 1) * TG_BK);
#pragma unroll
    for (int ks = 0; ks < TG_BK; ks += 4) {
      double fa[4], fb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) fa[i] = sm.a[buf][ks + q][wm + 8 * i + g];
#pragma unroll
      for (int j = 0; j < 4; ++j) fb[j] = sm.b[buf][ks + q][wn + 8 * j + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma884(acc[i][j][0], acc[i][j][1], fa[i], fb[j]);
    }
    if (it + 1 < nk) stash(buf ^ 1);
    __syncthreads();
  }
}

// Visit every accumulator with its tile coordinates: f(m, n, value).
template <class F>
__device__ __forceinline__ void tile_epilogue(const double (&acc)[4][4][2], const F& f) {
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) f(wm + 8 * i + g, wn + 8 * j + 2 * q + e, acc[i][j][e]);
}

}  // namespace psi
