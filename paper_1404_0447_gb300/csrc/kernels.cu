// Device kernels of the supernodal LDL^T and the selected inversion,
// templated on the scalar (double, or complex symmetric Cplx) and on the
// output tile width BN of the tile GEMMs.
//
// Storage (per batch member, offsets in SnMeta, elements of the scalar):
// L and X panels are (s + r) x s column-major blocks with ld = s + r whose
// rows are the supernode's own columns followed by R(K) = C; Lhat_{C,K} is
// r x s with ld = r; (L_KK)^{-1} is s x s with ld = s; D holds the pivots.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"
#include "selinv_steps.cuh"
#include "tile_gemm.cuh"

namespace psi {

// packed lower-triangular index, column-major: (i, j), i >= j, order s
__device__ __forceinline__ int pk(int i, int j, int s) { return j * s - (j * (j - 1)) / 2 + (i - j); }

// elements of the blocked inverse's scratch S for width s: (ceil(s/16) - 1)
// blocks of 16 x 16 (at least one)
__host__ __device__ __forceinline__ int fd_scratch(int s) {
  const int nb = (s + 15) / 16;
  return 256 * (nb > 1 ? nb - 1 : 1);
}

// Status words 0-1 hold one 64-bit key (column << 2 | kind), kind 1 = zero
// pivot, 2 = non-finite: the minimum is the first bad column and, within
// it, a zero pivot before its consequences.
__device__ void report_pivot(int* status, int col, bool zero) {
  atomicMin(reinterpret_cast<unsigned long long*>(status),
            ((unsigned long long)(unsigned)col << 2) | (zero ? 1ull : 2ull));
}

// --------------------------------------------------------------------------
// value scatter / selected-entry gather (HBM-bound, index driven)
// --------------------------------------------------------------------------

template <class T>
__global__ void k_scatter_values(const T* __restrict__ vals, const int64_t* __restrict__ vmap, int64_t nnz,
                                 T* __restrict__ L, int64_t panel_total) {
  const int b = blockIdx.y;
  const T* v = vals + (int64_t)b * nnz;
  T* Lb = L + (int64_t)b * panel_total;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
    Lb[vmap[q]] = v[q];
}

// Non-symmetric values: entry q's pair (A_ij, A_ji) goes to the L and U
// panels at its position, or to the U and L panels where the ordering
// transposed it.
template <class T>
__global__ void k_scatter_values_lu(const T* __restrict__ lo, const T* __restrict__ up,
                                    const int64_t* __restrict__ vmap, const uint8_t* __restrict__ flip,
                                    int64_t nnz, T* __restrict__ L, T* __restrict__ U, int64_t panel_total) {
  const int b = blockIdx.y;
  const T* vl = lo + (int64_t)b * nnz;
  const T* vu = up + (int64_t)b * nnz;
  T* Lb = L + (int64_t)b * panel_total;
  T* Ub = U + (int64_t)b * panel_total;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = vmap[q];
    const bool f = flip[q] != 0;
    Lb[p] = f ? vu[q] : vl[q];
    Ub[p] = f ? vl[q] : vu[q];
  }
}

// Non-symmetric gather: X_ij (upper = 0) or X_ji (upper = 1) for the stored
// entry q at (i, j), from the XL or XU panel depending on the flip.
template <class T>
__global__ void k_gather_values_lu(const T* __restrict__ XL, const T* __restrict__ XU, int64_t panel_total,
                                   const int64_t* __restrict__ vmap, const uint8_t* __restrict__ flip, int64_t nnz,
                                   int upper, T* __restrict__ out) {
  const int b = blockIdx.y;
  const T* Xl = XL + (int64_t)b * panel_total;
  const T* Xu = XU + (int64_t)b * panel_total;
  T* o = out + (int64_t)b * nnz;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
    o[q] = ((flip[q] != 0) != (upper != 0)) ? Xu[vmap[q]] : Xl[vmap[q]];
}

// out[q] = X at the panel position of stored entry q; with a diagonal mask,
// off-diagonal entries are doubled (gradient with respect to a stored value
// that stands for both A_ij and A_ji).
template <class T>
__global__ void k_gather_values(const T* __restrict__ X, int64_t panel_total, const int64_t* __restrict__ vmap,
                                const uint8_t* __restrict__ diagmask, int64_t nnz, T* __restrict__ out) {
  const int b = blockIdx.y;
  const T* Xb = X + (int64_t)b * panel_total;
  T* o = out + (int64_t)b * nnz;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    const T v = Xb[vmap[q]];
    o[q] = (diagmask && !diagmask[q]) ? 2.0 * v : v;
  }
}

// --------------------------------------------------------------------------
// diagonal blocks
// --------------------------------------------------------------------------

// V = (L_KK)^{-1} for the unit lower triangle held packed in Tp (shared
// memory), written column-major to global memory (ld s, zeros above the
// diagonal); one column per thread.
template <class T>
__device__ void unit_lower_inverse(const T* Tp, int s, T* V) {
  for (int c = threadIdx.x; c < s; c += blockDim.x) {
    for (int i = 0; i < c; ++i) V[i + c * s] = Sc<T>::zero();
    V[c + c * s] = Sc<T>::one();
    for (int i = c + 1; i < s; ++i) {
      T acc = Sc<T>::zero();
      for (int q = c; q < i; ++q) acc += Tp[pk(i, q, s)] * V[q + c * s];
      V[i + c * s] = -acc;
    }
  }
}

// Where unit_lower_inverse_blocked keeps V: column-major in global memory
// (ld s; the upper triangle is written as zeros), or packed lower in shared
// memory (the pk layout; only the lower triangle exists).
template <class T>
struct VGlobal {
  static constexpr bool kPacked = false;
  T* p;
  int s;
  __device__ __forceinline__ T& operator()(int i, int j) const { return p[i + (int64_t)j * s]; }
};
template <class T>
struct VPacked {
  static constexpr bool kPacked = true;
  T* p;
  int s;
  __device__ __forceinline__ T& operator()(int i, int j) const { return p[pk(i, j, s)]; }
};

// V = (L_KK)^{-1} for the unit lower triangle held packed in Tp (shared
// memory), by 16 x 16 blocks so that the whole CTA works at every step:
// first the diagonal blocks V_ii = (L_ii)^{-1} (one column per thread),
// then, for block distance d = 1, 2, ... (all block pairs (i, j) with
// i - j = d at once), S = sum_{k=j}^{i-1} L_ik V_kj and V_ij = -V_ii S.
// V (see VGlobal / VPacked) is read back by the later steps of this CTA;
// S (shared) holds (ceil(s/16) - 1) blocks of 16 x 16.
template <class T, class VA>
__device__ void unit_lower_inverse_blocked(const T* Tp, int s, const VA& V, T* S) {
  constexpr int B = 16;
  const int nb = (s + B - 1) / B;
  const int nt = blockDim.x, t = threadIdx.x;
  for (int c = t; c < s; c += nt) {
    const int i1 = min((c / B + 1) * B, s);
    if constexpr (!VA::kPacked)
      for (int i = 0; i < c; ++i) V(i, c) = Sc<T>::zero();
    V(c, c) = Sc<T>::one();
    for (int i = c + 1; i < i1; ++i) {
      T acc = Sc<T>::zero();
      for (int q = c; q < i; ++q) acc += Tp[pk(i, q, s)] * V(q, c);
      V(i, c) = -acc;
    }
  }
  __syncthreads();
  for (int d = 1; d < nb; ++d) {
    const int npair = nb - d;  // pairs (j + d, j), j = 0 .. nb - d - 1
    for (int e = t; e < npair * B * B; e += nt) {
      const int j = e / (B * B), rr = (e / B) % B, cc = e % B;
      const int row = (j + d) * B + rr, col = j * B + cc;
      T acc = Sc<T>::zero();
      if (row < s && col < s)  // V(q, col) = 0 above the diagonal: q from col
        for (int q = col; q < (j + d) * B; ++q) acc += Tp[pk(row, q, s)] * V(q, col);
      S[e] = acc;
    }
    __syncthreads();
    for (int e = t; e < npair * B * B; e += nt) {
      const int j = e / (B * B), rr = (e / B) % B, cc = e % B;
      const int i0 = (j + d) * B, row = i0 + rr, col = j * B + cc;
      if (row >= s || col >= s) continue;
      T acc = Sc<T>::zero();
      for (int q = 0; q <= rr; ++q) acc += V(row, i0 + q) * S[j * B * B + q * B + cc];
      V(row, col) = -acc;
    }
    __syncthreads();
  }
}

// Factorisation, one CTA per supernode of the level: right-looking LDL^T of
// the s x s diagonal block (lower part, already holding A_KK minus all
// descendant updates) in shared memory; L_KK (unit diagonal implied, d_j on
// the diagonal slot) back to the panel, d to D, (L_KK)^{-1} to linv.
// Column step j: u = column j below the diagonal, then L_ij = u_i / d_j and
// the trailing lower triangle T_ik -= L_ij u_k, one warp per column k (no
// integer division, only lower-triangle entries visited).
template <class T>
__global__ void k_factor_diag(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns, T* __restrict__ L,
                              T* __restrict__ D, T* __restrict__ Linv, Sizes sz, int* status) {
  extern __shared__ __align__(16) unsigned char shraw[];
  T* Tp = reinterpret_cast<T*>(shraw);
  const int k = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, ld = m.s + m.r;
  T* u = Tp + s * (s + 1) / 2;
  T* S = u + s;
  T* P = L + b * sz.panel + m.panel;
  const int nt = blockDim.x, t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5, nw = nt >> 5;
  for (int j = warp; j < s; j += nw) {
    const int cb = pk(j, j, s);
    for (int i = j + lane; i < s; i += 32) Tp[cb + i - j] = P[i + (int64_t)j * ld];
  }
  __syncthreads();
  // rd[0] = 1 / d_j of the current step: one division per column, by the
  // thread that last wrote the pivot (thread 0 here, then warp 0 lane 0 of
  // the update, which owns entry (j+1, j+1))
  T* rd = S;
  if (t == 0) rd[0] = Sc<T>::one() / Tp[0];
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    const int cj = pk(j, j, s);
    const T d = Tp[cj], rdj = rd[0];
    if (t == 0 && Sc<T>::bad(d)) report_pivot(status, m.f + j, Sc<T>::is_zero(d));
    for (int i = j + 1 + t; i < s; i += nt) {
      const T v = Tp[cj + i - j];
      u[i] = v;
      Tp[cj + i - j] = v * rdj;
    }
    __syncthreads();
    for (int kk = j + 1 + warp; kk < s; kk += nw) {
      const int ck = pk(kk, kk, s);
      const T uk = u[kk];
      for (int i = kk + lane; i < s; i += 32) {
        const T x = Tp[ck + i - kk] - Tp[cj + i - j] * uk;
        Tp[ck + i - kk] = x;
        if (i == j + 1 && kk == j + 1) rd[0] = Sc<T>::one() / x;
      }
    }
    __syncthreads();
  }
  T* Vg = Linv + b * sz.linv + m.linv;
  if constexpr (Sc<T>::P == 1) {
    // real: V packed in shared memory after S, then written out with its zeros
    T* Vs = S + fd_scratch(s);
    unit_lower_inverse_blocked(Tp, s, VPacked<T>{Vs, s}, S);
    for (int j = warp; j < s; j += nw)
      for (int i = lane; i < s; i += 32) Vg[i + (int64_t)j * s] = i < j ? Sc<T>::zero() : Vs[pk(i, j, s)];
  } else {
    unit_lower_inverse_blocked(Tp, s, VGlobal<T>{Vg, s}, S);
  }
  for (int j = warp; j < s; j += nw) {
    const int cb = pk(j, j, s);
    for (int i = j + lane; i < s; i += 32) P[i + (int64_t)j * ld] = Tp[cb + i - j];
  }
  for (int j = t; j < s; j += nt) D[b * sz.n + m.f + j] = Tp[pk(j, j, s)];
}

// Factorisation of a non-symmetric diagonal block, one CTA per supernode of
// the level: A_KK = L_KK D_K U'_KK by pivot-free Gaussian elimination in
// shared memory on two packed triangles, Tl (lower part and diagonal, from
// the L panel) and Tu (Tu(i, j) = A_ji for i > j, from the U panel).  For
// column j: d = Tl(j, j); L_ij = Tl(i, j) / d and U'_ji = Tu(i, j) / d; then
// A_ik -= L_ij d U'_jk for i, k > j, on whichever triangle holds (i, k).
// Back to the panels (L_KK with D on the diagonal, U'_KK^T), D, and the unit
// lower inverses (L_KK)^{-1} -> linv, (U'_KK^T)^{-1} -> uinv.  On symmetric
// input every operation matches k_factor_diag's.
template <class T>
__global__ void k_factor_diag_lu(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns, T* __restrict__ L,
                                 T* __restrict__ U, T* __restrict__ D, T* __restrict__ Linv, T* __restrict__ Uinv,
                                 Sizes sz, int* status) {
  extern __shared__ __align__(16) unsigned char shraw[];
  const int k = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, ld = m.s + m.r;
  T* Tl = reinterpret_cast<T*>(shraw);
  T* Tu = Tl + s * (s + 1) / 2;
  T* P = L + b * sz.panel + m.panel;
  T* Q = U + b * sz.panel + m.panel;
  const int nt = blockDim.x, t = threadIdx.x;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i >= j) {
      Tl[pk(i, j, s)] = P[i + (int64_t)j * ld];
      Tu[pk(i, j, s)] = i > j ? Q[i + (int64_t)j * ld] : Sc<T>::zero();
    }
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    const T d = Tl[pk(j, j, s)];
    if (t == 0 && Sc<T>::bad(d)) report_pivot(status, m.f + j, Sc<T>::is_zero(d));
    for (int i = j + 1 + t; i < s; i += nt) {
      Tl[pk(i, j, s)] = Tl[pk(i, j, s)] / d;
      Tu[pk(i, j, s)] = Tu[pk(i, j, s)] / d;
    }
    __syncthreads();
    // trailing block, one warp per column kk (no integer division)
    for (int kk = j + 1 + (t >> 5); kk < s; kk += nt >> 5) {
      const int ck = pk(kk, kk, s);
      for (int ii = kk + (t & 31); ii < s; ii += 32) {
        Tl[ck + ii - kk] -= Tl[pk(ii, j, s)] * Tu[pk(kk, j, s)] * d;                      // A_{ii,kk}
        if (ii > kk) Tu[ck + ii - kk] -= Tu[pk(ii, j, s)] * Tl[pk(kk, j, s)] * d;         // A_{kk,ii}
      }
    }
    __syncthreads();
  }
  if constexpr (Sc<T>::P == 1) {  // real: the blocked inverses (their 16 x 16 scratch after the triangles)
    T* S = Tu + s * (s + 1) / 2;
    unit_lower_inverse_blocked(Tl, s, VGlobal<T>{Linv + b * sz.linv + m.linv, s}, S);
    __syncthreads();
    unit_lower_inverse_blocked(Tu, s, VGlobal<T>{Uinv + b * sz.linv + m.linv, s}, S);
  } else {  // complex: both triangles fill the shared memory
    unit_lower_inverse(Tl, s, Linv + b * sz.linv + m.linv);
    unit_lower_inverse(Tu, s, Uinv + b * sz.linv + m.linv);
  }
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i >= j) P[i + (int64_t)j * ld] = Tl[pk(i, j, s)];
    if (i > j) Q[i + (int64_t)j * ld] = Tu[pk(i, j, s)];
  }
  for (int j = t; j < s; j += nt) D[b * sz.n + m.f + j] = Tl[pk(j, j, s)];
}

// Normalisation of a non-symmetric diagonal block (all supernodes, one CTA
// each): Vl = (L_KK)^{-1} -> linv, Vu = (U'_KK^T)^{-1} -> uinv, and the
// first term of step 3, U_KK^{-1} L_KK^{-1} = U'_KK^{-1} D_K^{-1} L_KK^{-1}
// = Vu^T D_K^{-1} Vl, to the full diagonal block of the X panel.
template <class T>
__global__ void k_norm_diag_lu(const SnMeta* __restrict__ meta, const T* __restrict__ L, const T* __restrict__ U,
                               const T* __restrict__ D, T* __restrict__ Linv, T* __restrict__ Uinv,
                               T* __restrict__ X, Sizes sz) {
  extern __shared__ __align__(16) unsigned char shraw[];
  T* Tp = reinterpret_cast<T*>(shraw);
  const int k = blockIdx.x;
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, ld = m.s + m.r;
  const T* d = D + b * sz.n + m.f;
  T* rd = Tp + s * (s + 1) / 2;
  const int nt = blockDim.x, t = threadIdx.x;
  T* Vl = Linv + b * sz.linv + m.linv;
  T* Vu = Uinv + b * sz.linv + m.linv;
  for (int side = 0; side < 2; ++side) {
    const T* P = (side == 0 ? L : U) + b * sz.panel + m.panel;
    for (int e = t; e < s * s; e += nt) {
      const int i = e % s, j = e / s;
      if (i > j) Tp[pk(i, j, s)] = P[i + (int64_t)j * ld];
    }
    __syncthreads();
    unit_lower_inverse(Tp, s, side == 0 ? Vl : Vu);
    __syncthreads();
  }
  for (int q = t; q < s; q += nt) rd[q] = Sc<T>::one() / d[q];
  __syncthreads();
  T* XK = X + b * sz.panel + m.panel;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    T acc = Sc<T>::zero();
    for (int q = i > j ? i : j; q < s; ++q) acc += Vu[q + i * s] * rd[q] * Vl[q + j * s];
    XK[i + (int64_t)j * ld] = acc;
  }
}

// Normalisation, diagonal part (all supernodes, one CTA each):
// (L_KK)^{-1} -> linv and M_K = L_KK^{-T} D_K^{-1} L_KK^{-1} -> the diagonal
// block of the X panel (Algorithm 1 step 3's first term; U_KK = D_K L_KK^T).
// A pivoted factor (ptype set): D_K has 2x2 blocks, so row q of D_K^{-1} V is
// c_q V_q + c'_q V_{q'} with q' the 2x2 partner, and M_K goes to the original
// columns (P(i), P(j)).
template <class T>
__global__ void k_norm_diag(const SnMeta* __restrict__ meta, const T* __restrict__ L, const T* __restrict__ D,
                            T* __restrict__ Linv, T* __restrict__ X, Sizes sz, const int32_t* __restrict__ piv,
                            const int8_t* __restrict__ ptype, const T* __restrict__ E) {
  extern __shared__ __align__(16) unsigned char shraw[];
  T* Tp = reinterpret_cast<T*>(shraw);
  const int k = blockIdx.x;
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, ld = m.s + m.r;
  const T* P = L + b * sz.panel + m.panel;
  const T* d = D + b * sz.n + m.f;
  T* rd = Tp + s * (s + 1) / 2;  // 1 / d_q, or the own coefficient of a 2x2 row
  T* rp = rd + s;                // partner coefficient (0 for a 1x1 pivot)
  int* pq = reinterpret_cast<int*>(rp + s);
  const int nt = blockDim.x, t = threadIdx.x;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i > j) Tp[pk(i, j, s)] = P[i + (int64_t)j * ld];
  }
  if (ptype) {
    const int8_t* ty = ptype + b * sz.n + m.f;
    const T* ee = E + b * sz.n + m.f;
    for (int q = t; q < s; q += nt) {
      if (ty[q] == 0) {
        rd[q] = Sc<T>::one() / d[q];
        rp[q] = Sc<T>::zero();
        pq[q] = q;
      } else {
        const int f0 = ty[q] == 1 ? q : q - 1;  // first column of the 2x2 block
        const T det = d[f0] * d[f0 + 1] - ee[f0] * ee[f0];
        const int o = ty[q] == 1 ? q + 1 : q - 1;
        rd[q] = d[o] / det;
        rp[q] = -ee[f0] / det;
        pq[q] = o;
      }
    }
  } else {
    for (int q = t; q < s; q += nt) rd[q] = Sc<T>::one() / d[q];
  }
  __syncthreads();
  T* V = Linv + b * sz.linv + m.linv;
  unit_lower_inverse(Tp, s, V);
  if (!X) return;  // inverse only (the adjoint recomputes it)
  __syncthreads();
  T* XK = X + b * sz.panel + m.panel;
  if (ptype) {
    const int32_t* pv = piv + b * sz.n + m.f;
    for (int e = t; e < s * s; e += nt) {
      const int i = e % s, j = e / s;
      if (i >= j) {
        T acc = Sc<T>::zero();
        for (int q = i; q < s; ++q)  // V_qi = 0 for q < i; row q of D^{-1} V vanishes in column j <= i below j - 1
          acc += V[q + i * s] * (rd[q] * V[q + j * s] + rp[q] * V[pq[q] + j * s]);
        XK[pv[i] + (int64_t)pv[j] * ld] = acc;
        XK[pv[j] + (int64_t)pv[i] * ld] = acc;
      }
    }
    return;
  }
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i >= j) {
      T acc = Sc<T>::zero();
      for (int q = i; q < s; ++q) acc += V[q + i * s] * rd[q] * V[q + j * s];
      XK[i + (int64_t)j * ld] = acc;
      XK[j + (int64_t)i * ld] = acc;
    }
  }
}

// |re| + |im|: the magnitude Bunch-Kaufman compares (plain |x| for real)
__device__ __forceinline__ double bk_abs(double x) { return fabs(x); }
__device__ __forceinline__ double bk_abs(Cplx x) { return fabs(x.re) + fabs(x.im); }

// Largest magnitude (first index on ties) over warp lanes; returns it to all lanes.
__device__ __forceinline__ void warp_argmax(double& v, int& idx) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (v2 > v || (v2 == v && i2 < idx)) {
      v = v2;
      idx = i2;
    }
  }
}

// Factorisation with Bunch-Kaufman pivoting restricted to the supernode's
// diagonal block (Bunch and Kaufman 1977, the lower form of LAPACK's
// xSYTF2), one CTA per supernode of the level, the block packed in shared
// memory.  For pivot position k of the reduced block: a = |T_kk|, colmax =
// max_{i>k} |T_ik| at imax; a >= alpha colmax -> 1x1; else with rowmax the
// largest off-diagonal magnitude of row/column imax: a rowmax >= alpha
// colmax^2 -> 1x1; |T_imax,imax| >= alpha rowmax -> 1x1 after swapping k
// and imax; else 2x2 on (k, k+1) after swapping k+1 and imax.  Swaps are
// symmetric interchanges of the whole block, including the computed L rows.
// Out: L_KK (pivot order, zero beside 2x2 blocks) and D to the panel's
// diagonal block, D, E (2x2 off-diagonals), pivot types, the local pivot
// order piv, (L_KK)^{-1} to linv.  A reduced column that is entirely zero, a
// singular 2x2 block or a non-finite value is reported in the status words.
template <class T>
__global__ void k_factor_diag_bk(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns, T* __restrict__ L,
                                 T* __restrict__ D, T* __restrict__ E, int8_t* __restrict__ ptype,
                                 int32_t* __restrict__ piv, T* __restrict__ Linv, Sizes sz, int* status) {
  extern __shared__ __align__(16) unsigned char shraw[];
  T* Tp = reinterpret_cast<T*>(shraw);
  const int k0 = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k0];
  const int s = m.s, ld = m.s + m.r;
  T* l1 = Tp + s * (s + 1) / 2;  // 2x2 step: new L columns
  T* l2 = l1 + s;
  int* perm = reinterpret_cast<int*>(l2 + s);
  __shared__ int sh_kp, sh_kstep, sh_bad;
  T* P = L + b * sz.panel + m.panel;
  const int nt = blockDim.x, t = threadIdx.x;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i >= j) Tp[pk(i, j, s)] = P[i + (int64_t)j * ld];
  }
  for (int q = t; q < s; q += nt) perm[q] = q;
  if (t == 0) sh_bad = 0;
  __syncthreads();
  T* dd = D + b * sz.n + m.f;
  T* ee = E + b * sz.n + m.f;
  int8_t* ty = ptype + b * sz.n + m.f;
  int k = 0;
  while (k < s) {
    // pivot search by warp 0
    if (t < 32) {
      double cv = -1.0;
      int ci = s;
      for (int i = k + 1 + t; i < s; i += 32) {
        const double v = bk_abs(Tp[pk(i, k, s)]);
        if (v > cv || (v == cv && i < ci)) {
          cv = v;
          ci = i;
        }
      }
      warp_argmax(cv, ci);
      const double absakk = bk_abs(Tp[pk(k, k, s)]);
      const double colmax = ci < s ? cv : 0.0;
      const int imax = ci < s ? ci : k;
      double rowmax = 0.0;
      if (absakk < alpha * colmax) {
        double rv = 0.0;
        for (int j = k + t; j < s; j += 32)
          if (j != imax) rv = fmax(rv, bk_abs(j < imax ? Tp[pk(imax, j, s)] : Tp[pk(j, imax, s)]));
        for (int o = 16; o > 0; o >>= 1) rv = fmax(rv, __shfl_xor_sync(0xffffffffu, rv, o));
        rowmax = rv;
      }
      if (t == 0) {
        int kp = k, kstep = 1;
        if (!(absakk == absakk) || !(colmax == colmax) || isinf(absakk) || isinf(colmax)) {
          sh_bad = 2;
        } else if (absakk == 0.0 && colmax == 0.0) {
          sh_bad = 1;
        } else if (absakk < alpha * colmax) {
          if (absakk * rowmax >= alpha * colmax * colmax) {
            kp = k;
          } else if (bk_abs(Tp[pk(imax, imax, s)]) >= alpha * rowmax) {
            kp = imax;
          } else {
            kp = imax;
            kstep = 2;
          }
        }
        sh_kp = kp;
        sh_kstep = kstep;
      }
    }
    __syncthreads();
    if (sh_bad) break;
    const int kstep = sh_kstep, kp = sh_kp, kk = k + kstep - 1;
    if (kp != kk) {  // symmetric interchange of kk and kp (kp > kk) in packed lower storage
      for (int j = t; j < kk; j += nt) {
        const T x = Tp[pk(kk, j, s)];
        Tp[pk(kk, j, s)] = Tp[pk(kp, j, s)];
        Tp[pk(kp, j, s)] = x;
      }
      for (int i = kk + 1 + t; i < kp; i += nt) {
        const T x = Tp[pk(i, kk, s)];
        Tp[pk(i, kk, s)] = Tp[pk(kp, i, s)];
        Tp[pk(kp, i, s)] = x;
      }
      for (int i = kp + 1 + t; i < s; i += nt) {
        const T x = Tp[pk(i, kk, s)];
        Tp[pk(i, kk, s)] = Tp[pk(i, kp, s)];
        Tp[pk(i, kp, s)] = x;
      }
      if (t == 0) {
        const T x = Tp[pk(kk, kk, s)];
        Tp[pk(kk, kk, s)] = Tp[pk(kp, kp, s)];
        Tp[pk(kp, kp, s)] = x;
        const int p = perm[kk];
        perm[kk] = perm[kp];
        perm[kp] = p;
      }
      __syncthreads();
    }
    if (kstep == 1) {
      const T d = Tp[pk(k, k, s)];
      for (int i = k + 1 + t; i < s; i += nt) Tp[pk(i, k, s)] = Tp[pk(i, k, s)] / d;
      __syncthreads();
      // trailing lower triangle, one warp per column (no integer division)
      for (int jj = k + 1 + (t >> 5); jj < s; jj += nt >> 5) {
        const int cj = pk(jj, jj, s);
        for (int ii = jj + (t & 31); ii < s; ii += 32) Tp[cj + ii - jj] -= Tp[pk(ii, k, s)] * Tp[pk(jj, k, s)] * d;
      }
      if (t == 0) {
        dd[k] = d;
        ee[k] = Sc<T>::zero();
        ty[k] = 0;
      }
    } else {
      const T a11 = Tp[pk(k, k, s)], a21 = Tp[pk(k + 1, k, s)], a22 = Tp[pk(k + 1, k + 1, s)];
      const T det = a11 * a22 - a21 * a21;
      if (t == 0 && Sc<T>::bad(det)) sh_bad = Sc<T>::is_zero(det) ? 1 : 2;
      for (int i = k + 2 + t; i < s; i += nt) {  // [l1 l2] = [w1 w2] D^{-1}
        const T w1 = Tp[pk(i, k, s)], w2 = Tp[pk(i, k + 1, s)];
        l1[i] = (w1 * a22 - w2 * a21) / det;
        l2[i] = (w2 * a11 - w1 * a21) / det;
      }
      __syncthreads();
      for (int jj = k + 2 + (t >> 5); jj < s; jj += nt >> 5) {
        const int cj = pk(jj, jj, s);
        for (int ii = jj + (t & 31); ii < s; ii += 32)
          Tp[cj + ii - jj] -= l1[ii] * Tp[pk(jj, k, s)] + l2[ii] * Tp[pk(jj, k + 1, s)];
      }
      __syncthreads();
      for (int i = k + 2 + t; i < s; i += nt) {
        Tp[pk(i, k, s)] = l1[i];
        Tp[pk(i, k + 1, s)] = l2[i];
      }
      if (t == 0) {
        Tp[pk(k + 1, k, s)] = Sc<T>::zero();
        dd[k] = a11;
        dd[k + 1] = a22;
        ee[k] = a21;
        ee[k + 1] = Sc<T>::zero();
        ty[k] = 1;
        ty[k + 1] = 2;
      }
    }
    __syncthreads();
    if (sh_bad) break;
    k += kstep;
  }
  if (sh_bad) {
    if (t == 0) report_pivot(status, m.f + k, sh_bad == 1);
    return;
  }
  unit_lower_inverse_blocked(Tp, s, VGlobal<T>{Linv + b * sz.linv + m.linv, s}, reinterpret_cast<T*>(perm + ((s + 3) & ~3)));
  for (int e = t; e < s * s; e += nt) {
    const int i = e % s, j = e / s;
    if (i > j) P[i + (int64_t)j * ld] = Tp[pk(i, j, s)];
    if (i == j) P[i + (int64_t)j * ld] = dd[i];
  }
  for (int q = t; q < s; q += nt) piv[b * sz.n + m.f + q] = perm[q];
}

// Pivoted factor: L_{C,K} = Z D_K^{-1} for the panel-solve output Z =
// A_{C,K P} L_KK^{-T} held in the factor scratch, with 2x2 blocks of D_K;
// written to the panel and back into the scratch (the Schur update reads it).
template <class T>
__global__ void k_copyback_bk(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns, T* __restrict__ L,
                              T* __restrict__ Ltmp, const T* __restrict__ D, const T* __restrict__ E,
                              const int8_t* __restrict__ ptype, Sizes sz) {
  const int k = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, r = m.r, ld = s + r;
  T* P = L + b * sz.panel + m.panel + s;
  T* Z = Ltmp + b * sz.lhat + m.lhat;
  const T* d = D + b * sz.n + m.f;
  const T* e = E + b * sz.n + m.f;
  const int8_t* ty = ptype + b * sz.n + m.f;
  for (int j = blockIdx.z; j < s; j += gridDim.z) {
    if (ty[j] == 2) continue;  // done with its partner
    if (ty[j] == 0) {
      for (int i = threadIdx.x; i < r; i += blockDim.x) {
        const T l = Z[i + (int64_t)j * r] / d[j];
        Z[i + (int64_t)j * r] = l;
        P[i + (int64_t)j * ld] = l;
      }
    } else {
      const T det = d[j] * d[j + 1] - e[j] * e[j];
      for (int i = threadIdx.x; i < r; i += blockDim.x) {
        const T z1 = Z[i + (int64_t)j * r], z2 = Z[i + (int64_t)(j + 1) * r];
        const T x1 = (z1 * d[j + 1] - z2 * e[j]) / det, x2 = (z2 * d[j] - z1 * e[j]) / det;
        Z[i + (int64_t)j * r] = x1;
        Z[i + (int64_t)(j + 1) * r] = x2;
        P[i + (int64_t)j * ld] = x1;
        P[i + (int64_t)(j + 1) * ld] = x2;
      }
    }
  }
}

// Pole sum in the write step (Section 4.4's expansion Gamma = sum_b w_b X_b,
// batch members b = poles): the finish is the last write of every panel
// entry (X_{C,K} is final since step 2, X_KK once the finish's CTAs have
// run), so after CTA `part` of supernode k has finished member b it counts
// itself on the counter of (k, part); the one that completes the batch forms
// Gamma over the entries this part owns (its X_KK pairs, both triangles, and
// a 1/nparts share of X_{C,K}), summing the members in order b = 0, 1, ...:
// no atomics on values, every Gamma entry written once, the same arithmetic
// as the separate pass (k_pole_sum).  Pivot-free symmetric factors only.
template <class T>
__device__ void pole_share(const KArgs& a, int k, int part, int nparts) {
  const Sizes& sz = a.sz;
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int* ctr = a.gctr + (int64_t)k * nparts + part;
    last = atomicAdd(ctr, 1) == sz.batch - 1;
    if (last) *ctr = 0;
    __threadfence();
  }
  __syncthreads();
  if (!last) return;
  const SnMeta m = a.meta[k];
  const int s = m.s, r = m.r, ld = s + r;
  const T* w = (const T*)a.gw;
  const T* X = (const T*)a.X + m.panel;
  T* G = (T*)a.gam + m.panel;
  auto gsum = [&](int64_t idx) {
    T acc = Sc<T>::zero();
    for (int q = 0; q < sz.batch; ++q) acc += w[q] * ld_cg(X + q * sz.panel + idx);
    G[idx] = acc;
  };
  for (int e = threadIdx.x + part * blockDim.x; e < s * s; e += nparts * blockDim.x) {
    const int i = e % s, j = e / s;
    if (i < j) continue;
    gsum(i + (int64_t)j * ld);
    if (i != j) gsum(j + (int64_t)i * ld);
  }
  const int64_t rs = (int64_t)r * s;
  for (int64_t q = threadIdx.x + (int64_t)part * blockDim.x; q < rs; q += (int64_t)nparts * blockDim.x)
    gsum(s + q % r + (q / r) * ld);
}

template <class T>
__global__ void k_diag_final(KArgs a, const int32_t* __restrict__ sns) {
  step3_finish<T>(a, sns[blockIdx.x], blockIdx.y, blockIdx.z, gridDim.z, false);
  if (a.gam) pole_share<T>(a, sns[blockIdx.x], blockIdx.z, gridDim.z);
}

// Copy the factor scratch back into the panels of the level's supernodes
// (blockIdx.z strides over the columns; threads run down a column).
template <class T>
__global__ void k_copyback(const SnMeta* __restrict__ meta, const int32_t* __restrict__ sns, T* __restrict__ L,
                           const T* __restrict__ Ltmp, Sizes sz) {
  const int k = sns[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[k];
  const int s = m.s, r = m.r, ld = s + r;
  T* P = L + b * sz.panel + m.panel + s;
  const T* src = Ltmp + b * sz.lhat + m.lhat;
  for (int j = blockIdx.z; j < s; j += gridDim.z)
    for (int i = threadIdx.x; i < r; i += blockDim.x) P[i + (int64_t)j * ld] = src[i + (int64_t)j * r];
}

// --------------------------------------------------------------------------
// tile GEMMs
// --------------------------------------------------------------------------

// Factorisation panel solve: Ltmp_{C,K} = A_{C,K} (L_KK)^{-T} D_K^{-1}, and,
// when W is set, W_{C,K} = A_{C,K} (L_KK)^{-T} itself (the Schur update's
// L_{C,K} D_K without a product per operand element; KArgs::W).
// Pivoted factor (piv set): the columns of A_{C,K} are read in pivot order
// and D^{-1} is left to k_copyback_bk (2x2 blocks can straddle tiles).
template <class T, int BN>
__global__ void __launch_bounds__(TG_THREADS, (tile_min_ctas<T, BN>())) k_trsm(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                     const T* __restrict__ L, const T* __restrict__ D,
                                                     const T* __restrict__ Linv, T* __restrict__ Ltmp, Sizes sz,
                                                     const int32_t* __restrict__ piv, T* __restrict__ W) {
  __shared__ TileSmem<T, BN> sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const T* A = L + b * sz.panel + m.panel + s;
  const T* Vi = Linv + b * sz.linv + m.linv;
  const T* d = D + b * sz.n + m.f;
  Acc<T, BN> acc;
  acc_zero<T, BN>(acc);
  const int32_t* pv = piv ? piv + b * sz.n + m.f : nullptr;
  auto la = [&](int mm, int kk) {
    const int row = tk.m0 + mm;
    return row < r ? A[row + (int64_t)(pv ? pv[kk] : kk) * ld] : Sc<T>::zero();
  };
  auto lb = [&](int kk, int nn) {
    const int col = tk.n0 + nn;
    return col < s ? Vi[col + kk * s] : Sc<T>::zero();
  };
  // (L_KK)^{-T} is upper triangular: output columns < n0 + BN need only k < n0 + BN
  tile_mma<T, BN>(sm, 0, min(s, tk.n0 + BN), [](int) { return false; }, la, lb, acc,
                  LiveRect{r - tk.m0, s - tk.n0}, KUpperB<BN>{tk.n0});
  T* out = Ltmp + b * sz.lhat + m.lhat;
  T* wout = W ? W + b * sz.panel + m.panel : nullptr;
  tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
    const int row = tk.m0 + mm, col = tk.n0 + nn;
    if (row < r && col < s) {
      out[row + (int64_t)col * r] = pv ? v : v / d[col];
      if (wout) wout[row + (int64_t)col * r] = v;
    }
  });
}

// Schur-complement update of the ancestors: lower tiles of
// U = L_{C,K} D_K L_{C,K}^T; U[i][k] (i >= k) is subtracted from the ancestor
// entry found through the column descriptor of k and the relative index of i.
// Task.c is the tile's column end (a tile covers columns [n0, c) of C).
// The task list of one launch is a group of supernodes whose C are disjoint
// (analysis), and inside one supernode the targets of different (i, k) are
// different entries, so each target is read-modified-written by exactly one
// thread of the launch: no atomics, and a fixed order of the updates.
// Non-symmetric factor: Ltmp2 is the second operand (U'_{K,C}^T), giving
// L_{C,K} D_K U'_{K,C} into the L panels and, called again with the operands
// swapped and `strict`, (U'_{K,C}^T D_K L_{C,K}^T) below the diagonal into the
// U panels.  W set: the first operand is W_{C,K} = L_{C,K} D_K (or
// U'_{K,C}^T D_K; pivoted: with D's 2 x 2 blocks) as the panel solve left it, so the loads carry no
// FP64 product (a product per A element is 64 x 16 FP64 operations per
// k-tile, 1/8 of the MMA work of a 64 x 8 tile on the same pipe).
template <class T, int BN>
__global__ void __launch_bounds__(TG_THREADS, (tile_min_ctas<T, BN>())) k_schur(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                      const ColDesc* __restrict__ desc,
                                                      const int32_t* __restrict__ relidx, T* __restrict__ L,
                                                      const T* __restrict__ D, const T* __restrict__ Ltmp,
                                                      const T* __restrict__ Ltmp2, int strict, Sizes sz,
                                                      const int8_t* __restrict__ ptype, const T* __restrict__ E,
                                                      const T* __restrict__ W) {
  __shared__ TileSmem<T, BN> sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r;
  const T* Lc = Ltmp + b * sz.lhat + m.lhat;
  const T* Lc2 = Ltmp2 + b * sz.lhat + m.lhat;
  const T* d = D + b * sz.n + m.f;
  Acc<T, BN> acc;
  acc_zero<T, BN>(acc);
  const int8_t* ty = ptype ? ptype + b * sz.n + m.f : nullptr;
  const T* ee = ptype ? E + b * sz.n + m.f : nullptr;
  const T* Wc = W ? W + b * sz.panel + m.panel : nullptr;
  auto la = [&](int mm, int kk) {
    const int row = tk.m0 + mm;
    if (row >= r) return Sc<T>::zero();
    if (Wc) return Wc[row + (int64_t)kk * r];
    T v = Lc[row + (int64_t)kk * r] * d[kk];
    if (ty && ty[kk] == 1) v += Lc[row + (int64_t)(kk + 1) * r] * ee[kk];       // (L D) with a 2x2 block
    if (ty && ty[kk] == 2) v += Lc[row + (int64_t)(kk - 1) * r] * ee[kk - 1];
    return v;
  };
  auto lb = [&](int kk, int nn) {
    const int col = tk.n0 + nn;
    return col < tk.c ? Lc2[col + (int64_t)kk * r] : Sc<T>::zero();
  };
  // live: fragments with a row and a column inside C and an entry on or below the diagonal
  const int dm = tk.m0 - tk.n0;
  tile_mma<T, BN>(sm, 0, s, [](int) { return false; }, la, lb, acc, [&](int r0, int c0) {
    return tk.m0 + r0 < r && tk.n0 + c0 < tk.c && c0 <= dm + r0 + 7;
  });
  T* Lb = L + b * sz.panel;
  const ColDesc* dk = desc + m.desc;
  tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
    const int i = tk.m0 + mm, kc = tk.n0 + nn;
    if (i < r && kc < tk.c && kc + strict <= i) {
      const ColDesc cd = dk[kc];
      T* dst = &Lb[cd.col + relidx[cd.rel + i]];
      *dst = *dst - v;
    }
  });
}

// Normalisation, off-diagonal part: Lhat_{C,K} = L_{C,K} (L_KK)^{-1}.
template <class T, int BN>
__global__ void __launch_bounds__(TG_THREADS, (tile_min_ctas<T, BN>())) k_lhat(const SnMeta* __restrict__ meta, const Task* __restrict__ tasks,
                                                     const T* __restrict__ L, const T* __restrict__ Linv,
                                                     T* __restrict__ Lhat, Sizes sz) {
  __shared__ TileSmem<T, BN> sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const T* A = L + b * sz.panel + m.panel + s;
  const T* Vi = Linv + b * sz.linv + m.linv;
  Acc<T, BN> acc;
  acc_zero<T, BN>(acc);
  auto la = [&](int mm, int kk) {
    const int row = tk.m0 + mm;
    return row < r ? A[row + (int64_t)kk * ld] : Sc<T>::zero();
  };
  auto lb = [&](int kk, int nn) {
    const int col = tk.n0 + nn;
    return col < s ? Vi[kk + col * s] : Sc<T>::zero();
  };
  // (L_KK)^{-1} is lower triangular: output columns >= n0 need only k >= n0
  tile_mma<T, BN>(sm, tk.n0, s, [](int) { return false; }, la, lb, acc, LiveRect{r - tk.m0, s - tk.n0},
                  KLowerB<BN>{tk.n0});
  T* out = Lhat + b * sz.lhat + m.lhat;
  tile_epilogue<T, BN>(acc, [&](int mm, int nn, T v) {
    const int row = tk.m0 + mm, col = tk.n0 + nn;
    if (row < r && col < s) out[row + (int64_t)col * r] = v;
  });
}

// Steps 2 and 3 as grouped per-level kernels (bodies in selinv_steps.cuh).
template <class T, int BN, bool UNSYM>
__global__ void __launch_bounds__(TG_THREADS, (tile_min_ctas<T, BN>())) k_gemm1(KArgs a, const Task* __restrict__ tasks) {
  __shared__ TileSmem<T, BN> sm;
  step2_tile<T, BN, UNSYM>(a, tasks[blockIdx.x], blockIdx.y, sm);
}

// blockIdx.z strides over the columns of the split supernodes of the level
template <class T>
__global__ void k_gemm1_reduce(KArgs a, const int32_t* __restrict__ sns) {
  step2_reduce<T>(a, sns[blockIdx.x], blockIdx.y, blockIdx.z, gridDim.z, false);
}

template <class T, int BN>
__global__ void __launch_bounds__(TG_THREADS, (tile_min_ctas<T, BN>())) k_gemm2(KArgs a, const Task* __restrict__ tasks) {
  __shared__ TileSmem<T, BN> sm;
  step3_tile<T, BN>(a, tasks[blockIdx.x], blockIdx.y, sm, false);
}

// --------------------------------------------------------------------------
// log det
// --------------------------------------------------------------------------

// Real: (sum log|d_j|, number of negative pivots); complex: sum of principal
// logs (log|d_j|, arg d_j), per batch member.
template <class T>
__global__ void k_logdet(const T* __restrict__ D, int64_t n, double* __restrict__ out,
                         const int8_t* __restrict__ ptype, const T* __restrict__ E) {
  __shared__ double s1[256];
  __shared__ double s2[256];
  const int b = blockIdx.x;
  double a = 0.0, c = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const int8_t ty = ptype ? ptype[b * n + j] : 0;
    if (ty == 2) continue;  // counted with its partner
    // a 2x2 pivot contributes the determinant of its block
    const T d = ty == 1 ? D[b * n + j] * D[b * n + j + 1] - E[b * n + j] * E[b * n + j] : D[b * n + j];
    if constexpr (Sc<T>::P == 1) {
      a += log(fabs(d));
      c += d < 0.0 ? 1.0 : 0.0;
    } else {
      a += log(hypot(d.re, d.im));
      c += atan2(d.im, d.re);
    }
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = c;
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
// pole sum and trace pairing
// --------------------------------------------------------------------------

// out[e] = sum_b w_b X_b[e]  (grid-stride, HBM-bound)
template <class T>
__global__ void k_pole_sum(const T* __restrict__ X, int64_t panel_total, int batch, const T* __restrict__ w,
                           T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < panel_total;
       e += (int64_t)gridDim.x * blockDim.x) {
    T acc = Sc<T>::zero();
    for (int b = 0; b < batch; ++b) acc += w[b] * X[(int64_t)b * panel_total + e];
    out[e] = acc;
  }
}

// S_b = sum_q m_q X(q) A_q with m_q = 1 on the diagonal, 2 off it; one CTA
// per batch member, fixed reduction order (deterministic).
template <class T>
__global__ void k_trace_sum(const T* __restrict__ X, int64_t panel_total, const int64_t* __restrict__ vmap,
                            const uint8_t* __restrict__ diagmask, const T* __restrict__ vals, int64_t nnz,
                            T* __restrict__ out) {
  __shared__ T red[1024];
  const int b = blockIdx.x;
  const T* Xb = X + (int64_t)b * panel_total;
  const T* v = vals + (int64_t)b * nnz;
  T acc = Sc<T>::zero();
  for (int64_t q = threadIdx.x; q < nnz; q += blockDim.x) {
    const T t = Xb[vmap[q]] * v[q];
    acc += diagmask[q] ? t : 2.0 * t;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = red[0];
}

cudaError_t launch_pole_sum(int dtype, const void* X, int64_t panel_total, int batch, const void* w, void* out,
                            cudaStream_t st) {
  const unsigned grid = 152 * 8;
  if (dtype == PSELINV_C128)
    k_pole_sum<Cplx><<<grid, 256, 0, st>>>((const Cplx*)X, panel_total, batch, (const Cplx*)w, (Cplx*)out);
  else
    k_pole_sum<double><<<grid, 256, 0, st>>>((const double*)X, panel_total, batch, (const double*)w, (double*)out);
  return cudaGetLastError();
}

cudaError_t launch_trace_sum(int dtype, const void* X, int64_t panel_total, const int64_t* vmap,
                             const uint8_t* diagmask, const void* vals, int64_t nnz, int batch, void* out,
                             cudaStream_t st) {
  if (dtype == PSELINV_C128)
    k_trace_sum<Cplx><<<batch, 1024, 0, st>>>((const Cplx*)X, panel_total, vmap, diagmask, (const Cplx*)vals, nnz,
                                              (Cplx*)out);
  else
    k_trace_sum<double><<<batch, 1024, 0, st>>>((const double*)X, panel_total, vmap, diagmask, (const double*)vals,
                                                nnz, (double*)out);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// launch wrappers
// --------------------------------------------------------------------------

static inline unsigned blocks_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

// packed lower triangle, two length-s vectors and s ints
template <class T>
static size_t diag_smem(int maxw) {
  return sizeof(T) * ((size_t)maxw * (maxw + 1) / 2 + 2 * (size_t)maxw) + sizeof(int) * (size_t)maxw;
}

// the symmetric diagonal factorisation: packed lower triangle, the column u,
// and the 16 x 16 blocks S of the blocked inverse
template <class T>
static size_t diag_smem_fd(int maxw) {
  // packed L_KK, u, S; real: the packed inverse too (complex keeps it in global memory)
  const size_t tri = (size_t)maxw * (maxw + 1) / 2;
  return sizeof(T) * (tri + (size_t)maxw + fd_scratch(maxw) + (Sc<T>::P == 1 ? tri : 0));
}

// the pivoted diagonal factorisation: diag_smem plus the blocks of the inverse
template <class T>
static size_t diag_smem_bk(int maxw) {
  const size_t nb = (size_t)(maxw + 15) / 16;
  return diag_smem<T>(maxw) + 16 + sizeof(T) * 256 * (nb > 1 ? nb - 1 : 1);
}

// two packed triangles of the non-symmetric diagonal factorisation
template <class T>
static size_t diag_smem_lu(int maxw) {
  const size_t nb = (size_t)(maxw + 15) / 16;
  return sizeof(T) * ((size_t)maxw * (maxw + 1) + (Sc<T>::P == 1 ? 256 * (nb > 1 ? nb - 1 : 1) : 0));
}

template <class T>
static cudaError_t setup_t() {
  cudaError_t e = cudaFuncSetAttribute(k_factor_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)diag_smem_fd<T>(kMaxWidth));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_norm_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)diag_smem<T>(kMaxWidth));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_norm_diag_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)diag_smem<T>(kMaxWidth));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_factor_diag_bk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)diag_smem_bk<T>(kMaxWidth));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_factor_diag_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)diag_smem_lu<T>(Sc<T>::P == 1 ? kMaxWidth : kMaxWidthLUComplex));
  return e;
}

cudaError_t setup_kernels() {
  cudaError_t e = setup_t<double>();
  if (e != cudaSuccess) return e;
  if ((e = setup_em_kernels()) != cudaSuccess) return e;
  return setup_t<Cplx>();
}

template <class T>
static cudaError_t scatter_t(const void* vals, const int64_t* vmap, int64_t nnz, void* L, const Sizes& sz,
                             cudaStream_t st) {
  k_scatter_values<T><<<dim3(blocks_for(nnz, 256), sz.batch), 256, 0, st>>>((const T*)vals, vmap, nnz, (T*)L,
                                                                           sz.panel);
  return cudaGetLastError();
}
cudaError_t launch_scatter_values(int dtype, const void* vals, const int64_t* vmap, int64_t nnz, void* L,
                                  const Sizes& sz, cudaStream_t st) {
  return dtype == PSELINV_C128 ? scatter_t<Cplx>(vals, vmap, nnz, L, sz, st)
                               : scatter_t<double>(vals, vmap, nnz, L, sz, st);
}

template <class T>
static cudaError_t scatter_lu_t(const void* lo, const void* up, const int64_t* vmap, const uint8_t* flip, int64_t nnz,
                                void* L, void* U, const Sizes& sz, cudaStream_t st) {
  k_scatter_values_lu<T><<<dim3(blocks_for(nnz, 256), sz.batch), 256, 0, st>>>(
      (const T*)lo, (const T*)up, vmap, flip, nnz, (T*)L, (T*)U, sz.panel);
  return cudaGetLastError();
}
cudaError_t launch_scatter_values_lu(int dtype, const void* lower, const void* upper, const int64_t* vmap,
                                     const uint8_t* flip, int64_t nnz, void* L, void* U, const Sizes& sz,
                                     cudaStream_t st) {
  return dtype == PSELINV_C128 ? scatter_lu_t<Cplx>(lower, upper, vmap, flip, nnz, L, U, sz, st)
                               : scatter_lu_t<double>(lower, upper, vmap, flip, nnz, L, U, sz, st);
}

template <class T>
static cudaError_t gather_lu_t(const void* XL, const void* XU, const int64_t* vmap, const uint8_t* flip, int64_t nnz,
                               int upper, void* out, const Sizes& sz, cudaStream_t st) {
  k_gather_values_lu<T><<<dim3(blocks_for(nnz, 256), sz.batch), 256, 0, st>>>(
      (const T*)XL, (const T*)XU, sz.panel, vmap, flip, nnz, upper, (T*)out);
  return cudaGetLastError();
}
cudaError_t launch_gather_values_lu(int dtype, const void* XL, const void* XU, const int64_t* vmap,
                                    const uint8_t* flip, int64_t nnz, int upper, void* out, const Sizes& sz,
                                    cudaStream_t st) {
  return dtype == PSELINV_C128 ? gather_lu_t<Cplx>(XL, XU, vmap, flip, nnz, upper, out, sz, st)
                               : gather_lu_t<double>(XL, XU, vmap, flip, nnz, upper, out, sz, st);
}

template <class T>
static cudaError_t gather_t(const void* X, const int64_t* vmap, const uint8_t* mask, int64_t nnz, void* out,
                            const Sizes& sz, cudaStream_t st) {
  k_gather_values<T><<<dim3(blocks_for(nnz, 256), sz.batch), 256, 0, st>>>((const T*)X, sz.panel, vmap, mask, nnz,
                                                                          (T*)out);
  return cudaGetLastError();
}
cudaError_t launch_gather_values(int dtype, const void* X, const int64_t* vmap, const uint8_t* diagmask, int64_t nnz,
                                 void* out, const Sizes& sz, cudaStream_t st) {
  return dtype == PSELINV_C128 ? gather_t<Cplx>(X, vmap, diagmask, nnz, out, sz, st)
                               : gather_t<double>(X, vmap, diagmask, nnz, out, sz, st);
}

// ---- tile-kernel launch for one task range of one variant ----

template <class T, int BN>
static cudaError_t tiles_tb(Kern k, const KArgs& a, const Task* t, int64_t n, cudaStream_t st) {
  const dim3 grid((unsigned)n, a.sz.batch);
  switch (k) {
    case Kern::Trsm:
      k_trsm<T, BN><<<grid, TG_THREADS, 0, st>>>(a.meta, t, (const T*)a.L, (const T*)a.D, (const T*)a.Linv,
                                                 (T*)a.Lhat, a.sz, a.piv, (T*)a.W);
      break;
    case Kern::Schur:
      k_schur<T, BN><<<grid, TG_THREADS, 0, st>>>(a.meta, t, a.desc, a.relidx, (T*)a.L, (const T*)a.D,
                                                  (const T*)a.Lhat, (const T*)(a.Uhat ? a.Uhat : a.Lhat),
                                                  a.strict, a.sz, a.ptype, (const T*)a.E, (const T*)a.W);
      break;
    case Kern::Lhat:
      k_lhat<T, BN><<<grid, TG_THREADS, 0, st>>>(a.meta, t, (const T*)a.L, (const T*)a.Linv, (T*)a.Lhat, a.sz);
      break;
    case Kern::Gemm1:
      if (a.XU)
        k_gemm1<T, BN, true><<<grid, TG_THREADS, 0, st>>>(a, t);
      else
        k_gemm1<T, BN, false><<<grid, TG_THREADS, 0, st>>>(a, t);
      break;
    default:
      k_gemm2<T, BN><<<grid, TG_THREADS, 0, st>>>(a, t);
      break;
  }
  return cudaGetLastError();
}

template <class T>
static cudaError_t tiles_t(Kern k, int var, const KArgs& a, const Task* t, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  switch (var) {
    case 0: return tiles_tb<T, 8>(k, a, t, n, st);
    case 1: return tiles_tb<T, 16>(k, a, t, n, st);
    case 2: return tiles_tb<T, 32>(k, a, t, n, st);
    default:
      if constexpr (Sc<T>::P == 1) return tiles_tb<T, 64>(k, a, t, n, st);
      return cudaErrorInvalidValue;  // complex tiles stop at BN = 32 (register budget)
  }
}

cudaError_t launch_tiles(Kern k, int var, const KArgs& a, const Task* t, int64_t n, cudaStream_t st) {
  return a.dtype == PSELINV_C128 ? tiles_t<Cplx>(k, var, a, t, n, st) : tiles_t<double>(k, var, a, t, n, st);
}

template <class T>
static cudaError_t per_sn_t(Kern k, const KArgs& a, const int32_t* sns, int nsn, cudaStream_t st, int threads) {
  if (nsn <= 0) return cudaSuccess;
  const dim3 grid(nsn, a.sz.batch);
  switch (k) {
    case Kern::FactorDiag:
      k_factor_diag<T><<<grid, threads, diag_smem_fd<T>(a.maxw), st>>>(a.meta, sns, (T*)a.L, (T*)a.D, (T*)a.Linv,
                                                                    a.sz, a.status);
      break;
    case Kern::CopyBack:
      k_copyback<T><<<dim3(nsn, a.sz.batch, 16), 256, 0, st>>>(a.meta, sns, (T*)a.L, (const T*)a.Lhat, a.sz);
      break;
    case Kern::NormDiag:  // every supernode: blockIdx.x is the supernode itself
      k_norm_diag<T><<<grid, 256, diag_smem<T>(a.maxw), st>>>(a.meta, (const T*)a.L, (const T*)a.D, (T*)a.Linv,
                                                              (T*)a.X, a.sz, a.piv, a.ptype, (const T*)a.E);
      break;
    case Kern::Gemm1Reduce:
      k_gemm1_reduce<T><<<dim3(nsn, a.sz.batch, 16), 256, 0, st>>>(a, sns);
      break;
    case Kern::FactorDiagLU:
      k_factor_diag_lu<T><<<grid, threads, diag_smem_lu<T>(a.maxw), st>>>(a.meta, sns, (T*)a.L, (T*)a.U, (T*)a.D,
                                                                      (T*)a.Linv, (T*)a.Uinv, a.sz, a.status);
      break;
    case Kern::FactorDiagBK:
      k_factor_diag_bk<T><<<grid, threads > 512 ? 512 : threads, diag_smem_bk<T>(a.maxw), st>>>(
          a.meta, sns, (T*)a.L, (T*)a.D, (T*)a.E, (int8_t*)a.ptype, (int32_t*)a.piv, (T*)a.Linv, a.sz, a.status);
      break;
    case Kern::CopyBackBK:
      k_copyback_bk<T><<<dim3(nsn, a.sz.batch, 16), 256, 0, st>>>(a.meta, sns, (T*)a.L, (T*)a.Lhat, (const T*)a.D,
                                                                  (const T*)a.E, a.ptype, a.sz);
      break;
    case Kern::NormDiagLU:
      k_norm_diag_lu<T><<<grid, 256, diag_smem<T>(a.maxw), st>>>(a.meta, (const T*)a.L, (const T*)a.U,
                                                                 (const T*)a.D, (T*)a.Linv, (T*)a.Uinv,
                                                                 (T*)a.X, a.sz);
      break;
    default:
      // 32 CTAs per supernode: the levels near the root hold one supernode whose
      // finish reads one s x s partial per row chunk of C
      k_diag_final<T><<<dim3(nsn, a.sz.batch, kFinishCtas), 256, 0, st>>>(a, sns);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_per_sn(Kern k, const KArgs& a, const int32_t* sns, int nsn, cudaStream_t st, int threads) {
  return a.dtype == PSELINV_C128 ? per_sn_t<Cplx>(k, a, sns, nsn, st, threads)
                                 : per_sn_t<double>(k, a, sns, nsn, st, threads);
}

cudaError_t launch_logdet(int dtype, const void* D, int64_t n, double* out, int batch, cudaStream_t st,
                          const int8_t* ptype, const void* E) {
  if (dtype == PSELINV_C128)
    k_logdet<Cplx><<<batch, 256, 0, st>>>((const Cplx*)D, n, out, ptype, (const Cplx*)E);
  else
    k_logdet<double><<<batch, 256, 0, st>>>((const double*)D, n, out, ptype, (const double*)E);
  return cudaGetLastError();
}

}  // namespace psi
