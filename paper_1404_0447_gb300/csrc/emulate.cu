// Steps 2 and 3 of the selected inversion (X_{C,K} = -X_{C,C} Lhat_{C,K} and
// the partial products Lhat_{C,K}^T X_{C,K}, Algorithm 1) in FP64 accuracy on
// the bf16 tensor cores, for real symmetric positive definite matrices.
//
// Scaling.  For X = A^{-1} SPD, |X_pq| <= sqrt(X_pp X_qq).  With the power of
// two 2^e_p >= sqrt(X_pp), e_p = ceil(E_p / 2) where X_pp < 2^E_p, every entry
// of Xt = 2^-(e_p + e_q) X satisfies |Xt| < 1, and X_{C,C} Lhat =
// diag(2^e_C) Xt_{C,C} B' with B' = diag(2^e_C) Lhat.  Column j of B' gets its
// own exponent F_j (|B'_{:,j}| < 2^F_j).
//
// Slices.  a = Xt and b = B' 2^-F are fixed-point numbers in (-1, 1):
// qa = floor(|a| 2^55), qb = floor(|b| 2^56), cut into 7 bytes from the top,
// a = sum_t a_t 2^(-7-8t), b = sum_u b_u 2^(-8-8u), every slice an integer in
// [-255, 255] carrying the entry's sign, exact in bf16.  The products
// a_t b_u with t + u = g <= 6 (28 of the 49) are formed by mma.sync bf16 with
// FP32 accumulation, one accumulator per g: over a chunk of 32 rows of C a
// group sum is an integer below 7 * 32 * 255^2 < 2^24, so FP32 holds it
// exactly.  After each chunk the seven group sums are folded into two 64-bit
// integers, hi = S0 2^16 + S1 2^8 + S2 and lo = S3 2^24 + S4 2^16 + S5 2^8 + S6,
// and at the end
//   (X_{C,C} Lhat)_{ij} = 2^(e_{C_i} + F_j - 31) (hi + lo 2^-32),
// the only FP64 arithmetic of the product.  The dropped products (g >= 7)
// and the truncation of the slices each contribute below 2^-53 of
// 2^(e_{C_i} + F_j) per term, the order of the FP64 rounding of the same sum.
//
// The slices of a supernode's X panel are cut once, right after its level
// has finished (k_em_split_x), those of its B' right before its step 2
// (k_em_split_lhat, once the exponents of the rows of C are known).  Step 3,
// Lhat^T X_{C,K} = B'^T X'' with X'' = diag(2^-e_C) X_{C,K}, takes B' and the
// slices of X'' over a per-column exponent G_j (k_em_split_xck, right after
// step 2): P_mn = 2^(F_m + G_n - 32) (hi + lo 2^-32), both operands cut at
// 2^56.  Step 2 runs on mma.sync (k_em_gemm1, 64-row tiles), step 3 on
// mma.sync (k_em_gemm2).
#include <cfloat>
#include <climits>
#include <cstdint>

#include "kernels.h"
#include "tile_gemm.cuh"

namespace psi {
namespace {

constexpr int kSl = 7;         // slices per entry
constexpr int kKC = 32;        // rows of C per exact FP32 chunk
constexpr int kEmThreads = 128;

// bf16 bits of the integer c in [0, 255] with sign bit sgn (0 or 0x8000):
// c has at most 8 significant bits, so the low half of float(c) is zero.
__device__ __forceinline__ uint32_t bf16_int(uint32_t c, uint32_t sgn) {
  return c ? (__float_as_uint((float)c) >> 16) | sgn : 0u;
}

// The 7 slices of v as bf16 (slice t in halfword t): q = floor(|v| 2^(56 - E))
// for |v| < 2^E, cut into bytes from the top.  Zero and subnormal v give
// zero slices; Inf, NaN or |v| >= 2^E set bad.
__device__ __forceinline__ uint4 split7(double v, int E, int& bad) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7FF);
  uint4 o = make_uint4(0u, 0u, 0u, 0u);
  if (ex == 0) return o;
  const int sh = ex - 1019 - E;  // |v| 2^(56 - E) = mant 2^sh; |v| < 2^E <=> sh <= 3
  if (ex == 0x7FF || sh > 3) {
    bad = 1;
    return o;
  }
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long q = sh >= 0 ? mant << sh : (sh > -64 ? mant >> (-sh) : 0ull);
  const uint32_t sgn = (uint32_t)(bits >> 63) << 15;
  uint32_t h[kSl];
#pragma unroll
  for (int t = 0; t < kSl; ++t) h[t] = bf16_int((uint32_t)(q >> (8 * (6 - t))) & 255u, sgn);
  o.x = h[0] | (h[1] << 16);
  o.y = h[2] | (h[3] << 16);
  o.z = h[4] | (h[5] << 16);
  o.w = h[6];
  return o;
}

// acc += x * scale (32 x 32 -> 64-bit signed multiply-add, one instruction)
__device__ __forceinline__ void madw(long long& acc, int x, int scale) {
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(x), "r"(scale));
}
// Fold the seven exact FP32 group sums of one entry into hi (groups 0-2) and
// lo (groups 3-6): hi += S0 2^16 + S1 2^8 + S2, lo += S3 2^24 + S4 2^16 + S5 2^8 + S6.
__device__ __forceinline__ void fold7(long long& hi, long long& lo, float s0, float s1, float s2, float s3,
                                      float s4, float s5, float s6) {
  madw(hi, __float2int_rn(s0), 65536);
  madw(hi, __float2int_rn(s1), 256);
  madw(hi, __float2int_rn(s2), 1);
  madw(lo, __float2int_rn(s3), 16777216);
  madw(lo, __float2int_rn(s4), 65536);
  madw(lo, __float2int_rn(s5), 256);
  madw(lo, __float2int_rn(s6), 1);
}

// Column groups of the split kernels: CTA z of a supernode handles its
// columns z, z + kSplitGroups, ... (the top levels hold few, tall supernodes).
constexpr int kSplitGroups = 32;

// After the level of supernode K: e_p of K's columns, then the slices of
// every panel entry of K that step 2 reads (the lower triangle of the
// diagonal block and the rows of C).  Grid (supernodes, batch, column groups);
// every CTA derives the s exponents itself, group 0 stores them.
__global__ void __launch_bounds__(256) k_em_split_x(KArgs a, EmArgs e, const int32_t* __restrict__ sns) {
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const SnMeta m = a.meta[k];
  const int s = m.s, r = m.r, ld = s + r;
  if ((int)blockIdx.z >= s) return;
  const double* X = (const double*)a.X + b * a.sz.panel + m.panel;
  uint4* xs = (uint4*)e.xs + b * a.sz.panel + m.panel;
  int32_t* sig = e.sig + b * e.n;
  const int32_t* crow = e.crow + m.desc;
  __shared__ int se[kMaxWidth];
  int bad = 0;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    const double d = X[j + (int64_t)j * ld];
    int E = 0;
    if (d > 0.0 && d <= DBL_MAX) {
      frexp(d, &E);      // d < 2^E
      E = (E + 1) >> 1;  // ceil(E / 2): 2^e >= sqrt(d)
    } else {
      bad = 1;
    }
    se[j] = E;
    if (blockIdx.z == 0) sig[m.f + j] = E;
  }
  __syncthreads();
  for (int j = blockIdx.z; j < s; j += gridDim.z) {
    const double* col = X + (int64_t)j * ld;
    uint4* out = xs + (int64_t)j * ld;
    const int ej = se[j] + 1;
    for (int p = threadIdx.x; p < ld; p += blockDim.x) {
      if (p < j) {
        out[p] = make_uint4(0u, 0u, 0u, 0u);  // above the diagonal: never read
        continue;
      }
      const int ep = p < s ? se[p] : sig[crow[p - s]];
      out[p] = split7(col[p], ep + ej, bad);  // |X_pq| < 2^(e_p + e_q + 1)
    }
  }
  if (bad) atomicOr(a.status + kEmStatusWord, kEmRange);
}

// Rows of C whose exponents k_em_split_lhat keeps in shared memory at most
// (a launch reserves the largest |C| of its supernodes, capped here; larger
// |C| reads them from global memory).
constexpr int kEcRows = 40960;

// The columns of an r x s block scaled by rows, V = diag(2^(esign e_C)) W,
// cut into slices column by column: exponent E_j with |V_{:,j}| < 2^E_j to
// exps[j], the slices of V_{:,j} 2^-E_j to dst.  Grid (supernodes, batch,
// column groups); a CTA takes the exponents e of the rows of C once, then its
// columns one at a time with all threads (block-wide maximum, then slices).
__device__ __forceinline__ void split_columns(const double* W, int64_t wld, uint4* dst, int64_t dld, int r, int s,
                                              int esign, int32_t* exps, const int32_t* sig, const int32_t* crow,
                                              int ec_cap, int* ec_smem, int* red, int* status) {
  const bool cached = r <= ec_cap;
  if (cached)
    for (int i = threadIdx.x; i < r; i += blockDim.x) ec_smem[i] = esign * sig[crow[i]];
  __syncthreads();
  auto ec = [&](int i) { return cached ? ec_smem[i] : esign * sig[crow[i]]; };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int bad = 0;
  for (int j = blockIdx.z; j < s; j += gridDim.z) {
    const double* col = W + (int64_t)j * wld;
    int mx = INT_MIN;
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(col[i]);
      const int ex = (int)((bits >> 52) & 0x7FF);
      if (ex == 0x7FF)
        bad = 1;
      else if (ex != 0)
        mx = max(mx, ex - 1023 + ec(i));  // floor(log2 |V_ij|)
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
    const int E = mx == INT_MIN ? 0 : mx + 1;
    if (threadIdx.x == 0) exps[j] = E;
    for (int i = threadIdx.x; i < r; i += blockDim.x) dst[i + (int64_t)j * dld] = split7(col[i], E - ec(i), bad);
    __syncthreads();  // red[] is rewritten by the next column
  }
  if (bad) atomicOr(status + kEmStatusWord, kEmRange);
}

// Before step 2 of supernode K: F_j and the slices of B' = diag(2^e_C) Lhat.
__global__ void __launch_bounds__(256) k_em_split_lhat(KArgs a, EmArgs e, const int32_t* __restrict__ sns,
                                                       int ec_cap) {
  extern __shared__ int ec_smem[];
  __shared__ int red[8];
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const SnMeta m = a.meta[k];
  if ((int)blockIdx.z >= m.s) return;
  split_columns((const double*)a.Lhat + b * a.sz.lhat + m.lhat, m.r, (uint4*)e.ls + b * a.sz.lhat + m.lhat, m.r,
                m.r, m.s, 1, e.lexp + b * e.n + m.f, e.sig + b * e.n, e.crow + m.desc, ec_cap, ec_smem, red,
                a.status);
}

// After step 2 of supernode K (before step 3): G_j and the slices of
// X'' = diag(2^-e_C) X_{C,K}, kept in the slice array at the rows of C of
// K's panel until the level's own slices replace them.
__global__ void __launch_bounds__(256) k_em_split_xck(KArgs a, EmArgs e, const int32_t* __restrict__ sns,
                                                      int ec_cap) {
  extern __shared__ int ec_smem[];
  __shared__ int red[8];
  const int k = sns[blockIdx.x], b = blockIdx.y;
  const SnMeta m = a.meta[k];
  if ((int)blockIdx.z >= m.s) return;
  const int64_t ld = m.s + m.r;
  split_columns((const double*)a.X + b * a.sz.panel + m.panel + m.s, ld,
                (uint4*)e.xs + b * a.sz.panel + m.panel + m.s, ld, m.r, m.s, -1, e.gexp + b * e.n + m.f,
                e.sig + b * e.n, e.crow + m.desc, ec_cap, ec_smem, red, a.status);
}

constexpr int kKP = kKC + 8;  // shared row stride of a slice plane in bf16 (80 bytes: ldmatrix rows conflict-free)

// A 64-row tile on mma.sync: the 7 slice planes of the A and B operands of
// one 32-row chunk of C (step 2: X_{C,C} and B'; step 3: B'^T and X''), the
// descriptors of the tile's rows and of the columns of the current and the
// next chunk (step 2 only), and the row / column exponents (step 2: e of the
// rows of C and F; step 3: F and G).
template <int NB>
struct EmSmem {
  uint16_t a[kSl][kTileM][kKP];  // X_{C,C} tile, [slice][m][k]
  uint16_t b[kSl][NB][kKP];      // B' tile, [slice][n][k]
  ColDesc rdesc[kTileM];         // desc of the tile's rows of C
  ColDesc cdesc[2][kKC];         // desc of the columns of chunk c, slot c & 1
  int32_t erow[kTileM];          // exponents of the tile's rows
  int32_t fcol[kTileN];          // exponents of the task's columns
};

__device__ __forceinline__ void ldsm_x4(uint32_t (&d)[4], const void* p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x2(uint32_t& d0, uint32_t& d1, const void* p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(d0), "=r"(d1) : "r"(s));
}
// D(16x8, f32) += A(16x16, bf16, row) B(16x8, bf16, col)
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Slice t of two entries (k, k+1 of one row) as one bf16x2 word.
__device__ __forceinline__ uint32_t pair_slice(const uint4& v0, const uint4& v1, int t) {
  const uint32_t w0 = t < 2 ? v0.x : t < 4 ? v0.y : t < 6 ? v0.z : v0.w;
  const uint32_t w1 = t < 2 ? v1.x : t < 4 ? v1.y : t < 6 ? v1.z : v1.w;
  return __byte_perm(w0, w1, (t & 1) ? 0x7632 : 0x5410);
}
template <int R>
__device__ __forceinline__ void stash_pair(uint16_t (&dst)[kSl][R][kKP], int row, int k, const uint4& v0,
                                           const uint4& v1) {
#pragma unroll
  for (int t = 0; t < kSl; ++t) *reinterpret_cast<uint32_t*>(&dst[t][row][k]) = pair_slice(v0, v1, t);
}

// The 28 slice products of the chunk in the planes (7 group sums per
// fragment entry, exact in FP32), folded into hi / lo.  Warp w takes rows
// 16w..16w+15 of the 64-row tile and all NB columns; accumulator x of
// fragment j is row g + 8 (x >> 1), column 8 j + 2 q + (x & 1).
template <int NB>
__device__ __forceinline__ void em_products(EmSmem<NB>& sm, long long (&hi)[NB / 8][4],
                                            long long (&lo)[NB / 8][4]) {
  constexpr int NF = NB / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float S[kSl][NF][4];
#pragma unroll
  for (int gi = 0; gi < kSl; ++gi)
#pragma unroll
    for (int j = 0; j < NF; ++j)
#pragma unroll
      for (int x = 0; x < 4; ++x) S[gi][j][x] = 0.f;
#pragma unroll
  for (int ks = 0; ks < kKC; ks += 16) {
    uint32_t B[kSl][NF][2];
#pragma unroll
    for (int u = 0; u < kSl; ++u) {
      if constexpr (NF == 2) {
        uint32_t d[4];
        ldsm_x4(d, &sm.b[u][(lane & 7) + ((lane >> 4) << 3)][ks + (((lane >> 3) & 1) << 3)]);
        B[u][0][0] = d[0];
        B[u][0][1] = d[1];
        B[u][1][0] = d[2];
        B[u][1][1] = d[3];
      } else {
        ldsm_x2(B[u][0][0], B[u][0][1], &sm.b[u][lane & 7][ks + (((lane >> 3) & 1) << 3)]);
      }
    }
#pragma unroll
    for (int ta = 0; ta < kSl; ++ta) {
      uint32_t A[4];
      ldsm_x4(A, &sm.a[ta][warp * 16 + (lane & 15)][ks + ((lane >> 4) << 3)]);
#pragma unroll
      for (int u = 0; u + ta < kSl; ++u)
#pragma unroll
        for (int j = 0; j < NF; ++j) mma_bf16(S[ta + u][j], A, B[u][j][0], B[u][j][1]);
    }
  }
#pragma unroll
  for (int j = 0; j < NF; ++j)
#pragma unroll
    for (int x = 0; x < 4; ++x)
      fold7(hi[j][x], lo[j][x], S[0][j][x], S[1][j][x], S[2][j][x], S[3][j][x], S[4][j][x], S[5][j][x],
            S[6][j][x]);
}

// One step-2 task (tile origin m0, n0, width NB in {8, 16}, k-slice c) on
// the slices.  Four warps; warp w owns rows 16w..16w+15 and all NB columns.
//
// Per chunk of 32 rows of C: the 16 entries of X_{C,C} a thread stages are
// fetched together (their relative indices were loaded during the previous
// chunk's products, the row descriptors are cached for the tile and the
// column descriptors one chunk ahead), written to the slice planes as
// 32-bit words holding one slice of two k-adjacent entries, and the 28
// slice products run on ldmatrix fragments.  Pair p of a thread: right of
// the tile's rows (entries above the diagonal of X_{C,C}, read along k) a
// warp covers 2 rows x 32 k, else (rows contiguous in the ancestors'
// panels) 8 rows x 8 k; both maps hit 32 distinct banks (row stride 20 words).
template <int NB>
__global__ void __launch_bounds__(kEmThreads, 3) k_em_gemm1(KArgs a, EmArgs e, const Task* __restrict__ tasks) {
  constexpr int NF = NB / 8;
  __shared__ __align__(16) EmSmem<NB> sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = a.meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const ColDesc* dk = a.desc + m.desc;
  const int32_t* relidx = a.relidx;
  const uint4* xs = (const uint4*)e.xs + b * a.sz.panel;
  const uint4* ls = (const uint4*)e.ls + b * a.sz.lhat + m.lhat;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, q = lane & 3;
  const int m0 = tk.m0, nb = tk.n0;
  const int kb = tk.c * m.kchunk, ke = min(r, kb + m.kchunk);
  const int nck = ke > kb ? (ke - kb + kKC - 1) / kKC : 0;
  if (t < kTileM) {
    const int i = m0 + t;
    sm.erow[t] = i < r ? e.sig[b * e.n + e.crow[m.desc + i]] : 0;
    if (i < r) sm.rdesc[t] = dk[i];
  } else {
    const int c = nb + (t - kTileM);
    sm.fcol[t - kTileM] = c < s ? e.lexp[b * e.n + m.f + c] : 0;
  }
  if (t < kKC && nck > 0 && kb + t < ke) sm.cdesc[0][t] = dk[kb + t];
  __syncthreads();

  // pair p (0..7) of this thread in chunk c: tile row and first k of the pair
  auto pair_at = [&](int c, int p, int& row, int& kk) {
    const int bi = warp * 8 + p;
    if (kb + c * kKC >= m0 + kTileM) {
      row = (bi & 3) + 8 * (bi >> 2) + 4 * (lane >> 4);
      kk = 2 * (lane & 15);
    } else {
      row = 8 * (bi & 7) + (lane & 7);
      kk = 2 * (4 * (bi >> 3) + (lane >> 3));
    }
  };
  // entry (i, kg), i >= kg, of X_{C,C} sits in column desc[kg] at row
  // relidx[desc[kg].rel + i]; above the diagonal the symmetric one
  auto load_ri = [&](int c, int (&ri)[16]) {
    const int kt = kb + c * kKC;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      int row, kk;
      pair_at(c, p, row, kk);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = m0 + row, kg = kt + kk + h;
        ri[2 * p + h] = 0;
        if (i < r && kg < ke) {
          const ColDesc& cd = i < kg ? sm.rdesc[row] : sm.cdesc[c & 1][kk + h];
          ri[2 * p + h] = __ldg(relidx + cd.rel + (i < kg ? kg : i));
        }
      }
    }
  };

  long long hi[NF][4], lo[NF][4];
#pragma unroll
  for (int j = 0; j < NF; ++j)
#pragma unroll
    for (int x = 0; x < 4; ++x) hi[j][x] = lo[j][x] = 0;
  int ri[16];
  if (nck > 0) load_ri(0, ri);
  for (int c = 0; c < nck; ++c) {
    const int kt = kb + c * kKC;
    // column descriptors of the next chunk (stored after this chunk's staging)
    ColDesc cdn{0, 0};
    const bool have_cdn = t < kKC && c + 1 < nck && kt + kKC + t < ke;
    if (have_cdn) cdn = dk[kt + kKC + t];
    {
      uint4 v[16];
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        int row, kk;
        pair_at(c, p, row, kk);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = m0 + row, kg = kt + kk + h;
          v[2 * p + h] = make_uint4(0u, 0u, 0u, 0u);
          if (i < r && kg < ke)
            v[2 * p + h] = __ldg(xs + (i < kg ? sm.rdesc[row].col : sm.cdesc[c & 1][kk + h].col) + ri[2 * p + h]);
        }
      }
      uint4 w[NB / 4];
#pragma unroll
      for (int j = 0; j < NB / 8; ++j) {
        const int pi = j * kEmThreads + t, nn = pi >> 4, kk = 2 * (pi & 15), col = nb + nn;
        w[2 * j] = w[2 * j + 1] = make_uint4(0u, 0u, 0u, 0u);
        if (col < s) {
          if (kt + kk < ke) w[2 * j] = __ldg(ls + kt + kk + (int64_t)col * r);
          if (kt + kk + 1 < ke) w[2 * j + 1] = __ldg(ls + kt + kk + 1 + (int64_t)col * r);
        }
      }
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        int row, kk;
        pair_at(c, p, row, kk);
        stash_pair<kTileM>(sm.a, row, kk, v[2 * p], v[2 * p + 1]);
      }
#pragma unroll
      for (int j = 0; j < NB / 8; ++j) {
        const int pi = j * kEmThreads + t;
        stash_pair<NB>(sm.b, pi >> 4, 2 * (pi & 15), w[2 * j], w[2 * j + 1]);
      }
    }
    if (have_cdn) sm.cdesc[(c + 1) & 1][t] = cdn;
    __syncthreads();
    // relative indices of the next chunk, in flight during the products
    if (c + 1 < nck) load_ri(c + 1, ri);
    em_products<NB>(sm, hi, lo);
    __syncthreads();
  }
  // accumulator x of fragment j: row g + 8 (x >> 1), column 8 j + 2 q + (x & 1)
#pragma unroll
  for (int j = 0; j < NF; ++j)
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int row = warp * 16 + g + 8 * (x >> 1), col = nb + 8 * j + 2 * q + (x & 1);
      const int i = m0 + row;
      if (i < r && col < s) {
        const double v = ldexp((double)hi[j][x] + (double)lo[j][x] * 0x1p-32,
                               sm.erow[row] + sm.fcol[col - nb] - 31);
        if (m.ksplit == 1)
          ((double*)a.X + b * a.sz.panel + m.panel + s)[i + (int64_t)col * ld] = -v;
        else
          ((double*)a.ypart + b * a.sz.ypart + m.ypart + (int64_t)tk.c * r * s)[i + (int64_t)col * r] = v;
      }
    }
}

// Step 3 partial product on the slices: P_c = Lhat_{rows c, K}^T X_{rows c, K}
// for one task of the step-3 list (tile origin m0, n0 of width BN over the
// s x s output, row chunk c of C), P_mn = 2^(F_m + G_n - 32) (hi + lo 2^-32)
// from the slices of B' (exponents F) and of X'' (exponents G).  Both
// operands are read along the rows of C (contiguous); columns in blocks of 16.
template <int BN>
__global__ void __launch_bounds__(kEmThreads, 3) k_em_gemm2(KArgs a, EmArgs e, const Task* __restrict__ tasks) {
  constexpr int NB = BN < 16 ? BN : 16;
  constexpr int NF = NB / 8;
  __shared__ __align__(16) EmSmem<NB> sm;
  const Task tk = tasks[blockIdx.x];
  const int b = blockIdx.y;
  const SnMeta m = a.meta[tk.sn];
  const int s = m.s, r = m.r, ld = s + r;
  const uint4* xk = (const uint4*)e.xs + b * a.sz.panel + m.panel + s;  // X'' slices, column stride ld
  const uint4* ls = (const uint4*)e.ls + b * a.sz.lhat + m.lhat;          // B' slices, column stride r
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, q = lane & 3;
  const int m0 = tk.m0;
  const int kb = tk.c * m.kchunk3, ke = min(r, kb + m.kchunk3);
  if (t < kTileM) {
    sm.erow[t] = m0 + t < s ? e.lexp[b * e.n + m.f + m0 + t] : 0;
  } else {
    const int c = tk.n0 + (t - kTileM);
    sm.fcol[t - kTileM] = c < s ? e.gexp[b * e.n + m.f + c] : 0;
  }
  __syncthreads();
  double* out = (double*)a.part + b * a.sz.part + m.part + (int64_t)tk.c * s * s;
  for (int nb = tk.n0; nb < tk.n0 + BN && nb < s; nb += NB) {
    long long hi[NF][4], lo[NF][4];
#pragma unroll
    for (int j = 0; j < NF; ++j)
#pragma unroll
      for (int x = 0; x < 4; ++x) hi[j][x] = lo[j][x] = 0;
    for (int kt = kb; kt < ke; kt += kKC) {
      // A = B'^T: row mm of the tile is column m0 + mm of B', read along k (2 rows x 32 k per warp)
      uint4 v[16];
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const int bi = warp * 8 + p;
        const int row = (bi & 3) + 8 * (bi >> 2) + 4 * (lane >> 4), kk = 2 * (lane & 15);
        const int i = m0 + row;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          v[2 * p + h] = make_uint4(0u, 0u, 0u, 0u);
          if (i < s && kt + kk + h < ke) v[2 * p + h] = __ldg(ls + kt + kk + h + (int64_t)i * r);
        }
      }
      uint4 w[NB / 4];
#pragma unroll
      for (int j = 0; j < NB / 8; ++j) {
        const int pi = j * kEmThreads + t, nn = pi >> 4, kk = 2 * (pi & 15), col = nb + nn;
        w[2 * j] = w[2 * j + 1] = make_uint4(0u, 0u, 0u, 0u);
        if (col < s) {
          if (kt + kk < ke) w[2 * j] = __ldg(xk + kt + kk + (int64_t)col * ld);
          if (kt + kk + 1 < ke) w[2 * j + 1] = __ldg(xk + kt + kk + 1 + (int64_t)col * ld);
        }
      }
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const int bi = warp * 8 + p;
        stash_pair<kTileM>(sm.a, (bi & 3) + 8 * (bi >> 2) + 4 * (lane >> 4), 2 * (lane & 15), v[2 * p],
                           v[2 * p + 1]);
      }
#pragma unroll
      for (int j = 0; j < NB / 8; ++j) {
        const int pi = j * kEmThreads + t;
        stash_pair<NB>(sm.b, pi >> 4, 2 * (pi & 15), w[2 * j], w[2 * j + 1]);
      }
      __syncthreads();
      em_products<NB>(sm, hi, lo);
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NF; ++j)
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int row = warp * 16 + g + 8 * (x >> 1), col = nb + 8 * j + 2 * q + (x & 1);
        const int i = m0 + row;
        if (i < s && col < s)
          out[i + (int64_t)col * s] = ldexp((double)hi[j][x] + (double)lo[j][x] * 0x1p-32,
                                            sm.erow[row] + sm.fcol[col - tk.n0] - 32);
      }
  }
}

}  // namespace

cudaError_t launch_em_split_x(const KArgs& a, const EmArgs& e, const int32_t* sns, int nsn, cudaStream_t st) {
  if (nsn <= 0) return cudaSuccess;
  k_em_split_x<<<dim3(nsn, a.sz.batch, kSplitGroups), 256, 0, st>>>(a, e, sns);
  return cudaGetLastError();
}

cudaError_t launch_em_split_lhat(const KArgs& a, const EmArgs& e, const int32_t* sns, int nsn, int max_r,
                                 cudaStream_t st) {
  if (nsn <= 0) return cudaSuccess;
  const int cap = max_r < kEcRows ? max_r : kEcRows;
  k_em_split_lhat<<<dim3(nsn, a.sz.batch, kSplitGroups), 256, sizeof(int) * cap, st>>>(a, e, sns, cap);
  return cudaGetLastError();
}

cudaError_t launch_em_split_xck(const KArgs& a, const EmArgs& e, const int32_t* sns, int nsn, int max_r,
                                cudaStream_t st) {
  if (nsn <= 0) return cudaSuccess;
  const int cap = max_r < kEcRows ? max_r : kEcRows;
  k_em_split_xck<<<dim3(nsn, a.sz.batch, kSplitGroups), 256, sizeof(int) * cap, st>>>(a, e, sns, cap);
  return cudaGetLastError();
}

cudaError_t launch_em_gemm2(int var, const KArgs& a, const EmArgs& e, const Task* t, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)n, a.sz.batch);
  switch (var) {
    case 0: k_em_gemm2<8><<<grid, kEmThreads, 0, st>>>(a, e, t); break;
    case 1: k_em_gemm2<16><<<grid, kEmThreads, 0, st>>>(a, e, t); break;
    case 2: k_em_gemm2<32><<<grid, kEmThreads, 0, st>>>(a, e, t); break;
    default: k_em_gemm2<64><<<grid, kEmThreads, 0, st>>>(a, e, t); break;
  }
  return cudaGetLastError();
}

cudaError_t setup_em_kernels() {
  cudaError_t err = cudaFuncSetAttribute(k_em_split_lhat, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(int) * kEcRows);
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(k_em_split_xck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(int) * kEcRows);
  if (err != cudaSuccess) return err;
  // static shared memory (< 48 KB): prefer the shared-memory carve-out (3 CTAs per SM)
  err = cudaFuncSetAttribute(k_em_gemm1<8>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err != cudaSuccess) return err;
  return cudaFuncSetAttribute(k_em_gemm1<16>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

cudaError_t launch_em_gemm1(int var, const KArgs& a, const EmArgs& e, const Task* t, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)n, a.sz.batch);
  switch (var) {  // the emulation's task lists hold 64 x 8 and 64 x 16 tiles only
    case 0: k_em_gemm1<8><<<grid, kEmThreads, 0, st>>>(a, e, t); break;
    case 1: k_em_gemm1<16><<<grid, kEmThreads, 0, st>>>(a, e, t); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace psi
