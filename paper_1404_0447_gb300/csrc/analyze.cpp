// Host symbolic analysis for the supernodal selected inversion.
//
//  - elimination tree (Section 2.2; column version), postorder;
//  - column counts |struct(j)| by row-subtree traversal;
//  - supernode partition (Section 2.1: fundamental supernodes, relaxed by
//    merging and a width cap; the rule is spelled out in pselinv.h);
//  - supernodal rows R(K) (the set C of Algorithm 1, step 0) by the
//    supernodal recursion R(K) = (A rows of K U R(children)) beyond K;
//  - priority lists of Algorithm 2;
//  - relative indices of each C inside its ancestor supernodes (Section 3.1's
//    non-contiguous row lists), the per-column gather descriptors and the
//    value map from A's entries into the panels;
//  - task lists of the grouped launches and the work counts.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace psi {
namespace {

int fail(pselinv_handle* h, int code, const std::string& msg) {
  h->err = msg;
  return code;
}

// Lower pattern of P A P^T with, for every entry, its position in the
// caller's arrays.
struct Pattern {
  std::vector<int64_t> cp;
  std::vector<int32_t> ri;
  std::vector<int64_t> src;
  std::vector<uint8_t> flip;  // entry transposed by the ordering
};

Pattern permute_pattern(int64_t n, const int64_t* cp, const int32_t* ri,
                        const std::vector<int32_t>& inv) {
  Pattern P;
  const int64_t nnz = cp[n];
  P.cp.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
      int32_t a = inv[ri[p]], b = inv[j];
      P.cp[std::min(a, b) + 1]++;
    }
  for (int64_t j = 0; j < n; ++j) P.cp[j + 1] += P.cp[j];
  P.ri.resize(nnz);
  P.src.resize(nnz);
  P.flip.resize(nnz);
  std::vector<int64_t> next(P.cp.begin(), P.cp.end() - 1);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
      int32_t a = inv[ri[p]], b = inv[j];
      int64_t q = next[std::min(a, b)]++;
      P.ri[q] = std::max(a, b);
      P.src[q] = p;
      P.flip[q] = a < b;  // the ordering moved this entry above the diagonal
    }
  // sort every column by row (columns are short; insertion sort on pairs)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t p = P.cp[j] + 1; p < P.cp[j + 1]; ++p) {
      int32_t r = P.ri[p];
      int64_t s = P.src[p];
      uint8_t f = P.flip[p];
      int64_t q = p - 1;
      while (q >= P.cp[j] && P.ri[q] > r) {
        P.ri[q + 1] = P.ri[q];
        P.src[q + 1] = P.src[q];
        P.flip[q + 1] = P.flip[q];
        --q;
      }
      P.ri[q + 1] = r;
      P.src[q + 1] = s;
      P.flip[q + 1] = f;
    }
  }
  return P;
}

// Row lists of a lower pattern (the columns j < i with (i, j) stored).
void row_lists(int64_t n, const Pattern& P, std::vector<int64_t>& rp, std::vector<int32_t>& rc) {
  rp.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = P.cp[j] + 1; p < P.cp[j + 1]; ++p) rp[P.ri[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  rc.resize(rp[n]);
  std::vector<int64_t> next(rp.begin(), rp.end() - 1);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = P.cp[j] + 1; p < P.cp[j + 1]; ++p) rc[next[P.ri[p]]++] = (int32_t)j;
}

// Elimination tree with a disjoint-set forest: scanning rows in order, each
// A_ij (j < i) joins the set holding j -- whose current tree root becomes a
// child of i -- to i's set.
std::vector<int32_t> etree(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& rc) {
  std::vector<int32_t> parent(n, -1), ds(n), top(n);
  auto find = [&](int32_t x) {
    while (ds[x] != x) {
      ds[x] = ds[ds[x]];  // path halving
      x = ds[x];
    }
    return x;
  };
  for (int64_t i = 0; i < n; ++i) {
    ds[i] = (int32_t)i;
    top[i] = (int32_t)i;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
      int32_t set = find(rc[q]);
      int32_t root = top[set];
      if (root != i) {
        parent[root] = (int32_t)i;
        int32_t mine = find((int32_t)i);
        ds[set] = mine;
        top[mine] = (int32_t)i;
      }
    }
  }
  return parent;
}

// Postorder (children in increasing order, roots in increasing order) by a
// stackless threaded walk over first-child / next-sibling links.
std::vector<int32_t> postorder(int64_t n, const std::vector<int32_t>& parent) {
  std::vector<int32_t> first(n, -1), sib(n, -1), roots;
  for (int64_t j = n - 1; j >= 0; --j) {
    if (parent[j] >= 0) {
      sib[j] = first[parent[j]];
      first[parent[j]] = (int32_t)j;
    }
  }
  for (int64_t j = 0; j < n; ++j)
    if (parent[j] < 0) roots.push_back((int32_t)j);
  std::vector<int32_t> post;
  post.reserve(n);
  for (int32_t r : roots) {
    int32_t v = r;
    while (first[v] >= 0) v = first[v];
    for (;;) {
      post.push_back(v);
      if (v == r) break;
      if (sib[v] >= 0) {
        v = sib[v];
        while (first[v] >= 0) v = first[v];
      } else {
        v = parent[v];
      }
    }
  }
  return post;
}

double sn_flops(double s, double r) { return 2 * r * r * s + 3 * r * s * s + 2.0 / 3.0 * s * s * s; }

}  // namespace

int analyze(pselinv_handle* h, int64_t n, const int64_t* cp, const int32_t* ri,
            const int32_t* uperm) {
  if (n < 1 || n >= (int64_t)1 << 31) return fail(h, PSELINV_ERR_ARG, "n out of range");
  if (!cp || !ri) return fail(h, PSELINV_ERR_ARG, "null pattern pointer");
  if (cp[0] != 0) return fail(h, PSELINV_ERR_NOT_LOWER, "colptr[0] != 0");
  for (int64_t j = 0; j < n; ++j) {
    if (cp[j + 1] <= cp[j]) return fail(h, PSELINV_ERR_NOT_LOWER, "empty column (missing diagonal)");
    if (ri[cp[j]] != j) return fail(h, PSELINV_ERR_NOT_LOWER, "diagonal not first in column " + std::to_string(j));
    for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p)
      if (ri[p] <= ri[p - 1] || ri[p] >= n)
        return fail(h, PSELINV_ERR_NOT_LOWER, "rows not increasing / out of range in column " + std::to_string(j));
  }
  const pselinv_opts& o = h->opts;
  int wcap = o.max_sn_width == 0 ? kMaxWidth : o.max_sn_width;
  if (wcap < 1 || wcap > kMaxWidth) return fail(h, PSELINV_ERR_ARG, "max_sn_width must be 0..128");
  if (o.unsym != 0 && o.unsym != 1) return fail(h, PSELINV_ERR_ARG, "unsym must be 0 or 1");
  if (o.unsym && o.dtype == PSELINV_C128) wcap = std::min(wcap, kMaxWidthLUComplex);
  if (o.fp64_emulation < 0 || o.fp64_emulation > 1) return fail(h, PSELINV_ERR_ARG, "fp64_emulation must be 0 or 1");
  if (o.fp64_emulation && (o.dtype != PSELINV_F64 || o.unsym))
    return fail(h, PSELINV_ERR_ARG, "fp64_emulation is for real symmetric handles");
  if (o.relax != PSELINV_RELAX_NONE && o.relax != PSELINV_RELAX_AMALG)
    return fail(h, PSELINV_ERR_ARG, "bad relax mode");

  h->n = n;
  h->nnz_a = cp[n];
  std::vector<int32_t> perm(n), inv(n, -1);
  if (uperm) {
    for (int64_t k = 0; k < n; ++k) {
      int32_t u = uperm[k];
      if (u < 0 || u >= n || inv[u] >= 0) return fail(h, PSELINV_ERR_NOT_LOWER, "perm is not a permutation");
      inv[u] = (int32_t)k;
      perm[k] = u;
    }
  } else {
    std::iota(perm.begin(), perm.end(), 0);
    std::iota(inv.begin(), inv.end(), 0);
  }

  // ---- elimination tree and postorder ----
  Pattern P = permute_pattern(n, cp, ri, inv);
  std::vector<int64_t> rp;
  std::vector<int32_t> rc;
  row_lists(n, P, rp, rc);
  std::vector<int32_t> parent = etree(n, rp, rc);
  std::vector<int32_t> post = postorder(n, parent);
  bool ident = true;
  for (int64_t k = 0; k < n && ident; ++k) ident = post[k] == k;
  if (!ident) {
    std::vector<int32_t> perm2(n);
    for (int64_t k = 0; k < n; ++k) perm2[k] = perm[post[k]];
    perm.swap(perm2);
    for (int64_t k = 0; k < n; ++k) inv[perm[k]] = (int32_t)k;
    P = permute_pattern(n, cp, ri, inv);
    row_lists(n, P, rp, rc);
    parent = etree(n, rp, rc);
  }

  // ---- column counts by row subtrees ----
  std::vector<int64_t> cnt(n, 0);
  {
    std::vector<int32_t> mark(n, -1);
    for (int64_t i = 0; i < n; ++i) {
      mark[i] = (int32_t)i;
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        for (int32_t k = rc[q]; mark[k] != i; k = parent[k]) {
          cnt[k]++;
          mark[k] = (int32_t)i;
        }
    }
  }

  // ---- supernodes ----
  std::vector<int32_t> nchild(n, 0);
  for (int64_t j = 0; j < n; ++j)
    if (parent[j] >= 0) nchild[parent[j]]++;
  std::vector<int32_t> fund;
  for (int64_t j = 0; j < n; ++j) {
    bool joins = j > 0 && parent[j - 1] == j && nchild[j] == 1 && cnt[j - 1] == cnt[j] + 1;
    if (!joins) fund.push_back((int32_t)j);
  }
  fund.push_back((int32_t)n);
  // true entries of columns [a, b): sum of 1 + |struct(j)|
  std::vector<int64_t> tpre(n + 1, 0);
  for (int64_t j = 0; j < n; ++j) tpre[j + 1] = tpre[j] + 1 + cnt[j];
  std::vector<int32_t> merged;
  if (o.relax == PSELINV_RELAX_AMALG) {
    const int64_t nf = (int64_t)fund.size() - 1;
    int32_t cur = fund[0];
    for (int64_t t = 0; t < nf; ++t) {
      const int32_t last = fund[t + 1] - 1;
      bool take = false;
      if (t + 1 < nf) {
        const int32_t pf = fund[t + 1], pl = fund[t + 2] - 1;
        const int32_t par = parent[last];
        if (par >= pf && par <= pl) {
          const int64_t s = pl - cur + 1;
          const int64_t stored = s * (s + 1) / 2 + s * cnt[pl];
          const int64_t zeros = stored - (tpre[pl + 1] - tpre[cur]);
          take = s <= wcap && (s <= 8 || 20 * zeros <= stored);
        }
      }
      if (!take) {
        merged.push_back(cur);
        if (t + 1 < nf) cur = fund[t + 1];
      }
    }
    merged.push_back((int32_t)n);
  } else {
    merged = fund;
  }
  std::vector<int32_t>& ss = h->sn_start;
  ss.clear();
  for (size_t t = 0; t + 1 < merged.size(); ++t)
    for (int32_t c = merged[t]; c < merged[t + 1]; c += wcap) ss.push_back(c);
  ss.push_back((int32_t)n);
  const int32_t nsn = (int32_t)ss.size() - 1;
  h->nsn = nsn;
  std::vector<int32_t> col2sn(n);
  for (int32_t k = 0; k < nsn; ++k)
    for (int32_t j = ss[k]; j < ss[k + 1]; ++j) col2sn[j] = k;

  // ---- supernodal rows R(K) and parents ----
  h->rowptr.assign(nsn + 1, 0);
  h->rows.clear();
  h->sn_parent.assign(nsn, -1);
  {
    std::vector<std::vector<int32_t>> kids(nsn);
    std::vector<int32_t> mark(n, -1), buf;
    for (int32_t k = 0; k < nsn; ++k) {
      const int32_t f = ss[k], l = ss[k + 1] - 1;
      buf.clear();
      for (int32_t j = f; j <= l; ++j)
        for (int64_t p = P.cp[j] + 1; p < P.cp[j + 1]; ++p) {
          int32_t i = P.ri[p];
          if (i > l && mark[i] != k) { mark[i] = k; buf.push_back(i); }
        }
      for (int32_t c : kids[k])
        for (int64_t p = h->rowptr[c]; p < h->rowptr[c + 1]; ++p) {
          int32_t i = h->rows[p];
          if (i > l && mark[i] != k) { mark[i] = k; buf.push_back(i); }
        }
      std::sort(buf.begin(), buf.end());
      h->rows.insert(h->rows.end(), buf.begin(), buf.end());
      h->rowptr[k + 1] = (int64_t)h->rows.size();
      if (!buf.empty()) {
        h->sn_parent[k] = col2sn[buf[0]];
        kids[h->sn_parent[k]].push_back(k);
      }
    }
  }

  // ---- metadata, work counts, priority lists (Algorithm 2) ----
  h->meta.assign(nsn, SnMeta{});
  h->panel_off.assign(nsn + 1, 0);
  std::vector<double> cost(nsn);
  h->flops_selinv = h->flops_gemm1 = h->bytes_selinv = 0;
  h->nnz_l = 0;
  h->max_r = 0;
  h->max_width = 0;
  int64_t lhat = 0, linv = 0;
  for (int32_t k = 0; k < nsn; ++k) {
    SnMeta& m = h->meta[k];
    m.f = ss[k];
    m.s = ss[k + 1] - ss[k];
    m.r = (int32_t)(h->rowptr[k + 1] - h->rowptr[k]);
    m.panel = h->panel_off[k];
    h->panel_off[k + 1] = h->panel_off[k] + (int64_t)(m.s + m.r) * m.s;
    m.lhat = lhat;
    lhat += (int64_t)m.r * m.s;
    m.linv = linv;
    linv += (int64_t)m.s * m.s;
    m.desc = h->rowptr[k];
    const double s = m.s, r = m.r;
    cost[k] = sn_flops(s, r);
    h->flops_selinv += o.unsym ? 4 * r * r * s + 4 * r * s * s + 4.0 / 3.0 * s * s * s : cost[k];
    h->flops_gemm1 += (o.unsym ? 4 : 2) * r * r * s;
    h->nnz_l += (int64_t)m.s * (m.s + 1) / 2 + (int64_t)m.s * m.r;
    h->max_r = std::max<int64_t>(h->max_r, m.r);
    h->max_width = std::max(h->max_width, m.s);
  }
  h->panel_total = h->panel_off[nsn];
  h->lhat_total = lhat;
  h->linv_total = linv;
  h->sigma.assign(nsn, 0);
  for (int32_t k = nsn - 1; k >= 0; --k)
    h->sigma[k] = h->sn_parent[k] < 0 ? 1 : h->sigma[h->sn_parent[k]] + 1;
  int32_t nl = 0;
  for (int32_t k = 0; k < nsn; ++k) nl = std::max(nl, h->sigma[k]);
  h->nlevels = nl;
  h->level_ptr.assign(nl + 1, 0);
  for (int32_t k = 0; k < nsn; ++k) h->level_ptr[h->sigma[k]]++;
  for (int32_t l = 0; l < nl; ++l) h->level_ptr[l + 1] += h->level_ptr[l];
  h->level_sn.assign(nsn, 0);
  {
    std::vector<int32_t> next(h->level_ptr.begin(), h->level_ptr.end() - 1);
    for (int32_t k = 0; k < nsn; ++k) h->level_sn[next[h->sigma[k] - 1]++] = k;
    for (int32_t l = 0; l < nl; ++l)
      std::stable_sort(h->level_sn.begin() + h->level_ptr[l], h->level_sn.begin() + h->level_ptr[l + 1],
                       [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  }

  // ---- relative indices, gather descriptors ----
  struct Blk {
    int32_t k, j, p;
    int64_t out;
  };
  std::vector<Blk> blks;
  h->relptr.assign(nsn + 1, 0);
  h->nblk.assign(nsn, 0);
  int64_t tot = 0;
  for (int32_t k = 0; k < nsn; ++k) {
    const int32_t* C = h->rows.data() + h->rowptr[k];
    const int32_t r = h->meta[k].r;
    for (int32_t p = 0; p < r;) {
      int32_t j = col2sn[C[p]];
      int32_t q = p;
      while (q < r && col2sn[C[q]] == j) ++q;
      blks.push_back({k, j, p, tot});
      tot += r - p;
      h->nblk[k]++;
      p = q;
    }
    h->relptr[k + 1] = tot;
  }
  h->relidx.assign(tot, -1);
  h->desc.assign(h->rowptr[nsn], ColDesc{0, 0});
  {
    // bucket the blocks by their ancestor J, then fill with a position map of J
    std::vector<int64_t> bptr(nsn + 1, 0);
    for (const Blk& b : blks) bptr[b.j + 1]++;
    for (int32_t k = 0; k < nsn; ++k) bptr[k + 1] += bptr[k];
    std::vector<int32_t> order(blks.size());
    std::vector<int64_t> next(bptr.begin(), bptr.end() - 1);
    for (size_t t = 0; t < blks.size(); ++t) order[next[blks[t].j]++] = (int32_t)t;
    std::vector<int32_t> pos(n, -1);
    for (int32_t j = 0; j < nsn; ++j) {
      if (bptr[j] == bptr[j + 1]) continue;
      const SnMeta& mj = h->meta[j];
      for (int32_t c = 0; c < mj.s; ++c) pos[mj.f + c] = c;
      for (int32_t t = 0; t < mj.r; ++t) pos[h->rows[h->rowptr[j] + t]] = mj.s + t;
      for (int64_t t = bptr[j]; t < bptr[j + 1]; ++t) {
        const Blk& b = blks[order[t]];
        const int32_t* C = h->rows.data() + h->rowptr[b.k];
        const int32_t r = h->meta[b.k].r;
        for (int32_t i = b.p; i < r; ++i) {
          int32_t v = pos[C[i]];
          if (v < 0) return fail(h, PSELINV_ERR_NOT_LOWER, "internal: structure not closed");
          h->relidx[b.out + (i - b.p)] = v;
        }
        for (int32_t i = b.p; i < r && col2sn[C[i]] == j; ++i) {
          ColDesc& d = h->desc[h->rowptr[b.k] + i];
          d.col = mj.panel + (int64_t)(C[i] - mj.f) * (mj.s + mj.r);
          d.rel = b.out - b.p;
        }
      }
      for (int32_t c = 0; c < mj.s; ++c) pos[mj.f + c] = -1;
      for (int32_t t = 0; t < mj.r; ++t) pos[h->rows[h->rowptr[j] + t]] = -1;
    }
  }
  for (int32_t k = 0; k < nsn; ++k) {
    const double s = h->meta[k].s, r = h->meta[k].r;
    const double idx = 4.0 * (h->relptr[k + 1] - h->relptr[k]);
    h->bytes_selinv += o.unsym ? 8.0 * (r * r + 4 * (s + r) * s) + 2 * idx
                               : 8.0 * (r * (r + 1) / 2 + 2 * (s + r) * s) + idx;
  }

  // ---- value map: A's stored entries -> panel offsets ----
  h->valmap.assign(h->nnz_a, -1);
  h->diagmask.assign(h->nnz_a, 0);
  if (o.unsym) h->flipmap.assign(h->nnz_a, 0);
  for (int64_t j = 0; j < n; ++j) h->diagmask[cp[j]] = 1;  // diagonal first in every column
  for (int64_t j = 0; j < n; ++j) {
    const SnMeta& m = h->meta[col2sn[j]];
    const int32_t* R = h->rows.data() + h->rowptr[col2sn[j]];
    const int32_t ld = m.s + m.r;
    for (int64_t p = P.cp[j]; p < P.cp[j + 1]; ++p) {
      const int32_t i = P.ri[p];
      int64_t pos;
      if (i < m.f + m.s) {
        pos = i - m.f;
      } else {
        const int32_t* it = std::lower_bound(R, R + m.r, i);
        if (it == R + m.r || *it != i) return fail(h, PSELINV_ERR_NOT_LOWER, "internal: entry outside L");
        pos = m.s + (it - R);
      }
      h->valmap[P.src[p]] = m.panel + (j - m.f) * (int64_t)ld + pos;
      if (o.unsym) h->flipmap[P.src[p]] = P.flip[p];
    }
  }

  h->perm = perm;
  h->parent = parent;
  return build_schedule(h);
}

// Schedule of the grouped launches (depends on the tuning options, not on the
// pattern): step-2 slices of wide C, the task lists and the level-local
// offsets of the partial-product buffers.
int build_schedule(pselinv_handle* h) {
  {
    // Step-2 slices: at most split_k_rows rows of C each; in a level whose
    // tiles cannot fill the GPU (fewer than opts.level_tiles, default
    // kTargetTiles) the slices shrink, down to opts.min_slice_rows (default
    // kMinSlice2) rows, until it can.  Step-3 row chunks likewise from
    // kChunkRows down to a quarter of that minimum.  Slice sizes are
    // multiples of 16.
    const pselinv_opts& o = h->opts;
    const bool cplx = o.dtype == PSELINV_C128;
    const int64_t target = o.level_tiles > 0 ? o.level_tiles : kTargetTiles;
    const int32_t min2 = o.min_slice_rows > 0 ? o.min_slice_rows : kMinSlice2;
    const int32_t min3 = std::max<int32_t>(16, min2 / 4);
    auto slices = [](int32_t r, int32_t rows, int32_t* chunk) {
      const int32_t parts = (r + rows - 1) / rows;
      *chunk = ((r + parts - 1) / parts + 15) / 16 * 16;
      return (r + *chunk - 1) / *chunk;
    };
    h->s2var.assign(h->nsn, 0);
    h->s3var.assign(h->nsn, 0);
    h->trvar.assign(h->nsn, 0);
    for (int32_t l = 0; l < h->nlevels; ++l) {
      int64_t t2 = 0, t3 = 0;
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
        SnMeta& m = h->meta[h->level_sn[t]];
        const int bn = 8 << pick_variant(m.s, cplx, o.small_cutoff);
        const int bn2 = 8 << step2_variant(m.s, cplx, o);
        const int64_t mt = (m.r + kTileM - 1) / kTileM, nt = (m.s + bn - 1) / bn, st = (m.s + kTileM - 1) / kTileM;
        const int64_t nt2 = (m.s + bn2 - 1) / bn2, mt2 = (m.r + step2_rows(o) - 1) / step2_rows(o);
        m.ksplit = 1;
        m.kchunk = m.r;
        if (o.split_k_rows > 0 && m.r > o.split_k_rows) m.ksplit = slices(m.r, o.split_k_rows, &m.kchunk);
        m.nchunk = m.r > 0 ? slices(m.r, kChunkRows, &m.kchunk3) : 0;
        if (m.r == 0) m.kchunk3 = kChunkRows;
        t2 += mt2 * nt2 * m.ksplit;
        t3 += (int64_t)m.nchunk * st * nt;
      }
      if (o.split_k_rows > 0 && t2 > 0 && t2 < target) {
        const int64_t f = (target + t2 - 1) / t2;
        for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
          SnMeta& m = h->meta[h->level_sn[t]];
          const int32_t rows = std::max<int32_t>(min2, (int32_t)((m.r + m.ksplit * f - 1) / (m.ksplit * f)));
          if (m.r > rows) m.ksplit = slices(m.r, rows, &m.kchunk);
        }
      }
      // step 3 aims at half the step-2 target: every extra row chunk is one
      // more s x s partial for the finish to read
      const int64_t target3 = target / 2;
      if (t3 > 0 && t3 < target3) {
        const int64_t f = (target3 + t3 - 1) / t3;
        for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
          SnMeta& m = h->meta[h->level_sn[t]];
          if (m.r == 0) continue;
          const int32_t rows = std::max<int32_t>(min3, (int32_t)((m.r + m.nchunk * f - 1) / (m.nchunk * f)));
          m.nchunk = slices(m.r, rows, &m.kchunk3);
        }
      }
      // A level that still offers fewer tiles than the target (short slices
      // cannot go below the minimum) takes the narrowest tiles, 64 x 8, for
      // steps 2 and 3: up to 8x the tiles at the same padding (dead 8 x 8
      // fragments are skipped), so the few wide supernodes near the root
      // spread over the SMs.
      int64_t t2f = 0, t3f = 0;
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
        const int32_t k = h->level_sn[t];
        const SnMeta& m = h->meta[k];
        h->s2var[k] = (int8_t)step2_variant(m.s, cplx, o);
        h->s3var[k] = (int8_t)pick_variant(m.s, cplx, o.small_cutoff);
        const int64_t bn2 = 8 << h->s2var[k], bn3 = 8 << h->s3var[k];
        t2f += (m.r + step2_rows(o) - 1) / step2_rows(o) * ((m.s + bn2 - 1) / bn2) * m.ksplit;
        t3f += (int64_t)m.nchunk * ((m.s + kTileM - 1) / kTileM) * ((m.s + bn3 - 1) / bn3);
      }
      // the factorisation's panel solve (r x s tiles, k <= s) likewise
      int64_t ttf = 0;
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
        const SnMeta& m = h->meta[h->level_sn[t]];
        const int64_t bn = 8 << pick_variant(m.s, cplx, o.small_cutoff);
        ttf += (m.r + kTileM - 1) / kTileM * ((m.s + bn - 1) / bn);
      }
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
        const int32_t k = h->level_sn[t];
        if (t2f < target && !o.fp64_emulation) h->s2var[k] = 0;
        if (t3f < target / 2 && !o.fp64_emulation) h->s3var[k] = 0;
        h->trvar[k] = (int8_t)(ttf < target ? 0 : pick_variant(h->meta[k].s, cplx, o.small_cutoff));
      }
    }
  }
  // ---- task lists ----
  // Level lists hold, per level, per tile variant, the supernodes in level
  // order (costliest first), each supernode's tiles contiguous.  The
  // normalisation list is variant-major over all levels (one launch per
  // variant).
  const pselinv_opts& o = h->opts;
  const bool cplx = o.dtype == PSELINV_C128;
  const int32_t nsn = h->nsn, nl = h->nlevels;
  auto build = [&](TaskList& tl, bool variant_major, auto&& var_of, auto&& emit) {
    tl.tasks.clear();
    tl.per_lv.assign((size_t)nl * kNumVar, Range{});
    tl.per_sn.assign(nsn, Range{});
    tl.var.assign(nsn, 0);
    for (int32_t k = 0; k < nsn; ++k) tl.var[k] = (int8_t)var_of(k);
    auto add_sn = [&](int32_t k) {
      tl.per_sn[k].begin = (int64_t)tl.tasks.size();
      emit(k, 8 << tl.var[k], tl.tasks);
      tl.per_sn[k].end = (int64_t)tl.tasks.size();
    };
    if (variant_major) {
      for (int v = 0; v < kNumVar; ++v) {
        tl.whole[v].begin = (int64_t)tl.tasks.size();
        for (int32_t t = 0; t < nsn; ++t)
          if (tl.var[h->level_sn[t]] == v) add_sn(h->level_sn[t]);
        tl.whole[v].end = (int64_t)tl.tasks.size();
      }
      return;
    }
    for (int32_t l = 0; l < nl; ++l)
      for (int v = 0; v < kNumVar; ++v) {
        Range& rg = tl.per_lv[(size_t)l * kNumVar + v];
        rg.begin = (int64_t)tl.tasks.size();
        for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t)
          if (tl.var[h->level_sn[t]] == v) add_sn(h->level_sn[t]);
        rg.end = (int64_t)tl.tasks.size();
      }
  };
  auto by_width = [&](int32_t k) { return pick_variant(h->meta[k].s, cplx, o.small_cutoff); };
  auto by_rows = [&](int32_t) { return cplx ? 2 : 3; };
  auto rect = [&](int32_t k, int bn, std::vector<Task>& out) {  // r x s output tiles
    const SnMeta& m = h->meta[k];
    for (int32_t m0 = 0; m0 < m.r; m0 += kTileM)
      for (int32_t n0 = 0; n0 < m.s; n0 += bn) out.push_back({k, m0, n0, 0});
  };
  build(h->t_lhat, true, by_width, rect);
  // the adjoint's r x s and s x s tile lists: 64 x 8 tiles on levels whose
  // tiles are too few to fill the GPU (as for steps 2 and 3)
  std::vector<int8_t> rvar(nsn), qvar(nsn);
  {
    const int64_t target = o.level_tiles > 0 ? o.level_tiles : kTargetTiles;
    for (int32_t l = 0; l < nl; ++l) {
      int64_t nr = 0, nq = 0;
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
        const SnMeta& m = h->meta[h->level_sn[t]];
        const int64_t bn = 8 << by_width(h->level_sn[t]);
        nr += (m.r + kTileM - 1) / kTileM * ((m.s + bn - 1) / bn);
        nq += (m.s + kTileM - 1) / kTileM * ((m.s + bn - 1) / bn);
      }
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
        const int32_t k = h->level_sn[t];
        rvar[k] = (int8_t)(nr < target ? 0 : by_width(k));
        qvar[k] = (int8_t)(nq < target ? 0 : by_width(k));
      }
    }
  }
  build(h->t_rect, false, [&](int32_t k) { return (int)rvar[k]; }, rect);
  auto step2_tiles = [&](int32_t k, int bn, std::vector<Task>& out) {  // step 2: + k-parts
    const SnMeta& m = h->meta[k];
    for (int32_t c = 0; c < m.ksplit; ++c)
      for (int32_t m0 = 0; m0 < m.r; m0 += step2_rows(o))
        for (int32_t n0 = 0; n0 < m.s; n0 += bn) out.push_back({k, m0, n0, c});
  };
  auto step3_tiles = [&](int32_t k, int bn, std::vector<Task>& out) {
    const SnMeta& m = h->meta[k];
    for (int32_t c = 0; c < m.nchunk; ++c)
      for (int32_t m0 = 0; m0 < m.s; m0 += kTileM)
        for (int32_t n0 = 0; n0 < m.s; n0 += bn) out.push_back({k, m0, n0, c});
  };
  build(h->t_gemm1, false, [&](int32_t k) { return (int)h->s2var[k]; }, step2_tiles);
  build(h->t_trsm, false, [&](int32_t k) { return (int)h->trvar[k]; }, rect);
  build(h->t_gemm2, false, [&](int32_t k) { return (int)h->s3var[k]; }, step3_tiles);
  build(h->t_sq, false, [&](int32_t k) { return (int)qvar[k]; }, [&](int32_t k, int bn, std::vector<Task>& out) {
    const SnMeta& m = h->meta[k];
    for (int32_t m0 = 0; m0 < m.s; m0 += kTileM)
      for (int32_t n0 = 0; n0 < m.s; n0 += bn) out.push_back({k, m0, n0, 0});
  });
  // the persistent kernel holds one shared-memory tile for every task kind,
  // so its lists stop at 64 x (8 << kPersistentMaxVar) tiles (register budget: more CTAs per SM)
  auto by_width_narrow = [&](int32_t k) { return std::min(by_width(k), kPersistentMaxVar); };
  build(h->t_pgemm1, false, by_width_narrow, step2_tiles);
  build(h->t_pgemm2, false, by_width_narrow, step3_tiles);
  {
    // Schur-update tiles (lower tiles of the r x r update of each supernode),
    // grouped so that the factorisation needs no atomics: two supernodes of a
    // level conflict when their C share a row (both then update entries of
    // that ancestor column); a greedy colouring in level order gives each
    // supernode the first group none of its conflicting predecessors holds.
    // Groups run one after the other (fixed order), the supernodes of a
    // group in parallel, every target entry read-modified-written by one
    // thread: the factor is bitwise reproducible.
    TaskList& tl = h->t_schur;
    const int var = by_rows(0);
    h->schur_var = var;
    tl.tasks.clear();
    tl.per_lv.assign((size_t)nl * kNumVar, Range{});
    tl.per_sn.assign(nsn, Range{});
    tl.var.assign(nsn, (int8_t)var);
    h->schur_gptr.assign(nl + 1, 0);
    h->schur_near.clear();
    h->schur_far.clear();
    h->schur_gvar.clear();
    h->schur_gsn_ptr.assign(1, 0);
    h->schur_gsn.clear();
    std::vector<uint64_t> used(h->n, 0);  // groups (< 64) holding a supernode with this row in C
    std::vector<int32_t> touched, color;
    for (int32_t l = 0; l < nl; ++l) {
      h->schur_gptr[l] = (int32_t)h->schur_near.size();
      const int32_t b = h->level_ptr[l], e = h->level_ptr[l + 1];
      color.assign(e - b, 0);
      int32_t ncol = 0;
      for (int32_t t = b; t < e; ++t) {
        const int32_t k = h->level_sn[t];
        const int32_t* C = h->rows.data() + h->rowptr[k];
        const int32_t r = h->meta[k].r;
        uint64_t busy = 0;
        for (int32_t i = 0; i < r; ++i) busy |= used[C[i]];
        int32_t c;
        if (~busy) {
          c = 0;
          while (busy >> c & 1) ++c;
          for (int32_t i = 0; i < r; ++i) {
            if (!used[C[i]]) touched.push_back(C[i]);
            used[C[i]] |= 1ull << c;
          }
        } else {
          c = 64 + (t - b);  // all 64 masks taken: a group of its own
        }
        color[t - b] = c;
        ncol = std::max(ncol, c + 1);
      }
      for (int32_t q : touched) used[q] = 0;
      touched.clear();
      // Each supernode's tiles split at np, the number of rows of C inside its
      // parent P: "near" tiles (target columns in P, level l - 1) and "far"
      // tiles (columns above P, levels <= l - 2).  Task.c holds the tile's
      // column end.  Per colour the near tiles, then the far tiles, adjacent:
      // near and far target different levels, so a colour's two ranges may
      // also run as one launch.
      Range& lv = tl.per_lv[(size_t)l * kNumVar + var];
      lv.begin = (int64_t)tl.tasks.size();
      for (int32_t c = 0; c < ncol; ++c) {
        // real: 64 x 8 tiles (9 CTAs per SM keep the FP64 pipe ~96% busy, and
        // the tail of a group is 8x shorter than with 64 x 64 tiles);
        // complex: 64 x 8 only for a group with few wide tiles (under ~4 waves
        // of its CTAs per SM)
        int64_t ntile = 0;
        for (int32_t t = b; t < e; ++t) {
          if (color[t - b] != c) continue;
          const int64_t rb = (h->meta[h->level_sn[t]].r + kTileM - 1) / kTileM;
          ntile += rb * (rb + 1) / 2;
        }
        const int gvar = (!cplx || ntile < 16 * 152) ? 0 : var;
        const int bn = 8 << gvar;
        Range ng, fg;
        for (int part = 0; part < 2; ++part) {
          Range& g = part == 0 ? ng : fg;
          g.begin = (int64_t)tl.tasks.size();
          for (int32_t t = b; t < e; ++t) {
            if (color[t - b] != c) continue;
            const int32_t k = h->level_sn[t];
            const SnMeta& m = h->meta[k];
            const int32_t* C = h->rows.data() + h->rowptr[k];
            int32_t np = m.r;
            const int32_t pk = h->sn_parent[k];
            if (pk >= 0) {
              const int32_t pend = h->meta[pk].f + h->meta[pk].s;
              np = (int32_t)(std::lower_bound(C, C + m.r, pend) - C);
            }
            const int32_t c0 = part == 0 ? 0 : np, c1 = part == 0 ? np : m.r;
            for (int32_t n0 = c0; n0 < c1; n0 += bn) {
              const int32_t ce = std::min(n0 + bn, c1);
              for (int32_t m0 = n0 / kTileM * kTileM; m0 < m.r; m0 += kTileM) tl.tasks.push_back({k, m0, n0, ce});
            }
          }
          g.end = (int64_t)tl.tasks.size();
        }
        if (fg.end > ng.begin) {
          h->schur_near.push_back(ng);
          h->schur_far.push_back(fg);
          h->schur_gvar.push_back((int8_t)gvar);
          for (int32_t t = b; t < e; ++t)
            if (color[t - b] == c) h->schur_gsn.push_back(h->level_sn[t]);
          h->schur_gsn_ptr.push_back((int32_t)h->schur_gsn.size());
        }
      }
      lv.end = (int64_t)tl.tasks.size();
    }
    h->schur_gptr[nl] = (int32_t)h->schur_near.size();
  }
  // counters of the split step-2 output tiles (one per (supernode, m-tile, n-tile))
  h->tctr_total = 0;
  for (int32_t k = 0; k < nsn; ++k) {
    SnMeta& m = h->meta[k];
    m.tctr = (int32_t)h->tctr_total;
    if (m.ksplit > 1) {
      const int64_t bn = 8 << h->t_gemm1.var[k];
      h->tctr_total += (m.r + step2_rows(o) - 1) / step2_rows(o) * ((m.s + bn - 1) / bn);
    }
  }
  // level-local offsets of the step-3 partial products
  h->part_max = 0;
  h->ypart_max = 0;
  h->level_split.assign(nl, 0);
  for (int32_t l = 0; l < nl; ++l) {
    int64_t off = 0, yoff = 0;
    for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
      SnMeta& m = h->meta[h->level_sn[t]];
      m.part = off;
      off += (int64_t)m.nchunk * m.s * m.s;
      m.ypart = yoff;
      if (m.ksplit > 1) {
        yoff += (int64_t)m.ksplit * m.r * m.s;
        h->level_split[l] = 1;
      }
    }
    h->part_max = std::max(h->part_max, off);
    h->ypart_max = std::max(h->ypart_max, yoff);
  }
  // persistent schedule: per level [step-2 tiles][slice reductions][step-3 tiles][finishes]
  h->plist.clear();
  h->plevel_ptr.assign(nl + 1, 0);
  h->pn1.assign(nsn, 0);
  h->pn2.assign(nsn, 0);
  for (int32_t k = 0; k < nsn; ++k) {
    h->pn1[k] = (int32_t)(h->t_pgemm1.per_sn[k].end - h->t_pgemm1.per_sn[k].begin);
    h->pn2[k] = (int32_t)(h->t_pgemm2.per_sn[k].end - h->t_pgemm2.per_sn[k].begin);
  }
  for (int32_t l = 0; l < nl; ++l) {
    h->plevel_ptr[l] = (int64_t)h->plist.size();
    for (int v = 0; v < kNumVar; ++v) {
      const Range rg = h->t_pgemm1.per_lv[(size_t)l * kNumVar + v];
      for (int64_t t = rg.begin; t < rg.end; ++t) h->plist.push_back({P_STEP2, (int16_t)v, (int32_t)t});
    }
    for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t)
      if (h->meta[h->level_sn[t]].ksplit > 1)
        for (int g = 0; g < kReduceGroups; ++g) h->plist.push_back({P_REDUCE, (int16_t)g, h->level_sn[t]});
    for (int v = 0; v < kNumVar; ++v) {
      const Range rg = h->t_pgemm2.per_lv[(size_t)l * kNumVar + v];
      for (int64_t t = rg.begin; t < rg.end; ++t) h->plist.push_back({P_STEP3, (int16_t)v, (int32_t)t});
    }
    for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t)
      for (int q = 0; q < kFinishParts; ++q) h->plist.push_back({P_FINISH, (int16_t)q, h->level_sn[t]});
  }
  h->plevel_ptr[nl] = (int64_t)h->plist.size();
  return PSELINV_OK;
}

}  // namespace psi
