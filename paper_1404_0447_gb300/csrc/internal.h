// Internal declarations of the pselinv library (host analysis, device
// kernels and the C ABI glue).  Not part of the public interface.
#pragma once

#include <cstdint>
#include <climits>
#include <string>
#include <vector>

#include "../../include/pselinv.h"

namespace psi {

// Per-supernode metadata, mirrored on the device.  Element offsets are per
// batch member; member b adds b * (total size of that array).
struct SnMeta {
  int32_t f;       // first column
  int32_t s;       // width
  int32_t r;       // |C| = rows below the diagonal block
  int32_t nchunk;  // row chunks of the step-3 product Lhat^T X_{C,K}
  int64_t panel;   // offset of the (s + r) x s column-major panel (ld = s + r)
  int64_t lhat;    // offset of Lhat_{C,K} (r x s, ld = r) in the normalised-factor buffer
  int64_t linv;    // offset of (L_KK)^{-1} (s x s, ld = s)
  int64_t desc;    // offset of this supernode's r column descriptors
  int64_t part;    // level-local offset of the step-3 partial products (nchunk * s * s)
  int32_t ksplit;  // step-2 partial products (1 = written directly)
  int32_t kchunk;  // rows of C per step-2 partial product
  int64_t ypart;   // level-local offset of the step-2 partial products (ksplit * r * s)
  int32_t kchunk3; // rows of C per step-3 partial product (nchunk = ceil(r / kchunk3))
  int32_t tctr;    // split step 2: first of this supernode's output-tile counters (per batch member)
};

// Where column k of X_{C,C} (k-th row of C) lives: element offset of that
// column inside its supernode J's panel, and the index into relidx such
// that relidx[rel + i] is the row position of C[i] in J's panel for every
// i >= the start of k's block.
struct ColDesc {
  int64_t col;
  int64_t rel;
};

// One unit of work of a grouped launch.  Meaning of m0/n0/c per kernel:
//   tile kernels: output tile origin (m0, n0); c = row chunk (step-3 product) or 0
struct Task {
  int32_t sn;
  int32_t m0;
  int32_t n0;
  int32_t c;
};

// One entry of a level's task list in the persistent schedule.
enum PKind : int16_t { P_STEP2 = 0, P_REDUCE = 1, P_STEP3 = 2, P_FINISH = 3 };
struct PTask {
  int16_t kind;  // PKind
  int16_t var;   // tile variant (STEP2 / STEP3) or column group (REDUCE)
  int32_t idx;   // index into the step-2 / step-3 task array, or the supernode
};
constexpr int kReduceGroups = 8;  // column groups of one slice reduction
constexpr int kFinishParts = 8;   // CTAs (or persistent tasks) sharing one step-3 finish

// Contiguous task ranges [begin, end) for a level and for a supernode.
struct Range {
  int64_t begin = 0, end = 0;
};

constexpr int kMaxWidth = 128;   // widest supernode the kernels accept
constexpr int kMaxWidthLUComplex = 112;  // complex non-symmetric: two packed triangles in shared memory
constexpr int kChunkRows = 512;  // rows per step-3 partial product (before the per-level boost)
constexpr int kTargetTiles = 128 * 152;  // tiles a level should offer the GPU (128 per SM: short tails)
constexpr int kMinSlice2 = 128;   // smallest step-2 slice the per-level boost makes
constexpr int kTileM = 64;       // output tile rows of the grouped GEMMs
constexpr int kTileN = 64;       // output tile columns

// Tile-width variants of the tile GEMMs: BN = 8 << var.
constexpr int kNumVar = 4;
constexpr int kPersistentMaxVar = 0;  // the persistent kernel's tiles stop at BN = 8

// Tile width of an output with `width` columns: the variant with the least
// padded width ceil(width / BN) * BN, the wider tile on ties; complex tiles
// stop at BN = 32 (register budget).
inline int pick_variant(int width, bool cplx, int small_cutoff = -1) {
  const int maxv = cplx ? 2 : 3;
  if (small_cutoff >= 0 && width >= small_cutoff) return maxv;  // wide supernodes: widest tile
  int best = 0;
  int64_t best_pad = INT64_MAX;
  for (int v = 0; v <= maxv; ++v) {
    const int bn = 8 << v;
    const int64_t pad = (int64_t)((width + bn - 1) / bn) * bn;
    if (pad <= best_pad) {
      best_pad = pad;
      best = v;
    }
  }
  return best;
}

// Step-2 tile width: the FP64 kernel's padding-minimal choice; with the bf16
// emulation 64 x 16 tiles for every supernode wider than 8 columns.
inline int step2_variant(int width, bool cplx, const pselinv_opts& o) {
  if (o.fp64_emulation) return width <= 8 ? 0 : 1;
  return pick_variant(width, cplx, o.small_cutoff);
}
// Step-2 tile rows.
inline int step2_rows(const pselinv_opts&) { return kTileM; }

struct TaskList {
  std::vector<Task> tasks;
  std::vector<Range> per_lv;  // [level * kNumVar + var] (level 0 = root level)
  std::vector<Range> per_sn;  // [supernode]
  std::vector<int8_t> var;    // [supernode] tile variant used for that supernode
  Range whole[kNumVar];       // lists built variant-major over all levels
};

}  // namespace psi

struct pselinv_handle {
  pselinv_opts opts{};
  std::string err;

  // ---- symbolic (host) ----
  int64_t n = 0;
  int64_t nnz_a = 0;
  int32_t nsn = 0;
  int32_t nlevels = 0;
  std::vector<int32_t> perm, parent, sn_start, sn_parent, sigma, level_ptr, level_sn;
  std::vector<int32_t> rows, relidx, nblk;
  std::vector<int64_t> rowptr, panel_off, relptr;
  std::vector<int64_t> valmap;  // user entry q -> panel offset of (i, j), i >= j internal
  std::vector<uint8_t> diagmask;  // user entry q is a diagonal entry
  std::vector<uint8_t> flipmap;   // non-symmetric: user entry q lies above the diagonal internally
  std::vector<psi::SnMeta> meta;
  std::vector<psi::ColDesc> desc;
  std::vector<int8_t> level_split;  // level holds a supernode whose step 2 is split
  std::vector<psi::PTask> plist;     // persistent schedule: task lists of all levels
  std::vector<int64_t> plevel_ptr;   // [nlevels+1] offsets into plist
  std::vector<int32_t> pn1, pn2;     // step-2 / step-3 tiles per supernode
  int64_t panel_total = 0, lhat_total = 0, linv_total = 0, part_max = 0, ypart_max = 0;
  int64_t nnz_l = 0, max_r = 0;
  int64_t tctr_total = 0;       // output-tile counters of the split step-2 supernodes (per batch member)
  int32_t max_width = 0;
  double flops_selinv = 0, flops_gemm1 = 0, bytes_selinv = 0;

  // task lists (levels in priority order; supernodes of a level costliest first)
  psi::TaskList t_lhat;   // normalisation tiles (all supernodes)
  psi::TaskList t_gemm1;  // step 2 tiles (with k-slices of split supernodes)
  psi::TaskList t_rect;   // r x s tiles per level, unsplit (adjoint)
  psi::TaskList t_gemm2;  // step 3 partial-product tiles
  psi::TaskList t_trsm;   // factorisation: off-diagonal panel solve tiles
  psi::TaskList t_schur;  // factorisation: Schur-complement update tiles
  // Schur groups: the supernodes of a level split into groups whose update
  // targets are disjoint (no two share a row of C), launched one after the
  // other; level l's groups are g = schur_gptr[l] .. schur_gptr[l+1], each
  // with its tiles updating the parents' columns (schur_near[g]) and those
  // updating the columns above the parents (schur_far[g]), adjacent in the
  // task list (far begins where near ends)
  std::vector<int32_t> schur_gptr;
  std::vector<psi::Range> schur_near, schur_far;
  std::vector<int8_t> schur_gvar;  // tile variant of each group (64 x 8 for groups with few tiles)
  std::vector<int32_t> schur_gsn_ptr, schur_gsn;  // supernodes of each group (pselinv_export_symbolic)
  int32_t schur_var = 0;  // tile variant of the Schur tiles of the larger groups
  std::vector<int8_t> s2var, s3var, trvar;  // step-2 / step-3 / panel-solve tile variant per supernode
  psi::TaskList t_sq;     // s x s tiles of each supernode's diagonal block (adjoint products)
  psi::TaskList t_pgemm1; // persistent schedule: step-2 tiles, widths <= 8 << kPersistentMaxVar
  psi::TaskList t_pgemm2; // persistent schedule: step-3 tiles, widths <= 8 << kPersistentMaxVar

  // ---- device state ----
  int device = -1;
  bool dev_sym = false;     // symbolic arrays uploaded
  bool factored = false;
  bool inverted = false;
  void* d_meta = nullptr;
  void* d_desc = nullptr;
  void* d_relidx = nullptr;
  void* d_valmap = nullptr;
  void* d_diagmask = nullptr;
  void* d_flipmap = nullptr;
  void* d_tasks = nullptr;  // all task arrays back to back
  int64_t off_lhat = 0, off_gemm1 = 0, off_gemm2 = 0, off_trsm = 0, off_schur = 0, off_rect = 0;
  int64_t off_pgemm1 = 0, off_pgemm2 = 0, off_sq = 0;
  void* d_levelsn = nullptr;
  void* d_L = nullptr;      // L panels (unit diagonal implied; D on the diagonal slots)
  void* d_X = nullptr;      // X panels
  void* d_D = nullptr;      // pivots, batch x n
  void* d_lhat = nullptr;   // normalised factor / factor scratch
  void* d_linv = nullptr;   // inverses of the diagonal blocks
  void* d_part = nullptr;   // step-3 partial products (level-local)
  void* d_ypart = nullptr;  // step-2 partial products (level-local)
  void* d_tctr = nullptr;   // int, batch x tctr_total: slices of a step-2 output tile finished (reset to 0)
  void* d_gctr = nullptr;   // int, nsn x kFinishCtas: batch members whose finish part is done (pole sum)
  void* pole_gam = nullptr; // set during pselinv_selinv_pole_sum: its Gamma output
  void* d_status = nullptr; // device status words
  // Bunch-Kaufman pivoted factor (pselinv_factor_bk), batch x n each
  bool pivoted = false;
  void* d_piv = nullptr;    // int32 local original column per pivot position
  void* d_ptype = nullptr;  // int8 pivot type
  void* d_E = nullptr;      // 2x2 off-diagonals
  // non-symmetric handles
  void* d_U = nullptr;      // U panels (U'_{j,i} at position (i, j))
  void* d_XU = nullptr;     // XU panels (X_{j,i} at position (i, j))
  void* d_uhat = nullptr;   // Uhat^T / factor scratch of the U side
  void* d_uinv = nullptr;   // (U'_KK^T)^{-1}
  // FP64 emulation of step 2 on the bf16 tensor cores (opts.fp64_emulation)
  void* d_xs = nullptr;     // slices of the scaled X panels (16 bytes per entry)
  void* d_ls = nullptr;     // slices of the scaled Lhat (16 bytes per entry)
  void* d_sig = nullptr;    // int32 column exponents e_p, batch x n
  void* d_lexp = nullptr;   // int32 column exponents F of B', batch x n
  void* d_gexp = nullptr;   // int32 column exponents G of the scaled X_{C,K} (step 3), batch x n
  void* d_crow = nullptr;   // int32 global rows of every C (rows, at rowptr)
  // adjoint work buffers (allocated on first pselinv_selinv_adjoint)
  void* d_xb = nullptr;     // X-bar, then F-bar (panel layout)
  void* d_lb = nullptr;     // L-bar (panel layout)
  void* d_db = nullptr;     // D-bar
  void* d_zb = nullptr;     // s x s per supernode
  void* d_w1 = nullptr;     // s x s per supernode
  void* d_yb = nullptr;     // r x s per supernode
  void* d_hb = nullptr;     // r x s per supernode
  int64_t device_bytes = 0;
  void* d_plist = nullptr;  // persistent schedule
  void* d_pn = nullptr;     // pn1 then pn2
  void* d_pctr = nullptr;   // c1, c2, cr, cf counters, per-level finish counts, dequeue head
  void* d_snlevel = nullptr; // level per supernode, supernodal parents, level offsets
  void* d_yring = nullptr;   // persistent schedule: kRing level slots of step-2 partials
  void* d_pring = nullptr;   // ... and of step-3 partials
  int pgrid = 0;
  void* pgraph_exec = nullptr;  // cudaGraphExec_t of the PERSISTENT schedule
  int debug_flags = 0;
  void* graph_exec = nullptr;  // cudaGraphExec_t of the LEVEL schedule
  void* graph_stream = nullptr;
  // pselinv_selinv_to_host: per-level copy plan of finished X panels
  std::vector<int64_t> xfer_off, xfer_len;  // element ranges of one panel array
  std::vector<int32_t> xfer_ptr;            // [nlevels + 2]: level l's ranges, then the tail
  void* xfer_stream = nullptr;              // copy stream (cudaStream_t)
  std::vector<void*> xfer_ev;               // [nlevels + 1] cudaEvent_t
  // factorisation look-ahead: high- and low-priority streams, events
  void* fs_hi = nullptr;
  void* fs_lo = nullptr;
  std::vector<void*> fev;
  std::vector<uint8_t> far_after_near;  // per level: far(l) waits for near(l) (factor_impl)

  // optional kernel timing (pselinv_set_timing)
  bool timing = false;
  std::vector<void*> ev_pool;              // cudaEvent_t, reused
  size_t ev_used = 0;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_spans;  // class, (start, stop) event slots
  int64_t launches[4] = {0, 0, 0, 0};
  int64_t graph_launches[4] = {0, 0, 0, 0};  // kernels in the captured graph, per class
};

namespace psi {
// analyze.cpp
int analyze(pselinv_handle* h, int64_t n, const int64_t* colptr, const int32_t* rowind,
            const int32_t* perm);
// Rebuild the tuning-dependent schedule (step-2 slices, task lists,
// partial-product offsets) from h->opts.
int build_schedule(pselinv_handle* h);
}  // namespace psi
