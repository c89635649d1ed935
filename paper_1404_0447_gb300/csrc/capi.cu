// C ABI of the pselinv library: handle lifetime, device buffers, the
// factorisation and selected-inversion schedules, results and errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <functional>
#include <string>

#include "internal.h"
#include "kernels.h"

namespace {

thread_local std::string g_last_err = "no error";
constexpr int kStatusWords = 8;   // [0] first bad pivot column, [1] kind, rest spare
constexpr unsigned long long kPivotKeyUnset = 0x7f7f7f7f7f7f7f7full;  // status words 0-1, see report_pivot

int set_err(pselinv_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  g_last_err = msg;
  return code;
}

int cuda_err(pselinv_handle* h, cudaError_t e, const char* where) {
  return set_err(h, e == cudaErrorMemoryAllocation ? PSELINV_ERR_OOM : PSELINV_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define PSI_CUDA(h, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_err((h), e_, #call); \
  } while (0)

size_t elem_size(const pselinv_handle* h) { return h->opts.dtype == PSELINV_C128 ? 16 : 8; }

psi::Sizes sizes(const pselinv_handle* h) {
  psi::Sizes s;
  s.panel = h->panel_total;
  s.lhat = h->lhat_total;
  s.linv = h->linv_total;
  s.n = h->n;
  s.part = h->part_max;
  s.ypart = h->ypart_max;
  s.batch = h->opts.batch;
  return s;
}

template <class T>
int upload(pselinv_handle* h, void** dst, const std::vector<T>& v) {
  size_t bytes = sizeof(T) * (v.empty() ? 1 : v.size());
  PSI_CUDA(h, cudaMalloc(dst, bytes));
  h->device_bytes += (int64_t)bytes;
  if (!v.empty()) PSI_CUDA(h, cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return PSELINV_OK;
}

int alloc(pselinv_handle* h, void** dst, int64_t bytes) {
  if (bytes < 16) bytes = 16;
  PSI_CUDA(h, cudaMalloc(dst, (size_t)bytes));
  h->device_bytes += bytes;
  return PSELINV_OK;
}

void free_device(pselinv_handle* h) {
  void** ptrs[] = {&h->d_meta, &h->d_desc, &h->d_relidx, &h->d_valmap, &h->d_diagmask, &h->d_tasks, &h->d_levelsn,
                   &h->d_L,    &h->d_X,    &h->d_D,      &h->d_lhat,   &h->d_linv,  &h->d_part, &h->d_ypart,
                   &h->d_status, &h->d_flipmap, &h->d_U, &h->d_XU, &h->d_uhat, &h->d_uinv,
                   &h->d_piv, &h->d_ptype, &h->d_E, &h->d_snlevel, &h->d_yring, &h->d_pring,
                   &h->d_xb,   &h->d_lb,   &h->d_db,     &h->d_zb,     &h->d_w1,    &h->d_yb,   &h->d_hb,
                   &h->d_plist, &h->d_pn,  &h->d_pctr, &h->d_xs, &h->d_ls, &h->d_sig, &h->d_lexp, &h->d_gexp, &h->d_crow,
                   &h->d_tctr, &h->d_gctr};
  for (void** p : ptrs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  for (void* e : h->ev_pool) cudaEventDestroy((cudaEvent_t)e);
  h->ev_pool.clear();
  h->ev_used = 0;
  h->ev_spans.clear();
  if (h->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)h->graph_exec);
  if (h->pgraph_exec) cudaGraphExecDestroy((cudaGraphExec_t)h->pgraph_exec);
  if (h->graph_stream) cudaStreamDestroy((cudaStream_t)h->graph_stream);
  h->graph_exec = h->pgraph_exec = h->graph_stream = nullptr;
  for (void* e : h->xfer_ev) cudaEventDestroy((cudaEvent_t)e);
  h->xfer_ev.clear();
  if (h->xfer_stream) cudaStreamDestroy((cudaStream_t)h->xfer_stream);
  h->xfer_stream = nullptr;
  for (void* e : h->fev) cudaEventDestroy((cudaEvent_t)e);
  h->fev.clear();
  if (h->fs_hi) cudaStreamDestroy((cudaStream_t)h->fs_hi);
  if (h->fs_lo) cudaStreamDestroy((cudaStream_t)h->fs_lo);
  h->fs_hi = h->fs_lo = nullptr;
  h->dev_sym = false;
  h->device_bytes = 0;
}

int upload_schedule(pselinv_handle* h);
int enqueue_selinv(pselinv_handle* h, int mode, cudaStream_t st, bool record,
                   const std::function<int(int32_t)>* after_level = nullptr);
const psi::Task* tasks_at(const pselinv_handle* h, int64_t base, int64_t off);
psi::KArgs kargs(pselinv_handle* h);
psi::KArgs kargs_uside(pselinv_handle* h);
psi::KArgs kargs_step4(pselinv_handle* h);

int ensure_device(pselinv_handle* h) {
  if (h->dev_sym) return PSELINV_OK;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) return set_err(h, PSELINV_ERR_CUDA, "no CUDA device available");
  PSI_CUDA(h, cudaGetDevice(&h->device));
  PSI_CUDA(h, psi::setup_kernels());
  PSI_CUDA(h, psi::persistent_grid(h->opts.dtype, &h->pgrid));
  int rc;
  if ((rc = upload(h, &h->d_desc, h->desc))) return rc;
  if ((rc = upload(h, &h->d_relidx, h->relidx))) return rc;
  if ((rc = upload(h, &h->d_valmap, h->valmap))) return rc;
  if ((rc = upload(h, &h->d_diagmask, h->diagmask))) return rc;
  if ((rc = upload(h, &h->d_levelsn, h->level_sn))) return rc;
  {
    // level of every supernode, supernodal parents, level offsets (persistent schedule)
    std::vector<int32_t> v(2 * (size_t)h->nsn + h->nlevels + 1);
    for (int32_t l = 0; l < h->nlevels; ++l)
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) v[h->level_sn[t]] = l;
    std::copy(h->sn_parent.begin(), h->sn_parent.end(), v.begin() + h->nsn);
    std::copy(h->level_ptr.begin(), h->level_ptr.end(), v.begin() + 2 * (size_t)h->nsn);
    if ((rc = upload(h, &h->d_snlevel, v))) return rc;
  }
  if ((rc = upload_schedule(h))) return rc;
  const int64_t B = h->opts.batch, es = (int64_t)elem_size(h);
  if ((rc = alloc(h, &h->d_L, B * h->panel_total * es))) return rc;
  if ((rc = alloc(h, &h->d_X, B * h->panel_total * es))) return rc;
  if ((rc = alloc(h, &h->d_D, B * h->n * es))) return rc;
  if ((rc = alloc(h, &h->d_lhat, B * h->lhat_total * es))) return rc;
  if ((rc = alloc(h, &h->d_linv, B * h->linv_total * es))) return rc;
  if ((rc = alloc(h, &h->d_status, sizeof(int) * kStatusWords + sizeof(double) * 6 * B))) return rc;
  if (h->opts.unsym) {
    if ((rc = upload(h, &h->d_flipmap, h->flipmap))) return rc;
    if ((rc = alloc(h, &h->d_U, B * h->panel_total * es))) return rc;
    if ((rc = alloc(h, &h->d_XU, B * h->panel_total * es))) return rc;
    if ((rc = alloc(h, &h->d_uhat, B * h->lhat_total * es))) return rc;
    if ((rc = alloc(h, &h->d_uinv, B * h->linv_total * es))) return rc;
  }
  if (h->opts.fp64_emulation) {
    if ((rc = upload(h, &h->d_crow, h->rows))) return rc;
    if ((rc = alloc(h, &h->d_xs, B * h->panel_total * 16))) return rc;
    if ((rc = alloc(h, &h->d_ls, B * h->lhat_total * 16))) return rc;
    if ((rc = alloc(h, &h->d_sig, B * h->n * (int64_t)sizeof(int32_t)))) return rc;
    if ((rc = alloc(h, &h->d_lexp, B * h->n * (int64_t)sizeof(int32_t)))) return rc;
    if ((rc = alloc(h, &h->d_gexp, B * h->n * (int64_t)sizeof(int32_t)))) return rc;
  }
  PSI_CUDA(h, cudaMemset(h->d_status, 0, sizeof(int) * kStatusWords));
  h->dev_sym = true;
  return PSELINV_OK;
}

// Upload the tuning-dependent part (metadata, task lists, partial buffers);
// called again by the autotuner after build_schedule.
int upload_schedule(pselinv_handle* h) {
  int rc;
  void** old[] = {&h->d_meta, &h->d_tasks, &h->d_part, &h->d_ypart, &h->d_plist, &h->d_pn, &h->d_pctr,
                   &h->d_yring, &h->d_pring, &h->d_tctr};
  for (void** p : old)
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  void** graphs[] = {&h->graph_exec, &h->pgraph_exec};
  for (void** g : graphs)
    if (*g) {
      cudaGraphExecDestroy((cudaGraphExec_t)*g);
      *g = nullptr;
    }
  if ((rc = upload(h, &h->d_meta, h->meta))) return rc;
  std::vector<psi::Task> all;
  h->off_lhat = (int64_t)all.size();
  all.insert(all.end(), h->t_lhat.tasks.begin(), h->t_lhat.tasks.end());
  h->off_gemm1 = (int64_t)all.size();
  all.insert(all.end(), h->t_gemm1.tasks.begin(), h->t_gemm1.tasks.end());
  h->off_gemm2 = (int64_t)all.size();
  all.insert(all.end(), h->t_gemm2.tasks.begin(), h->t_gemm2.tasks.end());
  h->off_trsm = (int64_t)all.size();
  all.insert(all.end(), h->t_trsm.tasks.begin(), h->t_trsm.tasks.end());
  h->off_schur = (int64_t)all.size();
  all.insert(all.end(), h->t_schur.tasks.begin(), h->t_schur.tasks.end());
  h->off_rect = (int64_t)all.size();
  all.insert(all.end(), h->t_rect.tasks.begin(), h->t_rect.tasks.end());
  h->off_pgemm1 = (int64_t)all.size();
  all.insert(all.end(), h->t_pgemm1.tasks.begin(), h->t_pgemm1.tasks.end());
  h->off_pgemm2 = (int64_t)all.size();
  all.insert(all.end(), h->t_pgemm2.tasks.begin(), h->t_pgemm2.tasks.end());
  h->off_sq = (int64_t)all.size();
  all.insert(all.end(), h->t_sq.tasks.begin(), h->t_sq.tasks.end());
  if ((rc = upload(h, &h->d_tasks, all))) return rc;
  const int64_t B = h->opts.batch, es = (int64_t)elem_size(h);
  if ((rc = alloc(h, &h->d_part, B * h->part_max * es))) return rc;
  if ((rc = alloc(h, &h->d_ypart, B * h->ypart_max * es))) return rc;
  if ((rc = alloc(h, &h->d_tctr, (int64_t)sizeof(int) * std::max<int64_t>(1, B * h->tctr_total)))) return rc;
  PSI_CUDA(h, cudaMemset(h->d_tctr, 0, sizeof(int) * std::max<int64_t>(1, B * h->tctr_total)));
  if ((rc = upload(h, &h->d_plist, h->plist))) return rc;
  std::vector<int32_t> pn(h->pn1);
  pn.insert(pn.end(), h->pn2.begin(), h->pn2.end());
  if ((rc = upload(h, &h->d_pn, pn))) return rc;
  if ((rc = alloc(h, &h->d_pctr, (int64_t)sizeof(int) * (4 * B * h->nsn + h->nlevels + 1)))) return rc;
  return PSELINV_OK;
}

// Ring of kRing level slots for the persistent schedule's partial products
// (allocated before its graph is captured; dropped with the schedule).
int ensure_ring(pselinv_handle* h) {
  if (h->d_yring) return PSELINV_OK;
  const int64_t B = h->opts.batch, es = (int64_t)elem_size(h);
  int rc;
  if ((rc = alloc(h, &h->d_yring, B * psi::kRing * h->ypart_max * es))) return rc;
  if ((rc = alloc(h, &h->d_pring, B * psi::kRing * h->part_max * es))) return rc;
  return PSELINV_OK;
}

// Persistent schedule: reset the counters, the normalisation pass, then one
// persistent launch over every level.
int enqueue_persistent(pselinv_handle* h, cudaStream_t st) {
  psi::KArgs a = kargs(h);
  const int64_t B = h->opts.batch;
  PSI_CUDA(h, cudaMemsetAsync(h->d_pctr, 0, sizeof(int) * (4 * B * h->nsn + h->nlevels + 1), st));
  PSI_CUDA(h, psi::launch_per_sn(psi::Kern::NormDiag, a, nullptr, h->nsn, st));
  for (int v = 0; v < psi::kNumVar; ++v) {
    const psi::Range r = h->t_lhat.whole[v];
    PSI_CUDA(h, psi::launch_tiles(psi::Kern::Lhat, v, a, tasks_at(h, h->off_lhat, r.begin), r.end - r.begin, st));
  }
  psi::PArgs p;
  int* ctr = (int*)h->d_pctr;
  p.g1 = tasks_at(h, h->off_pgemm1, 0);
  p.g2 = tasks_at(h, h->off_pgemm2, 0);
  p.c1 = ctr;
  p.c2 = ctr + B * h->nsn;
  p.cr = ctr + 2 * B * h->nsn;
  p.cf = ctr + 3 * B * h->nsn;
  p.lvl = ctr + 4 * B * h->nsn;
  p.head = p.lvl + h->nlevels;
  p.n1 = (const int32_t*)h->d_pn;
  p.n2 = (const int32_t*)h->d_pn + h->nsn;
  p.snlevel = (const int32_t*)h->d_snlevel;
  p.snparent = p.snlevel + h->nsn;
  p.level_ptr = p.snparent + h->nsn;
  p.nsn = h->nsn;
  p.yslot = h->ypart_max;
  p.pslot = h->part_max;
  p.spin_ns = h->opts.spin_limit_ns > 0 ? h->opts.spin_limit_ns : 1000000000LL;
  // partial products in the ring: member stride kRing slots
  a.ypart = h->d_yring;
  a.part = h->d_pring;
  a.sz.ypart = psi::kRing * h->ypart_max;
  a.sz.part = psi::kRing * h->part_max;
  const int64_t n = h->plevel_ptr[h->nlevels];
  const int grid = (int)std::min<int64_t>(h->pgrid, n * B);
  PSI_CUDA(h, psi::launch_persistent(a, p, (const psi::PTask*)h->d_plist, n, grid, st));
  return PSELINV_OK;
}

const psi::Task* tasks_at(const pselinv_handle* h, int64_t base, int64_t off) {
  return (const psi::Task*)h->d_tasks + base + off;
}

psi::KArgs kargs(pselinv_handle* h) {
  psi::KArgs a;
  a.dtype = h->opts.dtype;
  a.maxw = h->max_width;
  a.meta = (const psi::SnMeta*)h->d_meta;
  a.desc = (const psi::ColDesc*)h->d_desc;
  a.relidx = (const int32_t*)h->d_relidx;
  a.L = h->d_L;
  a.D = h->d_D;
  a.Linv = h->d_linv;
  a.Lhat = h->d_lhat;
  a.X = h->d_X;
  a.part = h->d_part;
  a.ypart = h->d_ypart;
  a.status = (int*)h->d_status;
  a.tctr = nullptr;  // step-2 slices reduced by the separate kernel unless a schedule sets it
  a.tctr_n = h->tctr_total;
  a.sz = sizes(h);
  a.U = h->d_U;
  a.Uinv = h->d_uinv;
  a.Uhat = nullptr;
  a.XU = h->d_XU;
  a.strict = 0;
  a.piv = h->pivoted ? (const int32_t*)h->d_piv : nullptr;
  a.ptype = h->pivoted ? (const int8_t*)h->d_ptype : nullptr;
  a.E = h->pivoted ? h->d_E : nullptr;
  a.W = nullptr;
  a.gw = nullptr;
  a.gam = nullptr;
  a.gctr = nullptr;
  return a;
}

// Non-symmetric handles: the same kernels run on the U side through swapped
// pointers.  Step 1 of the U side: Uhat^T = (U panel rows C) (U'_KK^T)^{-1}.
psi::KArgs kargs_uside(pselinv_handle* h) {
  psi::KArgs a = kargs(h);
  a.L = h->d_U;
  a.Linv = h->d_uinv;
  a.Lhat = h->d_uhat;
  return a;
}

// Step 4 as step 2 on the transposes: X and XU trade places, Uhat^T replaces Lhat.
psi::KArgs kargs_step4(pselinv_handle* h) {
  psi::KArgs a = kargs(h);
  a.X = h->d_XU;
  a.XU = h->d_X;
  a.Lhat = h->d_uhat;
  return a;
}

// Optional event bracketing of one kernel class (pselinv_set_timing).
struct Timer {
  pselinv_handle* h;
  cudaStream_t st;
  bool on;
  size_t slot(int* rc) {
    if (h->ev_used == h->ev_pool.size()) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) {
        *rc = cuda_err(h, err, "cudaEventCreate");
        return 0;
      }
      h->ev_pool.push_back((void*)e);
    }
    return h->ev_used++;
  }
  // run f() (which enqueues `count` launches of class cls) between two events
  template <class F>
  int run(int cls, int64_t count, F&& f) {
    if (count <= 0) return PSELINV_OK;
    int rc = PSELINV_OK;
    size_t a = 0, b = 0;
    if (on) {
      a = slot(&rc);
      if (rc) return rc;
      PSI_CUDA(h, cudaEventRecord((cudaEvent_t)h->ev_pool[a], st));
    }
    PSI_CUDA(h, f());
    if (on) {
      b = slot(&rc);
      if (rc) return rc;
      PSI_CUDA(h, cudaEventRecord((cudaEvent_t)h->ev_pool[b], st));
      h->ev_spans.push_back({cls, {a, b}});
    }
    h->launches[cls] += count;
    return PSELINV_OK;
  }
};

// Enqueue one schedule of the selected inversion on stream st.
int enqueue_selinv(pselinv_handle* h, int mode, cudaStream_t st, bool record,
                   const std::function<int(int32_t)>* after_level) {
  using psi::Kern;
  const psi::KArgs a = kargs(h);
  const auto* lsn = (const int32_t*)h->d_levelsn;
  Timer tm{h, st, record};
  int rc;
  // normalisation pass: every supernode at once (Algorithm 3, first loop)
  int64_t nlhat_launch = 0;
  for (int v = 0; v < psi::kNumVar; ++v) nlhat_launch += h->t_lhat.whole[v].end > h->t_lhat.whole[v].begin;
  const bool unsym = h->opts.unsym != 0;
  const psi::KArgs au = unsym ? kargs_uside(h) : a;   // U side of step 1
  const psi::KArgs a4 = unsym ? kargs_step4(h) : a;   // step 4
  psi::KArgs a3 = a;                                  // step 3: Uhat_{K,C} X_{C,K}
  if (unsym) a3.Lhat = h->d_uhat;
  rc = tm.run(0, (1 + nlhat_launch) * (unsym ? 2 : 1) - (unsym ? 1 : 0), [&] {
    cudaError_t e = psi::launch_per_sn(unsym ? Kern::NormDiagLU : Kern::NormDiag, a, nullptr, h->nsn, st);
    for (int side = 0; side < (unsym ? 2 : 1); ++side)
      for (int v = 0; v < psi::kNumVar && e == cudaSuccess; ++v) {
        const psi::Range r = h->t_lhat.whole[v];
        e = psi::launch_tiles(Kern::Lhat, v, side ? au : a, tasks_at(h, h->off_lhat, r.begin), r.end - r.begin,
                              st);
      }
    return e;
  });
  if (rc) return rc;
  // FP64 emulation of step 2: B' slices before it, X slices after the level
  const bool emul = h->opts.fp64_emulation != 0;
  const psi::EmArgs em{h->d_xs,         h->d_ls, (int32_t*)h->d_sig, (int32_t*)h->d_lexp, (int32_t*)h->d_gexp,
                       (const int32_t*)h->d_crow, h->n};
  // one step: the given supernodes, with per-variant task ranges of steps 2 and 3
  // maxr: the largest |C| among the step's supernodes
  // FP64 step 2 (and step 4): the last slice CTA of each split output tile
  // sums the slices in order (tile counters); the emulated step 2 keeps the
  // separate reduction kernel
  psi::KArgs a2 = a, a4f = a4;
  if (!emul) {
    a2.tctr = a4f.tctr = (int*)h->d_tctr;
  }
  // step-3 finish; pselinv_selinv_pole_sum: with the pole sum of its entries
  psi::KArgs af = a;
  if (h->pole_gam) {
    af.gw = (const double*)((int*)h->d_status + kStatusWords) + 2 * h->opts.batch;
    af.gam = h->pole_gam;
    af.gctr = (int*)h->d_gctr;
  }
  auto step = [&](const int32_t* sns, int nsn_step, const psi::Range* r1, const psi::Range* r2, bool split,
                  int maxr) {
    int n1 = (split && emul) ? 1 : 0, n2 = 0, e;
    for (int v = 0; v < psi::kNumVar; ++v) {
      n1 += r1[v].end > r1[v].begin;
      n2 += r2[v].end > r2[v].begin;
    }
    // step 2 (ka = a), or step 4 (ka = a4) of a non-symmetric handle
    auto gemm1 = [&](const psi::KArgs& ka) {
      return tm.run(1, n1 + (emul ? 1 : 0), [&] {
        cudaError_t x = emul ? psi::launch_em_split_lhat(ka, em, sns, nsn_step, maxr, st) : cudaSuccess;
        for (int v = 0; v < psi::kNumVar && x == cudaSuccess; ++v)
          x = emul ? psi::launch_em_gemm1(v, ka, em, tasks_at(h, h->off_gemm1, r1[v].begin), r1[v].end - r1[v].begin,
                                          st)
                   : psi::launch_tiles(Kern::Gemm1, v, ka, tasks_at(h, h->off_gemm1, r1[v].begin),
                                       r1[v].end - r1[v].begin, st);
        if (split && emul && x == cudaSuccess) x = psi::launch_per_sn(Kern::Gemm1Reduce, ka, sns, nsn_step, st);
        return x;
      });
    };
    if ((e = gemm1(a2))) return e;
    // step 3 partial products; emulated: slices of diag(2^-e_C) X_{C,K} first
    if ((e = tm.run(2, n2 + (emul && n2 > 0 ? 1 : 0), [&] {
           cudaError_t x = emul ? psi::launch_em_split_xck(a, em, sns, nsn_step, maxr, st) : cudaSuccess;
           for (int v = 0; v < psi::kNumVar && x == cudaSuccess; ++v)
             x = emul ? psi::launch_em_gemm2(v, a, em, tasks_at(h, h->off_gemm2, r2[v].begin),
                                             r2[v].end - r2[v].begin, st)
                      : psi::launch_tiles(Kern::Gemm2, v, a3, tasks_at(h, h->off_gemm2, r2[v].begin),
                                          r2[v].end - r2[v].begin, st);
           return x;
         })))
      return e;
    if ((e = tm.run(3, (nsn_step > 0) * (emul ? 2 : 1), [&] {
           cudaError_t x = psi::launch_per_sn(Kern::DiagFinal, af, sns, nsn_step, st);
           if (emul && x == cudaSuccess) x = psi::launch_em_split_x(a, em, sns, nsn_step, st);
           return x;
         })))
      return e;
    // step 4 reuses the step-2 partial-product buffer after step 2's reduction
    return unsym ? gemm1(a4f) : PSELINV_OK;
  };
  if (mode == PSELINV_PLAIN) {
    // one supernode per launch, reverse postorder (descending index)
    std::vector<int32_t> pos(h->nsn);
    for (int32_t t = 0; t < h->nsn; ++t) pos[h->level_sn[t]] = t;
    for (int32_t k = h->nsn - 1; k >= 0; --k) {
      psi::Range r1[psi::kNumVar], r2[psi::kNumVar];
      r1[h->t_gemm1.var[k]] = h->t_gemm1.per_sn[k];
      r2[h->t_gemm2.var[k]] = h->t_gemm2.per_sn[k];
      if ((rc = step(lsn + pos[k], 1, r1, r2, h->meta[k].ksplit > 1, h->meta[k].r))) return rc;
    }
  } else {
    for (int32_t l = 0; l < h->nlevels; ++l) {
      int maxr = 0;
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) maxr = std::max(maxr, h->meta[h->level_sn[t]].r);
      if ((rc = step(lsn + h->level_ptr[l], h->level_ptr[l + 1] - h->level_ptr[l],
                     &h->t_gemm1.per_lv[(size_t)l * psi::kNumVar], &h->t_gemm2.per_lv[(size_t)l * psi::kNumVar],
                     h->level_split[l] != 0, maxr)))
        return rc;
      if (after_level && (rc = (*after_level)(l))) return rc;
    }
  }
  return PSELINV_OK;
}

// Copy plan of pselinv_selinv_to_host.  The panels of a level's supernodes
// are final once that level's step 3 (and step 4) have run.  Levels whose
// supernodes form at most kXferRuns runs of adjacent panels are copied right
// after the level; the rest (the deep levels with thousands of scattered
// small supernodes) are copied after the last level as runs merged across
// gaps of already-copied panels shorter than kXferGap elements.
void build_xfer_plan(pselinv_handle* h) {
  constexpr int64_t kXferRuns = 1024, kXferGap = 1 << 17;
  h->xfer_off.clear();
  h->xfer_len.clear();
  h->xfer_ptr.assign(1, 0);
  std::vector<uint8_t> done(h->nsn, 0);
  std::vector<int32_t> s;
  for (int32_t l = 0; l < h->nlevels; ++l) {
    s.assign(h->level_sn.begin() + h->level_ptr[l], h->level_sn.begin() + h->level_ptr[l + 1]);
    std::sort(s.begin(), s.end());
    int64_t runs = s.empty() ? 0 : 1;
    for (size_t q = 1; q < s.size(); ++q) runs += s[q] != s[q - 1] + 1;
    if (runs <= kXferRuns) {
      for (size_t q = 0; q < s.size();) {
        size_t e = q + 1;
        while (e < s.size() && s[e] == s[e - 1] + 1) ++e;
        h->xfer_off.push_back(h->panel_off[s[q]]);
        h->xfer_len.push_back(h->panel_off[s[e - 1] + 1] - h->panel_off[s[q]]);
        for (size_t t = q; t < e; ++t) done[s[t]] = 1;
        q = e;
      }
    }
    h->xfer_ptr.push_back((int32_t)h->xfer_off.size());
  }
  int64_t b = -1, e = -1;  // current tail range [b, e) in elements
  for (int32_t k = 0; k < h->nsn; ++k) {
    if (done[k]) continue;
    const int64_t kb = h->panel_off[k], ke = h->panel_off[k + 1];
    if (b >= 0 && kb - e < kXferGap) {
      e = ke;
    } else {
      if (b >= 0) {
        h->xfer_off.push_back(b);
        h->xfer_len.push_back(e - b);
      }
      b = kb;
      e = ke;
    }
  }
  if (b >= 0) {
    h->xfer_off.push_back(b);
    h->xfer_len.push_back(e - b);
  }
  h->xfer_ptr.push_back((int32_t)h->xfer_off.size());
}

}  // namespace

namespace psi {
// Error text for entry points that have no handle (read by pselinv_last_error(NULL)).
void set_global_error(const std::string& msg) { g_last_err = msg; }
}  // namespace psi

extern "C" {

void pselinv_default_opts(pselinv_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dtype = PSELINV_F64;
  o->batch = 1;
  o->max_sn_width = psi::kMaxWidth;
  o->relax = PSELINV_RELAX_AMALG;
  o->small_cutoff = -1;
  o->split_k_rows = 1024;
  o->debug_checks = 0;
  o->unsym = 0;
  o->spin_limit_ns = 1000000000LL;
}

int pselinv_analyze(int64_t n, const int64_t* h_colptr, const int32_t* h_rowind, const int32_t* h_perm,
                    const pselinv_opts* opts, pselinv_handle** out) {
  if (!out) return set_err(nullptr, PSELINV_ERR_ARG, "out is NULL");
  *out = nullptr;
  auto* h = new pselinv_handle();
  if (opts)
    h->opts = *opts;
  else
    pselinv_default_opts(&h->opts);
  if (h->opts.dtype != PSELINV_F64 && h->opts.dtype != PSELINV_C128) {
    delete h;
    return set_err(nullptr, PSELINV_ERR_ARG, "dtype must be PSELINV_F64 or PSELINV_C128");
  }
  if (h->opts.batch < 1 || h->opts.batch > 65535) {
    delete h;
    return set_err(nullptr, PSELINV_ERR_ARG, "batch must be 1..65535");
  }
  int rc = psi::analyze(h, n, h_colptr, h_rowind, h_perm);
  if (rc != PSELINV_OK) {
    g_last_err = h->err;
    delete h;
    return rc;
  }
  *out = h;
  return PSELINV_OK;
}

int pselinv_analyze_batch(int32_t k, const int64_t* h_n, const int64_t* const* h_colptr,
                          const int32_t* const* h_rowind, const int32_t* const* h_perm, const pselinv_opts* opts,
                          pselinv_handle** out) {
  if (!out) return set_err(nullptr, PSELINV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (k < 1 || !h_n || !h_colptr || !h_rowind) return set_err(nullptr, PSELINV_ERR_ARG, "bad batch arguments");
  int64_t N = 0, NNZ = 0;
  for (int32_t b = 0; b < k; ++b) {
    if (h_n[b] < 1 || !h_colptr[b] || !h_rowind[b])
      return set_err(nullptr, PSELINV_ERR_ARG, "member " + std::to_string(b) + ": bad size or NULL pattern");
    N += h_n[b];
    NNZ += h_colptr[b][h_n[b]];
  }
  if (N >= ((int64_t)1 << 31)) return set_err(nullptr, PSELINV_ERR_ARG, "total order too large");
  std::vector<int64_t> cp(N + 1);
  std::vector<int32_t> ri(NNZ), perm(N);
  int64_t c0 = 0, q0 = 0;
  for (int32_t b = 0; b < k; ++b) {
    const int64_t nb = h_n[b];
    const int64_t* bcp = h_colptr[b];
    if (bcp[0] != 0) return set_err(nullptr, PSELINV_ERR_NOT_LOWER, "member " + std::to_string(b) + ": colptr[0] != 0");
    for (int64_t j = 0; j < nb; ++j) cp[c0 + j] = q0 + bcp[j];
    for (int64_t q = 0; q < bcp[nb]; ++q) {
      const int32_t r = h_rowind[b][q];
      if (r < 0 || r >= nb) return set_err(nullptr, PSELINV_ERR_NOT_LOWER, "member " + std::to_string(b) + ": row out of range");
      ri[q0 + q] = (int32_t)(c0 + r);
    }
    for (int64_t j = 0; j < nb; ++j) {
      const int32_t u = (h_perm && h_perm[b]) ? h_perm[b][j] : (int32_t)j;
      if (u < 0 || u >= nb) return set_err(nullptr, PSELINV_ERR_NOT_LOWER, "member " + std::to_string(b) + ": bad perm");
      perm[c0 + j] = (int32_t)(c0 + u);
    }
    c0 += nb;
    q0 += bcp[nb];
  }
  cp[N] = q0;
  return pselinv_analyze(N, cp.data(), ri.data(), perm.data(), opts, out);
}

}  // extern "C"

namespace {
// The factorisation's two streams (high and low priority) and its events
// (2 per level + 3), created on first use.
int ensure_factor_streams(pselinv_handle* h) {
  if (!h->fs_hi) {
    int least = 0, greatest = 0;
    PSI_CUDA(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    cudaStream_t s;
    PSI_CUDA(h, cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest));
    h->fs_hi = s;
    PSI_CUDA(h, cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, least));
    h->fs_lo = s;
  }
  const size_t need = 3 * (size_t)h->nlevels + 3;
  while (h->fev.size() < need) {
    cudaEvent_t e;
    PSI_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->fev.push_back(e);
  }
  if (h->far_after_near.empty()) {
    // Per level l: does far(l) wait for near(l), so that level l - 1's
    // diagonal blocks start beside it?  A diagonal-block CTA does not fit on
    // an SM beside resident Schur tiles, so when far(l) is already running the
    // next diagonal blocks wait for its end.  Worth it when far(l) is short
    // against the next level's diagonal blocks and panel solves (model: FP64
    // work at 1 TFLOP/s; a diagonal block of width w, 345 us (w / 128)^3 +
    // 30 us, measured on the 1,024-thread kernel).
    const int32_t nl = h->nlevels;
    std::vector<double> t_far(nl, 0.0), t_next(nl, 0.0);
    for (int32_t l = 0; l < nl; ++l) {
      double far = 0.0, solve = 0.0;
      int wmax = 0;
      for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) {
        const psi::SnMeta& m = h->meta[h->level_sn[t]];
        far += (double)m.r * (m.r + 1) * m.s;
        solve += (double)m.r * m.s * m.s;
        wmax = std::max(wmax, m.s);
      }
      const double w = wmax / 128.0;
      t_far[l] = far / 1e12;
      t_next[l] = 345e-6 * w * w * w + 30e-6 + solve / 1e12;
    }
    h->far_after_near.assign(nl, 0);
    for (int32_t l = 1; l < nl; ++l) h->far_after_near[l] = t_far[l] < 4.0 * t_next[l - 1];
  }
  return PSELINV_OK;
}

// Supernodal factorisation, level by level from the leaves.  Symmetric:
// A = L D L^T.  Non-symmetric (d_upper set): A = L D U', the U side running
// the same panel-solve, copy and Schur kernels through swapped pointers.
int factor_impl(pselinv_handle* h, const void* d_lower, const void* d_upper, cudaStream_t st, bool bk = false) {
  const psi::Sizes sz = sizes(h);
  const int64_t B = h->opts.batch;
  const bool unsym = d_upper != nullptr;
  h->factored = h->inverted = false;
  if (bk && !h->d_piv) {
    int rc;
    if ((rc = alloc(h, &h->d_piv, B * h->n * (int64_t)sizeof(int32_t)))) return rc;
    if ((rc = alloc(h, &h->d_ptype, B * h->n))) return rc;
    if ((rc = alloc(h, &h->d_E, B * h->n * (int64_t)elem_size(h)))) return rc;
  }
  h->pivoted = bk;
  PSI_CUDA(h, cudaMemsetAsync(h->d_L, 0, elem_size(h) * B * h->panel_total, st));
  if (unsym) PSI_CUDA(h, cudaMemsetAsync(h->d_U, 0, elem_size(h) * B * h->panel_total, st));
  PSI_CUDA(h, cudaMemsetAsync(h->d_status, 0x7f, 2 * sizeof(int), st));  // pivot key: unset
  PSI_CUDA(h, cudaMemsetAsync((int*)h->d_status + 2, 0, sizeof(int) * (kStatusWords - 2), st));
  psi::KArgs a = kargs(h);
  a.XU = nullptr;
  if (unsym)
    PSI_CUDA(h, psi::launch_scatter_values_lu(h->opts.dtype, d_lower, d_upper, (const int64_t*)h->d_valmap,
                                              (const uint8_t*)h->d_flipmap, h->nnz_a, h->d_L, h->d_U, sz, st));
  else
    PSI_CUDA(h, psi::launch_scatter_values(h->opts.dtype, d_lower, (const int64_t*)h->d_valmap, h->nnz_a, h->d_L,
                                           sz, st));
  // L side: L_{C,K} = A_{C,K} (L_KK^{-T} or U'_KK^{-1}) D^{-1} into lhat, copied to the L panels
  psi::KArgs al = a;
  if (unsym) al.Linv = h->d_uinv;
  // U side: U'_{K,C}^T = A_{K,C}^T L_KK^{-T} D^{-1} into uhat, copied to the U panels
  psi::KArgs au = a;
  au.L = h->d_U;
  au.Lhat = h->d_uhat;
  // the panel solves also keep W = L_{C,K} D_K (U'_{K,C}^T D_K; with pivots,
  // D_K's 1 x 1 and 2 x 2 blocks), in the X (XU) panels, which a factorisation
  // withdraws, as the Schur update's first operand
  al.W = h->d_X;
  if (unsym) au.W = h->d_XU;
  // Schur: L_{C,K} D U'_{K,C} into the L panels, and its strict upper part (transposed) into the U panels
  psi::KArgs sl = a, su = a;
  sl.W = al.W;
  su.W = au.W;
  if (unsym) {
    sl.Uhat = h->d_uhat;
    su.L = h->d_U;
    su.Lhat = h->d_uhat;
    su.Uhat = h->d_lhat;
    su.strict = 1;
  }
  // Two streams (look-ahead): `hi` (high priority) runs each level's
  // diagonal blocks, panel solves and "near" Schur tiles (those updating the
  // parents' columns, which the next level's diagonal blocks need); `lo` runs
  // the "far" Schur tiles (columns above the parents), so the far update of
  // level l overlaps the diagonal blocks and panel solves of level l - 1.
  // Events keep every target's updates in a fixed order: far(l) waits for
  // the panel solves of l (its operand); near(l) waits for far(l + 1), the
  // last earlier update of level l - 1's panels.  On levels whose far update
  // is short (far_after_near), far(l) waits for near(l) instead, so that the
  // diagonal blocks of l - 1 get their SMs before far(l)'s tiles fill them;
  // every target sees its updates in the same order either way.
  int rc;
  if ((rc = ensure_factor_streams(h))) return rc;
  cudaStream_t hi = (cudaStream_t)h->fs_hi, lo = (cudaStream_t)h->fs_lo;
  // [0] start, [1 + l] solves of l, [1 + nl + l] far of l, [3 + 2 nl + l] near of l
  cudaEvent_t* ev = (cudaEvent_t*)h->fev.data();
  const int32_t nl = h->nlevels;
  PSI_CUDA(h, cudaEventRecord(ev[0], st));
  PSI_CUDA(h, cudaStreamWaitEvent(hi, ev[0], 0));
  PSI_CUDA(h, cudaStreamWaitEvent(lo, ev[0], 0));
  const auto* lsn = (const int32_t*)h->d_levelsn;
  auto schur = [&](const std::vector<psi::Range>& grp, int32_t g0, int32_t g1, cudaStream_t s) -> cudaError_t {
    for (int side = 0; side < (unsym ? 2 : 1); ++side)
      for (int32_t g = g0; g < g1; ++g) {  // group by group: disjoint targets inside a group, no atomics
        const psi::Range r = grp[g];
        if (r.end == r.begin) continue;
        cudaError_t e = psi::launch_tiles(psi::Kern::Schur, h->schur_gvar[g], side ? su : sl,
                                          tasks_at(h, h->off_schur, r.begin), r.end - r.begin, s);
        if (e != cudaSuccess) return e;
      }
    return cudaSuccess;
  };
  for (int32_t l = nl - 1; l >= 0; --l) {
    const int32_t* sns = lsn + h->level_ptr[l];
    const int nsl = h->level_ptr[l + 1] - h->level_ptr[l];
    // a level holding a wide supernode gets wide CTAs: the column steps of the
    // diagonal factorisation are serial, the work inside each step is not
    int wmax = 0;
    for (int32_t t = h->level_ptr[l]; t < h->level_ptr[l + 1]; ++t) wmax = std::max(wmax, h->meta[h->level_sn[t]].s);
    // shared memory sized for the level's widest block: several CTAs per SM on levels of narrow supernodes
    psi::KArgs ad = a;
    ad.maxw = wmax;
    PSI_CUDA(h, psi::launch_per_sn(unsym ? psi::Kern::FactorDiagLU
                                         : bk  ? psi::Kern::FactorDiagBK
                                               : psi::Kern::FactorDiag,
                                   ad, sns, nsl, hi, wmax >= 64 ? 1024 : 256));
    for (int side = 0; side < (unsym ? 2 : 1); ++side) {
      const psi::KArgs& ka = side ? au : al;
      for (int v = 0; v < psi::kNumVar; ++v) {
        const psi::Range r = h->t_trsm.per_lv[(size_t)l * psi::kNumVar + v];
        PSI_CUDA(h, psi::launch_tiles(psi::Kern::Trsm, v, ka, tasks_at(h, h->off_trsm, r.begin), r.end - r.begin,
                                      hi));
      }
      // the pivoted copy-back also divides the scratch by 2x2 blocks of D, which the Schur
      // update reads: per level; the plain one only fills the panels (nothing in the
      // factorisation reads L_{C,K} from them): once for all levels, after the loop
      if (bk) PSI_CUDA(h, psi::launch_per_sn(psi::Kern::CopyBackBK, ka, sns, nsl, hi));
    }
    if (h->far_after_near[l]) {
      if (l + 1 < nl) PSI_CUDA(h, cudaStreamWaitEvent(hi, ev[1 + nl + l + 1], 0));
      PSI_CUDA(h, schur(h->schur_near, h->schur_gptr[l], h->schur_gptr[l + 1], hi));
      PSI_CUDA(h, cudaEventRecord(ev[3 + 2 * nl + l], hi));
      PSI_CUDA(h, cudaStreamWaitEvent(lo, ev[3 + 2 * nl + l], 0));
      PSI_CUDA(h, schur(h->schur_far, h->schur_gptr[l], h->schur_gptr[l + 1], lo));
      PSI_CUDA(h, cudaEventRecord(ev[1 + nl + l], lo));
    } else {
      PSI_CUDA(h, cudaEventRecord(ev[1 + l], hi));
      PSI_CUDA(h, cudaStreamWaitEvent(lo, ev[1 + l], 0));
      PSI_CUDA(h, schur(h->schur_far, h->schur_gptr[l], h->schur_gptr[l + 1], lo));
      PSI_CUDA(h, cudaEventRecord(ev[1 + nl + l], lo));
      if (l + 1 < nl) PSI_CUDA(h, cudaStreamWaitEvent(hi, ev[1 + nl + l + 1], 0));
      PSI_CUDA(h, schur(h->schur_near, h->schur_gptr[l], h->schur_gptr[l + 1], hi));
    }
  }
  PSI_CUDA(h, cudaEventRecord(ev[1 + 2 * nl], hi));
  PSI_CUDA(h, cudaStreamWaitEvent(st, ev[1 + 2 * nl], 0));
  PSI_CUDA(h, cudaEventRecord(ev[2 + 2 * nl], lo));
  PSI_CUDA(h, cudaStreamWaitEvent(st, ev[2 + 2 * nl], 0));
  if (!bk)
    for (int side = 0; side < (unsym ? 2 : 1); ++side)
      PSI_CUDA(h, psi::launch_per_sn(psi::Kern::CopyBack, side ? au : al, lsn, h->nsn, st));
  // no host synchronisation: the first bad pivot stays in status words 0-1
  // until the next factorisation and is reported by pselinv_sync_status (and
  // by pselinv_logdet, which synchronises anyway)
  h->factored = true;
  return PSELINV_OK;
}

// Pivot report of the last factorisation from status words 0-1 (host copy):
// an error with the first bad column, and the handle back to "not factored".
int pivot_error(pselinv_handle* h, unsigned long long key) {
  if (key == kPivotKeyUnset) return PSELINV_OK;
  h->factored = h->inverted = false;
  const bool zero = (key & 3) == 1;
  return set_err(h, zero ? PSELINV_ERR_ZERO_PIVOT : PSELINV_ERR_NONFINITE,
                 std::string(zero ? "zero" : "non-finite") + " pivot at column " + std::to_string(key >> 2) +
                     " (internal order)");
}
}  // namespace

extern "C" {

int pselinv_factor(pselinv_handle* h, const void* d_values, void* stream) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  if (!d_values) return set_err(h, PSELINV_ERR_ARG, "values pointer is NULL");
  if (h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "non-symmetric handle: use pselinv_factor_unsym");
  int rc = ensure_device(h);
  if (rc) return rc;
  return factor_impl(h, d_values, nullptr, (cudaStream_t)stream);
}

int pselinv_factor_bk(pselinv_handle* h, const void* d_values, void* stream) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  if (!d_values) return set_err(h, PSELINV_ERR_ARG, "values pointer is NULL");
  if (h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "pivoting is for symmetric handles");
  int rc = ensure_device(h);
  if (rc) return rc;
  return factor_impl(h, d_values, nullptr, (cudaStream_t)stream, true);
}

int pselinv_get_pivots(pselinv_handle* h, int32_t* h_piv, int8_t* h_type, void* stream) {
  if (!h || !h_piv || !h_type) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (!h->factored || !h->pivoted) return set_err(h, PSELINV_ERR_STATE, "no pivoted factor");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cnt = (size_t)h->opts.batch * (size_t)h->n;
  PSI_CUDA(h, cudaMemcpyAsync(h_piv, h->d_piv, cnt * sizeof(int32_t), cudaMemcpyDefault, st));
  PSI_CUDA(h, cudaMemcpyAsync(h_type, h->d_ptype, cnt, cudaMemcpyDefault, st));
  PSI_CUDA(h, cudaStreamSynchronize(st));
  return PSELINV_OK;
}

int pselinv_factor_unsym(pselinv_handle* h, const void* d_lower, const void* d_upper, void* stream) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  if (!d_lower || !d_upper) return set_err(h, PSELINV_ERR_ARG, "values pointer is NULL");
  if (!h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "symmetric handle: use pselinv_factor");
  int rc = ensure_device(h);
  if (rc) return rc;
  return factor_impl(h, d_lower, d_upper, (cudaStream_t)stream);
}

int pselinv_selinv(pselinv_handle* h, int32_t mode, void* stream) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  if (mode != PSELINV_PLAIN && mode != PSELINV_LEVEL && mode != PSELINV_GRAPH && mode != PSELINV_PERSISTENT)
    return set_err(h, PSELINV_ERR_ARG, "bad selinv mode");
  if (!h->factored) return set_err(h, PSELINV_ERR_STATE, "selinv called before a successful factor");
  if (mode == PSELINV_PERSISTENT && h->opts.unsym)
    return set_err(h, PSELINV_ERR_ARG, "the PERSISTENT schedule is for symmetric handles");
  if (h->opts.fp64_emulation) {
    if (mode == PSELINV_PERSISTENT)
      return set_err(h, PSELINV_ERR_ARG, "fp64_emulation runs with the PLAIN, LEVEL and GRAPH schedules");
    if (h->pivoted) return set_err(h, PSELINV_ERR_STATE, "fp64_emulation needs the pivot-free factor (SPD A)");
    if (h->max_r > (int64_t)1 << 21) return set_err(h, PSELINV_ERR_ARG, "fp64_emulation: |C| above 2^21");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == PSELINV_PERSISTENT) {
    int rrc = ensure_ring(h);
    if (rrc) return rrc;
    if (!h->pgraph_exec) {
      if (!h->graph_stream) {
        cudaStream_t cs;
        PSI_CUDA(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        h->graph_stream = cs;
      }
      cudaStream_t cs = (cudaStream_t)h->graph_stream;
      PSI_CUDA(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      int rc = enqueue_persistent(h, cs);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return cuda_err(h, e, "cudaStreamEndCapture");
      cudaGraphExec_t ex;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_err(h, e, "cudaGraphInstantiate");
      h->pgraph_exec = ex;
    }
    if (h->debug_flags & 2) {  // arm one never-satisfied wait (status word 3)
      PSI_CUDA(h, cudaMemsetAsync((int*)h->d_status + 3, 1, 1, st));
      h->debug_flags &= ~2;
    }
    PSI_CUDA(h, cudaGraphLaunch((cudaGraphExec_t)h->pgraph_exec, st));
    h->launches[1] += h->nlevels;
  } else if (mode != PSELINV_GRAPH) {
    int rc = enqueue_selinv(h, mode, st, h->timing);
    if (rc) return rc;
  } else {
    if (!h->graph_exec) {
      if (!h->graph_stream) {
        cudaStream_t ns;
        PSI_CUDA(h, cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking));
        h->graph_stream = ns;
      }
      cudaStream_t cs = (cudaStream_t)h->graph_stream;
      PSI_CUDA(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      int64_t before[4];
      std::memcpy(before, h->launches, sizeof(before));
      int rc = enqueue_selinv(h, PSELINV_LEVEL, cs, false);
      for (int q = 0; q < 4; ++q) {
        h->graph_launches[q] = h->launches[q] - before[q];
        h->launches[q] = before[q];
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return cuda_err(h, e, "cudaStreamEndCapture");
      cudaGraphExec_t ex;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_err(h, e, "cudaGraphInstantiate");
      h->graph_exec = ex;
    }
    PSI_CUDA(h, cudaGraphLaunch((cudaGraphExec_t)h->graph_exec, st));
    for (int q = 0; q < 4; ++q) h->launches[q] += h->graph_launches[q];
  }
  h->inverted = true;
  return PSELINV_OK;
}

int pselinv_selinv_to_host(pselinv_handle* h, void* h_x, void* h_xu, void* stream) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  if (!h_x) return set_err(h, PSELINV_ERR_ARG, "h_x is NULL");
  if (h_xu && !h->opts.unsym) return set_err(h, PSELINV_ERR_ARG, "h_xu is for non-symmetric handles");
  if (!h->factored) return set_err(h, PSELINV_ERR_STATE, "selinv called before a successful factor");
  cudaStream_t st = (cudaStream_t)stream;
  if (h->xfer_ev.empty()) {
    build_xfer_plan(h);
    cudaStream_t cs;
    PSI_CUDA(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    h->xfer_stream = cs;
    for (int32_t l = 0; l <= h->nlevels; ++l) {
      cudaEvent_t ev;
      PSI_CUDA(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      h->xfer_ev.push_back((void*)ev);
    }
  }
  cudaStream_t cs = (cudaStream_t)h->xfer_stream;
  const size_t es = elem_size(h), pitch = es * (size_t)h->panel_total;
  const int B = h->opts.batch;
  auto copy_ranges = [&](int32_t q0, int32_t q1) -> int {
    for (int32_t q = q0; q < q1; ++q)
      for (int side = 0; side < (h_xu ? 2 : 1); ++side) {
        const size_t o = es * (size_t)h->xfer_off[q];
        char* dst = (char*)(side ? h_xu : h_x) + o;
        const char* src = (const char*)(side ? h->d_XU : h->d_X) + o;
        PSI_CUDA(h, cudaMemcpy2DAsync(dst, pitch, src, pitch, es * (size_t)h->xfer_len[q], B, cudaMemcpyDefault,
                                      cs));
      }
    return PSELINV_OK;
  };
  // the copy stream must not start before the work already queued on st
  PSI_CUDA(h, cudaEventRecord((cudaEvent_t)h->xfer_ev[h->nlevels], st));
  PSI_CUDA(h, cudaStreamWaitEvent(cs, (cudaEvent_t)h->xfer_ev[h->nlevels], 0));
  const std::function<int(int32_t)> after = [&](int32_t l) -> int {
    if (h->xfer_ptr[l + 1] == h->xfer_ptr[l]) return PSELINV_OK;
    PSI_CUDA(h, cudaEventRecord((cudaEvent_t)h->xfer_ev[l], st));
    PSI_CUDA(h, cudaStreamWaitEvent(cs, (cudaEvent_t)h->xfer_ev[l], 0));
    return copy_ranges(h->xfer_ptr[l], h->xfer_ptr[l + 1]);
  };
  int rc = enqueue_selinv(h, PSELINV_LEVEL, st, h->timing, &after);
  if (rc) return rc;
  // tail: after the last level
  PSI_CUDA(h, cudaEventRecord((cudaEvent_t)h->xfer_ev[h->nlevels], st));
  PSI_CUDA(h, cudaStreamWaitEvent(cs, (cudaEvent_t)h->xfer_ev[h->nlevels], 0));
  if ((rc = copy_ranges(h->xfer_ptr[h->nlevels], h->xfer_ptr[h->nlevels + 1]))) return rc;
  // st completes after every copy
  PSI_CUDA(h, cudaEventRecord((cudaEvent_t)h->xfer_ev[h->nlevels], cs));
  PSI_CUDA(h, cudaStreamWaitEvent(st, (cudaEvent_t)h->xfer_ev[h->nlevels], 0));
  h->inverted = true;
  return PSELINV_OK;
}

int pselinv_sync_status(pselinv_handle* h, void* stream) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  if (!h->dev_sym) return PSELINV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int status[kStatusWords];
  PSI_CUDA(h, cudaMemcpyAsync(status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost, st));
  PSI_CUDA(h, cudaStreamSynchronize(st));
  {
    unsigned long long key;
    std::memcpy(&key, status, sizeof(key));
    const int rc = pivot_error(h, key);
    if (rc) return rc;
  }
  if (status[2]) {
    PSI_CUDA(h, cudaMemsetAsync((int*)h->d_status + 2, 0, 2 * sizeof(int), st));
    PSI_CUDA(h, cudaStreamSynchronize(st));
    h->inverted = false;
    return set_err(h, PSELINV_ERR_TIMEOUT,
                   "a bounded device wait of the persistent schedule ran out; that selinv's results are invalid");
  }
  if (status[psi::kEmStatusWord]) {
    const int em = status[psi::kEmStatusWord];
    PSI_CUDA(h, cudaMemsetAsync((int*)h->d_status + psi::kEmStatusWord, 0, sizeof(int), st));
    PSI_CUDA(h, cudaStreamSynchronize(st));
    h->inverted = false;
    return set_err(h, PSELINV_ERR_RANGE,
                   "FP64 emulation: X is not positive definite (a diagonal entry <= 0 or a scaled entry out of "
                   "range); that selinv's results are invalid -- use fp64_emulation = 0");
  }
  return PSELINV_OK;
}

int pselinv_set_debug(pselinv_handle* h, int32_t flags) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  h->debug_flags = flags;
  return PSELINV_OK;
}

int pselinv_get_panels(pselinv_handle* h, int32_t which, void* d_out, void* stream) {
  // d_out may be device or host memory: cudaMemcpyDefault resolves it (UVA)
  if (!h || !d_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  const int nwhich = h->opts.unsym ? 4 : 2;
  if (which < 0 || which >= nwhich)
    return set_err(h, PSELINV_ERR_ARG, "which must be 0 (X), 1 (L), or for non-symmetric handles 2 (XU), 3 (U)");
  if ((which == 0 || which == 2) && !h->inverted) return set_err(h, PSELINV_ERR_STATE, "no selected inverse yet");
  if ((which == 1 || which == 3) && !h->factored) return set_err(h, PSELINV_ERR_STATE, "no factor yet");
  const size_t bytes = elem_size(h) * (size_t)h->opts.batch * (size_t)h->panel_total;
  const void* src[4] = {h->d_X, h->d_L, h->d_XU, h->d_U};
  PSI_CUDA(h, cudaMemcpyAsync(d_out, src[which], bytes, cudaMemcpyDefault, (cudaStream_t)stream));
  return PSELINV_OK;
}

int pselinv_get_selected(pselinv_handle* h, void* d_out, void* stream) {
  if (!h || !d_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (!h->inverted) return set_err(h, PSELINV_ERR_STATE, "no selected inverse yet");
  if (h->opts.unsym)
    PSI_CUDA(h, psi::launch_gather_values_lu(h->opts.dtype, h->d_X, h->d_XU, (const int64_t*)h->d_valmap,
                                             (const uint8_t*)h->d_flipmap, h->nnz_a, 0, d_out, sizes(h),
                                             (cudaStream_t)stream));
  else
    PSI_CUDA(h, psi::launch_gather_values(h->opts.dtype, h->d_X, (const int64_t*)h->d_valmap, nullptr, h->nnz_a,
                                          d_out, sizes(h), (cudaStream_t)stream));
  return PSELINV_OK;
}

int pselinv_get_selected_upper(pselinv_handle* h, void* d_out, void* stream) {
  if (!h || !d_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (!h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "symmetric handle: use pselinv_get_selected");
  if (!h->inverted) return set_err(h, PSELINV_ERR_STATE, "no selected inverse yet");
  PSI_CUDA(h, psi::launch_gather_values_lu(h->opts.dtype, h->d_X, h->d_XU, (const int64_t*)h->d_valmap,
                                           (const uint8_t*)h->d_flipmap, h->nnz_a, 1, d_out, sizes(h),
                                           (cudaStream_t)stream));
  return PSELINV_OK;
}

int pselinv_logdet_grad(pselinv_handle* h, void* d_out, void* stream) {
  if (!h || !d_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "symmetric handles only");
  if (!h->inverted) return set_err(h, PSELINV_ERR_STATE, "no selected inverse yet");
  PSI_CUDA(h, psi::launch_gather_values(h->opts.dtype, h->d_X, (const int64_t*)h->d_valmap,
                                        (const uint8_t*)h->d_diagmask, h->nnz_a, d_out, sizes(h),
                                        (cudaStream_t)stream));
  return PSELINV_OK;
}

int pselinv_pole_sum(pselinv_handle* h, const double* h_weights, void* d_out, void* stream) {
  if (!h || !h_weights || !d_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "symmetric handles only");
  if (!h->inverted) return set_err(h, PSELINV_ERR_STATE, "no selected inverse yet");
  cudaStream_t st = (cudaStream_t)stream;
  const int B = h->opts.batch;
  double* w = (double*)((int*)h->d_status + kStatusWords) + 2 * B;
  const size_t wbytes = sizeof(double) * (h->opts.dtype == PSELINV_C128 ? 2 : 1) * B;
  PSI_CUDA(h, cudaMemcpyAsync(w, h_weights, wbytes, cudaMemcpyHostToDevice, st));
  PSI_CUDA(h, psi::launch_pole_sum(h->opts.dtype, h->d_X, h->panel_total, B, w, d_out, st));
  return PSELINV_OK;
}

int pselinv_selinv_pole_sum(pselinv_handle* h, const double* h_weights, void* d_out, void* stream) {
  if (!h || !h_weights || !d_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "symmetric handles only");
  if (!h->factored) return set_err(h, PSELINV_ERR_STATE, "selinv called before a successful factor");
  if (h->pivoted) return set_err(h, PSELINV_ERR_STATE, "the fused pole sum needs the pivot-free factor");
  if (h->opts.fp64_emulation) return set_err(h, PSELINV_ERR_ARG, "the fused pole sum runs without fp64_emulation");
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if (!h->d_gctr) {
    const int64_t n = (int64_t)h->nsn * psi::kFinishCtas;
    if ((rc = alloc(h, &h->d_gctr, (int64_t)sizeof(int) * n))) return rc;
    PSI_CUDA(h, cudaMemsetAsync(h->d_gctr, 0, sizeof(int) * n, st));
  }
  const int B = h->opts.batch;
  double* w = (double*)((int*)h->d_status + kStatusWords) + 2 * B;
  const size_t wbytes = sizeof(double) * (h->opts.dtype == PSELINV_C128 ? 2 : 1) * B;
  PSI_CUDA(h, cudaMemcpyAsync(w, h_weights, wbytes, cudaMemcpyHostToDevice, st));
  h->pole_gam = d_out;
  rc = enqueue_selinv(h, PSELINV_LEVEL, st, h->timing);
  h->pole_gam = nullptr;
  if (rc) return rc;
  h->inverted = true;
  return PSELINV_OK;
}

int pselinv_trace_sum(pselinv_handle* h, const void* d_values, double* h_out, void* stream) {
  if (!h || !d_values || !h_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "symmetric handles only");
  if (!h->inverted) return set_err(h, PSELINV_ERR_STATE, "no selected inverse yet");
  cudaStream_t st = (cudaStream_t)stream;
  const int B = h->opts.batch;
  double* dev = (double*)((int*)h->d_status + kStatusWords) + 4 * B;
  PSI_CUDA(h, psi::launch_trace_sum(h->opts.dtype, h->d_X, h->panel_total, (const int64_t*)h->d_valmap,
                                    (const uint8_t*)h->d_diagmask, d_values, h->nnz_a, B, dev, st));
  const bool cz = h->opts.dtype == PSELINV_C128;
  std::vector<double> tmp((cz ? 2 : 1) * B);
  PSI_CUDA(h, cudaMemcpyAsync(tmp.data(), dev, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, st));
  PSI_CUDA(h, cudaStreamSynchronize(st));
  for (int b = 0; b < B; ++b) {
    h_out[2 * b] = tmp[(cz ? 2 : 1) * b];
    h_out[2 * b + 1] = cz ? tmp[2 * b + 1] : 0.0;
  }
  return PSELINV_OK;
}

int pselinv_logdet(pselinv_handle* h, double* h_out, void* stream) {
  if (!h || !h_out) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (!h->factored) return set_err(h, PSELINV_ERR_STATE, "no factor yet");
  cudaStream_t st = (cudaStream_t)stream;
  double* dev = (double*)((int*)h->d_status + kStatusWords);
  PSI_CUDA(h, psi::launch_logdet(h->opts.dtype, h->d_D, h->n, dev, h->opts.batch, st,
                                  h->pivoted ? (const int8_t*)h->d_ptype : nullptr, h->pivoted ? h->d_E : nullptr));
  PSI_CUDA(h, cudaMemcpyAsync(h_out, dev, sizeof(double) * 2 * h->opts.batch, cudaMemcpyDeviceToHost, st));
  unsigned long long key = 0;
  PSI_CUDA(h, cudaMemcpyAsync(&key, h->d_status, sizeof(key), cudaMemcpyDeviceToHost, st));
  PSI_CUDA(h, cudaStreamSynchronize(st));
  return pivot_error(h, key);
}

int pselinv_selinv_adjoint(pselinv_handle* h, const void* d_G, int32_t g_kind, void* d_gradA, void* stream) {
  using psi::AdjKern;
  using psi::AdjSn;
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  if (!d_G || !d_gradA) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (g_kind != PSELINV_G_SYMMETRIC && g_kind != PSELINV_G_PANEL) return set_err(h, PSELINV_ERR_ARG, "bad g_kind");
  if (h->opts.unsym) return set_err(h, PSELINV_ERR_STATE, "symmetric handles only");
  if (h->pivoted) return set_err(h, PSELINV_ERR_STATE, "the adjoint needs the pivot-free factor (pselinv_factor)");
  if (!h->inverted) return set_err(h, PSELINV_ERR_STATE, "selinv_adjoint needs a prior pselinv_selinv");
  const int64_t B = h->opts.batch, es = (int64_t)elem_size(h);
  int rc;
  if (!h->d_xb) {
    if ((rc = alloc(h, &h->d_xb, B * h->panel_total * es))) return rc;
    if ((rc = alloc(h, &h->d_lb, B * h->panel_total * es))) return rc;
    if ((rc = alloc(h, &h->d_db, B * h->n * es))) return rc;
    if ((rc = alloc(h, &h->d_zb, B * h->linv_total * es))) return rc;
    if ((rc = alloc(h, &h->d_w1, B * h->linv_total * es))) return rc;
    if ((rc = alloc(h, &h->d_yb, B * h->lhat_total * es))) return rc;
    if ((rc = alloc(h, &h->d_hb, B * h->lhat_total * es))) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  psi::AdjArgs a;
  a.k = kargs(h);
  a.k.tctr = (int*)h->d_tctr;  // split X_CC Yb and (W + W^T) L_CK summed by their last slice CTA
  a.G = d_G;
  a.g_kind = g_kind;
  a.Xb = h->d_xb;
  a.Lb = h->d_lb;
  a.Db = h->d_db;
  a.Zb = h->d_zb;
  a.W1 = h->d_w1;
  a.Yb = h->d_yb;
  a.Hb = h->d_hb;
  // recompute (L_KK)^{-1} and Lhat from L (step 1) instead of trusting stored copies
  {
    psi::KArgs na = a.k;
    na.X = nullptr;
    PSI_CUDA(h, psi::launch_per_sn(psi::Kern::NormDiag, na, nullptr, h->nsn, st));
    for (int v = 0; v < psi::kNumVar; ++v) {
      const psi::Range r = h->t_lhat.whole[v];
      PSI_CUDA(h, psi::launch_tiles(psi::Kern::Lhat, v, na, tasks_at(h, h->off_lhat, r.begin), r.end - r.begin, st));
    }
  }
  PSI_CUDA(h, cudaMemsetAsync(h->d_lb, 0, B * h->panel_total * es, st));
  PSI_CUDA(h, cudaMemsetAsync(h->d_db, 0, B * h->n * es, st));
  PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::Seed, a, nullptr, h->nsn, st));
  const auto* lsn = (const int32_t*)h->d_levelsn;
  auto tiles = [&](AdjKern k, const psi::TaskList& tl, int64_t off, int32_t l) -> cudaError_t {
    for (int v = 0; v < psi::kNumVar; ++v) {
      const psi::Range r = tl.per_lv[(size_t)l * psi::kNumVar + v];
      cudaError_t e = psi::launch_adj_tiles(k, v, a, tasks_at(h, off, r.begin), r.end - r.begin, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // reverse sweep of the selected inversion, leaves -> root
  for (int32_t l = h->nlevels - 1; l >= 0; --l) {
    const int32_t* sns = lsn + h->level_ptr[l];
    const int nsl = h->level_ptr[l + 1] - h->level_ptr[l];
    PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::Zbar, a, sns, nsl, st));
    PSI_CUDA(h, tiles(AdjKern::Ybar, h->t_rect, h->off_rect, l));
    PSI_CUDA(h, tiles(AdjKern::Lhbar, h->t_gemm1, h->off_gemm1, l));  // step-2 slices of C
    // per Schur group, its near and far tiles (adjacent, different target levels) as one launch
    for (int32_t g = h->schur_gptr[l]; g < h->schur_gptr[l + 1]; ++g) {
      const int64_t b0 = h->schur_near[g].begin, b1 = h->schur_far[g].end;
      PSI_CUDA(h, psi::launch_adj_tiles(AdjKern::Syr2k, h->schur_gvar[g], a, tasks_at(h, h->off_schur, b0), b1 - b0, st));
    }
    PSI_CUDA(h, tiles(AdjKern::LbarOff, h->t_rect, h->off_rect, l));
    PSI_CUDA(h, tiles(AdjKern::Vpart, h->t_gemm2, h->off_gemm2, l));
    PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::SumParts, a, sns, nsl, st));
    // diagonal step: the s x s products as tiles over all supernodes of the level
    PSI_CUDA(h, tiles(AdjKern::Dr1, h->t_sq, h->off_sq, l));
    PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::Dr2, a, sns, nsl, st));
    PSI_CUDA(h, tiles(AdjKern::Dr3, h->t_sq, h->off_sq, l));
    PSI_CUDA(h, tiles(AdjKern::Dr4, h->t_sq, h->off_sq, l));
  }
  // adjoint of the supernodal LDL^T, root -> leaves
  PSI_CUDA(h, cudaMemsetAsync(h->d_xb, 0, B * h->panel_total * es, st));
  PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::Ev, a, nullptr, h->nsn, st));
  for (int32_t l = 0; l < h->nlevels; ++l) {
    const int32_t* sns = lsn + h->level_ptr[l];
    const int nsl = h->level_ptr[l + 1] - h->level_ptr[l];
    PSI_CUDA(h, tiles(AdjKern::T1, h->t_gemm1, h->off_gemm1, l));
    PSI_CUDA(h, tiles(AdjKern::Q, h->t_rect, h->off_rect, l));
    PSI_CUDA(h, tiles(AdjKern::Rpart, h->t_gemm2, h->off_gemm2, l));
    PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::SumParts, a, sns, nsl, st));
    PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::Df1, a, sns, nsl, st));
    PSI_CUDA(h, tiles(AdjKern::Df2, h->t_sq, h->off_sq, l));
    PSI_CUDA(h, tiles(AdjKern::Df3, h->t_sq, h->off_sq, l));
    PSI_CUDA(h, tiles(AdjKern::Df4, h->t_sq, h->off_sq, l));
    PSI_CUDA(h, psi::launch_adj_per_sn(AdjSn::Df5, a, sns, nsl, st));
  }
  PSI_CUDA(h, psi::launch_gather_values(h->opts.dtype, h->d_xb, (const int64_t*)h->d_valmap, nullptr, h->nnz_a,
                                        d_gradA, sizes(h), st));
  return PSELINV_OK;
}

int pselinv_set_timing(pselinv_handle* h, int32_t enable) {
  if (!h) return set_err(nullptr, PSELINV_ERR_ARG, "handle is NULL");
  h->timing = enable != 0;
  h->ev_used = 0;
  h->ev_spans.clear();
  for (int q = 0; q < 4; ++q) h->launches[q] = 0;
  return PSELINV_OK;
}

int pselinv_get_timing(pselinv_handle* h, double* h_ms, int64_t* h_launches) {
  if (!h || !h_ms || !h_launches) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  double ms[PSELINV_NTIMERS] = {0, 0, 0, 0};
  for (const auto& sp : h->ev_spans) {
    cudaEvent_t a = (cudaEvent_t)h->ev_pool[sp.second.first], b = (cudaEvent_t)h->ev_pool[sp.second.second];
    PSI_CUDA(h, cudaEventSynchronize(b));
    float t = 0.f;
    PSI_CUDA(h, cudaEventElapsedTime(&t, a, b));
    ms[sp.first] += t;
  }
  for (int q = 0; q < PSELINV_NTIMERS; ++q) {
    h_ms[q] = ms[q];
    h_launches[q] = h->launches[q];
    h->launches[q] = 0;
  }
  h->ev_used = 0;
  h->ev_spans.clear();
  return PSELINV_OK;
}

int pselinv_autotune(pselinv_handle* h, int32_t* h_best, double* h_best_ms, void* stream) {
  if (!h || !h_best || !h_best_ms) return set_err(h, PSELINV_ERR_ARG, "NULL argument");
  if (!h->factored) return set_err(h, PSELINV_ERR_STATE, "autotune needs a factored handle");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  PSI_CUDA(h, cudaEventCreate(&e0));
  PSI_CUDA(h, cudaEventCreate(&e1));
  const bool timing = h->timing;
  h->timing = false;
  auto measure = [&](int32_t split, int32_t cutoff, double* ms) -> int {
    h->opts.split_k_rows = split;
    h->opts.small_cutoff = cutoff;
    int rc = psi::build_schedule(h);
    if (!rc) rc = upload_schedule(h);
    if (!rc) rc = enqueue_selinv(h, PSELINV_LEVEL, st, false);  // warm-up
    double best = 1e300;
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      float t = 0.f;
      cudaError_t e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) rc = enqueue_selinv(h, PSELINV_LEVEL, st, false);
      if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (!rc && e != cudaSuccess) rc = cuda_err(h, e, "autotune timing");
      if (t < best) best = t;
    }
    *ms = best;
    return rc;
  };
  int32_t best_split = h->opts.split_k_rows, best_cut = h->opts.small_cutoff;
  double best_ms = 1e300, ms = 0;
  int rc = PSELINV_OK;
  for (int32_t split : {0, 512, 1024, 2048, 4096}) {
    if ((rc = measure(split, best_cut, &ms))) break;
    if (ms < best_ms) {
      best_ms = ms;
      best_split = split;
    }
  }
  for (int32_t cut : {-1, 32, 64}) {
    if (rc || cut == best_cut) continue;
    if ((rc = measure(best_split, cut, &ms))) break;
    if (ms < best_ms) {
      best_ms = ms;
      best_cut = cut;
    }
  }
  // third coordinate: the per-level tile target of the slice shrinking
  int32_t best_tiles = h->opts.level_tiles;
  for (int32_t tiles : {32 * 152, 64 * 152, 128 * 152}) {
    if (rc || tiles == (best_tiles > 0 ? best_tiles : psi::kTargetTiles)) continue;
    h->opts.level_tiles = tiles;
    if ((rc = measure(best_split, best_cut, &ms))) break;
    if (ms < best_ms) {
      best_ms = ms;
      best_tiles = tiles;
    }
  }
  if (!rc) {
    h->opts.split_k_rows = best_split;
    h->opts.small_cutoff = best_cut;
    h->opts.level_tiles = best_tiles;
    rc = psi::build_schedule(h);
    if (!rc) rc = upload_schedule(h);
  }
  // last: the schedule mode on the chosen parameters (LEVEL was measured above)
  int32_t best_mode = PSELINV_LEVEL;
  for (int32_t mode : {PSELINV_GRAPH, PSELINV_PERSISTENT}) {
    if (rc || (mode == PSELINV_PERSISTENT && (h->opts.unsym || h->opts.fp64_emulation))) continue;
    rc = pselinv_selinv(h, mode, st);  // warm-up (captures the graph)
    double best = 1e300;
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      float t = 0.f;
      cudaError_t e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) rc = pselinv_selinv(h, mode, st);
      if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (!rc && e != cudaSuccess) rc = cuda_err(h, e, "autotune timing");
      if (t < best) best = t;
    }
    if (!rc && mode == PSELINV_PERSISTENT) rc = pselinv_sync_status(h, st);
    if (!rc && best < best_ms) {
      best_ms = best;
      best_mode = mode;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->timing = timing;
  if (rc) return rc;
  h_best[0] = best_split;
  h_best[1] = best_cut;
  h_best[2] = best_tiles > 0 ? best_tiles : psi::kTargetTiles;
  h_best[3] = best_mode;
  *h_best_ms = best_ms;
  h->inverted = false;  // X was overwritten by the trial runs
  return PSELINV_OK;
}

int pselinv_get_info(const pselinv_handle* h, pselinv_info* info) {
  if (!h || !info) return PSELINV_ERR_ARG;
  info->n = h->n;
  info->nnz_a = h->nnz_a;
  info->nnz_l = h->nnz_l;
  info->panel_entries = h->panel_total;
  info->relidx_len = (int64_t)h->relidx.size();
  info->nsn = h->nsn;
  info->nlevels = h->nlevels;
  info->max_width = h->max_width;
  info->batch = h->opts.batch;
  info->max_r = h->max_r;
  info->flops_selinv = h->flops_selinv;
  info->flops_gemm1 = h->flops_gemm1;
  info->bytes_selinv = h->bytes_selinv;
  // device memory held now (the autotuner reallocates the schedule buffers)
  if (h->dev_sym) {
    const int64_t B = h->opts.batch, es = (int64_t)elem_size(h), tasks =
        (int64_t)(h->t_lhat.tasks.size() + h->t_gemm1.tasks.size() + h->t_gemm2.tasks.size() +
                  h->t_trsm.tasks.size() + h->t_schur.tasks.size() + h->t_rect.tasks.size() +
                  h->t_pgemm1.tasks.size() + h->t_pgemm2.tasks.size() + h->t_sq.tasks.size());
    int64_t bytes = (int64_t)(sizeof(psi::SnMeta) * h->meta.size() + sizeof(psi::ColDesc) * h->desc.size() +
                              4 * h->relidx.size() + 8 * h->valmap.size() + h->diagmask.size() +
                              4 * h->level_sn.size()) +
                    (int64_t)sizeof(psi::Task) * tasks +
                    B * es * (2 * h->panel_total + h->n + h->lhat_total + h->linv_total + h->part_max + h->ypart_max);
    if (h->d_xb) bytes += B * es * (2 * h->panel_total + h->n + 2 * h->linv_total + 2 * h->lhat_total);
    if (h->opts.unsym) bytes += h->flipmap.size() + B * es * (2 * h->panel_total + h->lhat_total + h->linv_total);
    if (h->d_yring) bytes += B * es * psi::kRing * (h->ypart_max + h->part_max);
    bytes += 4 * (2 * (int64_t)h->nsn + h->nlevels + 1);  // level / parent / level offsets
    info->device_bytes = bytes;
  } else {
    info->device_bytes = 0;
  }
  return PSELINV_OK;
}

int pselinv_export_symbolic(const pselinv_handle* h, pselinv_symbolic* v) {
  if (!h || !v) return PSELINV_ERR_ARG;
  v->n = h->n;
  v->nsn = h->nsn;
  v->nlevels = h->nlevels;
  v->perm = h->perm.data();
  v->parent = h->parent.data();
  v->sn_start = h->sn_start.data();
  v->sn_parent = h->sn_parent.data();
  v->sigma = h->sigma.data();
  v->rowptr = h->rowptr.data();
  v->rows = h->rows.data();
  v->panel_off = h->panel_off.data();
  v->relptr = h->relptr.data();
  v->relidx = h->relidx.data();
  v->nblk = h->nblk.data();
  v->level_ptr = h->level_ptr.data();
  v->level_sn = h->level_sn.data();
  v->ngroups = (int32_t)h->schur_near.size();
  v->group_ptr = h->schur_gptr.data();
  v->group_sn_ptr = h->schur_gsn_ptr.data();
  v->group_sn = h->schur_gsn.data();
  return PSELINV_OK;
}

void pselinv_destroy(pselinv_handle* h) {
  if (!h) return;
  free_device(h);
  delete h;
}

const char* pselinv_last_error(const pselinv_handle* h) {
  if (h) return h->err.empty() ? "no error" : h->err.c_str();
  return g_last_err.c_str();
}

}  // extern "C"
