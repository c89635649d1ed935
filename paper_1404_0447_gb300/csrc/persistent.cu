// Persistent schedule: one launch runs the whole level loop of Algorithm 3
// -- step-2 tiles (all tile widths and k-slices), slice reductions, step-3
// partial-product tiles and the step-3 finish of every supernode -- from one
// task list in level order (levels top-down, costliest supernode first
// inside a level).  CTAs take tasks with an atomic counter; there is no
// barrier between levels (the dynamic scheduling of Section 3.3 on one GPU):
//   * a supernode's step 2 reads X of its ancestors that hold rows of C, and
//     C_K lies in P and C_P for the supernodal parent P, so it waits only
//     until P's X is final (all finish parts of P done);
//   * partial products live in a ring of kRing level slots, so a level's
//     step 2 also waits until the level kRing above it has finished;
//   * reductions, step-3 tiles and the finish wait on per-supernode
//     completion counters of the tasks before them.
//
// Why this cannot deadlock: every CTA of the grid is resident; tasks are
// taken in list order and a task only waits on tasks earlier in the list,
// which are held by running CTAs that themselves only wait on still earlier
// tasks; the earliest unfinished task never waits.  Every wait is bounded in
// time (spin_limit_ns of %globaltimer); when one runs out the kernel raises a
// timeout flag in the status words, every other wait returns at once, the
// remaining tasks are skipped and the launch ends.  pselinv_sync_status
// reports it.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"
#include "selinv_steps.cuh"
#include "tile_gemm.cuh"

namespace psi {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until *ctr >= target (device-scope acquire), bounded by
// limit_ns; returns false for the whole CTA on timeout or abort.
__device__ bool cta_wait(const int* ctr, int target, long long limit_ns, int* status) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile const int* abort_flag = status + 2;
    const unsigned long long t0 = global_ns();
    for (;;) {
      if (*abort_flag) {
        ok = 0;
        break;
      }
      if (atomicAdd(const_cast<int*>(ctr), 0) >= target) break;
      if ((long long)(global_ns() - t0) > limit_ns) {
        atomicExch(status + 2, 1);  // timeout: abort the launch
        ok = 0;
        break;
      }
      __nanosleep(200);
    }
    __threadfence();
  }
  __syncthreads();
  const int r = ok;
  __syncthreads();
  return r != 0;
}

// Publish a finished task: all threads' writes, then a device-scope fence,
// then the counter.
__device__ void cta_signal(int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1);
  }
}

// Publish one finished finish part: the supernode's and the level's counters.
__device__ void cta_signal2(int* ctr1, int* ctr2) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr1, 1);
    atomicAdd(ctr2, 1);
  }
}

// 8 CTAs per SM for real data (64 registers, 20 KB of shared memory each), 5 for complex; 10 (48
// registers) measured slower.
template <class T>
__global__ void __launch_bounds__(TG_THREADS, Sc<T>::P == 1 ? 8 : 5) k_persistent(KArgs a, PArgs p, const PTask* __restrict__ list,
                                                           int64_t ntask) {
  constexpr int MAXBN = 8 << kPersistentMaxVar;  // the task lists stop at this width
  __shared__ __align__(16) unsigned char smraw[sizeof(TileSmem<T, MAXBN>)];
  __shared__ long long s_item;
  const int batch = a.sz.batch;
  const long long total = ntask * batch;
  int* status = a.status;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(p.head, 1);
    __syncthreads();
    const long long item = s_item;
    __syncthreads();
    if (item >= total) break;
    const PTask pt = list[item / batch];
    const int b = (int)(item % batch);
    const bool aborted = *(volatile int*)(status + 2) != 0;
    if (aborted) continue;  // drain the list
    const int64_t cb = (int64_t)b * p.nsn;
    switch (pt.kind) {
      case P_STEP2: {
        const Task tk = p.g1[pt.idx];
        const int k = tk.sn, l = p.snlevel[k];
        if (l >= kRing) {  // the level using the same partial-product slot has finished
          const int lr = l - kRing;
          const int target = (p.level_ptr[lr + 1] - p.level_ptr[lr]) * kFinishParts * batch;
          if (!cta_wait(p.lvl + lr, target, p.spin_ns, status)) break;
        }
        const int par = p.snparent[k];
        if (par >= 0 && !cta_wait(p.cf + cb + par, kFinishParts, p.spin_ns, status)) break;
        const int64_t yoff = (int64_t)(l % kRing) * p.yslot;
        if (pt.var == 0)
          step2_tile<T, 8>(a, tk, b, *reinterpret_cast<TileSmem<T, 8>*>(smraw), yoff);
        else
          step2_tile<T, MAXBN>(a, tk, b, *reinterpret_cast<TileSmem<T, MAXBN>*>(smraw), yoff);
        cta_signal(p.c1 + cb + k);
        break;
      }
      case P_REDUCE: {
        const int k = pt.idx;
        if (!cta_wait(p.c1 + cb + k, p.n1[k], p.spin_ns, status)) break;
        step2_reduce<T>(a, k, b, pt.var, kReduceGroups, true, (int64_t)(p.snlevel[k] % kRing) * p.yslot);
        cta_signal(p.cr + cb + k);
        break;
      }
      case P_STEP3: {
        const Task tk = p.g2[pt.idx];
        const int k = tk.sn;
        const bool split = a.meta[k].ksplit > 1;
        if (!cta_wait(split ? p.cr + cb + k : p.c1 + cb + k, split ? kReduceGroups : p.n1[k], p.spin_ns, status))
          break;
        const int64_t poff = (int64_t)(p.snlevel[k] % kRing) * p.pslot;
        if (pt.var == 0)
          step3_tile<T, 8>(a, tk, b, *reinterpret_cast<TileSmem<T, 8>*>(smraw), true, poff);
        else
          step3_tile<T, MAXBN>(a, tk, b, *reinterpret_cast<TileSmem<T, MAXBN>*>(smraw), true, poff);
        cta_signal(p.c2 + cb + k);
        break;
      }
      default: {  // P_FINISH
        const int k = pt.idx, l = p.snlevel[k];
        int target = p.n2[k];
        const int* ctr = p.c2 + cb + k;
        if (target == 0) {  // no step-3 tiles (r = 0): nothing to wait for
          ctr = nullptr;
        }
        // failure-detection support: one armed finish task waits for a
        // completion that never comes (status word 3, set by the host)
        __shared__ int inject;
        if (threadIdx.x == 0) inject = atomicExch(status + 3, 0);
        __syncthreads();
        if (inject) {
          ctr = p.c2 + cb + k;
          target = p.n2[k] + 1;
        }
        if (ctr && !cta_wait(ctr, target, p.spin_ns, status)) break;
        step3_finish<T>(a, k, b, pt.var, kFinishParts, true, (int64_t)(l % kRing) * p.pslot);
        cta_signal2(p.cf + cb + k, p.lvl + l);
        break;
      }
    }
  }
}

cudaError_t launch_persistent(const KArgs& a, const PArgs& p, const PTask* list, int64_t ntask, int grid,
                              cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  if (a.dtype == PSELINV_C128)
    k_persistent<Cplx><<<grid, TG_THREADS, 0, st>>>(a, p, list, ntask);
  else
    k_persistent<double><<<grid, TG_THREADS, 0, st>>>(a, p, list, ntask);
  return cudaGetLastError();
}

cudaError_t persistent_grid(int dtype, int* grid) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = dtype == PSELINV_C128
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<Cplx>, TG_THREADS, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<double>, TG_THREADS, 0);
  if (e == cudaSuccess) *grid = sms * (per > 0 ? per : 1);
  return e;
}

}  // namespace psi
