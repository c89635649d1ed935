// Persistent schedule: one launch per level of Algorithm 2 runs every piece
// of that level's work -- step-2 tiles (all tile widths and k-slices), the
// slice reductions, step-3 partial-product tiles and the step-3 finish --
// from one task list, in cost order.  CTAs take tasks with an atomic
// counter; a task whose inputs come from earlier tasks of the same launch
// waits on per-supernode completion counters.
//
// Why this cannot deadlock: tasks are taken in list order and a task only
// waits on tasks earlier in the list, which are already held by running
// CTAs that themselves only wait on still earlier tasks; the earliest
// unfinished task never waits.  Every wait is bounded in time (spin_limit_ns
// of %globaltimer); when one runs out the kernel raises a timeout flag in the
// status words, every other wait returns at once, the remaining tasks are
// skipped and the launch ends.  pselinv_sync_status reports it.
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

template <class T>
__global__ void __launch_bounds__(TG_THREADS) k_persistent_level(KArgs a, PArgs p, const PTask* __restrict__ list,
                                                                 int ntask, int level) {
  constexpr int MAXBN = Sc<T>::P == 1 ? 64 : 32;
  __shared__ __align__(16) unsigned char smraw[sizeof(TileSmem<T, MAXBN>)];
  __shared__ int s_item;
  const int batch = a.sz.batch;
  const int total = ntask * batch;
  int* status = a.status;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(p.head + level, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= total) break;
    const PTask pt = list[item / batch];
    const int b = item % batch;
    const bool aborted = *(volatile int*)(status + 2) != 0;
    if (aborted) continue;  // drain the list
    const int64_t cb = (int64_t)b * p.nsn;
    switch (pt.kind) {
      case P_STEP2: {
        const Task tk = p.g1[pt.idx];
        switch (pt.var) {
          case 0: step2_tile<T, 8>(a, tk, b, *reinterpret_cast<TileSmem<T, 8>*>(smraw)); break;
          case 1: step2_tile<T, 16>(a, tk, b, *reinterpret_cast<TileSmem<T, 16>*>(smraw)); break;
          case 2: step2_tile<T, 32>(a, tk, b, *reinterpret_cast<TileSmem<T, 32>*>(smraw)); break;
          default:
            if constexpr (MAXBN == 64) step2_tile<T, 64>(a, tk, b, *reinterpret_cast<TileSmem<T, 64>*>(smraw));
            break;
        }
        cta_signal(p.c1 + cb + tk.sn);
        break;
      }
      case P_REDUCE: {
        const int k = pt.idx;
        if (!cta_wait(p.c1 + cb + k, p.n1[k], p.spin_ns, status)) break;
        step2_reduce<T>(a, k, b, pt.var, kReduceGroups, true);
        cta_signal(p.cr + cb + k);
        break;
      }
      case P_STEP3: {
        const Task tk = p.g2[pt.idx];
        const int k = tk.sn;
        const bool split = a.meta[k].ksplit > 1;
        if (!cta_wait(split ? p.cr + cb + k : p.c1 + cb + k, split ? kReduceGroups : p.n1[k], p.spin_ns, status))
          break;
        switch (pt.var) {
          case 0: step3_tile<T, 8>(a, tk, b, *reinterpret_cast<TileSmem<T, 8>*>(smraw), true); break;
          case 1: step3_tile<T, 16>(a, tk, b, *reinterpret_cast<TileSmem<T, 16>*>(smraw), true); break;
          case 2: step3_tile<T, 32>(a, tk, b, *reinterpret_cast<TileSmem<T, 32>*>(smraw), true); break;
          default:
            if constexpr (MAXBN == 64) step3_tile<T, 64>(a, tk, b, *reinterpret_cast<TileSmem<T, 64>*>(smraw), true);
            break;
        }
        cta_signal(p.c2 + cb + k);
        break;
      }
      default: {  // P_FINISH
        const int k = pt.idx;
        int target = p.n2[k];
        const int* ctr = p.c2 + cb + k;
        if (target == 0) {  // no step-3 tiles (r = 0): nothing to wait for in this launch
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
        step3_finish<T>(a, k, b, pt.var, kFinishParts, true);
        break;
      }
    }
  }
}

cudaError_t launch_persistent_level(const KArgs& a, const PArgs& p, const PTask* list, int ntask, int level,
                                    int grid, cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  if (a.dtype == PSELINV_C128)
    k_persistent_level<Cplx><<<grid, TG_THREADS, 0, st>>>(a, p, list, ntask, level);
  else
    k_persistent_level<double><<<grid, TG_THREADS, 0, st>>>(a, p, list, ntask, level);
  return cudaGetLastError();
}

cudaError_t persistent_grid(int dtype, int* grid) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = dtype == PSELINV_C128
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent_level<Cplx>, TG_THREADS, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent_level<double>, TG_THREADS, 0);
  if (e == cudaSuccess) *grid = sms * (per > 0 ? per : 1);
  return e;
}

}  // namespace psi
