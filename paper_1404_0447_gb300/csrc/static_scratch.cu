// Allocation-free entry point: inverses of a batch of small dense blocks
// from their LDL^T factors, with the intermediate L^{-1} blocks kept in a
// fixed device array that belongs to this library instead of memory from
// cudaMalloc.
//
// Why: cudaMalloc can stall and cudaFree synchronises the whole device, and
// some callers may not call either -- code running inside another
// framework's memory pool or under a fixed memory budget, real-time loops
// that must never block on the allocator.  This entry point allocates
// nothing: the caller passes inputs and outputs, and the only scratch is
// g_block_scratch below (16 MiB, held by every GPU that loads the library
// until the process exits).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"
#include "tile_gemm.cuh"

namespace psi {
void set_global_error(const std::string& msg);  // capi.cu
}

namespace {

constexpr int64_t kScratchDoubles = int64_t(1) << 21;  // 16 MiB of doubles
constexpr int kMaxDevices = 64;

// The shared scratch: L^{-1} of every block of the current call, s x s
// column-major, block-major.  Every call overwrites what it uses.
__device__ __align__(256) double g_block_scratch[kScratchDoubles];

// Phase 1, one CTA per block: V = L^{-1} for the unit lower triangle of the
// block (entries on and above the diagonal of L are not read), one column of
// V per thread; every entry of V's s x s block is written (zeros above the
// diagonal), so nothing from an earlier call survives into this one.
__global__ void k_static_linv(int s, const double* __restrict__ L, double* __restrict__ scratch) {
  extern __shared__ double T[];
  const int b = blockIdx.x;
  const double* Lb = L + (int64_t)b * s * s;
  double* V = scratch + (int64_t)b * s * s;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) T[e] = Lb[e];
  __syncthreads();
  for (int c = threadIdx.x; c < s; c += blockDim.x) {
    for (int i = 0; i < c; ++i) V[i + c * s] = 0.0;
    V[c + c * s] = 1.0;
    for (int i = c + 1; i < s; ++i) {
      double acc = 0.0;
      for (int q = c; q < i; ++q) acc += T[i + q * s] * V[q + c * s];
      V[i + c * s] = -acc;
    }
  }
}

// Phase 2, one CTA per (block, 64 x 64 tile of M): M = V^T D^{-1} V on the
// FP64 tensor pipe.
__global__ void __launch_bounds__(psi::TG_THREADS) k_static_m(int s, int tiles_per_dim,
                                                              const double* __restrict__ scratch,
                                                              const double* __restrict__ d, double* __restrict__ M) {
  constexpr int BN = 64;
  __shared__ psi::TileSmem<double, BN> sm;
  const int per_block = tiles_per_dim * tiles_per_dim;
  const int b = blockIdx.x / per_block, t = blockIdx.x % per_block;
  const int m0 = (t % tiles_per_dim) * psi::TG_BM, n0 = (t / tiles_per_dim) * BN;
  const double* V = scratch + (int64_t)b * s * s;
  const double* db = d + (int64_t)b * s;
  psi::Acc<double, BN> acc;
  psi::acc_zero<double, BN>(acc);
  auto la = [&](int mm, int q) { const int i = m0 + mm; return i < s ? V[q + i * s] / db[q] : 0.0; };
  auto lb = [&](int q, int nn) { const int j = n0 + nn; return j < s ? V[q + j * s] : 0.0; };
  psi::tile_mma<double, BN>(sm, 0, s, [](int) { return true; }, la, lb, acc);
  double* Mb = M + (int64_t)b * s * s;
  psi::tile_epilogue<double, BN>(acc, [&](int mm, int nn, double v) {
    const int i = m0 + mm, j = n0 + nn;
    if (i < s && j < s) Mb[i + j * s] = v;
  });
}

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (the host-side symbol is only a stand-in) and the shared
// memory limit of phase 1.
cudaError_t setup_device(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_block_scratch);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_static_linv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * psi::kMaxWidth * psi::kMaxWidth));
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int fail(int code, const std::string& msg) {
  psi::set_global_error(msg);
  return code;
}

}  // namespace

extern "C" int pselinv_block_inverse_static(int32_t s, int32_t count, const double* d_L, const double* d_d,
                                            double* d_M, void* stream) {
  if (s < 1 || s > psi::kMaxWidth) return fail(PSELINV_ERR_ARG, "block order s must be 1..128");
  if (count < 1) return fail(PSELINV_ERR_ARG, "count must be >= 1");
  if ((int64_t)count * s * s > kScratchDoubles)
    return fail(PSELINV_ERR_ARG, "count * s * s exceeds the static scratch (2^21 doubles = 16 MiB): " +
                                     std::to_string((int64_t)count * s * s) + " requested");
  if (!d_L || !d_d || !d_M) return fail(PSELINV_ERR_ARG, "NULL pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(PSELINV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  e = setup_device(dev, &scratch);
  if (e != cudaSuccess) return fail(PSELINV_ERR_CUDA, std::string("static scratch set-up: ") + cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  k_static_linv<<<count, 128, sizeof(double) * s * s, st>>>(s, d_L, scratch);
  const int tpd = (s + psi::TG_BM - 1) / psi::TG_BM;
  k_static_m<<<count * tpd * tpd, psi::TG_THREADS, 0, st>>>(s, tpd, scratch, d_d, d_M);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PSELINV_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return PSELINV_OK;
}
