// Launch wrappers of the device kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace psi {

// Per-batch-member sizes (elements) of every batched array.
struct Sizes {
  int64_t panel;  // L and X panels
  int64_t lhat;   // normalised factor / factor scratch
  int64_t linv;   // diagonal-block inverses
  int64_t n;      // pivots
  int64_t part;   // step-3 partial products
  int batch;
};

cudaError_t setup_kernels();
cudaError_t launch_scatter_values(const double* vals, const int64_t* vmap, int64_t nnz, double* L, const Sizes& sz,
                                  cudaStream_t st);
cudaError_t launch_gather_values(const double* X, const int64_t* vmap, int64_t nnz, double* out, const Sizes& sz,
                                 cudaStream_t st);
cudaError_t launch_factor_level(const SnMeta* meta, const int32_t* sns, int nsn_level, const Task* trsm,
                                int64_t ntrsm, const Task* schur, int64_t nschur, const ColDesc* desc,
                                const int32_t* relidx, double* L, double* D, double* Linv, double* Ltmp, int maxw,
                                const Sizes& sz, int* status, cudaStream_t st);
cudaError_t launch_normalise(const SnMeta* meta, int nsn, const Task* lhat_tasks, int64_t nlhat, const double* L,
                             const double* D, double* Linv, double* Lhat, double* X, int maxw, const Sizes& sz,
                             cudaStream_t st);
cudaError_t launch_gemm1(const SnMeta* meta, const Task* g1, int64_t ng1, const ColDesc* desc, const int32_t* relidx,
                         const double* Lhat, double* X, const Sizes& sz, cudaStream_t st);
cudaError_t launch_gemm2(const SnMeta* meta, const Task* g2, int64_t ng2, const double* Lhat, const double* X,
                         double* part, const Sizes& sz, cudaStream_t st);
cudaError_t launch_diag_final(const SnMeta* meta, const int32_t* sns, int nsn_step, const double* part, double* X,
                              const Sizes& sz, cudaStream_t st);
cudaError_t launch_logdet(const double* D, int64_t n, double* out, int batch, cudaStream_t st);

}  // namespace psi
