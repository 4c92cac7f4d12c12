// Launch wrappers of the FP64 linear-algebra kernels (internal API).
#pragma once
#include "common.cuh"

namespace pepo {
cudaError_t launch_env_factor(const EnvFactorItem* items, int n_items, int chimax, int* ival,
                              cudaStream_t s);
cudaError_t launch_branch(const SiteFacItem* items, int n_items, int* ival, cudaStream_t s);
template <typename T>
// pass: the branch value of the sites processed (0: the Householder branch,
// 2: the sites the Cholesky branch handed over); only < 0: every site
cudaError_t launch_hh_level(const SiteFacItem* items, int n_items, int level, int grid_x, int nmax,
                            void* const* ptrs, const int* ival, cudaStream_t s, int pass);
// acct (may be null): 2 doubles accumulating the QR's algorithmic FLOPs and bytes
template <typename T>
cudaError_t launch_hh_extract(const SiteFacItem* items, int n_items, void* const* ptrs, int* ival,
                              cudaStream_t s, int pass, double* acct);
cudaError_t launch_form(const SiteFacItem* items, int n_items, int grid_x, const int* ival,
                        cudaStream_t s, int only);
// qcount (3 counters, may be null): sites per outcome of this pass, indexed
// by the final branch value (0 Householder, 1 Cholesky-QR, 2 handed back)
cudaError_t launch_factor(const SiteFacItem* items, int n_items, int rmax, int nmax, int* ival,
                          cudaStream_t s, int only, unsigned long long* qcount);
cudaError_t launch_core(const CoreItem* items, int n_items, int* ival, int* flags_base, cudaStream_t s);
}  // namespace pepo

namespace pepo {
// fp32 = 1: FP32 Jacobi in shared memory (FP32-storage modes), else FP64
cudaError_t launch_env_eig(const EnvEigItem* items, int n_items, int chimax, int fp32, const int* ival,
                           cudaStream_t s);
cudaError_t launch_rotate_back(const RotItem* items, int n_items, int chimax, const int* ival,
                               cudaStream_t s);
}  // namespace pepo
