// Launch wrappers of the libpepo kernels (host-callable, internal API).
#pragma once
#include "common.cuh"

namespace pepo {

// ---- k_tensor.cu (storage type T = float or double) ----------------------
template <typename T>
cudaError_t launch_leg_contract(const LegItem* items, int n_items, int grid_x, int chimax,
                                void* const* ptrs, const int* ival, cudaStream_t s);
template <typename T>
cudaError_t launch_copy(const TView* items, const int* out_refs, int n_items, int grid_x,
                        void* const* ptrs, const int* ival, cudaStream_t s);
template <typename T>
cudaError_t launch_gram_rows(const GramRowsItem* items, int n_items, int tiles_max, int splits_max,
                             int sym, void* const* ptrs, const int* ival, cudaStream_t s);
cudaError_t launch_gram_rows_reduce(const GramRowsItem* items, int n_items, int fmax,
                                    int splits_max, int sym, const int* ival, cudaStream_t s);
template <typename T>
cudaError_t launch_gram_leg(const GramLegItem* items, int n_items, int splits_max, int chimax,
                            void* const* ptrs, const int* ival, cudaStream_t s);
// canonical <-> stored site layout (perm[k] = canonical leg at layout position k)
template <typename T>
cudaError_t launch_permute(const void* in, void* out, int nlegs, const int* dims_canon, const int* perm,
                           int to_layout, cudaStream_t s);
// sum of the per-split partials; sym = 1 symmetrises the sum as (S + S^T) / 2
cudaError_t launch_gram_leg_reduce(const GramLegItem* items, int n_items, int chimax,
                                   int splits_max, int sym, const int* ival, cudaStream_t s);
template <typename T>
cudaError_t launch_reconstruct(const ReconItem* items, int n_items, int grid_x, int ntile_max,
                               void* const* ptrs, const int* ival, cudaStream_t s);
template <typename T>
cudaError_t launch_vec_contract(const VecItem* items, int n_items, int grid_x,
                                void* const* ptrs, const int* ival, cudaStream_t s);

// ---- k_umma.cu (FP32 storage, TF32x3 on tcgen05 tensor cores, chi <= 128)
bool umma_supported(int chimax);
// err: device int; bit 0 is set when a pipeline wait of the kernel ran
// longer than wait_ns (the kernel then leaves its loops, lets its own MMAs and
// copies in flight finish, frees its tensor memory and returns), bit 1 when a
// reconstruct item has no packed-W workspace, bit 2 when one of those exit
// drains itself ran out of time
cudaError_t launch_leg_umma(const LegItem* items, int n_items, int chimax, void* const* ptrs, const int* ival,
                            int* err, unsigned long long wait_ns, cudaStream_t s);
// floats of the packed W workspace of one reconstruct item for n, n' <= nmax
size_t recon_packed_floats(int nmax);
// psi_new = psi W into the next layout (Q-less reconstruct), W from the bond core
cudaError_t launch_recon_umma(const ReconItem* items, int n_items, int chimax, void* const* ptrs,
                              const int* ival, int* err, unsigned long long wait_ns, cudaStream_t s);
// writes per-split partial sums S; the reduction with sym = 1 returns (S + S^T) / 2
cudaError_t launch_gram_umma(const GramLegItem* items, int n_items, int splits_max, int chimax,
                             void* const* ptrs, const int* ival, int* err, unsigned long long wait_ns,
                             cudaStream_t s);

// Split count shared by the Gram kernels and their reductions.
__host__ __device__ inline int gram_rows_splits(long long K, int splits_max) {
  long long s = (K + 511) / 512;
  if (s < 1) s = 1;
  return (int)(s < splits_max ? s : splits_max);
}
// chunks of 32 (o, q) pairs: one o and 32 consecutive q when Q >= 32, else
// floor(32 / Q) consecutive o with all q (k_gram_leg's GL_BK)
__host__ __device__ inline long long gram_leg_chunks(long long O, long long Q) {
  return Q >= 32 ? O * ((Q + 31) / 32) : (O + (32 / Q) - 1) / (32 / Q);
}
// split count of a free-leg Gram from its summed extent K = O * Q (shared by
// every Gram variant and the reduction, independent of their chunk sizes)
__host__ __device__ inline int gram_leg_splits_k(long long K, int splits_max) {
  long long s = K / 2048;
  if (s < 1) s = 1;
  return (int)(s < splits_max ? s : splits_max);
}
__host__ __device__ inline int gram_leg_splits(long long chunks, int splits_max) {
  long long s = (chunks + 31) / 32;
  if (s < 1) s = 1;
  return (int)(s < splits_max ? s : splits_max);
}

}  // namespace pepo
