// Launch wrappers of the BP, Bethe, gate-table and bookkeeping kernels.
#pragma once
#include "common.cuh"

namespace pepo {
// `active` (per instance, may be null): converged instances of a batch keep their messages
cudaError_t launch_bp_finish(const MsgItem* items, int n, const int* ival, const int* active,
                             unsigned long long* delta, int* flags, cudaStream_t s);
cudaError_t launch_sl_init(const MsgItem* items, int n, const int* ival, cudaStream_t s);
cudaError_t launch_sl_finish(const MsgItem* items, int n, const int* ival, const int* active,
                             unsigned long long* delta, cudaStream_t s);
cudaError_t launch_site_scalars(const SiteScalarItem* items, int n, const int* ival, cudaStream_t s);
cudaError_t launch_edge_scalars(const EdgeItem* items, int n, const int* ival, cudaStream_t s);
template <typename T>
cudaError_t launch_pauli_weights(const PauliWItem* items, int n, void* const* ptrs, const int* ival,
                                 cudaStream_t s);
cudaError_t launch_bethe(const BetheItem* items, int n, cudaStream_t s);
cudaError_t launch_gates(const GateItem* items, int n, cudaStream_t s);
// swap pointer-table entries pairs[2i] <-> pairs[2i+1]; copy ival[moves[2i+1]] -> ival[moves[2i]]
cudaError_t launch_commit(const int* pairs, int npairs, const int* moves, int nmoves, void** ptrs,
                          int* ival, cudaStream_t s);
}  // namespace pepo
