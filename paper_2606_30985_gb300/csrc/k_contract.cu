// Register-tiled SIMT contractions of the BP and bond-update hot loop.
//
//   k_leg_contract  out[o, i, q] = sum_j A[i, j] in[o, j, q] on one layout leg
//                   (absorbing a message factor into a site tensor: Sec. 2.4
//                   step 1, and the products of Eq. 11)
//   k_gram_leg      out[i, i'] = sum_{o, q} X[o, i, q] Y[o, i', q]: a site tensor
//                   contracted with itself over every index but one leg, the
//                   Pauli leg traced (one double-layer message, Eq. 11)
//
// Both are GEMMs with one short dimension (chi <= 128).  A block owns a
// 128 x TC output tile; each of its 256 threads owns an 8 x MC register tile
// whose rows / columns are split in two halves 64 apart, so every 16-byte
// shared-memory load of a warp hits distinct banks.  A[i, j] is staged
// transposed in shared memory once per block and reused for every tile of the
// item.  FP32 storage accumulates in FP32 over the K <= 128 of a leg
// contraction; the Gram's long K is flushed into FP64 every 256 terms.
#include "kernels.h"

namespace pepo {

template <typename T> struct LCfg;
template <> struct LCfg<float> { static constexpr int TC = 128, MC = 8; };
template <> struct LCfg<double> { static constexpr int TC = 64, MC = 4; };

__device__ __forceinline__ int half_split(int t, int r) { return (r < 4) ? t * 4 + r : 64 + t * 4 + (r - 4); }

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T* v) {
  if constexpr (sizeof(T) == 4) {
    float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    double2 x = *reinterpret_cast<const double2*>(p);
    double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}

__device__ inline void load_dims4(const TView& v, const int* ival, int* d) {
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) d[k] = (k < v.nlegs) ? ival[v.dim[k]] : 1;
}

// ============================================================ leg contraction
template <typename T>
__global__ void __launch_bounds__(256)
k_leg_contract(const LegItem* __restrict__ items, void* const* ptrs, const int* __restrict__ ival) {
  constexpr int TR = 128, TC = LCfg<T>::TC, MC = LCfg<T>::MC;
  const LegItem it = items[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int d[PEPO_MAXLEG];
  load_dims4(it.in, ival, d);
  const int k = it.leg;
  const int Jin = d[k];
  const int Jout = ival[it.out_dim];
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.in.nlegs; ++i) Q *= d[i];
  T* At = reinterpret_cast<T*>(smem_raw);     // [Jin][TR]
  T* Bs = At + Jin * TR;                      // [Jin][TC]
  for (int e = threadIdx.x; e < Jin * TR; e += blockDim.x) {
    int j = e / TR, i = e - j * TR;
    At[e] = (i < Jout) ? (T)it.A[(long long)i * it.lda + j] : T(0);
  }
  long long G, nqb, units;
  if (Q >= TC) { G = 1; nqb = (Q + TC - 1) / TC; units = O * nqb; }
  else { G = TC / Q; nqb = 1; units = (O + G - 1) / G; }
  const T* __restrict__ in = static_cast<const T*>(ptrs[it.in.ref]);
  T* __restrict__ out = static_cast<T*>(ptrs[it.out_ref]);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __syncthreads();
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    long long o0, q0;
    int width;
    if (G == 1) { o0 = u / nqb; q0 = (u - o0 * nqb) * TC; width = (int)min((long long)TC, Q - q0); }
    else { o0 = u * G; q0 = 0; width = (int)(min(G, O - o0) * Q); }
    for (int e = threadIdx.x; e < Jin * TC; e += blockDim.x) {
      int j = e / TC, c = e - j * TC;
      T v = T(0);
      if (c < width) {
        long long o = (G == 1) ? o0 : o0 + c / Q;
        long long q = (G == 1) ? q0 + c : c % Q;
        v = in[(o * Jin + j) * Q + q];
      }
      Bs[e] = v;
    }
    __syncthreads();
    T acc[8][MC];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < MC; ++c) acc[r][c] = T(0);
#pragma unroll 2
    for (int j = 0; j < Jin; ++j) {
      T a[8], b[MC];
      lds4(At + j * TR + ty * 4, a);
      lds4(At + j * TR + 64 + ty * 4, a + 4);
      lds4(Bs + j * TC + tx * 4, b);
      if constexpr (MC == 8) lds4(Bs + j * TC + 64 + tx * 4, b + 4);
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
#pragma unroll
    for (int c = 0; c < MC; ++c) {
      const int col = (MC == 8) ? half_split(tx, c) : tx * 4 + c;
      if (col >= width) continue;
      const long long o = (G == 1) ? o0 : o0 + col / Q;
      const long long q = (G == 1) ? q0 + col : col % Q;
      T* dst = out + o * Jout * Q + q;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int i = half_split(ty, r);
        if (i < Jout) dst[(long long)i * Q] = acc[r][c];
      }
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_leg_contract(const LegItem* items, int n_items, int grid_x, int chimax,
                                void* const* ptrs, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = sizeof(T) * (size_t)chimax * (128 + LCfg<T>::TC);
  cudaError_t e = cudaFuncSetAttribute(k_leg_contract<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_leg_contract<T><<<dim3(grid_x, n_items), 256, smem, s>>>(items, ptrs, ival);
  return cudaGetLastError();
}

// ============================================================ Gram (free leg)
// X, Y as [O][F][Q], F <= 128: one 128 x 128 tile.  A chunk is 16 (o, q)
// pairs (one o and 16 consecutive q when Q >= 16, else floor(16/Q) o's).
constexpr int GL_BK = 16;
constexpr int GL_FLUSH = 256;

// product of the square-root weights sw[u][j_u] over layout legs u in [lo, hi)
// for the row-major multi-index `idx` of those legs
__device__ inline double leg_weight(const GramLegItem& it, const int* d, int lo, int hi, long long idx) {
  double w = 1.0;
  for (int u = hi - 1; u >= lo; --u) {
    const long long j = idx % d[u];
    idx /= d[u];
    if (it.sw[u]) w *= it.sw[u][j];
  }
  return w;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_gram_leg(const GramLegItem* __restrict__ items, int splits_max, void* const* ptrs,
           const int* __restrict__ ival) {
  const GramLegItem it = items[blockIdx.y];
  int d[PEPO_MAXLEG];
  load_dims4(it.x, ival, d);
  const int k = it.leg;
  const int F = d[k];
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.x.nlegs; ++i) Q *= d[i];
  const long long NC = gram_leg_chunks(O, Q);
  const int S = gram_leg_splits(NC, splits_max);
  const int s = blockIdx.x;
  if (s >= S) return;
  const long long c0 = NC * s / S, c1 = NC * (s + 1) / S;
  const T* __restrict__ X = static_cast<const T*>(ptrs[it.x.ref]);
  const T* __restrict__ Y = static_cast<const T*>(ptrs[it.y_ref]);
  const bool same = it.x.ref == it.y_ref;
  bool weighted = false;
  for (int u = 0; u < it.x.nlegs; ++u) weighted |= (u != k && it.sw[u] != nullptr);
  __shared__ __align__(16) T Xs[GL_BK][128];
  __shared__ __align__(16) T Ys[GL_BK][128];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool wideQ = Q >= GL_BK;
  const long long qpc = wideQ ? (Q + GL_BK - 1) / GL_BK : 0;
  const int opc = wideQ ? 1 : (int)(GL_BK / Q);
  // FP32 storage keeps an FP64 shadow of the accumulators, flushed every
  // GL_FLUSH terms; FP64 storage accumulates directly
  constexpr int NS = sizeof(T) == 4 ? 8 : 1;
  T acc[8][8];
  double acc64[NS][NS * 8 / NS];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = T(0);
#pragma unroll
  for (int r = 0; r < NS; ++r)
#pragma unroll
    for (int c = 0; c < NS * 8 / NS; ++c) acc64[r][c] = 0.0;
  int run = 0;
  for (long long cch = c0; cch < c1; ++cch) {
    long long o0, q0;
    if (wideQ) { o0 = cch / qpc; q0 = (cch - o0 * qpc) * GL_BK; }
    else { o0 = cch * opc; q0 = 0; }
    // zero the tile, then fill the live part
    for (int e = threadIdx.x; e < GL_BK * 128; e += blockDim.x) {
      (&Xs[0][0])[e] = T(0);
      if (!same) (&Ys[0][0])[e] = T(0);
    }
    __syncthreads();
    if (wideQ) {
      const double wo = weighted ? leg_weight(it, d, 0, k, o0) : 1.0;
      for (int e = threadIdx.x; e < GL_BK * F; e += blockDim.x) {
        int f = e / GL_BK, kk = e - f * GL_BK;
        long long q = q0 + kk;
        if (q < Q) {
          long long idx = (o0 * F + f) * Q + q;
          if (weighted) {
            const T w = (T)(wo * leg_weight(it, d, k + 1, it.x.nlegs, q >> 2));
            Xs[kk][f] = X[idx] * w;
            if (!same) Ys[kk][f] = Y[idx] * w;
          } else {
            Xs[kk][f] = X[idx];
            if (!same) Ys[kk][f] = Y[idx];
          }
        }
      }
    } else {
      const int Qi = (int)Q;
      for (int e = threadIdx.x; e < opc * F * Qi; e += blockDim.x) {
        int qq = e % Qi, rest = e / Qi;
        int f = rest % F, ol = rest / F;
        long long o = o0 + ol;
        if (o < O) {
          long long idx = (o * F + f) * Q + qq;
          if (weighted) {
            const T w = (T)(leg_weight(it, d, 0, k, o) * leg_weight(it, d, k + 1, it.x.nlegs, qq >> 2));
            Xs[ol * Qi + qq][f] = X[idx] * w;
            if (!same) Ys[ol * Qi + qq][f] = Y[idx] * w;
          } else {
            Xs[ol * Qi + qq][f] = X[idx];
            if (!same) Ys[ol * Qi + qq][f] = Y[idx];
          }
        }
      }
    }
    __syncthreads();
    const T* Yb = same ? &Xs[0][0] : &Ys[0][0];
#pragma unroll
    for (int kk = 0; kk < GL_BK; ++kk) {
      T a[8], b[8];
      lds4(&Xs[kk][0] + ty * 4, a);
      lds4(&Xs[kk][0] + 64 + ty * 4, a + 4);
      lds4(Yb + kk * 128 + tx * 4, b);
      lds4(Yb + kk * 128 + 64 + tx * 4, b + 4);
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      run += GL_BK;
      if (run >= GL_FLUSH) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) { acc64[r % NS][c] += (double)acc[r][c]; acc[r][c] = T(0); }
        run = 0;
      }
    }
  }
  double* P = it.partial + (long long)s * F * F;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int fi = half_split(ty, r);
    if (fi >= F) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int fj = half_split(tx, c);
      if (fj < F) {
        double v = (double)acc[r][c];
        if constexpr (sizeof(T) == 4) v += acc64[r % NS][c];
        P[(long long)fi * F + fj] = v;
      }
    }
  }
}

__global__ void k_gram_leg_reduce(const GramLegItem* __restrict__ items, int splits_max,
                                  const int* __restrict__ ival) {
  const GramLegItem it = items[blockIdx.y];
  int d[PEPO_MAXLEG];
  load_dims4(it.x, ival, d);
  const int k = it.leg;
  const int F = d[k];
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.x.nlegs; ++i) Q *= d[i];
  const int S = gram_leg_splits(gram_leg_chunks(O, Q), splits_max);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < F * F; e += gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int s = 0; s < S; ++s) sum += it.partial[(long long)s * F * F + e];
    int fi = e / F, fj = e - fi * F;
    it.out[(long long)fi * it.ldo + fj] = sum;
  }
}

template <typename T>
cudaError_t launch_gram_leg(const GramLegItem* items, int n_items, int splits_max,
                            void* const* ptrs, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_gram_leg<T><<<dim3(splits_max, n_items), 256, 0, s>>>(items, splits_max, ptrs, ival);
  return cudaGetLastError();
}

cudaError_t launch_gram_leg_reduce(const GramLegItem* items, int n_items, int chimax,
                                   int splits_max, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  int gx = ceil_div(chimax * chimax, 256);
  k_gram_leg_reduce<<<dim3(gx, n_items), 256, 0, s>>>(items, splits_max, ival);
  return cudaGetLastError();
}

template cudaError_t launch_leg_contract<float>(const LegItem*, int, int, int, void* const*,
                                                const int*, cudaStream_t);
template cudaError_t launch_leg_contract<double>(const LegItem*, int, int, int, void* const*,
                                                 const int*, cudaStream_t);
template cudaError_t launch_gram_leg<float>(const GramLegItem*, int, int, void* const*, const int*,
                                            cudaStream_t);
template cudaError_t launch_gram_leg<double>(const GramLegItem*, int, int, void* const*,
                                             const int*, cudaStream_t);

}  // namespace pepo
